// Tensor-core path (placeholder until the tcgen05 kernels land).
#include "jet_tc.h"

jet_status tc_plan_create(jet_plan_s*, jet::TcPlan** out, const cudaDeviceProp&, size_t, int) {
  *out = nullptr;
  return JET_ERR_UNSUPPORTED;
}
void tc_plan_destroy(jet::TcPlan*) {}
int tc_tile_points(const jet::TcPlan*) { return 0; }
int tc_grid(const jet::TcPlan*) { return 0; }
size_t tc_workspace_bytes(const jet::TcPlan*) { return 0; }
jet_status tc_forward(jet_plan_s*, jet::TcPlan*, const void*, const void*, long long, const void*, void*, double*,
                      cudaStream_t) { return JET_ERR_UNSUPPORTED; }
jet_status tc_backward(jet_plan_s*, jet::TcPlan*, const void*, const void*, long long, const void*, void*, void*,
                       double*, cudaStream_t) { return JET_ERR_UNSUPPORTED; }
jet_status tc_train_step(jet_plan_s*, jet::TcPlan*, void*, void*, void*, long long, float, const void*, long long,
                         const void*, double*, cudaStream_t) { return JET_ERR_UNSUPPORTED; }
jet_status tc_batch_create(const std::vector<jet_plan_s*>&, jet::TcBatch** out) {
  *out = nullptr;
  return JET_ERR_UNSUPPORTED;
}
void tc_batch_destroy(jet::TcBatch*) {}
jet_status tc_batch_run(jet::TcBatch*, const std::vector<jet_plan_s*>&, const void* const*, void* const*,
                        void* const*, long long, float, const void* const*, const int64_t*, const void* const*,
                        void* const*, double*, bool, cudaStream_t) { return JET_ERR_UNSUPPORTED; }
