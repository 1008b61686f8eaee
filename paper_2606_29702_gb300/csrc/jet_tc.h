// Tensor-core (tcgen05 / TMEM / TMA) path of libjet: declarations used by the
// host orchestration.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/jet.h"

struct jet_plan_s;
namespace jet {
struct TcPlan;
struct TcBatch;
}  // namespace jet

jet_status tc_plan_create(jet_plan_s* p, jet::TcPlan** out, const cudaDeviceProp& prop, size_t mem_budget,
                          int flags);
void tc_plan_destroy(jet::TcPlan* t);
int tc_tile_points(const jet::TcPlan* t);
int tc_grid(const jet::TcPlan* t);
int tc_ctas_per_sm(const jet::TcPlan* t);
int tc_threads(const jet::TcPlan* t);
int tc_wgrad_chunk_fp32(const jet::TcPlan* t);  // per-tile weight gradients use the FP32 chunk accumulator
size_t tc_workspace_bytes(const jet::TcPlan* t);
jet_status tc_forward(jet_plan_s* p, jet::TcPlan* t, const void* params, const void* X, long long N,
                      const void* source, void* r_out, double* loss_out, cudaStream_t s);
jet_status tc_backward(jet_plan_s* p, jet::TcPlan* t, const void* params, const void* X, long long N,
                       const void* source, void* grad_out, void* r_out, double* loss_out, cudaStream_t s);
jet_status tc_train_step(jet_plan_s* p, jet::TcPlan* t, void* params, void* m, void* v, long long step,
                         long long* step_ctr, float lr, const void* X, long long N, const void* source,
                         double* loss_out, cudaStream_t s);
jet_status tc_batch_create(const std::vector<jet_plan_s*>& plans, jet::TcBatch** out);
void tc_batch_destroy(jet::TcBatch* b);
jet_status tc_batch_run(jet::TcBatch* b, const std::vector<jet_plan_s*>& plans, const void* const* params,
                        void* const* m, void* const* v, long long step, long long* step_ctr, float lr,
                        const void* const* X,
                        const int64_t* N, const void* const* source, void* const* grad_out, double* loss_out,
                        bool adam, cudaStream_t s);
