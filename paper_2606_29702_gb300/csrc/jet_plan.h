// Plan object shared by the host units of libjet (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <utility>
#include <vector>

#include "../../include/jet.h"
#include "jet_internal.h"

namespace jet {
struct TcPlan;
}

struct jet_plan_s {
  int device = 0;
  int d = 0, L = 0, n_out = 0, n_res = 0;
  std::vector<int> widths;
  int cls = -1, C = 0;
  jet_precision prec = JET_FP32;
  bool fp64 = false;
  bool tc = false;
  std::vector<jet::DevTerm> terms;
  bool has_source = false;
  long long n_params = 0;
  std::vector<long long> off_W, off_b;
  int P = 0, pitch = 0, S = 0;
  size_t smem = 0;
  int grid = 0, ctas_per_sm = 0;
  size_t elem = 4;
  // workspace
  void* Wt = nullptr;
  double* grad_slices = nullptr;
  double* loss_slices = nullptr;
  void* scratch = nullptr;
  long long scratch_stride = 0;
  long long wacc_off = -1;  // FP32 weight-gradient accumulator in a scratch slot (elements)
  void* store = nullptr;
  long long store_max_points = 0;
  long long store_tile_stride = 0;
  size_t ws_bytes = 0;
  // identity of the forward call whose jets the store holds
  bool st_valid = false;
  const void* st_params = nullptr;
  const void* st_X = nullptr;
  const void* st_src = nullptr;
  long long st_N = -1;
  // tensor-core path state (jet_tc.cu)
  jet::TcPlan* tcp = nullptr;
  // measurement hook: event pairs around the dominant kernel
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof;
};

namespace jet {
// event pair around the dominant kernel of a call while profiling is enabled
void plan_prof_begin(jet_plan_s* p, cudaStream_t s);
void plan_prof_end(jet_plan_s* p, cudaStream_t s);
}  // namespace jet
