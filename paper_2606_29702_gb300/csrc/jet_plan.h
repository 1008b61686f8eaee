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
  // composite loss: its terms (monomial ranges, weights in `scale`) and the
  // point counts of the latest jet_plan_set_term_points; n_groups = 0 for a
  // plan with one residual
  int n_groups = 0;
  std::vector<jet::DevGroup> groups;
  std::vector<long long> group_counts;
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
// the loss terms of a call: point ranges from the counts, scale = weight /
// (residuals of the term); returns their number
inline int fill_groups(const jet_plan_s* p, DevGroup* out) {
  long long start = 0;
  for (int g = 0; g < p->n_groups; ++g) {
    DevGroup G = p->groups[g];
    const long long cnt = g < (int)p->group_counts.size() ? p->group_counts[g] : 0;
    const long long M = G.paired ? cnt / 2 : cnt;
    G.start = start;
    G.count = cnt;
    G.scale = M > 0 ? p->groups[g].scale / (double)M : 0.0;
    out[g] = G;
    start += cnt;
  }
  return p->n_groups;
}
// a composite-loss plan's term points (set by jet_plan_set_term_points) add up to N
inline bool group_counts_match(const jet_plan_s* p, long long N) {
  if (p->n_groups == 0) return true;
  if ((int)p->group_counts.size() != p->n_groups) return false;
  long long tot = 0;
  for (long long c : p->group_counts) tot += c;
  return tot == N;
}
// event pair around the dominant kernel of a call while profiling is enabled
void plan_prof_begin(jet_plan_s* p, cudaStream_t s);
void plan_prof_end(jet_plan_s* p, cudaStream_t s);
}  // namespace jet
