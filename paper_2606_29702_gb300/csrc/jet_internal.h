// Internal structures shared by the host orchestration (jet_api.cu) and the
// kernels.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace jet {

constexpr int kMaxLayers = 16;   // weight layers
constexpr int kMaxTerms = 32;    // residual monomials over all components
constexpr int kMaxRes = 4;
constexpr int kMaxOut = 4;
constexpr int kMaxC = 16;

// One residual monomial: coef * prod fac, fac = o * C + channel index; bit f
// of pmask: factor f is read at the second point of a pair (paired loss terms).
struct DevTerm {
  double coef;
  int comp;
  int nfac;
  int fac[4];
  int pmask;
};

// One term of a composite loss (Sec. 3.1.1: weighted IC, BC and PDE terms over
// their own blocks of the concatenated points): the points [start, start +
// count), its monomials [t0, t1), scale = weight / (residuals of the term).
// A paired term has one residual per consecutive pair of points, evaluated at
// the pair's first point.
constexpr int kMaxGroups = 4;
struct DevGroup {
  long long start, count;
  double scale;
  int t0, t1;
  int n_res, paired, has_source;
};

// Kernel modes
enum : int {
  MODE_FWD = 0,        // residual + loss (+ z-jet store when store != null)
  MODE_FWD_BWD = 1,    // residual + loss + gradient, hidden jets recomputed per tile
  MODE_BWD_STORE = 2,  // gradient from a z-jet store written by MODE_FWD
};

// Everything a kernel needs to know about one PINN instance for one call.
struct DevInstance {
  int L;               // weight layers
  int d, n_out, n_res;
  int widths[kMaxLayers + 1];
  long long off_W[kMaxLayers];  // offsets (elements) into the packed params
  long long off_b[kMaxLayers];
  long long n_params;
  const void* params;  // packed, value type T
  const void* Wt;      // weight workspace, value type T: the packed parameters
                       // with every W^l transposed, then (at weight_copy_offset)
                       // a 16-byte-aligned copy of the packed parameters
  const void* X;       // [N][d]
  const void* source;  // [N][n_res] or null
  void* r_out;         // [N][n_res] or null
  long long N;
  double inv_N;
  int n_terms;
  DevTerm terms[kMaxTerms];
  // composite loss (0: one residual over all points, mean over N)
  int n_groups;
  DevGroup groups[kMaxGroups];
  // tiling
  int P;               // points per tile
  int pitch;           // smem row pitch (elements) of a jet buffer, >= S * P
  int S;               // point stride within a jet row (SIMT forms)
  long long n_tiles;
  int tiles_per_chunk;
  int n_chunks;
  int chunk_base;      // first work-item index of this instance
  // outputs of the chunk reduction (FP64): [n_chunks][n_params], [n_chunks]
  double* grad_slices;
  double* loss_slices;
  // z-jet store for MODE_FWD / MODE_BWD_STORE: per tile, per hidden layer,
  // [w][C * P] (as the shared-memory rows); null if not stored
  void* store;
  long long store_tile_stride;  // elements per tile
  // FP32 forms: element offset, in a CTA's scratch slot, of the chunk's FP32
  // weight-gradient accumulator (simt_wacc_elems); -1: FP64 adds per tile
  long long wacc_off;
};

// Per-launch arguments of the fused SIMT kernel.
struct SimtArgs {
  int mode;
  int n_inst;
  const DevInstance* insts;   // device array (batched) or null
  DevInstance inst0;          // single-instance launches pass it by value
  int n_items;                // total work items (instance, chunk)
  const int* item_inst;       // [n_items] instance of each item (batched) or null
  void* scratch;              // per-CTA z-jet scratch
  long long scratch_stride;   // elements per CTA slot
  // batches: counter of the items taken after each CTA's first (zeroed before
  // the launch), so that a CTA that finishes takes the next item of the
  // cost-ordered list; null: a fixed stride
  int* item_next;
};

constexpr int kSimtThreads = 256;
// Point stride S of a SIMT shared-memory jet row [unit][n * S + alpha]: the
// lanes of a warp walk min(P, 32) points and must hit distinct banks, so S = C
// when C's power-of-two factor times those lanes fits in 32 banks (C = 6 at
// P = 16), else the odd C | 1 (pad columns stay zero).
inline int simt_point_stride(int C, int P) {
  const int lanes = P < 32 ? P : 32;
  return (C & -C) * lanes <= 32 ? C : (C | 1);
}
// share of L2 the per-chunk FP64 gradient slices may take before the kernels
// accumulate a chunk's weight gradients in FP32 instead of adding per tile
constexpr double kSimtSliceL2Bytes = 48.0 * 1024 * 1024;
// FP32 forms: elements of the per-CTA weight-gradient accumulator that
// follows a tile's z-jets in the CTA's scratch slot, one float per weight of
// every hidden-to-hidden layer W^l (l = 2 .. L-1, [w_l][w_{l-1}])
inline long long simt_wacc_elems(const int* widths, int L, bool fp64) {
  if (fp64) return 0;
  long long e = 0;
  for (int l = 2; l <= L - 1; ++l) e += (long long)widths[l] * widths[l - 1];
  return e;
}
// elements of the SIMT weight workspace: transposed copy, then aligned copy
__host__ __device__ inline long long weight_copy_offset(long long n_params) { return (n_params + 3) & ~3LL; }
__host__ __device__ inline long long weight_ws_elems(long long n_params) { return 2 * weight_copy_offset(n_params); }
// Dynamic shared memory of the fused SIMT kernel: three jet buffers
// [wmax][pitch], output jets and adjoints [n_out*C][P], tile points [P][d],
// and a small reduction area.
inline size_t simt_smem_bytes(int C, int P, int pitch, int wmax, int n_out, int d, size_t elem) {
  size_t e = 3 * (size_t)wmax * pitch + 2 * (size_t)n_out * C * P + (size_t)P * d;
  size_t bytes = (e * elem + 15) / 16 * 16;
  return bytes + 64 * sizeof(double);
}


// Reductions and elementwise kernels (jet_reduce.cu)
// One reduction job per instance: grad[p] = sum_c slices[c][p] in FP64 (fixed
// order), loss = inv_N * sum_c loss_slices[c]; optionally fused with Adam.
struct ReduceJob {
  const double* grad_slices;
  const double* loss_slices;
  int n_chunks;
  int grad_chunks;    // gradient slices to sum (0: n_chunks; 1: one shared accumulator)
  long long n_params;
  double inv_N;
  void* grad_out;     // value type T or null
  double* loss_out;   // or null
  void* params;       // Adam: updated in place (value type T)
  void* m;
  void* v;
};
cudaError_t launch_transpose_weights(const DevInstance& in, bool fp64, void* Wt, cudaStream_t s);
// jobs: host array copied by value when n == 1, else a device array.  Adam
// takes step t = `step`, or *step_ctr + 1 with a device counter, which the
// call then increments on the stream.
cudaError_t launch_reduce(const ReduceJob* dev_jobs, const ReduceJob& job0, int n, long long max_params, bool fp64,
                          bool adam, long long step, float lr, cudaStream_t s, long long* step_ctr = nullptr);

}  // namespace jet

namespace jet {
// Sets the thread-local message returned by jet_last_error() (jet_api.cu).
void set_last_error(const char* msg);

// Per-class entry points, one explicit specialisation per instantiation unit.
template <int ID> cudaError_t simt_launch_id(bool fp64, const SimtArgs& a, int grid, size_t smem, cudaStream_t s);
template <int ID> cudaError_t simt_max_active_id(bool fp64, size_t smem, int* blocks);
template <int ID> cudaError_t debug_activation_id(int kind, long long n, const double* z, const double* v,
                                                  double* out, cudaStream_t s);
}  // namespace jet
