// jet_backward_params_noalloc: the parameter gradient of the fused SIMT kernel
// without any device allocation.
//
// Who needs it: code that must not call cudaMalloc -- for example an
// embedding runtime that owns every device allocation itself, or a real-time
// loop that forbids allocator calls after start-up.  Such callers cannot create a plan
// (jet_plan_create allocates the plan's workspace), so this entry point takes
// the plan arguments and the call arguments together and keeps all of its
// working memory in one file-scope device array of fixed size.
//
// The array (kStaticScratchBytes) is reserved on every GPU that loads this
// library, for the life of the process.  Host code never dereferences its
// name: on the host the name is only a stand-in for the device symbol, so
// the address handed to kernels comes from cudaGetSymbolAddress, taken once
// per device (with that device current) on the first call made on it.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/jet.h"
#include "jet_closures_gen.h"
#include "jet_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 8u << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};
std::atomic<bool> g_ready[kMaxDevices];

// messages go to the library's thread-local jet_last_error()
jet_status nfail(jet_status st, const char* msg) {
  jet::set_last_error(msg);
  return st;
}

jet_status nfail_cuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  jet::set_last_error(buf);
  return JET_ERR_CUDA;
}

// Device address of g_static_scratch on the current device (set-up on first use).
jet_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return nfail(JET_ERR_UNSUPPORTED, "device index above 63");
  if (!g_ready[dev].load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_ready[dev].load(std::memory_order_relaxed)) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return nfail_cuda(e, "cudaGetSymbolAddress(static scratch)");
      g_scratch_ptr[dev] = p;
      g_ready[dev].store(true, std::memory_order_release);
    }
  }
  *out = g_scratch_ptr[dev];
  return JET_OK;
}

bool class_has(const jet::ClassInfo& ci, int d, const int* alpha) {
  for (int c = 0; c < ci.C; ++c) {
    bool eq = true;
    for (int j = 0; j < d; ++j) eq = eq && ci.alpha[c][j] == alpha[j];
    if (eq) return true;
  }
  return false;
}

int chan_of(const jet::ClassInfo& ci, int d, const uint8_t* alpha) {
  for (int c = 0; c < ci.C; ++c) {
    bool eq = true;
    for (int j = 0; j < d; ++j) eq = eq && ci.alpha[c][j] == alpha[j];
    if (eq) return c;
  }
  return -1;
}

cudaError_t launch_by_class(int cls, bool fp64, const jet::SimtArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (cls) {
#define CASE(id, cl) \
  case id:           \
    return jet::simt_launch_id<id>(fp64, a, grid, smem, s);
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_by_class(int cls, bool fp64, size_t smem, int* blocks) {
  switch (cls) {
#define CASE(id, cl) \
  case id:           \
    return jet::simt_max_active_id<id>(fp64, smem, blocks);
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

}  // namespace

extern "C" jet_status jet_backward_params_noalloc(const jet_residual_spec* spec, int32_t d_in, int32_t n_layers,
                                                  const int32_t* widths, int32_t n_needed, const jet_chan* needed,
                                                  jet_precision prec, const void* params, const void* X, int64_t N,
                                                  const void* source, void* grad_out, double* loss_out,
                                                  jet_stream_t stream, size_t* scratch_bytes_used) {
  using namespace jet;
  if (scratch_bytes_used) *scratch_bytes_used = 0;
  if (!spec || !widths || !params || !grad_out || (N > 0 && !X) || (n_needed > 0 && !needed))
    return nfail(JET_ERR_INVALID, "NULL argument");
  if (prec != JET_FP64 && prec != JET_FP32) return nfail(JET_ERR_UNSUPPORTED, "only JET_FP64 and JET_FP32");
  if (d_in < 1 || d_in > 3 || n_layers < 2 || n_layers > kMaxLayers || widths[0] != d_in || N < 1)
    return nfail(JET_ERR_INVALID, "bad shape (d_in 1..3, 2 <= n_layers <= 16, widths[0] == d_in, N >= 1)");
  const int n_out = widths[n_layers];
  if (n_out < 1 || n_out > kMaxOut) return nfail(JET_ERR_INVALID, "n_out must be 1..4");
  int wmax = 0;
  for (int l = 1; l < n_layers; ++l) {
    if (widths[l] < 4 || widths[l] > 256 || widths[l] % 4) return nfail(JET_ERR_UNSUPPORTED, "hidden width");
    wmax = widths[l] > wmax ? widths[l] : wmax;
  }
  if (spec->n_res < 1 || spec->n_res > kMaxRes || !spec->n_mono || !spec->mono)
    return nfail(JET_ERR_INVALID, "residual spec");
  if ((spec->has_source != 0) != (source != nullptr)) return nfail(JET_ERR_INVALID, "source does not match spec");
  // the same spec and multi-index checks as jet_plan_create, before anything
  // below dereferences the monomial lists
  for (int c = 0; c < spec->n_res; ++c)
    if (spec->n_mono[c] < 0 || (spec->n_mono[c] > 0 && !spec->mono[c]))
      return nfail(JET_ERR_INVALID, "residual component with a bad monomial list");
  for (int i = 0; i < n_needed; ++i)
    for (int j = d_in; j < 4; ++j)
      if (needed[i].alpha[j]) return nfail(JET_ERR_INVALID, "a needed multi-index differentiates a coordinate >= d_in");
  // smallest compiled channel set containing every needed multi-index and
  // every multi-index below them (checked componentwise, no heap)
  int best = -1;
  for (int k = 0; k < kNumClasses; ++k) {
    const ClassInfo& ci = kClassInfo[k];
    if (ci.d != d_in) continue;
    bool ok = true;
    for (int i = 0; i < n_needed && ok; ++i) {
      int lim[3] = {0, 0, 0};
      for (int j = 0; j < d_in; ++j) lim[j] = needed[i].alpha[j];
      int a[3] = {0, 0, 0};
      for (a[0] = 0; a[0] <= lim[0] && ok; ++a[0])
        for (a[1] = 0; a[1] <= lim[1] && ok; ++a[1])
          for (a[2] = 0; a[2] <= lim[2] && ok; ++a[2]) ok = class_has(ci, d_in, a);
    }
    if (ok && (best < 0 || ci.C < kClassInfo[best].C)) best = k;
  }
  if (best < 0) return nfail(JET_ERR_UNSUPPORTED, "no compiled channel set contains the needed multi-indices");
  const ClassInfo& ci = kClassInfo[best];
  const int C = ci.C;
  const bool fp64 = prec == JET_FP64;
  const size_t elem = fp64 ? 8 : 4;

  DevInstance I;
  memset(&I, 0, sizeof(I));
  I.L = n_layers;
  I.d = d_in;
  I.n_out = n_out;
  I.n_res = spec->n_res;
  long long off = 0;
  for (int l = 0; l <= n_layers; ++l) I.widths[l] = widths[l];
  for (int l = 0; l < n_layers; ++l) {
    I.off_W[l] = off;
    off += (long long)widths[l] * widths[l + 1];
    I.off_b[l] = off;
    off += widths[l + 1];
  }
  I.n_params = off;
  int nt = 0;
  for (int c = 0; c < spec->n_res; ++c) {
    for (int m = 0; m < spec->n_mono[c]; ++m) {
      const jet_monomial& mo = spec->mono[c][m];
      if (nt >= kMaxTerms || mo.n_fac < 0 || mo.n_fac > 4) return nfail(JET_ERR_UNSUPPORTED, "residual monomials");
      DevTerm& t = I.terms[nt++];
      t.coef = mo.coef;
      t.comp = c;
      t.nfac = mo.n_fac;
      for (int f = 0; f < mo.n_fac; ++f) {
        for (int j = d_in; j < 4; ++j)
          if (mo.fac[f].alpha[j]) return nfail(JET_ERR_INVALID, "a residual factor differentiates a coordinate >= d_in");
        const int ch = chan_of(ci, d_in, mo.fac[f].alpha);
        if (ch < 0 || mo.fac[f].out < 0 || mo.fac[f].out >= n_out)
          return nfail(JET_ERR_INVALID, "residual factor outside the carried channels");
        t.fac[f] = mo.fac[f].out * C + ch;
      }
    }
  }
  I.n_terms = nt;
  I.params = params;
  I.X = X;
  I.source = source;
  I.r_out = nullptr;
  I.N = N;
  I.inv_N = 1.0 / (double)N;
  // tiling: same rule as the plan path
  const int TP = fp64 ? 2 : 4;
  const int P = TP * (kSimtThreads / wmax > 0 ? kSimtThreads / wmax : 1);
  const int S = simt_point_stride(C, P);
  int pitch = S * P;
  while (pitch % (fp64 ? 16 : 32) != (fp64 ? 2 : 4)) ++pitch;
  I.P = P;
  I.pitch = pitch;
  I.S = S;
  I.n_tiles = (N + P - 1) / P;
  const size_t smem = simt_smem_bytes(C, P, pitch, wmax, n_out, d_in, elem);
  long long jet_elems = 0;
  for (int l = 1; l < n_layers; ++l) jet_elems += (long long)C * P * widths[l];

  // carve the static array: Wt | loss slices | grad slices | per-CTA scratch
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_wt = up((size_t)weight_ws_elems(I.n_params) * elem);
  const size_t per_chunk = (size_t)I.n_params * sizeof(double) + sizeof(double) + (size_t)jet_elems * elem;
  const size_t fixed = b_wt + 3 * 256;
  if (fixed + per_chunk > kStaticScratchBytes)
    return nfail(JET_ERR_UNSUPPORTED, "shape needs more than the 8 MiB static scratch of the no-alloc path");
  int per_sm = 0, dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = occupancy_by_class(best, fp64, smem, &per_sm);
  if (e != cudaSuccess) return nfail_cuda(e, "occupancy");
  if (per_sm < 1) return nfail(JET_ERR_UNSUPPORTED, "tile does not fit one SM");
  long long fit = (long long)((kStaticScratchBytes - fixed) / per_chunk);
  long long chunks = I.n_tiles;
  if (chunks > (long long)sms * per_sm) chunks = (long long)sms * per_sm;
  if (chunks > fit) chunks = fit;
  I.tiles_per_chunk = (int)((I.n_tiles + chunks - 1) / chunks);
  I.n_chunks = (int)((I.n_tiles + I.tiles_per_chunk - 1) / I.tiles_per_chunk);

  void* base = nullptr;
  jet_status st = scratch_address(&base);
  if (st != JET_OK) return st;
  unsigned char* b = static_cast<unsigned char*>(base);
  I.Wt = b;
  I.loss_slices = reinterpret_cast<double*>(b + b_wt);
  I.grad_slices = reinterpret_cast<double*>(b + b_wt + up((size_t)I.n_chunks * sizeof(double)));
  unsigned char* scr = b + b_wt + up((size_t)I.n_chunks * sizeof(double)) +
                       up((size_t)I.n_chunks * I.n_params * sizeof(double));
  const size_t used = (size_t)(scr - b) + (size_t)I.n_chunks * jet_elems * elem;
  if (used > kStaticScratchBytes) return nfail(JET_ERR_UNSUPPORTED, "static scratch overflow");
  if (scratch_bytes_used) *scratch_bytes_used = used;
  I.chunk_base = 0;
  I.store = nullptr;
  I.wacc_off = -1;  // its few chunks' FP64 slices stay in L2: FP64 adds per tile

  cudaStream_t s = (cudaStream_t)stream;
  // every buffer below is fully written before it is read: the transpose
  // fills Wt, each chunk zeroes its gradient slice and writes its loss slice,
  // and each tile writes its scratch jets before reading them
  e = launch_transpose_weights(I, fp64, b, s);
  if (e != cudaSuccess) return nfail_cuda(e, "transpose launch");
  SimtArgs a;
  memset(&a, 0, sizeof(a));
  a.mode = MODE_FWD_BWD;
  a.n_inst = 1;
  a.inst0 = I;
  a.n_items = I.n_chunks;
  a.scratch = scr;
  a.scratch_stride = jet_elems;
  e = launch_by_class(best, fp64, a, I.n_chunks, smem, s);
  if (e != cudaSuccess) return nfail_cuda(e, "kernel launch");
  ReduceJob j;
  memset(&j, 0, sizeof(j));
  j.grad_slices = I.grad_slices;
  j.loss_slices = I.loss_slices;
  j.n_chunks = I.n_chunks;
  j.n_params = I.n_params;
  j.inv_N = I.inv_N;
  j.grad_out = grad_out;
  j.loss_out = loss_out;
  e = launch_reduce(nullptr, j, 1, I.n_params, fp64, false, 1, 0.f, s);
  if (e != cudaSuccess) return nfail_cuda(e, "reduce launch");
  return JET_OK;
}
