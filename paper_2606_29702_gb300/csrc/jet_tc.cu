// Host side of the tensor-core path: plan set-up (tile size under the shared-
// memory and TMEM budgets, BF16 weight copies and their TMA tensor maps),
// per-call weight preparation and launches of the fused tcgen05 kernel.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "jet_closures_gen.h"
#include "jet_internal.h"
#include "jet_plan.h"
#include "jet_tc.h"
#include "jet_tc_kernel.cuh"

using namespace jet;

namespace jet {

template <int ID> cudaError_t tc_launch_id(const TcArgs& a, int grid, size_t smem, cudaStream_t s);
template <int ID> cudaError_t tc_max_active_id(size_t smem, int threads, int* blocks);
template <int ID> cudaError_t tc_attrs_id(cudaFuncAttributes* a);

struct TcPlan {
  int w = 0, H = 1, P = 0, cols = 0, cols_pad = 0, top_cols = 0, split3 = 0;
  // packing: G = 128 / wu sub-tiles of Pc points each share the MMA rows
  // (block-diagonal weights); w = G * wu is the width the MMAs see
  int wu = 0, G = 1, Pc = 0;
  // store-mode plans whose tile only fits with one activation buffer: the
  // weight gradient always runs as the separate GEMM (never per tile), so
  // the layer input and its adjoint never need to be in shared memory together
  bool single_act = false;
  int tmem_cols = 0, ctas_per_sm = 1, grid = 0;
  int nthreads = 512;  // CTA size: 512 (one CTA per SM) or 256 (two)
  size_t smem = 0;
  int o_w, o_wlo, o_a0, o_a1, o_alo0, o_alo1, o_uo, o_ub, o_xs, o_red, o_part;
  int act_bytes = 0, alo_bytes = 0, r0w = 0, r1w = 0;
  long long scratch_stride = 0;
  // per-CTA scratch slot: A^1..A^{L-3} copies, then (plans that can run the
  // weight gradient per tile) the chunk's FP32 weight-gradient accumulator
  long long wacc_off = -1;
  // workspace
  __nv_bfloat16* Wh = nullptr;   // hidden weights [L-2][w][w]
  __nv_bfloat16* Wl = nullptr;   // output weights [n_out][w]
  __nv_bfloat16* Wlo = nullptr;  // low parts [L-2][w][w]
  double* grad_slices = nullptr;
  double* loss_slices = nullptr;
  unsigned char* scratch = nullptr;
  int* err = nullptr;
  int* h_err = nullptr;
  cudaEvent_t err_ev = nullptr;
  size_t ws_bytes = 0;
  CUtensorMap wmap, wlmap, wlomap;
  // per-chunk FP64 gradient slices when they fit in a share of L2, else one
  // accumulator that every chunk adds into (atomic order not fixed)
  bool shared_acc = false;
  // store mode of the weight gradient (JET_FLAG_STORE with a memory budget):
  // per tile A^1..A^{L-2} and Zbar^2..Zbar^{L-1} in HBM, reduced by the
  // weight-gradient GEMM kernel into one FP64 partial per work item
  unsigned char* wstore = nullptr;
  long long wstore_tile_stride = 0, wstore_tiles = 0;
  size_t wstore_budget = 0;  // grown on demand up to this many bytes
  float* wg_out = nullptr;  // [max_items][w*w]
  int wg_max_items = 0, wg_sms = 0;
};

// budget of the per-chunk gradient slices (their bias, output-layer and
// first-layer entries take FP64 adds every tile, so they should stay in L2)
constexpr double kSliceBudgetBytes = 48.0 * 1024 * 1024;

// ------------------------------------------------------------------ weight-gradient GEMM
// Wbar^l = sum over the tiles of a K range of Zbar^l A^{l-1}^T, both operands
// read from the store in the fused kernel's swizzled layout, 64 columns
// (one layout chunk) per pipeline stage; the accumulator stays in TMEM for
// the whole range and is written once to the item's partial, in FP32 (the
// accumulator's own precision).
struct WgArgs {
  const unsigned char* wstore;
  long long tile_stride;  // bytes per tile in the store
  long long a_slot;       // bytes between consecutive A^l copies
  long long z_off;        // offset of Zbar^2 within a tile
  int act_bytes, chunk_bytes, ach, stages;
  int L, w, H;
  long long n_tiles;
  int items_per_layer, n_items;
  long long tiles_per_item;
  float* out;
  int* err;
  int tmem_cols;
};

constexpr int kWgThreads = 128;
constexpr int kWgMaxStages = 4;

__global__ void __launch_bounds__(kWgThreads, 1) wgrad_kernel(const __grid_constant__ WgArgs a) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full[kWgMaxStages], empty[kWgMaxStages], done;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int abort_s;
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    abort_s = 0;
    for (int s = 0; s < kWgMaxStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(&done, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_s, (uint32_t)a.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = tmem_s;
  // phase parities of the full / empty barriers, one bit per stage (registers, not a local array)
  uint32_t fph = 0, eph = 0, dph = 0;
  const int ww = a.w * a.w;
  const uint32_t id = tc::idesc_bf16(128, a.w, 0, 0);
  for (int item = blockIdx.x; item < a.n_items && !abort_s; item += gridDim.x) {
    const int l = item / a.items_per_layer + 2;
    const long long t0 = (long long)(item % a.items_per_layer) * a.tiles_per_item;
    const long long t1 = t0 + a.tiles_per_item < a.n_tiles ? t0 + a.tiles_per_item : a.n_tiles;
    const long long nch = t1 > t0 ? (t1 - t0) * a.ach : 0;
    float* out = a.out + (long long)item * ww;
    if (nch == 0) {
      for (int i = tid; i < ww; i += kWgThreads) out[i] = 0.f;
      continue;
    }
    if (tid == 0) {
      uint32_t pending = 0;  // stages whose MMAs are not yet known complete, one bit each
      auto load = [&](long long i, int st) {
        const long long t = t0 + i / a.ach;
        const int cc = (int)(i % a.ach);
        const unsigned char* base = a.wstore + t * a.tile_stride;
        unsigned char* zs = sm + (size_t)st * 2 * a.chunk_bytes;
        tc::mbar_arrive_expect_tx(&full[st], (uint32_t)(2 * a.chunk_bytes));
        tc::bulk_g2s(zs, base + a.z_off + (long long)(l - 2) * a.act_bytes + (long long)cc * a.chunk_bytes,
                     (uint32_t)a.chunk_bytes, &full[st]);
        tc::bulk_g2s(zs + a.chunk_bytes, base + (long long)(l - 2) * a.a_slot + (long long)cc * a.chunk_bytes,
                     (uint32_t)a.chunk_bytes, &full[st]);
      };
      const int S = a.stages;
      for (long long i = 0; i < S && i < nch; ++i) load(i, (int)i);
      for (long long i = 0; i < nch && !abort_s; ++i) {
        const int st = (int)(i % S);
        if (!tc::mbar_wait(&full[st], (fph >> st) & 1u, &abort_s, a.err, 71)) break;
        fph ^= 1u << st;
        tc::tc_fence_after();
        const uint32_t zs = tc::smem_u32(sm + (size_t)st * 2 * a.chunk_bytes);
        const uint32_t as = zs + (uint32_t)a.chunk_bytes;
        for (int h = 0; h < a.H; ++h)
          for (int s = 0; s < 4; ++s)
            tc::mma_f16(tmem + (uint32_t)(h * a.w), tc::sdesc(zs + (uint32_t)h * 16384u + (uint32_t)s * 32u, 16, 1024),
                        tc::sdesc(as + (uint32_t)s * 32u, 16, 1024), id, (i > 0 || s > 0) ? 1u : 0u);
        tc::mma_commit(&empty[st]);
        pending |= 1u << st;
        // refill the previous chunk's stage once its MMAs (queued before this
        // chunk's) are done: the tensor pipe keeps a chunk queued meanwhile
        const long long j = i - 1;
        if (j >= 0 && j + S < nch) {
          const int sj = (int)(j % S);
          if (!tc::mbar_wait(&empty[sj], (eph >> sj) & 1u, &abort_s, a.err, 72)) break;
          eph ^= 1u << sj;
          pending &= ~(1u << sj);
          load(j + S, sj);
        }
      }
      for (int st = 0; st < S; ++st)
        if ((pending >> st) & 1u) {
          tc::mbar_wait(&empty[st], (eph >> st) & 1u, &abort_s, a.err, 73);
          eph ^= 1u << st;
        }
      tc::mma_commit(&done);
    }
    if (!tc::mbar_wait(&done, dph & 1u, &abort_s, a.err, 74)) break;
    ++dph;
    tc::tc_fence_after();
    for (int h = 0; h < a.H; ++h) {
      const int row = h * 128 + tid;
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(h * a.w);
      float* orow = out + (long long)row * a.w;
      int k0 = 0;
      // four loads of 8 columns in flight per wait, 128-byte row segments out
      for (; k0 + 32 <= a.w; k0 += 32) {
        float v[32];
        tc::tmem_ld8(ta + (uint32_t)k0, v);
        tc::tmem_ld8(ta + (uint32_t)(k0 + 8), v + 8);
        tc::tmem_ld8(ta + (uint32_t)(k0 + 16), v + 16);
        tc::tmem_ld8(ta + (uint32_t)(k0 + 24), v + 24);
        tc::tmem_wait_ld();
        if (row < a.w)
#pragma unroll
          for (int i = 0; i < 32; i += 4)
            *reinterpret_cast<float4*>(orow + k0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      }
      for (; k0 < a.w; k0 += 8) {
        float v[8];
        tc::tmem_ld8(ta + (uint32_t)k0, v);
        tc::tmem_wait_ld();
        if (row < a.w)
#pragma unroll
          for (int i = 0; i < 8; ++i) orow[k0 + i] = v[i];
      }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// dst[off_W[l-1] + i*wu + k] += sum over the items of layer l and over the
// G diagonal blocks of out[item] (w = G * wu: packed sub-tiles contribute
// only within their own block)
struct OffWl {
  long long v[kMaxLayers];
};

// Four consecutive elements of a row per thread (hidden widths are multiples
// of 32), 16-byte loads; each element's items in item order, eight at a time
// in FP32 before each FP64 add.  offW is a __grid_constant__: read in place,
// not copied to local memory for its runtime index.
__global__ void wgrad_sum4_kernel(const float* out, int L, int w, int wu, int G, int ipl,
                                  const __grid_constant__ OffWl offW, double* dst) {
  const long long ww = (long long)w * w, uu = (long long)wu * wu, total4 = (long long)(L - 2) * uu / 4;
  for (long long e4 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e4 < total4;
       e4 += (long long)gridDim.x * blockDim.x) {
    const long long e = e4 * 4;
    const int li = (int)(e / uu);
    const long long r = e % uu;
    const int i = (int)(r / wu), k = (int)(r % wu);
    const float* src = out + (long long)li * ipl * ww;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int b = 0; b < G; ++b) {
      const float* p = src + (long long)(b * wu + i) * w + b * wu + k;
      int it = 0;
      // eight items' loads in flight; their FP32 sum (in item order) takes
      // one FP64 add, since FP64 arithmetic, not HBM, bounds a per-item add
      for (; it + 8 <= ipl; it += 8) {
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = __ldg(reinterpret_cast<const float4*>(p + (it + q) * ww));
        float4 f = v[0];
#pragma unroll
        for (int q = 1; q < 8; ++q) {
          f.x += v[q].x;
          f.y += v[q].y;
          f.z += v[q].z;
          f.w += v[q].w;
        }
        s0 += (double)f.x;
        s1 += (double)f.y;
        s2 += (double)f.z;
        s3 += (double)f.w;
      }
      for (; it < ipl; ++it) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p + it * ww));
        s0 += (double)v.x;
        s1 += (double)v.y;
        s2 += (double)v.z;
        s3 += (double)v.w;
      }
    }
    double* d = dst + offW.v[li + 1] + r;
    d[0] += s0;
    d[1] += s1;
    d[2] += s2;
    d[3] += s3;
  }
}

}  // namespace jet

namespace {

cudaError_t tc_launch(int cls, const TcArgs& a, int grid, size_t smem, cudaStream_t s) {
  switch (cls) {
#define CASE(id, cl) \
  case id:           \
    return tc_launch_id<id>(a, grid, smem, s);
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t tc_occupancy(int cls, size_t smem, int threads, int* blocks) {
  switch (cls) {
#define CASE(id, cl) \
  case id:           \
    return tc_max_active_id<id>(smem, threads, blocks);
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  return cudaErrorInvalidValue;
}

// CTAs of the fused kernel that fit one SM by registers and shared memory.
// The runtime's occupancy query reports one CTA per SM for any kernel that
// contains TMEM instructions; measured residency shows two such CTAs running
// on one SM at once when their TMEM allocations fit together (the plan keeps
// the sum at or below 512 columns), so the count is derived here from the
// kernel's own attributes.
cudaError_t tc_fit(int cls, size_t smem, int threads, int* blocks) {
  cudaFuncAttributes a;
  cudaError_t e = cudaErrorInvalidValue;
  switch (cls) {
#define CASE(id, cl)            \
  case id:                      \
    e = tc_attrs_id<id>(&a);    \
    break;
    JET_FOR_EACH_CLASS(CASE)
#undef CASE
  }
  if (e != cudaSuccess) return e;
  int dev = 0, smem_sm = 0, regs_sm = 0, reserved = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess) return e;
  const int warps = (threads + 31) / 32;
  const int regs_warp = (a.numRegs * 32 + 255) / 256 * 256;  // 256-register allocation unit
  const size_t smem_cta = smem + a.sharedSizeBytes + (size_t)reserved;
  const int by_regs = regs_sm / std::max(1, warps * regs_warp);
  const int by_smem = (int)((size_t)smem_sm / std::max<size_t>(1, smem_cta));
  *blocks = std::min(by_regs, by_smem);
  return cudaSuccess;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// bf16 tensor [n2][n1][n0] (n0 contiguous), box (64, box1, 1), 128-byte swizzle
bool encode(CUtensorMap* m, void* base, cuuint64_t n0, cuuint64_t n1, cuuint64_t n2, cuuint32_t box1, int rank) {
  EncodeTiledFn fn = encoder();
  if (!fn) return false;
  cuuint64_t dims[3] = {n0, n1, n2};
  cuuint64_t strides[2] = {n0 * 2, n0 * n1 * 2};
  cuuint32_t box[3] = {64, box1, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// fp32 packed params -> bf16 hidden / output weights (and split low parts)
struct OffW {
  long long v[kMaxLayers];
};

// One plan's weight preparation: elements [start, start + nh + nl) of a
// (batched) preparation launch.
struct PrepJob {
  const float* params;
  OffW offW;
  __nv_bfloat16* Wh;
  __nv_bfloat16* Wl;
  __nv_bfloat16* Wlo;
  long long nh, nl, start;
  int L, w, wu, n_out;
};

// BF16 copies of the weights in the MMA's view: W^l (l = 2..L-1) as a
// [w][w] block-diagonal matrix of G copies of the wu x wu weights, and the
// output weights as [128][w]: in every 32-row lane quadrant, row s * n_out + o
// holds W^L[o] in the columns of sub-tile s (G = 1: plain copies), so that
// the output rows of D sit in all four TMEM lane quadrants.  Element i < nh of
// the job is a hidden weight, the rest output weights.
__device__ __forceinline__ void prep_element(const PrepJob& j, long long i) {
  const int w = j.w, wu = j.wu;
  if (i < j.nh) {
    const long long l = i / ((long long)w * w), r = i % ((long long)w * w);
    const int row = (int)(r / w), col = (int)(r % w);
    const float v = row / wu == col / wu ? j.params[j.offW.v[l + 1] + (long long)(row % wu) * wu + col % wu] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    j.Wh[i] = hi;
    if (j.Wlo) j.Wlo[i] = __float2bfloat16_rn(v - __bfloat162float(hi));
  } else {
    const long long r = i - j.nh;
    const int row = (int)(r / w) & 31, col = (int)(r % w);
    const int sub = row / j.n_out, o = row % j.n_out;
    const bool live = row < (w / wu) * j.n_out && col / wu == sub;
    j.Wl[r] = __float2bfloat16_rn(live ? j.params[j.offW.v[j.L - 1] + (long long)o * wu + col % wu] : 0.f);
  }
}

__global__ void tc_prep_kernel_v(const PrepJob j) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < j.nh + j.nl;
       i += (long long)gridDim.x * blockDim.x)
    prep_element(j, i);
}

// all plans of a batch in one launch: element i belongs to the last job
// whose start is <= i (jobs ordered by start)
__global__ void tc_prep_batch_kernel(const PrepJob* jobs, int n, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (jobs[mid].start <= i) lo = mid;
      else hi = mid - 1;
    }
    prep_element(jobs[lo], i - jobs[lo].start);
  }
}

jet_status tfail(jet_status st, const char* msg) {
  jet::set_last_error(msg);
  return st;
}

jet_status tcuda(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  jet::set_last_error(buf);
  return e == cudaErrorMemoryAllocation ? JET_ERR_OOM : JET_ERR_CUDA;
}

// shared-memory carve for tile size P; returns total bytes (without the 1 KB alignment slack)
size_t carve(TcPlan& t, int C, int n_out, int d) {
  const int R = 128 * t.H;
  const int nck = std::max(2, t.w / 64);
  const int ach = (t.cols_pad + 63) / 64;
  const int lch = t.split3 ? (t.top_cols + 63) / 64 : 0;
  size_t off = 0;
  t.o_w = (int)off;
  off += (size_t)nck * R * 128;
  t.o_wlo = (int)off;
  if (t.split3) off += (size_t)nck * R * 128;
  t.act_bytes = ach * (R / 8) * 1024;
  t.alo_bytes = lch * (R / 8) * 1024;
  t.o_a0 = (int)off;
  off += t.act_bytes;
  t.o_a1 = t.single_act ? t.o_a0 : (int)off;
  if (!t.single_act) off += t.act_bytes;
  t.o_alo0 = (int)off;
  off += t.alo_bytes;
  t.o_alo1 = t.single_act ? t.o_alo0 : (int)off;
  if (!t.single_act) off += t.alo_bytes;
  t.o_uo = (int)off;
  off += (size_t)n_out * C * t.P * 4;
  t.o_ub = (int)off;
  off += (size_t)n_out * C * t.P * 4;
  t.o_xs = (int)off;
  off += (size_t)t.P * d * 4;
  off = (off + 15) / 16 * 16;
  t.o_red = (int)off;
  off += 64;
  t.o_part = (int)off;
  off += (size_t)(t.nthreads / 128) * 4 * 256 * sizeof(float);
  return off;
}

}  // namespace

jet_status tc_plan_create(jet_plan_s* p, TcPlan** out, const cudaDeviceProp& prop, size_t mem_budget, int flags) {
  *out = nullptr;
  if (p->prec == JET_TF32) return tfail(JET_ERR_UNSUPPORTED, "JET_TF32 is not provided by this build");
  const int L = p->L, w = p->widths[1];
  for (int l = 1; l < L; ++l)
    if (p->widths[l] != w) return tfail(JET_ERR_UNSUPPORTED, "tensor-core path needs equal hidden widths");
  if (w % 32 || w < 32 || w > 256) return tfail(JET_ERR_UNSUPPORTED, "tensor-core path needs hidden width 32..256, multiple of 32");
  if (!encoder()) return tfail(JET_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
  if (p->prec == JET_BF16X3 && w > 128)
    return tfail(JET_ERR_UNSUPPORTED, "JET_BF16X3 needs hidden width <= 128 (high and low weights share shared memory)");
  const int C = p->C, maxord = kClassInfo[p->cls].maxord;
  int top_begin = 0;
  for (int c = 0; c < C; ++c) {
    int o = 0;
    for (int j = 0; j < 3; ++j) o += kClassInfo[p->cls].alpha[c][j];
    if (o == maxord) {
      top_begin = c;
      break;
    }
  }
  TcPlan* t = new TcPlan();
  // widths 32 and 64 pack 4 or 2 sub-tiles into the 128 MMA rows, so that
  // every TMEM lane quadrant (and so every epilogue warp) holds units
  t->wu = w;
  t->G = w <= 64 ? 128 / w : 1;
  t->w = t->G * w;
  t->H = t->w > 128 ? 2 : 1;
  t->split3 = p->prec == JET_BF16X3 ? 1 : 0;
  const int ntop = C - top_begin;
  // choose the CTA shape and P: most points in flight per SM (P x CTAs per
  // SM, doubled for tiles that give every warpgroup whole epilogue passes)
  // within shared memory and TMEM (512 columns per SM); on a tie one CTA of
  // 16 warps with the larger tile wins (measured faster than two CTAs of 8
  // warps with half the tile on the KS and NS workloads)
  int best_score = -1;
  TcPlan best = *t;
  const int p8 = JET_FLAG_TILE_GET(flags), want_ctas = JET_FLAG_CTAS_GET(flags);
  const bool want_store = (flags & JET_FLAG_STORE) && mem_budget > 0 && L >= 3;
  if (want_ctas > 2) {
    delete t;
    return tfail(JET_ERR_INVALID, "JET_FLAG_CTAS takes 0, 1 or 2");
  }
  char why[160] = "no candidate tile";  // last rejection, for the error message
  for (int ctas = 1; ctas <= 2; ++ctas) {
    if (want_ctas && ctas != want_ctas) continue;
    for (int Pc = 8; Pc <= 64; Pc += 8) {
      const int P = t->G * Pc;  // points per tile; Pc per sub-tile
      if (p8 && P != 8 * p8) {
        if (8 * p8 % (8 * t->G)) snprintf(why, sizeof(why), "P=%d is not a multiple of %d (packed sub-tiles)", 8 * p8, 8 * t->G);
        continue;
      }
      TcPlan c = *t;
      c.nthreads = 512 / ctas;
      c.P = P;
      c.Pc = Pc;
      c.cols = C * Pc;
      c.cols_pad = (c.cols + 15) / 16 * 16;
      if (c.cols_pad > 256) break;
      c.top_cols = ntop * Pc;
      if (c.split3 && c.top_cols % 16) {
        snprintf(why, sizeof(why), "P=%d: split columns not a multiple of 16", P);
        continue;
      }
      size_t sm = carve(c, C, p->n_out, p->d) + 1024;
      if (sm > (size_t)(226 * 1024) / ctas && want_store) {
        c.single_act = true;  // store mode: one activation buffer may be enough
        sm = carve(c, C, p->n_out, p->d) + 1024;
      }
      if (sm > (size_t)(226 * 1024) / ctas) {
        snprintf(why, sizeof(why), "P=%d, %d CTA/SM: %zu B of shared memory", P, ctas, sm);
        continue;
      }
      const int NB = c.H == 2 ? 128 : c.w;  // N of the weight-gradient MMA (the MMA width)
      c.r0w = c.single_act ? c.cols_pad : std::max(c.cols_pad, NB);
      c.r1w = c.cols_pad;
      const int need = c.H * (c.r0w + c.r1w);
      int tm = 32;
      while (tm < need) tm *= 2;
      if (tm > 512 / ctas) {
        snprintf(why, sizeof(why), "P=%d, %d CTA/SM: %d TMEM columns", P, ctas, tm);
        continue;
      }
      c.tmem_cols = tm;
      int by_occ = 0;  // registers and shared memory
      const cudaError_t oe = ctas == 1 ? tc_occupancy(p->cls, sm, c.nthreads, &by_occ)
                                       : tc_fit(p->cls, sm, c.nthreads, &by_occ);
      if (oe != cudaSuccess || by_occ < ctas) {
        snprintf(why, sizeof(why), "P=%d, %d CTA/SM: occupancy %d (%s, %zu B shared)", P, ctas, by_occ,
                 cudaGetErrorString(oe), sm);
        cudaGetLastError();
        continue;
      }
      c.ctas_per_sm = ctas;
      // the epilogues give each warpgroup passes of 4 points (up to 7
      // channels) or 2: a tile that splits into whole passes counts double
      const int pw = C <= 7 ? 4 : 2;
      const bool whole = Pc % (pw * (c.nthreads / 128)) == 0;
      const int score = 2 * P * ctas * (whole ? 2 : 1) + (ctas == 1 ? 1 : 0);
      if (score > best_score) {
        best_score = score;
        best = c;
      }
    }
  }
  if (best_score < 0) {
    delete t;
    char msg[224];
    snprintf(msg, sizeof(msg), "no tile size fits shared memory and TMEM (%s)", why);
    return tfail(JET_ERR_UNSUPPORTED, msg);
  }
  *t = best;
  // pad the shared-memory request so that no more CTAs share an SM than TMEM allows
  size_t sm = carve(*t, C, p->n_out, p->d) + 1024;
  const size_t floor_sm = (228 * 1024) / (t->ctas_per_sm + 1) + 1024;
  t->smem = std::max(sm, floor_sm);
  int occ = 0;
  cudaError_t e = t->ctas_per_sm == 1 ? tc_occupancy(p->cls, t->smem, t->nthreads, &occ)
                                      : tc_fit(p->cls, t->smem, t->nthreads, &occ);
  if (e != cudaSuccess || occ < 1) {
    delete t;
    return e != cudaSuccess ? tcuda(e, "tc occupancy") : tfail(JET_ERR_UNSUPPORTED, "tensor-core tile does not fit");
  }
  t->ctas_per_sm = std::min(t->ctas_per_sm, occ);
  t->grid = prop.multiProcessorCount * t->ctas_per_sm;
  t->scratch_stride = ((long long)std::max(0, L - 3) * (t->act_bytes + t->alo_bytes) + 15) / 16 * 16;
  if (!t->single_act) {
    t->wacc_off = t->scratch_stride;
    t->scratch_stride += (long long)std::max(0, L - 2) * t->G * t->wu * t->wu * (long long)sizeof(float);
  }
  // workspace
  const long long nh = (long long)std::max(0, L - 2) * t->w * t->w, nl = 128LL * t->w;
  size_t b_wh = std::max<long long>(nh, 1) * 2, b_wl = nl * 2, b_wlo = t->split3 ? b_wh : 0;
  t->shared_acc = (double)t->grid * p->n_params * 8.0 > kSliceBudgetBytes;
  size_t b_gs = (size_t)(t->shared_acc ? 1 : t->grid) * p->n_params * 8, b_ls = (size_t)t->grid * 8;
  size_t b_sc = (size_t)t->grid * std::max<long long>(t->scratch_stride, 16);
  e = cudaMalloc((void**)&t->Wh, b_wh);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->Wl, b_wl);
  if (e == cudaSuccess && t->split3) e = cudaMalloc((void**)&t->Wlo, b_wlo);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->grad_slices, b_gs);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->loss_slices, b_ls);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->scratch, b_sc);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(t->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&t->h_err, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&t->err_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    tc_plan_destroy(t);
    return tcuda(e, "tensor-core workspace");
  }
  *t->h_err = 0;
  t->ws_bytes = b_wh + b_wl + b_wlo + b_gs + b_ls + b_sc;
  if (want_store) {
    t->wstore_tile_stride = (long long)(L - 2) * (t->act_bytes + t->alo_bytes) + (long long)(L - 2) * t->act_bytes;
    t->wstore_budget = mem_budget;
    if ((long long)(mem_budget / (size_t)t->wstore_tile_stride) > 0) {
      t->wg_sms = prop.multiProcessorCount;
      // items of equal size, (L - 2) * ipl of them a multiple of the CTAs, so
      // that every CTA takes the same number (no tail of a few CTAs running
      // one more item): ipl = wg_sms / gcd(wg_sms, L - 2)
      int a = t->wg_sms, b = L - 2;
      while (b) {
        const int r = a % b;
        a = b;
        b = r;
      }
      const int ipl = std::max(1, t->wg_sms / a);
      t->wg_max_items = (L - 2) * ipl;
      const size_t b_wo = (size_t)t->wg_max_items * t->w * t->w * sizeof(float);
      e = cudaMalloc((void**)&t->wg_out, b_wo);
      if (e != cudaSuccess) {
        tc_plan_destroy(t);
        return tcuda(e, "weight-gradient partials");
      }
      t->ws_bytes += b_wo;
    }
  }
  const int R = 128 * t->H;
  const int we = t->w;
  bool ok = encode(&t->wmap, t->Wh, we, we, std::max(1, L - 2), R, 3) &&
            encode(&t->wlmap, t->Wl, we, 128, 1, 128, 2);
  if (ok && t->split3) ok = encode(&t->wlomap, t->Wlo, we, we, std::max(1, L - 2), R, 3);
  if (!ok) {
    tc_plan_destroy(t);
    return tfail(JET_ERR_UNSUPPORTED, "tensor map encoding failed");
  }
  if (!t->split3) t->wlomap = t->wmap;
  *out = t;
  return JET_OK;
}

void tc_plan_destroy(TcPlan* t) {
  if (!t) return;
  cudaFree(t->Wh);
  cudaFree(t->Wl);
  cudaFree(t->Wlo);
  cudaFree(t->grad_slices);
  cudaFree(t->loss_slices);
  cudaFree(t->scratch);
  cudaFree(t->wstore);
  cudaFree(t->wg_out);
  cudaFree(t->err);
  cudaFreeHost(t->h_err);
  if (t->err_ev) cudaEventDestroy(t->err_ev);
  delete t;
}

int tc_tile_points(const TcPlan* t) { return t ? t->P : 0; }
int tc_grid(const TcPlan* t) { return t ? t->grid : 0; }
int tc_ctas_per_sm(const TcPlan* t) { return t ? t->ctas_per_sm : 0; }
int tc_threads(const TcPlan* t) { return t ? t->nthreads : 0; }
int tc_wgrad_chunk_fp32(const TcPlan* t) { return t && t->wacc_off >= 0 ? 1 : 0; }
size_t tc_workspace_bytes(const TcPlan* t) { return t ? t->ws_bytes : 0; }

namespace {

bool is_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// Device-side wait time-outs of an earlier call surface here.  While the
// stream is being captured into a CUDA graph the event query (and the
// read-back in run) would invalidate the capture: a time-out inside a replayed
// graph surfaces at the next call made outside capture.
jet_status check_err(TcPlan* t, cudaStream_t s) {
  if (is_capturing(s)) return JET_OK;
  if (cudaEventQuery(t->err_ev) == cudaSuccess && *t->h_err != 0) {
    char buf[128];
    snprintf(buf, sizeof(buf), "a bounded device wait timed out in an earlier call (code %d)", *t->h_err);
    *t->h_err = 0;
    cudaMemset(t->err, 0, sizeof(int));
    jet::set_last_error(buf);
    return JET_ERR_TIMEOUT;
  }
  return JET_OK;
}

void fill_tc(const jet_plan_s* p, const TcPlan* t, const void* params, const void* X, long long N, const void* source,
             void* r_out, TcInst& I) {
  memset(&I, 0, sizeof(I));
  I.wmap = t->wmap;
  I.wlmap = t->wlmap;
  I.wlomap = t->wlomap;
  I.L = p->L;
  I.d = p->d;
  I.n_out = p->n_out;
  I.n_res = p->n_res;
  I.w = t->w;
  I.wu = t->wu;
  I.G = t->G;
  I.Pc = t->Pc;
  I.H = t->H;
  I.P = t->P;
  I.cols = t->cols;
  I.cols_pad = t->cols_pad;
  I.top_cols = t->top_cols;
  I.split3 = t->split3;
  I.n_terms = (int)p->terms.size();
  for (int m = 0; m < I.n_terms; ++m) {
    I.terms[m] = p->terms[m];
    I.coef_f[m] = (float)p->terms[m].coef;
  }
  I.n_groups = p->n_groups > 0 ? jet::fill_groups(p, I.groups) : 0;
  {  // per output-jet slot, the (monomial, factor) pairs that read it, in (m, f) order
    int e = 0;
    const int nslot = p->n_out * p->C;
    for (int k = 0; k < nslot; ++k) {
      I.adj_off[k] = (short)e;
      for (int m = 0; m < I.n_terms; ++m)
        for (int f = 0; f < I.terms[m].nfac; ++f)
          if (I.terms[m].fac[f] == k) I.adj_mf[e++] = (unsigned char)(m * 4 + f);
    }
    I.adj_off[nslot] = (short)e;
  }
  I.params = reinterpret_cast<const float*>(params);
  for (int l = 0; l < p->L; ++l) {
    I.off_W[l] = p->off_W[l];
    I.off_b[l] = p->off_b[l];
  }
  I.n_params = p->n_params;
  I.X = reinterpret_cast<const float*>(X);
  I.source = reinterpret_cast<const float*>(source);
  I.r_out = reinterpret_cast<float*>(r_out);
  I.N = N;
  I.inv_N = p->n_groups > 0 ? 1.0 : (N > 0 ? 1.0 / (double)N : 0.0);  // a composite loss scales per term
  I.n_tiles = (N + t->P - 1) / t->P;
  long long chunks = std::min<long long>(std::max<long long>(I.n_tiles, 1), t->grid);
  I.tiles_per_chunk = (int)((I.n_tiles + chunks - 1) / chunks);
  if (I.tiles_per_chunk < 1) I.tiles_per_chunk = 1;
  I.n_chunks = (int)((I.n_tiles + I.tiles_per_chunk - 1) / I.tiles_per_chunk);
  I.chunk_base = 0;
  I.grad_slices = t->grad_slices;
  I.loss_slices = t->loss_slices;
  I.scratch = t->scratch;
  I.scratch_stride = t->scratch_stride;
  I.wacc_off = t->wacc_off;
  I.o_w = t->o_w;
  I.o_wlo = t->o_wlo;
  I.o_a0 = t->o_a0;
  I.o_a1 = t->o_a1;
  I.o_alo0 = t->o_alo0;
  I.o_alo1 = t->o_alo1;
  I.o_uo = t->o_uo;
  I.o_ub = t->o_ub;
  I.o_xs = t->o_xs;
  I.o_red = t->o_red;
  I.o_part = t->o_part;
  I.act_bytes = t->act_bytes;
  I.alo_bytes = t->alo_bytes;
  I.r0w = t->r0w;
  I.r1w = t->r1w;
  I.slice_shared = t->shared_acc ? 1 : 0;
  const bool use_store = t->wstore && I.n_tiles <= t->wstore_tiles;
  I.wstore = use_store ? t->wstore : nullptr;
  I.wstore_tile_stride = t->wstore_tile_stride;
}

// Grow the weight-gradient store to the tiles of N points when the plan's
// budget allows; otherwise the call runs in per-tile mode.  A call that grows
// it allocates (and cudaFree synchronises): make the first call with the
// largest N before any stream capture.
jet_status store_too_small(const TcPlan* t, long long N) {
  char msg[200];
  snprintf(msg, sizeof(msg),
           "this plan's tile keeps one activation buffer and needs the weight-gradient store, which cannot hold "
           "%lld points within mem_budget (%zu bytes): raise mem_budget or use a smaller tile",
           N, t->wstore_budget);
  return tfail(JET_ERR_OOM, msg);
}

void ensure_store(TcPlan* t, long long N, cudaStream_t s) {
  if (!t->wstore_budget || !t->wg_out || N < 1 || is_capturing(s)) return;
  const long long tiles = (N + t->P - 1) / t->P;
  if (tiles <= t->wstore_tiles) return;
  const size_t need = (size_t)tiles * (size_t)t->wstore_tile_stride;
  if (need > t->wstore_budget) return;
  if (t->wstore) {
    cudaFree(t->wstore);
    t->ws_bytes -= (size_t)t->wstore_tiles * (size_t)t->wstore_tile_stride;
    t->wstore = nullptr;
    t->wstore_tiles = 0;
  }
  if (cudaMalloc((void**)&t->wstore, need) == cudaSuccess) {
    t->wstore_tiles = tiles;
    t->ws_bytes += need;
  } else {
    t->wstore = nullptr;
    cudaGetLastError();  // clear: this N runs in per-tile mode
  }
}

PrepJob prep_job(const jet_plan_s* p, const TcPlan* t, const void* params, long long start) {
  PrepJob j;
  memset(&j, 0, sizeof(j));
  j.params = reinterpret_cast<const float*>(params);
  for (int l = 0; l < p->L; ++l) j.offW.v[l] = p->off_W[l];
  j.Wh = t->Wh;
  j.Wl = t->Wl;
  j.Wlo = t->Wlo;
  j.nh = (long long)std::max(0, p->L - 2) * t->w * t->w;
  j.nl = 128LL * t->w;
  j.start = start;
  j.L = p->L;
  j.w = t->w;
  j.wu = t->wu;
  j.n_out = p->n_out;
  return j;
}

jet_status prep(const jet_plan_s* p, TcPlan* t, const void* params, cudaStream_t s) {
  const PrepJob j = prep_job(p, t, params, 0);
  int grid = (int)std::min<long long>((j.nh + j.nl + 255) / 256, 1024);
  tc_prep_kernel_v<<<grid, 256, 0, s>>>(j);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? JET_OK : tcuda(e, "tc prep launch");
}

jet_status run(jet_plan_s* p, TcPlan* t, int mode, const TcInst& I, cudaStream_t s) {
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.inst0 = I;
  a.shape[0] = I.Pc;
  a.shape[1] = I.G;
  a.shape[2] = I.H;
  a.shape[3] = I.w;
  a.mode = mode;
  a.n_items = I.n_chunks;
  a.insts = nullptr;
  a.item_inst = nullptr;
  a.err = t->err;
  a.tmem_cols = t->tmem_cols;
  a.nthreads = t->nthreads;
  const int grid = std::min(t->grid, I.n_chunks);
  if (mode != MODE_FWD && t->shared_acc) {
    cudaError_t z = cudaMemsetAsync(t->grad_slices, 0, (size_t)p->n_params * sizeof(double), s);
    if (z != cudaSuccess) return tcuda(z, "accumulator reset");
  }
  jet::plan_prof_begin(p, s);
  cudaError_t e = tc_launch(p->cls, a, grid, t->smem, s);
  if (e == cudaSuccess && mode != MODE_FWD && I.wstore) {
    // weight gradients of the hidden-to-hidden layers from the store
    WgArgs w;
    memset(&w, 0, sizeof(w));
    const int L = p->L, R = 128 * t->H;
    w.wstore = I.wstore;
    w.tile_stride = t->wstore_tile_stride;
    w.a_slot = t->act_bytes + t->alo_bytes;
    w.z_off = (long long)(L - 2) * w.a_slot;
    w.act_bytes = t->act_bytes;
    w.chunk_bytes = (R / 8) * 1024;
    w.ach = t->act_bytes / w.chunk_bytes;
    w.stages = std::min(kWgMaxStages, (int)((200 * 1024) / (2 * w.chunk_bytes)));
    w.L = L;
    w.w = t->w;
    w.H = t->H;
    w.n_tiles = I.n_tiles;
    w.items_per_layer = t->wg_max_items / (L - 2);
    w.tiles_per_item = (I.n_tiles + w.items_per_layer - 1) / w.items_per_layer;
    w.items_per_layer = (int)((I.n_tiles + w.tiles_per_item - 1) / w.tiles_per_item);
    w.n_items = (L - 2) * w.items_per_layer;
    w.out = t->wg_out;
    w.err = t->err;
    int tm = 32;
    while (tm < t->H * t->w) tm *= 2;
    w.tmem_cols = tm;
    const size_t smem = (size_t)w.stages * 2 * w.chunk_bytes + 1024;
    e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      wgrad_kernel<<<std::min(w.n_items, t->wg_sms), kWgThreads, smem, s>>>(w);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      OffWl ow;
      for (int l = 0; l < L; ++l) ow.v[l] = p->off_W[l];
      const long long tot = (long long)(L - 2) * t->wu * t->wu;
      wgrad_sum4_kernel<<<(int)std::min<long long>((tot / 4 + 255) / 256, 2048), 256, 0, s>>>(
          t->wg_out, L, t->w, t->wu, t->G, w.items_per_layer, ow, t->grad_slices);
      e = cudaGetLastError();
    }
  }
  jet::plan_prof_end(p, s);
  if (e != cudaSuccess) return tcuda(e, "tc kernel launch");
  if (is_capturing(s)) return JET_OK;
  e = cudaMemcpyAsync(t->h_err, t->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(t->err_ev, s);
  return e == cudaSuccess ? JET_OK : tcuda(e, "tc error read-back");
}

}  // namespace

jet_status tc_forward(jet_plan_s* p, TcPlan* t, const void* params, const void* X, long long N, const void* source,
                      void* r_out, double* loss_out, cudaStream_t s) {
  jet_status st = check_err(t, s);
  if (st != JET_OK) return st;
  if (N == 0) {
    if (loss_out && cudaMemsetAsync(loss_out, 0, sizeof(double), s) != cudaSuccess) return tcuda(cudaGetLastError(), "memset");
    return JET_OK;
  }
  st = prep(p, t, params, s);
  if (st != JET_OK) return st;
  TcInst I;
  fill_tc(p, t, params, X, N, source, r_out, I);
  st = run(p, t, MODE_FWD, I, s);
  if (st != JET_OK) return st;
  if (loss_out) {
    ReduceJob j;
    memset(&j, 0, sizeof(j));
    j.loss_slices = I.loss_slices;
    j.n_chunks = I.n_chunks;
    j.inv_N = I.inv_N;
    j.loss_out = loss_out;
    cudaError_t e = launch_reduce(nullptr, j, 1, 1, false, false, 1, 0.f, s);
    if (e != cudaSuccess) return tcuda(e, "reduce");
  }
  return JET_OK;
}

jet_status tc_backward(jet_plan_s* p, TcPlan* t, const void* params, const void* X, long long N, const void* source,
                       void* grad_out, void* r_out, double* loss_out, cudaStream_t s) {
  jet_status st = check_err(t, s);
  if (st != JET_OK) return st;
  if (N == 0) {
    cudaMemsetAsync(grad_out, 0, p->n_params * 4, s);
    if (loss_out) cudaMemsetAsync(loss_out, 0, sizeof(double), s);
    return JET_OK;
  }
  ensure_store(t, N, s);
  st = prep(p, t, params, s);
  if (st != JET_OK) return st;
  TcInst I;
  fill_tc(p, t, params, X, N, source, r_out, I);
  if (t->single_act && !I.wstore) return store_too_small(t, N);
  st = run(p, t, MODE_FWD_BWD, I, s);
  if (st != JET_OK) return st;
  ReduceJob j;
  memset(&j, 0, sizeof(j));
  j.grad_slices = I.grad_slices;
  j.loss_slices = I.loss_slices;
  j.n_chunks = I.n_chunks;
  j.n_params = p->n_params;
  j.grad_chunks = t->shared_acc ? 1 : 0;
  j.inv_N = I.inv_N;
  j.grad_out = grad_out;
  j.loss_out = loss_out;
  cudaError_t e = launch_reduce(nullptr, j, 1, p->n_params, false, false, 1, 0.f, s);
  return e == cudaSuccess ? JET_OK : tcuda(e, "reduce");
}

jet_status tc_train_step(jet_plan_s* p, TcPlan* t, void* params, void* m, void* v, long long step,
                         long long* step_ctr, float lr, const void* X, long long N, const void* source,
                         double* loss_out, cudaStream_t s) {
  jet_status st = check_err(t, s);
  if (st != JET_OK) return st;
  ensure_store(t, N, s);
  st = prep(p, t, params, s);
  if (st != JET_OK) return st;
  TcInst I;
  fill_tc(p, t, params, X, N, source, nullptr, I);
  if (t->single_act && !I.wstore) return store_too_small(t, N);
  st = run(p, t, MODE_FWD_BWD, I, s);
  if (st != JET_OK) return st;
  ReduceJob j;
  memset(&j, 0, sizeof(j));
  j.grad_slices = I.grad_slices;
  j.loss_slices = I.loss_slices;
  j.n_chunks = I.n_chunks;
  j.n_params = p->n_params;
  j.grad_chunks = t->shared_acc ? 1 : 0;
  j.inv_N = I.inv_N;
  j.loss_out = loss_out;
  j.params = params;
  j.m = m;
  j.v = v;
  cudaError_t e = launch_reduce(nullptr, j, 1, p->n_params, false, true, step, lr, s, step_ctr);
  return e == cudaSuccess ? JET_OK : tcuda(e, "reduce/adam");
}

// ------------------------------------------------------------------ batches
// Many plans (same channel set, any widths/depths/point counts) run as one
// persistent launch of the fused kernel over a cost-ordered list of
// (instance, chunk of tiles) items; every instance keeps its own tile size,
// BF16 weight copies and TMA tensor maps.

namespace jet {
struct TcBatch {
  int n = 0, cls = 0, grid = 0, tmem_cols = 0, max_chunks = 16, max_items = 0, n_items = 0;
  int nthreads = 512;  // smallest CTA of the member plans (their partial-sum areas fit it)
  size_t smem = 0;
  TcInst* d_insts = nullptr;
  TcInst* h_insts = nullptr;
  int* d_items = nullptr;
  int* h_items = nullptr;
  int* d_next = nullptr;  // the kernel's item counter
  ReduceJob* d_jobs = nullptr;
  ReduceJob* h_jobs = nullptr;
  PrepJob* d_prep = nullptr;  // weight preparation of every member, one launch
  PrepJob* h_prep = nullptr;
  double* grad_slices = nullptr;
  double* loss_slices = nullptr;
  std::vector<long long> slice_off;
  unsigned char* scratch = nullptr;
  long long scratch_stride = 0;
  int* err = nullptr;
  cudaEvent_t copied = nullptr;  // descriptor upload of the previous call
  bool have_prev = false;
};
}  // namespace jet

jet_status tc_batch_create(const std::vector<jet_plan_s*>& plans, TcBatch** out) {
  *out = nullptr;
  TcBatch* b = new TcBatch();
  b->n = (int)plans.size();
  b->cls = plans[0]->cls;
  long long slices = 0;
  for (jet_plan_s* p : plans)
    if (p->tcp->single_act) {
      delete b;
      return tfail(JET_ERR_UNSUPPORTED, "a plan whose tile needs the weight-gradient store cannot be batched "
                                        "(batches flush weight gradients per tile): create it without JET_FLAG_STORE");
    }
  for (jet_plan_s* p : plans) {
    TcPlan* t = p->tcp;
    b->smem = std::max(b->smem, t->smem);
    b->tmem_cols = std::max(b->tmem_cols, t->tmem_cols);
    b->nthreads = std::min(b->nthreads, t->nthreads);
    b->scratch_stride = std::max(b->scratch_stride, t->scratch_stride);
    b->slice_off.push_back(slices);
    slices += (long long)b->max_chunks * p->n_params;
  }
  int dev = 0, sms = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = b->nthreads < 512 ? tc_fit(b->cls, b->smem, b->nthreads, &occ) : tc_occupancy(b->cls, b->smem, b->nthreads, &occ);
  if (e != cudaSuccess || occ < 1) {
    delete b;
    return e != cudaSuccess ? tcuda(e, "batch occupancy") : tfail(JET_ERR_UNSUPPORTED, "batch tile does not fit");
  }
  b->grid = sms * std::max(1, std::min(occ, 512 / b->tmem_cols));
  b->max_items = b->n * b->max_chunks;
  e = cudaMalloc((void**)&b->d_insts, sizeof(TcInst) * b->n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_insts, sizeof(TcInst) * b->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_items, sizeof(int) * 2 * b->max_items);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_next, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_items, sizeof(int) * 2 * b->max_items);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_jobs, sizeof(ReduceJob) * b->n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_jobs, sizeof(ReduceJob) * b->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_prep, sizeof(PrepJob) * b->n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_prep, sizeof(PrepJob) * b->n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->grad_slices, sizeof(double) * std::max<long long>(slices, 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->loss_slices, sizeof(double) * b->max_items);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->scratch, (size_t)b->grid * std::max<long long>(b->scratch_stride, 16));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    tc_batch_destroy(b);
    return tcuda(e, "batch workspace");
  }
  memset(b->h_insts, 0, sizeof(TcInst) * b->n);
  memset(b->h_prep, 0, sizeof(PrepJob) * b->n);
  *out = b;
  return JET_OK;
}

void tc_batch_destroy(TcBatch* b) {
  if (!b) return;
  cudaFree(b->d_insts);
  cudaFreeHost(b->h_insts);
  cudaFree(b->d_items);
  cudaFree(b->d_next);
  cudaFreeHost(b->h_items);
  cudaFree(b->d_jobs);
  cudaFreeHost(b->h_jobs);
  cudaFree(b->d_prep);
  cudaFreeHost(b->h_prep);
  cudaFree(b->grad_slices);
  cudaFree(b->loss_slices);
  cudaFree(b->scratch);
  cudaFree(b->err);
  if (b->copied) cudaEventDestroy(b->copied);
  delete b;
}

jet_status tc_batch_run(TcBatch* bb, const std::vector<jet_plan_s*>& plans, const void* const* params, void* const* m,
                        void* const* v, long long step, long long* step_ctr, float lr, const void* const* X,
                        const int64_t* N,
                        const void* const* source, void* const* grad_out, double* loss_out, bool adam,
                        cudaStream_t s) {
  TcBatch* b = bb;
  const int n = b->n;
  long long total_tiles = 0;
  for (int i = 0; i < n; ++i) {
    if (N[i] < 1) return tfail(JET_ERR_INVALID, "batched calls need N >= 1 for every instance");
    if (!jet::group_counts_match(plans[i], N[i]))
      return tfail(JET_ERR_INVALID, "a composite-loss member's term points do not add up to its N");
    if (!params[i] || !X[i]) return tfail(JET_ERR_INVALID, "NULL params or X in batch");
    if (plans[i]->has_source != (source && source[i])) return tfail(JET_ERR_INVALID, "source does not match spec");
    total_tiles += (N[i] + plans[i]->tcp->P - 1) / plans[i]->tcp->P;
  }
  // weight preparation of every member: one launch over all their elements
  std::vector<PrepJob> prep_jobs(n);
  long long prep_total = 0;
  for (int i = 0; i < n; ++i) {
    prep_jobs[i] = prep_job(plans[i], plans[i]->tcp, params[i], prep_total);
    prep_total += prep_jobs[i].nh + prep_jobs[i].nl;
  }
  // work list: about eight items per CTA, cost-ordered, largest first (CTAs take
  // them from a shared counter, so the smaller ones fill the tail)
  const long long target = std::max<long long>(1, (total_tiles + 8LL * b->grid - 1) / (8LL * b->grid));
  std::vector<TcInst> insts(n);
  std::vector<std::pair<double, int>> cost;
  std::vector<int> inst_of;
  int base = 0;
  for (int i = 0; i < n; ++i) {
    jet_plan_s* p = plans[i];
    TcPlan* t = p->tcp;
    TcInst& I = insts[i];
    fill_tc(p, t, params[i], X[i], N[i], source ? source[i] : nullptr, nullptr, I);
    const long long chunks = std::min<long long>(b->max_chunks, std::max<long long>(1, (I.n_tiles + target - 1) / target));
    I.tiles_per_chunk = (int)((I.n_tiles + chunks - 1) / chunks);
    I.n_chunks = (int)((I.n_tiles + I.tiles_per_chunk - 1) / I.tiles_per_chunk);
    I.chunk_base = base;
    I.grad_slices = b->grad_slices + b->slice_off[i];
    I.loss_slices = b->loss_slices + (long long)i * b->max_chunks;
    I.scratch = b->scratch;
    I.scratch_stride = b->scratch_stride;
    I.slice_shared = 0;  // batches keep one deterministic slice per chunk
    I.wstore = nullptr;  // and flush weight gradients per tile
    double per_tile = (double)(p->L - 1) * t->w * t->w * t->cols_pad + 2000.0 * t->w * t->P * (p->L - 1);
    for (int c = 0; c < I.n_chunks; ++c) {
      const long long t0 = (long long)c * I.tiles_per_chunk;
      const long long nt = std::min<long long>(I.n_tiles, t0 + I.tiles_per_chunk) - t0;
      cost.push_back({per_tile * (double)nt, base + c});
      inst_of.push_back(i);
    }
    base += I.n_chunks;
  }
  std::stable_sort(cost.begin(), cost.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first > y.first;
  });
  const bool capturing = [&] {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    return cs != cudaStreamCaptureStatusNone;
  }();
  // upload the descriptors only when they changed; wait for the previous
  // upload to have read the staging buffers before rewriting them
  bool same = b->have_prev && b->n_items == base && memcmp(b->h_insts, insts.data(), sizeof(TcInst) * n) == 0 &&
              memcmp(b->h_prep, prep_jobs.data(), sizeof(PrepJob) * n) == 0;
  if (same)
    for (int k = 0; k < base && same; ++k) same = b->h_items[k] == cost[k].second && b->h_items[base + k] == inst_of[k];
  if (!same) {
    if (b->have_prev && !capturing) cudaEventSynchronize(b->copied);
    memcpy(b->h_insts, insts.data(), sizeof(TcInst) * n);
    memcpy(b->h_prep, prep_jobs.data(), sizeof(PrepJob) * n);
    for (int k = 0; k < base; ++k) {
      b->h_items[k] = cost[k].second;
      b->h_items[base + k] = inst_of[k];
    }
    b->n_items = base;
    cudaError_t e = cudaMemcpyAsync(b->d_insts, b->h_insts, sizeof(TcInst) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_items, b->h_items, sizeof(int) * 2 * base, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_prep, b->h_prep, sizeof(PrepJob) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !capturing) e = cudaEventRecord(b->copied, s);
    if (e != cudaSuccess) return tcuda(e, "batch descriptor upload");
    b->have_prev = b->have_prev || !capturing;
  }
  {
    const int pgrid = (int)std::min<long long>((prep_total + 255) / 256, 2048);
    tc_prep_batch_kernel<<<pgrid, 256, 0, s>>>(b->d_prep, n, prep_total);
    cudaError_t pe = cudaGetLastError();
    if (pe != cudaSuccess) return tcuda(pe, "batched weight preparation");
  }
  TcArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < 4; ++k) {  // the members' common tile shape (0 where they differ)
    auto field = [&](const TcInst& I) { return k == 0 ? I.Pc : k == 1 ? I.G : k == 2 ? I.H : I.w; };
    a.shape[k] = field(insts[0]);
    for (int i = 1; i < n; ++i)
      if (field(insts[i]) != a.shape[k]) a.shape[k] = 0;
  }
  a.mode = MODE_FWD_BWD;
  a.n_items = base;
  a.insts = b->d_insts;
  a.item_inst = b->d_items;
  a.item_next = b->d_next;
  a.err = b->err;
  a.tmem_cols = b->tmem_cols;
  a.nthreads = b->nthreads;
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(int), s);
  if (e != cudaSuccess) return tcuda(e, "batch item counter reset");
  e = tc_launch(b->cls, a, std::min(b->grid, base), b->smem, s);
  if (e != cudaSuccess) return tcuda(e, "batched tc kernel launch");
  long long maxp = 0;
  bool jobs_same = !capturing;
  for (int i = 0; i < n; ++i) {
    ReduceJob j;
    memset(&j, 0, sizeof(j));
    j.grad_slices = insts[i].grad_slices;
    j.loss_slices = insts[i].loss_slices;
    j.n_chunks = insts[i].n_chunks;
    j.n_params = plans[i]->n_params;
    j.inv_N = insts[i].inv_N;
    j.grad_out = adam ? nullptr : grad_out[i];
    j.loss_out = loss_out ? loss_out + i : nullptr;
    if (adam) {
      j.params = const_cast<void*>(params[i]);
      j.m = m[i];
      j.v = v[i];
    }
    if (jobs_same && memcmp(&b->h_jobs[i], &j, sizeof(j)) != 0) {
      jobs_same = false;
      if (b->have_prev && !capturing) cudaEventSynchronize(b->copied);
    }
    if (!jobs_same || capturing) b->h_jobs[i] = j;
    maxp = std::max(maxp, j.n_params);
  }
  if (!jobs_same || capturing) {
    e = cudaMemcpyAsync(b->d_jobs, b->h_jobs, sizeof(ReduceJob) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !capturing) e = cudaEventRecord(b->copied, s);
    if (e != cudaSuccess) return tcuda(e, "batch job upload");
  }
  e = launch_reduce(b->d_jobs, b->h_jobs[0], n, maxp, false, adam, step, lr, s, step_ctr);
  return e == cudaSuccess ? JET_OK : tcuda(e, "batch reduce");
}

// ------------------------------------------------------------------ failure-detection hook
namespace {
__global__ void wait_timeout_kernel(unsigned long long budget_ns, int* err) {
  __shared__ uint64_t bar;
  __shared__ volatile int abort_s;
  if (threadIdx.x == 0) {
    abort_s = 0;
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  // nothing arrives at the barrier: the bounded wait must give up
  const bool ok = tc::mbar_wait(&bar, 0u, &abort_s, err, 90, budget_ns);
  if (ok && threadIdx.x == 0) atomicExch(err, -1);  // a wait that "completed" is a failure of the hook
}
}  // namespace

extern "C" jet_status jet_debug_wait_timeout(int64_t budget_ns) {
  if (budget_ns < 1000 || budget_ns > 1000000000) return tfail(JET_ERR_INVALID, "budget_ns must be in [1e3, 1e9]");
  int* d_err = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(int));
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32>>>((unsigned long long)budget_ns, d_err);
    e = cudaGetLastError();
  }
  int h = 0;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d_err);
  if (e != cudaSuccess) return tcuda(e, "wait-timeout hook");
  if (h == 90) return tfail(JET_ERR_TIMEOUT, "bounded device wait gave up after its budget (as intended)");
  return tfail(JET_ERR_CUDA, "bounded wait did not report a time-out");
}
