// Fused tensor-core partial-jet kernel (BF16 operands, FP32 accumulation in
// TMEM), one persistent launch over (instance, chunk of point tiles) items.
//
// Hidden widths 32 and 64 are packed: G = 128 / width sub-tiles of the tile's
// points share the 128 MMA rows (operand row = sub-tile * width + unit) with
// block-diagonal BF16 weights, so that every TMEM lane quadrant holds units.
//
// Per tile of P collocation points the CTA keeps the jets of one layer in
// shared memory as a [unit][column] bf16 matrix in the 128-byte-swizzled
// layout of tc_ptx.cuh, columns = (channel block, point): the channels of the
// highest derivative order come first, so that the split-precision products
// of JET_BF16X3 cover one leading column range.  For every hidden layer:
//
//   forward  TMA loads W^l (bf16) into shared memory; one thread issues
//            tcgen05.mma  Z^l[unit][col] = W^l A^{l-1}  (M = 128 units per
//            half, N = all columns, K = 16 per instruction) into TMEM; the
//            four epilogue warps read their TMEM lanes (one unit per thread,
//            all channels of a point in that thread's registers), add the bias
//            on the value channel, compose the tanh jet in closed form
//            (Eq. 2-3 recursion) and write A^l back as the next B operand;
//   output   one more MMA with the output weights (rows >= n_out zero),
//            residual monomials and the FP64 loss partial;
//   backward residual adjoint, output-layer gradients, then per layer:
//            z^l (kept in TMEM for the last layer, recomputed by MMA from the
//            stored A^{l-1} for the others), activation-jet adjoint in the
//            epilogue (Zbar^l to shared memory), data gradient
//            Abar^{l-1} = W^l^T Zbar^l (MN-major A) and weight gradient
//            Wbar^l = Zbar^l A^{l-1}^T (both operands K-major) by MMA; the
//            weight gradient is added from TMEM into the CTA's FP32
//            accumulator, which reaches the chunk's FP64 slice once per chunk.
//
// The layer inputs A^l of a tile are saved to a per-CTA global scratch slot by
// bulk copies during the forward and read back during the backward, so memory
// is bounded by the number of CTAs.  Every mbarrier wait is bounded: on time-
// out the kernel records an error code, stops issuing work, waits (bounded) for
// its own MMAs, releases TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "jet_closures_gen.h"
#include "jet_internal.h"
#include "jet_simt.cuh"
#include "tc_ptx.cuh"

namespace jet {

// A CTA has 2 or 4 warpgroups (TcArgs::nthreads = 256 or 512); each
// warpgroup covers the four TMEM lane quadrants and a share of the points.
constexpr int kTcThreads = 512;  // largest CTA
constexpr int kTcWG = 4;         // largest warpgroup count

// p[k] = tanh^(k)(z) for the tensor-core epilogue.  q = 1 - tanh|z| =
// 2 / (exp(2|z|) + 1) is formed with the approximate exp2 and reciprocal
// units; tanh z = sign(z) (1 - q) and s = 1 - tanh^2 z = q (2 - q), which keeps
// s accurate in relative terms where |z| is large (no 1 - a^2 cancellation).
template <int NP>
__device__ __forceinline__ void tanh_derivs_fast(float z, float* p) {
  const float az = fabsf(z);
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(az * 2.8853900817779268f));  // exp(2|z|)
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
  const float q = 2.0f * r;
  const float a = copysignf(1.0f - q, z);
  const float s = q * (2.0f - q);
  const float a2 = a * a;
  p[0] = a;
  if (NP > 1) p[1] = s;
  if (NP > 2) p[2] = -2.0f * a * s;
  if (NP > 3) p[3] = s * (6.0f * a2 - 2.0f);
  if (NP > 4) p[4] = 8.0f * a * s * (2.0f - 3.0f * a2);
  if (NP > 5) p[5] = 8.0f * s * (15.0f * a2 * a2 - 15.0f * a2 + 2.0f);
}

// tanh_derivs_fast for two points at once (the exponential and reciprocal
// per point, the polynomials in a and s packed)
template <int NP>
__device__ __forceinline__ void tanh_derivs_fast2(f2 z, f2* p) {
  float e0, e1, r0, r1;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(fabsf(z.v.x) * 2.8853900817779268f));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(fabsf(z.v.y) * 2.8853900817779268f));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(1.0f + e0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(1.0f + e1));
  const f2 q(2.0f * r0, 2.0f * r1);
  const f2 a(copysignf(1.0f - q.v.x, z.v.x), copysignf(1.0f - q.v.y, z.v.y));
  const f2 s = q * jfma(q, f2(-1.0f), f2(2.0f));
  const f2 a2 = a * a;
  p[0] = a;
  if (NP > 1) p[1] = s;
  if (NP > 2) p[2] = f2(-2.0f) * a * s;
  if (NP > 3) p[3] = s * jfma(f2(6.0f), a2, f2(-2.0f));
  if (NP > 4) p[4] = f2(8.0f) * a * s * jfma(f2(-3.0f), a2, f2(2.0f));
  if (NP > 5) p[5] = f2(8.0f) * s * jfma(a2, jfma(f2(15.0f), a2, f2(-15.0f)), f2(2.0f));
}

struct alignas(64) TcInst {
  CUtensorMap wmap;    // hidden weights bf16 [L-2][w][w]: dims (in, out, layer), box (64, R_W, 1)
  CUtensorMap wlmap;   // output weights bf16 [128][w] (rows repeated per lane quadrant): box (64, 128)
  CUtensorMap wlomap;  // low parts of the hidden weights (JET_BF16X3), like wmap
  int L, d, n_out, n_res, w, H, P, cols, cols_pad, top_cols, split3;
  // packing: operand row r holds unit r % wu of sub-tile r / wu; G = w / wu
  // sub-tiles of Pc points each (P = G * Pc); w is the width the MMAs see
  int wu, G, Pc;
  int n_terms;
  DevTerm terms[kMaxTerms];
  int n_groups;  // composite loss (0: one residual over all points)
  DevGroup groups[kMaxGroups];
  // residual adjoint lists: for output-jet slot k (o * C + channel), the
  // factors (monomial m, factor f) that read it, packed m * 4 + f, in (m, f)
  // order at adj_mf[adj_off[k] .. adj_off[k + 1]); monomial coefficients in FP32
  short adj_off[kMaxOut * kMaxC + 1];
  unsigned char adj_mf[kMaxTerms * 4];
  float coef_f[kMaxTerms];
  const float* params;
  long long off_W[kMaxLayers], off_b[kMaxLayers];
  long long n_params;
  const float* X;
  const float* source;
  float* r_out;
  long long N;
  double inv_N;
  long long n_tiles;
  int tiles_per_chunk, n_chunks, chunk_base;
  double* grad_slices;
  double* loss_slices;
  unsigned char* scratch;
  long long scratch_stride;  // bytes per CTA slot
  // FP32 weight-gradient accumulator of the running chunk, at this byte
  // offset in the CTA's scratch slot (-1: none; such plans never run the
  // weight gradient per tile)
  long long wacc_off;
  // shared-memory carve (bytes from the 1024-aligned base)
  int o_w, o_wlo, o_a0, o_a1, o_alo0, o_alo1, o_uo, o_ub, o_xs, o_red;
  int o_part;  // per-warpgroup partial sums, float [warpgroups][4][256]
  int act_bytes, alo_bytes;
  int r0w, r1w;  // TMEM column widths of regions R0 and R1 per half
  int slice_shared;  // 1: all chunks add into grad_slices[0 .. n_params)
  // store mode: per tile, the layer inputs A^1..A^{L-2} (and their split low
  // parts) and the adjoints Zbar^2..Zbar^{L-1} go to HBM for the separate
  // weight-gradient GEMM; null = per-tile weight-gradient MMA and flush
  unsigned char* wstore;
  long long wstore_tile_stride;  // bytes per tile
};

struct TcArgs {
  TcInst inst0;
  // tile shape shared by every work item of the launch (points per sub-tile,
  // packed sub-tiles, 128-row halves, MMA width), 0 where they differ: selects
  // a fixed-shape kernel when one is compiled
  int shape[4];
  int mode;
  int n_items;
  const TcInst* insts;
  const int* item_inst;
  int* err;
  int tmem_cols;
  int nthreads;  // launch block size: 256 or 512
  // batches: counter of the items taken after each CTA's first (zeroed before
  // the launch); a CTA that finishes an item takes the next in the
  // cost-ordered list, so the work balances itself.  Null: a fixed stride.
  int* item_next;
};

// Tile shape of a launch: points per sub-tile PC, packed sub-tiles G, 128-row
// halves H, MMA width W and CTA threads NT as compile-time constants, or 0 for
// the runtime values of the work item's descriptor and launch (a batch of
// members with different packings fixes PC, H, W and NT and leaves G).  Fixed shapes let the compiler fold
// the TMEM column and swizzled shared-memory offsets of every epilogue access.
template <int PC_, int G_, int H_, int W_, int NT_>
struct TcShape {
  static constexpr int PC = PC_, G = G_, H = H_, W = W_, NT = NT_;
};
using TcShapeAny = TcShape<0, 0, 0, 0, 0>;

template <class Cls, class Shape = TcShapeAny>
struct TcTile {
  static constexpr int C = Cls::C;
  static constexpr int NP = Cls::NP;
  static constexpr int TOP = Cls::TOP_BEGIN;
  // points per epilogue pass: four below seven channels (forward) or five
  // (adjoint); four where a compiled shape gives every warpgroup whole
  // passes of four (the adjoint only up to seven channels, where its three
  // arrays of jets still fit the registers); two otherwise, so that small
  // tiles keep every warpgroup busy
  static constexpr bool BAL4 = Shape::PC != 0 && Shape::NT != 0 && Shape::PC % (Shape::NT / 128 * 4) == 0;
  static constexpr int PPF = (C < 7 || BAL4) ? 4 : 2;
  static constexpr int PPB = (C < 5 || (C <= 7 && BAL4)) ? 4 : 2;

  // the tile shape: compile-time when the launch fixes it, else the descriptor's
  __device__ __forceinline__ int pc() const { return Shape::PC ? Shape::PC : I.Pc; }
  __device__ __forceinline__ int gg() const { return Shape::G ? Shape::G : I.G; }
  __device__ __forceinline__ int hh() const { return Shape::H ? Shape::H : I.H; }
  __device__ __forceinline__ int ww() const { return Shape::W ? Shape::W : I.w; }
  __device__ __forceinline__ int wuu() const { return Shape::W && Shape::G ? Shape::W / Shape::G : I.wu; }
  __device__ __forceinline__ int pp() const { return pc() * gg(); }
  __device__ __forceinline__ int rr() const { return Shape::H ? 128 * Shape::H : R_; }  // rows of every operand buffer
  __device__ __forceinline__ int cpad() const { return Shape::PC ? (C * Shape::PC + 15) / 16 * 16 : I.cols_pad; }
  __device__ __forceinline__ int ctop() const { return Shape::PC ? (C - TOP) * Shape::PC : I.top_cols; }
  __device__ __forceinline__ int nth() const { return Shape::NT ? Shape::NT : nthr; }   // threads of the CTA
  __device__ __forceinline__ int nw() const { return Shape::NT ? Shape::NT / 128 : nwg; }  // warpgroups

  const TcInst& I;      // the work item's descriptor, copied to shared memory
  const TcInst* Imap;   // the same descriptor in param or global space: its tensor maps serve TMA
  unsigned char* sm;
  uint64_t* bar_tma;
  uint64_t* bar_mma;
  uint64_t* bar_ld;
  uint64_t* bar_wg;  // the weight-gradient MMA of a backward layer (per-tile schedule)
  volatile int* abort_f;
  int* err;
  uint32_t tmem;
  uint32_t ph_tma, ph_mma, ph_ld, ph_wg;
  int tid, warp;
  int R_;       // rows of every operand buffer (128 * H), for a runtime shape
  float* part;  // per-warpgroup partial sums [nwg][4][256]
  int q, wg, ul;  // TMEM lane quadrant, warpgroup, unit within a 128-row half
  int nwg, nthr;  // warpgroups and threads of the CTA
  // descriptor fields of the epilogues' hot accesses, read once per tile: the
  // shared addresses of the operand buffers and the TMEM region widths
  uint32_t act_s0 = tc::smem_u32(sm + I.o_a0), act_s1 = tc::smem_u32(sm + I.o_a1);
  uint32_t alo_s0 = tc::smem_u32(sm + I.o_alo0), alo_s1 = tc::smem_u32(sm + I.o_alo1);
  uint32_t r0w_ = (uint32_t)I.r0w, r1w_ = (uint32_t)I.r1w;
  __device__ __forceinline__ uint32_t act_s(int i) const { return i ? act_s1 : act_s0; }
  __device__ __forceinline__ uint32_t alo_s(int i) const { return i ? alo_s1 : alo_s0; }

  // column block of channel c: highest-order channels first
  static __device__ __forceinline__ int blk(int c) { return c >= TOP ? c - TOP : c + (C - TOP); }

  __device__ float* UO() const { return reinterpret_cast<float*>(sm + I.o_uo); }
  __device__ float* UB() const { return reinterpret_cast<float*>(sm + I.o_ub); }
  __device__ float* XS() const { return reinterpret_cast<float*>(sm + I.o_xs); }
  __device__ unsigned char* ACT(int i) const { return sm + (i ? I.o_a1 : I.o_a0); }
  __device__ unsigned char* ALO(int i) const { return sm + (i ? I.o_alo1 : I.o_alo0); }
  __device__ uint32_t R0(int h) const { return tmem + (uint32_t)h * r0w_; }
  __device__ uint32_t R1(int h) const { return tmem + (uint32_t)hh() * r0w_ + (uint32_t)h * r1w_; }
  __device__ uint32_t lane_base() const { return (uint32_t)(q * 32) << 16; }
  __device__ float& PART(int w, int k, int u) const { return part[(w * 4 + k) * 256 + u]; }

  __device__ bool wait(uint64_t* bar, uint32_t& ph, int code) {
    const bool ok = tc::mbar_wait(bar, ph & 1u, abort_f, err, code);
    ++ph;
    return ok;
  }

  __device__ void sync() {
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
  }

  // ------------------------------------------------------------ loads (thread 0)
  __device__ void load_hidden_w(int l) {  // W^l, l = 2..L-1 -> W buffer (and W_lo)
    const int nck = ww() / 64 > 2 ? ww() / 64 : 2;
    const uint32_t box = 64u * rr() * 2u;
    tc::mbar_arrive_expect_tx(bar_tma, box * nck * (I.split3 ? 2u : 1u));
    for (int kc = 0; kc < nck; ++kc) {
      tc::tma_load_3d(sm + I.o_w + kc * box, &Imap->wmap, bar_tma, kc * 64, 0, l - 2);
      if (I.split3) tc::tma_load_3d(sm + I.o_wlo + kc * box, &Imap->wlomap, bar_tma, kc * 64, 0, l - 2);
    }
  }

  __device__ void load_out_w() {  // W^L -> W buffer, 128-row boxes
    const int nck = (ww() + 63) / 64;
    const uint32_t box = 64u * 128u * 2u;
    tc::mbar_arrive_expect_tx(bar_tma, box * nck);
    for (int kc = 0; kc < nck; ++kc) tc::tma_load_2d(sm + I.o_w + kc * box, &Imap->wlmap, bar_tma, kc * 64, 0);
  }

  long long cur_tile = 0;

  // copy of A^l (l = 1..L-3; with the store also L-2): per-CTA scratch slot,
  // or the tile's place in the store
  __device__ unsigned char* slot(int l) const {
    const long long off = (long long)(l - 1) * (I.act_bytes + I.alo_bytes);
    if (I.wstore) return I.wstore + cur_tile * I.wstore_tile_stride + off;
    return I.scratch + (long long)blockIdx.x * I.scratch_stride + off;
  }
  // layer-input copies: the per-CTA scratch slot is rewritten every tile and
  // stays in L2 (evict_last); the store streams through it (default policy)
  __device__ void scratch_out(unsigned char* dst, const unsigned char* src, uint32_t bytes) const {
    if (I.wstore) tc::bulk_s2g(dst, src, bytes);
    else tc::bulk_s2g_hint(dst, src, bytes, tc::policy_evict_last());
  }
  __device__ void scratch_in(unsigned char* dst, const unsigned char* src, uint32_t bytes) const {
    if (I.wstore) tc::bulk_g2s(dst, src, bytes, bar_ld);
    else tc::bulk_g2s_hint(dst, src, bytes, bar_ld, tc::policy_evict_last());
  }

  // adjoint Zbar^l (l = 2..L-1) of the tile in the store
  __device__ unsigned char* zslot(int l) const {
    return I.wstore + cur_tile * I.wstore_tile_stride + (long long)(I.L - 2) * (I.act_bytes + I.alo_bytes) +
           (long long)(l - 2) * I.act_bytes;
  }

  // ------------------------------------------------------------ MMAs (thread 0)
  // D[R0] = W^l (K-major) x B (MN-major rows = units), plus the split terms
  __device__ void mma_layer(int bi) {
    const uint32_t sW = tc::smem_u32(sm + I.o_w), sWlo = tc::smem_u32(sm + I.o_wlo);
    const uint32_t sB = tc::smem_u32(ACT(bi)), sBlo = tc::smem_u32(ALO(bi));
    const uint32_t chunkW = (uint32_t)(rr() / 8) * 1024u, chunkA = chunkW;
    const uint32_t id = tc::idesc_bf16(128, cpad(), 0, 1);
    const uint32_t id_top = tc::idesc_bf16(128, ctop(), 0, 1);
    const int ks = ww() / 16;
    for (int h = 0; h < hh(); ++h) {
      for (int s = 0; s < ks; ++s) {
        const uint32_t aoff = (uint32_t)(s / 4) * chunkW + (uint32_t)h * 16384u + (uint32_t)(s % 4) * 32u;
        const uint64_t ad = tc::sdesc(sW + aoff, 16, 1024);
        const uint64_t bd = tc::sdesc(sB + (uint32_t)s * 2048u, chunkA, 1024);
        tc::mma_f16(R0(h), ad, bd, id, s > 0);
      }
      if (I.split3) {
        for (int s = 0; s < ks; ++s) {
          const uint32_t aoff = (uint32_t)(s / 4) * chunkW + (uint32_t)h * 16384u + (uint32_t)(s % 4) * 32u;
          tc::mma_f16(R0(h), tc::sdesc(sWlo + aoff, 16, 1024), tc::sdesc(sB + (uint32_t)s * 2048u, chunkA, 1024),
                      id_top, 1);
          tc::mma_f16(R0(h), tc::sdesc(sW + aoff, 16, 1024), tc::sdesc(sBlo + (uint32_t)s * 2048u, chunkA, 1024),
                      id_top, 1);
        }
      }
    }
  }

  __device__ void mma_out(int bi) {  // D[R1(0)] = W^L (rows >= n_out zero) x A^{L-1}
    const uint32_t sW = tc::smem_u32(sm + I.o_w), sB = tc::smem_u32(ACT(bi));
    const uint32_t chunkA = (uint32_t)(rr() / 8) * 1024u;
    const uint32_t id = tc::idesc_bf16(128, cpad(), 0, 1);
    for (int s = 0; s < ww() / 16; ++s) {
      const uint64_t ad = tc::sdesc(sW + (uint32_t)(s / 4) * 16384u + (uint32_t)(s % 4) * 32u, 16, 1024);
      const uint64_t bd = tc::sdesc(sB + (uint32_t)s * 2048u, chunkA, 1024);
      tc::mma_f16(R1(0), ad, bd, id, s > 0);
    }
  }

  // D[R1] = W^l^T (MN-major A) x Zbar (MN-major B)
  __device__ void mma_dgrad(int zi) {
    const uint32_t sW = tc::smem_u32(sm + I.o_w), sZ = tc::smem_u32(ACT(zi));
    const uint32_t chunk = (uint32_t)(rr() / 8) * 1024u;
    const uint32_t id = tc::idesc_bf16(128, cpad(), 1, 1);
    for (int h = 0; h < hh(); ++h)
      for (int s = 0; s < ww() / 16; ++s) {
        const uint64_t ad = tc::sdesc(sW + (uint32_t)(2 * h) * chunk + (uint32_t)s * 2048u, chunk, 1024);
        const uint64_t bd = tc::sdesc(sZ + (uint32_t)s * 2048u, chunk, 1024);
        tc::mma_f16(R1(h), ad, bd, id, s > 0);
      }
  }

  // D[R0] = Zbar (K-major, M = out units) x A^{l-1} (K-major, N block nb of in units)
  __device__ void mma_wgrad(int zi, int ai, int nb, int NB) {
    const uint32_t sZ = tc::smem_u32(ACT(zi)), sA = tc::smem_u32(ACT(ai));
    const uint32_t chunk = (uint32_t)(rr() / 8) * 1024u;
    const uint32_t id = tc::idesc_bf16(128, NB, 0, 0);
    for (int h = 0; h < hh(); ++h)
      for (int s = 0; s < cpad() / 16; ++s) {
        const uint32_t koff = (uint32_t)(s / 4) * chunk + (uint32_t)(s % 4) * 32u;
        const uint64_t ad = tc::sdesc(sZ + koff + (uint32_t)h * 16384u, 16, 1024);
        const uint64_t bd = tc::sdesc(sA + koff + (uint32_t)(nb * NB / 8) * 1024u, 16, 1024);
        tc::mma_f16(R0(h), ad, bd, id, s > 0);
      }
  }

  // ------------------------------------------------------------ epilogue helpers
  // PP values of one operand row (consecutive columns) as BF16; buf is the
  // buffer's shared address
  template <int PP>
  __device__ void st_bf16(uint32_t buf, int row, int col, const float* v) const {
    const uint32_t p = buf + tc::swz_off(row, col & ~7, rr()) + (uint32_t)(col & 7) * 2u;
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    if (PP == 4) {
      __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
      tc::sts_v2_b32(p, *reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
    } else {
      tc::sts_b32(p, *reinterpret_cast<uint32_t*>(&a));
    }
  }

  template <int PP>
  __device__ void st_lo(uint32_t buf, int row, int col, const float* v) const {
    float lo[PP];
#pragma unroll
    for (int j = 0; j < PP; ++j) lo[j] = v[j] - __bfloat162float(__float2bfloat16_rn(v[j]));
    st_bf16<PP>(buf, row, col, lo);
  }

  // ------------------------------------------------------------ per-row parameters
  // Parameters of this thread's operand rows (one per 128-row half), loaded
  // ahead of the wait or barrier that precedes their epilogue, so that the
  // global loads' latency hides behind it.  Which ones pay was measured per
  // shape class: the biases and the first layer's weights of the forward for
  // 128-wide and packed shapes, the first layer's weights of the backward for
  // 256-wide shapes (whose registers are tighter: two row halves).
  static constexpr bool PRELOAD = Shape::H != 2;    // biases
  static constexpr bool PRELOAD1 = Shape::H != 2;   // W^1, b^1 of the layer-1 forward
  static constexpr bool PRELOAD1B = Shape::H == 2;  // W^1, b^1 of the layer-1 backward
  struct RowBias {
    float v[2];
  };
  __device__ RowBias row_bias(int l) const {  // b^l
    RowBias b{};
    if (!PRELOAD) return b;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h * 128 + ul;
      b.v[h] = (h < hh() && r < ww()) ? I.params[I.off_b[l - 1] + r % wuu()] : 0.f;
    }
    return b;
  }
  struct Row1 {  // W^1 and b^1
    float w[2][Cls::D];
    float b[2];
  };
  __device__ Row1 row_l1(bool on) const {
    Row1 w{};
    if (!on) return w;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h * 128 + ul;
      const bool ok = h < hh() && r < ww();
      const int u = r % wuu();
#pragma unroll
      for (int i = 0; i < Cls::D; ++i) w.w[h][i] = ok ? I.params[I.off_W[0] + u * Cls::D + i] : 0.f;
      w.b[h] = ok ? I.params[I.off_b[0] + u] : 0.f;
    }
    return w;
  }

  // ------------------------------------------------------------ forward pieces
  __device__ void layer1_fwd(int out_buf, const Row1& w1p) {
    const int Pc = pc();
    const bool split3 = I.split3;
    constexpr int d = Cls::D;  // the plan's input dimension
    for (int h = 0; h < hh(); ++h) {
      const int r = h * 128 + ul;  // operand row
      if (r >= ww()) continue;
      const int sub = r / wuu(), u = r - sub * wuu();
      float w1[d];
#pragma unroll
      for (int i = 0; i < d; ++i) w1[i] = PRELOAD1 ? w1p.w[h][i] : I.params[I.off_W[0] + u * d + i];
      const float b1 = PRELOAD1 ? w1p.b[h] : I.params[I.off_b[0] + u];
      const float* xs = XS() + sub * Pc * d;
      // the warpgroups split the points; a fixed shape makes the pass count a
      // compile-time constant, so the passes unroll with constant offsets
#pragma unroll
      for (int k = 0; k < (Pc + nw() * PPF - 1) / (nw() * PPF); ++k) {
        const int g = wg * PPF + k * nw() * PPF;
        if (g >= Pc) break;
        float av[C][PPF];
#pragma unroll
        for (int j = 0; j < PPF; j += 2) {
          f2 z[C], p[NP], a[C];
#pragma unroll
          for (int c = 0; c < C; ++c) z[c] = f2(0.f);
          float v0 = b1, v1 = b1;
#pragma unroll
          for (int i = 0; i < d; ++i) {
            v0 = fmaf(w1[i], xs[(g + j) * d + i], v0);
            v1 = fmaf(w1[i], xs[(g + j + 1) * d + i], v1);
          }
          z[0] = f2(v0, v1);
#pragma unroll
          for (int i = 0; i < Cls::D; ++i) {
            const int fo = Cls::first_order(i);
            if (fo >= 0) z[fo] = f2(w1[i]);
          }
          tanh_derivs_fast2<NP>(z[0], p);
          Cls::compose(z, p, a);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            av[c][j] = a[c].v.x;
            av[c][j + 1] = a[c].v.y;
          }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          st_bf16<PPF>(act_s(out_buf), r, blk(c) * Pc + g, av[c]);
          if (split3 && c >= TOP) st_lo<PPF>(alo_s(out_buf), r, blk(c) * Pc + g, av[c]);
        }
      }
    }
  }

  // a^l = compose(D[R0] + b^l) -> ACT(out_buf)
  __device__ void hidden_epilogue(int l, int out_buf, const RowBias& bias) {
    const int Pc = pc();
    const bool split3 = I.split3;
    for (int h = 0; h < hh(); ++h) {
      const int r = h * 128 + ul;
      if (h * 128 + q * 32 >= ww()) continue;  // warp-uniform
      const float bu = PRELOAD ? bias.v[h] : I.params[I.off_b[l - 1] + r % wuu()];
      // the warpgroups split the points; a fixed shape makes the pass count a
      // compile-time constant, so the passes unroll with constant offsets
#pragma unroll
      for (int k = 0; k < (Pc + nw() * PPF - 1) / (nw() * PPF); ++k) {
        const int g = wg * PPF + k * nw() * PPF;
        if (g >= Pc) break;
        float zv[C][PPF];
#pragma unroll
        for (int c = 0; c < C; ++c) tc::tmem_ld<PPF>(R0(h) + lane_base() + (uint32_t)(blk(c) * Pc + g), zv[c]);
        tc::tmem_wait_ld();
        float av[C][PPF];
#pragma unroll
        for (int j = 0; j < PPF; j += 2) {
          f2 z[C], p[NP], a[C];
#pragma unroll
          for (int c = 0; c < C; ++c) z[c] = f2(zv[c][j], zv[c][j + 1]);
          z[0] = z[0] + f2(bu);
          tanh_derivs_fast2<NP>(z[0], p);
          Cls::compose(z, p, a);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            av[c][j] = a[c].v.x;
            av[c][j + 1] = a[c].v.y;
          }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
          st_bf16<PPF>(act_s(out_buf), r, blk(c) * Pc + g, av[c]);
          if (split3 && c >= TOP) st_lo<PPF>(alo_s(out_buf), r, blk(c) * Pc + g, av[c]);
        }
      }
    }
  }

  // UO[o*C + c][s*Pc + n] = D[R1(0)][row s*n_out + o] (+ b^L on the value
  // channel).  The output weights repeat in every 32-row lane quadrant, so
  // the rows sit in lanes 0..G*n_out-1 of every quadrant: each warp reads its
  // own quadrant, and all warps split the column groups.
  __device__ void out_epilogue() {
    float* uo = UO();
    const int Pc = pc(), ng = Pc / 8, nrow = gg() * I.n_out, lane = tid & 31;
    for (int k = wg * 4 + q; k < C * ng; k += nw() * 4) {
      const int c = k / ng, g = (k - c * ng) * 8;
      float v[8];
      tc::tmem_ld8(R1(0) + lane_base() + (uint32_t)(blk(c) * Pc + g), v);
      tc::tmem_wait_ld();
      if (lane < nrow) {
        const int sub = lane / I.n_out, o = lane - sub * I.n_out;
        const float b = c == 0 ? I.params[I.off_b[I.L - 1] + o] : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) uo[(o * C + c) * pp() + sub * Pc + g + j] = v[j] + b;
      }
    }
  }

  // Residual r_c = sum of the monomials - source, the loss partial and (bwd)
  // ub = dL/du.  Three parallel passes over (point, monomial) products, per
  // point sums and per (point, output channel) adjoints, which keep every
  // sum's operands and order those of a per-point loop over the monomials;
  // the products and scaled residuals live in the partial-sum area (free
  // here).  Spec-sized work that does not fit takes the per-point loop.
  __device__ double residual(long long n0, int nvalid, bool bwd) {
    float* uo = UO();
    float* ub = UB();
    const int P = pp(), nt = I.n_terms, nslot = I.n_out * C;
    const float two_over_n = (float)(2.0 * I.inv_N);
    double loss = 0.0;
    if (I.n_groups > 0) {  // composite loss: every term over its own points
      if (bwd)
        for (int i = tid; i < nslot * P; i += nth()) ub[i] = 0.f;
      __syncthreads();
      return grouped_residual<float>(I.terms, I.groups, I.n_groups, I.n_res, uo, ub, P, n0, nvalid, I.source,
                                     I.r_out, bwd, tid, nth());
    }
    if ((nt + I.n_res) * P > nw() * 4 * 256) {
      if (bwd)
        for (int i = tid; i < nslot * P; i += nth()) ub[i] = 0.f;
      __syncthreads();
      for (int n = tid; n < nvalid; n += nth()) {
        float r[kMaxRes];
        for (int c = 0; c < I.n_res; ++c) r[c] = I.source ? -I.source[(n0 + n) * I.n_res + c] : 0.f;
        for (int m = 0; m < nt; ++m) {
          const DevTerm& tm = I.terms[m];
          float prod = (float)tm.coef;
          for (int f = 0; f < tm.nfac; ++f) prod *= uo[tm.fac[f] * P + n];
          r[tm.comp] += prod;
        }
        for (int c = 0; c < I.n_res; ++c) {
          if (I.r_out) I.r_out[(n0 + n) * I.n_res + c] = r[c];
          loss += (double)r[c] * (double)r[c];
        }
        if (bwd)
          for (int m = 0; m < nt; ++m) {
            const DevTerm& tm = I.terms[m];
            const float gg = two_over_n * r[tm.comp] * (float)tm.coef;
            for (int f = 0; f < tm.nfac; ++f) {
              float prod = gg;
              for (int q = 0; q < tm.nfac; ++q)
                if (q != f) prod *= uo[tm.fac[q] * P + n];
              ub[tm.fac[f] * P + n] += prod;
            }
          }
      }
      return loss;
    }
    float* prodm = part;            // [n_terms][P] monomial values
    float* rg = part + nt * P;      // [n_res][P] 2 r / N
    for (int i = tid; i < nt * nvalid; i += nth()) {
      const int m = i / nvalid, n = i - m * nvalid;
      const DevTerm& tm = I.terms[m];
      float prod = I.coef_f[m];
      for (int f = 0; f < tm.nfac; ++f) prod *= uo[tm.fac[f] * P + n];
      prodm[m * P + n] = prod;
    }
    __syncthreads();
    for (int n = tid; n < nvalid; n += nth()) {
      const int nres = I.n_res;
      float r[kMaxRes];
#pragma unroll
      for (int c = 0; c < kMaxRes; ++c) r[c] = (c < nres && I.source) ? -ub[n * nres + c] : 0.f;  // source, staged
      for (int m = 0; m < nt; ++m) {
        const int cm = I.terms[m].comp;
        const float v = prodm[m * P + n];
#pragma unroll
        for (int c = 0; c < kMaxRes; ++c)
          if (c == cm) r[c] += v;
      }
#pragma unroll
      for (int c = 0; c < kMaxRes; ++c) {
        if (c >= nres) break;
        if (I.r_out) I.r_out[(n0 + n) * nres + c] = r[c];
        loss += (double)r[c] * (double)r[c];
        rg[c * P + n] = two_over_n * r[c];
      }
    }
    if (!bwd) return loss;
    __syncthreads();
    for (int i = tid; i < nslot * P; i += nth()) {
      const int k = i / P, n = i - k * P;
      float acc = 0.f;
      if (n < nvalid)
        for (int e = I.adj_off[k]; e < I.adj_off[k + 1]; ++e) {  // the factors reading slot k, in (m, f) order
          const int m = I.adj_mf[e] >> 2, f = I.adj_mf[e] & 3;
          const DevTerm& tm = I.terms[m];
          float prod = rg[tm.comp * P + n] * I.coef_f[m];
          for (int q = 0; q < tm.nfac; ++q)
            if (q != f) prod *= uo[tm.fac[q] * P + n];
          acc += prod;
        }
      ub[i] = acc;
    }
    return loss;
  }

  // ------------------------------------------------------------ backward pieces
  // dW^L[o][k] += sum_cols ub[o][col] a^{L-1}[k][col]; db^L[o] += sum_n ub[o][0][n]
  // (warpgroups split the channel blocks; partials go to PART per operand
  // row and are summed in a fixed order, over warpgroups and sub-tiles, by
  // out_grads_flush after a barrier)
  __device__ void out_grads(int a_buf) {
    const float* ub = UB();
    const int P = pp(), Pc = pc();
    for (int h = 0; h < hh(); ++h) {
      const int r = h * 128 + ul;
      if (r >= ww()) continue;
      const int sub = r / wuu();
      const int nout = I.n_out;
      float acc[kMaxOut] = {0.f, 0.f, 0.f, 0.f};
      for (int c = wg; c < C; c += nw())
        for (int q8 = 0; q8 < Pc; q8 += 8) {
          const int col = blk(c) * Pc + q8;
          const uint4 raw = tc::lds_v4_b32(act_s(a_buf) + tc::swz_off(r, col, rr()));
          const __nv_bfloat16* bv = reinterpret_cast<const __nv_bfloat16*>(&raw);
          const float* ubc = ub + c * P + sub * Pc + q8;
#pragma unroll
          for (int o = 0; o < kMaxOut; ++o) {
            if (o >= nout) break;
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[o] = fmaf(__bfloat162float(bv[j]), ubc[o * C * P + j], acc[o]);
          }
        }
#pragma unroll
      for (int o = 0; o < kMaxOut; ++o)
        if (o < nout) PART(wg, o, r) = acc[o];
    }
  }

  // sum of slot k of PART over warpgroups and sub-tiles for true unit u, in
  // FP32 and a fixed order (at most 16 FP32 partials of one tile; the FP64
  // adds across tiles follow)
  __device__ double part_sum(int k, int u) const {
    float s = 0.f;
    for (int sub = 0; sub < gg(); ++sub)
      for (int w2 = 0; w2 < nw(); ++w2) s += PART(w2, k, sub * wuu() + u);
    return (double)s;
  }

  __device__ void out_grads_flush(double* g) {
    const float* ub = UB();
    const int P = pp(), L = I.L;
    if (wg == 0)
      for (int h = 0; h < hh(); ++h) {
        const int k = h * 128 + ul;
        if (k >= wuu()) continue;
        for (int o = 0; o < I.n_out; ++o) tc::red_add_f64(g + I.off_W[L - 1] + (long long)o * wuu() + k, part_sum(o, k));
      }
    if (tid < I.n_out) {
      float s = 0.f;
      for (int n = 0; n < P; ++n) s += ub[(tid * C + 0) * P + n];
      tc::red_add_f64(g + I.off_b[L - 1] + tid, (double)s);
    }
  }

  // slot k of PART summed over warpgroups and sub-tiles -> FP64 slice at dst[u * stride]
  __device__ void part_flush(int k, double* dst, int stride) {
    if (wg != 0) return;
    for (int h = 0; h < hh(); ++h) {
      const int u = h * 128 + ul;
      if (u >= wuu()) continue;
      tc::red_add_f64(dst + (long long)u * stride, part_sum(k, u));
    }
  }

  // Zbar^l = (d compose/dz)^T Abar^l -> ACT(z_buf); db^l += sum_n Zbar_0.
  // Abar^l from TMEM (the data-gradient MMA), or for the last hidden layer
  // from the output-layer adjoint ub (ABAR_FROM_UB): one instantiation each.
  template <bool ABAR_FROM_UB>
  __device__ void adjoint_epilogue(int l, int z_buf, const RowBias& bias) {
    constexpr bool abar_from_ub = ABAR_FROM_UB;
    const float* ub = UB();
    const int P = pp(), Pc = pc();
    for (int h = 0; h < hh(); ++h) {
      const int r = h * 128 + ul;
      if (h * 128 + q * 32 >= ww()) continue;
      const int sub = r / wuu(), u = r - sub * wuu();
      const float bu = PRELOAD ? bias.v[h] : I.params[I.off_b[l - 1] + r % wuu()];
      const int nout = I.n_out;
      float wl[kMaxOut] = {0.f, 0.f, 0.f, 0.f};
      if (abar_from_ub) {
#pragma unroll
        for (int o = 0; o < kMaxOut; ++o)
          if (o < nout) wl[o] = I.params[I.off_W[I.L - 1] + (long long)o * wuu() + u];
      }
      float gb = 0.f;
      // the warpgroups split the points; a fixed shape makes the pass count a
      // compile-time constant, so the passes unroll with constant offsets
#pragma unroll
      for (int k = 0; k < (Pc + nw() * PPB - 1) / (nw() * PPB); ++k) {
        const int g = wg * PPB + k * nw() * PPB;
        if (g >= Pc) break;
        float zv[C][PPB], abv[C][PPB];
#pragma unroll
        for (int c = 0; c < C; ++c) tc::tmem_ld<PPB>(R0(h) + lane_base() + (uint32_t)(blk(c) * Pc + g), zv[c]);
        if (!abar_from_ub) {
#pragma unroll
          for (int c = 0; c < C; ++c) tc::tmem_ld<PPB>(R1(h) + lane_base() + (uint32_t)(blk(c) * Pc + g), abv[c]);
        }
        tc::tmem_wait_ld();
        if (abar_from_ub) {
#pragma unroll
          for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < PPB; ++j) {
              float s = 0.f;
#pragma unroll
              for (int o = 0; o < kMaxOut; ++o)
                if (o < nout) s = fmaf(wl[o], ub[(o * C + c) * P + sub * Pc + g + j], s);
              abv[c][j] = s;
            }
        }
        float zbv[C][PPB];
#pragma unroll
        for (int j = 0; j < PPB; j += 2) {
          f2 z[C], p[NP], ab[C], zb[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            z[c] = f2(zv[c][j], zv[c][j + 1]);
            ab[c] = f2(abv[c][j], abv[c][j + 1]);
          }
          z[0] = z[0] + f2(bu);
          tanh_derivs_fast2<NP>(z[0], p);
          Cls::adjoint(z, p, ab, zb);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            zbv[c][j] = zb[c].v.x;
            zbv[c][j + 1] = zb[c].v.y;
          }
          gb += zb[0].v.x;
          gb += zb[0].v.y;
        }
#pragma unroll
        for (int c = 0; c < C; ++c) st_bf16<PPB>(act_s(z_buf), r, blk(c) * Pc + g, zbv[c]);
      }
      PART(wg, 0, r) = gb;
    }
  }

  // Weight gradients of a chunk's tiles add up in FP32 in the CTA's scratch
  // slot and reach the FP64 slice once per chunk (chunk_flush): per-CTA FP32
  // partials, FP64 across chunks.  Layer l (2..L-1) takes G * wu * wu floats,
  // laid out [sub][k / 4][u][4], so that the 32 rows of a warp cover 512
  // contiguous bytes per vector add.  The adds are fire-and-forget FP32
  // vector reductions; every element belongs to one thread, which adds the
  // tiles in program order, so the sums are deterministic.
  __device__ float* wacc(int l) const {
    return reinterpret_cast<float*>(I.scratch + (long long)blockIdx.x * I.scratch_stride + I.wacc_off) +
           (long long)(l - 2) * gg() * wuu() * wuu();
  }
  __device__ void wacc_zero() {
    float4* a = reinterpret_cast<float4*>(wacc(2));
    const long long n4 = (long long)(I.L - 2) * gg() * wuu() * wuu() / 4;
    for (long long i = tid; i < n4; i += nth()) a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }

  // TMEM columns of lane row (8, from taddr) -> accumulator columns k0 .. k0+7
  // of row u in the [k / 4][u][4] block at acc
  __device__ void acc8(float* acc, int u, int k0, uint32_t taddr, uint64_t pol) const {
    float v[8];
    tc::tmem_ld8(taddr, v);
    tc::tmem_wait_ld();
    const int wu = wuu();
    tc::red_add_v4_hint(acc + ((long long)(k0 / 4) * wu + u) * 4, v[0], v[1], v[2], v[3], pol);
    tc::red_add_v4_hint(acc + ((long long)(k0 / 4 + 1) * wu + u) * 4, v[4], v[5], v[6], v[7], pol);
  }

  // D[R0] (weight-gradient columns nb*NB .. of layer l) -> accumulator.  With
  // packed sub-tiles only the diagonal block of the lane's sub-tile is read:
  // D holds Zbar A^T over all operand rows, and rows of different sub-tiles
  // belong to different points.
  __device__ void acc_wgrad(int l, int nb, int NB) {
    float* acc = wacc(l);
    const int wu = wuu();
    const uint64_t pol = tc::policy_evict_last();
    if (gg() > 1) {  // packed plans have H == 1
      const int sub = ul / wu, j = ul - sub * wu;
      float* a = acc + (long long)sub * wu * wu;
      for (int k0 = wg * 8; k0 < wu; k0 += nw() * 8)
        acc8(a, j, k0, R0(0) + lane_base() + (uint32_t)(sub * wu + k0), pol);
      return;
    }
    for (int h = 0; h < hh(); ++h) {
      if (h * 128 + q * 32 >= ww()) continue;  // warp-uniform
      for (int k0 = wg * 8; k0 < NB; k0 += nw() * 8)
        acc8(acc, h * 128 + ul, nb * NB + k0, R0(h) + lane_base() + (uint32_t)k0, pol);
    }
  }

  // accumulator (summed over sub-tiles) -> FP64 slice, once per chunk;
  // consecutive threads take consecutive weights, eight per batch with their
  // loads in flight before the adds
  __device__ void chunk_flush(double* g) {
    const int wu = wuu(), per = wu * wu;
    for (int l = 2; l <= I.L - 1; ++l) {
      const float* acc = wacc(l);
      double* gW = g + I.off_W[l - 1];
      for (int e0 = tid; e0 < per; e0 += 8 * nth()) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e = e0 + j * nth();
          v[j] = 0.f;
          if (e < per) {
            const int u = e / wu, k = e - u * wu;
            for (int sub = 0; sub < gg(); ++sub)
              v[j] += __ldcg(acc + ((long long)(sub * (wu / 4) + k / 4) * wu + u) * 4 + (k & 3));
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (e0 + j * nth() < per) tc::red_add_f64(gW + e0 + j * nth(), (double)v[j]);
      }
    }
  }

  // layer-1 backward with z^1 recomputed from the points
  __device__ void layer1_bwd(bool abar_from_ub, const Row1& w1p) {
    const float* Pm = I.params;
    const float* ub = UB();
    const int P = pp(), Pc = pc();
    constexpr int d = Cls::D;  // the plan's input dimension
    for (int h = 0; h < hh(); ++h) {
      const int r = h * 128 + ul;
      if (h * 128 + q * 32 >= ww()) continue;
      const int sub = r / wuu(), u = r - sub * wuu();
      float w1[d];
#pragma unroll
      for (int i = 0; i < d; ++i) w1[i] = PRELOAD1B ? w1p.w[h][i] : Pm[I.off_W[0] + u * d + i];
      const float b1 = PRELOAD1B ? w1p.b[h] : Pm[I.off_b[0] + u];
      const int nout = I.n_out;
      float wl[kMaxOut] = {0.f, 0.f, 0.f, 0.f};
      if (abar_from_ub) {
#pragma unroll
        for (int o = 0; o < kMaxOut; ++o)
          if (o < nout) wl[o] = Pm[I.off_W[I.L - 1] + (long long)o * wuu() + u];
      }
      const float* xs = XS() + sub * Pc * d;
      float gw[d], gb = 0.f;
#pragma unroll
      for (int i = 0; i < d; ++i) gw[i] = 0.f;
      // the warpgroups split the points; a fixed shape makes the pass count a
      // compile-time constant, so the passes unroll with constant offsets
#pragma unroll
      for (int k = 0; k < (Pc + nw() * PPB - 1) / (nw() * PPB); ++k) {
        const int g = wg * PPB + k * nw() * PPB;
        if (g >= Pc) break;
        float abv[C][PPB];
        if (!abar_from_ub) {
#pragma unroll
          for (int c = 0; c < C; ++c) tc::tmem_ld<PPB>(R1(h) + lane_base() + (uint32_t)(blk(c) * Pc + g), abv[c]);
          tc::tmem_wait_ld();
        } else {
#pragma unroll
          for (int c = 0; c < C; ++c)
#pragma unroll
            for (int j = 0; j < PPB; ++j) {
              float s = 0.f;
#pragma unroll
              for (int o = 0; o < kMaxOut; ++o)
                if (o < nout) s = fmaf(wl[o], ub[(o * C + c) * P + sub * Pc + g + j], s);
              abv[c][j] = s;
            }
        }
#pragma unroll
        for (int j = 0; j < PPB; j += 2) {
          f2 z[C], p[NP], ab[C], zb[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            z[c] = f2(0.f);
            ab[c] = f2(abv[c][j], abv[c][j + 1]);
          }
          float v0 = b1, v1 = b1;
#pragma unroll
          for (int i = 0; i < d; ++i) {
            v0 = fmaf(w1[i], xs[(g + j) * d + i], v0);
            v1 = fmaf(w1[i], xs[(g + j + 1) * d + i], v1);
          }
          z[0] = f2(v0, v1);
#pragma unroll
          for (int i = 0; i < Cls::D; ++i) {
            const int fo = Cls::first_order(i);
            if (fo >= 0) z[fo] = f2(w1[i]);
          }
          tanh_derivs_fast2<NP>(z[0], p);
          Cls::adjoint(z, p, ab, zb);
          gb += zb[0].v.x;
          gb += zb[0].v.y;
#pragma unroll
          for (int i = 0; i < d; ++i) {
            gw[i] = fmaf(zb[0].v.x, xs[(g + j) * d + i], gw[i]);
            gw[i] = fmaf(zb[0].v.y, xs[(g + j + 1) * d + i], gw[i]);
          }
#pragma unroll
          for (int i = 0; i < Cls::D; ++i) {
            const int fo = Cls::first_order(i);
            if (fo >= 0) {
              gw[i] += zb[fo].v.x;
              gw[i] += zb[fo].v.y;
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < d; ++i) PART(wg, i, r) = gw[i];
      PART(wg, 3, r) = gb;
    }
  }

  __device__ void layer1_flush(double* g) {
    for (int i = 0; i < Cls::D; ++i) part_flush(i, g + I.off_W[0] + i, Cls::D);
    part_flush(3, g + I.off_b[0], 1);
  }

  // ------------------------------------------------------------ one tile
  __device__ double tile(long long t, int mode, double* g) {
    const int P = pp(), L = I.L, d = I.d;
    const bool bwd = mode != MODE_FWD;
    const long long n0 = t * P;
    const long long rem = I.N - n0;
    const int nvalid = rem < (long long)P ? (int)rem : P;
    cur_tile = t;
    const bool store = bwd && I.wstore != nullptr;
    const int last_a = store ? L - 2 : L - 3;  // highest A^l copied out of shared memory
    const Row1 w1 = row_l1(PRELOAD1);
    float* xs = XS();
    for (int i = tid; i < P * d; i += nth()) {
      const int n = i / d;
      xs[i] = n < nvalid ? I.X[(n0 + n) * d + (i % d)] : 0.f;
    }
    // the residual's source rows, staged in the output-adjoint area (free
    // until the residual writes it) while the points load
    if (I.source && I.n_groups == 0 && (I.n_terms + I.n_res) * P <= nw() * 4 * 256) {
      float* ub = UB();
      const int nr = I.n_res;
      for (int i = tid; i < nvalid * nr; i += nth()) ub[i] = I.source[n0 * nr + i];
    }
    if (tid == 0 && !*abort_f) {
      tc::bulk_wait_read0();  // earlier bulk stores must have read ACT(0) before it is rewritten
      if (L >= 3) load_hidden_w(2);
      else load_out_w();
    }
    __syncthreads();
    // ---- forward
    layer1_fwd(0, w1);
    tc::fence_proxy_async_smem();
    sync();
    // scratch keeps A^l for l <= L-3 (A^{L-2} stays in shared memory for the
    // backward); the store keeps A^{L-2} as well, for the weight-gradient GEMM
    if (tid == 0 && bwd && 1 <= last_a && !*abort_f) {
      scratch_out(slot(1), ACT(0), (uint32_t)I.act_bytes);
      if (I.split3) scratch_out(slot(1) + I.act_bytes, ALO(0), (uint32_t)I.alo_bytes);
      tc::bulk_commit();
    }
    int cur = 0;
    for (int l = 2; l <= L - 1; ++l) {
      if (!wait(bar_tma, ph_tma, 10 + l)) break;
      if (tid == 0) {
        tc::tc_fence_after();
        mma_layer(cur);
        // This layer's epilogue rewrites ACT(cur^1) once the MMAs are complete:
        // every copy that read it must be done reading before the commit that
        // releases the epilogue.  With two buffers that is the copy two layers
        // back (the newest copies ACT(cur), which the MMAs only read); with one
        // buffer it is the newest, whose read overlaps the MMAs issued above.
        if (bwd && l - 1 <= last_a && I.o_a0 != I.o_a1) tc::bulk_wait_read1();
        else tc::bulk_wait_read0();
        tc::mma_commit(bar_mma);
      }
      const RowBias bias = row_bias(l);
      if (!wait(bar_mma, ph_mma, 30 + l)) break;
      tc::tc_fence_after();
      if (tid == 0) {
        if (l + 1 <= L - 1) load_hidden_w(l + 1);
        else load_out_w();
      }
      hidden_epilogue(l, cur ^ 1, bias);
      tc::fence_proxy_async_smem();
      sync();
      if (tid == 0 && bwd && l <= last_a) {
        scratch_out(slot(l), ACT(cur ^ 1), (uint32_t)I.act_bytes);
        if (I.split3) scratch_out(slot(l) + I.act_bytes, ALO(cur ^ 1), (uint32_t)I.alo_bytes);
        tc::bulk_commit();
      }
      cur ^= 1;
    }
    // ---- output layer
    if (!*abort_f && wait(bar_tma, ph_tma, 50)) {
      if (tid == 0) {
        tc::tc_fence_after();
        mma_out(cur);
        tc::mma_commit(bar_mma);
      }
      if (wait(bar_mma, ph_mma, 51)) {
        tc::tc_fence_after();
        if (tid == 0 && bwd && L >= 3) load_hidden_w(L - 1);
        out_epilogue();
      }
    }
    sync();
    double loss = 0.0;
    if (!*abort_f) loss = residual(n0, nvalid, bwd);
    __syncthreads();
    if (!bwd || *abort_f) return loss;
    // ---- backward
    out_grads(cur);
    __syncthreads();
    out_grads_flush(g);
    __syncthreads();  // PART is rewritten by the first adjoint epilogue
    const int zb = cur, ain = cur ^ 1;
    // thread 0: A^{l-1} and W^l for the recompute of layer l, requested as
    // soon as the MMAs of layer l+1 have released both buffers.  The layer
    // inputs were written by this CTA's own bulk copies, which must be
    // complete; the nz adjoint copies to the store committed after them may
    // still be writing.
    int nz = 0;
    auto reload_act = [&](int l) {
      tc::bulk_wait_n(nz);
      tc::mbar_arrive_expect_tx(bar_ld, (uint32_t)(I.act_bytes + (I.split3 ? I.alo_bytes : 0)));
      scratch_in(ACT(ain), slot(l - 1), (uint32_t)I.act_bytes);
      if (I.split3) scratch_in(ALO(ain), slot(l - 1) + I.act_bytes, (uint32_t)I.alo_bytes);
    };
    auto request_reload = [&](int l) {
      reload_act(l);
      load_hidden_w(l);
    };
    Row1 w1b;  // W^1, b^1 for the layer-1 backward, loaded before the last MMA wait
    for (int l = L - 1; l >= 2; --l) {
      const RowBias bias = row_bias(l);
      if (l < L - 1) {
        // recompute z^l = W^l A^{l-1} into R0
        if (!wait(bar_ld, ph_ld, 60)) break;
        if (!wait(bar_tma, ph_tma, 61)) break;
        if (tid == 0) {
          tc::tc_fence_after();
          mma_layer(ain);
          tc::mma_commit(bar_mma);
        }
        if (!wait(bar_mma, ph_mma, 62)) break;
        tc::tc_fence_after();
      } else {
        if (!wait(bar_tma, ph_tma, 63)) break;  // W^{L-1} for the data gradient
      }
      if (l == L - 1) adjoint_epilogue<true>(l, zb, bias);
      else adjoint_epilogue<false>(l, zb, bias);
      tc::fence_proxy_async_smem();
      sync();
      if (store) {
        // Zbar^l goes to the store; the weight gradient is a separate GEMM
        if (tid == 0) {
          tc::bulk_s2g(zslot(l), ACT(zb), (uint32_t)I.act_bytes);
          tc::bulk_commit();
          ++nz;
          mma_dgrad(zb);
          tc::mma_commit(bar_mma);
        }
        part_flush(0, g + I.off_b[l - 1], 1);  // bias gradient of layer l, during the MMA
        if (l == 2) w1b = row_l1(PRELOAD1B);
        if (!wait(bar_mma, ph_mma, 66)) break;
        tc::tc_fence_after();
        if (tid == 0) {
          if (l > 2) load_hidden_w(l - 1);  // W^l is free: W^{l-1} loads while the copy reads
          tc::bulk_wait_read0();  // ACT(zb) is rewritten by the reload or the next adjoint
          if (l > 2) reload_act(l - 1);
          // the layer input of the next reload, from HBM into L2 a layer ahead
          if (l > 3) tc::bulk_prefetch_l2(slot(l - 3), (uint32_t)I.act_bytes);
        }
        sync();
        continue;
      }
      const int NB = hh() == 2 ? 128 : ww();
      const int nblk = ww() / NB;
      if (nblk == 1) {
        // weight gradient first, with its own barrier: its flush from TMEM
        // runs while the data-gradient MMA does, and A^{l-2} reloads into
        // ACT(ain) as soon as the weight-gradient MMA has read A^{l-1}; W^{l-1}
        // loads once the data-gradient MMA has read W^l
        if (tid == 0) {
          mma_wgrad(zb, ain, 0, NB);
          tc::mma_commit(bar_wg);
          mma_dgrad(zb);
          tc::mma_commit(bar_mma);
        }
        part_flush(0, g + I.off_b[l - 1], 1);  // bias gradient of layer l, during the MMAs
        if (!wait(bar_wg, ph_wg, 67)) break;
        tc::tc_fence_after();
        if (tid == 0 && l > 2) reload_act(l - 1);
        acc_wgrad(l, 0, NB);
        if (l == 2) w1b = row_l1(PRELOAD1B);
        if (!wait(bar_mma, ph_mma, 64)) break;
        tc::tc_fence_after();
        if (tid == 0 && l > 2) load_hidden_w(l - 1);
        sync();
        continue;
      }
      if (tid == 0) {
        mma_dgrad(zb);
        mma_wgrad(zb, ain, 0, NB);
        tc::mma_commit(bar_mma);
      }
      part_flush(0, g + I.off_b[l - 1], 1);  // bias gradient of layer l, during the MMAs
      if (l == 2) w1b = row_l1(PRELOAD1B);
      if (!wait(bar_mma, ph_mma, 64)) break;
      tc::tc_fence_after();
      acc_wgrad(l, 0, NB);
      for (int nb = 1; nb < nblk; ++nb) {
        sync();
        if (tid == 0) {
          mma_wgrad(zb, ain, nb, NB);
          tc::mma_commit(bar_mma);
        }
        if (!wait(bar_mma, ph_mma, 65)) break;
        tc::tc_fence_after();
        if (tid == 0 && nb == nblk - 1 && l > 2) request_reload(l - 1);
        acc_wgrad(l, nb, NB);
      }
      sync();
    }
    if (L == 2) w1b = row_l1(PRELOAD1B);
    if (!*abort_f) layer1_bwd(L == 2, w1b);
    sync();
    if (!*abort_f) layer1_flush(g);
    __syncthreads();
    return loss;
  }
};

template <class Cls, class Shape>
__global__ void __launch_bounds__(kTcThreads, 1) tc_kernel(const __grid_constant__ TcArgs args) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bars[4];
  // the running work item's descriptor: every epilogue reads its fields, and
  // shared-memory loads keep those reads off the global/param path
  __shared__ TcInst inst_s;
  __shared__ uint32_t tmem_s;
  __shared__ volatile int abort_s;
  __shared__ double red_s[kTcThreads / 32];
  // 1024-byte aligned base, derived from the shared array by pointer arithmetic
  // only, so that every pointer computed from it is known to be shared
  // (loads and stores through it compile to LDS / STS)
  unsigned char* sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nthr = args.nthreads, nwg = nthr / 128;
  if (tid == 0) {
    abort_s = 0;
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::mbar_init(&bars[2], 1);
    tc::mbar_init(&bars[3], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tmem_s, (uint32_t)args.tmem_cols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  uint32_t ph_tma = 0, ph_mma = 0, ph_ld = 0, ph_wg = 0;
  int prev_inst = -1;
  __shared__ int k_s;
  for (int k = blockIdx.x; k < args.n_items && !abort_s;) {
    const int item = args.item_inst ? args.item_inst[k] : k;
    const int ii = args.insts ? args.item_inst[args.n_items + item] : 0;
    const TcInst& Ig = args.insts ? args.insts[ii] : args.inst0;
    if (ii != prev_inst) {
      // the previous item's readers of inst_s passed the barrier at its end
      const uint4* src = reinterpret_cast<const uint4*>(&Ig);
      uint4* dst = reinterpret_cast<uint4*>(&inst_s);
      for (int i = tid; i < (int)(sizeof(TcInst) / 16); i += nthr) dst[i] = src[i];
      __syncthreads();
    }
    const TcInst& I = inst_s;
    const int chunk = item - I.chunk_base;
    if (ii != prev_inst) {
      // zero both activation buffers (and split buffers) once per instance:
      // padding rows and columns must read as zero in every MMA
      uint4 z4 = make_uint4(0, 0, 0, 0);
      for (int i = tid; i < I.act_bytes / 16; i += nthr) {
        reinterpret_cast<uint4*>(sm + I.o_a0)[i] = z4;
        reinterpret_cast<uint4*>(sm + I.o_a1)[i] = z4;
      }
      if (I.split3)
        for (int i = tid; i < I.alo_bytes / 16; i += nthr) {
          reinterpret_cast<uint4*>(sm + I.o_alo0)[i] = z4;
          reinterpret_cast<uint4*>(sm + I.o_alo1)[i] = z4;
        }
      if (tid == 0) {
        tc::prefetch_tensormap(&Ig.wmap);
        tc::prefetch_tensormap(&Ig.wlmap);
      }
      tc::fence_proxy_async_smem();
      __syncthreads();
      prev_inst = ii;
    }
    TcTile<Cls, Shape> T{I,
                  &Ig,
                  sm,
                  &bars[0],
                  &bars[1],
                  &bars[2],
                  &bars[3],
                  &abort_s,
                  args.err,
                  tmem_s,
                  ph_tma,
                  ph_mma,
                  ph_ld,
                  ph_wg,
                  tid,
                  warp,
                  128 * I.H,
                  reinterpret_cast<float*>(sm + I.o_part),
                  warp & 3,
                  warp >> 2,
                  tid & 127,
                  nwg,
                  nthr};
    const bool bwd = args.mode != MODE_FWD;
    // one FP64 slice per chunk (fixed summation order), or one accumulator
    // shared by every chunk, zeroed by the host, when the slices would not
    // fit in L2
    double* g = bwd ? I.grad_slices + (I.slice_shared ? 0LL : (long long)chunk * I.n_params) : nullptr;
    if (bwd && !I.slice_shared)
      for (long long i = tid; i < I.n_params; i += nthr) g[i] = 0.0;
    const bool wacc_on = bwd && !I.wstore && I.L >= 3;  // weight gradients per tile
    if (wacc_on) T.wacc_zero();
    __syncthreads();
    double loss = 0.0;
    const long long t0 = (long long)chunk * I.tiles_per_chunk;
    const long long t1 = (t0 + I.tiles_per_chunk < I.n_tiles) ? t0 + I.tiles_per_chunk : I.n_tiles;
    for (long long t = t0; t < t1 && !abort_s; ++t) loss += T.tile(t, args.mode, g);
    // hidden-layer weight gradients of the chunk's tiles -> FP64 slice
    if (wacc_on && !abort_s) {
      __threadfence();
      __syncthreads();
      T.chunk_flush(g);
    }
    ph_tma = T.ph_tma;
    ph_mma = T.ph_mma;
    ph_ld = T.ph_ld;
    ph_wg = T.ph_wg;
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0) red_s[warp] = loss;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < nthr / 32; ++w) s += red_s[w];
      I.loss_slices[chunk] = s;
    }
    // the next item: from the shared counter, or a fixed stride
    if (args.item_next) {
      if (tid == 0) k_s = (int)gridDim.x + atomicAdd(args.item_next, 1);
      __syncthreads();
      k = k_s;
    } else {
      k += gridDim.x;
    }
    __syncthreads();
  }
  // teardown: drain our own bulk copies and MMAs (bounded), release TMEM
  if (tid == 0) tc::bulk_wait0();
  if (abort_s && tid == 0) {
    volatile int dummy = 0;
    tc::mma_commit(&bars[1]);
    tc::mbar_wait(&bars[1], ph_mma & 1u, &dummy, args.err, 99, 100000000ull);
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem_s, (uint32_t)args.tmem_cols);
}

}  // namespace jet
