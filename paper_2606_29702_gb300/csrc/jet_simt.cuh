// Fused SIMT partial-jet kernel (FP64 and plain FP32 forms).
//
// One persistent launch walks a list of work items (instance, chunk of point
// tiles).  For every tile of P collocation points a CTA runs, on chip:
//
//   forward   layer 1 seed (z^1_0 = W^1 x + b^1, z^1_{e_i} = W^1[:, i], higher
//             channels 0), then for every hidden layer the jet GEMM
//             Z^l = W^l A^{l-1} over all C channels with the bias on the value
//             channel only (Eq. 1-3, Sec. 2.2 "fused GEMM"), and the closed-
//             form tanh jet composition in registers (Eq. 2-3 recursion);
//   output    linear output layer on every channel, residual monomials,
//             loss partial (FP64);
//   backward  residual adjoint ub = (2 r / N) dr/du, output-layer adjoint,
//             then for l = L-1 .. 1: activation-jet adjoint (transpose of the
//             composition), weight gradient sum_cols Zb A^T, bias gradient on
//             the value channel, data gradient W^T Zb.
//
// Jets live in shared memory as [unit][point-major column] rows: column =
// n * S + alpha with an odd point stride S >= C (the pad columns stay zero).
// A thread owns one point and TP consecutive units with every channel, so the
// composition and its adjoint are thread-local and each jet-GEMM activation
// load is one conflict-free wavefront.  The hidden z-jets of a tile are
// written to a per-CTA global scratch slot (or to a full-size store) as
// [unit][alpha * P + n] in the forward and read back in the backward, cached
// in L2 only so that L1 keeps the layer's weights: the memory of the backward
// is bounded by the number of CTAs, not by N.
// Gradient partial sums go to a per-(instance, chunk) FP64 slice; every slice
// element is added by one thread in tile order (fire-and-forget FP64 adds),
// so the final FP64 reduction is deterministic.
#pragma once

#include "jet_closures_gen.h"
#include "jet_f2.cuh"
#include "jet_groups.cuh"
#include "jet_internal.h"

namespace jet {

template <class T> struct Vec;
template <> struct Vec<float> { static constexpr int N = 4; using type = float4; };
template <> struct Vec<double> { static constexpr int N = 2; using type = double2; };

template <class T> __device__ __forceinline__ T dev_tanh(T z);
template <> __device__ __forceinline__ float dev_tanh<float>(float z) { return tanhf(z); }
template <> __device__ __forceinline__ double dev_tanh<double>(double z) { return tanh(z); }

// p[k] = tanh^(k)(z) for k < NP, as polynomials of a = tanh z and s = 1 - a^2.
template <class T, int NP>
__device__ __forceinline__ void tanh_derivs(T z, T* p) {
  const T a = dev_tanh<T>(z);
  const T a2 = a * a;
  const T s = T(1) - a2;
  p[0] = a;
  if (NP > 1) p[1] = s;
  if (NP > 2) p[2] = T(-2) * a * s;
  if (NP > 3) p[3] = s * (T(6) * a2 - T(2));
  if (NP > 4) p[4] = T(8) * a * s * (T(2) - T(3) * a2);
  if (NP > 5) p[5] = T(8) * s * (T(15) * a2 * a2 - T(15) * a2 + T(2));
}

// tanh_derivs of two values in a packed pair (accurate tanhf per value, the
// derivative polynomials in a and s packed)
template <int NP>
__device__ __forceinline__ void tanh_derivs_pair(f2 z, f2* p) {
  const f2 a(tanhf(z.v.x), tanhf(z.v.y));
  const f2 a2 = a * a;
  const f2 s = jfma(f2(-1.0f), a2, f2(1.0f));
  p[0] = a;
  if (NP > 1) p[1] = s;
  if (NP > 2) p[2] = f2(-2.0f) * a * s;
  if (NP > 3) p[3] = s * jfma(f2(6.0f), a2, f2(-2.0f));
  if (NP > 4) p[4] = f2(8.0f) * a * s * jfma(f2(-3.0f), a2, f2(2.0f));
  if (NP > 5) p[5] = f2(8.0f) * s * jfma(a2, jfma(f2(15.0f), a2, f2(-15.0f)), f2(2.0f));
}

template <class T>
__device__ __forceinline__ void vload(const T* p, T* out) {
  using V = typename Vec<T>::type;
  V v = *reinterpret_cast<const V*>(p);
  const T* q = reinterpret_cast<const T*>(&v);
#pragma unroll
  for (int j = 0; j < Vec<T>::N; ++j) out[j] = q[j];
}

// Vec<T>::N consecutive values through the read-only path (16-byte aligned)
template <class T>
__device__ __forceinline__ void vldg(const T* p, T* out) {
  using V = typename Vec<T>::type;
  V v = __ldg(reinterpret_cast<const V*>(p));
  const T* q = reinterpret_cast<const T*>(&v);
#pragma unroll
  for (int j = 0; j < Vec<T>::N; ++j) out[j] = q[j];
}

template <class T>
__device__ __forceinline__ void vstore(T* p, const T* in) {
  using V = typename Vec<T>::type;
  V v;
  T* q = reinterpret_cast<T*>(&v);
#pragma unroll
  for (int j = 0; j < Vec<T>::N; ++j) q[j] = in[j];
  *reinterpret_cast<V*>(p) = v;
}

// p[0..3] += (a, b, c, d) in global memory as one fire-and-forget FP32
// vector reduction (16-byte aligned; no value comes back, so nothing waits)
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

struct SimtSmem {
  int P, pitch, wmax, C, nout, d;
  __device__ size_t buf_elems() const { return (size_t)wmax * pitch; }
};

template <class Cls, class T>
struct SimtTile {
  static constexpr int C = Cls::C;
  static constexpr int NP = Cls::NP;
  static constexpr int TP = Vec<T>::N;
  static constexpr int NT = kSimtThreads;
  static constexpr int RU = TP;  // consecutive units per thread
  // k-steps of the jet GEMMs unrolled together (loads in flight): wide
  // channel sets gain from four, KS-sized ones lose (measured)
  static constexpr int UK = C >= 7 ? 4 : 2;

  const DevInstance& I;
  const SimtArgs& A;
  T* B[3];   // jet buffers [wmax][pitch]
  T* UO;     // output jets [n_out*C][P]
  T* UB;     // output adjoints [n_out*C][P]
  T* XS;     // tile points [P][d]
  double* RED;
  int P, pitch, wmax, S;  // S: point stride within a jet row
  const T* params;
  const T* Wt;  // transposed weights [in][out] per layer
  const T* Wc;  // aligned copy of the packed parameters
  // FP32 forms: the chunk's hidden-layer weight gradients add up in FP32 in
  // this CTA's scratch slot (fire-and-forget vector reductions; every element
  // belongs to one thread, which adds the tiles in program order) and reach
  // the FP64 slice once per chunk.  Null: FP64 adds per tile.
  float* wacc_base = nullptr;

  __device__ SimtTile(const DevInstance& I_, const SimtArgs& A_, unsigned char* smem) : I(I_), A(A_) {
    P = I.P;
    pitch = I.pitch;
    S = I.S;
    wmax = 0;
    for (int l = 1; l < I.L; ++l) wmax = max(wmax, I.widths[l]);
    T* base = reinterpret_cast<T*>(smem);
    size_t be = (size_t)wmax * pitch;
    B[0] = base;
    B[1] = base + be;
    B[2] = base + 2 * be;
    UO = base + 3 * be;
    UB = UO + (size_t)I.n_out * C * P;
    XS = UB + (size_t)I.n_out * C * P;
    size_t off = (size_t)(XS - base) + (size_t)P * I.d;
    off = (off * sizeof(T) + 15) / 16 * 16;
    RED = reinterpret_cast<double*>(smem + off);
    params = reinterpret_cast<const T*>(I.params);
    Wt = reinterpret_cast<const T*>(I.Wt);
    Wc = Wt + weight_copy_offset(I.n_params);
    if (sizeof(T) == 4 && I.wacc_off >= 0)
      wacc_base = reinterpret_cast<float*>(A.scratch) + (long long)blockIdx.x * A.scratch_stride + I.wacc_off;
  }

  // accumulator of W^l (l = 2..L-1): [item][4][4] per thread item of wgrad
  __device__ float* wacc(int l) const {
    long long off = 0;
    for (int k = 2; k < l; ++k) off += (long long)I.widths[k] * I.widths[k - 1];
    return wacc_base + off;
  }
  __device__ __noinline__ void wacc_zero() {
    float4* a = reinterpret_cast<float4*>(wacc_base);
    const long long n4 = (wacc(I.L) - wacc_base) / 4;
    for (long long i = threadIdx.x; i < n4; i += NT) a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // accumulator -> FP64 slice (consecutive threads read consecutive floats;
  // eight loads in flight before their adds)
  __device__ __noinline__ void wacc_flush(double* g) {
    for (int l = 2; l <= I.L - 1; ++l) {
      const int wo = I.widths[l], wi = I.widths[l - 1], nkb = wi / 4, n = wo * wi;
      const float* a = wacc(l);
      double* gW = g + I.off_W[l - 1];
      for (int e0 = threadIdx.x; e0 < n; e0 += 8 * NT) {
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = e0 + j * NT < n ? __ldcg(a + e0 + j * NT) : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int e = e0 + j * NT;
          if (e >= n) break;
          const int it = e >> 4, r = (e >> 2) & 3, s = e & 3;
          const int kb = it % nkb, ub = it / nkb;
          atomicAdd(gW + (ub * 4 + r) * wi + kb + s * nkb, (double)v[j]);
        }
      }
    }
  }

  __device__ const T* W(int l) const { return params + I.off_W[l - 1]; }   // l = 1..L
  __device__ const T* bias(int l) const { return params + I.off_b[l - 1]; }
  __device__ const T* WtL(int l) const { return Wt + I.off_W[l - 1]; }

  // hidden layer z-jet location for tile t, hidden layer l (1..L-1)
  __device__ T* zjet(long long tile, int l, bool to_store) const {
    long long off = 0;
    for (int k = 1; k < l; ++k) off += (long long)C * P * I.widths[k];
    if (to_store) return reinterpret_cast<T*>(I.store) + tile * I.store_tile_stride + off;
    return reinterpret_cast<T*>(A.scratch) + (long long)blockIdx.x * A.scratch_stride + off;
  }

  // acc[r][c] += w[r] * a[c] for RU units and C channels.  FP32: channel
  // pairs use the packed FMA, with the unit's weight in both halves.
  static __device__ __forceinline__ void rank1(T (&acc)[RU][C], const T* w, const T* a) {
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int r = 0; r < RU; ++r) {
        const f2 wr(w[r]);
#pragma unroll
        for (int c = 0; c + 1 < C; c += 2) {
          const f2 s = jfma(wr, f2(a[c], a[c + 1]), f2(acc[r][c], acc[r][c + 1]));
          acc[r][c] = s.v.x;
          acc[r][c + 1] = s.v.y;
        }
        if (C & 1) acc[r][C - 1] = fma(w[r], a[C - 1], acc[r][C - 1]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < RU; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = fma(w[r], a[c], acc[r][c]);
    }
  }

  // ---------------------------------------------------------------- forward
  // Every elementwise phase and both jet GEMMs map a thread to one point n of
  // the tile and RU consecutive units u0 .. u0+RU, with all C channels of each
  // (unit, point) in registers: lanes walk points, so a point's channels sit
  // at fixed offsets from one row pointer, shared-memory rows (odd stride S)
  // are read and written conflict-free, the z-jet scratch rows
  // [unit][alpha * P + n] are coalesced, and with RU = TP every thread has
  // exactly one item when the tile fills the CTA (P = TP * threads / width).
  __device__ void layer1(T* out, T* zdst) {
    const int w = I.widths[1], d = I.d, CP = C * P;
    const T* W1 = W(1);
    const T* b1 = bias(1);
    for (int it = threadIdx.x; it < (w / RU) * P; it += NT) {
      const int n = it % P, u0 = (it / P) * RU;
      T x[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) x[i] = i < d ? XS[n * d + i] : T(0);
#pragma unroll
      for (int r = 0; r < RU; ++r) {
        const int u = u0 + r;
        T wrow[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) wrow[i] = i < d ? W1[u * d + i] : T(0);
        T z[C], p[NP], a[C];
#pragma unroll
        for (int c = 0; c < C; ++c) z[c] = T(0);
        T v = b1[u];
#pragma unroll
        for (int i = 0; i < 3; ++i) v += wrow[i] * x[i];
        z[0] = v;
#pragma unroll
        for (int i = 0; i < Cls::D; ++i) {
          const int fo = Cls::first_order(i);
          if (fo >= 0) z[fo] = wrow[i];
        }
        tanh_derivs<T, NP>(z[0], p);
        Cls::compose(z, p, a);
#pragma unroll
        for (int c = 0; c < C; ++c) out[u * pitch + n * S + c] = a[c];
        if (zdst) {
#pragma unroll
          for (int c = 0; c < C; ++c) __stcg(zdst + (long long)u * CP + c * P + n, z[c]);
        }
      }
    }
  }

  // Z^l = W^l A^{l-1} (+ b on channel 0), then a^l = compose(z^l).  Per k a
  // thread reads its point's C activations (one shared-memory wavefront per
  // load: lanes walk points) and RU weights as one vector, for RU * C FMAs.
  __device__ void hidden_fwd(int l, const T* in, T* out, T* zdst) {
    const int wi = I.widths[l - 1], wo = I.widths[l], CP = C * P;
    const T* Wtl = WtL(l);  // [wi][wo]
    const T* bl = bias(l);
    for (int it = threadIdx.x; it < (wo / RU) * P; it += NT) {
      const int n = it % P, u0 = (it / P) * RU;
      T acc[RU][C];
#pragma unroll
      for (int r = 0; r < RU; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[r][c] = T(0);
      const T* ap = in + n * S;  // row k of A^{l-1}, this point's channels
      const T* wp = Wtl + u0;    // row k of W^l^T, this thread's units
#pragma unroll(UK)
      for (int k = 0; k < wi; ++k, ap += pitch, wp += wo) {
        T wv[RU], av[C];
        vldg<T>(wp, wv);
#pragma unroll
        for (int c = 0; c < C; ++c) av[c] = ap[c];
        rank1(acc, wv, av);
      }
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int r = 0; r < RU; r += 2) {
          const int u = u0 + r;
          f2 z[C], p[NP], a[C];
#pragma unroll
          for (int c = 0; c < C; ++c) z[c] = f2(acc[r][c], acc[r + 1][c]);
          z[0] = z[0] + f2(bl[u], bl[u + 1]);
          tanh_derivs_pair<NP>(z[0], p);
          Cls::compose(z, p, a);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            out[u * pitch + n * S + c] = a[c].v.x;
            out[(u + 1) * pitch + n * S + c] = a[c].v.y;
          }
          if (zdst) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
              __stcg(zdst + (long long)u * CP + c * P + n, z[c].v.x);
              __stcg(zdst + (long long)(u + 1) * CP + c * P + n, z[c].v.y);
            }
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const int u = u0 + r;
          T z[C], p[NP], a[C];
#pragma unroll
          for (int c = 0; c < C; ++c) z[c] = acc[r][c];
          z[0] += bl[u];
          tanh_derivs<T, NP>(z[0], p);
          Cls::compose(z, p, a);
#pragma unroll
          for (int c = 0; c < C; ++c) out[u * pitch + n * S + c] = a[c];
          if (zdst) {
#pragma unroll
            for (int c = 0; c < C; ++c) __stcg(zdst + (long long)u * CP + c * P + n, z[c]);
          }
        }
      }
    }
  }

  // a^l = compose(z^l) from a stored z-jet [w][C*P]
  __device__ void compose_from(int l, const T* zsrc, T* out) {
    const int w = I.widths[l], CP = C * P;
    for (int it = threadIdx.x; it < (w / RU) * P; it += NT) {
      const int n = it % P, u0 = (it / P) * RU;
      // all loads first, so that they are in flight together
      T zz[RU][C];
#pragma unroll
      for (int r = 0; r < RU; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) zz[r][c] = __ldcg(zsrc + (long long)(u0 + r) * CP + c * P + n);
      if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int r = 0; r < RU; r += 2) {
          f2 z[C], p[NP], a[C];
#pragma unroll
          for (int c = 0; c < C; ++c) z[c] = f2(zz[r][c], zz[r + 1][c]);
          tanh_derivs_pair<NP>(z[0], p);
          Cls::compose(z, p, a);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            out[(u0 + r) * pitch + n * S + c] = a[c].v.x;
            out[(u0 + r + 1) * pitch + n * S + c] = a[c].v.y;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          T p[NP], a[C];
          tanh_derivs<T, NP>(zz[r][0], p);
          Cls::compose(zz[r], p, a);
#pragma unroll
          for (int c = 0; c < C; ++c) out[(u0 + r) * pitch + n * S + c] = a[c];
        }
      }
    }
  }

  // u_{o,alpha} = W^L a^{L-1}_alpha (+ b^L on the value channel)
  __device__ void output_layer(const T* in) {
    const int L = I.L, wi = I.widths[L - 1], no = I.n_out;
    const T* WL = W(L);
    const T* bL = bias(L);
    const int ncol = C * P;
    for (int it = threadIdx.x; it < no * ncol; it += NT) {
      const int o = it / ncol, col = it % ncol;  // col = alpha * P + n
      const T* ap = in + (col % P) * S + col / P;
      T s = col < P ? bL[o] : T(0);
      for (int k = 0; k < wi; ++k) s = fma(WL[o * wi + k], ap[k * pitch], s);
      UO[o * ncol + col] = s;
    }
  }

  // residual r_c = sum terms - source, loss partial, and (if bwd) ub = dL/du.
  // Residual r_c = sum of the monomials - source, the loss partial and (bwd)
  // UB = dL/du.  When the monomial values fit the UB area and 2 r / N the
  // reduction area: three parallel passes, (point, monomial) products, per
  // point sums, per (point, output channel) adjoints, each keeping the
  // operands and order of a per-point loop over the monomials (which is the
  // fallback).
  __device__ double residual(long long n0, int nvalid, bool bwd) {
    const int ncol = C * P, nt = I.n_terms;
    double loss = 0.0;
    const T* src = reinterpret_cast<const T*>(I.source);
    T* rout = reinterpret_cast<T*>(I.r_out);
    if (I.n_groups > 0) {  // composite loss: every term over its own points
      if (bwd)
        for (int i = threadIdx.x; i < I.n_out * ncol; i += NT) UB[i] = T(0);
      __syncthreads();
      return grouped_residual<T>(I.terms, I.groups, I.n_groups, I.n_res, UO, UB, P, n0, nvalid, src, rout, bwd,
                                 threadIdx.x, NT);
    }
    const T two_over_n = T(2.0 * I.inv_N);
    const bool parallel = nt <= I.n_out * C && I.n_res * P * (int)sizeof(T) <= 64 * (int)sizeof(double);
    if (!parallel) {
      if (bwd)
        for (int i = threadIdx.x; i < I.n_out * ncol; i += NT) UB[i] = T(0);
      __syncthreads();
      for (int n = threadIdx.x; n < nvalid; n += NT) {
        T r[kMaxRes];
        for (int c = 0; c < I.n_res; ++c) r[c] = src ? -src[(n0 + n) * I.n_res + c] : T(0);
        for (int m = 0; m < nt; ++m) {
          const DevTerm& tm = I.terms[m];
          T prod = T(tm.coef);
          for (int f = 0; f < tm.nfac; ++f) prod *= UO[tm.fac[f] * P + n];
          r[tm.comp] += prod;
        }
        for (int c = 0; c < I.n_res; ++c) {
          if (rout) rout[(n0 + n) * I.n_res + c] = r[c];
          loss += (double)r[c] * (double)r[c];
        }
        if (bwd)
          for (int m = 0; m < nt; ++m) {
            const DevTerm& tm = I.terms[m];
            const T g = two_over_n * r[tm.comp] * T(tm.coef);
            for (int f = 0; f < tm.nfac; ++f) {
              T prod = g;
              for (int h = 0; h < tm.nfac; ++h)
                if (h != f) prod *= UO[tm.fac[h] * P + n];
              UB[tm.fac[f] * P + n] += prod;
            }
          }
      }
      return loss;
    }
    T* prodm = UB;                         // [n_terms][P]
    T* rg = reinterpret_cast<T*>(RED);     // [n_res][P]: 2 r / N
    for (int i = threadIdx.x; i < nt * nvalid; i += NT) {
      const int m = i / nvalid, n = i - m * nvalid;
      const DevTerm& tm = I.terms[m];
      T prod = T(tm.coef);
      for (int f = 0; f < tm.nfac; ++f) prod *= UO[tm.fac[f] * P + n];
      prodm[m * P + n] = prod;
    }
    __syncthreads();
    for (int n = threadIdx.x; n < nvalid; n += NT) {
      T r[kMaxRes];
      for (int c = 0; c < I.n_res; ++c) r[c] = src ? -src[(n0 + n) * I.n_res + c] : T(0);
      for (int m = 0; m < nt; ++m) r[I.terms[m].comp] += prodm[m * P + n];
      for (int c = 0; c < I.n_res; ++c) {
        if (rout) rout[(n0 + n) * I.n_res + c] = r[c];
        loss += (double)r[c] * (double)r[c];
        rg[c * P + n] = two_over_n * r[c];
      }
    }
    __syncthreads();  // the products in UB are consumed
    if (!bwd) return loss;
    for (int i = threadIdx.x; i < I.n_out * ncol; i += NT) {
      const int k = i / P, n = i - k * P;
      T acc = T(0);
      if (n < nvalid)
        for (int m = 0; m < nt; ++m) {
          const DevTerm& tm = I.terms[m];
          for (int f = 0; f < tm.nfac; ++f) {
            if (tm.fac[f] != k) continue;
            T prod = rg[tm.comp * P + n] * T(tm.coef);
            for (int h = 0; h < tm.nfac; ++h)
              if (h != f) prod *= UO[tm.fac[h] * P + n];
            acc += prod;
          }
        }
      UB[i] = acc;
    }
    return loss;
  }

  // ---------------------------------------------------------------- backward
  // Abar^{L-1} = W^L^T ub; dW^L = sum_cols ub a^{L-1}^T; db^L = sum_n ub_0
  __device__ void output_bwd(const T* a_last, T* abar, double* g) {
    const int L = I.L, wi = I.widths[L - 1], no = I.n_out;
    const T* WL = W(L);
    const int ncol = C * P;
    // Abar[k][n*S + c], one (unit, point) per item with all channels
    for (int it = threadIdx.x; it < wi * P; it += NT) {
      const int n = it % P, k = it / P;
      T s[C];
#pragma unroll
      for (int c = 0; c < C; ++c) s[c] = T(0);
      for (int o = 0; o < no; ++o) {
        const T w = WL[o * wi + k];
#pragma unroll
        for (int c = 0; c < C; ++c) s[c] = fma(w, UB[o * ncol + c * P + n], s[c]);
      }
#pragma unroll
      for (int c = 0; c < C; ++c) abar[k * pitch + n * S + c] = s[c];
    }
    // dW^L[o][k]: four lanes share a weight, each summing a quarter of the
    // points; the partials combine by shuffles in a fixed order
    // (the loop runs whole warps: every lane of a warp reaches the shuffles)
    const int items = 4 * no * wi, items_w = (items + 31) & ~31;
    for (int it = threadIdx.x; it < items_w; it += NT) {
      const bool act = it < items;
      const int part = it & 3, ok = it >> 2, o = act ? ok / wi : 0, k = act ? ok % wi : 0;
      T s = T(0);
      if (act)
        for (int n = part; n < P; n += 4)
#pragma unroll
          for (int c = 0; c < C; ++c) s = fma(UB[o * ncol + c * P + n], a_last[k * pitch + n * S + c], s);
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (act && part == 0) atomicAdd(g + I.off_W[L - 1] + o * wi + k, (double)s);
    }
    for (int o = threadIdx.x; o < no; o += NT) {
      T s = T(0);
      for (int n = 0; n < P; ++n) s += UB[o * ncol + n];
      atomicAdd(g + I.off_b[L - 1] + o, (double)s);
    }
  }

  // Zbar^l = (d compose / dz)^T Abar^l, per (unit, point), z^l read from zsrc.
  __device__ void act_adjoint(int l, const T* zsrc, const T* abar, T* zbar) {
    const int w = I.widths[l], CP = C * P;
    for (int it = threadIdx.x; it < (w / RU) * P; it += NT) {
      const int n = it % P, u0 = (it / P) * RU;
      // all global loads first, so that they overlap
      T zz[RU][C];
#pragma unroll
      for (int r = 0; r < RU; ++r)
#pragma unroll
        for (int c = 0; c < C; ++c) zz[r][c] = __ldcg(zsrc + (long long)(u0 + r) * CP + c * P + n);
      if constexpr (sizeof(T) == 4) {
        // FP32: units (r, r+1) in packed pairs
#pragma unroll
        for (int r = 0; r < RU; r += 2) {
          const int u = u0 + r;
          f2 z[C], p[NP], ab[C], zb[C];
#pragma unroll
          for (int c = 0; c < C; ++c) {
            z[c] = f2(zz[r][c], zz[r + 1][c]);
            ab[c] = f2(abar[u * pitch + n * S + c], abar[(u + 1) * pitch + n * S + c]);
          }
          tanh_derivs_pair<NP>(z[0], p);
          Cls::adjoint(z, p, ab, zb);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            zbar[u * pitch + n * S + c] = zb[c].v.x;
            zbar[(u + 1) * pitch + n * S + c] = zb[c].v.y;
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const int u = u0 + r;
          T p[NP], ab[C], zb[C];
#pragma unroll
          for (int c = 0; c < C; ++c) ab[c] = abar[u * pitch + n * S + c];
          tanh_derivs<T, NP>(zz[r][0], p);
          Cls::adjoint(zz[r], p, ab, zb);
#pragma unroll
          for (int c = 0; c < C; ++c) zbar[u * pitch + n * S + c] = zb[c];
        }
      }
    }
  }

  // dW^l[u][k] += sum_cols Zbar[u][col] A[k][col]; db^l[u] += sum_n Zbar[u][n]
  __device__ void wgrad(int l, const T* zbar, const T* aprev, double* g) {
    const int wo = I.widths[l], wi = I.widths[l - 1];
    const int ncol = S * P;  // every column, the zero pads of odd S included
    const int nkb = wi / 4;
    double* gW = g + I.off_W[l - 1];
    for (int it = threadIdx.x; it < (wo / 4) * nkb; it += NT) {
      const int kb = it % nkb, ub = it / nkb;
      T acc[4][4];
      if constexpr (sizeof(T) == 4) {
        // FP32: even and odd columns accumulate in the two halves of a
        // packed pair (the 16-byte loads deliver the pairs), summed at the end
        f2 ap2[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) ap2[r][s] = f2(0.f);
        for (int col = 0; col < ncol; col += TP) {
          T zv[4][TP], av[4][TP];
#pragma unroll
          for (int r = 0; r < 4; ++r) vload<T>(zbar + (ub * 4 + r) * pitch + col, zv[r]);
#pragma unroll
          for (int s = 0; s < 4; ++s) vload<T>(aprev + (kb + s * nkb) * pitch + col, av[s]);
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
              for (int j = 0; j < TP; j += 2)
                ap2[r][s] = jfma(f2(zv[r][j], zv[r][j + 1]), f2(av[s][j], av[s][j + 1]), ap2[r][s]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) acc[r][s] = ap2[r][s].v.x + ap2[r][s].v.y;
      } else {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s = 0; s < 4; ++s) acc[r][s] = T(0);
        for (int col = 0; col < ncol; col += TP) {
          T zv[4][TP], av[4][TP];
#pragma unroll
          for (int r = 0; r < 4; ++r) vload<T>(zbar + (ub * 4 + r) * pitch + col, zv[r]);
#pragma unroll
          for (int s = 0; s < 4; ++s) vload<T>(aprev + (kb + s * nkb) * pitch + col, av[s]);
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
              for (int j = 0; j < TP; ++j) acc[r][s] = fma(zv[r][j], av[s][j], acc[r][s]);
        }
      }
      // fire-and-forget adds: every element belongs to one thread, which adds
      // the tiles in order, so the sums stay deterministic
      if constexpr (sizeof(T) == 4) {
        if (wacc_base) {
          float* a = wacc(l) + (long long)it * 16;
#pragma unroll
          for (int r = 0; r < 4; ++r) red_add_v4(a + 4 * r, acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
          continue;
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) atomicAdd(gW + (ub * 4 + r) * wi + kb + s * nkb, (double)acc[r][s]);
    }
    double* gb = g + I.off_b[l - 1];
    for (int u = threadIdx.x; u < wo; u += NT) {
      T s = T(0);
      for (int n = 0; n < P; ++n) s += zbar[u * pitch + n * S];
      atomicAdd(gb + u, (double)s);
    }
  }

  // Abar^{l-1}[k][col] = sum_u W^l[u][k] Zbar^l[u][col].  A thread owns one
  // point and RU consecutive input units (the mapping of hidden_fwd); the
  // weights W^l[u][k0 .. k0+RU) come from the aligned parameter copy.
  __device__ void dgrad(int l, const T* zbar, T* abar) {
    const int wo = I.widths[l], wi = I.widths[l - 1];
    const T* Wl = Wc + I.off_W[l - 1];  // [wo][wi]
    for (int it = threadIdx.x; it < (wi / RU) * P; it += NT) {
      const int n = it % P, k0 = (it / P) * RU;
      T acc[RU][C];
#pragma unroll
      for (int i = 0; i < RU; ++i)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[i][c] = T(0);
      const T* zp = zbar + n * S;  // row u of Zbar^l, this point's channels
      const T* wp = Wl + k0;       // row u of W^l, this thread's input units
#pragma unroll(UK)
      for (int u = 0; u < wo; ++u, zp += pitch, wp += wi) {
        T wv[RU], zv[C];
        vldg<T>(wp, wv);
#pragma unroll
        for (int c = 0; c < C; ++c) zv[c] = zp[c];
        rank1(acc, wv, zv);
      }
#pragma unroll
      for (int i = 0; i < RU; ++i)
#pragma unroll
        for (int c = 0; c < C; ++c) abar[(k0 + i) * pitch + n * S + c] = acc[i][c];
    }
  }

  // dW^1[u][i] += sum_n Zbar_0[u][n] x_i[n] + Zbar_{e_i}[u][n]; db^1[u] += sum_n Zbar_0[u][n]
  __device__ void layer1_bwd(const T* zbar, double* g) {
    const int w = I.widths[1], d = I.d;
    double* gW = g + I.off_W[0];
    double* gb = g + I.off_b[0];
    for (int u = threadIdx.x; u < w; u += NT) {
      T sb = T(0), sw[3] = {T(0), T(0), T(0)};
      for (int n = 0; n < P; ++n) {
        const T z0 = zbar[u * pitch + n * S];
        sb += z0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (i < d) sw[i] = fma(z0, XS[n * d + i], sw[i]);
      }
#pragma unroll
      for (int i = 0; i < Cls::D; ++i) {
        const int fo = Cls::first_order(i);
        if (fo >= 0 && i < d)
          for (int n = 0; n < P; ++n) sw[i] += zbar[u * pitch + n * S + fo];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < d) atomicAdd(gW + u * d + i, (double)sw[i]);
      atomicAdd(gb + u, (double)sb);
    }
  }

  // ---------------------------------------------------------------- driver
  __device__ double tile(long long t, double* g) {
    const int mode = A.mode;
    const long long n0 = t * P;
    const long long rem = I.N - n0;
    const int nvalid = rem < (long long)P ? (int)rem : P;
    const int d = I.d;
    const T* X = reinterpret_cast<const T*>(I.X);
    for (int i = threadIdx.x; i < P * d; i += NT) {
      const int n = i / d;
      XS[i] = n < nvalid ? X[(n0 + n) * d + (i % d)] : T(0);
    }
    __syncthreads();
    const bool use_store = (mode == MODE_BWD_STORE) || (mode == MODE_FWD && I.store != nullptr);
    const bool write_z = (mode == MODE_FWD_BWD) || (mode == MODE_FWD && I.store != nullptr);
    const int L = I.L;
    int cur = 0;
    if (mode != MODE_BWD_STORE) {
      layer1(B[0], write_z ? zjet(t, 1, use_store) : nullptr);
      for (int l = 2; l <= L - 1; ++l) {
        __syncthreads();
        hidden_fwd(l, B[cur], B[cur ^ 1], write_z ? zjet(t, l, use_store) : nullptr);
        cur ^= 1;
      }
    } else {
      compose_from(L - 1, zjet(t, L - 1, true), B[0]);
    }
    __syncthreads();
    output_layer(B[cur]);
    __syncthreads();
    const bool bwd = mode != MODE_FWD;
    double loss = residual(n0, nvalid, bwd);
    __syncthreads();
    if (!bwd) return loss;
    const int ab = (cur + 1) % 3, zb = (cur + 2) % 3, ap = cur;
    output_bwd(B[cur], B[ab], g);
    __syncthreads();
    const bool from_store = mode == MODE_BWD_STORE;
    for (int l = L - 1; l >= 1; --l) {
      act_adjoint(l, zjet(t, l, from_store), B[ab], B[zb]);
      if (l >= 2) compose_from(l - 1, zjet(t, l - 1, from_store), B[ap]);
      __syncthreads();
      if (l >= 2) {
        wgrad(l, B[zb], B[ap], g);
        dgrad(l, B[zb], B[ab]);
      } else {
        layer1_bwd(B[zb], g);
      }
      __syncthreads();
    }
    return loss;
  }
};

constexpr int kWaccTiles = 64;  // tiles per FP32 weight-gradient run (FP32 forms)

template <class Cls, class T>
__device__ __forceinline__ void simt_body(const SimtArgs& args) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int k_s;
  for (int k = blockIdx.x; k < args.n_items;) {
    // batched launches walk a cost-ordered list: position k -> item id, and
    // item id -> instance (second half of item_inst)
    const int item = args.item_inst ? args.item_inst[k] : k;
    const DevInstance& I = args.insts ? args.insts[args.item_inst[args.n_items + item]] : args.inst0;
    const int chunk = item - I.chunk_base;
    SimtTile<Cls, T> S(I, args, smem);
    // the pad columns of the odd point stride are never written: zero them
    // (and everything else) once per item so that the weight-gradient sums
    // over whole rows see zeros there
    for (int i = threadIdx.x; i < 3 * S.wmax * S.pitch; i += kSimtThreads) S.B[0][i] = T(0);
    const bool bwd = args.mode != MODE_FWD;
    double* g = bwd ? I.grad_slices + (long long)chunk * I.n_params : nullptr;
    if (bwd)
      for (long long i = threadIdx.x; i < I.n_params; i += kSimtThreads) g[i] = 0.0;
    const bool wacc_on = bwd && S.wacc_base != nullptr;
    if (wacc_on) S.wacc_zero();
    __syncthreads();
    double loss = 0.0;
    const long long t0 = (long long)chunk * I.tiles_per_chunk;
    const long long t1 = (t0 + I.tiles_per_chunk < I.n_tiles) ? t0 + I.tiles_per_chunk : I.n_tiles;
    if constexpr (Cls::C >= 7) {
      // FP32 runs of at most kWaccTiles tiles: the FP32 rounding of a
      // weight's sum stays below kWaccTiles * 2^-24 of its magnitudes at any N
      long long t = t0;
      while (t < t1) {
        const long long r1 = (wacc_on && t1 - t > kWaccTiles) ? t + kWaccTiles : t1;
        for (; t < r1; ++t) {
          loss += S.tile(t, g);
          __syncthreads();
        }
        if (wacc_on) {
          __threadfence();
          __syncthreads();
          S.wacc_flush(g);
          if (t < t1) {
            __syncthreads();
            S.wacc_zero();
            __syncthreads();
          }
        }
      }
    } else {
      // smaller channel sets keep every register for the tile and flush
      // once per chunk; their accumulator serves only nets too wide for
      // L2-resident FP64 slices
      for (long long t = t0; t < t1; ++t) {
        loss += S.tile(t, g);
        __syncthreads();
      }
      if (wacc_on) {
        __threadfence();
        __syncthreads();
        S.wacc_flush(g);
      }
    }
    // block reduction of the loss partial (fixed order)
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if ((threadIdx.x & 31) == 0) S.RED[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kSimtThreads / 32; ++w) s += S.RED[w];
      I.loss_slices[chunk] = s;
    }
    // the next item: from the shared counter, or a fixed stride
    if (args.item_next) {
      if (threadIdx.x == 0) k_s = (int)gridDim.x + atomicAdd(args.item_next, 1);
      __syncthreads();
      k = k_s;
    } else {
      k += gridDim.x;
    }
    __syncthreads();
  }
}

template <class Cls, class T>
__global__ void __launch_bounds__(kSimtThreads) simt_kernel(const __grid_constant__ SimtArgs args) {
  simt_body<Cls, T>(args);
}

// Channel sets of 10 or more: their tiles take most of the shared memory
// with one CTA per SM, so the registers are sized for one.
template <class Cls, class T>
__global__ void __launch_bounds__(kSimtThreads, 1) simt_kernel_wide(const __grid_constant__ SimtArgs args) {
  simt_body<Cls, T>(args);
}

template <class Cls, class T>
constexpr auto simt_entry() {
  if constexpr (Cls::C >= 10) return &simt_kernel_wide<Cls, T>;
  else return &simt_kernel<Cls, T>;
}

// Elementwise activation rule on [n][C] FP64 jets (verification hook, Eq. 15).
template <class Cls>
__global__ void debug_activation_kernel(int kind, long long n, const double* z, const double* v, double* out) {
  constexpr int C = Cls::C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double zz[C], vv[C], oo[C], p[Cls::NP];
    for (int c = 0; c < C; ++c) {
      zz[c] = z[i * C + c];
      vv[c] = v ? v[i * C + c] : 0.0;
    }
    tanh_derivs<double, Cls::NP>(zz[0], p);
    if (kind == 0) Cls::compose(zz, p, oo);
    else if (kind == 1) Cls::tangent(zz, p, vv, oo);
    else Cls::adjoint(zz, p, vv, oo);
    for (int c = 0; c < C; ++c) out[i * C + c] = oo[c];
  }
}

}  // namespace jet
