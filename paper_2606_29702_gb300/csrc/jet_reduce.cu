// Weight transposition (plus an aligned copy of the parameters), deterministic FP64 gradient/loss reduction over the
// chunk slices, and the fused full-batch Adam update (Sec. 3.1.1).
#include <cmath>

#include "jet_internal.h"

namespace jet {

template <class T>
__global__ void transpose_weights_kernel(const __grid_constant__ DevInstance I, T* Wt) {
  const T* P = reinterpret_cast<const T*>(I.params);
  T* Wc = Wt + weight_copy_offset(I.n_params);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < I.n_params;
       e += (long long)gridDim.x * blockDim.x) {
    Wc[e] = P[e];
    for (int l = 0; l < I.L; ++l) {
      const long long off = I.off_W[l];
      const int fi = I.widths[l], fo = I.widths[l + 1];
      if (e >= off && e < off + (long long)fi * fo) {
        const long long r = e - off;
        const int o = (int)(r / fi), i = (int)(r % fi);
        Wt[off + (long long)i * fo + o] = P[e];
        break;
      }
    }
  }
}

cudaError_t launch_transpose_weights(const DevInstance& in, bool fp64, void* Wt, cudaStream_t s) {
  int grid = (int)((in.n_params + 255) / 256);
  if (grid > 2048) grid = 2048;
  if (grid < 1) grid = 1;
  if (fp64) transpose_weights_kernel<double><<<grid, 256, 0, s>>>(in, reinterpret_cast<double*>(Wt));
  else transpose_weights_kernel<float><<<grid, 256, 0, s>>>(in, reinterpret_cast<float*>(Wt));
  return cudaGetLastError();
}

// Adam (Kingma & Ba 2015) with beta1 = 0.9, beta2 = 0.999, eps = 1e-8; the
// paper fixes only the learning rate (1e-3).  The update runs in the value
// type of the parameters (FP32 for the FP32 and BF16 forms); the gradient it
// takes is the FP64 sum over chunks.
// The 1-based step t is `step`, or *step_ctr + 1 when the counter lives in
// device memory; the bias corrections 1 - beta^t = -expm1(t ln beta) are
// formed on the device in both cases (ln beta from the host), so the two give
// identical updates for the same t.
struct AdamConst {
  double lr, beta1, beta2, eps;
  double ln_beta1, ln_beta2;
  float lr_f, beta1_f, beta2_f, eps_f;
  long long step;
  const long long* step_ctr;
};

// One block takes 32 consecutive parameters (lanes over parameters, so every
// slice row is read coalesced); its 8 warps sum every 8th chunk slice in FP64
// and warp 0 adds the 8 partials in a fixed order: deterministic, and enough
// blocks to fill the GPU when there are many chunks.
constexpr int kRedWarps = 8;

template <class T, bool ADAM>
__global__ void __launch_bounds__(32 * kRedWarps) reduce_kernel(const __grid_constant__ ReduceJob job0,
                                                                const ReduceJob* jobs, AdamConst ac) {
  const ReduceJob& J = jobs ? jobs[blockIdx.y] : job0;
  // the grid covers the largest job: blocks past this job's parameters have
  // nothing to do (block 0 stays: it writes the loss, also of loss-only jobs)
  if (blockIdx.x > 0 && (long long)blockIdx.x * 32 >= J.n_params) return;
  __shared__ double part[kRedWarps][32];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int gc = J.grad_chunks > 0 ? J.grad_chunks : J.n_chunks;
  // bias corrections: one thread per block, one expm1 each (FP32 for the
  // FP32 update; FP64 arithmetic is slow on this GPU)
  __shared__ double bc_s[2];
  if (ADAM) {
    if (threadIdx.x == 0) {
      const long long t = ac.step_ctr ? *ac.step_ctr + 1 : ac.step;
      if (sizeof(T) == 4) {
        bc_s[0] = (double)-expm1f((float)((double)t * ac.ln_beta1));
        bc_s[1] = (double)-expm1f((float)((double)t * ac.ln_beta2));
      } else {
        bc_s[0] = -expm1((double)t * ac.ln_beta1);
        bc_s[1] = -expm1((double)t * ac.ln_beta2);
      }
    }
    __syncthreads();
  }
  const double bc1 = ADAM ? bc_s[0] : 1.0, bc2 = ADAM ? bc_s[1] : 1.0;
  const float bc1_f = (float)bc1, bc2_f = (float)bc2;
  for (long long p0 = (long long)blockIdx.x * 32; p0 < J.n_params; p0 += (long long)gridDim.x * 32) {
    const long long p = p0 + lane;
    double g = 0.0;
    if (p < J.n_params)
      for (int c = wp; c < gc; c += kRedWarps) g += J.grad_slices[(long long)c * J.n_params + p];
    part[wp][lane] = g;
    __syncthreads();
    if (wp == 0 && p < J.n_params) {
      g = 0.0;
#pragma unroll
      for (int w = 0; w < kRedWarps; ++w) g += part[w][lane];
      if (J.grad_out) reinterpret_cast<T*>(J.grad_out)[p] = (T)g;
      if (ADAM) {
        T* th = reinterpret_cast<T*>(J.params);
        T* m = reinterpret_cast<T*>(J.m);
        T* v = reinterpret_cast<T*>(J.v);
        if constexpr (sizeof(T) == 4) {
          const float gf = (float)g;
          const float mm = ac.beta1_f * m[p] + (1.0f - ac.beta1_f) * gf;
          const float vv = ac.beta2_f * v[p] + (1.0f - ac.beta2_f) * gf * gf;
          m[p] = mm;
          v[p] = vv;
          th[p] = th[p] - ac.lr_f * (mm / bc1_f) / (sqrtf(vv / bc2_f) + ac.eps_f);
        } else {
          const double mm = ac.beta1 * (double)m[p] + (1.0 - ac.beta1) * g;
          const double vv = ac.beta2 * (double)v[p] + (1.0 - ac.beta2) * g * g;
          m[p] = (T)mm;
          v[p] = (T)vv;
          const double mhat = mm / bc1, vhat = vv / bc2;
          th[p] = (T)((double)th[p] - ac.lr * mhat / (sqrt(vhat) + ac.eps));
        }
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && J.loss_out) {
    double s = 0.0;
    for (int c = 0; c < J.n_chunks; ++c) s += J.loss_slices[c];
    *J.loss_out = s * J.inv_N;
  }
}

// the device step counter advances once the update that read it is done
__global__ void adam_advance_kernel(long long* step_ctr) { *step_ctr += 1; }

cudaError_t launch_reduce(const ReduceJob* dev_jobs, const ReduceJob& job0, int n, long long max_params, bool fp64,
                          bool adam, long long step, float lr, cudaStream_t s, long long* step_ctr) {
  AdamConst ac;
  ac.lr = lr;
  ac.beta1 = 0.9;
  ac.beta2 = 0.999;
  ac.eps = 1e-8;
  ac.ln_beta1 = std::log(ac.beta1);
  ac.ln_beta2 = std::log(ac.beta2);
  ac.lr_f = lr;
  ac.beta1_f = 0.9f;
  ac.beta2_f = 0.999f;
  ac.eps_f = 1e-8f;
  ac.step = step < 1 ? 1 : step;
  ac.step_ctr = adam ? step_ctr : nullptr;
  long long gx = (max_params + 31) / 32;
  if (gx > 4096) gx = 4096;
  if (gx < 1) gx = 1;
  dim3 grid((unsigned)gx, (unsigned)(n > 0 ? n : 1));
  const ReduceJob* jobs = n == 1 ? nullptr : dev_jobs;
  const int threads = 32 * kRedWarps;
  if (fp64) {
    if (adam) reduce_kernel<double, true><<<grid, threads, 0, s>>>(job0, jobs, ac);
    else reduce_kernel<double, false><<<grid, threads, 0, s>>>(job0, jobs, ac);
  } else {
    if (adam) reduce_kernel<float, true><<<grid, threads, 0, s>>>(job0, jobs, ac);
    else reduce_kernel<float, false><<<grid, threads, 0, s>>>(job0, jobs, ac);
  }
  if (adam && step_ctr) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    adam_advance_kernel<<<1, 1, 0, s>>>(step_ctr);
  }
  return cudaGetLastError();
}

}  // namespace jet
