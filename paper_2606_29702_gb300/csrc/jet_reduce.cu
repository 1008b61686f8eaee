// Weight transposition (plus an aligned copy of the parameters), deterministic FP64 gradient/loss reduction over the
// chunk slices, and the fused full-batch Adam update (Sec. 3.1.1).
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
// paper fixes only the learning rate (1e-3).
struct AdamConst {
  double lr, beta1, beta2, eps, bc1, bc2;
};

template <class T, bool ADAM>
__global__ void reduce_kernel(const __grid_constant__ ReduceJob job0, const ReduceJob* jobs, AdamConst ac) {
  const ReduceJob& J = jobs ? jobs[blockIdx.y] : job0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < J.n_params;
       p += (long long)gridDim.x * blockDim.x) {
    double g = 0.0;
    const int gc = J.grad_chunks > 0 ? J.grad_chunks : J.n_chunks;
    for (int c = 0; c < gc; ++c) g += J.grad_slices[(long long)c * J.n_params + p];
    if (J.grad_out) reinterpret_cast<T*>(J.grad_out)[p] = (T)g;
    if (ADAM) {
      T* th = reinterpret_cast<T*>(J.params);
      T* m = reinterpret_cast<T*>(J.m);
      T* v = reinterpret_cast<T*>(J.v);
      const double mm = ac.beta1 * (double)m[p] + (1.0 - ac.beta1) * g;
      const double vv = ac.beta2 * (double)v[p] + (1.0 - ac.beta2) * g * g;
      m[p] = (T)mm;
      v[p] = (T)vv;
      const double mhat = mm / ac.bc1, vhat = vv / ac.bc2;
      th[p] = (T)((double)th[p] - ac.lr * mhat / (sqrt(vhat) + ac.eps));
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && J.loss_out) {
    double s = 0.0;
    for (int c = 0; c < J.n_chunks; ++c) s += J.loss_slices[c];
    *J.loss_out = s * J.inv_N;
  }
}

cudaError_t launch_reduce(const ReduceJob* dev_jobs, const ReduceJob& job0, int n, long long max_params, bool fp64,
                          bool adam, long long step, float lr, cudaStream_t s) {
  AdamConst ac;
  ac.lr = lr;
  ac.beta1 = 0.9;
  ac.beta2 = 0.999;
  ac.eps = 1e-8;
  ac.bc1 = 1.0 - pow(ac.beta1, (double)(step < 1 ? 1 : step));
  ac.bc2 = 1.0 - pow(ac.beta2, (double)(step < 1 ? 1 : step));
  long long gx = (max_params + 255) / 256;
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  dim3 grid((unsigned)gx, (unsigned)(n > 0 ? n : 1));
  const ReduceJob* jobs = n == 1 ? nullptr : dev_jobs;
  if (fp64) {
    if (adam) reduce_kernel<double, true><<<grid, 256, 0, s>>>(job0, jobs, ac);
    else reduce_kernel<double, false><<<grid, 256, 0, s>>>(job0, jobs, ac);
  } else {
    if (adam) reduce_kernel<float, true><<<grid, 256, 0, s>>>(job0, jobs, ac);
    else reduce_kernel<float, false><<<grid, 256, 0, s>>>(job0, jobs, ac);
  }
  return cudaGetLastError();
}

}  // namespace jet
