// Instantiates the SIMT kernels for one closure class; compiled once per class
// with -DJET_CLASS_ID=<id> so the classes build in parallel.
#include "jet_simt.cuh"

#ifndef JET_CLASS_ID
#error "JET_CLASS_ID must be defined"
#endif

namespace jet {

using ThisCls = ClassById<JET_CLASS_ID>::type;

namespace {
// Dynamic shared memory and an L1/shared split that holds just the CTAs the
// kernel can keep resident (the rest of the SM's 256 KB stays L1, which
// serves the per-k weight vectors of the jet GEMMs).
template <class K>
cudaError_t prepare(K kernel, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int blocks = 0, dev = 0, smem_sm = 0, reserved = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, kSimtThreads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e != cudaSuccess || blocks < 1 || smem_sm < 1) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const size_t need = (size_t)blocks * (smem + fa.sharedSizeBytes + (size_t)reserved);
  int pct = (int)((need * 100 + (size_t)smem_sm - 1) / (size_t)smem_sm);
  if (pct > 100) pct = 100;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}
}  // namespace

template <>
cudaError_t simt_launch_id<JET_CLASS_ID>(bool fp64, const SimtArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e;
  if (fp64) {
    e = prepare(simt_entry<ThisCls, double>(), smem);
    if (e != cudaSuccess) return e;
    simt_entry<ThisCls, double>()<<<grid, kSimtThreads, smem, s>>>(a);
  } else {
    e = prepare(simt_entry<ThisCls, float>(), smem);
    if (e != cudaSuccess) return e;
    simt_entry<ThisCls, float>()<<<grid, kSimtThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <>
cudaError_t simt_max_active_id<JET_CLASS_ID>(bool fp64, size_t smem, int* blocks) {
  cudaError_t e;
  if (fp64) {
    e = cudaFuncSetAttribute(simt_entry<ThisCls, double>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, simt_entry<ThisCls, double>(), kSimtThreads, smem);
  }
  e = cudaFuncSetAttribute(simt_entry<ThisCls, float>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, simt_entry<ThisCls, float>(), kSimtThreads, smem);
}

template <>
cudaError_t debug_activation_id<JET_CLASS_ID>(int kind, long long n, const double* z, const double* v, double* out,
                                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  debug_activation_kernel<ThisCls><<<grid, 256, 0, s>>>(kind, n, z, v, out);
  return cudaGetLastError();
}

}  // namespace jet
