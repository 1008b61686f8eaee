// Instantiates the SIMT kernels for one closure class; compiled once per class
// with -DJET_CLASS_ID=<id> so the classes build in parallel.
#include "jet_simt.cuh"

#ifndef JET_CLASS_ID
#error "JET_CLASS_ID must be defined"
#endif

namespace jet {

using ThisCls = ClassById<JET_CLASS_ID>::type;

template <>
cudaError_t simt_launch_id<JET_CLASS_ID>(bool fp64, const SimtArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e;
  if (fp64) {
    e = cudaFuncSetAttribute(simt_kernel<ThisCls, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    simt_kernel<ThisCls, double><<<grid, kSimtThreads, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(simt_kernel<ThisCls, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    simt_kernel<ThisCls, float><<<grid, kSimtThreads, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <>
cudaError_t simt_max_active_id<JET_CLASS_ID>(bool fp64, size_t smem, int* blocks) {
  cudaError_t e;
  if (fp64) {
    e = cudaFuncSetAttribute(simt_kernel<ThisCls, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, simt_kernel<ThisCls, double>, kSimtThreads, smem);
  }
  e = cudaFuncSetAttribute(simt_kernel<ThisCls, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, simt_kernel<ThisCls, float>, kSimtThreads, smem);
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
