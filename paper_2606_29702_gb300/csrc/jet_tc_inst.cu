// Instantiates the tensor-core kernel for one closure class; compiled once per
// class with -DJET_CLASS_ID=<id>.
#include "jet_tc_kernel.cuh"

#ifndef JET_CLASS_ID
#error "JET_CLASS_ID must be defined"
#endif

namespace jet {

template <int ID> cudaError_t tc_launch_id(const TcArgs& a, int grid, size_t smem, cudaStream_t s);
template <int ID> cudaError_t tc_max_active_id(size_t smem, int threads, int* blocks);
template <int ID> cudaError_t tc_attrs_id(cudaFuncAttributes* a);

using TcCls = ClassById<JET_CLASS_ID>::type;

template <>
cudaError_t tc_launch_id<JET_CLASS_ID>(const TcArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(tc_kernel<TcCls>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_kernel<TcCls><<<grid, a.nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <>
cudaError_t tc_max_active_id<JET_CLASS_ID>(size_t smem, int threads, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(tc_kernel<TcCls>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tc_kernel<TcCls>, threads, smem);
}

template <>
cudaError_t tc_attrs_id<JET_CLASS_ID>(cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, tc_kernel<TcCls>);
}

}  // namespace jet
