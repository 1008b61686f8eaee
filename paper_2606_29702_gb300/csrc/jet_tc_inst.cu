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

template <class Shape>
static cudaError_t launch_shape(const TcArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(tc_kernel<TcCls, Shape>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_kernel<TcCls, Shape><<<grid, a.nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

#define JET_CAT2(a, b) a##b
#define JET_CAT(a, b) JET_CAT2(a, b)

// A launch whose work items share a tile shape with a compiled fixed-shape
// kernel runs it (a compiled G of 0 accepts any packing); every other launch
// runs the general kernel.
template <>
cudaError_t tc_launch_id<JET_CLASS_ID>(const TcArgs& a, int grid, size_t smem, cudaStream_t s) {
#define JET_TRY_SHAPE(PC_, G_, H_, W_, NT_)                                                     \
  if (a.shape[0] == (PC_) && ((G_) == 0 || a.shape[1] == (G_)) && a.shape[2] == (H_) &&          \
      a.shape[3] == (W_) && a.nthreads == (NT_))                                                \
    return launch_shape<TcShape<PC_, G_, H_, W_, NT_>>(a, grid, smem, s);
  JET_CAT(JET_TC_SHAPES_, JET_CLASS_ID)(JET_TRY_SHAPE)
#undef JET_TRY_SHAPE
  return launch_shape<TcShapeAny>(a, grid, smem, s);
}

// occupancy and attributes of the general kernel (the fixed shapes use the
// same shared-memory carve and register bound)
template <>
cudaError_t tc_max_active_id<JET_CLASS_ID>(size_t smem, int threads, int* blocks) {
  cudaError_t e = cudaFuncSetAttribute(tc_kernel<TcCls, TcShapeAny>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tc_kernel<TcCls, TcShapeAny>, threads, smem);
}

template <>
cudaError_t tc_attrs_id<JET_CLASS_ID>(cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, tc_kernel<TcCls, TcShapeAny>);
}

}  // namespace jet
