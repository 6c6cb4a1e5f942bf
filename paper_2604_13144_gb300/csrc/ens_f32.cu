// Instantiations of the ensemble kernel for float tensor arithmetic: one that
// may hold TMEM for the tensor-core launch shape, one without any TMEM code
// for the CUDA-core shapes.
#include "ensemble.cuh"

namespace tepai {

// Dynamic shared memory of the ensemble kernel, with the SM's carveout set to
// the largest shared-memory share: the staged shapes place two CTAs of about
// 110 KB on one SM, which the default carveout preference need not allow.
template <bool TC>
static cudaError_t ensemble_smem_attr_f32(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(ensemble_kernel<float, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(ensemble_kernel<float, TC>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

cudaError_t launch_ensemble_f32(const KArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  cudaError_t e = a.use_tc ? ensemble_smem_attr_f32<true>(smem) : ensemble_smem_attr_f32<false>(smem);
  if (e != cudaSuccess) return e;
  if (a.use_tc) ensemble_kernel<float, true><<<grid, block, smem, st>>>(a);
  else ensemble_kernel<float, false><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

// Launch without touching the function attribute (set beforehand), for use
// inside a CUDA-graph capture.
cudaError_t launch_ensemble_captured_f32(const KArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  if (a.use_tc) ensemble_kernel<float, true><<<grid, block, smem, st>>>(a);
  else ensemble_kernel<float, false><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

// The kernel's address, to find its node in a captured CUDA graph.
const void* ensemble_kernel_fn_f32(int use_tc) {
  return use_tc ? reinterpret_cast<const void*>(ensemble_kernel<float, true>)
                : reinterpret_cast<const void*>(ensemble_kernel<float, false>);
}

cudaError_t set_ensemble_smem_f32(size_t smem, int use_tc) {
  return use_tc ? ensemble_smem_attr_f32<true>(smem) : ensemble_smem_attr_f32<false>(smem);
}

cudaError_t launch_canon_f32(const KArgs& a, int block, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(canon_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  canon_kernel<float><<<1, block, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_ensemble_f32(int block, size_t smem, int use_tc, int* ctas_per_sm) {
  cudaError_t e = use_tc ? ensemble_smem_attr_f32<true>(smem) : ensemble_smem_attr_f32<false>(smem);
  if (e != cudaSuccess) return e;
  return use_tc ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, ensemble_kernel<float, true>, block, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, ensemble_kernel<float, false>, block, smem);
}

}  // namespace tepai
