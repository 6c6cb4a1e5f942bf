// Instantiation of the ensemble kernel for double tensor arithmetic (no
// tensor-core shape: the use_tc arguments are accepted for symmetry).
#include "ensemble.cuh"

namespace tepai {

// Dynamic shared memory of the ensemble kernel, with the SM's carveout set to
// the largest shared-memory share: the staged shapes place two CTAs of about
// 110 KB on one SM, which the default carveout preference need not allow.
static cudaError_t ensemble_smem_attr_f64(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(ensemble_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(ensemble_kernel<double, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

cudaError_t launch_ensemble_f64(const KArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  cudaError_t e = ensemble_smem_attr_f64(smem);
  if (e != cudaSuccess) return e;
  ensemble_kernel<double, false><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

// Launch without touching the function attribute (set beforehand), for use
// inside a CUDA-graph capture.
cudaError_t launch_ensemble_captured_f64(const KArgs& a, int grid, int block, size_t smem, cudaStream_t st) {
  ensemble_kernel<double, false><<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

// The kernel's address, to find its node in a captured CUDA graph.
const void* ensemble_kernel_fn_f64(int) { return reinterpret_cast<const void*>(ensemble_kernel<double, false>); }

cudaError_t set_ensemble_smem_f64(size_t smem, int) { return ensemble_smem_attr_f64(smem); }

cudaError_t launch_canon_f64(const KArgs& a, int block, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(canon_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  canon_kernel<double><<<1, block, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_ensemble_f64(int block, size_t smem, int, int* ctas_per_sm) {
  cudaError_t e = ensemble_smem_attr_f64(smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, ensemble_kernel<double, false>, block, smem);
}

}  // namespace tepai
