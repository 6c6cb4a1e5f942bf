// Throughput microbenchmarks of the pipes the ensemble kernel runs on: FP32
// and FP64 fused multiply-add on the CUDA cores, and TF32 MMA on the tensor
// cores (tcgen05.mma kind::tf32, M = 128, N = 256, K = 8, operands in shared
// memory, accumulator in TMEM). They give the measured denominators of the
// roofline fractions. Each kernel keeps every SM busy with independent work
// and is timed with CUDA events on a stream of its own, after a warm-up launch.
#include <cstdint>

#include "../../include/tepai.h"
#include "common.cuh"
#include "tc.cuh"

namespace tepai {

// 8 independent FMA chains per thread, `iters` rounds: 16 iters flops per thread.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T* out, int iters, T seed) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = seed + (T)(threadIdx.x + j);
  const T a = (T)0.999999, b = (T)1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)-12345.0) out[blockIdx.x] = s;   // keeps the chains live
}

// One CTA per SM: thread 0 issues `iters` rounds of four K = 8 MMAs into a
// 128 x 256 FP32 accumulator and commits once; every wait is bounded.
__global__ void __launch_bounds__(128, 1) tf32_peak_kernel(int iters, int* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_bar;
  float* A = reinterpret_cast<float*>(smem);           // 128 x 32
  float* B = A + 128 * 32;                              // 256 x 32
  for (int e = threadIdx.x; e < 384 * 32; e += blockDim.x) A[e] = tc::tf32_rna(1.0f / (float)(1 + (e & 63)));
  if (threadIdx.x < 32) { tc::alloc(&s_tmem, 256); tc::relinquish(); }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::saddr(&s_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_smem_to_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  if (threadIdx.x == 0) {
    const uint32_t idesc = tc::idesc_tf32(128, 256);
    for (int it = 0; it < iters; ++it)
      for (int s = 0; s < 4; ++s) {
        const uint64_t da = tc::desc(tc::saddr(A) + s * 256, 128, 32 * 32);
        const uint64_t db = tc::desc(tc::saddr(B) + s * 256, 128, 32 * 32);
        tc::mma_tf32(tmem, da, db, idesc, (it > 0 || s > 0) ? 1u : 0u);
      }
    tc::commit(&s_bar);
  }
  bool ok = false;
  for (int i = 0; i < (1 << 26) && !ok; ++i) {
    uint32_t r;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(r) : "r"(tc::saddr(&s_bar)) : "memory");
    ok = r != 0;
  }
  if (!ok && threadIdx.x == 0) atomicExch(status, 1);
  tc::fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tc::dealloc(tmem, 256);
}

namespace {

template <class Launch>
int time_launch(Launch launch, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return TEPAI_ERR_CUDA;
  launch();                                   // warm-up
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  const cudaError_t e = cudaEventSynchronize(e1);
  cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? TEPAI_OK : TEPAI_ERR_CUDA;
}

}  // namespace
}  // namespace tepai

using namespace tepai;

extern "C" int tepai_measure_peaks(int cuda_device, double* fp32_tflops, double* fp64_tflops,
                                   double* tf32_tflops) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TEPAI_ERR_NO_DEVICE;
  if (cuda_device < 0 || cuda_device >= ndev) return TEPAI_ERR_INVALID_ARG;
  if (cudaSetDevice(cuda_device) != cudaSuccess) return TEPAI_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cuda_device) != cudaSuccess) return TEPAI_ERR_CUDA;
  cudaStream_t st;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return TEPAI_ERR_CUDA;
  void* scratch = nullptr;
  if (cudaMalloc(&scratch, 4096 * sizeof(double) + 16) != cudaSuccess) { cudaStreamDestroy(st); return TEPAI_ERR_OUT_OF_MEMORY; }
  int rc = TEPAI_OK;
  const int blocks = sms * 8, threads = 256;
  float ms = 0.f;
  if (fp32_tflops && rc == TEPAI_OK) {
    const int iters = 1 << 16;
    rc = time_launch([&] { fma_peak_kernel<float><<<blocks, threads, 0, st>>>((float*)scratch, iters, 1.f); }, st, &ms);
    *fp32_tflops = rc == TEPAI_OK ? 16.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12 : 0.0;
  }
  if (fp64_tflops && rc == TEPAI_OK) {
    const int iters = 1 << 11;
    rc = time_launch([&] { fma_peak_kernel<double><<<blocks, threads, 0, st>>>((double*)scratch, iters, 1.0); }, st, &ms);
    *fp64_tflops = rc == TEPAI_OK ? 16.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12 : 0.0;
  }
  if (tf32_tflops && rc == TEPAI_OK) {
    const int iters = 1 << 12;
    const size_t smem = 384 * 32 * sizeof(float);
    int* status = reinterpret_cast<int*>(static_cast<char*>(scratch) + 4096 * sizeof(double));
    if (cudaFuncSetAttribute(tf32_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) {
      rc = TEPAI_ERR_CUDA;
    } else {
      rc = time_launch([&] { tf32_peak_kernel<<<sms, 128, smem, st>>>(iters, status); }, st, &ms);
      int bad = 0;
      if (rc == TEPAI_OK && cudaMemcpy(&bad, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = TEPAI_ERR_CUDA;
      if (bad) rc = TEPAI_ERR_DEVICE_CHECK;
      *tf32_tflops = rc == TEPAI_OK ? 2.0 * 128 * 256 * 8 * 4.0 * iters * (double)sms / (ms * 1e-3) / 1e12 : 0.0;
    }
  }
  cudaFree(scratch);
  cudaStreamDestroy(st);
  return rc;
}
