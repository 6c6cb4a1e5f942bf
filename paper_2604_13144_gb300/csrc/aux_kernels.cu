// Signed, ||g||_1-weighted ensemble reduction (Sec. II.B; App. B; Statement 2)
// and the device circuit export used by parity checks.
#include "ensemble.cuh"

namespace tepai {

__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x;
  else c += (x - t) + s;
  s = t;
}

// One thread per (snapshot m, observable o): sums sign * v over the samples in
// fixed sample order with Neumaier compensation, in FP64.
// mean = ||g(t_m)||_1 (S + C) / N_s;  stderr = ||g(t_m)||_1 sqrt(Var[v] / N_s).
__global__ void signed_reduce_kernel(const double* __restrict__ v, const signed char* __restrict__ sign,
                                     long long ns, int M, int nobs, const double* __restrict__ gnorm,
                                     double* mean, double* se, double* part) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * nobs) return;
  const int m = e / nobs, o = e - m * nobs;
  double s = 0.0, c = 0.0, q = 0.0, qc = 0.0;
  for (long long i = 0; i < ns; ++i) {
    const double x = (double)sign[i * M + m] * v[(i * M + m) * nobs + o];
    neumaier_add(s, c, x);
    neumaier_add(q, qc, x * x);
  }
  const double mu = (s + c) / (double)ns;
  if (mean) mean[e] = gnorm[m] * mu;
  if (se) {
    double var = 0.0;
    if (ns > 1) var = fmax(0.0, ((q + qc) - (double)ns * mu * mu) / (double)(ns - 1));
    se[e] = gnorm[m] * sqrt(var / (double)ns);
  }
  if (part) { part[3 * e] = s; part[3 * e + 1] = c; part[3 * e + 2] = q + qc; }
}

cudaError_t launch_signed_reduce(const double* v, const signed char* sign, long long ns, int M, int nobs,
                                 const double* gnorm, double* mean, double* se, double* part,
                                 cudaStream_t st) {
  const int tot = M * nobs;
  signed_reduce_kernel<<<(tot + 127) / 128, 128, 0, st>>>(v, sign, ns, M, nobs, gnorm, mean, se, part);
  return cudaGetLastError();
}

// Events of one sample in gate order, drawn with the same device sampler as the
// ensemble kernel. One CTA; thread 0 appends in k order after each step.
__global__ void export_circuit_kernel(const __grid_constant__ KArgs a, unsigned long long s, int* buf,
                                      long long cap, unsigned long long* count) {
  extern __shared__ __align__(16) unsigned char flags[];
  unsigned long long cnt = 0;
  if (a.variant == 3) {
    // N -> infinity sampler: thread 0 merges the terms' events in time order;
    // an event's j is its snapshot index m (first m with t <= t_m)
    double* tn = reinterpret_cast<double*>(flags + ((a.L + 15) / 16) * 16);
    unsigned* ic = reinterpret_cast<unsigned*>(tn + a.L);
    if (threadIdx.x == 0) {
      for (int k = 0; k < a.L; ++k) { ic[k] = 0; tn[k] = clock_next(a, s, k, 0u, 0.0, flags + k); }
      int m = 1;
      while (true) {
        int kb = a.L;
        double tb = __longlong_as_double(0x7ff0000000000000ll);
        for (int k = 0; k < a.L; ++k)
          if (tn[k] < tb) { tb = tn[k]; kb = k; }
        while (m <= a.M && tb > clock_snap_time(a, m)) ++m;
        if (m > a.M) break;
        if ((long long)cnt < cap) {
          buf[4 * cnt] = m; buf[4 * cnt + 1] = kb; buf[4 * cnt + 2] = flags[kb]; buf[4 * cnt + 3] = 0;
        }
        ++cnt;
        ic[kb] += 1;
        tn[kb] = clock_next(a, s, kb, ic[kb], tn[kb], flags + kb);
      }
      *count = cnt;
    }
    return;
  }
  for (long long j = 1; j <= a.run_steps; ++j) {
    for (int k = threadIdx.x; k < a.L; k += blockDim.x) flags[k] = (unsigned char)draw_gate(a, s, j, k);
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 0; k < a.L; ++k) {
        if (flags[k]) {
          if ((long long)cnt < cap) {
            buf[4 * cnt] = (int)j; buf[4 * cnt + 1] = k; buf[4 * cnt + 2] = flags[k]; buf[4 * cnt + 3] = 0;
          }
          ++cnt;
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = cnt;
}

cudaError_t launch_export_circuit(const KArgs& a, unsigned long long s, int* buf, long long cap,
                                  unsigned long long* count, cudaStream_t st) {
  const size_t smem = a.variant == 3 ? (size_t)((a.L + 15) / 16) * 16 + (size_t)a.L * 12 : (size_t)a.L;
  cudaError_t e = cudaFuncSetAttribute(export_circuit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  export_circuit_kernel<<<1, 256, smem, st>>>(a, s, buf, cap, count);
  return cudaGetLastError();
}

}  // namespace tepai
