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

// Predicted cost of every sample of the call, for longest-first scheduling:
// its two-site updates, 1 per B event of a bond gate whose sites are adjacent
// in the chain and 3 (swap, gate, swap back) when they are two apart. Z and C
// events need no SVD and cost 0. One warp per sample; the lanes split the
// (step, term) draws, which are the kernel's own draws.
constexpr int kCostBuckets = 4096;

__global__ void sample_cost_kernel(const __grid_constant__ KArgs a) {
  const long long q = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= a.n_samples) return;
  const unsigned long long s = (unsigned long long)(a.sample_offset + q);
  const long long draws = a.run_steps * (long long)a.L;
  int c = 0;
  for (long long e = lane; e < draws; e += 32) {
    const long long j = 1 + e / a.L;
    const int k = (int)(e - (j - 1) * a.L);
    if (draw_gate(a, s, j, k) == 1) {
      const TermDev& T = a.terms[k];
      if (T.kind == 1) c += (T.b - T.a == 1) ? 1 : 3;
    }
  }
#pragma unroll
  for (int off = 16; off; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  if (lane == 0) a.cost[q] = c < kCostBuckets - 1 ? c : kCostBuckets - 1;
}

// order[0..n) = the samples by decreasing cost: a counting sort in one CTA
// (the order within one cost is left to the atomics; results do not depend
// on it, since every sample writes only its own outputs).
__global__ void order_by_cost_kernel(const int* __restrict__ cost, int* __restrict__ order, long long n) {
  __shared__ int pos[kCostBuckets];
  for (int b = threadIdx.x; b < kCostBuckets; b += blockDim.x) pos[b] = 0;
  __syncthreads();
  for (long long q = threadIdx.x; q < n; q += blockDim.x) {
    int c = cost[q];
    c = c < 0 ? 0 : (c >= kCostBuckets ? kCostBuckets - 1 : c);
    atomicAdd(&pos[c], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // exclusive prefix from the highest cost down
    int run = 0;
    for (int b = kCostBuckets - 1; b >= 0; --b) {
      const int h = pos[b];
      pos[b] = run;
      run += h;
    }
  }
  __syncthreads();
  for (long long q = threadIdx.x; q < n; q += blockDim.x) {
    int c = cost[q];
    c = c < 0 ? 0 : (c >= kCostBuckets ? kCostBuckets - 1 : c);
    const int p = atomicAdd(&pos[c], 1);
    order[p] = (int)q;
  }
}

cudaError_t launch_order_samples(const KArgs& a, cudaStream_t st) {
  const int wpb = 8;
  const long long blocks = (a.n_samples + wpb - 1) / wpb;
  sample_cost_kernel<<<(unsigned)blocks, 32 * wpb, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  order_by_cost_kernel<<<1, 1024, 0, st>>>(a.cost, const_cast<int*>(a.order), a.n_samples);
  return cudaGetLastError();
}

const void* sample_cost_kernel_fn() { return reinterpret_cast<const void*>(&sample_cost_kernel); }

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
