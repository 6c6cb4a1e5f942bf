// Dense products on the tensor cores for the single-precision engine: a real
// 3xTF32 GEMM with FP32 accumulators in TMEM (tc_gemm), and a complex GEMM
// built on it by the real embedding of complex products (tc_cgemm).
#pragma once
#include "svd_update.cuh"
#include "tc.cuh"

namespace tepai {

// One staged chunk of a 128-row operand: element (r, k) of the chunk, r < 128,
// k < KT, is written to float offset kmajor_off(r, k, KT) of the hi and lo
// tiles. Thread t handles elements t, t + nt, ...; consecutive elements fill
// one core matrix (8 rows x 4 elements, 128 contiguous bytes) per warp. The
// operand reads of a thread's elements are all issued before the first
// conversion, so their latencies overlap.
template <class F>
__device__ __forceinline__ void tc_stage(float* hi, float* lo, int rows, F f) {
  constexpr int PER = 8;
  constexpr int TOTAL = 128 * TcJac::KT;
  const int cores_k = TcJac::KT / 4;
  for (int e0 = threadIdx.x; e0 < TOTAL; e0 += blockDim.x * PER) {
    float x[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = e0 + u * blockDim.x;
      const int core = e >> 5, w = e & 31;
      const int r = (core / cores_k) * 8 + (w >> 2), k = (core % cores_k) * 4 + (w & 3);
      x[u] = (e < TOTAL && r < rows) ? f(r, k) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < TOTAL) {
        const float h = tc::tf32_rna(x[u]);
        hi[e] = h;
        lo[e] = tc::tf32_rna(x[u] - h);
      }
    }
  }
}

// D (TMEM columns 0 .. N-1, 128 lanes) = sum_k A(i, k) B(j, k), i < 128, j < N
// (N a multiple of 16, <= 128), in 3xTF32 with FP32 accumulation, over nch
// chunks of KT along k. stage(c, Ahi, Alo, Bhi, Blo) fills the operand tiles
// of chunk c (128 x KT and N x KT, hi and lo parts, K-major core-matrix
// layout); with same = true only A is staged and B is A itself. Chunks go
// through TcJac::STAGES stages in turn; a stage is refilled only after the
// MMAs that read it have completed (tcgen05.commit on the stage's mbarrier).
// With more than one stage the staging of chunk c + 1 overlaps the MMAs of
// chunk c; with one, the other CTA on the SM fills that time. Returns once the
// accumulator is complete; on a wait that runs out the CTA records
// ST_MMA_TIMEOUT and failed() is set.
template <typename R, bool TC>
template <class STAGE>
__device__ void Engine<R, TC>::tc_pipeline(int N, int nch, bool same, STAGE stage) {
  float* base = reinterpret_cast<float*>(sm.x);
  const uint32_t idesc = tc::idesc_tf32(128, N);
  const uint32_t sbo = TcJac::KT * 32;
  for (int c = 0; c < nch && !failed(); ++c) {
    const int s = c % TcJac::STAGES;
    if (c >= TcJac::STAGES && !tc_wait(s)) return;
    float* Ahi = base + (size_t)s * 4 * TcJac::OP_FLOATS;
    float* Alo = Ahi + TcJac::OP_FLOATS;
    float* Bhi = Alo + TcJac::OP_FLOATS;
    float* Blo = Bhi + TcJac::OP_FLOATS;
    stage(c, Ahi, Alo, Bhi, Blo);
    tc::fence_smem_to_async();
    __syncthreads();
    if (tid() == 0) {
      tc::fence_after();
      const float* bh = same ? Ahi : Bhi;
      const float* bl = same ? Alo : Blo;
      for (int st4 = 0; st4 < TcJac::KT / 8; ++st4) {
        const uint32_t off = (uint32_t)st4 * 256;
        const uint64_t dah = tc::desc(tc::saddr(Ahi) + off, 128, sbo), dal = tc::desc(tc::saddr(Alo) + off, 128, sbo);
        const uint64_t dbh = tc::desc(tc::saddr(bh) + off, 128, sbo), dbl = tc::desc(tc::saddr(bl) + off, 128, sbo);
        tc::mma_tf32(tmem, dah, dbh, idesc, (c > 0 || st4 > 0) ? 1u : 0u);
        tc::mma_tf32(tmem, dah, dbl, idesc, 1u);
        tc::mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      tc::commit(tcbar + s);
      st.tc_flops += 3.0 * (TcJac::KT / 8) * 2.0 * 128.0 * N * 8.0;
    }
    tc_cnt[s]++;
  }
  if (failed()) return;
  // the last commit covers every MMA issued before it
  if (!tc_wait((nch - 1) % TcJac::STAGES)) return;
  tc::fence_after();
}

// tc_pipeline with operands given element by element: fa(i, k) and fb(j, k)
// (callers return 0 outside their extents; k >= K is padded here).
template <typename R, bool TC>
template <class FA, class FB>
__device__ void Engine<R, TC>::tc_gemm(int N, int K, bool same, FA fa, FB fb) {
  const int nch = (K + TcJac::KT - 1) / TcJac::KT;
  tc_pipeline(N, nch, same, [&](int c, float* Ahi, float* Alo, float* Bhi, float* Blo) {
    const int k0 = c * TcJac::KT;
    tc_stage(Ahi, Alo, 128, [&](int i, int k) { return k0 + k < K ? fa(i, k0 + k) : 0.f; });
    if (!same) tc_stage(Bhi, Blo, N, [&](int j, int k) { return k0 + k < K ? fb(j, k0 + k) : 0.f; });
  });
}

// Bounded wait for the latest commit on stage barrier s (idempotent). Returns
// false after recording ST_MMA_TIMEOUT when the MMAs did not complete.
template <typename R, bool TC>
__device__ bool Engine<R, TC>::tc_wait(int s) {
  if (tc_cnt[s] == 0) return true;
  const uint32_t parity = (tc_cnt[s] - 1) & 1u;
  bool ok = false;
  for (int it = 0; it < (1 << 24) && !ok; ++it) ok = bulk::try_wait(tcbar + s, parity);
  if (__syncthreads_and(ok)) return true;
  fail(ST_MMA_TIMEOUT, s);
  return false;
}

// out(i, j) = sum_{k < K} A(i, k) B(k, j) for complex i < M, j < N, through
// the real 3xTF32 GEMM: [Re C, Im C] = [Re A, Im A] [[Re B, Im B], [-Im B, Re B]],
// one 128-row tile of C and 64 complex columns (128 TMEM columns) at a time.
// fa(i, k) and fb(k, j) return complex elements (called only inside the
// extents); fo(i, j, v) stores one. Called by all threads of the CTA.
template <typename R, bool TC>
template <class FA, class FB, class FO>
__device__ void Engine<R, TC>::tc_cgemm(int M, int N, int K, FA fa, FB fb, FO fo) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  for (int m0 = 0; m0 < M && !failed(); m0 += 128) {
    for (int n0 = 0; n0 < N && !failed(); n0 += 64) {
      const int nn = min(64, N - n0);
      tc_gemm(128, 2 * K, false,
              [&](int i, int k) {
                const int r = m0 + i;
                if (r >= M) return 0.f;
                if (k < K) return (float)fa(r, k).re;
                return (float)fa(r, k - K).im;
              },
              [&](int j, int k) {
                const int jj = j & 63;
                if (jj >= nn) return 0.f;
                const bool im_out = j >= 64;
                if (k < K) {
                  const auto v = fb(k, n0 + jj);
                  return (float)(im_out ? v.im : v.re);
                }
                const auto v = fb(k - K, n0 + jj);
                return (float)(im_out ? v.re : -v.im);
              });
      if (failed()) return;
      const int quad = w & 3, r = m0 + quad * 32 + lane;
      for (int cg = w >> 2; cg < 8; cg += nw >> 2) {
        float vr[8], vi[8];
        tc::ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cg * 8), vr);
        tc::ld8(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(64 + cg * 8), vi);
        if (r < M) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = n0 + cg * 8 + j;
            if (c < N) fo(r, c, C{(R)vr[j], (R)vi[j]});
          }
        }
      }
      tc::fence_before();
      __syncthreads();
    }
  }
}

}  // namespace tepai
