// Block-wide complex matrix product through shared memory, for the dense
// contractions around the SVD and the centre moves (R times the neighbour
// site, U^H theta and theta V).
#pragma once
#include "common.cuh"

namespace tepai {

// Shared-memory elements block_gemm needs for a CTA of nt threads.
__host__ __device__ inline int gemm_tile_elems(int nt) { return 16 * 64 + 16 * 4 * (nt / 16); }

// out(i, j) = sum_k fa(i, k) fb(k, j) for 0 <= i < M, 0 <= j < N.
// The CTA walks output tiles of 64 x 4TX (TX = threads / 16) and stages
// 16-deep slices of both operands in `tile` (gemm_tile_elems complex). Thread
// (ty, tx) accumulates rows ty + 16 a and columns tx + TX b (a, b < 4) in
// registers: a warp then reads one broadcast row slice of A and contiguous
// elements of B, free of bank conflicts. The sum over k runs in increasing k
// for every output, as a plain loop would. fa / fb return one element and
// carry the operand's layout, conjugation and masking; fo(i, j, v) stores a
// result. Called by all threads of the CTA; tile must not alias the operands.
template <typename R, class FA, class FB, class FO>
__device__ __forceinline__ void block_gemm(int M, int N, int K, cplx<R>* tile, FA fa, FB fb, FO fo) {
  using C = cplx<R>;
  const int t = threadIdx.x, nt = blockDim.x;
  const int TX = nt / 16;
  const int tx = t % TX, ty = t / TX;
  const int NT = 4 * TX;
  C* As = tile;            // [16][64]
  C* Bs = tile + 16 * 64;  // [16][NT]
  for (int i0 = 0; i0 < M; i0 += 64) {
    for (int j0 = 0; j0 < N; j0 += NT) {
      C acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = C{0, 0};
      for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = t; e < 16 * 64; e += nt) {
          const int kk = e >> 6, ii = e & 63;
          const int i = i0 + ii, k = k0 + kk;
          As[e] = (i < M && k < K) ? fa(i, k) : C{0, 0};
        }
        for (int e = t; e < 16 * NT; e += nt) {
          const int kk = e / NT, jj = e - kk * NT;
          const int j = j0 + jj, k = k0 + kk;
          Bs[e] = (j < N && k < K) ? fb(k, j) : C{0, 0};
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
          C av[4], bv[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) av[a] = As[kk * 64 + ty + 16 * a];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = Bs[kk * NT + tx + TX * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) fma_c(acc[a][b], av[a], bv[b]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + ty + 16 * a, j = j0 + tx + TX * b;
          if (i < M && j < N) fo(i, j, acc[a][b]);
        }
    }
  }
}

}  // namespace tepai
