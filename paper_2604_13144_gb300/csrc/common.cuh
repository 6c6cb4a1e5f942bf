// Shared device/host definitions of the MPS TE-PAI CUDA path.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tepai {

// ---------------------------------------------------------------- complex
template <typename R> struct cplx { R re, im; };

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { return {a, b}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> add(cplx<R> a, cplx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> sub(cplx<R> a, cplx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> mul(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename R> __host__ __device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R> __host__ __device__ __forceinline__ cplx<R> scale(cplx<R> a, R s) { return {a.re * s, a.im * s}; }
template <typename R> __host__ __device__ __forceinline__ R abs2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <typename R> __host__ __device__ __forceinline__ void fma_c(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R> __host__ __device__ __forceinline__ void fma_cc(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}

// ---------------------------------------------------------------- Philox4x64-10
// Salmon et al., SC'11: ten rounds of two 64x64->128-bit products with Weyl
// key increments. Key = (seed, global sample index); counter = (j, k, 0, 0).
struct u64x4 { unsigned long long x0, x1, x2, x3; };

__device__ __forceinline__ u64x4 philox4x64_10(u64x4 c, unsigned long long k0, unsigned long long k1) {
  const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    unsigned long long hi0 = __umul64hi(M0, c.x0), lo0 = M0 * c.x0;
    unsigned long long hi1 = __umul64hi(M1, c.x2), lo1 = M1 * c.x2;
    c = u64x4{hi1 ^ c.x1 ^ k0, lo1, hi0 ^ c.x3 ^ k1, lo0};
  }
  return c;
}

// ---------------------------------------------------------------- tables
// One Hamiltonian term k, built by the host planner (FP64).
struct TermDev {
  int kind;       // 0 = single-site Z_a, 1 = bond term P_a P_b
  int a, b;       // sites acted on (b == a for kind 0)
  int pauli;      // 0 = X, 1 = Y, 2 = Z
  int pad;
  unsigned long long thr_event;  // gate (j,k) is not A when x0 < thr_event
  unsigned long long thr_c;      // ... and is C when x1 < thr_c
  double lam;     // N -> infinity sampler: rate of the term's events per unit time
  double g[32];   // gate of setting B (or the Trotter gate): 4x4 complex row-major,
                  // basis |s_a s_b>, (re,im) interleaved; kind 0 uses g[0..7] as 2x2.
};

// Phases timed with clock64 by thread 0 of every CTA (SM cycles, summed over CTAs).
enum : int { PH_INIT = 0, PH_SAMPLER, PH_SINGLE, PH_THETA, PH_JACOBI, PH_TRUNC, PH_QR, PH_MEASURE, PH_N };
// Sub-phases, nested inside the phases above (counted separately): Householder
// panel factorisation, trailing block-reflector updates, explicit Q, R times
// the neighbour site, SVD projection and write-back, waits on bulk copies,
// Jacobi passes, singular-value ranking and truncation bookkeeping.
// The last four split the tensor-core Jacobi: Gram GEMMs, assembly of the
// complex Gram matrix from TMEM, rotation rounds, block-update GEMMs and
// write-back.
enum : int { SP_QR_PANEL = 0, SP_QR_APPLY, SP_QR_FORMQ, SP_QR_RMUL, SP_PROJ, SP_BULK, SP_PASSES, SP_RANK,
             SP_TC_GRAM, SP_TC_ASSEMBLE, SP_TC_ROUNDS, SP_TC_UPDATE, SP_N };

struct DevStats {
  unsigned long long events, gate_updates, swap_updates, qr_moves, sweeps, not_converged;
  int max_chi, pad;
  double max_discarded;
  double alg_flops;
  unsigned long long cycles[PH_N];
  unsigned long long jac_pairs, jac_rots;  // Jacobi pair checks and rotations
  unsigned long long sub_cycles[SP_N];
  unsigned long long reorth;               // SVDs finished by the FP64 re-orthogonalisation pass
  double tc_flops;                         // flops of the tcgen05 MMAs issued (2 M N K each)
  unsigned long long three_site;           // bond-2 gates applied as three-site updates
};

struct KArgs {
  int n, L, M, n_obs, chi_cap, periodic, variant, max_sweeps;
  long long N, run_steps, n_samples, sample_offset;
  unsigned long long seed;
  double t_run;              // N -> infinity sampler: evolved time; snapshot m at t_run * m / M
  double cutoff, floor_rel, tol, gap_rel;
  const TermDev* terms;
  const int* snaps;          // [M] snapshot steps
  const int* obs;            // [n_obs]
  const int* init_dims;      // [n+1] or nullptr
  const char* canon;         // arena slot holding the start state in canonical form, or nullptr
  int* canon_meta;           // [n+2]: its bond dimensions, then its centre
  const unsigned char* obs_ops;  // [n_obs][n] Pauli codes in chain order, or nullptr (Z on obs)
  double* state_out;         // final MPS of the call's first sample (FP64, dims-packed), or nullptr
  int* state_dims;           // [n+1] its bond dimensions
  const double* init_tensors;// complex interleaved FP64, or nullptr
  const unsigned char* init_bits;  // [n]
  char* arena;               // per-CTA arena base
  size_t arena_stride;       // bytes per CTA
  double* v;                 // [n_samples][M][n_obs]
  signed char* sign;         // [n_samples][M]
  DevStats* stats;
  unsigned long long* counter;  // work-queue head
  const int* order;          // [n_samples] queue slot -> sample, costliest first; nullptr = identity
  int* cost;                 // [n_samples] predicted two-site updates per sample (when order is set)
  int x_in_smem;             // the SVD working matrix lives in shared memory
  int smem_x_elems;          // capacity of that buffer (complex elements)
  int* status;               // [4]: first failure (code, detail, sample, 0); 0 = ok
  int precondition;          // 1 = QR-preconditioned Jacobi where the shapes allow it
  int use_tc;                // 1 = tensor-core Jacobi where it applies (launch shape with its staging room)
  int wait_limit;            // spin iterations of a Jacobi column handoff wait before it gives up
  int wait_bias;             // added to every handoff target (0; tests set it so that no wait is met)
  int three_site;            // 1 = bond-2 gates as one three-site update (arena holds W3), 0 = swap routing
};

// Device status codes. A CTA that detects a broken invariant records the first
// failure, touches no more memory for that sample, and leaves the kernel.
enum : int { ST_OK = 0, ST_BAD_DIM = 1, ST_BAD_RANK = 2, ST_NONFINITE = 3, ST_COPY_TIMEOUT = 4, ST_HANDOFF_TIMEOUT = 5,
             ST_BAD_ORDER = 6, ST_MMA_TIMEOUT = 7 };

__host__ __device__ inline size_t align_up(size_t x, size_t al) { return (x + al - 1) / al * al; }

// Shared-memory plan of the tensor-core Jacobi inside the staging area (byte
// offsets): one operand stage (A hi, A lo, B hi, B lo of 128 rows x KT FP32),
// the 64 x 64 complex Gram matrix G (row stride GS) and the accumulated
// rotation V; TMEM columns held by the CTA. Sized so that two 256-thread CTAs
// share an SM.
struct TcJac {
  static constexpr int KT = 16;
  static constexpr int STAGES = 1;
  static constexpr int OP_FLOATS = 128 * KT;
  static constexpr size_t STAGE_BYTES = 4 * OP_FLOATS * 4;
  static constexpr int GS = 65;                 // row stride of G (complex): rows fall on distinct banks
  static constexpr size_t G_OFF = STAGES * STAGE_BYTES;
  static constexpr size_t V_OFF = G_OFF + 64 * GS * 8;
  static constexpr size_t BYTES = V_OFF + 64 * 64 * 8;
  static constexpr uint32_t TMEM_COLS = 128;
  static constexpr int THREADS = 256;
};

// Fixed shared-memory bytes of the engine for (n, L, cap, sizeof complex).
// n_clocks: terms with a Poisson clock (the N -> infinity sampler), else 0.
__host__ __device__ inline size_t smem_fixed_bytes(int n, int L, int n_clocks, int cap, int csize) {
  size_t b = 0;
  b += align_up((size_t)(n + 1) * 4, 16);          // dims
  b += align_up((size_t)L, 16);                     // flags
  b += align_up((size_t)n_clocks * 8, 16);          // next event time per term
  b += align_up((size_t)n_clocks * 4, 16);          // events drawn per term
  b += 64 * 8;                                      // red
  b += 32;                                          // mbarriers of the bulk copies (3 slots)
  b += align_up((size_t)2 * cap * 8, 16);           // wn
  b += align_up((size_t)2 * cap * 4, 16);           // perm
  b += align_up((size_t)n * 8, 16);                 // zval
  b += 16 * 4 + 16 * 8;                             // ibuf, dbuf
  b += align_up((size_t)3 * 2 * cap * csize, 16);   // Householder scalars
  return align_up(b, 128);
}

}  // namespace tepai
