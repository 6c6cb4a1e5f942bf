// Per-sample MPS engine: one CTA evolves one TE-PAI circuit at a time.
//
// State of the CTA, in global memory (the CTA's arena slot, mostly L2-resident):
//   sites  n slots of 2*cap*cap complex, A_i[d_i][2][d_{i+1}] dense row-major
//   TH     4*cap*cap complex: theta' row-major, also QR panel / environments
//   XG     4*cap*cap complex: SVD working matrix when it does not fit in shared
//          memory, also the Q factor and temporaries
//   W3     16*cap*cap complex, only with three-site updates: theta3' of the
//          first split and its conjugate transpose
// State in shared memory: bond dims, step flags, sort keys, reductions, and
// either the whole SVD working matrix X (when it fits) or two staged column
// blocks of it.
// Every member function is called by all threads of the CTA with uniform
// arguments; they synchronise internally.
#pragma once
#include "gemm.cuh"
#include "common.cuh"

namespace tepai {

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of several scalars at once by a transposing butterfly: each xor
// level halves the number of values a lane carries (it keeps one half and
// sends the other to its partner), so 4 values take 2 + 1 shuffles and 8 take
// 4 + 2 + 1 before the last levels reduce the single survivor. Every lane ends
// with the totals, read from one lane each, so all lanes hold bit-identical
// sums and take the same branch on them.
template <typename R>
__device__ __forceinline__ void warp_sum4(R v[4], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8;
  R w[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const R send = b4 ? v[j] : v[j + 2], keep = b4 ? v[j + 2] : v[j];
    w[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  // w[j] carries value j + 2*b4
  R z;
  {
    const R send = b3 ? w[0] : w[1], keep = b3 ? w[1] : w[0];
    z = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  // z carries value b3 + 2*b4, summed over lanes that differ in bits 4 and 3
  z += __shfl_xor_sync(0xffffffffu, z, 4);
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = __shfl_sync(0xffffffffu, z, 8 * j);
}

template <typename R>
__device__ __forceinline__ void warp_sum8(R v[8], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  R w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const R send = b4 ? v[j] : v[j + 4], keep = b4 ? v[j + 4] : v[j];
    w[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  // w[j] carries value j + 4*b4
  R u[2];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const R send = b3 ? w[j] : w[j + 2], keep = b3 ? w[j + 2] : w[j];
    u[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  // u[j] carries value j + 2*b3 + 4*b4
  R z;
  {
    const R send = b2 ? u[0] : u[1], keep = b2 ? u[1] : u[0];
    z = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  // z carries value b2 + 2*b3 + 4*b4, summed over lanes that differ in bits 4..2
  z += __shfl_xor_sync(0xffffffffu, z, 2);
  z += __shfl_xor_sync(0xffffffffu, z, 1);
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __shfl_sync(0xffffffffu, z, 4 * j);
}

// Sum over the CTA; every thread gets the result. `red` holds >= 33 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double r = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    r = warp_sum(r);
    if (threadIdx.x == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }

// SVD tolerances and floors of one precision.
template <typename R> struct Prec;
template <> struct Prec<float>  { static constexpr double eps = 5.9604644775390625e-08; };
template <> struct Prec<double> { static constexpr double eps = 1.1102230246251565e-16; };

struct LocalStats {
  unsigned long long events = 0, gate_updates = 0, swap_updates = 0, qr_moves = 0, sweeps = 0,
                     not_converged = 0;
  int max_chi = 1;
  double max_discarded = 0.0, alg_flops = 0.0;
  unsigned long long cycles[PH_N] = {0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long jac_pairs = 0, jac_rots = 0;
  unsigned long long sub_cycles[SP_N] = {};
  unsigned long long reorth = 0;
  double tc_flops = 0.0;
  unsigned long long three_site = 0;
};

// Adds the SM cycles of a scope to one phase counter (thread 0 only).
struct SubTimer {
  LocalStats& st;
  int sp;
  long long t0 = 0;
  __device__ SubTimer(LocalStats& s, int p) : st(s), sp(p) {
#ifdef __CUDA_ARCH__
    if (threadIdx.x == 0) t0 = clock64();
#endif
  }
  __device__ void stop() {
#ifdef __CUDA_ARCH__
    if (threadIdx.x == 0 && sp >= 0) st.sub_cycles[sp] += (unsigned long long)(clock64() - t0);
#endif
    sp = -1;
  }
  __device__ ~SubTimer() { stop(); }
};

struct PhaseTimer {
  LocalStats& st;
  int ph;
  long long t0 = 0;
  __device__ PhaseTimer(LocalStats& s, int p) : st(s), ph(p) {
#ifdef __CUDA_ARCH__
    if (threadIdx.x == 0) t0 = clock64();
#endif
  }
  __device__ ~PhaseTimer() {
#ifdef __CUDA_ARCH__
    if (threadIdx.x == 0) st.cycles[ph] += (unsigned long long)(clock64() - t0);
#endif
  }
};

// Bulk copies between global and shared memory through the copy engine
// (cp.async.bulk, sm_90+): a load completes on an mbarrier with a byte count,
// a store completes as a bulk async-group. Addresses 16-byte aligned, sizes
// multiples of 16 bytes.
namespace bulk {
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(saddr(dst)), "l"(src), "r"(bytes), "r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ bool try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
__device__ __forceinline__ void store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(saddr(src)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void store_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
}  // namespace bulk

// Column handoff between the warps of one CTA: a shared-memory counter per
// column, written with release and read with acquire semantics (CTA scope).
namespace handoff {
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.b32 %0, [%1];" : "=r"(v) : "r"(bulk::saddr(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.cta.shared::cta.b32 [%0], %1;" ::"r"(bulk::saddr(p)), "r"(v) : "memory");
}
}  // namespace handoff

// Global load that bypasses L1: for data the bulk copy engine may have
// written behind L1's back (it also works for ordinary global data).
template <typename R>
__device__ __forceinline__ cplx<R> ldcg_c(const cplx<R>* p) {
  if constexpr (sizeof(R) == 4) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return cplx<R>{v.x, v.y};
  } else {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return cplx<R>{v.x, v.y};
  }
}

// Shared-memory scratch of the engine (fixed part); X follows when it fits.
struct SmemLayout {
  int* dims;          // [n+1]
  unsigned char* flags;  // [L]
  double* tnext;      // [L] next event time per term (N -> infinity sampler only)
  unsigned* tcnt;     // [L] events drawn per term (N -> infinity sampler only)
  double* red;        // [64]
  unsigned long long* mbar;  // mbarrier of the bulk copies
  double* wn;         // [2*cap] squared column norms
  int* perm;          // [2*cap]
  double* zval;       // [n]
  int* ibuf;          // [16]
  double* dbuf;       // [16]
  void* hh;           // Householder scalars: 3 arrays of [2*cap] complex<double>-sized slots
  void* x;            // SVD working matrix (optional)
};

// TC = true: the engine of the kernel that may hold TMEM, whose single-precision
// SVDs and products can run on the tensor cores. With TC = false no tcgen05
// code is compiled into the engine at all: a kernel that contains any
// tcgen05 instruction is limited to one CTA per SM.
template <typename R, bool TC = false>
struct Engine {
  using C = cplx<R>;
  static constexpr bool kTC = TC && sizeof(R) == 4;
  const KArgs& a;
  SmemLayout sm;
  C* site0;
  size_t slot;        // complex elements per site slot
  C* TH;
  C* XG;
  int cap;            // bond-dimension cap (chi_max)
  int centre;
  LocalStats st;
  // tensor cores: TMEM base address, the two stage mbarriers of tc_gemm and
  // the commits issued on each (uniform across the CTA); tc_ok once TMEM is held
  bool tc_ok = false;
  uint32_t tmem = 0;
  unsigned long long* tcbar = nullptr;
  uint32_t tc_cnt[2] = {0, 0};

  __device__ Engine(const KArgs& args, SmemLayout s, char* arena)
      : a(args), sm(s), cap(args.chi_cap), centre(0) {
    slot = (size_t)2 * cap * cap;
    site0 = reinterpret_cast<C*>(arena);
    TH = site0 + (size_t)a.n * slot;
    XG = TH + (size_t)4 * cap * cap;
  }

  __device__ __forceinline__ C* S(int i) const { return site0 + (size_t)i * slot; }
  // three-site buffers (arenas sized with KArgs::three_site): theta3' and its
  // conjugate transpose, 8 cap^2 complex values each, after XG
  __device__ __forceinline__ C* W3() const { return XG + (size_t)4 * cap * cap; }
  // Failure state of this CTA (sm.ibuf[15]); uniform across the CTA after a barrier.
  __device__ __forceinline__ bool failed() const { return sm.ibuf[15] != 0; }
  // Record a broken invariant. Called by every thread with uniform arguments.
  __device__ void fail(int code, int detail) {
    __syncthreads();
    if (tid() == 0) {
      if (atomicCAS(a.status, 0, code) == 0) { a.status[1] = detail; a.status[2] = (int)blockIdx.x; }
      sm.ibuf[15] = code;
    }
    __syncthreads();
  }
  __device__ bool dim_ok(int d) const { return d >= 1 && d <= cap; }
  // Bulk copies through the copy engine. A load is issued on one of three
  // completion slots (mbarriers; the phase of slot s is bit s of ibuf[13]) and
  // waited for later, so that it overlaps compute. Stores are issued by thread
  // 0 as bulk async-groups: bulk_wait_store_read() frees their shared-memory
  // sources, bulk_drain() waits until their writes are complete. A load must
  // not read global memory written by a store that has not been drained.
  // Every thread fences its own generic accesses before a copy is issued.
  __device__ void bulk_issue_load(int slot, void* dst, const void* src, uint32_t bytes) {
    bulk::fence_proxy();
    __syncthreads();
    if (tid() == 0) bulk::load(dst, src, bytes, sm.mbar + slot);
  }
  // Bounded wait for the load on `slot`: on timeout the CTA records
  // ST_COPY_TIMEOUT, waits once more (bounded) for the copy in flight, and the
  // caller sees failed().
  __device__ void bulk_wait_load(int slot, uint32_t bytes) {
    SubTimer sbt(st, SP_BULK);
    const uint32_t parity = (uint32_t)((sm.ibuf[13] >> slot) & 1);
    bool ok = false;
    for (int it = 0; it < (1 << 22) && !ok; ++it) ok = bulk::try_wait(sm.mbar + slot, parity);
    const int timed_out = __syncthreads_or(!ok);
    if (tid() == 0) sm.ibuf[13] ^= (1 << slot);
    if (timed_out) {
      bool again = false;
      for (int it = 0; it < (1 << 22) && !again; ++it) again = bulk::try_wait(sm.mbar + slot, parity);
      fail(ST_COPY_TIMEOUT, (int)bytes);
      return;
    }
    __syncthreads();
  }
  __device__ void bulk_issue_store(void* dst, const void* src, uint32_t bytes) {
    bulk::fence_proxy();
    __syncthreads();
    if (tid() == 0) bulk::store(dst, src, bytes);
  }
  __device__ void bulk_wait_store_read() {
    SubTimer sbt(st, SP_BULK);
    if (tid() == 0) bulk::store_wait_read();
    __syncthreads();
  }
  __device__ void bulk_drain() {
    SubTimer sbt(st, SP_BULK);
    if (tid() == 0) {
      bulk::store_wait();
      bulk::fence_proxy();
    }
    __syncthreads();
  }
  // After a failure: bounded waits for the loads still in flight on the slots
  // of `pend`, so that no copy lands in shared memory after the CTA has left.
  __device__ void bulk_settle(int pend) {
    for (int sl = 0; sl < 3; ++sl) {
      if (!(pend & (1 << sl))) continue;
      const uint32_t parity = (uint32_t)((sm.ibuf[13] >> sl) & 1);
      bool ok = false;
      for (int it = 0; it < (1 << 22) && !ok; ++it) ok = bulk::try_wait(sm.mbar + sl, parity);
      __syncthreads();
      if (tid() == 0) sm.ibuf[13] ^= (1 << sl);
      __syncthreads();
    }
  }
  // Synchronous forms: every thread returns after the data has landed.
  __device__ void bulk_load(void* dst, const void* src, uint32_t bytes) {
    bulk_issue_load(0, dst, src, bytes);
    bulk_wait_load(0, bytes);
  }
  __device__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    bulk_issue_store(dst, src, bytes);
    bulk_drain();
  }
  // Bounded wait until column counter *ver reaches r (every lane polls). A
  // wait that runs out (ibuf[7] polls; ibuf[8] is added to the target, 0
  // except in tests of this path) records ibuf[5] = 1 and returns; the pass
  // then finishes without further waits and the caller fails the sample.
  __device__ __forceinline__ void wait_col(const int* ver, int r) {
    for (int it = 0; handoff::ld_acquire(ver) < r + sm.ibuf[8]; ++it) {
      if (it >= sm.ibuf[7] || sm.ibuf[5]) { sm.ibuf[5] = 1; return; }
    }
  }
  __device__ __forceinline__ int tid() const { return threadIdx.x; }
  __device__ __forceinline__ int nt() const { return blockDim.x; }

  // state preparation
  __device__ void init_product();
  __device__ void init_from_tensors();
  __device__ void init_from_canonical();
  __device__ void export_state(double* out, int* dims);
  __device__ void normalise_centre();
  // single-site unitary u (2x2 row-major) on site i
  __device__ void apply_1site(int i, const C u[4]);
  // centre moves
  __device__ void move_centre(int target);
  __device__ void qr_right();
  __device__ void qr_left();
  __device__ void householder(C* Y, int m, int nq, C* Q, double tiny2);
  __device__ void ts_combine(C* Tm, C* Bm, int ld, int n, double tiny2);
  __device__ void householder_blocked(C* Y, int m, int nq, C* Q, double tiny2);
  __device__ void panel_t(const C* V, int m, int j0, int bp, C* T);
  __device__ void apply_block_reflector(const C* V, int m, int j0, int bp, const C* T, bool herm,
                                        C* G, int c0, int c1, C* CH, C* CH1, C* Wm);
  // QR of Y (global or shared): blocked when Y is in global memory, the
  // staging buffer holds a panel and a chunk, and the CTA has the 256 threads
  // the 16 x 16 block-reflector steps use
  __device__ void qr_factor(C* Y, int m, int nq, C* Q, double tiny2) {
    const C* xs = reinterpret_cast<const C*>(sm.x);
    const bool y_in_smem = Y >= xs && Y < xs + a.smem_x_elems;
    if (!y_in_smem && m >= 64 && nt() >= 256 && (size_t)m * 32 + 512 <= (size_t)a.smem_x_elems)
      householder_blocked(Y, m, nq, Q, tiny2);
    else
      householder(Y, m, nq, Q, tiny2);
  }
  // two-site update on bond (i, i+1) with gate g (basis |s_i s_{i+1}>); with
  // theta_in_th, theta' is already in TH and g is not read
  __device__ void two_site(int i, const C g[16], bool end_left, bool is_swap, bool theta_in_th = false);
  // gate g (basis |s_i s_{i+2}>) on positions i, i+2 as one three-site update
  __device__ void three_site(int i, const C g[16]);
  __device__ bool svd_truncate(C* Y, C*& X, int& ncx, bool& x_sh, bool pre, bool x_smem, int m, int nc, bool is_swap,
                               double flops_theta, bool factored = false, int y_ld = 0);
  __device__ void project_left(const C* Ai, int m, int k, const C* theta, int ncol, R renorm, C* out);
  __device__ void theta_from_th(int dl, int dr, bool end_left, bool zh, C* X);
  __device__ void form_theta(int i, const C g[16], bool end_left, bool zh, C* X);
  __device__ int jacobi(C* X, int m, int nc, bool x_in_smem);
  __device__ int jacobi_tc(C* X, int m, int nc, R tol, R thr);
  template <class STAGE>
  __device__ void tc_pipeline(int N, int nch, bool same, STAGE stage);
  template <class FA, class FB>
  __device__ void tc_gemm(int N, int K, bool same, FA fa, FB fb);
  template <class FA, class FB, class FO>
  __device__ void tc_cgemm(int M, int N, int K, FA fa, FB fb, FO fo);
  // a complex product goes to the tensor cores when the CTA holds TMEM and the
  // product is large enough to fill 128-row tiles (below that, block_gemm)
  __device__ bool tc_worth(int M, int N, int K) const {
    return kTC && tc_ok && (long long)M * N * K >= 64LL * 64 * 64;
  }
  __device__ bool tc_wait(int s);
  __device__ void reorth_pass_f64(C* X, int m, int nc, bool x_in_smem, double thr);
  __device__ void rr_pass(C* X, int m, int nc, R tol, R thr);
  __device__ void cross_pass(C* XA, int na, C* XB, int nb, int m, R tol, R thr);
  template <int RPL>
  __device__ void cross_pass_regs(C* XA, int na, C* XB, int nb, int m, R tol, R thr);
  // events
  __device__ void apply_event(int k, int v, int& sign_count);
  // measurement
  __device__ void measure_z(double* out_v);
  __device__ void measure_strings(double* out_v);
};

}  // namespace tepai
