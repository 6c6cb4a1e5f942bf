// Sample initialisation, events, <Z_i> measurement and the persistent
// ensemble kernel (one CTA per sample at a time, samples pulled from an
// atomic work queue).
#pragma once
#include "qr.cuh"
#include "svd_update.cuh"
#include "tc_gemm.cuh"
#include "jacobi_tc.cuh"

namespace tepai {

template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::init_product() {
  for (int i = tid(); i <= a.n; i += nt()) sm.dims[i] = 1;
  // single-site codes 0 |0>, 1 |1>, 2 |+>, 3 |->, 4 |+i>, 5 |-i>
  const R r = (R)0.70710678118654752440;
  for (int i = tid(); i < a.n; i += nt()) {
    C* p = S(i);
    const int b = a.init_bits[i];
    if (b <= 1) {
      p[0] = C{b == 0 ? R(1) : R(0), 0};
      p[1] = C{b == 1 ? R(1) : R(0), 0};
    } else {
      p[0] = C{r, 0};
      p[1] = b == 2 ? C{r, 0} : b == 3 ? C{-r, 0} : b == 4 ? C{0, r} : C{0, -r};
    }
  }
  centre = 0;
  __syncthreads();
}

// Copy the shared initial tensors, bring them to right-canonical form with the
// centre on site 0 (LQ sweep from the right), and normalise the state. The
// centre is rescaled to unit norm after every step of the sweep: the norm of an
// unnormalised input grows geometrically along the chain and would overflow
// FP32 long before site 0.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::init_from_tensors() {
  for (int i = tid(); i <= a.n; i += nt()) sm.dims[i] = a.init_dims[i];
  __syncthreads();
  for (int i = 0; i <= a.n; ++i)
    if (!dim_ok(sm.dims[i]) || (i == 0 || i == a.n) && sm.dims[i] != 1) { fail(ST_BAD_DIM, 7000 + i); return; }
  size_t off = 0;
  for (int i = 0; i < a.n; ++i) {
    const int cnt = sm.dims[i] * 2 * sm.dims[i + 1];
    C* p = S(i);
    for (int e = tid(); e < cnt; e += nt())
      p[e] = C{(R)a.init_tensors[2 * (off + e)], (R)a.init_tensors[2 * (off + e) + 1]};
    off += cnt;
  }
  centre = a.n - 1;
  __syncthreads();
  normalise_centre();
  while (centre > 0 && !failed()) {
    qr_left();
    normalise_centre();
  }
}

// Start from the canonical form that canon_kernel left in a.canon: bond
// dimensions, centre and site tensors are copied (16-byte vectors; every site
// slot starts 16-byte aligned and holds a multiple of 16 bytes when the
// dimensions are even, else the tail is copied element-wise).
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::init_from_canonical() {
  for (int i = tid(); i <= a.n; i += nt()) sm.dims[i] = a.canon_meta[i];
  __syncthreads();
  for (int i = 0; i <= a.n; ++i)
    if (!dim_ok(sm.dims[i])) { fail(ST_BAD_DIM, 7500 + i); return; }
  const C* src0 = reinterpret_cast<const C*>(a.canon);
  for (int i = 0; i < a.n; ++i) {
    const size_t cnt = (size_t)sm.dims[i] * 2 * sm.dims[i + 1];
    const size_t bytes = cnt * sizeof(C);
    const float4* s4 = reinterpret_cast<const float4*>(src0 + (size_t)i * slot);
    float4* d4 = reinterpret_cast<float4*>(S(i));
    for (size_t e = tid(); e < bytes / 16; e += nt()) d4[e] = s4[e];
    if (bytes % 16 && tid() == 0) {
      const C* s = src0 + (size_t)i * slot;
      for (size_t e = (bytes / 16) * 16 / sizeof(C); e < cnt; ++e) S(i)[e] = s[e];
    }
  }
  centre = a.canon_meta[a.n + 1];
  if (centre < 0 || centre >= a.n) { fail(ST_BAD_DIM, 7600); return; }
  __syncthreads();
}

// Write the MPS (any gauge; normalised) to out in the start-state layout:
// site tensors A_p[d_p][2][d_{p+1}] concatenated over chain positions, complex
// interleaved in FP64; bond dimensions to dims[0..n].
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::export_state(double* out, int* dims) {
  for (int i = tid(); i <= a.n; i += nt()) dims[i] = sm.dims[i];
  size_t off = 0;
  for (int i = 0; i < a.n; ++i) {
    const size_t cnt = (size_t)sm.dims[i] * 2 * sm.dims[i + 1];
    const C* p = S(i);
    for (size_t e = tid(); e < cnt; e += nt()) {
      const C v = p[e];
      out[2 * (off + e)] = (double)v.re;
      out[2 * (off + e) + 1] = (double)v.im;
    }
    off += cnt;
  }
  __syncthreads();
}

// Rescale the centre tensor (and so the state) to unit norm.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::normalise_centre() {
  if (failed()) return;
  const int c = centre;
  const int cnt = sm.dims[c] * 2 * sm.dims[c + 1];
  C* p = S(c);
  double s2 = 0.0;
  for (int e = tid(); e < cnt; e += nt()) s2 += (double)abs2(p[e]);
  s2 = block_sum(s2, sm.red);
  if (!(s2 > 0.0 && s2 < 1.0e300)) { fail(ST_NONFINITE, 8000 + c); return; }
  const R inv = (R)(1.0 / sqrt(s2));
  for (int e = tid(); e < cnt; e += nt()) p[e] = scale(p[e], inv);
  __syncthreads();
}

template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::apply_1site(int i, const C u[4]) {
  PhaseTimer pt(st, PH_SINGLE);
  const int dl = sm.dims[i], dr = sm.dims[i + 1];
  C* p = S(i);
  for (int e = tid(); e < dl * dr; e += nt()) {
    const int aa = e / dr, bb = e - aa * dr;
    C* x0p = p + (size_t)(aa * 2) * dr + bb;
    C* x1p = x0p + dr;
    const C x0 = *x0p, x1 = *x1p;
    C y0 = {0, 0}, y1 = {0, 0};
    fma_c(y0, u[0], x0); fma_c(y0, u[1], x1);
    fma_c(y1, u[2], x0); fma_c(y1, u[3], x1);
    *x0p = y0; *x1p = y1;
  }
  __syncthreads();
}

template <typename R> __device__ __forceinline__ void pauli2(int p, cplx<R> u[4]) {
  if (p == 0) { u[0] = {0, 0}; u[1] = {1, 0}; u[2] = {1, 0}; u[3] = {0, 0}; }
  else if (p == 1) { u[0] = {0, 0}; u[1] = {0, -1}; u[2] = {0, 1}; u[3] = {0, 0}; }
  else { u[0] = {1, 0}; u[1] = {0, 0}; u[2] = {0, 0}; u[3] = {-1, 0}; }
}

// Event (j, k, v): v = 1 setting B, 2 setting C, 3 deterministic Trotter gate.
// Setting C is R_k(pi) = -i h_k, applied as the Pauli string h_k (the global
// phase drops out of every expectation value) and flips sign(g_l) (App. B).
// Sites are chain positions: a ring is stored in the folded order 0, n-1, 1,
// n-2, ..., so a bond term joins positions one or two apart. A gate two apart
// swaps the far site next to the near one, acts, and swaps it back; every swap
// is a truncated two-site update.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::apply_event(int k, int v, int& sign_count) {
  if (failed()) return;
  const TermDev& T = a.terms[k];
  if (tid() == 0) st.events++;
  if (v == 2) sign_count++;
  if (T.kind == 0) {
    C u[4];
    if (v == 2) pauli2<R>(2, u);
    else for (int q = 0; q < 4; ++q) u[q] = C{(R)T.g[2 * q], (R)T.g[2 * q + 1]};
    apply_1site(T.a, u);
    return;
  }
  if (v == 2) {
    C u[4];
    pauli2<R>(T.pauli, u);
    apply_1site(T.a, u);
    apply_1site(T.b, u);
    return;
  }
  C g[16];
  for (int q = 0; q < 16; ++q) g[q] = C{(R)T.g[2 * q], (R)T.g[2 * q + 1]};
  // sites are chain positions with T.a < T.b and the gate in basis |s_a s_b>
  if (T.b == T.a + 1) { two_site(T.a, g, false, false); return; }
  if (T.b != T.a + 2) { fail(ST_BAD_DIM, 10000 + k); return; }
  if (a.three_site) { three_site(T.a, g); return; }
  // two positions apart: bring the site at a+2 next to a, apply, move it back
  C sw[16];
  for (int q = 0; q < 16; ++q) sw[q] = C{0, 0};
  sw[0] = C{1, 0}; sw[6] = C{1, 0}; sw[9] = C{1, 0}; sw[15] = C{1, 0};
  two_site(T.a + 1, sw, true, true);
  two_site(T.a, g, false, false);
  two_site(T.a + 1, sw, false, true);
}

// <Z_p> / <psi|psi> for every chain position p. With the centre on site c, sites left of c
// are left-orthonormal and sites right of c are right-orthonormal, so a
// transfer-matrix sweep rightward from c (E <- sum_s A^s^H E A^s) gives
// <Z_i> for i >= c and a sweep leftward from c (F <- sum_s A^s F A^s^H) gives
// <Z_i> for i < c.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::measure_z(double* zout) {
  if (failed()) return;
  PhaseTimer pt(st, PH_MEASURE);
  const int n = a.n, c = centre;
  C* E = TH;
  C* Tm = TH + (size_t)cap * cap;
  double nrm = 1.0;
  // dense products through shared-memory tiles when the staging room holds one
  const bool use_gemm = a.smem_x_elems >= gemm_tile_elems(nt());
  C* tile = reinterpret_cast<C*>(sm.x);
  // rightward sweep
  {
    const int d = sm.dims[c];
    for (int e = tid(); e < d * d; e += nt()) E[e] = C{(e / d == e % d) ? R(1) : R(0), 0};
    __syncthreads();
    for (int i = c; i < n; ++i) {
      const int dl = sm.dims[i], dr = sm.dims[i + 1];
      const C* A = S(i);
      if (use_gemm) {
        // Tm^s[aa][bb] = sum_q E[aa][q] A[q][s][bb]: columns j = s dr + bb of A's rows
        block_gemm<R>(dl, 2 * dr, dl, tile,
            [=](int ii, int kk) { return E[(size_t)ii * dl + kk]; },
            [=](int kk, int jj) { return A[(size_t)kk * 2 * dr + jj]; },
            [=](int ii, int jj, C v) {
              const int s = jj >= dr, bb = jj - s * dr;
              Tm[(size_t)s * dl * dr + (size_t)ii * dr + bb] = v;
            });
      } else {
        for (int e = tid(); e < 2 * dl * dr; e += nt()) {
          const int s = e / (dl * dr), rem = e - s * dl * dr, aa = rem / dr, bb = rem - aa * dr;
          C acc = {0, 0};
          for (int q = 0; q < dl; ++q) fma_c(acc, E[(size_t)aa * dl + q], A[(size_t)(q * 2 + s) * dr + bb]);
          Tm[e] = acc;
        }
      }
      __syncthreads();
      double zp = 0.0, np_ = 0.0;
      for (int e = tid(); e < 2 * dl * dr; e += nt()) {
        const int s = e / (dl * dr), rem = e - s * dl * dr, aa = rem / dr, bb = rem - aa * dr;
        const C av = A[(size_t)(aa * 2 + s) * dr + bb];
        const double re = (double)av.re * (double)Tm[e].re + (double)av.im * (double)Tm[e].im;
        zp += s ? -re : re;
        np_ += re;
      }
      const double z = block_sum(zp, sm.red);
      const double nn = block_sum(np_, sm.red);
      if (i == c) nrm = nn;
      if (tid() == 0) sm.zval[i] = z;
      if (i + 1 < n) {
        if (use_gemm) {
          // E'[b1][b2] = sum_{s,q} conj(A[q][s][b1]) Tm^s[q][b2], k = s dl + q (E is not read here)
          block_gemm<R>(dr, dr, 2 * dl, tile,
              [=](int ii, int kk) {
                const int s = kk >= dl, q = kk - s * dl;
                const C u = A[(size_t)(q * 2 + s) * dr + ii];
                return C{u.re, -u.im};
              },
              [=](int kk, int jj) { return Tm[(size_t)kk * dr + jj]; },
              [=](int ii, int jj, C v) { E[(size_t)ii * dr + jj] = v; });
          __syncthreads();
        } else {
          for (int e = tid(); e < dr * dr; e += nt()) {
            const int b1 = e / dr, b2 = e - b1 * dr;
            C acc = {0, 0};
            for (int s = 0; s < 2; ++s)
              for (int q = 0; q < dl; ++q)
                fma_cc(acc, A[(size_t)(q * 2 + s) * dr + b1], Tm[(size_t)s * dl * dr + (size_t)q * dr + b2]);
            XG[e] = acc;
          }
          __syncthreads();
          for (int e = tid(); e < dr * dr; e += nt()) E[e] = XG[e];
          __syncthreads();
        }
      }
    }
  }
  // leftward sweep
  if (c > 0) {
    const int d = sm.dims[c + 1];
    for (int e = tid(); e < d * d; e += nt()) E[e] = C{(e / d == e % d) ? R(1) : R(0), 0};
    __syncthreads();
    for (int i = c; i >= 0; --i) {
      const int dl = sm.dims[i], dr = sm.dims[i + 1];
      const C* A = S(i);
      // U^s[a][b'] = sum_b A[a][s][b] F[b][b']
      if (use_gemm) {
        // rows i = 2 a + s of A times F
        block_gemm<R>(2 * dl, dr, dr, tile,
            [=](int ii, int kk) { return A[(size_t)ii * dr + kk]; },
            [=](int kk, int jj) { return E[(size_t)kk * dr + jj]; },
            [=](int ii, int jj, C v) { Tm[(size_t)(ii & 1) * dl * dr + (size_t)(ii >> 1) * dr + jj] = v; });
      } else {
        for (int e = tid(); e < 2 * dl * dr; e += nt()) {
          const int s = e / (dl * dr), rem = e - s * dl * dr, aa = rem / dr, bb = rem - aa * dr;
          C acc = {0, 0};
          const C* ar = A + (size_t)(aa * 2 + s) * dr;
          for (int q = 0; q < dr; ++q) fma_c(acc, ar[q], E[(size_t)q * dr + bb]);
          Tm[e] = acc;
        }
      }
      __syncthreads();
      if (i < c) {
        double zp = 0.0;
        for (int e = tid(); e < 2 * dl * dr; e += nt()) {
          const int s = e / (dl * dr), rem = e - s * dl * dr, aa = rem / dr, bb = rem - aa * dr;
          const C av = A[(size_t)(aa * 2 + s) * dr + bb];
          const double re = (double)av.re * (double)Tm[e].re + (double)av.im * (double)Tm[e].im;
          zp += s ? -re : re;
        }
        const double z = block_sum(zp, sm.red);
        if (tid() == 0) sm.zval[i] = z;
      }
      if (i == 0) break;
      // F'[a][a'] = sum_s sum_b' U^s[a][b'] conj(A[a'][s][b'])
      if (use_gemm) {
        // k = s dr + q (F is not read here)
        block_gemm<R>(dl, dl, 2 * dr, tile,
            [=](int ii, int kk) {
              const int s = kk >= dr, q = kk - s * dr;
              return Tm[(size_t)s * dl * dr + (size_t)ii * dr + q];
            },
            [=](int kk, int jj) {
              const int s = kk >= dr, q = kk - s * dr;
              const C u = A[(size_t)(jj * 2 + s) * dr + q];
              return C{u.re, -u.im};
            },
            [=](int ii, int jj, C v) { E[(size_t)ii * dl + jj] = v; });
        __syncthreads();
      } else {
        for (int e = tid(); e < dl * dl; e += nt()) {
          const int a1 = e / dl, a2 = e - a1 * dl;
          C acc = {0, 0};
          for (int s = 0; s < 2; ++s)
            for (int q = 0; q < dr; ++q)
              fma_cc(acc, A[(size_t)(a2 * 2 + s) * dr + q], Tm[(size_t)s * dl * dr + (size_t)a1 * dr + q]);
          XG[e] = acc;
        }
        __syncthreads();
        for (int e = tid(); e < dl * dl; e += nt()) E[e] = XG[e];
        __syncthreads();
      }
    }
  }
  __syncthreads();
  for (int o = tid(); o < a.n_obs; o += nt()) zout[o] = sm.zval[a.obs[o]] / nrm;
  __syncthreads();
}

// <P_o> / <psi|psi> for Pauli-string observables (a.obs_ops: codes 0 I, 1 X,
// 2 Y, 3 Z per chain position). With the centre on site c, sites left of c are
// left-orthonormal and sites right of c right-orthonormal, so the contraction
// only runs over chain positions lo = min(first, c) .. hi = max(last, c) of
// the string's support: E = I at bond lo, then per site
//   T^t[a][d] = sum_b E[a][b] A[b][t][d],  U^s = sum_t O[s][t] T^t,
//   E'[c][d]  = sum_{a,s} conj(A[a][s][c]) U^s[a][d],
// and <P> = Tr E at bond hi + 1, divided by |centre|^2.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::measure_strings(double* out) {
  if (failed()) return;
  PhaseTimer pt(st, PH_MEASURE);
  const int n = a.n, c = centre;
  C* E = TH;
  C* Tm = TH + (size_t)cap * cap;
  const bool use_gemm = a.smem_x_elems >= gemm_tile_elems(nt());
  C* tile = reinterpret_cast<C*>(sm.x);
  double nrm = 0.0;
  {
    const int cnt = sm.dims[c] * 2 * sm.dims[c + 1];
    const C* p = S(c);
    for (int e2 = tid(); e2 < cnt; e2 += nt()) nrm += (double)abs2(p[e2]);
    nrm = block_sum(nrm, sm.red);
  }
  for (int o = 0; o < a.n_obs; ++o) {
    const unsigned char* ops = a.obs_ops + (size_t)o * n;
    int first = n, last = -1;
    for (int p = 0; p < n; ++p)
      if (ops[p]) { if (first == n) first = p; last = p; }
    if (last < 0) {
      if (tid() == 0) out[o] = 1.0;
      continue;
    }
    const int lo = min(first, c), hi = max(last, c);
    {
      const int d = sm.dims[lo];
      for (int e2 = tid(); e2 < d * d; e2 += nt()) E[e2] = C{(e2 / d == e2 % d) ? R(1) : R(0), 0};
    }
    __syncthreads();
    for (int p = lo; p <= hi; ++p) {
      const int dl = sm.dims[p], dr = sm.dims[p + 1];
      const C* A = S(p);
      if (use_gemm) {
        block_gemm<R>(dl, 2 * dr, dl, tile,
            [=](int ii, int kk) { return E[(size_t)ii * dl + kk]; },
            [=](int kk, int jj) { return A[(size_t)kk * 2 * dr + jj]; },
            [=](int ii, int jj, C v) {
              const int s = jj >= dr, bb = jj - s * dr;
              Tm[(size_t)s * dl * dr + (size_t)ii * dr + bb] = v;
            });
      } else {
        for (int e2 = tid(); e2 < 2 * dl * dr; e2 += nt()) {
          const int s = e2 / (dl * dr), rem = e2 - s * dl * dr, aa = rem / dr, bb = rem - aa * dr;
          C acc = {0, 0};
          for (int q = 0; q < dl; ++q) fma_c(acc, E[(size_t)aa * dl + q], A[(size_t)(q * 2 + s) * dr + bb]);
          Tm[e2] = acc;
        }
      }
      __syncthreads();
      const int code = ops[p];
      if (code) {
        const size_t h = (size_t)dl * dr;
        for (size_t e2 = tid(); e2 < h; e2 += nt()) {
          const C t0 = Tm[e2], t1 = Tm[h + e2];
          C u0, u1;
          if (code == 1) { u0 = t1; u1 = t0; }                                      // X
          else if (code == 2) { u0 = C{t1.im, -t1.re}; u1 = C{-t0.im, t0.re}; }    // Y: -i t1, i t0
          else { u0 = t0; u1 = C{-t1.re, -t1.im}; }                                // Z
          Tm[e2] = u0;
          Tm[h + e2] = u1;
        }
        __syncthreads();
      }
      if (use_gemm) {
        block_gemm<R>(dr, dr, 2 * dl, tile,
            [=](int ii, int kk) {
              const int s = kk >= dl, q = kk - s * dl;
              const C u = A[(size_t)(q * 2 + s) * dr + ii];
              return C{u.re, -u.im};
            },
            [=](int kk, int jj) { return Tm[(size_t)kk * dr + jj]; },
            [=](int ii, int jj, C v) { E[(size_t)ii * dr + jj] = v; });
        __syncthreads();
      } else {
        for (int e2 = tid(); e2 < dr * dr; e2 += nt()) {
          const int b1 = e2 / dr, b2 = e2 - b1 * dr;
          C acc = {0, 0};
          for (int s = 0; s < 2; ++s)
            for (int q = 0; q < dl; ++q)
              fma_cc(acc, A[(size_t)(q * 2 + s) * dr + b1], Tm[(size_t)s * dl * dr + (size_t)q * dr + b2]);
          XG[e2] = acc;
        }
        __syncthreads();
        for (int e2 = tid(); e2 < dr * dr; e2 += nt()) E[e2] = XG[e2];
        __syncthreads();
      }
    }
    const int d = sm.dims[hi + 1];
    double tr = 0.0;
    for (int i = tid(); i < d; i += nt()) tr += (double)E[(size_t)i * d + i].re;
    tr = block_sum(tr, sm.red);
    if (tid() == 0) out[o] = tr / nrm;
    __syncthreads();
  }
}

// The TE-PAI sampler draw of gate (j, k) for global sample s: Philox4x64-10 with
// key (seed, s) and counter (j, k, 0, 0); word 0 against floor(q_k 2^64) decides
// "not A", word 1 against floor(r_k 2^64) decides C over B.
__device__ __forceinline__ int draw_gate(const KArgs& a, unsigned long long s, long long j, int k) {
  if (a.variant == 2) return 3;
  const u64x4 x = philox4x64_10(u64x4{(unsigned long long)j, (unsigned long long)k, 0ull, 0ull}, a.seed, s);
  const TermDev& T = a.terms[k];
  if (x.x0 < T.thr_event) return (x.x1 < T.thr_c) ? 2 : 1;
  return 0;
}

// The N -> infinity sampler: event i (from 0) of term k in global sample s
// comes a waiting time -ln(u) / lam_k after time t, with u = ((x0 >> 11) + 1)
// 2^-53 in (0, 1] from Philox4x64-10 counter (k, i, 1, 0) under key (seed, s);
// *ev is set to 2 (C) when x1 < floor(r_inf 2^64), else 1 (B). A term with
// lam_k = 0 never fires: its next time is +infinity.
__device__ __forceinline__ double clock_next(const KArgs& a, unsigned long long s, int k, unsigned i, double t,
                                             unsigned char* ev) {
  const TermDev& T = a.terms[k];
  if (!(T.lam > 0.0)) {
    *ev = 1;
    return __longlong_as_double(0x7ff0000000000000ll);
  }
  const u64x4 x = philox4x64_10(u64x4{(unsigned long long)k, (unsigned long long)i, 1ull, 0ull}, a.seed, s);
  const double u = ((double)(x.x0 >> 11) + 1.0) * 0x1p-53;
  *ev = x.x1 < T.thr_c ? 2 : 1;
  return t + (-log(u) / T.lam);
}

// Snapshot time t_m = t_run m / M (m from 1) of the N -> infinity sampler.
__device__ __forceinline__ double clock_snap_time(const KArgs& a, int m) {
  return a.t_run * (double)m / (double)a.M;
}

// The term whose next event comes first, ties to the lower index; L when no
// term fires. Called by all threads of the CTA, returns the same to all;
// red holds 2 x 32 doubles of scratch.
__device__ __forceinline__ int clock_argmin(const double* tn, int L, double* red) {
  const int t = threadIdx.x, nw = blockDim.x >> 5;
  double bt = __longlong_as_double(0x7ff0000000000000ll);
  int bk = L;
  for (int k = t; k < L; k += blockDim.x)
    if (tn[k] < bt) { bt = tn[k]; bk = k; }
#pragma unroll
  for (int off = 16; off; off >>= 1) {
    const double ot = __shfl_down_sync(0xffffffffu, bt, off);
    const int ok = __shfl_down_sync(0xffffffffu, bk, off);
    if (ot < bt || (ot == bt && ok < bk)) { bt = ot; bk = ok; }
  }
  if ((t & 31) == 0) { red[t >> 5] = bt; red[32 + (t >> 5)] = (double)bk; }
  __syncthreads();
  bt = red[0];
  bk = (int)red[32];
  for (int w = 1; w < nw; ++w) {
    const double ot = red[w];
    const int ok = (int)red[32 + w];
    if (ot < bt || (ot == bt && ok < bk)) { bt = ot; bk = ok; }
  }
  __syncthreads();
  return bk;
}

__host__ __device__ inline SmemLayout carve_smem(unsigned char* base, const KArgs& a, int csize) {
  SmemLayout s;
  size_t o = 0;
  s.dims = reinterpret_cast<int*>(base + o); o += align_up((size_t)(a.n + 1) * 4, 16);
  s.flags = base + o; o += align_up((size_t)a.L, 16);
  const int nclk = a.variant == 3 ? a.L : 0;
  s.tnext = reinterpret_cast<double*>(base + o); o += align_up((size_t)nclk * 8, 16);
  s.tcnt = reinterpret_cast<unsigned*>(base + o); o += align_up((size_t)nclk * 4, 16);
  s.red = reinterpret_cast<double*>(base + o); o += 64 * 8;
  s.mbar = reinterpret_cast<unsigned long long*>(base + o); o += 32;
  s.wn = reinterpret_cast<double*>(base + o); o += align_up((size_t)2 * a.chi_cap * 8, 16);
  s.perm = reinterpret_cast<int*>(base + o); o += align_up((size_t)2 * a.chi_cap * 4, 16);
  s.zval = reinterpret_cast<double*>(base + o); o += align_up((size_t)a.n * 8, 16);
  s.ibuf = reinterpret_cast<int*>(base + o); o += 16 * 4;
  s.dbuf = reinterpret_cast<double*>(base + o); o += 16 * 8;
  s.hh = base + o; o += align_up((size_t)3 * 2 * a.chi_cap * csize, 16);
  o = align_up(o, 128);
  s.x = base + o;
  return s;
}

// One sample of the N -> infinity sampler: the events of all terms merged in
// time order; snapshot m is taken once the next event lies beyond t_m.
template <typename R, bool TC>
__device__ __noinline__ void run_continuous(Engine<R, TC>& eng, const KArgs& a, const SmemLayout& sm, long long si,
                                            unsigned long long s) {
  int sign_count = 0;
  int mi = 0;
  {
    PhaseTimer pt(eng.st, PH_SAMPLER);
    for (int k = threadIdx.x; k < a.L; k += blockDim.x) {
      sm.tcnt[k] = 0;
      sm.tnext[k] = clock_next(a, s, k, 0u, 0.0, sm.flags + k);
    }
    __syncthreads();
  }
  while (true) {
    int k;
    {
      PhaseTimer pt(eng.st, PH_SAMPLER);
      k = clock_argmin(sm.tnext, a.L, sm.red);
    }
    const double tk = k < a.L ? sm.tnext[k] : __longlong_as_double(0x7ff0000000000000ll);
    while (mi < a.M && tk > clock_snap_time(a, mi + 1)) {
      if (a.obs_ops) eng.measure_strings(a.v + ((size_t)si * a.M + mi) * a.n_obs);
      else eng.measure_z(a.v + ((size_t)si * a.M + mi) * a.n_obs);
      if (threadIdx.x == 0) a.sign[(size_t)si * a.M + mi] = (sign_count & 1) ? -1 : 1;
      ++mi;
    }
    if (mi >= a.M) break;
    eng.apply_event(k, sm.flags[k], sign_count);
    __syncthreads();
    if (eng.failed()) break;
    if (threadIdx.x == 0) {
      const unsigned i = ++sm.tcnt[k];
      sm.tnext[k] = clock_next(a, s, k, i, sm.tnext[k], sm.flags + k);
    }
    __syncthreads();
  }
}

// TC selects the instantiation that may hold TMEM (single precision, the
// tensor-core launch shape). The instantiation without it contains no TMEM
// allocation, which the occupancy of the CUDA-core launch shapes depends on.
template <typename R, bool TC>
__global__ void __launch_bounds__(512, 1) ensemble_kernel(const __grid_constant__ KArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ long long s_next;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) unsigned long long s_tcbar[2];
  SmemLayout sm = carve_smem(smem_raw, a, (int)sizeof(cplx<R>));
  char* arena = a.arena + (size_t)blockIdx.x * a.arena_stride;
  Engine<R, TC> eng(a, sm, arena);
  // single precision with the tensor-core launch shape: hold TMEM for the
  // whole kernel (one warp allocates and, at the end, frees it)
  bool use_tc = false;
  if constexpr (TC && sizeof(R) == 4) use_tc = a.use_tc && blockDim.x >= 128;
  if constexpr (TC && sizeof(R) == 4) {
    if (use_tc && threadIdx.x < 32) { tc::alloc(&s_tmem, TcJac::TMEM_COLS); tc::relinquish(); }
  }
  if (threadIdx.x == 0) {
    sm.ibuf[13] = 0; sm.ibuf[14] = 0; sm.ibuf[15] = 0;
    sm.ibuf[7] = a.wait_limit > 0 ? a.wait_limit : (1 << 22);
    sm.ibuf[8] = a.wait_bias > 0 ? a.wait_bias : 0;
    for (int b = 0; b < 3; ++b) bulk::mbar_init(sm.mbar + b);
    if (use_tc) { bulk::mbar_init(s_tcbar); bulk::mbar_init(s_tcbar + 1); }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (use_tc) { eng.tc_ok = true; eng.tmem = s_tmem; eng.tcbar = s_tcbar; }
  while (!eng.failed()) {
    if (threadIdx.x == 0) {
      // queue slot -> sample: with an order, the costliest samples go first
      // (longest-processing-time-first), so the grid ends on short samples
      const long long q = (long long)atomicAdd(a.counter, 1ull);
      long long si = q;
      if (a.order && q < a.n_samples) {
        si = a.order[q];
        if (si < 0 || si >= a.n_samples) si = -1;
      }
      s_next = si;
    }
    __syncthreads();
    const long long si = s_next;
    __syncthreads();
    if (si < 0) {
      eng.fail(ST_BAD_ORDER, 0);
      break;
    }
    if (si >= a.n_samples) break;
    const unsigned long long s = (unsigned long long)(a.sample_offset + si);
    {
      PhaseTimer pt(eng.st, PH_INIT);
      if (a.canon) eng.init_from_canonical();
      else if (a.init_tensors) eng.init_from_tensors();
      else eng.init_product();
    }
    int sign_count = 0;
    int mi = 0;
    if (a.variant == 3) {
      run_continuous(eng, a, sm, si, s);
      if (a.state_out && si == 0 && !eng.failed()) eng.export_state(a.state_out, a.state_dims);
      continue;
    }
    for (long long j = 1; j <= a.run_steps; ++j) {
      {
        PhaseTimer pt(eng.st, PH_SAMPLER);
        for (int k = threadIdx.x; k < a.L; k += blockDim.x) sm.flags[k] = (unsigned char)draw_gate(a, s, j, k);
        __syncthreads();
      }
      for (int k = 0; k < a.L; ++k) {
        const int f = sm.flags[k];
        if (f) eng.apply_event(k, f, sign_count);
      }
      __syncthreads();
      if (eng.failed()) break;
      while (mi < a.M && a.snaps[mi] == j) {
        if (a.obs_ops) eng.measure_strings(a.v + ((size_t)si * a.M + mi) * a.n_obs);
        else eng.measure_z(a.v + ((size_t)si * a.M + mi) * a.n_obs);
        if (threadIdx.x == 0) a.sign[(size_t)si * a.M + mi] = (sign_count & 1) ? -1 : 1;
        ++mi;
      }
    }
    if (a.state_out && si == 0 && !eng.failed()) eng.export_state(a.state_out, a.state_dims);
  }
  if (threadIdx.x == 0) {
    const LocalStats& st = eng.st;
    atomicAdd(&a.stats->events, st.events);
    atomicAdd(&a.stats->gate_updates, st.gate_updates);
    atomicAdd(&a.stats->swap_updates, st.swap_updates);
    atomicAdd(&a.stats->qr_moves, st.qr_moves);
    atomicAdd(&a.stats->sweeps, st.sweeps);
    atomicAdd(&a.stats->not_converged, st.not_converged);
    atomicMax(&a.stats->max_chi, st.max_chi);
    atomicMax(reinterpret_cast<unsigned long long*>(&a.stats->max_discarded),
              (unsigned long long)__double_as_longlong(st.max_discarded));
    atomicAdd(&a.stats->alg_flops, st.alg_flops);
    for (int p = 0; p < PH_N; ++p) atomicAdd(&a.stats->cycles[p], st.cycles[p]);
    atomicAdd(&a.stats->jac_pairs, st.jac_pairs);
    atomicAdd(&a.stats->jac_rots, st.jac_rots);
    for (int p = 0; p < SP_N; ++p) atomicAdd(&a.stats->sub_cycles[p], st.sub_cycles[p]);
    atomicAdd(&a.stats->reorth, st.reorth);
    atomicAdd(&a.stats->tc_flops, st.tc_flops);
    atomicAdd(&a.stats->three_site, st.three_site);
  }
  if constexpr (TC && sizeof(R) == 4) {
    if (use_tc) {
      // no MMA may still be writing TMEM when it is freed: bounded waits for
      // the latest commit on each stage barrier (already complete unless a
      // wait timed out), then the allocating warp frees the columns
      for (int s = 0; s < 2; ++s) {
        if (eng.tc_cnt[s] == 0) continue;
        bool ok = false;
        for (int it = 0; it < (1 << 24) && !ok; ++it) ok = bulk::try_wait(s_tcbar + s, (eng.tc_cnt[s] - 1) & 1u);
      }
      tc::fence_before();
      __syncthreads();
      if (threadIdx.x < 32) tc::dealloc(eng.tmem, TcJac::TMEM_COLS);
    }
  }
}

// The canonical form of a shared start state, computed once per prepared
// problem by one CTA: the same steps as init_from_tensors in every sample
// (right-canonical, centre on site 0, unit norm), written to the arena slot
// a.canon with its bond dimensions and centre in a.canon_meta.
template <typename R>
__global__ void __launch_bounds__(512, 1) canon_kernel(const __grid_constant__ KArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemLayout sm = carve_smem(smem_raw, a, (int)sizeof(cplx<R>));
  Engine<R> eng(a, sm, const_cast<char*>(a.canon));
  if (threadIdx.x == 0) {
    sm.ibuf[13] = 0; sm.ibuf[14] = 0; sm.ibuf[15] = 0;
    sm.ibuf[7] = 1 << 22; sm.ibuf[8] = 0;
    for (int b = 0; b < 3; ++b) bulk::mbar_init(sm.mbar + b);
  }
  __syncthreads();
  eng.init_from_tensors();
  __syncthreads();
  if (threadIdx.x == 0 && !eng.failed()) {
    for (int i = 0; i <= a.n; ++i) a.canon_meta[i] = sm.dims[i];
    a.canon_meta[a.n + 1] = eng.centre;
  }
}

}  // namespace tepai
