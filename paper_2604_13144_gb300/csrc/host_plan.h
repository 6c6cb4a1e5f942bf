// Host planner of the CUDA path (FP64): term list, rotation angles, PAI
// coefficients, sampler thresholds, gate matrices and ||g(t_m)||_1.
// Follows App. A.3 (Eq. productFormula, Eq. settings, Eq. gammas), App. A.4
// (no-pi variant) and App. A.6 (Eq. overhead-bound).
#pragma once
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "../../include/tepai.h"
#include "common.cuh"

namespace tepai {

// Jacobi tolerance (scaled by sqrt(m) in the kernel, m = rows of the
// orthogonalised matrix), singular-value floor (values at or below
// floor_rel * s_0 are zero to working precision), sweep cap and complex
// element size per precision.
struct NumCfg { double tol, floor_rel; int max_sweeps; int csize; };
inline NumCfg num_cfg(int precision) {
  if (precision == TEPAI_FP64) return {2 * 1.1102230246251565e-16, 1e-14, 60, 16};
  return {2 * 5.9604644775390625e-08, 4e-6, 40, 8};
}

// Tie band at truncation cuts: the caller's tie_rel, else the paper's rule
// (only values equal to working precision, 1e-12 s_0, are tied).
inline double tie_band(const tepai_params* Q) { return Q->tie_rel > 0.0 ? Q->tie_rel : 1e-12; }

// QR preconditioning of the Jacobi SVD: on unless TEPAI_JACOBI_PRECONDITION=0
// (kept switchable for A/B timing of the two SVD variants).
inline int jacobi_precondition() {
  const char* e = std::getenv("TEPAI_JACOBI_PRECONDITION");
  return (e && e[0] == '0') ? 0 : 1;
}

// Fixed-capacity vector for plans that must not touch the heap.
template <typename T, size_t N>
struct FixedVec {
  T buf[N];
  size_t n = 0;
  bool overflow = false;
  void clear() { n = 0; overflow = false; }
  void push_back(const T& v) { if (n < N) buf[n++] = v; else overflow = true; }
  const T* data() const { return buf; }
  size_t size() const { return n; }
  bool empty() const { return n == 0; }
  const T& operator[](size_t i) const { return buf[i]; }
  T& operator[](size_t i) { return buf[i]; }
};

template <template <typename> class Vec>
struct PlanT {
  int n = 0, L = 0, M = 0, n_obs = 0, periodic = 0;
  long long N = 0, run_steps = 0;
  Vec<TermDev> terms;
  Vec<int> snaps;
  Vec<double> gnorm;
  Vec<int> obs;
  Vec<unsigned char> bits;
  Vec<unsigned char> obs_ops;   // Pauli-string observables: [n_obs][n] codes in chain order
  double gnorm_step = 1.0, expected_nu = 0.0;
  double t_run = 0.0;           // N -> infinity sampler: evolved time T run_steps / N
  void reset() {
    n = L = M = n_obs = periodic = 0; N = run_steps = 0; gnorm_step = 1.0; expected_nu = 0.0; t_run = 0.0;
    terms.clear(); snaps.clear(); gnorm.clear(); obs.clear(); bits.clear(); obs_ops.clear();
  }
  bool overflowed() const;
  void bits_set(int p, unsigned char v) { if ((size_t)p < bits.size()) bits[p] = v; }
  void ops_set(size_t p, unsigned char v) { if (p < obs_ops.size()) obs_ops[p] = v; }
};

template <typename T> using HeapVec = std::vector<T>;
using HostPlan = PlanT<HeapVec>;
template <> inline bool HostPlan::overflowed() const { return false; }

// Plan capacity without heap storage: n <= 1024 spins, M <= 4096 snapshots.
constexpr size_t kFixedMaxN = 1024, kFixedMaxM = 4096;
template <typename T> struct FixedCap { static constexpr size_t value = 4 * kFixedMaxN; };
template <> struct FixedCap<double> { static constexpr size_t value = kFixedMaxM; };
template <typename T> using FixedVecT = FixedVec<T, FixedCap<T>::value>;
using FixedPlan = PlanT<FixedVecT>;
template <> inline bool FixedPlan::overflowed() const {
  return terms.overflow || snaps.overflow || gnorm.overflow || obs.overflow || bits.overflow ||
         obs_ops.overflow;
}

inline bool finite_arr(const double* p, int n) {
  if (!p) return false;
  for (int i = 0; i < n; ++i) if (!std::isfinite(p[i])) return false;
  return true;
}

// floor(p * 2^64), saturated: a uniform 64-bit word x selects the event when
// x < threshold, so the event probability is threshold / 2^64.
inline unsigned long long threshold_u64(double p) {
  if (!(p > 0.0)) return 0ull;
  const double v = std::ldexp(p, 64);
  if (v >= 18446744073709551616.0) return ~0ull;
  return (unsigned long long)std::floor(v);
}

// Pauli rotation R(phi) = exp(-i phi P/2) = cos(phi/2) I - i sin(phi/2) P for a
// Pauli string P with P^2 = I, written into TermDev::g.
inline void rotation_gate(int pauli, bool two_site, double phi, double* g) {
  using cd = std::complex<double>;
  cd P1[2][2];
  if (pauli == 0) { P1[0][0] = 0; P1[0][1] = 1; P1[1][0] = 1; P1[1][1] = 0; }
  else if (pauli == 1) { P1[0][0] = 0; P1[0][1] = cd(0, -1); P1[1][0] = cd(0, 1); P1[1][1] = 0; }
  else { P1[0][0] = 1; P1[0][1] = 0; P1[1][0] = 0; P1[1][1] = -1; }
  const double c = std::cos(phi / 2), s = std::sin(phi / 2);
  const int d = two_site ? 4 : 2;
  for (int r = 0; r < d; ++r)
    for (int q = 0; q < d; ++q) {
      cd p;
      if (two_site) p = P1[r >> 1][q >> 1] * P1[r & 1][q & 1];
      else p = P1[r][q];
      const cd v = (r == q ? cd(c, 0) : cd(0, 0)) - cd(0, s) * p;
      g[2 * (r * d + q)] = v.real();
      g[2 * (r * d + q) + 1] = v.imag();
    }
}

// Chain position of ring site `site`: natural order for an open chain; for a
// ring the folded order 0, n-1, 1, n-2, 2, ... (every ring bond within chain
// distance 2, every cut crossing two ring bonds).
inline int chain_pos(int site, int n, bool periodic) {
  if (!periodic) return site;
  return site <= (n - 1) / 2 ? 2 * site : 2 * (n - 1 - site) + 1;
}

// The same gate in the basis |s_b s_a> instead of |s_a s_b>.
inline void swap_gate_basis(double* g) {
  double t[32];
  for (int r = 0; r < 4; ++r)
    for (int q = 0; q < 4; ++q) {
      const int rs = ((r & 1) << 1) | (r >> 1), qs = ((q & 1) << 1) | (q >> 1);
      t[2 * (r * 4 + q)] = g[2 * (rs * 4 + qs)];
      t[2 * (r * 4 + q) + 1] = g[2 * (rs * 4 + qs) + 1];
    }
  for (int e = 0; e < 32; ++e) g[e] = t[e];
}

template <class Plan>
inline int build_plan(const tepai_problem* P, const tepai_params* Q, Plan& hp) {
  if (!P || !Q) return TEPAI_ERR_INVALID_ARG;
  const int n = P->n;
  if (n < 2) return TEPAI_ERR_INVALID_ARG;
  const int nb = P->periodic ? n : n - 1;
  if (!finite_arr(P->Jx, nb) || !finite_arr(P->Jy, nb) || !finite_arr(P->Jz, nb) || !finite_arr(P->h, n))
    return TEPAI_ERR_INVALID_ARG;
  if (!P->init_bits) return TEPAI_ERR_INVALID_ARG;
  if (!(std::isfinite(Q->T) && Q->T >= 0.0) || Q->n_steps < 1) return TEPAI_ERR_INVALID_ARG;
  if (!(std::isfinite(Q->delta) && Q->delta > 0.0)) return TEPAI_ERR_INVALID_ARG;
  if (Q->chi_max < 1 || !(std::isfinite(Q->cutoff) && Q->cutoff >= 0.0)) return TEPAI_ERR_INVALID_ARG;
  if (!(std::isfinite(Q->tie_rel) && Q->tie_rel >= 0.0 && Q->tie_rel < 1.0)) return TEPAI_ERR_INVALID_ARG;
  if (Q->variant < 0 || Q->variant > 3 || Q->precision < 0 || Q->precision > 1) return TEPAI_ERR_INVALID_ARG;
  if (Q->variant == TEPAI_CONTINUOUS && !(Q->delta < M_PI)) return TEPAI_ERR_INVALID_ARG;
  if (Q->launch_variant < 0 || Q->launch_variant > 7) return TEPAI_ERR_INVALID_ARG;
  if (Q->three_site != 0 && Q->three_site != 1) return TEPAI_ERR_INVALID_ARG;
  if (Q->n_samples < 0 || Q->sample_offset < 0) return TEPAI_ERR_INVALID_ARG;
  const long long S = Q->run_steps ? Q->run_steps : Q->n_steps;
  if (S < 1 || S > Q->n_steps) return TEPAI_ERR_INVALID_ARG;
  if (Q->n_snapshots < 1 || S % Q->n_snapshots != 0) return TEPAI_ERR_INVALID_ARG;
  hp.reset();
  hp.n = n; hp.periodic = P->periodic ? 1 : 0; hp.N = Q->n_steps; hp.run_steps = S; hp.M = Q->n_snapshots;
  if (Q->obs_strings) {
    // observable o = Pauli string over physical sites, stored in chain order
    if (Q->n_obs < 1) return TEPAI_ERR_INVALID_ARG;
    for (int o = 0; o < Q->n_obs; ++o) {
      hp.obs.push_back(0);
      for (int p = 0; p < n; ++p) hp.obs_ops.push_back(0);
    }
    for (int o = 0; o < Q->n_obs; ++o)
      for (int i = 0; i < n; ++i) {
        const unsigned char code = Q->obs_strings[(size_t)o * n + i];
        if (code > 3) return TEPAI_ERR_INVALID_ARG;
        hp.ops_set((size_t)o * n + chain_pos(i, n, P->periodic), code);
      }
  } else if (Q->obs_sites) {
    if (Q->n_obs < 1) return TEPAI_ERR_INVALID_ARG;
    for (int o = 0; o < Q->n_obs; ++o) {
      if (Q->obs_sites[o] < 0 || Q->obs_sites[o] >= n) return TEPAI_ERR_INVALID_ARG;
      hp.obs.push_back(chain_pos(Q->obs_sites[o], n, P->periodic));
    }
  } else {
    for (int i = 0; i < n; ++i) hp.obs.push_back(chain_pos(i, n, P->periodic));
  }
  hp.n_obs = (int)hp.obs.size();
  // initial bits in chain order
  for (int p = 0; p < n; ++p) hp.bits.push_back(0);
  for (int i = 0; i < n; ++i) {
    if (P->init_bits[i] > 5) return TEPAI_ERR_INVALID_ARG;
    hp.bits_set(chain_pos(i, n, P->periodic), P->init_bits[i]);
  }
  // term list: Z_0..Z_{n-1}, then per bond b: XX_b, YY_b, ZZ_b
  struct T0 { int kind, a, b, pauli; double c; };
  hp.L = n + 3 * nb;
  const double delta = Q->delta;
  const bool cont = Q->variant == TEPAI_CONTINUOUS;
  // N -> infinity limit of the draw probabilities built from Eq. gammas: the
  // rate of "not A" per unit time is |c_k| (3 - cos Delta) / sin Delta, the
  // share of C among those events (1 - cos Delta) / (3 - cos Delta).
  const double rate = cont ? (3.0 - std::cos(delta)) / std::sin(delta) : 0.0;
  const double r_inf = cont ? (1.0 - std::cos(delta)) / (3.0 - std::cos(delta)) : 0.0;
  double sumq = 0.0, gstep = 1.0, c1 = 0.0, sumlam = 0.0;
  for (int k = 0; k < hp.L; ++k) {
    T0 t;
    if (k < n) {
      t = {0, k, k, 2, P->h[k]};
    } else {
      const int b = (k - n) / 3, p = (k - n) % 3;
      const double cc = p == 0 ? P->Jx[b] : (p == 1 ? P->Jy[b] : P->Jz[b]);
      t = {1, b, (b + 1) % n, p, cc};
    }
    TermDev td{};
    td.kind = t.kind; td.a = t.a; td.b = t.b; td.pauli = t.pauli;
    const double th = 2.0 * t.c * Q->T / (double)Q->n_steps;
    double q, r, gn, phi;
    td.lam = 0.0;
    if (cont) {
      q = 0.0; r = r_inf; gn = 1.0;
      phi = t.c != 0.0 ? std::copysign(delta, t.c) : delta;
      td.lam = std::fabs(t.c) * rate;
      c1 += std::fabs(t.c);
      sumlam += td.lam;
    } else if (Q->variant == TEPAI_TROTTER) {
      q = 1.0; r = 0.0; gn = 1.0; phi = th;
    } else {
      if (std::fabs(th) > delta || delta > M_PI) return TEPAI_ERR_THETA_EXCEEDS_DELTA;
      double g1, g2, g3;
      if (Q->variant == TEPAI_NO_PI) {
        const double lam = std::fabs(th) / delta;
        g1 = 1.0 - lam; g2 = lam; g3 = 0.0;
      } else {
        const double ta = std::fabs(th);
        g1 = std::cos(ta / 2) * std::sin(delta / 2 - ta / 2) / std::sin(delta / 2);
        g2 = std::sin(ta) / std::sin(delta);
        g3 = -std::sin(ta / 2) * std::sin(delta / 2 - ta / 2) / std::cos(delta / 2);
      }
      const double a1 = std::fabs(g1), a2 = std::fabs(g2), a3 = std::fabs(g3);
      gn = a1 + a2 + a3;
      const double nonid = a2 + a3;
      q = nonid / gn;
      r = nonid > 0.0 ? a3 / nonid : 0.0;
      phi = th != 0.0 ? std::copysign(delta, th) : delta;
    }
    td.thr_event = threshold_u64(q);
    td.thr_c = threshold_u64(r);
    rotation_gate(t.pauli, t.kind == 1, phi, td.g);
    // sites as chain positions; a bond gate in the basis |s_lower s_upper>
    td.a = chain_pos(t.a, n, P->periodic);
    td.b = chain_pos(t.b, n, P->periodic);
    if (t.kind == 1 && td.a > td.b) {
      const int tmp = td.a; td.a = td.b; td.b = tmp;
      swap_gate_basis(td.g);
    }
    hp.terms.push_back(td);
    sumq += q;
    gstep *= gn;
  }
  hp.gnorm_step = gstep;
  hp.expected_nu = (double)S * sumq;
  if (cont) {
    // snapshot m at t_m = t_run m / M, with ||g(t_m)||_1 of Eq. overhead
    hp.t_run = Q->T * (double)S / (double)Q->n_steps;
    hp.gnorm_step = 1.0;
    hp.expected_nu = sumlam * hp.t_run;
    // every sample runs about expected_nu events in one CTA: refuse problems
    // whose samples would not end in reasonable time
    if (!(hp.expected_nu <= 1e7)) return TEPAI_ERR_INVALID_ARG;
    for (int m = 1; m <= hp.M; ++m) {
      const double tm = hp.t_run * (double)m / (double)hp.M;
      hp.snaps.push_back(m);
      hp.gnorm.push_back(std::exp(2.0 * std::tan(delta / 2) * c1 * tm));
    }
    if (hp.overflowed()) return TEPAI_ERR_INVALID_ARG;
    return TEPAI_OK;
  }
  for (int m = 1; m <= hp.M; ++m) {
    const long long j = (long long)m * S / hp.M;
    hp.snaps.push_back((int)j);
    hp.gnorm.push_back(std::pow(gstep, (double)j));
  }
  if (hp.overflowed()) return TEPAI_ERR_INVALID_ARG;
  return TEPAI_OK;
}

// Launch shape of the ensemble kernel: threads per CTA, dynamic shared memory,
// where the SVD working matrix lives, and resident CTAs per SM (per_sm).
struct LaunchShape { int grid, block; size_t smem; int x_in_smem, x_elems, per_sm, use_tc; };

// Picks the shape for bond cap `cap` and complex size `csize` bytes. `occ`
// reports resident CTAs per SM of a (block, smem) pair. When the whole SVD
// working matrix (2cap x 2cap) fits in shared memory it stays there, with 512
// threads per CTA from cap 64, 128 up to cap 32 (a 64 x 64 SVD keeps few warps
// busy, and smaller CTAs put more samples on an SM: measured 16% faster at cap
// 32 in single precision, equal in double) and 256 between;
// otherwise it lives in global memory and column blocks are staged.
//   - Staged shapes first try two samples per SM (256 threads each,
//     staging room for a 16-column Householder panel and one 16-column update
//     chunk, which also holds two 16-column Jacobi blocks): two independent
//     CTAs fill each other's barrier, latency and copy-wait stalls, and the
//     modest staging leaves L1 room for the global operands. If two do not
//     fit, one 512-thread CTA per SM stages blocks within 128 KB.
// `variant` forces a shape. For a staged working matrix: 1 = two 256-thread
// CTAs per SM, 2 = one 512-thread CTA per SM (both with the CUDA-core Jacobi
// passes), 7 = the tensor-core shape (single precision, at most 256 rows:
// 256-thread CTAs whose staging room holds the tensor-core Jacobi's operand
// stage, Gram matrix and rotation, TcJac::BYTES; each CTA holds TMEM, and a
// kernel with tcgen05 code runs one CTA per SM, which makes this shape slower
// than the CUDA-core ones, so it is used only on request). When the working matrix fits in shared
// memory: 3, 4, 5, 6 = 64, 128, 256, 512 threads per CTA (smaller CTAs at small
// bond dimensions run several samples per SM). 0 (or a variant that does not
// apply) = the rule above.
template <class Occ>
inline cudaError_t choose_launch_shape(int n, int L, int n_clocks, int cap, int csize, int optin, Occ occ,
                                       LaunchShape& ls, int variant = 0) {
  const size_t fixed = smem_fixed_bytes(n, L, n_clocks, cap, csize);
  const size_t xbytes = (size_t)4 * cap * cap * csize;
  int per_sm = 1;
  cudaError_t e;
  ls.use_tc = 0;
  if (fixed + xbytes <= (size_t)optin) {
    ls.block = variant >= 3 && variant <= 6 ? (64 << (variant - 3)) : (cap >= 64 ? 512 : cap <= 32 ? 128 : 256);
    ls.x_in_smem = 1;
    ls.x_elems = 4 * cap * cap;
    ls.smem = fixed + xbytes;
    e = occ(ls.block, ls.smem, ls.use_tc, &per_sm);
  } else if (csize == 8 && 2 * cap <= 256 && variant == 7 &&
             fixed + align_up(TcJac::BYTES, 8) <= (size_t)optin) {
    ls.block = TcJac::THREADS;
    ls.x_in_smem = 0;
    ls.x_elems = (int)(align_up(TcJac::BYTES, 8) / 8);
    ls.smem = fixed + (size_t)ls.x_elems * 8;
    ls.use_tc = 1;
    e = occ(ls.block, ls.smem, ls.use_tc, &per_sm);
  } else {
    ls.block = 256;
    ls.x_in_smem = 0;
    ls.x_elems = 2 * cap * 32 + 512;
    ls.smem = fixed + (size_t)ls.x_elems * csize;
    e = ls.smem <= (size_t)optin ? occ(ls.block, ls.smem, ls.use_tc, &per_sm) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (ls.smem > (size_t)optin || (per_sm < 2 && variant != 1) || variant == 2) {
      int bw = 1;
      while ((size_t)2 * (2 * bw) * (2 * cap) * csize <= 131072 && 2 * bw < 2 * cap) bw *= 2;
      ls.block = 512;
      ls.x_elems = 2 * bw * 2 * cap;
      ls.smem = fixed + (size_t)ls.x_elems * csize;
      per_sm = 1;
      e = occ(ls.block, ls.smem, ls.use_tc, &per_sm);
    }
  }
  ls.per_sm = per_sm < 1 ? 1 : per_sm;
  return e;
}

}  // namespace tepai
