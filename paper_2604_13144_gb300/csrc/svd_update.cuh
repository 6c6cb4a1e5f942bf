// Two-site update of the mixed-canonical MPS (Sec. II.A): theta contraction,
// Pauli-rotation gate, one-sided Jacobi SVD, truncation to chi_max / cutoff,
// renormalisation and write-back of the two site tensors.
#pragma once
#include "engine.cuh"

namespace tepai {

// theta'[(a,s),(t,b)] = sum_{s't'} g[st][s't'] sum_c A_i[a,s',c] A_{i+1}[c,t',b].
// TH receives theta' row-major (2dl x 2dr). X receives, column-major, the
// matrix Z whose left singular vectors become the orthonormal site: Z = theta'
// when the centre ends on the right site, Z = theta'^T when it ends on the
// left. With zh set, X receives Z^H instead (the input of the preconditioning
// QR): theta'^H (ld 2dr) or conj(theta') (ld 2dl).
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::form_theta(int i, const C g[16], bool end_left, bool zh, C* X) {
  const int dl = sm.dims[i], dc = sm.dims[i + 1], dr = sm.dims[i + 2];
  const C* A = S(i);
  const C* B = S(i + 1);
  const int m = 2 * dl, ncol = 2 * dr;
  // The shared-memory staging room is free before the SVD: when it holds a
  // GEMM tile, T[(a,s),(t,b)] = sum_c A_i[a,s,c] A_{i+1}[c,t,b] goes into TH
  // first (rows 2a+s, columns t dr + b: the natural layouts of both sites) and
  // the gate pass below reads it back in place.
  const bool use_gemm = a.smem_x_elems >= gemm_tile_elems(nt()) && X != TH;
  if (use_gemm) {
    C* thp = TH;
    auto fa = [=](int ii, int kk) { return A[(size_t)ii * dc + kk]; };
    auto fb = [=](int kk, int jj) { return B[(size_t)kk * ncol + jj]; };
    auto fo = [=](int ii, int jj, C v) { thp[(size_t)ii * ncol + jj] = v; };
    bool done = false;
    if constexpr (kTC) {
      if (tc_worth(m, ncol, dc)) { tc_cgemm(m, ncol, dc, fa, fb, fo); done = true; }
    }
    if (!done) block_gemm<R>(m, ncol, dc, reinterpret_cast<C*>(sm.x), fa, fb, fo);
    __syncthreads();
  }
  for (int e = tid(); e < dl * dr; e += nt()) {
    const int aa = e / dr, bb = e - aa * dr;
    C t[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    if (use_gemm) {
      // T[(a,s'),(t',b)] at row 2a+s', column t' dr + b; index s4 = 2 s' + t'
#pragma unroll
      for (int s4 = 0; s4 < 4; ++s4) t[s4] = TH[(size_t)(aa * 2 + (s4 >> 1)) * ncol + (s4 & 1) * dr + bb];
    } else {
      const C* a0p = A + (size_t)(aa * 2) * dc;
      const C* a1p = a0p + dc;
      for (int c = 0; c < dc; ++c) {
        const C a0 = a0p[c], a1 = a1p[c];
        const C b0 = B[(size_t)(c * 2) * dr + bb], b1 = B[(size_t)(c * 2 + 1) * dr + bb];
        fma_c(t[0], a0, b0); fma_c(t[1], a0, b1); fma_c(t[2], a1, b0); fma_c(t[3], a1, b1);
      }
    }
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4) {
      C o = {0, 0};
#pragma unroll
      for (int q = 0; q < 4; ++q) fma_c(o, g[s4 * 4 + q], t[q]);
      const int row = aa * 2 + (s4 >> 1), col = (s4 & 1) * dr + bb;
      TH[(size_t)row * ncol + col] = o;
      if (!zh) {
        if (end_left) X[(size_t)row * ncol + col] = o;
        else X[(size_t)col * m + row] = o;
      } else {
        const C oc = {o.re, -o.im};
        if (end_left) X[(size_t)col * m + row] = oc;
        else X[(size_t)row * ncol + col] = oc;
      }
    }
  }
  __syncthreads();
}

// Rotation parameters of a pair from its Gram entries (al = |x_p|^2,
// be = |x_q|^2, g = x_p^H x_q = gr + i gi). Returns false when no rotation is
// due; otherwise c, s and e^{-i phi} = (er, ei). The angle follows the
// classical Jacobi formulas: zeta = (be - al) / (2|g|), t = sign(zeta) /
// (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2), s = c t.
template <typename R>
__device__ __forceinline__ bool rot_params(R al, R be, R gr, R gi, R tol, R thr, R& c, R& s, R& er, R& ei) {
  if (al < thr || be < thr) return false;
  if constexpr (sizeof(R) == 4) {
    // Single precision: 1/|g| from one reciprocal square root serves the
    // rotation test, zeta and the phase, so the dependent chain between the
    // warp sums and the rotation holds no division and no square root. The
    // phase has unit modulus and c^2 + s^2 = 1 to rsqrt accuracy (a few ulp).
    // A zero or non-finite g gives NaN in the test and no rotation.
    // Below |g| ~ 1e-15 the squares approach the subnormal range, where they
    // keep few significant bits and the phase g / |g| would lose unit modulus
    // (a non-unitary rotation); g is then scaled by 2^60 before squaring.
    float h = fmaf(gr, gr, gi * gi);
    float ig, ag;
    if (h >= 1.0e-30f) {
      ig = rsqrtf(h);
      ag = h * ig;
    } else {
      const float S = 1152921504606846976.0f;  // 2^60
      const float grs = gr * S, gis = gi * S;
      h = fmaf(grs, grs, gis * gis);
      const float igs = rsqrtf(h);
      ig = igs * S;
      ag = (h * igs) * (1.0f / S);
    }
    const float cosv = ag * (rsqrtf(al) * rsqrtf(be));
    if (!(cosv > tol)) return false;
    const float zeta = 0.5f * (be - al) * ig;
    const float az = fabsf(zeta);
    float tt;
    if (az < 1.0e15f) {
      const float q = fmaf(az, az, 1.0f);
      tt = __fdividef(1.0f, az + q * rsqrtf(q));
    } else {
      tt = __fdividef(0.5f, az);
    }
    if (zeta < 0.0f) tt = -tt;
    c = rsqrtf(fmaf(tt, tt, 1.0f));
    s = c * tt;
    er = gr * ig;
    ei = -gi * ig;
    return true;
  } else {
    const R g = sqrt(gr * gr + gi * gi);
    if (!(g > tol * sqrt(al * be))) return false;
    const R zeta = (be - al) / (R(2) * g);
    const R az = fabs(zeta);
    R tt = az > R(1) ? R(1) / (az * (R(1) + sqrt(R(1) + R(1) / (az * az))))
                     : R(1) / (az + sqrt(R(1) + az * az));
    if (zeta < R(0)) tt = -tt;
    c = rsqrt_<R>(R(1) + tt * tt);
    s = c * tt;
    er = gr / g;
    ei = -gi / g;
    return true;
  }
}

// One Jacobi rotation of the column pair (xp, xq), by one warp: the pair is
// rotated when |x_p^H x_q| > tol |x_p||x_q| and neither column is below thr
// (zero to working precision). The complex rotation first removes the phase
// of x_p^H x_q from x_q, then applies the real Jacobi rotation that zeroes the
// off-diagonal of the 2x2 Gram matrix. Each lane keeps its RPL rows of both
// columns in registers between the inner products and the rotation
// (m <= 32 * RPL). Returns true (warp-uniform) if rotated.
template <typename R, int RPL>
__device__ __forceinline__ bool rotate_pair(cplx<R>* xp, cplx<R>* xq, int m, R tol, R thr, int lane) {
  using C = cplx<R>;
  C u[RPL], v[RPL];
  R al = 0, be = 0, gr = 0, gi = 0;
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    if (row < m) { u[t] = xp[row]; v[t] = xq[row]; }
    else { u[t] = C{0, 0}; v[t] = C{0, 0}; }
    al = fma(u[t].re, u[t].re, fma(u[t].im, u[t].im, al));
    be = fma(v[t].re, v[t].re, fma(v[t].im, v[t].im, be));
    gr = fma(u[t].re, v[t].re, fma(u[t].im, v[t].im, gr));
    gi = fma(u[t].re, v[t].im, fma(-u[t].im, v[t].re, gi));
  }
  {
    R v4[4] = {al, be, gr, gi};
    warp_sum4<R>(v4, lane);
    al = v4[0]; be = v4[1]; gr = v4[2]; gi = v4[3];
  }
  R c, s, er, ei;
  if (!rot_params<R>(al, be, gr, gi, tol, thr, c, s, er, ei)) return false;
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    const C w = {er * v[t].re - ei * v[t].im, er * v[t].im + ei * v[t].re};
    if (row < m) {
      xp[row] = C{c * u[t].re - s * w.re, c * u[t].im - s * w.im};
      xq[row] = C{s * u[t].re + c * w.re, s * u[t].im + c * w.im};
    }
  }
  return true;
}

template <typename R>
__device__ __forceinline__ bool rotate_pair_m(cplx<R>* xp, cplx<R>* xq, int m, R tol, R thr, int lane) {
  if (m <= 64) return rotate_pair<R, 2>(xp, xq, m, tol, thr, lane);
  if (m <= 128) return rotate_pair<R, 4>(xp, xq, m, tol, thr, lane);
  if (m <= 256) return rotate_pair<R, 8>(xp, xq, m, tol, thr, lane);
  return rotate_pair<R, 16>(xp, xq, m, tol, thr, lane);
}

// Single-precision round-robin pass with two slots per warp processed together
// (slots w and w + nw of every round): the four columns are loaded, the eight
// Gram sums share one warp reduction, and both rotations run before the
// columns are stored and released. Same schedule, handoff and rotation rule as
// Engine::rr_pass; FULL drops the row bounds when m = 32 RPL.
template <int RPL, bool FULL>
__device__ __noinline__ void rr_pass_f32(float2* X, int m, int nc, float tol, float thr, int* ver, int* ibuf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int np = nc + (nc & 1), half = np / 2;
  for (int c = threadIdx.x; c < np; c += blockDim.x) ver[c] = 0;
  __syncthreads();
  const int t0 = w, t1 = w + nw;
  const bool o0 = t0 < half, o1 = t1 < half;
  const float2 zero = make_float2(0.f, 0.f);
  auto wait = [&](const int* vp, int need) {
    for (int it = 0; handoff::ld_acquire(vp) < need + ibuf[8]; ++it) {
      if (it >= ibuf[7] || ibuf[5]) { ibuf[5] = 1; return; }
    }
  };
  auto slot = [&](int t, int r, int& p, int& q) {
    if (t == 0) { p = np - 1; q = r; }
    else { p = (r + t) % (np - 1); q = (r - t + np - 1) % (np - 1); }
  };
  int rot = 0, chk = 0;
  for (int r = 0; r < np - 1 && o0; ++r) {
    int p0, q0, p1 = 0, q1 = 0;
    slot(t0, r, p0, q0);
    if (o1) slot(t1, r, p1, q1);
    wait(ver + p0, r);
    wait(ver + q0, r);
    if (o1) { wait(ver + p1, r); wait(ver + q1, r); }
    const bool d0 = p0 < nc && q0 < nc, d1 = o1 && p1 < nc && q1 < nc;
    chk += (int)d0 + (int)d1;
    float2* xp0 = X + (size_t)p0 * m;
    float2* xq0 = X + (size_t)q0 * m;
    float2* xp1 = X + (size_t)p1 * m;
    float2* xq1 = X + (size_t)q1 * m;
    float2 u0[RPL], v0[RPL], u1[RPL], v1[RPL];
    float al0 = 0, be0 = 0, gr0 = 0, gi0 = 0, al1 = 0, be1 = 0, gr1 = 0, gi1 = 0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      const bool in = FULL || row < m;
      u0[t] = (d0 && in) ? xp0[row] : zero;
      v0[t] = (d0 && in) ? xq0[row] : zero;
      u1[t] = (d1 && in) ? xp1[row] : zero;
      v1[t] = (d1 && in) ? xq1[row] : zero;
      al0 = fmaf(u0[t].x, u0[t].x, fmaf(u0[t].y, u0[t].y, al0));
      be0 = fmaf(v0[t].x, v0[t].x, fmaf(v0[t].y, v0[t].y, be0));
      gr0 = fmaf(u0[t].x, v0[t].x, fmaf(u0[t].y, v0[t].y, gr0));
      gi0 = fmaf(u0[t].x, v0[t].y, fmaf(-u0[t].y, v0[t].x, gi0));
      al1 = fmaf(u1[t].x, u1[t].x, fmaf(u1[t].y, u1[t].y, al1));
      be1 = fmaf(v1[t].x, v1[t].x, fmaf(v1[t].y, v1[t].y, be1));
      gr1 = fmaf(u1[t].x, v1[t].x, fmaf(u1[t].y, v1[t].y, gr1));
      gi1 = fmaf(u1[t].x, v1[t].y, fmaf(-u1[t].y, v1[t].x, gi1));
    }
    float v8[8] = {al0, be0, gr0, gi0, al1, be1, gr1, gi1};
    warp_sum8<float>(v8, lane);
    float c0, s0, er0, ei0, c1, s1, er1, ei1;
    const bool r0 = d0 && rot_params<float>(v8[0], v8[1], v8[2], v8[3], tol, thr, c0, s0, er0, ei0);
    const bool r1 = d1 && rot_params<float>(v8[4], v8[5], v8[6], v8[7], tol, thr, c1, s1, er1, ei1);
    if (r0) {
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        if (!(FULL || row < m)) continue;
        const float2 vv = v0[t], u = u0[t];
        const float wx = er0 * vv.x - ei0 * vv.y, wy = er0 * vv.y + ei0 * vv.x;
        xp0[row] = make_float2(c0 * u.x - s0 * wx, c0 * u.y - s0 * wy);
        xq0[row] = make_float2(s0 * u.x + c0 * wx, s0 * u.y + c0 * wy);
      }
      ++rot;
    }
    if (r1) {
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        if (!(FULL || row < m)) continue;
        const float2 vv = v1[t], u = u1[t];
        const float wx = er1 * vv.x - ei1 * vv.y, wy = er1 * vv.y + ei1 * vv.x;
        xp1[row] = make_float2(c1 * u.x - s1 * wx, c1 * u.y - s1 * wy);
        xq1[row] = make_float2(s1 * u.x + c1 * wx, s1 * u.y + c1 * wy);
      }
      ++rot;
    }
    __syncwarp();
    if (lane == 0) {
      handoff::st_release(ver + p0, r + 1);
      handoff::st_release(ver + q0, r + 1);
      if (o1) { handoff::st_release(ver + p1, r + 1); handoff::st_release(ver + q1, r + 1); }
    }
  }
  if (lane == 0) { if (rot) atomicAdd(&ibuf[0], rot); if (chk) atomicAdd(&ibuf[6], chk); }
  __syncthreads();
}

// One cyclic pass over all pairs of the nc columns of X (m rows, column-major)
// in parallel round-robin order (Brent & Luk, SIAM J. Sci. Stat. Comput. 6,
// 1985): np-1 rounds of disjoint pairs (np = nc rounded up to even), slot t
// of every round owned by warp t mod nw. Rounds are not separated by CTA
// barriers: every column is touched by exactly one slot per round, and a slot
// waits only until both of its columns have finished the previous round
// (counter ver[c] = rounds completed on column c, in sm.perm). Warps therefore
// drift apart and overlap their latency-bound phases, while every pair sees
// exactly the column values of the barrier-separated schedule. Rotations are
// counted in ibuf[0].
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::rr_pass(C* X, int m, int nc, R tol, R thr) {
  if constexpr (sizeof(R) == 4) if (m <= 256 && nc + (nc & 1) <= 2 * cap) {
    float2* xf = reinterpret_cast<float2*>(X);
    if (m <= 64) { if (m == 64) rr_pass_f32<2, true>(xf, m, nc, tol, thr, sm.perm, sm.ibuf);
                   else rr_pass_f32<2, false>(xf, m, nc, tol, thr, sm.perm, sm.ibuf); }
    else if (m <= 128) { if (m == 128) rr_pass_f32<4, true>(xf, m, nc, tol, thr, sm.perm, sm.ibuf);
                         else rr_pass_f32<4, false>(xf, m, nc, tol, thr, sm.perm, sm.ibuf); }
    else { if (m == 256) rr_pass_f32<8, true>(xf, m, nc, tol, thr, sm.perm, sm.ibuf);
           else rr_pass_f32<8, false>(xf, m, nc, tol, thr, sm.perm, sm.ibuf); }
    return;
  }
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int np = nc + (nc & 1);
  int* ver = sm.perm;
  for (int c = tid(); c < np; c += nt()) ver[c] = 0;
  __syncthreads();
  int rot = 0, chk = 0;
  for (int r = 0; r < np - 1; ++r) {
    for (int t = w; t < np / 2; t += nw) {
      int p, q;
      if (t == 0) { p = np - 1; q = r; }
      else { p = (r + t) % (np - 1); q = (r - t + np - 1) % (np - 1); }
      wait_col(ver + p, r);
      wait_col(ver + q, r);
      if (p < nc && q < nc) {
        ++chk;
        if (rotate_pair_m<R>(X + (size_t)p * m, X + (size_t)q * m, m, tol, thr, lane)) ++rot;
      }
      __syncwarp();
      if (lane == 0) {
        handoff::st_release(ver + p, r + 1);
        handoff::st_release(ver + q, r + 1);
      }
    }
  }
  if (lane == 0) { if (rot) atomicAdd(&sm.ibuf[0], rot); if (chk) atomicAdd(&sm.ibuf[6], chk); }
  __syncthreads();
}

// All pairs (p in block A, q in block B): round r pairs p with (p + r) mod nmax.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::cross_pass(C* XA, int na, C* XB, int nb, int m, R tol, R thr) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int nmax = max(na, nb);
  for (int r = 0; r < nmax; ++r) {
    for (int p = w; p < nmax; p += nw) {
      const int q = (p + r) % nmax;
      if (p >= na || q >= nb) continue;
      if (lane == 0) atomicAdd(&sm.ibuf[6], 1);
      if (rotate_pair_m<R>(XA + (size_t)p * m, XB + (size_t)q * m, m, tol, thr, lane) && lane == 0)
        atomicAdd(&sm.ibuf[0], 1);
    }
    __syncthreads();
  }
}

// Load of the SVD working matrix after the Jacobi: from global memory it
// bypasses L1 (the bulk copy engine wrote it to L2 behind L1's back).
template <typename R>
__device__ __forceinline__ cplx<R> ld_x(const cplx<R>* p, bool in_smem) {
  if (in_smem) return *p;
  if constexpr (sizeof(R) == 4) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return cplx<R>{v.x, v.y};
  } else {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return cplx<R>{v.x, v.y};
  }
}

// Single-precision cross pass: warp w holds A columns p0 = w and p1 = w + nw in
// registers for the whole pass and, in round r, takes one B column
// q = (w + r) mod nbp (nbp = max(nb, warps)). The column is loaded once and
// meets both A columns in turn: pair (p0, q) first, then (p1, q') with q' the
// column after the first rotation. The Gram entries of the second pair follow
// from those of the first without touching the data again:
//   |q'|^2 = s^2 |a0|^2 + c^2 |q|^2 + 2 s c |a0^H q|,
//   a1^H q' = s a1^H a0 + c e^{-i phi} a1^H q,
// which costs one extra inner product (a1^H a0) per round. When the first pair
// does not rotate, q' = q and the second pair uses the exact inner products, so
// a sweep that rotates nothing (the convergence test) decides on exact values.
// Every (A, B) pair is met once per pass. Column q's previous user is warp
// w + 1 one round earlier, or, for the last warp, warp 0 nbp - nw + 1 rounds
// earlier: a warp waits (acquire) until that round has released the column.
// FULL drops the row bounds when m = 32 RPL.
template <int RPL, bool FULL>
__device__ __noinline__ void cross_pass_f32(float2* XA, int na, float2* XB, int nb, int m, float tol, float thr,
                                            int* ver, int* ibuf) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nbp = max(nb, nw);
  for (int c = threadIdx.x; c < nbp; c += blockDim.x) ver[c] = 0;
  __syncthreads();
  const int p0 = w, p1 = w + nw;
  const bool h0 = p0 < na, h1 = p1 < na;
  const float2 zero = make_float2(0.f, 0.f);
  float2 a0[RPL], a1[RPL], qv[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    const bool in = FULL || row < m;
    a0[t] = (h0 && in) ? XA[(size_t)p0 * m + row] : zero;
    a1[t] = (h1 && in) ? XA[(size_t)p1 * m + row] : zero;
  }
  auto wait = [&](const int* vp, int need) {
    for (int it = 0; handoff::ld_acquire(vp) < need + ibuf[8]; ++it) {
      if (it >= ibuf[7] || ibuf[5]) { ibuf[5] = 1; return; }
    }
  };
  const int gap = nbp - nw;
  int rot = 0, chk = 0;
  int q = w;
  for (int r = 0; r < nbp; ++r) {
    const int prev = (w + 1 < nw) ? r - 1 : r - 1 - gap;
    if (prev >= 0) wait(ver + q, prev + 1);
    const bool dq = q < nb;
    chk += (int)(dq && h0) + (int)(dq && h1);
    float2* xq = XB + (size_t)q * m;
    float al0 = 0, al1 = 0, be = 0, gr0 = 0, gi0 = 0, gr1 = 0, gi1 = 0, cr = 0, ci = 0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      qv[t] = (dq && (FULL || row < m)) ? xq[row] : zero;
      const float2 u0 = a0[t], u1 = a1[t], vv = qv[t];
      al0 = fmaf(u0.x, u0.x, fmaf(u0.y, u0.y, al0));
      al1 = fmaf(u1.x, u1.x, fmaf(u1.y, u1.y, al1));
      be = fmaf(vv.x, vv.x, fmaf(vv.y, vv.y, be));
      gr0 = fmaf(u0.x, vv.x, fmaf(u0.y, vv.y, gr0));
      gi0 = fmaf(u0.x, vv.y, fmaf(-u0.y, vv.x, gi0));
      gr1 = fmaf(u1.x, vv.x, fmaf(u1.y, vv.y, gr1));
      gi1 = fmaf(u1.x, vv.y, fmaf(-u1.y, vv.x, gi1));
      cr = fmaf(u1.x, u0.x, fmaf(u1.y, u0.y, cr));
      ci = fmaf(u1.x, u0.y, fmaf(-u1.y, u0.x, ci));
    }
    float v8[8] = {al0, al1, be, gr0, gi0, gr1, gi1, cr};
    warp_sum8<float>(v8, lane);
    ci = warp_sum(ci);
    al0 = v8[0]; al1 = v8[1]; be = v8[2]; gr0 = v8[3]; gi0 = v8[4]; gr1 = v8[5]; gi1 = v8[6]; cr = v8[7];
    float c0, s0, er0, ei0, c1, s1, er1, ei1;
    const bool r0 = dq && h0 && rot_params<float>(al0, be, gr0, gi0, tol, thr, c0, s0, er0, ei0);
    if (r0) {
      const float g0 = sqrtf(fmaf(gr0, gr0, gi0 * gi0));
      const float ngr = s0 * cr + c0 * (er0 * gr1 - ei0 * gi1);
      const float ngi = s0 * ci + c0 * (er0 * gi1 + ei0 * gr1);
      be = s0 * s0 * al0 + c0 * c0 * be + 2.f * s0 * c0 * g0;
      gr1 = ngr;
      gi1 = ngi;
      // w = e^{-i phi} q; a0 <- c a0 - s w; q <- s a0 + c w
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const float2 vv = qv[t], u = a0[t];
        const float wx = er0 * vv.x - ei0 * vv.y, wy = er0 * vv.y + ei0 * vv.x;
        a0[t] = make_float2(c0 * u.x - s0 * wx, c0 * u.y - s0 * wy);
        qv[t] = make_float2(s0 * u.x + c0 * wx, s0 * u.y + c0 * wy);
      }
      ++rot;
    }
    const bool r1 = dq && h1 && rot_params<float>(al1, be, gr1, gi1, tol, thr, c1, s1, er1, ei1);
    if (r1) {
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const float2 vv = qv[t], u = a1[t];
        const float wx = er1 * vv.x - ei1 * vv.y, wy = er1 * vv.y + ei1 * vv.x;
        a1[t] = make_float2(c1 * u.x - s1 * wx, c1 * u.y - s1 * wy);
        qv[t] = make_float2(s1 * u.x + c1 * wx, s1 * u.y + c1 * wy);
      }
      ++rot;
    }
    if (r0 || r1) {
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        if (FULL || row < m) xq[row] = qv[t];
      }
    }
    __syncwarp();
    if (lane == 0) handoff::st_release(ver + q, r + 1);
    q = q + 1 == nbp ? 0 : q + 1;
  }
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    if (FULL || row < m) {
      if (h0) XA[(size_t)p0 * m + row] = a0[t];
      if (h1) XA[(size_t)p1 * m + row] = a1[t];
    }
  }
  if (lane == 0) { if (rot) atomicAdd(&ibuf[0], rot); if (chk) atomicAdd(&ibuf[6], chk); }
  __syncthreads();
}

// Cross pairs of blocks A and B (na, nb <= 2 * warps) with the warp-owned A
// columns held in registers: warp w owns A slots w and w + nw for the whole
// pass; in round r slot p meets B column (p + r) mod nmax. Only B columns move
// through shared memory, and the two pairs of a warp are processed together.
// As in rr_pass, rounds are ordered per column instead of by CTA barriers: B
// column q is touched by one slot per round, and the slot waits until q has
// finished the previous round (ver[q], in sm.perm).
template <typename R, bool TC>
template <int RPL>
__device__ __noinline__ void Engine<R, TC>::cross_pass_regs(C* XA, int na, C* XB, int nb, int m, R tol, R thr) {
  // the column counters live in sm.perm (2 cap entries)
  if constexpr (sizeof(R) == 4) if (max(nb, (int)(nt() >> 5)) <= 2 * cap) {
    float2* xa = reinterpret_cast<float2*>(XA);
    float2* xb = reinterpret_cast<float2*>(XB);
    if (m == 32 * RPL) cross_pass_f32<RPL, true>(xa, na, xb, nb, m, tol, thr, sm.perm, sm.ibuf);
    else cross_pass_f32<RPL, false>(xa, na, xb, nb, m, tol, thr, sm.perm, sm.ibuf);
    return;
  }
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int nmax = max(na, nb);
  int* ver = sm.perm;
  for (int c = tid(); c < nmax; c += nt()) ver[c] = 0;
  __syncthreads();
  const int p0 = w, p1 = w + nw;
  const bool o0 = p0 < nmax, o1 = p1 < nmax;  // slots this warp owns
  const bool h0 = p0 < na, h1 = p1 < na;
  C a0[RPL], a1[RPL], b0[RPL], b1[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    a0[t] = (h0 && row < m) ? XA[(size_t)p0 * m + row] : C{0, 0};
    a1[t] = (h1 && row < m) ? XA[(size_t)p1 * m + row] : C{0, 0};
  }
  int rot = 0, chk = 0;
  for (int r = 0; r < nmax && o0; ++r) {
    const int q0 = (p0 + r) % nmax, q1 = (p1 + r) % nmax;
    wait_col(ver + q0, r);
    if (o1) wait_col(ver + q1, r);
    const bool d0 = h0 && q0 < nb, d1 = h1 && q1 < nb;
    chk += (int)d0 + (int)d1;
    C* xb0 = XB + (size_t)q0 * m;
    C* xb1 = XB + (size_t)q1 * m;
    R al0 = 0, be0 = 0, gr0 = 0, gi0 = 0, al1 = 0, be1 = 0, gr1 = 0, gi1 = 0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      b0[t] = (d0 && row < m) ? xb0[row] : C{0, 0};
      b1[t] = (d1 && row < m) ? xb1[row] : C{0, 0};
      al0 = fma(a0[t].re, a0[t].re, fma(a0[t].im, a0[t].im, al0));
      be0 = fma(b0[t].re, b0[t].re, fma(b0[t].im, b0[t].im, be0));
      gr0 = fma(a0[t].re, b0[t].re, fma(a0[t].im, b0[t].im, gr0));
      gi0 = fma(a0[t].re, b0[t].im, fma(-a0[t].im, b0[t].re, gi0));
      al1 = fma(a1[t].re, a1[t].re, fma(a1[t].im, a1[t].im, al1));
      be1 = fma(b1[t].re, b1[t].re, fma(b1[t].im, b1[t].im, be1));
      gr1 = fma(a1[t].re, b1[t].re, fma(a1[t].im, b1[t].im, gr1));
      gi1 = fma(a1[t].re, b1[t].im, fma(-a1[t].im, b1[t].re, gi1));
    }
    {
      R v8[8] = {al0, be0, gr0, gi0, al1, be1, gr1, gi1};
      warp_sum8<R>(v8, lane);
      al0 = v8[0]; be0 = v8[1]; gr0 = v8[2]; gi0 = v8[3];
      al1 = v8[4]; be1 = v8[5]; gr1 = v8[6]; gi1 = v8[7];
    }
    R c0, s0, er0, ei0, c1, s1, er1, ei1;
    const bool r0 = d0 && rot_params<R>(al0, be0, gr0, gi0, tol, thr, c0, s0, er0, ei0);
    const bool r1 = d1 && rot_params<R>(al1, be1, gr1, gi1, tol, thr, c1, s1, er1, ei1);
    if (r0) {
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const C wv = {er0 * b0[t].re - ei0 * b0[t].im, er0 * b0[t].im + ei0 * b0[t].re};
        const C u = a0[t];
        a0[t] = C{c0 * u.re - s0 * wv.re, c0 * u.im - s0 * wv.im};
        const C nb0 = {s0 * u.re + c0 * wv.re, s0 * u.im + c0 * wv.im};
        const int row = lane + 32 * t;
        if (row < m) xb0[row] = nb0;
      }
      ++rot;
    }
    if (r1) {
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const C wv = {er1 * b1[t].re - ei1 * b1[t].im, er1 * b1[t].im + ei1 * b1[t].re};
        const C u = a1[t];
        a1[t] = C{c1 * u.re - s1 * wv.re, c1 * u.im - s1 * wv.im};
        const C nb1 = {s1 * u.re + c1 * wv.re, s1 * u.im + c1 * wv.im};
        const int row = lane + 32 * t;
        if (row < m) xb1[row] = nb1;
      }
      ++rot;
    }
    __syncwarp();
    if (lane == 0) {
      handoff::st_release(ver + q0, r + 1);
      if (o1) handoff::st_release(ver + q1, r + 1);
    }
  }
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int row = lane + 32 * t;
    if (row < m) {
      if (h0) XA[(size_t)p0 * m + row] = a0[t];
      if (h1) XA[(size_t)p1 * m + row] = a1[t];
    }
  }
  if (lane == 0) { if (rot) atomicAdd(&sm.ibuf[0], rot); if (chk) atomicAdd(&sm.ibuf[6], chk); }
  __syncthreads();
}

// Cyclic one-sided Jacobi SVD (Hestenes, J. SIAM 6, 1958) on the columns of X
// (m x nc, column-major). When X lives in shared memory, each sweep is one
// round-robin pass. When it does not fit, X stays in global memory and is
// processed in column blocks of bw: block I is staged in shared memory, its
// internal pairs are rotated, then every later block J is staged beside it for
// the cross pairs and written back, and finally I is written back. Every pair
// is visited once per sweep. Sweeps stop when one rotates nothing; ibuf[1] = 1
// then, 0 if the sweep cap was hit.
template <typename R, bool TC>
__device__ __noinline__ int Engine<R, TC>::jacobi(C* X, int m, int nc, bool x_in_smem) {
  // rotate a pair when |x_p^H x_q| > tol |x_p||x_q|, tol = a.tol * sqrt(m): the
  // rounding noise of a length-m dot product grows like sqrt(m) eps, so a fixed
  // tolerance would leave the last sweeps rotating pairs on noise alone
  const R tol = (R)(a.tol * sqrt((double)m));
  const int lane = tid() & 31, nw = nt() >> 5;
  // squared column norms (FP64 accumulation) and ||X||_F^2
  for (int col = tid() >> 5; col < nc; col += nw) {
    const C* x = X + (size_t)col * m;
    double s2 = 0.0;
    for (int row = lane; row < m; row += 32) s2 += (double)abs2(ld_x(x + row, x_in_smem));
    s2 = warp_sum(s2);
    if (lane == 0) sm.wn[col] = s2;
  }
  __syncthreads();
  double fro = 0.0;
  for (int col = tid(); col < nc; col += nt()) fro += sm.wn[col];
  fro = block_sum(fro, sm.red);
  // columns below floor_rel/4 of the matrix norm are zero to working precision
  // (they will be discarded): they are not rotated, so that the nc - m null
  // columns of a wide matrix settle instead of shrinking towards underflow
  const R thr = (R)(0.0625 * a.floor_rel * a.floor_rel * fro);
  // A pair is rotated only when both of its columns are at or above thr, so a
  // column that starts below thr keeps its values through every sweep. Those
  // columns are swapped behind the active ones and the sweeps visit only the
  // active prefix: a two-site theta of rank ~chi plus a small gate term has
  // about half of its R^H columns below thr, and skipping them removes most
  // of the pair checks of a sweep without changing any rotation's arithmetic.
  if (tid() == 0) {
    const double thr_d = (double)thr;
    int na = 0;
    for (int j = 0; j < nc; ++j) na += sm.wn[j] >= thr_d;
    int ns = 0, q = na;
    for (int j = 0; j < na; ++j) {
      if (sm.wn[j] >= thr_d) continue;
      while (q < nc && sm.wn[q] < thr_d) ++q;
      if (q >= nc) break;  // unreachable: the counts of the two sides agree
      sm.perm[2 * ns] = j;
      sm.perm[2 * ns + 1] = q;
      ++ns;
      ++q;
    }
    sm.ibuf[3] = na;
    sm.ibuf[4] = ns;
    sm.ibuf[1] = 0;
    sm.ibuf[5] = 0;  // column handoff timeout flag of the passes
  }
  __syncthreads();
  const int n_act = sm.ibuf[3], n_swap = sm.ibuf[4];
  for (int sidx = tid() >> 5; sidx < n_swap; sidx += nw) {
    C* xp = X + (size_t)sm.perm[2 * sidx] * m;
    C* xq = X + (size_t)sm.perm[2 * sidx + 1] * m;
    for (int row = lane; row < m; row += 32) {
      const C u = ld_x(xp + row, x_in_smem), v = ld_x(xq + row, x_in_smem);
      xp[row] = v;
      xq[row] = u;
    }
  }
  __syncthreads();
  nc = n_act;
  int sweep = 0;
  if (nc < 2) { __syncthreads(); if (tid() == 0) sm.ibuf[1] = 1; __syncthreads(); return 0; }
  if constexpr (kTC) {
    // single precision, staged in global memory, up to 256 rows and more than
    // one 32-column block: Gram matrices and block updates on the tensor cores
    if (tc_ok && nt() == TcJac::THREADS && !x_in_smem && m <= 256 && nc > 32) {
      SubTimer spt(st, SP_PASSES);
      return jacobi_tc(X, m, nc, tol, thr);
    }
  }
  C* xs = reinterpret_cast<C*>(sm.x);
  // column blocks of bw: the width the staging buffer allows, at most 2 columns
  // per warp so that a block's warp-owned columns fit in registers
  // Staged blocks: two (I and J) fit in the staging room. (A third block for
  // double-buffered loads of J measured no faster with two CTAs per SM, whose
  // co-resident CTA already covers the copy latency.)
  int bw = 1;
  if (!x_in_smem) {
    while (4 * bw * m <= a.smem_x_elems && 2 * bw < nc) bw *= 2;
  } else {
    bw = nc;
  }
  if (bw > 2 * nw) bw = 2 * nw;
  const int nbk = (nc + bw - 1) / bw;
  auto cross = [&](C* XA, int na, C* XB, int nbb) {
    if (m <= 64) cross_pass_regs<2>(XA, na, XB, nbb, m, tol, thr);
    else if (m <= 128) cross_pass_regs<4>(XA, na, XB, nbb, m, tol, thr);
    else if (m <= 256) cross_pass_regs<8>(XA, na, XB, nbb, m, tol, thr);
    else cross_pass(XA, na, XB, nbb, m, tol, thr);
  };
  SubTimer spt(st, SP_PASSES);
  int prev_rot = 1 << 30;   // no stall test before the second sweep
  while (sweep < a.max_sweeps) {
    if (tid() == 0) { sm.ibuf[0] = 0; sm.ibuf[6] = 0; }
    __syncthreads();
    if (x_in_smem) {
      for (int I = 0; I < nbk; ++I) {
        const int nI = min(bw, nc - I * bw);
        C* xI = X + (size_t)I * bw * m;
        rr_pass(xI, m, nI, tol, thr);
        for (int J = I + 1; J < nbk; ++J) cross(xI, nI, X + (size_t)J * bw * m, min(bw, nc - J * bw));
      }
    } else {
      // Blocks are contiguous column ranges of X, moved by whole-block bulk
      // copies into sa (block I) and sb (block J), which are adjacent in
      // shared memory. Blocks 2k and 2k+1 form a super-block: one round-robin
      // pass over its 2 bw columns covers the pairs inside both blocks and
      // those between them, with two pairs per warp in every round. Every pair
      // of columns is still visited exactly once per sweep.
      C* sa = xs;
      C* sb = xs + (size_t)bw * m;
      for (int I = 0; I < nbk && !failed(); ++I) {
        const int nI = min(bw, nc - I * bw);
        C* gI = X + (size_t)I * bw * m;
        const bool lead = (I % 2 == 0) && (I + 1 < nbk);
        bulk_load(sa, gI, (uint32_t)(sizeof(C) * nI * m));
        if (failed()) break;
        if (lead) {
          const int n1 = min(bw, nc - (I + 1) * bw);
          bulk_load(sb, gI + (size_t)bw * m, (uint32_t)(sizeof(C) * n1 * m));
          if (failed()) break;
          rr_pass(xs, m, nI + n1, tol, thr);
          bulk_store(gI + (size_t)bw * m, sb, (uint32_t)(sizeof(C) * n1 * m));
        } else if (I % 2 == 0) {
          rr_pass(sa, m, nI, tol, thr);
        }
        for (int J = lead ? I + 2 : I + 1; J < nbk; ++J) {
          const int nJ = min(bw, nc - J * bw);
          C* gJ = X + (size_t)J * bw * m;
          bulk_load(sb, gJ, (uint32_t)(sizeof(C) * nJ * m));
          if (failed()) break;
          cross(sa, nI, sb, nJ);
          bulk_store(gJ, sb, (uint32_t)(sizeof(C) * nJ * m));
        }
        bulk_store(gI, sa, (uint32_t)(sizeof(C) * nI * m));
      }
    }
    ++sweep;
    if (failed()) break;
    if (sm.ibuf[5]) { fail(ST_HANDOFF_TIMEOUT, sweep); break; }
    const int rot = sm.ibuf[0];
    if (tid() == 0) { st.jac_rots += (unsigned long long)rot; st.jac_pairs += (unsigned long long)sm.ibuf[6]; }
    __syncthreads();
    if (rot == 0) { if (tid() == 0) sm.ibuf[1] = 1; break; }
    // Single precision: near convergence (fewer than 1 in 20 pairs rotating)
    // a rotation count that stops falling means the FP32 inner products are
    // deciding on their own rounding; one pass in FP64 arithmetic then
    // finishes the SVD, as it does at the sweep cap.
    if constexpr (sizeof(R) == 4) {
      if ((rot >= prev_rot && 20 * rot < sm.ibuf[6]) || sweep >= a.max_sweeps) {
        reorth_pass_f64(X, m, nc, x_in_smem, (double)thr);
        if (tid() == 0) { st.reorth++; sm.ibuf[1] = 1; }
        __syncthreads();
        break;
      }
    }
    prev_rot = rot;
  }
  __syncthreads();
  return sweep;
}

// The FP64 re-orthogonalisation pass of a single-precision Jacobi whose FP32
// residual stalled: one cyclic round-robin pass (Brent & Luk order, rounds
// separated by CTA barriers, one warp per pair) over the nc active columns of
// X, with FP64 inner products, FP64 rotation parameters and the rotation
// evaluated in FP64 before the columns are rounded back to FP32. A pair is
// rotated when its cosine exceeds 2^-24, the orthogonality FP32 columns can
// hold, and both columns lie at or above thr. X is in shared memory or, when
// staged, in global memory with every bulk copy already drained.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::reorth_pass_f64(C* X, int m, int nc, bool x_in_smem, double thr) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int np = nc + (nc & 1);
  const double tol = 5.9604644775390625e-08;
  for (int r = 0; r < np - 1; ++r) {
    for (int t = w; t < np / 2; t += nw) {
      int p, q;
      if (t == 0) { p = np - 1; q = r; }
      else { p = (r + t) % (np - 1); q = (r - t + np - 1) % (np - 1); }
      if (p >= nc || q >= nc) continue;
      C* xp = X + (size_t)p * m;
      C* xq = X + (size_t)q * m;
      double al = 0, be = 0, gr = 0, gi = 0;
      for (int row = lane; row < m; row += 32) {
        const C u = ld_x(xp + row, x_in_smem), v = ld_x(xq + row, x_in_smem);
        const double ur = u.re, ui = u.im, vr = v.re, vi = v.im;
        al = fma(ur, ur, fma(ui, ui, al));
        be = fma(vr, vr, fma(vi, vi, be));
        gr = fma(ur, vr, fma(ui, vi, gr));
        gi = fma(ur, vi, fma(-ui, vr, gi));
      }
      al = warp_sum(al); be = warp_sum(be); gr = warp_sum(gr); gi = warp_sum(gi);
      double c, sn, er, ei;
      if (!rot_params<double>(al, be, gr, gi, tol, thr, c, sn, er, ei)) continue;
      for (int row = lane; row < m; row += 32) {
        const C u = ld_x(xp + row, x_in_smem), v = ld_x(xq + row, x_in_smem);
        const double wr = er * (double)v.re - ei * (double)v.im, wi = er * (double)v.im + ei * (double)v.re;
        xp[row] = C{(R)(c * (double)u.re - sn * wr), (R)(c * (double)u.im - sn * wi)};
        xq[row] = C{(R)(sn * (double)u.re + c * wr), (R)(sn * (double)u.im + c * wi)};
      }
    }
    __syncthreads();
  }
}

// SVD and truncation of one working matrix Z (m x nc; its left singular
// vectors become the orthonormal site). With pre set, Y holds Z^H (nc x m,
// column-major, destroyed): Z^H = Q R by Householder (Q not formed), then
// one-sided Jacobi on the columns of X = R^H (Drmac & Veselic, SIAM J. Matrix
// Anal. Appl. 29, 2008). Z = R^H Q^H, so the normalised columns of X J are the
// left singular vectors of Z, after far fewer sweeps than Z itself needs.
// X = R^H goes to shared memory when x_smem is set, replaces R in place when Y
// is square and in shared memory, and goes to XG otherwise. Without pre, X
// already holds Z (column-major) and is rotated as it is.
// Truncation keeps k = max(1, min(chi_max, k_floor, k_cut, min(m, nc))) sorted
// singular values (descending, ties by column index):
//   k_cut   = the smallest k with sum_{j>=k} s_j^2 <= cutoff * sum_j s_j^2,
//   k_floor = #{j : s_j > floor_rel * s_0};
// then, if s_{k-1} - s_k <= gap_rel * s_0, k drops to the largest k' < k with a
// clear gap (a cut never splits a group of equal singular values), unless no
// such k' >= 1 exists. The kept values are rescaled to unit norm, so every
// sample stays normalised.
// On return: the singular vectors scaled by the singular values are the
// columns of X (ncx columns, in shared memory when x_sh), sm.wn their squared
// norms, sm.perm their ranking, sm.ibuf[2] = k and sm.dbuf[0] = 1/sqrt(kept
// weight). flops_theta is added to the algorithmic flop count. With factored
// set, Y already holds R (strict upper triangle, leading dimension y_ld;
// diagonal in the alpha array), and the QR is not run again. Returns false
// after a recorded failure.
template <typename R, bool TC>
__device__ __noinline__ bool Engine<R, TC>::svd_truncate(C* Y, C*& X, int& ncx, bool& x_sh, bool pre, bool x_smem,
                                                         int m, int nc, bool is_swap, double flops_theta,
                                                         bool factored, int y_ld) {
  const int r = min(m, nc);
  C* xs = reinterpret_cast<C*>(sm.x);
  if (pre) {
    PhaseTimer pt(st, PH_QR);
    if (!factored) {
      double fro = 0.0;
      for (int e = tid(); e < m * nc; e += nt()) fro += (double)abs2(Y[e]);
      fro = block_sum(fro, sm.red);
      // skip only reflectors whose 1/|x|^2 scale would overflow; smaller
      // columns are still rotated exactly (dropping them would lose their weight)
      qr_factor(Y, nc, m, nullptr, (sizeof(R) == 4 ? 1e-30 : 1e-280) * fro);
    }
    const int ld = y_ld > 0 ? y_ld : nc;
    const C* alpha = reinterpret_cast<const C*>(sm.hh) + 4 * cap;
    X = x_smem ? xs : XG;
    if (X == Y) {
      // square: move the upper triangle of R to X = R^H in place
      const bool y_sm = Y == xs;
      for (int e = tid(); e < m * m; e += nt()) {
        const int ca = e / m, rj = e - ca * m;
        if (ca > rj) {
          const C u = y_sm ? Y[(size_t)ca * m + rj] : ldcg_c(Y + (size_t)ca * m + rj);
          X[(size_t)rj * m + ca] = C{u.re, -u.im};
          X[(size_t)ca * m + rj] = C{0, 0};
        } else if (ca == rj) {
          X[(size_t)rj * m + rj] = C{alpha[rj].re, -alpha[rj].im};
        }
      }
    } else {
      for (int e = tid(); e < m * r; e += nt()) {
        const int j = e / m, aa = e - j * m;
        C v = {0, 0};
        if (aa > j) { const C u = ldcg_c(Y + (size_t)aa * ld + j); v = C{u.re, -u.im}; }
        else if (aa == j) v = C{alpha[j].re, -alpha[j].im};
        X[e] = v;
      }
    }
    __syncthreads();
    ncx = r;
  } else {
    ncx = nc;
  }
  if (failed()) return false;
  int sweeps;
  { PhaseTimer pt(st, PH_JACOBI); sweeps = jacobi(X, m, ncx, X == xs); }
  const int converged = sm.ibuf[1];
  PhaseTimer pt_trunc(st, PH_TRUNC);
  SubTimer srt(st, SP_RANK);
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  // squared column norms (FP64 accumulation)
  x_sh = X == xs;
  for (int col = w; col < ncx; col += nw) {
    const C* x = X + (size_t)col * m;
    double s2 = 0.0;
    for (int row = lane; row < m; row += 32) s2 += (double)abs2(ld_x(x + row, x_sh));
    s2 = warp_sum(s2);
    if (lane == 0) {
      if (!(s2 >= 0.0 && s2 <= 1.0e300)) { s2 = 0.0; sm.ibuf[14] = 1; }
      sm.wn[col] = s2;
    }
  }
  __syncthreads();
  const int bad_norm = sm.ibuf[14];
  __syncthreads();
  if (bad_norm) { if (tid() == 0) sm.ibuf[14] = 0; fail(ST_NONFINITE, 2000 + m); return false; }
  for (int j = tid(); j < ncx; j += nt()) sm.perm[j] = -1;
  __syncthreads();
  for (int j = tid(); j < ncx; j += nt()) {
    const double wj = sm.wn[j];
    int rank = 0;
    for (int q = 0; q < ncx; ++q) {
      const double wq = sm.wn[q];
      rank += (wq > wj) || (wq == wj && q < j);
    }
    sm.perm[rank] = j;
  }
  __syncthreads();
  // the ranks of finite keys form a permutation; check before indexing with it
  int bad_perm = 0;
  for (int j = tid(); j < ncx; j += nt()) bad_perm |= (sm.perm[j] < 0 || sm.perm[j] >= ncx);
  if (__syncthreads_or(bad_perm)) { fail(ST_BAD_RANK, 9000 + m); return false; }
  if (tid() == 0) {
    double tot = 0.0;
    for (int j = ncx - 1; j >= 0; --j) tot += sm.wn[sm.perm[j]];
    const double thr = a.cutoff * tot;
    int kcut = ncx;
    double acc = 0.0;
    for (int j = ncx - 1; j >= 1; --j) {
      acc += sm.wn[sm.perm[j]];
      if (acc <= thr) kcut = j; else break;
    }
    const double s0 = sqrt(sm.wn[sm.perm[0]]);
    int kfloor = 0;
    while (kfloor < ncx && sqrt(sm.wn[sm.perm[kfloor]]) > a.floor_rel * s0) ++kfloor;
    int k = min(min(cap, kfloor), min(kcut, min(m, ncx)));
    if (k < 1) k = 1;
    // never split a group of equal singular values: drop the whole group
    if (k < ncx && sqrt(sm.wn[sm.perm[k]]) > a.floor_rel * s0) {
      int kk = k;
      while (kk >= 1 && sqrt(sm.wn[sm.perm[kk - 1]]) - sqrt(sm.wn[sm.perm[kk]]) <= a.gap_rel * s0) --kk;
      if (kk >= 1) k = kk;
    }
    double kept = 0.0;
    for (int j = k - 1; j >= 0; --j) kept += sm.wn[sm.perm[j]];
    sm.ibuf[2] = k;
    sm.dbuf[0] = kept > 0.0 ? 1.0 / sqrt(kept) : 0.0;
    const double disc = tot > 0.0 ? (tot - kept) / tot : 0.0;
    if (disc > st.max_discarded) st.max_discarded = disc;
    if (k > st.max_chi) st.max_chi = k;
    st.sweeps += sweeps;
    if (!converged) st.not_converged++;
    if (is_swap) st.swap_updates++; else st.gate_updates++;
    const double mx = (double)max(m, nc), mn = (double)min(m, nc);
    st.alg_flops += flops_theta + 4.0 * (14.0 * mx * mn * mn + 8.0 * mn * mn * mn);
  }
  __syncthreads();
  return true;
}

// Gate on bond (i, i+1). The centre is first moved onto site i or i+1, so that
// theta holds it and the environments are orthonormal (mixed-canonical form).
// After the SVD (svd_truncate) the centre sits on site i (end_left) or i+1.
// With theta_in_th the gate is not applied: theta' (2 d_i x 2 d_{i+2},
// row-major) is already in TH (the second split of a three-site update) and g
// is not read.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::two_site(int i, const C g[16], bool end_left, bool is_swap,
                                                     bool theta_in_th) {
  if (failed()) return;
  if (i < 0 || i > a.n - 2) { fail(ST_BAD_DIM, i); return; }
  if (centre < i) move_centre(i);
  else if (centre > i + 1) move_centre(i + 1);
  if (failed()) return;
  const int dl = sm.dims[i], dc = sm.dims[i + 1], dr = sm.dims[i + 2];
  if (!dim_ok(dl) || !dim_ok(dc) || !dim_ok(dr)) { fail(ST_BAD_DIM, 1000 + i); return; }
  const int m = end_left ? 2 * dr : 2 * dl;
  const int nc = end_left ? 2 * dl : 2 * dr;
  // X = R^H lives in shared memory when it fits, or replaces R in place when
  // Z is square; other shapes run plain Jacobi on Z.
  const int r = min(m, nc);
  const bool y_smem = (m == nc) && (m * nc <= a.smem_x_elems);
  const bool x_smem = y_smem || (m * r <= a.smem_x_elems);
  const bool pre = a.precondition && (x_smem || m == nc);
  C* xs = reinterpret_cast<C*>(sm.x);
  C* X;
  C* Y = nullptr;
  if (pre) {
    Y = y_smem ? xs : XG;
    PhaseTimer pt(st, PH_THETA);
    if (theta_in_th) theta_from_th(dl, dr, end_left, true, Y);
    else form_theta(i, g, end_left, true, Y);
  } else {
    const bool x_in = m * nc <= a.smem_x_elems;
    X = x_in ? xs : XG;
    PhaseTimer pt(st, PH_THETA);
    if (theta_in_th) theta_from_th(dl, dr, end_left, false, X);
    else form_theta(i, g, end_left, false, X);
  }
  int ncx = 0;
  bool x_sh = false;
  const double flops_theta = theta_in_th ? 0.0 : 32.0 * dl * dc * dr;
  if (!svd_truncate(Y, X, ncx, x_sh, pre, x_smem, m, nc, is_swap, flops_theta)) return;
  PhaseTimer pt_proj(st, PH_TRUNC);
  SubTimer sjt(st, SP_PROJ);
  const int k = sm.ibuf[2];
  const R renorm = (R)sm.dbuf[0];
  if (!dim_ok(k)) { fail(ST_BAD_RANK, k); return; }
  if (!end_left) {
    // site i <- U[:, :k] (2dl x k); site i+1 <- renorm * U^H theta' (k x 2dr)
    C* Ai = S(i);
    for (int e = tid(); e < m * k; e += nt()) {
      const int row = e / k, mm = e - row * k;
      const int col = sm.perm[mm];
      const double wv = sm.wn[col];
      const R inv = wv > 0.0 ? (R)(1.0 / sqrt(wv)) : R(0);
      Ai[e] = scale(ld_x(X + (size_t)col * m + row, x_sh), inv);
    }
    __syncthreads();
    project_left(Ai, m, k, TH, 2 * dr, renorm, S(i + 1));
    if (tid() == 0) sm.dims[i + 1] = k;
    centre = i + 1;
  } else {
    // site i+1 <- V^H[:k, :] (k x 2dr); site i <- renorm * theta' V (2dl x k)
    C* Bi = S(i + 1);
    const int ncol = 2 * dr;  // == m
    for (int e = tid(); e < k * ncol; e += nt()) {
      const int mm = e / ncol, col = e - mm * ncol;
      const int src = sm.perm[mm];
      const double wv = sm.wn[src];
      const R inv = wv > 0.0 ? (R)(1.0 / sqrt(wv)) : R(0);
      Bi[e] = scale(ld_x(X + (size_t)src * m + col, x_sh), inv);
    }
    __syncthreads();
    C* Ai = S(i);
    const int rows = 2 * dl;
    if (a.smem_x_elems >= gemm_tile_elems(nt())) {
      // Ai = renorm theta' V (V^H = Bi)
      const C* thp = TH;
      const C* bip = Bi;
      auto fa = [=](int ii, int kk) { return thp[(size_t)ii * ncol + kk]; };
      auto fb = [=](int kk, int jj) { const C u = bip[(size_t)jj * ncol + kk]; return C{u.re, -u.im}; };
      auto fo = [=](int ii, int jj, C v) { Ai[(size_t)ii * k + jj] = scale(v, renorm); };
      bool done = false;
      if constexpr (kTC) {
        if (tc_worth(rows, k, ncol)) { tc_cgemm(rows, k, ncol, fa, fb, fo); done = true; }
      }
      if (!done) block_gemm<R>(rows, k, ncol, reinterpret_cast<C*>(sm.x), fa, fb, fo);
    } else {
      for (int e = tid(); e < rows * k; e += nt()) {
        const int row = e / k, mm = e - row * k;
        C acc2 = {0, 0};
        const C* th = TH + (size_t)row * ncol;
        const C* bv = Bi + (size_t)mm * ncol;
        for (int col = 0; col < ncol; ++col) fma_cc(acc2, bv[col], th[col]);
        Ai[e] = scale(acc2, renorm);
      }
    }
    __syncthreads();
    if (tid() == 0) sm.dims[i + 1] = k;
    centre = i;
  }
  __syncthreads();
}

// out = renorm * U^H theta (k x ncol, row-major), with U = Ai (m x k,
// row-major) and theta (m x ncol, row-major). out must not alias either.
template <typename R, bool TC>
__device__ void Engine<R, TC>::project_left(const C* Ai, int m, int k, const C* theta, int ncol, R renorm, C* out) {
  if (a.smem_x_elems >= gemm_tile_elems(nt())) {
    // the working matrix in shared memory is no longer needed: it stages the GEMM
    auto fa = [=](int ii, int kk) { const C u = Ai[(size_t)kk * k + ii]; return C{u.re, -u.im}; };
    auto fb = [=](int kk, int jj) { return theta[(size_t)kk * ncol + jj]; };
    auto fo = [=](int ii, int jj, C v) { out[(size_t)ii * ncol + jj] = scale(v, renorm); };
    bool done = false;
    if constexpr (kTC) {
      if (tc_worth(k, ncol, m)) { tc_cgemm(k, ncol, m, fa, fb, fo); done = true; }
    }
    if (!done) block_gemm<R>(k, ncol, m, reinterpret_cast<C*>(sm.x), fa, fb, fo);
  } else {
    for (int e = tid(); e < k * ncol; e += nt()) {
      const int mm = e / ncol, col = e - mm * ncol;
      C acc2 = {0, 0};
      for (int row = 0; row < m; ++row) fma_cc(acc2, Ai[(size_t)row * k + mm], theta[(size_t)row * ncol + col]);
      out[e] = scale(acc2, renorm);
    }
  }
  __syncthreads();
}

// The working matrix of a two-site SVD from a theta' already in TH
// (2 dl x 2 dr, row-major): the layouts form_theta writes (Z or Z^H, with
// Z = theta' or theta'^T).
template <typename R, bool TC>
__device__ void Engine<R, TC>::theta_from_th(int dl, int dr, bool end_left, bool zh, C* X) {
  const int m = 2 * dl, ncol = 2 * dr;
  for (int e = tid(); e < m * ncol; e += nt()) {
    const int row = e / ncol, col = e - row * ncol;
    const C o = TH[e];
    if (!zh) {
      if (end_left) X[(size_t)row * ncol + col] = o;
      else X[(size_t)col * m + row] = o;
    } else {
      const C oc = {o.re, -o.im};
      if (end_left) X[(size_t)col * m + row] = oc;
      else X[(size_t)row * ncol + col] = oc;
    }
  }
  __syncthreads();
}

// Gate g (basis |s_i s_{i+2}>) on chain positions i and i+2 as one three-site
// update (the bond-2 alternative to swap routing): with the centre on i, i+1
// or i+2,
//   theta3[a, s, t, u, b] = sum_{c,d} A_i[a,s,c] A_{i+1}[c,t,d] A_{i+2}[d,u,b],
//   M1[(a,x), (t,y,b)]    = sum_{s,u} g[(x,y),(s,u)] theta3[a,s,t,u,b]
// (2 d_i x 4 d_{i+3}). The first split is the SVD of M1 with the two-site
// keep rule: site i <- U1 (2 d_i x k1), and renorm * U1^H M1 (k1 x 4 d_{i+3},
// row-major) is the theta' of bond (i+1, i+2) read as (2 k1 x 2 d_{i+3}).
// The second split is the two-site SVD of that theta'. The centre ends on i+2.
// Arena: M1 in W3 (8 cap^2), Y = M1^H in W3 + 8 cap^2 (8 cap^2), or its two
// row halves at W3 + 8 cap^2 and W3 + 12 cap^2 for the two-level QR.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::three_site(int i, const C g[16]) {
  if (failed()) return;
  if (i < 0 || i > a.n - 3) { fail(ST_BAD_DIM, 11000 + i); return; }
  if (centre < i) move_centre(i);
  else if (centre > i + 2) move_centre(i + 2);
  if (failed()) return;
  const int dl = sm.dims[i], d1 = sm.dims[i + 1], d2 = sm.dims[i + 2], dr = sm.dims[i + 3];
  if (!dim_ok(dl) || !dim_ok(d1) || !dim_ok(d2) || !dim_ok(dr)) { fail(ST_BAD_DIM, 12000 + i); return; }
  const int m = 2 * dl, nc = 4 * dr;
  C* M1 = W3();
  C* Y = W3() + (size_t)8 * cap * cap;
  // two-level QR when Z^H's two row halves (2 dr x 2 dl each) are at least square
  const bool two_level = dr >= dl;
  C* Yt = Y;
  C* Yb = Y + (size_t)4 * cap * cap;
  {
    PhaseTimer pt(st, PH_THETA);
    const C* A = S(i);
    const C* B = S(i + 1);
    const C* Cs = S(i + 2);
    // T1[(a,s), (t,d)] = A_i (2dl x d1) A_{i+1} (d1 x 2 d2), row-major in TH
    // T2[(a,s,t), (u,b)] = T1 (4 dl x d2) A_{i+2} (d2 x 2 dr), row-major in Y
    C* T1 = TH;
    const bool gemm = a.smem_x_elems >= gemm_tile_elems(nt());
    {
      auto fa = [=](int ii, int kk) { return A[(size_t)ii * d1 + kk]; };
      auto fb = [=](int kk, int jj) { return B[(size_t)kk * 2 * d2 + jj]; };
      auto fo = [=](int ii, int jj, C v) { T1[(size_t)ii * 2 * d2 + jj] = v; };
      if (gemm) block_gemm<R>(2 * dl, 2 * d2, d1, reinterpret_cast<C*>(sm.x), fa, fb, fo);
      else
        for (int e = tid(); e < 2 * dl * 2 * d2; e += nt()) {
          const int ii = e / (2 * d2), jj = e - ii * 2 * d2;
          C acc = {0, 0};
          for (int kk = 0; kk < d1; ++kk) fma_c(acc, fa(ii, kk), fb(kk, jj));
          fo(ii, jj, acc);
        }
      __syncthreads();
    }
    {
      auto fa = [=](int ii, int kk) { return T1[(size_t)ii * d2 + kk]; };
      auto fb = [=](int kk, int jj) { return Cs[(size_t)kk * 2 * dr + jj]; };
      auto fo = [=](int ii, int jj, C v) { Y[(size_t)ii * 2 * dr + jj] = v; };
      if (gemm) block_gemm<R>(4 * dl, 2 * dr, d2, reinterpret_cast<C*>(sm.x), fa, fb, fo);
      else
        for (int e = tid(); e < 4 * dl * 2 * dr; e += nt()) {
          const int ii = e / (2 * dr), jj = e - ii * 2 * dr;
          C acc = {0, 0};
          for (int kk = 0; kk < d2; ++kk) fma_c(acc, fa(ii, kk), fb(kk, jj));
          fo(ii, jj, acc);
        }
      __syncthreads();
    }
    // gate on s and u: M1[(a,x), (t,y,b)] = sum_{s,u} g[(x,y),(s,u)] T2[(a,s,t), (u,b)]
    for (int e = tid(); e < dl * 2 * dr; e += nt()) {
      const int aa = e / (2 * dr), tb = e - aa * 2 * dr;
      const int t = tb / dr, bb = tb - t * dr;
      C tv[4];
#pragma unroll
      for (int su = 0; su < 4; ++su) {
        const int s_ = su >> 1, u = su & 1;
        tv[su] = Y[(size_t)((aa * 2 + s_) * 2 + t) * 2 * dr + u * dr + bb];
      }
#pragma unroll
      for (int xy = 0; xy < 4; ++xy) {
        C o = {0, 0};
#pragma unroll
        for (int q = 0; q < 4; ++q) fma_c(o, g[xy * 4 + q], tv[q]);
        const int x = xy >> 1, y = xy & 1;
        M1[(size_t)(aa * 2 + x) * nc + (t * 2 + y) * dr + bb] = o;
      }
    }
    __syncthreads();
    // Y = Z^H of Z = M1 (nc x m column-major): the conjugate of M1, element by
    // element. For the two-level QR its rows are split into two halves of
    // 2 dr rows, each column-major with leading dimension 2 dr.
    if (!two_level) {
      for (int e = tid(); e < m * nc; e += nt()) { const C o = M1[e]; Y[e] = C{o.re, -o.im}; }
    } else {
      const int h = 2 * dr;
      for (int e = tid(); e < m * nc; e += nt()) {
        const int aa = e / nc, c = e - aa * nc;
        const C o = M1[e];
        (c < h ? Yt : Yb)[(size_t)aa * h + (c < h ? c : c - h)] = C{o.re, -o.im};
      }
    }
    __syncthreads();
  }
  if (two_level) {
    // Two-level QR of Z^H (4 dr x 2 dl): the R factors of its two row halves
    // (blocked Householder where the staging room allows), then the R of the
    // stacked pair (ts_combine). Only R is needed: the Jacobi yields U1.
    PhaseTimer pt(st, PH_QR);
    double fro = 0.0;
    for (int e = tid(); e < m * nc; e += nt()) fro += (double)abs2(M1[e]);
    fro = block_sum(fro, sm.red);
    const double tiny2 = (sizeof(R) == 4 ? 1e-30 : 1e-280) * fro;
    const int h = 2 * dr;
    C* alpha = reinterpret_cast<C*>(sm.hh) + 4 * cap;
    for (int half = 0; half < 2 && !failed(); ++half) {
      C* Yh = half ? Yb : Yt;
      qr_factor(Yh, h, m, nullptr, tiny2);
      if (failed()) return;
      // the diagonal of this half's R into its array (the next QR reuses alpha)
      for (int j = tid(); j < m; j += nt()) Yh[(size_t)j * h + j] = alpha[j];
      __syncthreads();
    }
    if (failed()) return;
    ts_combine(Yt, Yb, h, m, tiny2);
  }
  const bool x_smem = m * m <= a.smem_x_elems;
  C* X = nullptr;
  int ncx = 0;
  bool x_sh = false;
  const double flops_theta = 32.0 * dl * d1 * d2 + 64.0 * dl * d2 * dr;
  if (!svd_truncate(two_level ? Yt : Y, X, ncx, x_sh, true, x_smem, m, nc, false, flops_theta, two_level,
                    two_level ? 2 * dr : 0))
    return;
  {
    PhaseTimer pt_proj(st, PH_TRUNC);
    SubTimer sjt(st, SP_PROJ);
    const int k1 = sm.ibuf[2];
    const R renorm = (R)sm.dbuf[0];
    if (!dim_ok(k1)) { fail(ST_BAD_RANK, k1); return; }
    // site i <- U1[:, :k1]; TH <- renorm U1^H M1 (k1 x 4 dr)
    C* Ai = S(i);
    for (int e = tid(); e < m * k1; e += nt()) {
      const int row = e / k1, mm = e - row * k1;
      const int col = sm.perm[mm];
      const double wv = sm.wn[col];
      const R inv = wv > 0.0 ? (R)(1.0 / sqrt(wv)) : R(0);
      Ai[e] = scale(ld_x(X + (size_t)col * m + row, x_sh), inv);
    }
    __syncthreads();
    project_left(Ai, m, k1, M1, nc, renorm, TH);
    if (tid() == 0) { sm.dims[i + 1] = k1; st.three_site++; }
    centre = i + 1;
    __syncthreads();
  }
  // second split: theta' of bond (i+1, i+2) = TH as (2 k1) x (2 dr)
  two_site(i + 1, g, false, false, true);
}

}  // namespace tepai
