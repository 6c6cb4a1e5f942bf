// Orthogonality-centre moves of the mixed-canonical MPS by Householder QR
// (Sec. II.A: gates act on an MPS in mixed-canonical form).
#pragma once
#include "engine.cuh"

namespace tepai {

// Householder QR of Y (m x nq, column-major, ld m): Y = Q R with r = min(m, nq).
// Reflector j is H_j = I - tau_j v_j v_j^H, v_j = (vhead_j, Y[j+1.., j]); it maps
// the column onto alpha_j e_j with alpha_j = -e^{i arg x_0} |x|. On return the
// strict upper triangle of R is in Y, its diagonal in alpha[], and Q (m x r,
// column-major) is formed explicitly by backward accumulation unless Q is null.
// A reflector is skipped (tau = 0) when the remaining column has |x|^2 <= tiny2,
// or when tau = 1/(|x|(|x|+|x_0|)) is not finite: an evolved state carries
// amplitudes like sin(Delta/2)^k whose squares underflow FP32, and the scale
// would overflow.
template <typename R>
__device__ void Engine<R>::householder(C* Y, int m, int nq, C* Q, double tiny2) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int r = min(m, nq);
  C* vhead = reinterpret_cast<C*>(sm.hh);
  C* tau = vhead + 2 * cap;
  C* alpha = tau + 2 * cap;
  for (int j = 0; j < r; ++j) {
    if (w == 0) {
      const C* y = Y + (size_t)j * m;
      R nr2 = 0;
      for (int row = j + lane; row < m; row += 32) nr2 += abs2(y[row]);
      nr2 = warp_sum(nr2);
      if (lane == 0) {
        const C x0 = y[j];
        const R ax0 = sqrt(abs2(x0));
        const R nrm = sqrt(nr2);
        const R tj = R(1) / (nrm * (nrm + ax0));
        if (!((double)nr2 > tiny2) || !(nrm > R(0)) || !isfinite(tj)) {
          vhead[j] = C{1, 0}; tau[j] = C{0, 0}; alpha[j] = x0;
        } else {
          const C ph = ax0 > R(0) ? C{x0.re / ax0, x0.im / ax0} : C{1, 0};
          alpha[j] = C{-ph.re * nrm, -ph.im * nrm};
          vhead[j] = C{ph.re * (ax0 + nrm), ph.im * (ax0 + nrm)};
          tau[j] = C{tj, 0};
        }
      }
    }
    __syncthreads();
    const C vh = vhead[j];
    const R tj = tau[j].re;
    if (tj != R(0)) {
      const C* vj = Y + (size_t)j * m;
      for (int c = j + 1 + w; c < nq; c += nw) {
        C* y = Y + (size_t)c * m;
        R sr = 0, si = 0;
        for (int row = j + lane; row < m; row += 32) {
          const C vv = row == j ? vh : vj[row];
          const C yy = y[row];
          sr = fma(vv.re, yy.re, fma(vv.im, yy.im, sr));
          si = fma(vv.re, yy.im, fma(-vv.im, yy.re, si));
        }
        sr = warp_sum(sr) * tj; si = warp_sum(si) * tj;
        const C sc = {sr, si};
        for (int row = j + lane; row < m; row += 32) {
          const C vv = row == j ? vh : vj[row];
          y[row] = sub(y[row], mul(vv, sc));
        }
      }
    }
    __syncthreads();
  }
  if (Q == nullptr) return;
  for (int e = tid(); e < m * r; e += nt()) {
    const int col = e / m, row = e - col * m;
    Q[e] = C{row == col ? R(1) : R(0), 0};
  }
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    const C vh = vhead[j];
    const R tj = tau[j].re;
    if (tj != R(0)) {
      const C* vj = Y + (size_t)j * m;
      for (int c = j + w; c < r; c += nw) {
        C* qc = Q + (size_t)c * m;
        R sr = 0, si = 0;
        for (int row = j + lane; row < m; row += 32) {
          const C vv = row == j ? vh : vj[row];
          const C yy = qc[row];
          sr = fma(vv.re, yy.re, fma(vv.im, yy.im, sr));
          si = fma(vv.re, yy.im, fma(-vv.im, yy.re, si));
        }
        sr = warp_sum(sr) * tj; si = warp_sum(si) * tj;
        const C sc = {sr, si};
        for (int row = j + lane; row < m; row += 32) {
          const C vv = row == j ? vh : vj[row];
          qc[row] = sub(qc[row], mul(vv, sc));
        }
      }
    }
    __syncthreads();
  }
}

// Centre c -> c+1: A_c (2 d_c x d_{c+1}) = Q R; A_c <- Q, A_{c+1} <- R A_{c+1}.
template <typename R>
__device__ void Engine<R>::qr_right() {
  PhaseTimer pt(st, PH_QR);
  const int c = centre;
  if (c < 0 || c > a.n - 2) { fail(ST_BAD_DIM, 3000 + c); return; }
  const int dl = sm.dims[c], dr = sm.dims[c + 1], d2 = sm.dims[c + 2];
  if (!dim_ok(dl) || !dim_ok(dr) || !dim_ok(d2)) { fail(ST_BAD_DIM, 4000 + c); return; }
  const int m = 2 * dl, nq = dr, r = min(m, nq);
  C* Y = TH;
  C* Q = XG;
  const C* Ac = S(c);
  for (int e = tid(); e < m * nq; e += nt()) {
    const int row = e / nq, b = e - row * nq;
    Y[(size_t)b * m + row] = Ac[e];
  }
  __syncthreads();
  householder(Y, m, nq, Q, 0.0);
  C* Acw = S(c);
  for (int e = tid(); e < m * r; e += nt()) {
    const int row = e / r, col = e - row * r;
    Acw[e] = Q[(size_t)col * m + row];
  }
  __syncthreads();
  const C* alpha = reinterpret_cast<const C*>(sm.hh) + 4 * cap;
  const int ncol = 2 * d2;
  const C* B = S(c + 1);
  for (int e = tid(); e < r * ncol; e += nt()) {
    const int ii = e / ncol, col = e - ii * ncol;
    C s = {0, 0};
    fma_c(s, alpha[ii], B[(size_t)ii * ncol + col]);
    for (int b = ii + 1; b < nq; ++b) fma_c(s, Y[(size_t)b * m + ii], B[(size_t)b * ncol + col]);
    XG[e] = s;
  }
  __syncthreads();
  C* Bw = S(c + 1);
  for (int e = tid(); e < r * ncol; e += nt()) Bw[e] = XG[e];
  if (tid() == 0) { sm.dims[c + 1] = r; st.qr_moves++; }
  centre = c + 1;
  __syncthreads();
}

// Centre c -> c-1: A_c (d_c x 2 d_{c+1}) = L Q via A_c^H = Q' R;
// A_c <- Q'^H (right-orthonormal rows), A_{c-1} <- A_{c-1} R^H.
template <typename R>
__device__ void Engine<R>::qr_left() {
  PhaseTimer pt(st, PH_QR);
  const int c = centre;
  if (c < 1 || c > a.n - 1) { fail(ST_BAD_DIM, 5000 + c); return; }
  const int dl = sm.dims[c], dr = sm.dims[c + 1], d0 = sm.dims[c - 1];
  if (!dim_ok(dl) || !dim_ok(dr) || !dim_ok(d0)) { fail(ST_BAD_DIM, 6000 + c); return; }
  const int m = 2 * dr, nq = dl, r = min(m, nq);
  C* Y = TH;
  C* Q = XG;
  const C* Ac = S(c);
  for (int e = tid(); e < m * nq; e += nt()) { const C v = Ac[e]; Y[e] = C{v.re, -v.im}; }
  __syncthreads();
  householder(Y, m, nq, Q, 0.0);
  C* Acw = S(c);
  for (int e = tid(); e < r * m; e += nt()) { const C v = Q[e]; Acw[e] = C{v.re, -v.im}; }
  __syncthreads();
  const C* alpha = reinterpret_cast<const C*>(sm.hh) + 4 * cap;
  const int rows = 2 * d0;
  const C* Ap = S(c - 1);
  for (int e = tid(); e < rows * r; e += nt()) {
    const int row = e / r, mm = e - row * r;
    // out[row][mm] = sum_{a >= mm} A[row][a] conj(R[mm][a])
    C s = {0, 0};
    const C* ar = Ap + (size_t)row * nq;
    fma_c(s, ar[mm], C{alpha[mm].re, -alpha[mm].im});
    for (int aa = mm + 1; aa < nq; ++aa) {
      const C rv = Y[(size_t)aa * m + mm];
      fma_c(s, ar[aa], C{rv.re, -rv.im});
    }
    XG[e] = s;
  }
  __syncthreads();
  C* Apw = S(c - 1);
  for (int e = tid(); e < rows * r; e += nt()) Apw[e] = XG[e];
  if (tid() == 0) { sm.dims[c] = r; st.qr_moves++; }
  centre = c - 1;
  __syncthreads();
}

template <typename R>
__device__ void Engine<R>::move_centre(int target) {
  while (centre < target && !failed()) qr_right();
  while (centre > target && !failed()) qr_left();
}

}  // namespace tepai
