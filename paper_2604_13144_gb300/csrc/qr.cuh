// Orthogonality-centre moves of the mixed-canonical MPS by Householder QR
// (Sec. II.A: gates act on an MPS in mixed-canonical form).
#pragma once
#include "engine.cuh"

namespace tepai {

// Reflector of a column x with |x|^2 = nr2 and leading entry x_0: vhead,
// tau and alpha of H = I - tau v v^H, H x = alpha e_0. Squares, sums, |x_0|
// and the phase x_0 / |x_0| are taken in FP64 whatever R is: the square of an
// FP32 entry below about 1e-19 falls into the subnormal range and keeps only a
// few significant bits, and a norm or phase taken from it would make H
// non-unitary (tau |v|^2 != 2), so that a Q formed from it is no longer an
// isometry. In FP64 the squares of FP32 values are always exact enough. The
// reflector is skipped (tau = 0, H = I) when |x|^2 is at most tiny2 or tau
// does not fit R.
template <typename R>
__device__ __forceinline__ void reflector_params(double nr2, cplx<R> x0, double tiny2, cplx<R>& vhead,
                                                 cplx<R>& tau, cplx<R>& alpha) {
  const double xr = (double)x0.re, xi = (double)x0.im;
  const double a2 = fma(xr, xr, xi * xi);
  if constexpr (sizeof(R) == 4) {
    // FP32 square root and divisions (FP64 ones are long sequences on this
    // part) wherever |x|^2 and |x_0|^2 (unless x_0 = 0) are normal FP32 numbers
    // far from both ends of the range: then they hold full relative precision
    if (nr2 > tiny2 && nr2 >= 1e-30 && nr2 <= 1e30 && (a2 == 0.0 || a2 >= 1e-30)) {
      const float ax0 = sqrtf((float)a2), nrm = sqrtf((float)nr2);
      const float tj = 1.0f / (nrm * (nrm + ax0));
      const float pr = ax0 > 0.f ? x0.re / ax0 : 1.f, pi = ax0 > 0.f ? x0.im / ax0 : 0.f;
      alpha = cplx<R>{-pr * nrm, -pi * nrm};
      vhead = cplx<R>{pr * (ax0 + nrm), pi * (ax0 + nrm)};
      tau = cplx<R>{tj, 0};
      return;
    }
  }
  const double ax0 = sqrt(a2);
  const double nrm = sqrt(nr2);
  const double tj = 1.0 / (nrm * (nrm + ax0));
  if (!(nr2 > tiny2) || !(nrm > 0.0) || !isfinite((R)tj)) {
    vhead = cplx<R>{1, 0}; tau = cplx<R>{0, 0}; alpha = x0;
    return;
  }
  const double pr = ax0 > 0.0 ? xr / ax0 : 1.0, pi = ax0 > 0.0 ? xi / ax0 : 0.0;
  alpha = cplx<R>{(R)(-pr * nrm), (R)(-pi * nrm)};
  vhead = cplx<R>{(R)(pr * (ax0 + nrm)), (R)(pi * (ax0 + nrm))};
  tau = cplx<R>{(R)tj, 0};
}

// Reflector of column y at row j (rows j..m-1, warp-collective; lane 0 writes
// vhead[j], tau[j] and alpha[j]). In single precision |x|^2 is summed in FP32
// first: when the sum is at least 1e-30, squares that underflow change it by
// less than 1e-13 relative. Only smaller sums are taken again in FP64.
template <typename R>
__device__ __forceinline__ void householder_reflector(const cplx<R>* y, int j, int m, int lane, double tiny2,
                                                      cplx<R>* vhead, cplx<R>* tau, cplx<R>* alpha) {
  double nr2 = 0.0;
  bool done = false;
  if constexpr (sizeof(R) == 4) {
    float nf = 0.f;
    for (int row = j + lane; row < m; row += 32) nf = fmaf(y[row].re, y[row].re, fmaf(y[row].im, y[row].im, nf));
    nf = warp_sum(nf);              // the same value in every lane
    if (nf >= 1e-30f) { nr2 = (double)nf; done = true; }
  }
  if (!done) {
    for (int row = j + lane; row < m; row += 32) {
      const double re = (double)y[row].re, im = (double)y[row].im;
      nr2 = fma(re, re, fma(im, im, nr2));
    }
    nr2 = warp_sum(nr2);
  }
  if (lane == 0) reflector_params<R>(nr2, y[j], tiny2, vhead[j], tau[j], alpha[j]);
}

// Householder QR of Y (m x nq, column-major, ld m): Y = Q R with r = min(m, nq).
// Reflector j is H_j = I - tau_j v_j v_j^H, v_j = (vhead_j, Y[j+1.., j]); it maps
// the column onto alpha_j e_j with alpha_j = -e^{i arg x_0} |x|. On return the
// strict upper triangle of R is in Y, its diagonal in alpha[], and Q (m x r,
// column-major) is formed explicitly by backward accumulation unless Q is null.
// A reflector is skipped (tau = 0) when the remaining column has |x|^2 <= tiny2,
// or when tau = 1/(|x|(|x|+|x_0|)) does not fit R: an evolved state carries
// amplitudes like sin(Delta/2)^k far below 1e-19, and the scale would
// overflow FP32 (householder_reflector takes the norms themselves in FP64).
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::householder(C* Y, int m, int nq, C* Q, double tiny2) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int r = min(m, nq);
  C* vhead = reinterpret_cast<C*>(sm.hh);
  C* tau = vhead + 2 * cap;
  C* alpha = tau + 2 * cap;
  {
  SubTimer spt(st, SP_QR_PANEL);
  for (int j = 0; j < r; ++j) {
    if (w == 0) householder_reflector<R>(Y + (size_t)j * m, j, m, lane, tiny2, vhead, tau, alpha);
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
  }
  if (Q == nullptr) return;
  SubTimer sqt(st, SP_QR_FORMQ);
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
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::qr_right() {
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
  qr_factor(Y, m, nq, Q, 0.0);
  if (failed()) return;
  SubTimer smt(st, SP_QR_RMUL);
  C* Acw = S(c);
  for (int e = tid(); e < m * r; e += nt()) {
    const int row = e / r, col = e - row * r;
    Acw[e] = ldcg_c(Q + (size_t)col * m + row);
  }
  __syncthreads();
  const C* alpha = reinterpret_cast<const C*>(sm.hh) + 4 * cap;
  const int ncol = 2 * d2;
  const C* B = S(c + 1);
  C* out = XG;
  if (a.smem_x_elems >= gemm_tile_elems(nt())) {
    // R (upper triangle in Y above the diagonal, diagonal in alpha) times A_{c+1}
    const C* yp = Y;
    block_gemm<R>(r, ncol, nq, reinterpret_cast<C*>(sm.x),
        [=](int ii, int kk) {
          return kk < ii ? C{0, 0} : (kk == ii ? alpha[ii] : ldcg_c(yp + (size_t)kk * m + ii));
        },
        [=](int kk, int jj) { return B[(size_t)kk * ncol + jj]; },
        [=](int ii, int jj, C v) { out[(size_t)ii * ncol + jj] = v; });
  } else {
    for (int e = tid(); e < r * ncol; e += nt()) {
      const int ii = e / ncol, col = e - ii * ncol;
      C s = {0, 0};
      fma_c(s, alpha[ii], B[(size_t)ii * ncol + col]);
      for (int b = ii + 1; b < nq; ++b) fma_c(s, ldcg_c(Y + (size_t)b * m + ii), B[(size_t)b * ncol + col]);
      XG[e] = s;
    }
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
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::qr_left() {
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
  qr_factor(Y, m, nq, Q, 0.0);
  if (failed()) return;
  SubTimer smt(st, SP_QR_RMUL);
  C* Acw = S(c);
  for (int e = tid(); e < r * m; e += nt()) { const C v = ldcg_c(Q + e); Acw[e] = C{v.re, -v.im}; }
  __syncthreads();
  const C* alpha = reinterpret_cast<const C*>(sm.hh) + 4 * cap;
  const int rows = 2 * d0;
  const C* Ap = S(c - 1);
  C* out = XG;
  if (a.smem_x_elems >= gemm_tile_elems(nt())) {
    // A_{c-1} times R^H (R: upper triangle in Y above the diagonal, diagonal in alpha)
    const C* yp = Y;
    block_gemm<R>(rows, r, nq, reinterpret_cast<C*>(sm.x),
        [=](int ii, int kk) { return Ap[(size_t)ii * nq + kk]; },
        [=](int kk, int jj) {
          if (kk < jj) return C{0, 0};
          const C u = kk == jj ? alpha[jj] : ldcg_c(yp + (size_t)kk * m + jj);
          return C{u.re, -u.im};
        },
        [=](int ii, int jj, C v) { out[(size_t)ii * r + jj] = v; });
  } else {
    for (int e = tid(); e < rows * r; e += nt()) {
      const int row = e / r, mm = e - row * r;
      // out[row][mm] = sum_{a >= mm} A[row][a] conj(R[mm][a])
      C s = {0, 0};
      const C* ar = Ap + (size_t)row * nq;
      fma_c(s, ar[mm], C{alpha[mm].re, -alpha[mm].im});
      for (int aa = mm + 1; aa < nq; ++aa) {
        const C rv = ldcg_c(Y + (size_t)aa * m + mm);
        fma_c(s, ar[aa], C{rv.re, -rv.im});
      }
      XG[e] = s;
    }
  }
  __syncthreads();
  C* Apw = S(c - 1);
  for (int e = tid(); e < rows * r; e += nt()) Apw[e] = XG[e];
  if (tid() == 0) { sm.dims[c] = r; st.qr_moves++; }
  centre = c - 1;
  __syncthreads();
}

template <typename R, bool TC>
__device__ void Engine<R, TC>::move_centre(int target) {
  while (centre < target && !failed()) qr_right();
  while (centre > target && !failed()) qr_left();
}

}  // namespace tepai

namespace tepai {

// Compact WY factor of the panel (Schreiber & Van Loan, SIAM J. Sci. Stat.
// Comput. 10, 1989): H_{j0} ... H_{j0+bp-1} = I - V T V^H with T upper
// triangular, T_kk = tau_k, T_{0:k,k} = -tau_k T_{0:k,0:k} (V_{:,0:k}^H v_k).
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::panel_t(const C* V, int m, int j0, int bp, C* T) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const C* tau = reinterpret_cast<const C*>(sm.hh) + 2 * cap;
  // z_{k,jj} = V_{:,k}^H v_jj for k < jj, stored in T[k][jj] (T row-major 16 x 16)
  for (int e = w; e < bp * bp; e += nw) {
    const int k = e / bp, jj = e - k * bp;
    if (k >= jj) continue;
    const C* vk = V + (size_t)k * m;
    const C* vj = V + (size_t)jj * m;
    R sr = 0, si = 0;
    for (int row = j0 + jj + lane; row < m; row += 32) {
      const C a = vk[row], b = vj[row];
      sr = fma(a.re, b.re, fma(a.im, b.im, sr));
      si = fma(a.re, b.im, fma(-a.im, b.re, si));
    }
    sr = warp_sum(sr); si = warp_sum(si);
    if (lane == 0) T[k * 16 + jj] = C{sr, si};
  }
  __syncthreads();
  // Column jj needs the finished columns < jj of T and the raw z column jj, so
  // one warp forms it with lane k computing row k; the sum over q runs in the
  // same order as a serial loop would take it.
  if (w == 0) {
    const int k = lane;
    for (int jj = 0; jj < bp; ++jj) {
      const R tj = tau[j0 + jj].re;
      C acc = {0, 0};
      if (k < jj)
        for (int q = k; q < jj; ++q) fma_c(acc, T[k * 16 + q], T[q * 16 + jj]);
      __syncwarp();
      if (k < jj) T[k * 16 + jj] = C{-tj * acc.re, -tj * acc.im};
      else if (k == jj) T[k * 16 + jj] = C{tj, 0};
      else if (k < 16) T[k * 16 + jj] = C{0, 0};
      __syncwarp();
    }
  }
  __syncthreads();
}

// Single-precision compute of one block-reflector chunk (cb <= 16 columns of
// C in shared memory, m = 32 RPL rows at most): W = V^H C, W <- op(T) W,
// C <- C - V W. For W, warp w keeps the rows of reflectors k = w and w + nw in
// registers across the chunk's columns and forms both inner products with
// paired FP32 FMA; the update gives each thread a 4 x 4 block of (rows,
// columns) so that every loaded V or W element feeds four products.
template <int RPL>
__device__ __noinline__ void apply_chunk_f32(const float2* V, int m, int bp, const float2* T, bool herm,
                                             float2* ch, int cb, float2* Wm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float2 zero = make_float2(0.f, 0.f);
  for (int k0 = w; k0 < bp; k0 += 2 * nw) {
    const int k1 = k0 + nw;
    const bool has1 = k1 < bp;
    float2 v0[RPL], v1[RPL];
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int row = lane + 32 * t;
      v0[t] = row < m ? V[(size_t)k0 * m + row] : zero;
      v1[t] = (has1 && row < m) ? V[(size_t)k1 * m + row] : zero;
    }
    for (int c = 0; c < cb; ++c) {
      const float2* x = ch + (size_t)c * m;
      float2 r0 = zero, i0 = zero, r1 = zero, i1 = zero;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int row = lane + 32 * t;
        const float2 xv = row < m ? x[row] : zero;
        const float2 xs = make_float2(xv.y, xv.x);
        // conj(v) x = (v.re x.re + v.im x.im) + i (v.re x.im - v.im x.re)
        r0 = __ffma2_rn(v0[t], xv, r0);
        i0 = __ffma2_rn(v0[t], xs, i0);
        r1 = __ffma2_rn(v1[t], xv, r1);
        i1 = __ffma2_rn(v1[t], xs, i1);
      }
      float s4[4] = {r0.x + r0.y, i0.x - i0.y, r1.x + r1.y, i1.x - i1.y};
      warp_sum4<float>(s4, lane);
      if (lane == 0) {
        Wm[k0 * 16 + c] = make_float2(s4[0], s4[1]);
        if (has1) Wm[k1 * 16 + c] = make_float2(s4[2], s4[3]);
      }
    }
  }
  __syncthreads();
  // W2 = op(T) W, kept in registers of threads (k, c), then written back
  float2 w2 = zero;
  const int kk = threadIdx.x / 16, cc = threadIdx.x % 16;
  const bool act = threadIdx.x < 256 && kk < bp && cc < cb;
  if (act) {
    cplx<float> acc = {0.f, 0.f};
    const cplx<float>* Tc = reinterpret_cast<const cplx<float>*>(T);
    const cplx<float>* Wc = reinterpret_cast<const cplx<float>*>(Wm);
    if (herm) {
      for (int q = 0; q <= kk; ++q) fma_cc(acc, Tc[q * 16 + kk], Wc[q * 16 + cc]);
    } else {
      for (int q = kk; q < bp; ++q) fma_c(acc, Tc[kk * 16 + q], Wc[q * 16 + cc]);
    }
    w2 = make_float2(acc.re, acc.im);
  }
  __syncthreads();
  if (act) Wm[kk * 16 + cc] = w2;
  __syncthreads();
  // C <- C - V W: item (rbase, column group) covers rows rbase + R4 i (i < 4)
  // and columns 4 g .. 4 g + 3
  const int R4 = (m + 3) / 4, ng = (cb + 3) / 4;
  for (int e = threadIdx.x; e < R4 * ng; e += blockDim.x) {
    const int g = e / R4, rbase = e - g * R4;
    float accr[4][4], acci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { accr[i][j] = 0.f; acci[i][j] = 0.f; }
    for (int k = 0; k < bp; ++k) {
      float2 vv[4], ww[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int row = rbase + R4 * i;
        vv[i] = row < m ? V[(size_t)k * m + row] : zero;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) ww[j] = Wm[k * 16 + 4 * g + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accr[i][j] = fmaf(vv[i].x, ww[j].x, fmaf(-vv[i].y, ww[j].y, accr[i][j]));
          acci[i][j] = fmaf(vv[i].x, ww[j].y, fmaf(vv[i].y, ww[j].x, acci[i][j]));
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int row = rbase + R4 * i;
      if (row >= m) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = 4 * g + j;
        if (c < cb) {
          float2 x = ch[(size_t)c * m + row];
          x.x -= accr[i][j];
          x.y -= acci[i][j];
          ch[(size_t)c * m + row] = x;
        }
      }
    }
  }
}

// Apply I - V op(T) V^H to columns [c0, c1) of the global matrix G (ld m),
// rows j0..m-1, in shared-memory chunks of 16 columns: W = V^H C,
// W <- op(T) W (T^H when herm), C <- C - V W. V is dense in shared memory
// (V[k*m + row], zero above its diagonal, vhead on it). Chunks move by bulk
// copies; with a second chunk buffer CH1 the load of chunk i+1 overlaps the
// update of chunk i. Starts and ends with every earlier bulk store drained.
template <typename R, bool TC>
__device__ void Engine<R, TC>::apply_block_reflector(const C* V, int m, int j0, int bp, const C* T, bool herm,
                                                 C* G, int c0, int c1, C* CH, C* CH1, C* Wm) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int nch = (c1 - c0 + 15) / 16;
  const bool dbl = CH1 != nullptr;
  C* buf[2] = {CH, dbl ? CH1 : CH};
  auto bytes_of = [&](int ci) { return (uint32_t)(sizeof(C) * min(16, c1 - c0 - 16 * ci) * m); };
  bulk_drain();
  int pend = 0;
  if (nch > 0) {
    bulk_issue_load(1, buf[0], G + (size_t)c0 * m, bytes_of(0));
    pend = 2;
  }
  for (int ci = 0; ci < nch; ++ci) {
    const int b = dbl ? (ci & 1) : 0;
    const int cs = c0 + 16 * ci;
    const int cb = min(16, c1 - cs);
    C* ch = buf[b];
    if (dbl && ci + 1 < nch) {
      bulk_wait_store_read();  // the store of chunk ci-1 has read buf[b^1]
      bulk_issue_load(1 + (b ^ 1), buf[b ^ 1], G + (size_t)(cs + 16) * m, bytes_of(ci + 1));
      pend |= 2 << (b ^ 1);
    }
    bulk_wait_load(1 + b, bytes_of(ci));
    pend &= ~(2 << b);
    if (failed()) { bulk_settle(pend); bulk_drain(); return; }
    bool done = false;
    if constexpr (sizeof(R) == 4) {
      const float2* Vf = reinterpret_cast<const float2*>(V);
      const float2* Tf = reinterpret_cast<const float2*>(T);
      float2* chf = reinterpret_cast<float2*>(ch);
      float2* Wf = reinterpret_cast<float2*>(Wm);
      done = true;
      if (m <= 64) apply_chunk_f32<2>(Vf, m, bp, Tf, herm, chf, cb, Wf);
      else if (m <= 128) apply_chunk_f32<4>(Vf, m, bp, Tf, herm, chf, cb, Wf);
      else if (m <= 256) apply_chunk_f32<8>(Vf, m, bp, Tf, herm, chf, cb, Wf);
      else done = false;
    }
    if (!done) {
    for (int e = w; e < bp * cb; e += nw) {
      const int k = e / cb, c = e - k * cb;
      const C* vk = V + (size_t)k * m;
      const C* x = ch + (size_t)c * m;
      R sr = 0, si = 0;
      for (int row = j0 + k + lane; row < m; row += 32) {
        const C a = vk[row], bb = x[row];
        sr = fma(a.re, bb.re, fma(a.im, bb.im, sr));
        si = fma(a.re, bb.im, fma(-a.im, bb.re, si));
      }
      sr = warp_sum(sr); si = warp_sum(si);
      if (lane == 0) Wm[k * 16 + c] = C{sr, si};
    }
    __syncthreads();
    // W2 = op(T) W, kept in registers of threads (k, c), then written back
    C w2 = {0, 0};
    const int kk = tid() / 16, cc = tid() % 16;
    const bool act = tid() < 256 && kk < bp && cc < cb;
    if (act) {
      if (herm) {
        for (int q = 0; q <= kk; ++q) fma_cc(w2, T[q * 16 + kk], Wm[q * 16 + cc]);
      } else {
        for (int q = kk; q < bp; ++q) fma_c(w2, T[kk * 16 + q], Wm[q * 16 + cc]);
      }
    }
    __syncthreads();
    if (act) Wm[kk * 16 + cc] = w2;
    __syncthreads();
    for (int e = tid(); e < cb * m; e += nt()) {
      const int c = e / m, row = e - c * m;
      if (row < j0) continue;
      C x = ch[(size_t)c * m + row];
      const int kmax = min(bp, row - j0 + 1);
      for (int k = 0; k < kmax; ++k) {
        const C vk = V[(size_t)k * m + row];
        const C wv = Wm[k * 16 + c];
        x.re -= vk.re * wv.re - vk.im * wv.im;
        x.im -= vk.re * wv.im + vk.im * wv.re;
      }
      ch[(size_t)c * m + row] = x;
    }
    }
    bulk_issue_store(G + (size_t)cs * m, ch, bytes_of(ci));
    if (!dbl && ci + 1 < nch) {
      bulk_wait_store_read();
      bulk_issue_load(1, buf[0], G + (size_t)(cs + 16) * m, bytes_of(ci + 1));
      pend |= 2;
    }
  }
  bulk_drain();
}

// Turn the factored panel in P (rows >= j0 of columns j0..j0+bp-1) into the
// dense reflector block V: zero above each diagonal, vhead on it.
template <typename R>
__device__ __forceinline__ void densify_panel(cplx<R>* P, const cplx<R>* vhead, int m, int j0, int bp) {
  for (int e = threadIdx.x; e < bp * m; e += blockDim.x) {
    const int k = e / m, row = e - k * m;
    const int d = j0 + k;
    if (row < d) P[e] = cplx<R>{0, 0};
    else if (row == d) P[e] = vhead[d];
  }
  __syncthreads();
}

// Blocked Householder QR of Y (m x nq, column-major, global memory): 16-column
// panels are factored in shared memory, then the trailing columns are updated
// with the panel's block reflector. Same output convention as householder().
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::householder_blocked(C* Y, int m, int nq, C* Q, double tiny2) {
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  const int r = min(m, nq);
  C* vhead = reinterpret_cast<C*>(sm.hh);
  C* tau = vhead + 2 * cap;
  C* alpha = tau + 2 * cap;
  // staging: panel P, one or two update chunks, T and W (16 x 16 each)
  const bool dbl = (size_t)m * 48 + 512 <= (size_t)a.smem_x_elems;
  C* P = reinterpret_cast<C*>(sm.x);
  C* CH = P + (size_t)m * 16;
  C* CH1 = dbl ? CH + (size_t)m * 16 : nullptr;
  C* T = CH + (size_t)m * (dbl ? 32 : 16);
  C* Wm = T + 256;
  for (int j0 = 0; j0 < r && !failed(); j0 += 16) {
    const int bp = min(16, r - j0);
    SubTimer spt(st, SP_QR_PANEL);
    bulk_load(P, Y + (size_t)j0 * m, (uint32_t)(sizeof(C) * bp * m));
    if (failed()) return;
    for (int jj = 0; jj < bp; ++jj) {
      const int j = j0 + jj;
      if (w == 0) householder_reflector<R>(P + (size_t)jj * m, j, m, lane, tiny2, vhead, tau, alpha);
      __syncthreads();
      const C vh = vhead[j];
      const R tj = tau[j].re;
      if (tj != R(0)) {
        const C* vj = P + (size_t)jj * m;
        for (int c = jj + 1 + w; c < bp; c += nw) {
          C* y = P + (size_t)c * m;
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
    bulk_store(Y + (size_t)j0 * m, P, (uint32_t)(sizeof(C) * bp * m));
    if (j0 + bp < nq) {
      densify_panel(P, vhead, m, j0, bp);
      panel_t(P, m, j0, bp, T);
      spt.stop();  // the trailing update is counted apart from the panel
      SubTimer sat(st, SP_QR_APPLY);
      apply_block_reflector(P, m, j0, bp, T, true, Y, j0 + bp, nq, CH, CH1, Wm);
    }
  }
  if (Q == nullptr) return;
  SubTimer sqt(st, SP_QR_FORMQ);
  for (int e = tid(); e < m * r; e += nt()) {
    const int col = e / m, row = e - col * m;
    Q[e] = C{row == col ? R(1) : R(0), 0};
  }
  __syncthreads();
  const int last = ((r - 1) / 16) * 16;
  for (int j0 = last; j0 >= 0 && !failed(); j0 -= 16) {
    const int bp = min(16, r - j0);
    bulk_load(P, Y + (size_t)j0 * m, (uint32_t)(sizeof(C) * bp * m));
    if (failed()) return;
    densify_panel(P, vhead, m, j0, bp);
    panel_t(P, m, j0, bp, T);
    apply_block_reflector(P, m, j0, bp, T, false, Q, j0, r, CH, CH1, Wm);
  }
  (void)alpha;
}

// The triangle-on-triangle step of a two-level QR: the R factor of
// S = [T; B], where T and B are n x n upper-triangular (column-major, leading
// dimension ld, diagonal included in the arrays; entries below the diagonal
// are ignored). Column j's reflector (householder_reflector's convention)
// maps (T[j][j], B[0..j][j]) onto alpha_j e_j: every other entry of that
// column of S is zero, so step j costs O(j (n - j)) instead of O((2n - j)(n - j)).
// On return the strict upper triangle of R is in T and its diagonal in the
// alpha array (sm.hh + 4 cap), as householder() leaves them.
template <typename R, bool TC>
__device__ __noinline__ void Engine<R, TC>::ts_combine(C* Tm, C* Bm, int ld, int n, double tiny2) {
  SubTimer spt(st, SP_QR_PANEL);
  const int lane = tid() & 31, w = tid() >> 5, nw = nt() >> 5;
  C* vhead = reinterpret_cast<C*>(sm.hh);
  C* tau = vhead + 2 * cap;
  C* alpha = tau + 2 * cap;
  for (int j = 0; j < n; ++j) {
    const C* bj = Bm + (size_t)j * ld;
    if (w == 0) {
      double nr2 = 0.0;
      for (int b = lane; b <= j; b += 32) {
        const double re = (double)bj[b].re, im = (double)bj[b].im;
        nr2 = fma(re, re, fma(im, im, nr2));
      }
      const C x0 = Tm[(size_t)j * ld + j];
      if (lane == 0) nr2 += fma((double)x0.re, (double)x0.re, (double)x0.im * (double)x0.im);
      nr2 = warp_sum(nr2);
      if (lane == 0) reflector_params<R>(nr2, x0, tiny2, vhead[j], tau[j], alpha[j]);
    }
    __syncthreads();
    const C vh = vhead[j];
    const R tj = tau[j].re;
    if (tj != R(0)) {
      for (int c = j + 1 + w; c < n; c += nw) {
        C* tcol = Tm + (size_t)c * ld;
        C* bc = Bm + (size_t)c * ld;
        R sr = 0, si = 0;
        if (lane == 0) {
          const C yy = tcol[j];
          sr = vh.re * yy.re + vh.im * yy.im;
          si = vh.re * yy.im - vh.im * yy.re;
        }
        for (int b = lane; b <= j; b += 32) {
          const C vv = bj[b], yy = bc[b];
          sr = fma(vv.re, yy.re, fma(vv.im, yy.im, sr));
          si = fma(vv.re, yy.im, fma(-vv.im, yy.re, si));
        }
        sr = warp_sum(sr) * tj; si = warp_sum(si) * tj;
        const C sc = {sr, si};
        if (lane == 0) tcol[j] = sub(tcol[j], mul(vh, sc));
        for (int b = lane; b <= j; b += 32) bc[b] = sub(bc[b], mul(bj[b], sc));
      }
    }
    __syncthreads();
  }
}

}  // namespace tepai
