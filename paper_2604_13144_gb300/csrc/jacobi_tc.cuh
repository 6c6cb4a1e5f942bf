// Blocked one-sided Jacobi SVD on the tensor cores (single precision, working
// matrix X staged in global memory, m <= 256 rows, CTAs of 256 threads, two
// per SM).
//
// Same method as Engine::jacobi (Hestenes' one-sided Jacobi: rotate column
// pairs until every pair is orthogonal to tol * |x_p| |x_q|), with the column
// pairs visited block pair by block pair. For blocks I and J of 32 columns,
// P = [X_I X_J] (m x 64 complex):
//   1. G = P^H P, the 64 x 64 Gram matrix of the pair, on tcgen05 (3xTF32,
//      FP32 accumulators in TMEM): the real GEMM Pt^T Pt, where row 2x + c of
//      Pt^T holds the real (c = 0) or imaginary (c = 1) part of column x.
//   2. The pairs (p in I, q in J), and the pairs inside I (inside J) when I
//      (J) is met for the first time in the sweep, are rotated in parallel
//      rounds of disjoint pairs. A rotation is decided from G exactly as the
//      column Jacobi decides it from inner products, and is applied to G on
//      both sides (G <- J^H G J) and accumulated into V (V <- V J).
//   3. If any pair rotated, P <- P V on tcgen05 (3xTF32) and P is written back.
// A sweep visits every pair once; sweeps stop when one rotates nothing. The
// convergence decision is therefore taken on Gram matrices computed afresh
// from the current columns, at the start of each block pair.
//
// Shared memory (inside the staging area sm.x): one operand stage (A hi,
// A lo, B hi, B lo of 128 x KT FP32, K-major core-matrix layout of tc.cuh),
// G (64 x 64 complex, row stride TcJac::GS) and V (64 x 64 complex). TMEM:
// 128 FP32 columns x 128 lanes.
#pragma once
#include "tc_gemm.cuh"

namespace tepai {

// Gram operand, one chunk: tile row 2x + c is the real (c = 0) or imaginary
// (c = 1) part of local column x (0..63), tile column k is row k0 + k of X.
// A warp task fills two K-adjacent core matrices (4 columns x 8 rows of X):
// lane (h, xx, kk) = (lane >> 4, (lane >> 2) & 3, lane & 3) loads the complex
// X[col(4 rg + xx)][k0 + 4 (kg + h) + kk] once and writes its two parts to
// core rows 2 xx and 2 xx + 1. The half-warps write the two parts in opposite
// order, so every store instruction covers the 32 banks once.
template <class COL>
__device__ __forceinline__ void stage_gram(float* hi, float* lo, const float2* X, int m, int k0, COL col) {
  constexpr int CK = TcJac::KT / 4, TASKS = 16 * (CK / 2), PER = 4;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int h = lane >> 4, xx = (lane >> 2) & 3, kk = lane & 3;
  for (int t0 = w; t0 < TASKS; t0 += nw * PER) {
    float2 v[PER];
    int off[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int t = t0 + u * nw;
      v[u] = make_float2(0.f, 0.f);
      off[u] = -1;
      if (t < TASKS) {
        const int rg = t / (CK / 2), kg = 2 * (t % (CK / 2)) + h;
        const int cx = col(4 * rg + xx), k = k0 + 4 * kg + kk;
        if (cx >= 0 && k < m) v[u] = __ldcg(X + (size_t)cx * m + k);
        off[u] = (rg * CK + kg) * 32 + 8 * xx + kk;
      }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (off[u] < 0) continue;
      const float a = h ? v[u].y : v[u].x, b = h ? v[u].x : v[u].y;
      const int oa = off[u] + (h ? 4 : 0), ob = off[u] + (h ? 0 : 4);
      const float ah = tc::tf32_rna(a), bh = tc::tf32_rna(b);
      hi[oa] = ah; hi[ob] = bh;
      lo[oa] = tc::tf32_rna(a - ah); lo[ob] = tc::tf32_rna(b - bh);
    }
  }
}

// Block-update A operand, one chunk: tile row i is row r0 + i of P, tile
// column k = 2 x' + c the real or imaginary part of local column x0 + x'. A
// warp task fills two M-adjacent core matrices (16 rows x 2 columns of X):
// lane (h, ii, xx) = (lane >> 4, (lane >> 1) & 7, lane & 1) loads the complex
// X[col(x0 + 2 kg + xx)][r0 + 8 (2 rgp + h) + ii] once; half-warps again
// write the two parts in opposite order.
template <class COL>
__device__ __forceinline__ void stage_update_a(float* hi, float* lo, const float2* X, int m, int r0, int x0,
                                               COL col) {
  constexpr int CK = TcJac::KT / 4, TASKS = 8 * CK, PER = 4;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int h = lane >> 4, ii = (lane >> 1) & 7, xx = lane & 1;
  for (int t0 = w; t0 < TASKS; t0 += nw * PER) {
    float2 v[PER];
    int off[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int t = t0 + u * nw;
      v[u] = make_float2(0.f, 0.f);
      off[u] = -1;
      if (t < TASKS) {
        const int rg = 2 * (t / CK) + h, kg = t % CK;
        const int row = r0 + 8 * rg + ii, cx = col(x0 + 2 * kg + xx);
        if (cx >= 0 && row < m) v[u] = __ldcg(X + (size_t)cx * m + row);
        off[u] = (rg * CK + kg) * 32 + 4 * ii + 2 * xx;
      }
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      if (off[u] < 0) continue;
      const float a = h ? v[u].y : v[u].x, b = h ? v[u].x : v[u].y;
      const int oa = off[u] + (h ? 1 : 0), ob = off[u] + (h ? 0 : 1);
      const float ah = tc::tf32_rna(a), bh = tc::tf32_rna(b);
      hi[oa] = ah; hi[ob] = bh;
      lo[oa] = tc::tf32_rna(a - ah); lo[ob] = tc::tf32_rna(b - bh);
    }
  }
}

// Jacobi sweeps on X (m x nc complex FP32, column-major, global memory,
// 32 < nc <= 256, m <= 256) through the tensor cores, by a CTA of exactly 8
// warps (TcJac::THREADS); tol and thr as in Engine::jacobi. Returns the number of sweeps; sets
// ibuf[1] = 1 on convergence.
template <typename R, bool TC>
__device__ __noinline__ int Engine<R, TC>::jacobi_tc(C* X, int m, int nc, R tol, R thr) {
  float2* Xf = reinterpret_cast<float2*>(X);
  unsigned char* xs = reinterpret_cast<unsigned char*>(sm.x);
  float2* G = reinterpret_cast<float2*>(xs + TcJac::G_OFF);
  float2* V = reinterpret_cast<float2*>(xs + TcJac::V_OFF);
  constexpr int GS = TcJac::GS;
  const int lane = tid() & 31, w = tid() >> 5;
  const int nb = (nc + 31) / 32;
  const int ntiles = (m + 127) / 128;
  const uint32_t tq = tmem + ((uint32_t)((w & 3) * 32) << 16);   // this warp's TMEM lane quarter
  int sweep = 0, prev_rot = 1 << 30;   // no stall test before the second sweep
  while (sweep < a.max_sweeps && !failed()) {
    if (tid() == 0) { sm.ibuf[0] = 0; sm.ibuf[6] = 0; }
    __syncthreads();
    for (int I = 0; I < nb - 1 && !failed(); ++I) {
      for (int J = I + 1; J < nb && !failed(); ++J) {
        const int nI = min(32, nc - I * 32), nJ = min(32, nc - J * 32);
        const bool intI = J == I + 1, intJ = J == nb - 1 && I == nb - 2;
        // local column x (0..63) -> column of X, or -1 when padding
        auto col = [=](int x) { return x < 32 ? (x < nI ? I * 32 + x : -1) : (x - 32 < nJ ? J * 32 + x - 32 : -1); };
        // 1. Gram matrix of the pair
        SubTimer t_gram(st, SP_TC_GRAM);
        tc_pipeline(128, (m + TcJac::KT - 1) / TcJac::KT, true,
                    [&](int c, float* Ahi, float* Alo, float*, float*) {
                      stage_gram(Ahi, Alo, Xf, m, c * TcJac::KT, col);
                    });
        t_gram.stop();
        if (failed()) return sweep;
        // G[p][q] = Gt[2p][2q] + Gt[2p+1][2q+1] + i (Gt[2p][2q+1] - Gt[2p+1][2q]): rows 2p and
        // 2p + 1 are neighbouring lanes; even lanes finish q = 4 cg, 4 cg + 1 and
        // odd lanes 4 cg + 2, 4 cg + 3 of each 8-column group cg
        SubTimer t_asm(st, SP_TC_ASSEMBLE);
        {
          const int p = (w & 3) * 16 + (lane >> 1);
          const bool odd = lane & 1;
          for (int cg = w >> 2; cg < 16; cg += 2) {
            float v[8], u[8];
            tc::ld8(tq + (uint32_t)(cg * 8), v);
#pragma unroll
            for (int j = 0; j < 8; ++j) u[j] = __shfl_xor_sync(0xffffffffu, v[j], 1);
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
              // columns 2q, 2q + 1 of this group: 2qq, 2qq + 1 (even lanes) or 2qq + 4, 2qq + 5 (odd lanes)
              const float ere = odd ? u[2 * qq + 4] : v[2 * qq], eim = odd ? u[2 * qq + 5] : v[2 * qq + 1];  // row 2p
              const float ore = odd ? v[2 * qq + 4] : u[2 * qq], oim = odd ? v[2 * qq + 5] : u[2 * qq + 1];  // row 2p + 1
              G[p * GS + cg * 4 + qq + (odd ? 2 : 0)] = make_float2(ere + oim, eim - ore);
            }
          }
        }
        for (int e = tid(); e < 64 * 64; e += nt()) V[e] = make_float2((e >> 6) == (e & 63) ? 1.f : 0.f, 0.f);
        tc::fence_before();
        __syncthreads();
        t_asm.stop();
        // 2. rounds of disjoint pairs: the internal rounds first (Brent & Luk
        // order on 32 columns), then 32 cross rounds (p, 32 + (p + r) mod 32).
        // Every warp decides all 32 rotations of a round (lane t: pair t) from
        // the same G, so the decisions agree across warps without being shared.
        // After a barrier, warp w applies the rotations to the 2 x 2 blocks
        // (pairs 4w .. 4w + 3) x (pair lane) of G and to rows 8w .. 8w + 7 of V
        // in pair lane; a second barrier ends the round.
        SubTimer t_rounds(st, SP_TC_ROUNDS);
        int rot_pair = 0;
        const int n_int = (intI || intJ) ? 31 : 0;
        // When no pair of this visit passes the rotation test on the fresh G, no
        // round can rotate (rounds only change G through rotations): skip them,
        // counting the pairs as examined.
        bool any = false;
        for (int e = tid(); e < 64 * 64; e += nt()) {
          const int p = e >> 6, q = e & 63;
          const bool cross = p < 32 && q >= 32;
          const bool inner = p < q && ((p < 32 && q < 32 && intI) || (p >= 32 && intJ));
          if (!(cross || inner) || col(p) < 0 || col(q) < 0) continue;
          const float2 g = G[p * GS + q];
          const float al = G[p * GS + p].x, be = G[q * GS + q].x;
          if (al < thr || be < thr) continue;
          // 0.9 tol: a borderline pair is left to the rounds' own test
          any = any || fmaf(g.x, g.x, g.y * g.y) > 0.81f * tol * tol * al * be;
        }
        if (!__syncthreads_or(any)) {
          if (tid() == 0) {
            const int ni = intI ? nI * (nI - 1) / 2 : 0, nj = intJ ? nJ * (nJ - 1) / 2 : 0;
            sm.ibuf[6] += nI * nJ + ni + nj;
          }
          continue;
        }
        for (int rr = 0; rr < n_int + 32; ++rr) {
          int p = -1, q = -1;
          if (rr < n_int) {
            const int tt = lane & 15;
            const int pa = tt == 0 ? 31 : (rr + tt) % 31, qa = tt == 0 ? rr : (rr - tt + 31) % 31;
            if (lane < 16 && intI) { p = pa; q = qa; }
            if (lane >= 16 && intJ) { p = 32 + pa; q = 32 + qa; }
          } else {
            p = lane;
            q = 32 + ((lane + rr - n_int) & 31);
          }
          const bool valid = p >= 0 && col(p) >= 0 && col(q) >= 0;
          // an idle slot takes the identity on (2 lane, 2 lane + 1): slots 0..15
          // then cover block I and 16..31 block J, so a round's pairs always
          // partition the 64 local columns
          if (p < 0) { p = 2 * lane; q = p + 1; }
          float c = 1.f, s = 0.f, er = 1.f, ei = 0.f;
          bool rot = false;
          if (valid) {
            const float2 g = G[p * GS + q];
            rot = rot_params<float>(G[p * GS + p].x, G[q * GS + q].x, g.x, g.y, tol, thr, c, s, er, ei);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, rot);
          const unsigned chk = __ballot_sync(0xffffffffu, valid);
          if (tid() == 0) sm.ibuf[6] += __popc(chk);
          // every warp has read the G entries its decisions need before any warp
          // writes G in this round; the barrier also makes the skip of a round
          // without rotations one decision of the whole CTA
          if (!__syncthreads_or(bal != 0)) continue;
          rot_pair += __popc(bal);
          const int pb = p, qb = q;
          // the four blocks (pairs 4w + hh) x (pair lane) are disjoint: they are
          // taken two at a time, both loaded before either is written
#pragma unroll
          for (int h0 = 0; h0 < 4; h0 += 2) {
          float2 bk[2][4];
          float ca[2], sa[2], era[2], eia[2];
          int pa[2], qa[2];
          bool act[2];
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int a2 = 4 * w + h0 + hh;
            ca[hh] = __shfl_sync(0xffffffffu, c, a2);
            sa[hh] = __shfl_sync(0xffffffffu, s, a2);
            era[hh] = __shfl_sync(0xffffffffu, er, a2);
            eia[hh] = __shfl_sync(0xffffffffu, ei, a2);
            pa[hh] = __shfl_sync(0xffffffffu, p, a2);
            qa[hh] = __shfl_sync(0xffffffffu, q, a2);
            act[hh] = ((bal >> a2) & 1) || rot;
            if (act[hh]) {
              bk[hh][0] = G[pa[hh] * GS + pb]; bk[hh][1] = G[pa[hh] * GS + qb];
              bk[hh][2] = G[qa[hh] * GS + pb]; bk[hh][3] = G[qa[hh] * GS + qb];
            }
          }
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            if (!act[hh]) continue;
            const float2 b00 = bk[hh][0], b01 = bk[hh][1], b10 = bk[hh][2], b11 = bk[hh][3];
            // T = B J_b: T[:,0] = c B[:,0] - s e B[:,1]; T[:,1] = s B[:,0] + c e B[:,1]
            const float2 w01 = make_float2(er * b01.x - ei * b01.y, er * b01.y + ei * b01.x);
            const float2 w11 = make_float2(er * b11.x - ei * b11.y, er * b11.y + ei * b11.x);
            const float2 t00 = make_float2(c * b00.x - s * w01.x, c * b00.y - s * w01.y);
            const float2 t01 = make_float2(s * b00.x + c * w01.x, s * b00.y + c * w01.y);
            const float2 t10 = make_float2(c * b10.x - s * w11.x, c * b10.y - s * w11.y);
            const float2 t11 = make_float2(s * b10.x + c * w11.x, s * b10.y + c * w11.y);
            // new = J_a^H T: row 0 = ca T[0,:] - sa conj(ea) T[1,:]; row 1 = sa T[0,:] + ca conj(ea) T[1,:]
            const float2 u10 = make_float2(era[hh] * t10.x + eia[hh] * t10.y, era[hh] * t10.y - eia[hh] * t10.x);
            const float2 u11 = make_float2(era[hh] * t11.x + eia[hh] * t11.y, era[hh] * t11.y - eia[hh] * t11.x);
            const float2 n00 = make_float2(ca[hh] * t00.x - sa[hh] * u10.x, ca[hh] * t00.y - sa[hh] * u10.y);
            const float2 n01 = make_float2(ca[hh] * t01.x - sa[hh] * u11.x, ca[hh] * t01.y - sa[hh] * u11.y);
            const float2 n10 = make_float2(sa[hh] * t00.x + ca[hh] * u10.x, sa[hh] * t00.y + ca[hh] * u10.y);
            const float2 n11 = make_float2(sa[hh] * t01.x + ca[hh] * u11.x, sa[hh] * t01.y + ca[hh] * u11.y);
            const int pah = pa[hh], qah = qa[hh];
            if (4 * w + h0 + hh == lane) {
              // diagonal block: Hermitian 2 x 2, real diagonal
              G[pah * GS + pah] = make_float2(n00.x, 0.f);
              G[qah * GS + qah] = make_float2(n11.x, 0.f);
              G[pah * GS + qah] = n01;
              G[qah * GS + pah] = make_float2(n01.x, -n01.y);
            } else {
              G[pah * GS + pb] = n00; G[pah * GS + qb] = n01; G[qah * GS + pb] = n10; G[qah * GS + qb] = n11;
            }
          }
          }
          if (rot) {
#pragma unroll
            for (int r0 = 0; r0 < 8; r0 += 4) {
              float2 vp[4], vq[4];
#pragma unroll
              for (int u2 = 0; u2 < 4; ++u2) {
                vp[u2] = V[(8 * w + r0 + u2) * 64 + pb];
                vq[u2] = V[(8 * w + r0 + u2) * 64 + qb];
              }
#pragma unroll
              for (int u2 = 0; u2 < 4; ++u2) {
                const float wx = er * vq[u2].x - ei * vq[u2].y, wy = er * vq[u2].y + ei * vq[u2].x;
                V[(8 * w + r0 + u2) * 64 + pb] = make_float2(c * vp[u2].x - s * wx, c * vp[u2].y - s * wy);
                V[(8 * w + r0 + u2) * 64 + qb] = make_float2(s * vp[u2].x + c * wx, s * vp[u2].y + c * wy);
              }
            }
          }
          __syncthreads();
        }
        t_rounds.stop();
        if (tid() == 0) sm.ibuf[0] += rot_pair;
        if (!__syncthreads_or(rot_pair != 0)) continue;
        // 3. P <- P V, one 128-row tile at a time. Real column k = 2x + c of the
        // A operand is the real or imaginary part of P's column x; output column
        // 2y + d the real or imaginary part of P'(:, y) = sum_x P(:, x) V(x, y).
        SubTimer t_upd(st, SP_TC_UPDATE);
        for (int tile = 0; tile < ntiles && !failed(); ++tile) {
          const int r0 = tile * 128;
          constexpr int XC = TcJac::KT / 2;   // complex columns of P per chunk
          tc_pipeline(128, 64 / XC, false, [&](int c, float* Ahi, float* Alo, float* Bhi, float* Blo) {
            stage_update_a(Ahi, Alo, Xf, m, r0, c * XC, col);
            tc_stage(Bhi, Blo, 128, [&](int j, int k) {
              const float2 v = V[(c * XC + (k >> 1)) * 64 + (j >> 1)];
              const int cin = k & 1, dout = j & 1;
              return cin == dout ? v.x : (cin ? -v.y : v.y);
            });
          });
          if (failed()) return sweep;
          const int row = r0 + (w & 3) * 32 + lane;
          for (int cg = w >> 2; cg < 16; cg += 2) {
            float v[8];
            tc::ld8(tq + (uint32_t)(cg * 8), v);
            if (row < m) {
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                const int cx = col(cg * 4 + j);
                if (cx >= 0) Xf[(size_t)cx * m + row] = make_float2(v[2 * j], v[2 * j + 1]);
              }
            }
          }
          tc::fence_before();
          __syncthreads();
        }
      }
    }
    ++sweep;
    if (failed()) break;
    const int rot = sm.ibuf[0];
    if (tid() == 0) { st.jac_rots += (unsigned long long)rot; st.jac_pairs += (unsigned long long)sm.ibuf[6]; }
    __syncthreads();
    if (rot == 0) { if (tid() == 0) sm.ibuf[1] = 1; break; }
    // near convergence (fewer than 1 in 20 pairs rotating) a rotation count that
    // stops falling means FP32 rounding decides; one FP64 pass finishes the SVD
    if ((rot >= prev_rot && 20 * rot < sm.ibuf[6]) || sweep >= a.max_sweeps) {
      reorth_pass_f64(X, m, nc, false, (double)thr);
      if (tid() == 0) { st.reorth++; sm.ibuf[1] = 1; }
      __syncthreads();
      break;
    }
    prev_rot = rot;
  }
  __syncthreads();
  return sweep;
}

}  // namespace tepai
