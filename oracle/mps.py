"""Plain FP64 matrix-product-state simulator of one TE-PAI circuit (Sec. II.A).

Site tensors are A_p[chi_{p-1}][2][chi_p] over chain positions p, in
mixed-canonical form with an explicit orthogonality centre. An open chain uses
the natural site order. A ring (periodic boundary of Sec. III, Eq. spinRing)
uses the folded order 0, n-1, 1, n-2, 2, ..., so that every ring bond joins
chain positions at distance 1 or 2 and every cut crosses two ring bonds, as
in the natural order.

- A two-site gate on bond (i, i+1) moves the centre to site i (Householder
  QR / LQ through numpy.linalg.qr) and forms theta = A_i A_{i+1}. It applies
  the 4x4 gate and factorises theta by SVD (numpy.linalg.svd, LAPACK). It
  keeps at most chi_max singular values, renormalises the kept ones to unit
  norm, and leaves the centre on site i+1 (Sec. II.A, bond-dimension and
  truncation paragraphs).
- Truncation keeps the k largest singular values, with
  k = max(1, min(chi_max, k_floor, k_cut, len(s))):
    k_cut   = the smallest k with sum_{j>=k} s_j^2 <= cutoff * sum_j s_j^2;
    k_floor = #{j : s_j > floor_rel * s_0}, which drops singular values that
              are zero to working precision.
  A cut never splits a group of singular values that are equal to working
  precision: when s_{k-1} - s_k <= gap_rel * s_0, k drops to the largest
  k' < k with a gap there (the whole tied group is discarded); if no such
  k' >= 1 exists, k stays as it is. The paper keeps "the chi largest"
  singular values and says nothing of ties; the default gap_rel = 1e-12
  (PAPER_TIE_REL) only settles exactly degenerate groups, whose kept state
  the paper's rule leaves undefined. A wider band (e.g. 1e-4) is an explicit
  option, taken by both this oracle and the CUDA path when set.
- A single-site gate, and a pi-rotation of a bond term (a product of two
  single-site Paulis), act on the physical index directly. A unitary on one
  site keeps every canonical condition.
- A gate on sites two chain positions apart (p, p+2) swaps positions p+1 and
  p+2, acts on chain bond (p, p+1), and swaps back. Every swap is a two-site
  update with truncation.
- Alternatively (three_site=True) such a gate is one three-site update: with
  the centre on p, theta3 = A_p A_{p+1} A_{p+2} takes the gate on its first
  and third physical indices and is split back left to right by two truncated
  SVDs, (chi_l 2) x (4 chi_r) and then (k 2) x (2 chi_r), each under the same
  keep rule and renormalisation; the centre ends on p+2. This is the cheapest
  form of applying the bond-2 gate as an operator on three sites (a
  three-site MPO of bond dimension 1 to 4) instead of routing it by swaps; it
  truncates twice instead of three times.
- <Z_i> is contracted with left and right environments. This makes no
  canonical-form assumption.
"""
from __future__ import annotations

import numpy as np

from . import gates
from .sampler import EV_B, EV_C, EV_T

ZDIAG = np.array([1.0, -1.0])

# Tie band of the paper's truncation rule: only groups of singular values equal
# to working precision (relative gaps <= 1e-12) count as ties at a cut.
PAPER_TIE_REL = 1e-12


def chain_order(n: int, periodic: bool) -> list:
    """Ring site held by each chain position: natural for an open chain;
    0, n-1, 1, n-2, 2, ... for a ring."""
    if not periodic:
        return list(range(n))
    out, lo, hi = [], 0, n - 1
    while lo <= hi:
        out.append(lo)
        lo += 1
        if lo <= hi:
            out.append(hi)
            hi -= 1
    return out


class MPS:
    def __init__(self, tensors, centre: int, periodic: bool = False):
        self.A = [np.asarray(a, dtype=np.complex128) for a in tensors]
        self.c = centre
        self.order = chain_order(len(self.A), periodic)
        self.pos = [0] * len(self.A)
        for p, site in enumerate(self.order):
            self.pos[site] = p
        self.stats = {"gate_updates": 0, "swap_updates": 0, "three_site_updates": 0, "qr_moves": 0,
                      "max_discarded": 0.0, "max_chi": 1, "min_cut_gap": float("inf")}

    @property
    def n(self):
        return len(self.A)

    def bond_dims(self):
        return [1] + [a.shape[2] for a in self.A[:-1]] + [1]


def product_state(bits, periodic: bool = False) -> MPS:
    """Product state of single-site codes (gates.STATE_CODE: |0>, |1>, |+>,
    |->, |+i>, |-i>) over ring sites, stored in chain order."""
    order = chain_order(len(bits), periodic)
    ts = []
    for site in order:
        a = np.zeros((1, 2, 1), dtype=np.complex128)
        a[0, :, 0] = gates.STATE_CODE[int(bits[site])]
        ts.append(a)
    return MPS(ts, 0, periodic)


def _move_right(m: MPS):
    c = m.c
    A = m.A[c]
    chl, d, chr_ = A.shape
    Q, R = np.linalg.qr(A.reshape(chl * d, chr_))
    m.A[c] = Q.reshape(chl, d, Q.shape[1])
    m.A[c + 1] = np.tensordot(R, m.A[c + 1], axes=(1, 0))
    m.c = c + 1
    m.stats["qr_moves"] += 1


def _move_left(m: MPS):
    c = m.c
    A = m.A[c]
    chl, d, chr_ = A.shape
    # A = L Q with Q right-orthonormal rows: QR of A^H.
    Q, R = np.linalg.qr(A.reshape(chl, d * chr_).conj().T)
    m.A[c] = Q.conj().T.reshape(Q.shape[1], d, chr_)
    m.A[c - 1] = np.tensordot(m.A[c - 1], R.conj().T, axes=(2, 0))
    m.c = c - 1
    m.stats["qr_moves"] += 1


def move_centre(m: MPS, target: int):
    while m.c < target:
        _move_right(m)
    while m.c > target:
        _move_left(m)


def canonicalize(tensors, periodic: bool = False) -> MPS:
    """Bring arbitrary site tensors (given in chain order) to right-canonical
    form with the centre on chain position 0, then normalise the state."""
    m = MPS(tensors, len(tensors) - 1, periodic)
    move_centre(m, 0)
    m.A[0] = m.A[0] / np.linalg.norm(m.A[0])
    m.stats["qr_moves"] = 0
    return m


def keep_count(s: np.ndarray, chi_max: int, cutoff: float, floor_rel: float,
               gap_rel: float = PAPER_TIE_REL) -> int:
    if s.size == 0 or s[0] <= 0.0:
        return 1
    w = s.astype(np.float64) ** 2
    tot = float(np.sum(w))
    # tail[k] = sum_{j >= k} w_j, accumulated from the smallest value upward
    tail = np.zeros(s.size + 1)
    acc = 0.0
    for j in range(s.size - 1, -1, -1):
        acc += w[j]
        tail[j] = acc
    k_cut = s.size
    for k in range(1, s.size + 1):
        if tail[k] <= cutoff * tot:
            k_cut = k
            break
    k_floor = int(np.count_nonzero(s > floor_rel * s[0]))
    k = max(1, min(chi_max, k_floor, k_cut, s.size))
    if k < s.size and s[k] > floor_rel * s[0]:
        kk = k
        while kk >= 1 and s[kk - 1] - s[kk] <= gap_rel * s[0]:
            kk -= 1
        if kk >= 1:
            k = kk
    return k


def apply_two(m: MPS, i: int, g: np.ndarray, chi_max: int, cutoff: float,
              floor_rel: float, swap: bool = False, gap_rel: float = PAPER_TIE_REL,
              regauge: bool = False):
    """Two-site update on bond (i, i+1) with a 4x4 gate g (basis |s_i s_{i+1}>).
    regauge=True moves the centre back to site i afterwards: an exact change of
    gauge that leaves the state unchanged, used to measure how strongly a run
    amplifies rounding-level perturbations."""
    move_centre(m, i)
    A, B = m.A[i], m.A[i + 1]
    chl, chr_ = A.shape[0], B.shape[2]
    th = np.tensordot(A, B, axes=(2, 0))                          # (chl,2,2,chr)
    th = np.einsum('stuv,auvb->astb', g.reshape(2, 2, 2, 2), th)
    M = th.reshape(chl * 2, 2 * chr_)
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    k = keep_count(s, chi_max, cutoff, floor_rel, gap_rel)
    tot = float(np.sum(s.astype(np.float64) ** 2))
    kept = s[:k]
    disc = 0.0 if tot == 0.0 else float(np.sum(s[k:] ** 2)) / tot
    if k < s.size and s[k] > floor_rel * s[0]:
        # relative gap at a cut that discards weight: small gaps make the kept
        # subspace sensitive to rounding-level perturbations
        m.stats["min_cut_gap"] = min(m.stats["min_cut_gap"], float((s[k - 1] - s[k]) / s[0]))
    kept = kept / np.sqrt(np.sum(kept ** 2))
    m.A[i] = U[:, :k].reshape(chl, 2, k)
    m.A[i + 1] = (kept[:, None] * Vh[:k, :]).reshape(k, 2, chr_)
    m.c = i + 1
    m.stats["swap_updates" if swap else "gate_updates"] += 1
    m.stats["max_discarded"] = max(m.stats["max_discarded"], disc)
    m.stats["max_chi"] = max(m.stats["max_chi"], k)
    if regauge:
        move_centre(m, i)


def _split(m: MPS, M: np.ndarray, chi_max: int, cutoff: float, floor_rel: float, gap_rel: float):
    """Truncated SVD of one split of a three-site update: the keep rule of
    keep_count, kept singular values renormalised to unit norm; returns
    (U_k, s_k, Vh_k, discarded weight fraction) and records it, the cut gap
    and k."""
    U, s, Vh = np.linalg.svd(M, full_matrices=False)
    k = keep_count(s, chi_max, cutoff, floor_rel, gap_rel)
    tot = float(np.sum(s ** 2))
    disc = 0.0 if tot == 0.0 else float(np.sum(s[k:] ** 2)) / tot
    if k < s.size and s[k] > floor_rel * s[0]:
        m.stats["min_cut_gap"] = min(m.stats["min_cut_gap"], float((s[k - 1] - s[k]) / s[0]))
    kept = s[:k] / np.sqrt(np.sum(s[:k] ** 2))
    m.stats["max_discarded"] = max(m.stats["max_discarded"], disc)
    m.stats["max_chi"] = max(m.stats["max_chi"], k)
    return U[:, :k], kept, Vh[:k, :], disc


def apply_three(m: MPS, i: int, g: np.ndarray, chi_max: int, cutoff: float, floor_rel: float,
                gap_rel: float = PAPER_TIE_REL):
    """Gate g (4x4, basis |s_i s_{i+2}>) on chain positions i and i+2 as one
    three-site update (see the module notes); the centre ends on i+2.
    Returns the discarded weight fractions of the two splits."""
    move_centre(m, i)
    A, B, C3 = m.A[i], m.A[i + 1], m.A[i + 2]
    chl, chr_ = A.shape[0], C3.shape[2]
    th = np.einsum('asc,ctd,dub->astub', A, B, C3)                  # (chl,2,2,2,chr)
    th = np.einsum('xysu,astub->axtyb', g.reshape(2, 2, 2, 2), th)  # gate on s and u
    U1, s1, V1, e1 = _split(m, th.reshape(chl * 2, 4 * chr_), chi_max, cutoff, floor_rel, gap_rel)
    k1 = s1.size
    m.A[i] = U1.reshape(chl, 2, k1)
    rest = (s1[:, None] * V1).reshape(k1 * 2, 2 * chr_)
    U2, s2, V2, e2 = _split(m, rest, chi_max, cutoff, floor_rel, gap_rel)
    k2 = s2.size
    m.A[i + 1] = U2.reshape(k1, 2, k2)
    m.A[i + 2] = (s2[:, None] * V2).reshape(k2, 2, chr_)
    m.c = i + 2
    m.stats["three_site_updates"] += 1
    return e1, e2


def apply_one(m: MPS, i: int, u: np.ndarray):
    m.A[i] = np.einsum('st,atb->asb', u, m.A[i])


class GateCache:
    """Gate matrices per (term, setting), built once from the gate module."""

    def __init__(self, plan):
        self.plan = plan
        self.cache = {}

    def get(self, k: int, v: int) -> np.ndarray:
        key = (k, v)
        if key not in self.cache:
            t = self.plan.terms[k]
            if v == EV_C:
                self.cache[key] = gates.PAULI[t.pauli[0]]   # one factor per site
            elif v == EV_B:
                self.cache[key] = gates.rotation(t.pauli, self.plan.phi[k])
            else:
                self.cache[key] = gates.rotation(t.pauli, self.plan.theta[k])
        return self.cache[key]


def apply_event(m: MPS, plan, cache: GateCache, k: int, v: int, chi_max: int,
                cutoff: float, floor_rel: float, gap_rel: float = PAPER_TIE_REL, regauge: bool = False,
                three_site: bool = False):
    t = plan.terms[k]
    g = cache.get(k, v)
    if t.pauli == 'Z':
        apply_one(m, m.pos[t.a], g)
        return
    pa, pb = m.pos[t.a], m.pos[t.b]
    if v == EV_C:
        # R_k(pi) = -i P (x) P: one Pauli on each site, global phase dropped
        apply_one(m, pa, g)
        apply_one(m, pb, g)
        return
    # gate basis |s_lo s_hi> over the lower and upper chain position
    lo, hi = (pa, pb) if pa < pb else (pb, pa)
    if pa > pb:
        g = gates.SWAP @ g @ gates.SWAP
    if hi - lo == 1:
        apply_two(m, lo, g, chi_max, cutoff, floor_rel, gap_rel=gap_rel, regauge=regauge)
        return
    assert hi - lo == 2
    if three_site:
        apply_three(m, lo, g, chi_max, cutoff, floor_rel, gap_rel=gap_rel)
        if regauge:
            move_centre(m, lo)
        return
    # bring the site at hi next to lo, apply the gate, move it back
    apply_two(m, lo + 1, gates.SWAP, chi_max, cutoff, floor_rel, swap=True, gap_rel=gap_rel,
              regauge=regauge)
    apply_two(m, lo, g, chi_max, cutoff, floor_rel, gap_rel=gap_rel, regauge=regauge)
    apply_two(m, lo + 1, gates.SWAP, chi_max, cutoff, floor_rel, swap=True, gap_rel=gap_rel,
              regauge=regauge)


def expect_z(m: MPS) -> np.ndarray:
    """<Z_i> / <psi|psi> for every ring site i (chain position pos[i]), by
    left and right environments,
    contracted pairwise:
      L_{i+1}[c,d] = sum_{a,b,s} L_i[a,b] conj(A[a,s,c]) A[b,s,d]
      R_i[a,b]     = sum_{c,d,s} conj(A[a,s,c]) A[b,s,d] R_{i+1}[c,d]
      <Z_i>        = sum L_i[a,b] conj(A[a,s,c]) z_s A[b,s,d] R_{i+1}[c,d] / L_n."""
    n = m.n
    Lenv = [np.ones((1, 1), dtype=np.complex128)]
    for i in range(n):
        A = m.A[i]
        T = np.tensordot(Lenv[i], A, axes=(1, 0))                    # [a,s,d]
        Lenv.append(np.tensordot(A.conj(), T, axes=([0, 1], [0, 1])))  # [c,d]
    Renv = [None] * (n + 1)
    Renv[n] = np.ones((1, 1), dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        A = m.A[i]
        U = np.tensordot(A, Renv[i + 1], axes=(2, 1))                # [b,s,c]
        Renv[i] = np.tensordot(A.conj(), U, axes=([1, 2], [1, 2]))   # [a,b]
    norm = Lenv[n][0, 0].real
    out = np.zeros(n)
    for i in range(n):
        A = m.A[i]
        T = np.tensordot(Lenv[i], A, axes=(1, 0))                    # [a,s,d]
        T2 = np.tensordot(T, Renv[i + 1], axes=(2, 1))              # [a,s,c]
        out[i] = np.sum(A.conj() * ZDIAG[None, :, None] * T2).real / norm
    return out[np.array(m.pos)]


def expect_string(m: MPS, codes) -> float:
    """<psi| (x)_i P_{codes[i]} |psi> / <psi|psi> for a Pauli string given per
    ring site i (gates.PAULI_CODE), by one left-to-right transfer-matrix
    contraction over the whole chain (no use of the canonical form):
      E_{p+1}[c,d] = sum_{a,b,s,t} E_p[a,b] conj(A_p[a,s,c]) O_p[s,t] A_p[b,t,d],
    with O_p the operator at chain position p (identity where none)."""
    n = m.n
    ops = [gates.I2] * n
    for site, c in enumerate(codes):
        ops[m.pos[site]] = gates.PAULI_CODE[int(c)]
    E = np.ones((1, 1), dtype=np.complex128)
    N = np.ones((1, 1), dtype=np.complex128)
    for p in range(n):
        A = m.A[p]
        OA = np.einsum('st,btd->bsd', ops[p], A)
        E = np.einsum('ab,asc,bsd->cd', E, A.conj(), OA)
        N = np.einsum('ab,asc,bsd->cd', N, A.conj(), A)
    return float((E[0, 0] / N[0, 0]).real)


def run_events(m: MPS, plan, events, snap_steps, chi_max: int, cutoff: float,
               floor_rel: float = 1e-14, gap_rel: float = PAPER_TIE_REL, regauge: bool = False,
               strings=None, three_site: bool = False) -> np.ndarray:
    cache = GateCache(plan)
    out = []
    e = 0
    ne = len(events)
    for js in snap_steps:
        while e < ne and events[e, 0] <= js:
            apply_event(m, plan, cache, int(events[e, 1]), int(events[e, 2]),
                        chi_max, cutoff, floor_rel, gap_rel, regauge, three_site)
            e += 1
        out.append(expect_z(m) if strings is None else np.array([expect_string(m, r) for r in strings]))
    return np.array(out)
