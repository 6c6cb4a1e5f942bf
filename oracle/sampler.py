"""TE-PAI circuit sampler (Sec. II.B protocol, step 2; App. A.3).

Every rotation R_k(theta_kj) of the N-step product formula is replaced by
one of three settings, drawn independently per gate:
  A = I                          with probability |gamma_1| / ||gamma||_1
  B = R_k(sign(theta) Delta)     with probability |gamma_2| / ||gamma||_1
  C = R_k(pi)                    with probability |gamma_3| / ||gamma||_1
The draw is split in two steps with identical law: first "not A" with
probability q_k = (|g2|+|g3|)/||g||_1, then "C" with probability
r_k = |g3| / (|g2|+|g3|). Each gate (j, k) uses one Philox4x64-10 block with
key (seed, global sample index s) and counter (j, k, 0, 0), where j is
1-based. Word x0 decides "not A" (x0 < floor(q_k 2^64)). Word x1 decides
"C" (x1 < floor(r_k 2^64)). This costs O(N L) per sample, the
circuit-generation cost stated in Sec. II.B.

Events are returned in gate order (j ascending, then k ascending) as
(j, k, v) with v = 1 for B, 2 for C and 3 for a deterministic Trotter gate.
"""
from __future__ import annotations

import math

import numpy as np

from . import planner
from .philox import philox4x64_vec

EV_B, EV_C, EV_T = 1, 2, 3


def sample_events(plan: planner.Plan, seed: int, s: int, run_steps: int) -> np.ndarray:
    """Return an (nu, 3) int64 array of events for global sample s."""
    L = len(plan.terms)
    if plan.variant == planner.TROTTER:
        j = np.repeat(np.arange(1, run_steps + 1), L)
        k = np.tile(np.arange(L), run_steps)
        return np.stack([j, k, np.full_like(j, EV_T)], axis=1).astype(np.int64)
    j = np.repeat(np.arange(1, run_steps + 1, dtype=np.uint64), L)
    k = np.tile(np.arange(L, dtype=np.uint64), run_steps)
    zero = np.zeros_like(j)
    x0, x1, _, _ = philox4x64_vec(j, k, zero, zero, seed, s)
    thr_e = np.array(plan.thr_event, dtype=np.uint64)[k.astype(np.int64)]
    thr_c = np.array(plan.thr_c, dtype=np.uint64)[k.astype(np.int64)]
    ev = x0 < thr_e
    isc = x1 < thr_c
    sel = np.nonzero(ev)[0]
    v = np.where(isc[sel], EV_C, EV_B)
    return np.stack([j[sel].astype(np.int64), k[sel].astype(np.int64),
                     v.astype(np.int64)], axis=1)


def sample_events_continuous(plan: planner.Plan, seed: int, s: int, t_snaps) -> tuple:
    """N -> infinity sampler (variant CONTINUOUS): term k emits events as a
    Poisson process of rate lam_k on [0, t_snaps[-1]]. Event i (0-based) of term
    k uses one Philox4x64-10 block with key (seed, s) and counter (k, i, 1, 0):
    u = ((x0 >> 11) + 1) 2^-53 in (0, 1] gives the gap -ln(u) / lam_k since the
    previous event (or t = 0), and x1 < floor(r_inf 2^64) makes it C. Events
    are returned in time order as (m, k, v): m is the first snapshot with
    t <= t_m, so (m, k, v) rows work with sign_after and the snapshot loops;
    the times are returned alongside."""
    t_end = float(t_snaps[-1])
    L = len(plan.terms)
    lam = np.asarray(plan.lam, dtype=np.float64)
    live = [k for k in range(L) if lam[k] > 0.0]
    rows, times = [], []
    if not live:
        return np.zeros((0, 3), dtype=np.int64), np.zeros(0)
    # draw events i = 0 .. C-1 of every live term at once; a term whose C
    # events all fall before t_end draws the next C (rare: C is the mean
    # count plus eight standard deviations)
    mu = float(np.max(lam)) * t_end
    C = int(mu + 8.0 * math.sqrt(mu) + 16)

    def draw(ks, i0):
        kk = np.repeat(np.array(ks, dtype=np.uint64), C)
        ii = np.tile(np.arange(i0, i0 + C, dtype=np.uint64), len(ks))
        x0, x1, _, _ = philox4x64_vec(kk, ii, np.ones_like(kk), np.zeros_like(kk), seed, s)
        return x0.reshape(len(ks), C), x1.reshape(len(ks), C)

    X0, X1 = draw(live, 0)
    for row, k in enumerate(live):
        t, i0 = 0.0, 0
        x0, x1 = X0[row], X1[row]
        while True:
            u = ((x0 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
            gap = -np.log(u) / lam[k]
            tk = np.empty(C)
            for e in range(C):          # t accumulates one gap at a time
                t = t + gap[e]
                tk[e] = t
            n_ok = int(np.count_nonzero(tk <= t_end))
            times.extend(tk[:n_ok].tolist())
            isc = x1[:n_ok] < np.uint64(plan.thr_c[k])
            rows.extend((k, EV_C if c else EV_B) for c in isc)
            if n_ok < C:
                break
            i0 += C
            x0, x1 = (a[0] for a in draw([k], i0))
    order = sorted(range(len(times)), key=lambda e: (times[e], rows[e][0]))
    ts = np.array([times[e] for e in order])
    ev = np.zeros((len(order), 3), dtype=np.int64)
    for r, e in enumerate(order):
        m = 1
        while ts[r] > t_snaps[m - 1]:
            m += 1
        ev[r] = (m, rows[e][0], rows[e][1])
    return ev, ts


def sign_after(events: np.ndarray, j: int) -> int:
    """sign(g_l) = (-1)^(number of pi-rotations C so far) (App. B)."""
    if len(events) == 0:
        return 1
    nc = int(np.count_nonzero((events[:, 0] <= j) & (events[:, 2] == EV_C)))
    return -1 if nc % 2 else 1
