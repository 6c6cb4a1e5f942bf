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


def sign_after(events: np.ndarray, j: int) -> int:
    """sign(g_l) = (-1)^(number of pi-rotations C so far) (App. B)."""
    if len(events) == 0:
        return 1
    nc = int(np.count_nonzero((events[:, 0] <= j) & (events[:, 2] == EV_C)))
    return -1 if nc % 2 else 1
