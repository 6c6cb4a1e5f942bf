"""Brute-force sum over every gate-setting configuration (Statement 1;
App. B, multi-index l in {1,2,3}^{LN}).

For tiny systems this visits all 3^{L N} circuits U_l. It weights each
circuit by g_l = prod gamma_{l_kj}(|theta_k|) and returns
sum_l g_l <Z_i>_l together with sum_l |g_l|. By Statement 1 the first equals
the N-step Trotter value, and by Eq. overhead-bound the second equals
||g||_1. The traversal is a depth-first search that carries the state vector.
"""
from __future__ import annotations

import numpy as np

from . import gates
from . import statevector as sv


def enumerate_all(prob, plan, n_steps: int):
    L = len(plan.terms)
    ops = []
    for k, t in enumerate(plan.terms):
        sites = (t.a,) if t.pauli == 'Z' else (t.a, t.b)
        gB = gates.rotation(t.pauli, plan.phi[k])
        gC = gates.pauli_string(t.pauli)
        ops.append((sites, plan.gam[k], gB, gC))
    total_z = np.zeros(prob.n)
    total_abs = [0.0]

    def apply(psi, sites, g):
        if len(sites) == 1:
            return sv.apply_1(psi, g, sites[0])
        return sv.apply_2(psi, g, sites[0], sites[1])

    def rec(depth, psi, weight):
        nonlocal total_z
        if depth == n_steps * L:
            total_z = total_z + weight * sv.expect_z(psi)
            total_abs[0] += abs(weight)
            return
        sites, gam, gB, gC = ops[depth % L]
        if gam[0] != 0.0:
            rec(depth + 1, psi, weight * gam[0])
        if gam[1] != 0.0:
            rec(depth + 1, apply(psi, sites, gB), weight * gam[1])
        if gam[2] != 0.0:
            rec(depth + 1, apply(psi, sites, gC), weight * gam[2])

    rec(0, sv.basis_state(prob.init_bits), 1.0)
    return total_z, total_abs[0]
