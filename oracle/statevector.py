"""Dense FP64 state-vector simulator (n <= 14) for the oracle.

A state is a complex128 array of shape (2,)*n with axis i = site i. It
applies the same ordered gate list as one TE-PAI sample, or the
deterministic N-step first-order product formula (Eq. Trotter-Suzuki). It
also computes exact exp(-iHt)|psi_0> by dense Hermitian eigendecomposition.
"""
from __future__ import annotations

import numpy as np

from . import gates
from .sampler import EV_B, EV_C, EV_T


def basis_state(bits) -> np.ndarray:
    """Product state of single-site codes (gates.STATE_CODE): 0/1 are the
    basis states, 2..5 are |+>, |->, |+i>, |-i>."""
    psi = np.ones((), dtype=np.complex128)
    for b in bits:
        psi = np.multiply.outer(psi, gates.STATE_CODE[int(b)])
    return psi


def expect_string(psi: np.ndarray, codes) -> float:
    """<psi| (x)_i P_{codes[i]} |psi> / <psi|psi> for a Pauli string given per site
    (gates.PAULI_CODE): the operators are applied to a copy of the state."""
    phi = psi
    for i, c in enumerate(codes):
        if int(c):
            phi = apply_1(phi, gates.PAULI_CODE[int(c)], i)
    return float((np.vdot(psi, phi) / np.vdot(psi, psi)).real)


def apply_1(psi: np.ndarray, u: np.ndarray, i: int) -> np.ndarray:
    out = np.tensordot(u, psi, axes=([1], [i]))
    return np.moveaxis(out, 0, i)


def apply_2(psi: np.ndarray, g: np.ndarray, i: int, j: int) -> np.ndarray:
    """Apply a 4x4 gate with basis |s_i s_j> to sites i and j (any pair)."""
    g4 = g.reshape(2, 2, 2, 2)
    out = np.tensordot(g4, psi, axes=([2, 3], [i, j]))
    return np.moveaxis(out, [0, 1], [i, j])


def expect_z(psi: np.ndarray) -> np.ndarray:
    n = psi.ndim
    p = np.abs(psi) ** 2
    norm = p.sum()
    out = np.zeros(n)
    for i in range(n):
        pi = np.moveaxis(p, i, 0).reshape(2, -1).sum(axis=1)
        out[i] = (pi[0] - pi[1]) / norm
    return out


def apply_event(psi: np.ndarray, plan, k: int, v: int) -> np.ndarray:
    """Setting B: R_k(sign(theta) Delta). Setting C: R_k(pi) = -i h_k, applied
    as h_k (a global phase does not change any expectation value).
    Trotter gate: R_k(theta_k)."""
    t = plan.terms[k]
    if v == EV_C:
        g = gates.pauli_string(t.pauli)
    elif v == EV_B:
        g = gates.rotation(t.pauli, plan.phi[k])
    elif v == EV_T:
        g = gates.rotation(t.pauli, plan.theta[k])
    else:
        raise ValueError(v)
    if t.pauli == 'Z':
        return apply_1(psi, g, t.a)
    return apply_2(psi, g, t.a, t.b)


def run_events(bits, plan, events, snap_steps, strings=None) -> np.ndarray:
    """<Z_i> (or, with `strings`, each Pauli string's expectation) after each
    snapshot step; events in gate order."""
    psi = basis_state(bits)
    out = []
    e = 0
    ne = len(events)
    for js in snap_steps:
        while e < ne and events[e, 0] <= js:
            psi = apply_event(psi, plan, int(events[e, 1]), int(events[e, 2]))
            e += 1
        out.append(expect_z(psi) if strings is None else np.array([expect_string(psi, r) for r in strings]))
    return np.array(out)


def hamiltonian(prob) -> np.ndarray:
    """Dense H = sum_k c_k h_k (Eq. spinRing), basis index = bits read with
    site 0 as the most significant bit (matches psi.reshape(-1))."""
    from .planner import term_list
    n = prob.n
    dim = 2 ** n
    H = np.zeros((dim, dim), dtype=np.complex128)
    for t in term_list(prob):
        ops = [gates.I2] * n
        for ch, site in zip(t.pauli, (t.a, t.b)[:len(t.pauli)]):
            ops[site] = gates.PAULI[ch]
        m = ops[0]
        for o in ops[1:]:
            m = np.kron(m, o)
        H += t.c * m
    return H


def exact_z(prob, times) -> np.ndarray:
    """<Z_i>(t) under exact exp(-iHt) from |init_bits>."""
    H = hamiltonian(prob)
    w, V = np.linalg.eigh(H)
    psi0 = basis_state(prob.init_bits).reshape(-1)
    c = V.conj().T @ psi0
    out = []
    for t in times:
        psi = V @ (np.exp(-1j * w * t) * c)
        out.append(expect_z(psi.reshape((2,) * prob.n)))
    return np.array(out)
