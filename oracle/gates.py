"""Pauli rotation gates of the product formula (App. A.3, Eq. productFormula):
R_k(theta) = exp(-i h_k theta / 2) for a Pauli string h_k. Because h_k^2 = I,
the exponential equals cos(theta/2) I - i sin(theta/2) h_k. The gate is
formed here as an explicit matrix exponential (scipy.linalg.expm), which is
the definition itself; tests pin it against the closed form.

Basis: single site |0>, |1> with Z|0> = |0>. Two sites |s_a s_b> ordered
(first site, second site), index 2*s_a + s_b.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {'X': X, 'Y': Y, 'Z': Z}
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]],
                dtype=np.complex128)


# Single-site codes of initial product states and of observables (Pauli
# strings given per site): states |0>, |1>, |+>, |->, |+i>, |-i>; operators
# I, X, Y, Z.
_R2 = 1.0 / np.sqrt(2.0)
STATE_CODE = {0: np.array([1, 0], dtype=np.complex128), 1: np.array([0, 1], dtype=np.complex128),
              2: np.array([_R2, _R2], dtype=np.complex128), 3: np.array([_R2, -_R2], dtype=np.complex128),
              4: np.array([_R2, 1j * _R2], dtype=np.complex128), 5: np.array([_R2, -1j * _R2], dtype=np.complex128)}
PAULI_CODE = {0: I2, 1: X, 2: Y, 3: Z}


def pauli_string(name: str) -> np.ndarray:
    """'Z' -> Z (2x2); 'XX' -> X (x) X (4x4)."""
    m = PAULI[name[0]]
    for ch in name[1:]:
        m = np.kron(m, PAULI[ch])
    return m


def rotation(name: str, theta: float) -> np.ndarray:
    """R(theta) = exp(-i theta h / 2)."""
    return scipy.linalg.expm(-0.5j * theta * pauli_string(name))
