"""Signed, ||g||_1-weighted ensemble mean (App. B; Sec. II.B; Statement 2).

o_l = ||g(t)||_1 sign(g_l) Tr[O U_l rho_0 U_l^dag]. The estimate is the mean
over samples. The per-configuration value is v_l = sign(g_l) <O>_l, so that
Var[o] = ||g||_1^2 Var[v] (Eq. config_var).

Sums run in fixed sample order with Neumaier's compensated summation
(A. Neumaier, ZAMM 54, 1974), in FP64.
"""
from __future__ import annotations

import math

import numpy as np


def neumaier(values) -> tuple[float, float]:
    """Return (sum, compensation); the compensated total is sum + comp."""
    s = 0.0
    c = 0.0
    for x in values:
        x = float(x)
        t = s + x
        if abs(s) >= abs(x):
            c += (s - t) + x
        else:
            c += (x - t) + s
        s = t
    return s, c


def estimate(v: np.ndarray, sign: np.ndarray, gnorm: np.ndarray):
    """v: (Ns, M, n_obs) per-sample <Z_i>; sign: (Ns, M) in {+1, -1};
    gnorm: (M,). Returns (mean, stderr, partials) with partials (M, n_obs, 3)
    holding (sum, compensation, sum of squares) of sign * v."""
    Ns, M, nobs = v.shape
    mean = np.zeros((M, nobs))
    se = np.zeros((M, nobs))
    part = np.zeros((M, nobs, 3))
    for m in range(M):
        for i in range(nobs):
            x = sign[:, m].astype(np.float64) * v[:, m, i]
            s, c = neumaier(x)
            sq, sqc = neumaier(x * x)
            part[m, i] = (s, c, sq + sqc)
            mu = (s + c) / Ns
            mean[m, i] = gnorm[m] * mu
            if Ns > 1:
                var = max(0.0, ((sq + sqc) - Ns * mu * mu) / (Ns - 1))
                se[m, i] = gnorm[m] * math.sqrt(var / Ns)
    return mean, se, part
