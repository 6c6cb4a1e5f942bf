"""Single precision with entries whose squares underflow FP32.

A TE-PAI state carries amplitudes far below 1e-19 (rounding residues of exact
zeros, products of sin(Delta/2)); the square of such an FP32 entry lies in
the subnormal range and keeps only a few significant bits. A Householder
reflector whose leading entry x_0 is that small, in a column of O(1) norm,
must still be unitary: its phase x_0/|x_0| needs |x_0| to full relative
precision. These tests plant such entries (1e-23 .. 1e-20, random phases) at
the leading positions of the columns that the canonicalisation of the start
state factors (the (a = 0, s = 0) slice of every site), then check on the
single-precision path that every site the centre has left is an isometry,
that the state keeps unit norm, and that <Z_i> matches the FP64 oracle at
1e-4. The planted entries change the state by less than 1e-19, so the oracle
sees the same physics."""
import math

import numpy as np
import pytest

import workloads as W
from oracle_rule import oracle_rule
from oracle import run as oracle_run

pytestmark = pytest.mark.gpu

TOLMIX = 1e-4
N = 8
CHI = 4


@pytest.fixture(scope="module")
def T():
    from paper_2604_13144_gb300 import build
    build.build()
    from paper_2604_13144_gb300 import tepai
    return tepai


@pytest.fixture(scope="module")
def ctx(T):
    c = T.tepai_create(0)
    yield c
    T.tepai_destroy(c)


def _planted(seed=11):
    tens, dims = W.random_mps_tensors(N, CHI, seed=seed)
    rng = np.random.default_rng(seed + 1)
    mags = [3e-23, 1e-21, 5e-22, 2e-20, 3e-23, 1e-22, 4e-21, 3e-23]
    for p, A in enumerate(tens):
        slab = A[0, 0, :]
        ph = np.exp(2j * np.pi * rng.random(slab.shape))
        A[0, 0, :] = mags[p] * ph * (1.0 + rng.random(slab.shape))
    return tens, dims


def _case(steps):
    prob = W.spin_ring(N, 1.0, seed=3, Jz=0.5)
    par = W.Params(T=1.0, n_steps=400, delta=math.pi / 256, n_samples=1, chi_max=CHI,
                   cutoff=1e-12, n_snapshots=1, seed=9, precision=1, run_steps=steps)
    return prob, par


def _dense(ts):
    v = np.ones((1,), dtype=complex)
    for t in ts:
        v = np.tensordot(v.reshape(-1, t.shape[0]), t, axes=(1, 0)).reshape(-1, t.shape[2])
    return v.reshape(-1)


@pytest.mark.parametrize("steps", [1, 3])
def test_tiny_leading_entries_keep_isometries(T, ctx, steps):
    prob, par = _case(steps)
    init = _planted()
    tens, dims = T.tepai_evolve_state(ctx, prob, par, init)
    left = right = 0
    for A in tens:
        a, d, b = A.shape
        L = A.reshape(a * d, b)
        Rm = A.reshape(a, d * b)
        el = np.abs(L.conj().T @ L - np.eye(b)).max()
        er = np.abs(Rm @ Rm.conj().T - np.eye(a)).max()
        left += el < 1e-5
        right += er < 1e-5
        assert min(el, er) < 1e-5 or np.isclose(np.linalg.norm(A), 1.0, atol=1e-5), (A.shape, el, er)
    # mixed-canonical: all sites but the centre are isometries of one kind or the other
    assert left + right >= N - 1
    assert abs(np.linalg.norm(_dense(tens)) - 1.0) < 1e-5


def test_tiny_leading_entries_match_oracle(T, ctx):
    prob, par = _case(4)
    par = W.Params(**{**par.__dict__, "n_samples": 8})
    init = _planted()
    got = T.tepai_sample_values(ctx, prob, par, init)
    assert got["stats"]["device_status"][0] == 0
    ref = oracle_run.run(prob, par, init_tensors=init[0], **oracle_rule(par))
    assert np.array_equal(got["sign"], ref["sign"])
    assert np.max(np.abs(got["v"] - ref["v"])) <= TOLMIX
