"""General observables and initial states through the C-ABI: Pauli strings
(X, Y, Z on any sites, 2- and 3-local) and product starts |0>, |1>, |+>, |->,
|+i>, |-i>, including the |+...+ - +...+> / <X_0> workload of Sec. III.
Same seeded circuits as the FP64 oracle: 1e-10 in FP64 mode, 1e-4 in mixed
mode at a short horizon."""
import math

import numpy as np
import pytest

import workloads as W
from oracle_rule import oracle_rule
from oracle import run as oracle_run

pytestmark = pytest.mark.gpu


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


def _strings(n, rng, count):
    out = np.zeros((count, n), dtype=np.uint8)
    for o in range(count):
        k = 1 + o % 3
        sites = rng.choice(n, size=k, replace=False)
        out[o, sites] = rng.integers(1, 4, size=k)
    return out


@pytest.mark.parametrize("periodic", [True, False])
def test_pauli_strings_from_product_codes_fp64(T, ctx, periodic):
    n = 8
    rng = np.random.default_rng(11)
    prob = W.spin_ring(n, 1.0, seed=2, periodic=periodic)
    prob.init_bits = np.array([2, 0, 5, 1, 3, 4, 2, 0], dtype=np.uint8)
    strings = _strings(n, rng, 9)
    strings[0] = 0                                   # the identity string is 1
    strings[1, :3] = [1, 1, 1]                       # X_0 X_1 X_2
    par = W.Params(T=0.4, n_steps=80, delta=math.pi / 64, n_samples=4, chi_max=16, cutoff=0.0,
                   n_snapshots=4, seed=7, precision=0, obs_strings=strings)
    got = T.tepai_sample_values(ctx, prob, par)
    want = oracle_run.run(prob, par)
    assert got["v"].shape == (4, 4, 9)
    assert np.allclose(got["v"][:, :, 0], 1.0, atol=1e-12)
    assert float(np.max(np.abs(got["v"] - want["v"]))) <= 1e-10
    assert np.array_equal(got["sign"], want["sign"])


def test_plus_minus_start_with_x0_fp64(T, ctx):
    n = 10
    prob = W.spin_ring(n, 1.0, seed=0)
    prob.init_bits = W.plus_minus_codes(n)
    strings = np.zeros((2, n), dtype=np.uint8)
    strings[0, 0] = 1                                # X_0
    strings[1, n // 2] = 1                           # X on the flipped site
    par = W.Params(T=0.5, n_steps=100, delta=math.pi / 64, n_samples=3, chi_max=32, cutoff=0.0,
                   n_snapshots=5, seed=2, precision=0, obs_strings=strings)
    got = T.tepai_sample_values(ctx, prob, par)
    want = oracle_run.run(prob, par)
    assert float(np.max(np.abs(got["v"] - want["v"]))) <= 1e-10
    # the ensemble estimate carries the same weights as for <Z_i>
    r = T.tepai_run(ctx, prob, W.Params(**{**par.__dict__, "n_samples": 3}))
    assert np.allclose(r["mean"], want["mean"], atol=1e-10, rtol=0)


def test_pauli_strings_mixed_from_random_mps(T, ctx):
    n = 12
    rng = np.random.default_rng(5)
    prob = W.spin_ring(n, 1.0, seed=6)
    init = W.random_mps_tensors(n, 64, seed=21)
    strings = _strings(n, rng, 6)
    par = W.Params(T=0.05, n_steps=16, delta=math.pi / 64, n_samples=3, chi_max=64, cutoff=1e-10,
                   n_snapshots=2, seed=4, precision=1, obs_strings=strings)
    got = T.tepai_sample_values(ctx, prob, par, init)
    want = oracle_run.run(prob, par, init_tensors=init[0], **oracle_rule(par))
    assert float(np.max(np.abs(got["v"] - want["v"]))) <= 1e-4
