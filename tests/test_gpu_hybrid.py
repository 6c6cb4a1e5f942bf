"""Hybrid run (Sec. IV): a deterministic Trotter prefix evolved as one circuit,
its final MPS exported through tepai_evolve_state, then TE-PAI samples started
from it. The exported state equals the oracle's prefix state (up to a global
phase), and the continuation matches the oracle started from its own prefix
state, sample by sample, to 1e-10 in FP64."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import run as oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2604_13144_gb300 import build
    build.build()
    from paper_2604_13144_gb300 import tepai
    return tepai


def _vector(tensors):
    psi = np.asarray(tensors[0]).reshape(-1, tensors[0].shape[2])
    for a in tensors[1:]:
        psi = (psi @ a.reshape(a.shape[0], -1)).reshape(-1, a.shape[2])
    return psi.reshape(-1)


@pytest.mark.parametrize("periodic", [True, False])
def test_trotter_prefix_then_tepai_matches_oracle(T, periodic):
    n = 8
    prob = W.spin_ring(n, 1.0, seed=0, periodic=periodic)
    pre = W.Params(T=0.5, n_steps=50, delta=math.pi / 64, n_samples=1, chi_max=16, cutoff=0.0,
                   n_snapshots=1, seed=0, precision=0, variant=2)
    ctx = T.tepai_create(0)
    try:
        tens, dims = T.tepai_evolve_state(ctx, prob, pre)
        ro = oracle_run.run(prob, pre)
        ref = ro["states"][0]
        assert list(dims) == [1] + [a.shape[2] for a in ref]
        a, b = _vector(tens), _vector(ref)
        assert abs(np.linalg.norm(a) - 1.0) <= 1e-12
        assert abs(abs(np.vdot(a, b)) - 1.0) <= 1e-12
        te = W.Params(T=0.5, n_steps=200, delta=math.pi / 64, n_samples=4, chi_max=16, cutoff=0.0,
                      n_snapshots=4, seed=3, precision=0)
        got = T.tepai_sample_values(ctx, prob, te, init=(tens, dims))
        want = oracle_run.run(prob, te, init_tensors=ref)
        assert float(np.max(np.abs(got["v"] - want["v"]))) <= 1e-10
        assert np.array_equal(got["sign"], want["sign"])
    finally:
        T.tepai_destroy(ctx)
