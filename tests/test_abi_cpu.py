"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and its FP64 host planner agrees with the oracle's."""
import math
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import planner

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def T():
    from paper_2604_13144_gb300 import build
    build.build()
    from paper_2604_13144_gb300 import tepai
    return tepai


def _declared():
    src = open(os.path.join(ROOT, "include", "tepai.h")).read()
    return sorted(set(re.findall(r"\b(tepai_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(T):
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(T._lib, name), name
    assert set(T.EXPORTED) == set(names)


@pytest.mark.parametrize("cfg", [W.RING8, W.RING32, W.RING64_XXZ, W.RING100, W.RING64_HYBRID])
def test_host_planner_matches_oracle(T, cfg):
    prob, par, _ = W.workload(cfg)
    g, nu = T.tepai_gnorm(prob, par)
    plan = planner.make_plan(prob, par.T, par.n_steps, par.delta, par.variant)
    snaps = planner.snapshot_steps(par.n_steps, par.n_snapshots)
    want = np.array([planner.gnorm_at(plan, j) for j in snaps])
    assert np.allclose(g, want, rtol=1e-13, atol=0)
    assert abs(nu - planner.expected_nu(plan, par.n_steps)) <= 1e-9 * nu


def test_invalid_arguments_are_rejected(T):
    prob, par, _ = W.workload(W.RING8)
    bad = W.Params(**{**par.__dict__, "n_steps": 100})      # theta = 0.02 > Delta = pi/256
    with pytest.raises(T.TepaiError) as e:
        T.tepai_gnorm(prob, bad)
    assert e.value.code == 2
    bad = W.Params(**{**par.__dict__, "n_snapshots": 7})    # 7 does not divide 2000
    with pytest.raises(T.TepaiError) as e:
        T.tepai_gnorm(prob, bad)
    assert e.value.code == 1
    p2 = W.spin_ring(8, 1.0)
    p2.h = p2.h.copy()
    p2.h[3] = float("nan")
    with pytest.raises(T.TepaiError):
        T.tepai_gnorm(p2, par)
    bad = W.Params(**par.__dict__)
    bad.launch_variant = 8                                  # variants are 0 .. 7
    with pytest.raises(T.TepaiError) as e:
        T.tepai_gnorm(prob, bad)
    assert e.value.code == 1
    for tie in (-1e-4, float("nan"), 1.0):                  # tie band must lie in [0, 1)
        bad = W.Params(**{**par.__dict__, "tie_rel": tie})
        with pytest.raises(T.TepaiError) as e:
            T.tepai_gnorm(prob, bad)
        assert e.value.code == 1
    bad = W.Params(**{**par.__dict__, "three_site": 2})     # a flag: 0 or 1
    with pytest.raises(T.TepaiError) as e:
        T.tepai_gnorm(prob, bad)
    assert e.value.code == 1
    trot = W.Params(**{**par.__dict__, "n_steps": 100, "variant": 2})   # Trotter has no Delta bound
    g, nu = T.tepai_gnorm(prob, trot)
    assert np.all(g == 1.0) and nu == 100 * 32


def test_no_pi_gnorm_is_one(T):
    prob, par, _ = W.workload(W.RING32)
    g, _ = T.tepai_gnorm(prob, W.Params(**{**par.__dict__, "variant": 1}))
    assert np.all(np.abs(g - 1.0) < 1e-15)


@pytest.mark.parametrize("cfg", [W.RING8, W.RING32])
def test_continuous_host_planner_matches_oracle(T, cfg):
    """N -> infinity sampler: ||g(t_m)||_1 and E[nu] from the host planner equal
    the oracle's to rounding (the oracle sums ||c||_1 with Python's compensated
    sum, the planner plainly); small Delta is no obstacle (no theta <= Delta
    bound), Delta >= pi and runaway event counts are refused."""
    prob, par, _ = W.workload(cfg)
    cp = W.Params(**{**par.__dict__, "n_steps": 10, "n_snapshots": 5, "variant": 3})
    g, nu = T.tepai_gnorm(prob, cp)
    plan = planner.make_plan(prob, cp.T, cp.n_steps, cp.delta, planner.CONTINUOUS)
    ts = planner.snapshot_times(plan, cp.steps_run(), cp.n_snapshots)
    want = np.array([planner.gnorm_time(plan, t) for t in ts])
    assert np.allclose(g, want, rtol=1e-14, atol=0)
    assert abs(nu / (np.sum(plan.lam) * ts[-1]) - 1) < 1e-14
    assert abs(nu / planner.nu_infinity(prob, cp.T, cp.delta) - 1) < 1e-14
    for bad in (W.Params(**{**cp.__dict__, "delta": math.pi}),
                W.Params(**{**cp.__dict__, "delta": 1e-9})):     # ~1e10 events per sample
        with pytest.raises(T.TepaiError) as e:
            T.tepai_gnorm(prob, bad)
        assert e.value.code == 1
    bad = W.Params(**{**cp.__dict__, "variant": 4})
    with pytest.raises(T.TepaiError):
        T.tepai_gnorm(prob, bad)
