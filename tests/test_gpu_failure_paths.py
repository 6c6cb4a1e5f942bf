"""Bounded device waits that run out, and the run statistics of the C-ABI.

The Jacobi column handoff waits are bounded; a test-only knob
(TEPAI_TEST_HANDOFF_LIMIT, read when a workspace is prepared) gives every
handoff wait a few polls and a target no column reaches. The first wait of the
first Jacobi pass then runs out: the kernel must record device status 5,
stop the sample without touching memory, return, and leave the context usable
for the next run. No GPU fault or hang is involved."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2604_13144_gb300 import build
    build.build()
    from paper_2604_13144_gb300 import tepai
    return tepai


def _par(**kw):
    base = dict(T=0.5, n_steps=200, delta=math.pi / 64, n_samples=4, chi_max=8, cutoff=0.0,
                n_snapshots=4, seed=1, precision=1)
    base.update(kw)
    return W.Params(**base)


@pytest.mark.parametrize("precision", [1, 0])
def test_handoff_wait_runs_out_and_reports_status_5(T, monkeypatch, precision):
    import torch
    prob = W.spin_ring(6, 1.0, seed=0)
    par = _par(precision=precision)
    monkeypatch.setenv("TEPAI_TEST_HANDOFF_LIMIT", "16")
    run = T.DeviceRun(prob, par)
    v = torch.zeros((4, 4, 6), dtype=torch.float64, device="cuda")
    run.execute(v=v)
    torch.cuda.synchronize()                      # the kernel returned
    st = run.stats()
    assert st["device_status"][0] == 5, st["device_status"]
    run.release()
    monkeypatch.delenv("TEPAI_TEST_HANDOFF_LIMIT")
    # the context is still usable: the same problem now runs clean
    ctx = T.tepai_create(0)
    try:
        out = T.tepai_sample_values(ctx, prob, par)
        assert out["stats"]["device_status"][0] == 0
        assert np.all(np.isfinite(out["v"]))
    finally:
        T.tepai_destroy(ctx)


def test_host_call_returns_device_check_on_timeout(T, monkeypatch):
    prob = W.spin_ring(6, 1.0, seed=0)
    monkeypatch.setenv("TEPAI_TEST_HANDOFF_LIMIT", "16")
    ctx = T.tepai_create(0)
    try:
        with pytest.raises(T.TepaiError) as e:
            T.tepai_sample_values(ctx, prob, _par())
        assert e.value.code == 8
    finally:
        T.tepai_destroy(ctx)


def test_stats_report_seconds_and_mean_nu(T):
    prob = W.spin_ring(6, 1.0, seed=3)
    par = _par(n_samples=16)
    ctx = T.tepai_create(0)
    try:
        out = T.tepai_run(ctx, prob, par)
    finally:
        T.tepai_destroy(ctx)
    st = out["stats"]
    assert st["seconds"] > 0.0
    assert st["mean_nu"] == pytest.approx(st["events"] / 16)
    _, expected_nu = T.tepai_gnorm(prob, par)
    assert abs(st["mean_nu"] - expected_nu) < 6 * math.sqrt(expected_nu / 16) + 1
    assert st["jacobi_reorth"] >= 0
