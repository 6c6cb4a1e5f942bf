"""The entry point that allocates no device memory, for callers that cannot
call cudaMalloc: a host application that gives each component a fixed device
budget, a plug-in that only receives buffers its framework allocated, or code
that must not pay cudaMalloc's implicit device synchronisation. Its scratch is
a fixed static device array. Its results
must equal those of the allocating entry point within the parity tolerances:
1e-10 in FP64 and 1e-4 in mixed precision. Two calls run back to back,
because every call reuses the same array."""
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


def _params(**kw):
    base = dict(T=0.5, n_steps=200, delta=math.pi / 64, n_samples=6, chi_max=8, cutoff=1e-12,
                n_snapshots=4, seed=3, precision=0)
    base.update(kw)
    return W.Params(**base)


def test_static_scratch_matches_allocating_entry_point_twice(T):
    import torch
    cases = [(W.spin_ring(6, 1.0, seed=1), _params(), 1e-10),
             (W.spin_ring(8, 1.0, seed=2), _params(chi_max=16, precision=1, seed=4), 1e-4)]
    ctx = T.tepai_create(0)
    try:
        for prob, par, tol in cases:
            want = T.tepai_sample_values(ctx, prob, par)
            v = torch.zeros((par.n_samples, par.n_snapshots, prob.n), dtype=torch.float64, device="cuda")
            sg = torch.zeros((par.n_samples, par.n_snapshots), dtype=torch.int8, device="cuda")
            T.tepai_sample_values_static(prob, par, v, sg)
            torch.cuda.synchronize()
            assert np.max(np.abs(v.cpu().numpy() - want["v"])) <= tol
            assert np.array_equal(sg.cpu().numpy(), want["sign"])
    finally:
        T.tepai_destroy(ctx)


def test_static_scratch_rejects_sizes_beyond_its_limit(T):
    import torch
    prob = W.spin_ring(64, 1.0, seed=0)
    par = _params(chi_max=512, n_samples=1, precision=1)      # one MPS arena exceeds 64 MiB
    v = torch.zeros((1, 4, 64), dtype=torch.float64, device="cuda")
    sg = torch.zeros((1, 4), dtype=torch.int8, device="cuda")
    with pytest.raises(T.TepaiError) as e:
        T.tepai_sample_values_static(prob, par, v, sg)
    assert e.value.code == 6


def test_static_scratch_with_pauli_string_observables(T):
    import torch
    n = 8
    prob = W.spin_ring(n, 1.0, seed=1)
    strings = np.zeros((3, n), dtype=np.uint8)
    strings[0, 1] = 2
    strings[1, [2, 3]] = [3, 3]
    strings[2, [0, 4, 7]] = [1, 2, 3]
    par = W.Params(T=0.3, n_steps=60, delta=math.pi / 64, n_samples=4, chi_max=16, cutoff=0.0,
                   n_snapshots=3, seed=9, precision=0, obs_strings=strings)
    ctx = T.tepai_create(0)
    try:
        ref = T.tepai_sample_values(ctx, prob, par)["v"]
    finally:
        T.tepai_destroy(ctx)
    dv = torch.zeros((4, 3, 3), dtype=torch.float64, device="cuda")
    ds = torch.zeros((4, 3), dtype=torch.int8, device="cuda")
    T.tepai_sample_values_static(prob, par, dv, ds)
    torch.cuda.synchronize()
    assert float(np.max(np.abs(dv.cpu().numpy() - ref))) <= 1e-12
