"""The tensor-core Jacobi (launch variant 7, single precision, staged working
matrix of up to 256 rows): parity with the FP64 oracle on the same seeded
circuits at 1e-4 on every <Z_i>, with the Gram matrices and block updates
running on tcgen05 (tc_flops > 0), at bond caps that give full 32-column
blocks and 128-row tiles (chi = 128), and ragged ones (chi = 100: partial
blocks, a 72-row second tile)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle_rule import oracle_rule
from oracle import run as oracle_run

pytestmark = pytest.mark.gpu

TOLMIX = 1e-4


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


def _case(chi, n=16, seed=5, n_samples=2, steps=2):
    prob = W.spin_ring(n, 1.0, seed=seed, Jz=0.5)
    tens, dims = W.random_mps_tensors(n, chi, seed=seed + 100)
    par = W.Params(T=3.0, n_steps=18000, delta=math.pi / 1024, n_samples=n_samples, chi_max=chi,
                   cutoff=1e-10, n_snapshots=1, seed=7, precision=1, run_steps=steps)
    return prob, par, (tens, dims)


@pytest.mark.parametrize("chi", [128, 100])
def test_tensor_core_jacobi_matches_oracle(T, ctx, chi):
    prob, par, init = _case(chi)
    got = T.tepai_sample_values(ctx, prob, W.Params(**{**par.__dict__, "launch_variant": 7}), init)
    st = got["stats"]
    assert st["tc_flops"] > 0, st
    assert st["device_status"][0] == 0
    assert st["max_chi"] == chi
    ref = oracle_run.run(prob, par, init_tensors=init[0], **oracle_rule(par))
    err = np.abs(got["v"] - ref["v"])
    print("per-sample max |gpu - oracle|:", err.max(axis=(1, 2)), "sweeps/svd:",
          st["jacobi_sweeps"] / max(1.0, st["gate_updates"] + st["swap_updates"]), "reorth:", st["jacobi_reorth"])
    assert np.array_equal(got["sign"], ref["sign"])
    assert err.max() <= TOLMIX


def test_tensor_core_and_cuda_core_jacobi_agree(T, ctx):
    """The same circuits through launch variants 7 (tensor cores) and 2 (CUDA-core
    passes): two FP32 evaluations of the same SVDs agree within 1e-4."""
    prob, par, init = _case(128, n_samples=3, steps=1)
    a = T.tepai_sample_values(ctx, prob, W.Params(**{**par.__dict__, "launch_variant": 7}), init)
    b = T.tepai_sample_values(ctx, prob, W.Params(**{**par.__dict__, "launch_variant": 2}), init)
    assert a["stats"]["tc_flops"] > 0 and b["stats"]["tc_flops"] == 0
    assert np.max(np.abs(a["v"] - b["v"])) <= TOLMIX
