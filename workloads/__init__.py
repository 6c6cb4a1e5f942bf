"""Seeded synthetic inputs shared by the oracle-based tests, the CUDA parity
tests and the benchmark.

This module draws random numbers and lays out problem descriptions. It holds
none of the method's arithmetic: no rotation angles, no quasi-probabilities,
no gates and no tensor-network operations.

The workloads are disordered spin rings of the form given in Sec. III,
Eq. (spinRing): H = sum_k h_k Z_k + sum_bonds (Jx XX + Jy YY + Jz ZZ). The
on-site fields are drawn uniformly from [-a, a]. The initial states are
computational basis states such as |0101...>.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    """Hamiltonian and initial product state of one spin chain or ring."""
    n: int
    periodic: bool
    Jx: np.ndarray          # one coupling per bond: n bonds (ring) or n-1 (chain)
    Jy: np.ndarray
    Jz: np.ndarray
    h: np.ndarray           # one Z field per site
    init_bits: np.ndarray   # uint8, one computational-basis bit per site

    @property
    def n_bonds(self) -> int:
        return self.n if self.periodic else self.n - 1


@dataclasses.dataclass
class Params:
    """Run parameters of one TE-PAI ensemble (names follow the paper)."""
    T: float                  # total evolution time
    n_steps: int              # N, Trotter steps of the sampled product formula
    delta: float              # Delta, the fixed rotation angle of setting B
    n_samples: int            # N_s
    chi_max: int
    cutoff: float             # discarded-weight fraction allowed per update
    n_snapshots: int          # M, snapshots at j_m = m * run_steps / M
    seed: int = 0             # circuit-sampler seed
    sample_offset: int = 0    # global index of the first sample
    variant: int = 0          # 0 unbiased TE-PAI, 1 no-pi TE-PAI, 2 Trotter, 3 N -> infinity TE-PAI
    precision: int = 0        # 0 FP64, 1 mixed (FP32 tensors, FP64 bookkeeping)
    run_steps: int = 0        # steps actually run (0 = all n_steps)
    obs_sites: np.ndarray | None = None   # Z_i sites; None = all sites
    obs_strings: np.ndarray | None = None  # (n_obs, n) Pauli codes 0 I, 1 X, 2 Y, 3 Z per site;
                                           # replaces obs_sites when given
    tie_rel: float = 0.0      # tie band at truncation cuts (0 = only equal values are tied)
    launch_variant: int = 0   # launch shape of the CUDA path (0 = its default rule)
    three_site: int = 0       # 1 = bond-2 gates as one three-site update (0 = swap routing)

    def steps_run(self) -> int:
        return self.n_steps if self.run_steps == 0 else self.run_steps


def plus_minus_codes(n: int) -> np.ndarray:
    """|+...+ - +...+>: |+> on every site except |-> on site n // 2 (single-site
    state codes 2 and 3 of the product-state table)."""
    c = np.full(n, 2, dtype=np.uint8)
    c[n // 2] = 3
    return c


def neel_bits(n: int) -> np.ndarray:
    """|0101...>: site i holds bit (i mod 2)."""
    return (np.arange(n) % 2).astype(np.uint8)


def spin_ring(n: int, field_range: float, seed: int = 0, Jz: float = 1.0,
              J: float = 1.0, periodic: bool = True) -> Problem:
    """Disordered Heisenberg / XXZ ring with h_i ~ U[-a, a] drawn with
    numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    h = rng.uniform(-field_range, field_range, n)
    nb = n if periodic else n - 1
    return Problem(n=n, periodic=periodic,
                   Jx=np.full(nb, J), Jy=np.full(nb, J), Jz=np.full(nb, J * Jz),
                   h=h.astype(np.float64), init_bits=neel_bits(n))


def uniform_chain(n: int, c: float, periodic: bool = True) -> Problem:
    """All couplings and fields equal to c (every |c_k| equal)."""
    nb = n if periodic else n - 1
    return Problem(n=n, periodic=periodic, Jx=np.full(nb, c), Jy=np.full(nb, c),
                   Jz=np.full(nb, c), h=np.full(n, c), init_bits=neel_bits(n))


def random_mps_tensors(n: int, chi: int, seed: int, dtype=np.complex128):
    """Gaussian random site tensors A_i[chi_{i-1}][2][chi_i] with bond
    dimensions chi_i = min(chi, 2^(i+1), 2^(n-1-i)). No normalisation or
    canonical form is imposed; each consumer brings them to canonical form
    with its own code."""
    rng = np.random.default_rng(seed)
    dims = [1] + [min(chi, 2 ** (i + 1), 2 ** (n - 1 - i)) for i in range(n - 1)] + [1]
    out = []
    for i in range(n):
        shape = (dims[i], 2, dims[i + 1])
        a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        out.append(a.astype(dtype))
    return out, dims


# --------------------------------------------------------------------------
# The paper-scale workloads (all synthetic), by name.
# N for TE-PAI follows the deep-Trotter baseline N(T) = N_dT (T/dT)^2 with
# dT = 0.1 and N_dT = 20 (Sec. II.D, Eq. trotter-baseline-scaling).
# --------------------------------------------------------------------------

def trotter_baseline_steps(T: float, dT: float = 0.1, N_dT: int = 20) -> int:
    return int(round(N_dT * (T / dT) ** 2))


RING8 = "ring8_heisenberg_T1"
RING32 = "ring32_heisenberg_T2"
RING64_XXZ = "ring64_xxz_T3"
RING100 = "ring100_heisenberg_T4"
RING64_HYBRID = "ring64_hybrid_T2to5"


def workload(name: str) -> tuple[Problem, Params, dict]:
    """Return (problem, params, extra) of a named workload:
    ring8_heisenberg_T1    n = 8 Heisenberg ring, T = 1, chi 16, 1000 samples, <Z_0>;
    ring32_heisenberg_T2   n = 32, fields U[-2, 2], T = 2, chi 64, 10^4 samples;
    ring64_xxz_T3          n = 64 XXZ (Jz = 0.5), T = 3, chi 128, 10^5 samples;
    ring100_heisenberg_T4  n = 100, fields U[-3, 3], T = 4, chi 32 (and 256);
    ring64_hybrid_T2to5    n = 64, chi 256, TE-PAI on [2, 5] after a Trotter prefix."""
    if name == RING8:
        prob = spin_ring(8, 1.0, seed=0)
        par = Params(T=1.0, n_steps=trotter_baseline_steps(1.0), delta=math.pi / 256,
                     n_samples=1000, chi_max=16, cutoff=0.0, n_snapshots=10,
                     seed=0, precision=0, obs_sites=np.array([0], dtype=np.int32))
        return prob, par, {"trotter_steps": 100, "name": "ring8_heisenberg_T1"}
    if name == RING32:
        prob = spin_ring(32, 2.0, seed=0)
        par = Params(T=2.0, n_steps=trotter_baseline_steps(2.0), delta=math.pi / 512,
                     n_samples=10_000, chi_max=64, cutoff=1e-10, n_snapshots=20,
                     seed=0, precision=1)
        return prob, par, {"name": "ring32_heisenberg_T2"}
    if name == RING64_XXZ:
        prob = spin_ring(64, 1.0, seed=0, Jz=0.5)
        par = Params(T=3.0, n_steps=trotter_baseline_steps(3.0), delta=math.pi / 1024,
                     n_samples=100_000, chi_max=128, cutoff=1e-10, n_snapshots=1,
                     seed=0, precision=1)
        return prob, par, {"name": "ring64_xxz_T3"}
    if name == RING100:
        prob = spin_ring(100, 3.0, seed=0)
        par = Params(T=4.0, n_steps=trotter_baseline_steps(4.0), delta=math.pi / 1024,
                     n_samples=50_000, chi_max=32, cutoff=1e-10, n_snapshots=1,
                     seed=0, precision=1)
        return prob, par, {"name": "ring100_heisenberg_T4", "chi_alt": 256}
    if name == RING64_HYBRID:
        prob = spin_ring(64, 1.0, seed=0)
        par = Params(T=3.0, n_steps=trotter_baseline_steps(3.0), delta=math.pi / 1024,
                     n_samples=20_000, chi_max=256, cutoff=1e-10, n_snapshots=1,
                     seed=0, precision=1)
        return prob, par, {"name": "ring64_hybrid_T2to5", "t0": 2.0}
    raise ValueError(name)


# --------------------------------------------------------------------------
# Benchmark workload: steady state at chi = 128.
# The ring64_xxz_T3 ring (n = 64 XXZ, Jz = 0.5, h ~ U[-1, 1], T = 3,
# Delta = pi/1024, N = 18000, chi_max = 128, cutoff 1e-10). Every sample starts
# from one shared random MPS whose bonds are already at the cap, so that every
# two-site update runs at chi = 128. Each sample then evolves a window of the
# first `window_steps` Trotter steps of its own TE-PAI circuit and is measured
# once at the end of the window.
# --------------------------------------------------------------------------

def bench_workload(n_samples: int, window_steps: int = 2, sample_offset: int = 0,
                   chi: int = 128, mps_seed: int = 1234, n: int = 64):
    prob, par, extra = workload(RING64_XXZ)
    if n != prob.n:
        prob = spin_ring(n, 1.0, seed=0, Jz=0.5)
    par = Params(T=par.T, n_steps=par.n_steps, delta=par.delta, n_samples=n_samples,
                 chi_max=chi, cutoff=par.cutoff, n_snapshots=1, seed=par.seed,
                 sample_offset=sample_offset, precision=1, run_steps=window_steps)
    tensors, dims = random_mps_tensors(prob.n, chi, seed=mps_seed)
    return prob, par, (tensors, dims)
