"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, brute force, library routines). CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize

import workloads as W
from oracle import enumerate as en
from oracle import estimator, gates, planner, sampler
from oracle import mps as M
from oracle import run as R
from oracle import statevector as sv
from oracle.philox import philox4x64_scalar, philox4x64_vec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator
@pytest.mark.parametrize("key,ctr", [((0, 0), (1, 0, 0, 0)), ((5, 7), (3, 9, 0, 0)),
                                     ((2**64 - 1, 12345), (2**63 + 5, 2**40, 7, 1))])
def test_philox_matches_numpy_bitgenerator(key, ctr):
    # numpy's Philox (4x64-10) increments the counter before producing a block
    c = list(ctr)
    c[0] = (c[0] - 1) % 2**64
    ref = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(c, dtype=np.uint64)).random_raw(4)
    got = philox4x64_scalar(ctr, key)
    assert [int(x) for x in ref] == list(got)
    vec = philox4x64_vec(np.array([ctr[0]], np.uint64), np.array([ctr[1]], np.uint64),
                         np.array([ctr[2]], np.uint64), np.array([ctr[3]], np.uint64), *key)
    assert [int(v[0]) for v in vec] == list(got)


# ---------------------------------------------------------------- gates
@pytest.mark.parametrize("name", ["Z", "XX", "YY", "ZZ"])
def test_rotation_closed_form(name):
    P = gates.pauli_string(name)
    for th in (0.3, -1.1, math.pi):
        want = math.cos(th / 2) * np.eye(P.shape[0]) - 1j * math.sin(th / 2) * P
        assert np.allclose(gates.rotation(name, th), want, atol=1e-14)


# ---------------------------------------------------------------- P1: gammas
def _rand_rho(d, rng):
    a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    r = a @ a.conj().T
    return r / np.trace(r)


@pytest.mark.parametrize("name", ["Z", "XX", "YY", "ZZ"])
def test_pai_superoperator_identity(name):
    """gamma_1 A + gamma_2 B + gamma_3 C = R(theta) as superoperators (App. A.3)."""
    rng = np.random.default_rng(1)
    d = 2 ** len(name)
    for _ in range(20):
        delta = rng.uniform(0.01, math.pi)
        theta = rng.uniform(-delta, delta)
        g1, g2, g3 = planner.gammas(theta, delta)
        assert abs(g1 + g2 + g3 - 1.0) < 1e-14
        rho = _rand_rho(d, rng)
        Rt = gates.rotation(name, theta)
        B = gates.rotation(name, math.copysign(delta, theta))
        C = gates.rotation(name, math.pi)
        lhs = g1 * rho + g2 * B @ rho @ B.conj().T + g3 * C @ rho @ C.conj().T
        assert np.allclose(lhs, Rt @ rho @ Rt.conj().T, atol=1e-14)


def test_pai_signs_and_norm_under_assumption():
    for delta in (0.01, 0.5, 2.0):
        for t in np.linspace(0, delta, 7):
            g1, g2, g3 = planner.gammas(t, delta)
            assert g1 >= -1e-15 and g2 >= 0 and g3 <= 1e-15
            # ||gamma||_1 = 1 - 2 gamma_3 >= 1
            assert abs(abs(g1) + abs(g2) + abs(g3) - (1 - 2 * g3)) < 1e-14


# ---------------------------------------------------------------- golden: App. A.5
def test_nu_inf_minimum_matches_paper_constants():
    gold = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    f = lambda d: (3 - math.cos(d)) / math.sin(d)
    res = scipy.optimize.minimize_scalar(f, bounds=(0.05, 3.0), method="bounded",
                                         options={"xatol": 1e-12})
    assert abs(res.fun - gold["nu_inf_min_prefactor"]) < 1e-10
    assert abs(res.x - gold["nu_inf_argmin_delta"]) < 1e-5
    assert abs(res.x / math.pi - gold["nu_inf_argmin_delta_over_pi_printed"]) < 5e-4
    # the oracle's nu_inf reproduces the bound with ||c||_1 T = 1
    prob = W.uniform_chain(2, 0.2, periodic=False)        # 5 terms, ||c||_1 = 1
    assert abs(planner.nu_infinity(prob, 1.0, gold["nu_inf_argmin_delta"])
               - gold["nu_inf_min_prefactor"]) < 1e-12


# ---------------------------------------------------------------- P2
def test_delta_equals_theta_is_deterministic_trotter():
    prob = W.uniform_chain(5, 0.5, periodic=True)
    T, N = 1.0, 20
    delta = 2 * 0.5 * T / N
    plan = planner.make_plan(prob, T, N, delta)
    assert np.allclose(plan.gam, [[0.0, 1.0, 0.0]] * len(plan.terms), atol=1e-15)
    ev = sampler.sample_events(plan, 3, 11, N)
    assert len(ev) == N * len(plan.terms) and np.all(ev[:, 2] == sampler.EV_B)
    tplan = planner.make_plan(prob, T, N, delta, planner.TROTTER)
    snaps = planner.snapshot_steps(N, 4)
    z_tepai = sv.run_events(prob.init_bits, plan, ev, snaps)
    z_trot = sv.run_events(prob.init_bits, tplan, sampler.sample_events(tplan, 0, 0, N), snaps)
    assert np.max(np.abs(z_tepai - z_trot)) < 1e-12


# ---------------------------------------------------------------- P3
@pytest.mark.parametrize("n,N", [(2, 2), (3, 1)])
def test_enumeration_is_unbiased(n, N):
    """Statement 1: sum_l g_l <Z>_l over all settings = N-step Trotter value."""
    prob = W.spin_ring(n, 1.0, seed=4, periodic=False)
    T, delta = 0.2 * N, 0.5
    plan = planner.make_plan(prob, T, N, delta)
    assert planner.check_theta(plan)
    z, gabs = en.enumerate_all(prob, plan, N)
    tplan = planner.make_plan(prob, T, N, delta, planner.TROTTER)
    z_trot = sv.run_events(prob.init_bits, tplan, sampler.sample_events(tplan, 0, 0, N), [N])[0]
    assert np.max(np.abs(z - z_trot)) < 1e-12
    assert abs(gabs - plan.gnorm_step ** N) < 1e-12


# ---------------------------------------------------------------- P4
def test_mean_gate_count_and_setting_frequencies():
    prob = W.spin_ring(4, 1.0, seed=2)
    T, N, delta = 1.0, 200, math.pi / 64
    plan = planner.make_plan(prob, T, N, delta)
    Ns = 3000
    nus, ncs = [], []
    for s in range(Ns):
        ev = sampler.sample_events(plan, 7, s, N)
        nus.append(len(ev))
        ncs.append(int(np.count_nonzero(ev[:, 2] == sampler.EV_C)))
    nus = np.array(nus, dtype=float)
    mean_exact = N * plan.q.sum()
    var_exact = N * np.sum(plan.q * (1 - plan.q))
    assert abs(nus.mean() - mean_exact) < 4 * math.sqrt(var_exact / Ns)
    assert abs(nus.var(ddof=1) / var_exact - 1) < 0.1
    pc = N * np.sum(plan.q * plan.r)
    assert abs(np.mean(ncs) - pc) < 4 * math.sqrt(pc / Ns) + 1e-9


def test_expected_gate_count_tends_to_nu_inf():
    prob, par, _ = W.workload(W.RING32)
    prev = None
    for N in (2000, 8000, 32000):
        plan = planner.make_plan(prob, par.T, N, par.delta)
        rel = abs(planner.expected_nu(plan, N) - planner.nu_infinity(prob, par.T, par.delta)) \
            / planner.nu_infinity(prob, par.T, par.delta)
        if prev is not None:
            assert rel < prev
        prev = rel
    assert prev < 1e-3


# ---------------------------------------------------------------- P5
def test_gnorm_tends_to_limit():
    prob, par, _ = W.workload(W.RING8)
    lim = planner.gnorm_infinity(prob, par.T, par.delta)
    rels = []
    for N in (2000, 20000, 200000):
        plan = planner.make_plan(prob, par.T, N, par.delta)
        rels.append(abs(plan.gnorm_step ** N / lim - 1))
    assert rels[0] > rels[1] > rels[2] and rels[2] < 5e-4


# ---------------------------------------------------------------- P6
@pytest.mark.parametrize("n", [5, 6])
def test_untruncated_mps_equals_statevector(n):
    prob = W.spin_ring(n, 1.0, seed=n)
    T, N, delta = 1.0, 60, math.pi / 24
    par = W.Params(T=T, n_steps=N, delta=delta, n_samples=3, chi_max=2 ** (n // 2),
                   cutoff=0.0, n_snapshots=3, seed=5)
    r1 = R.run(prob, par)
    r2 = R.run(prob, par, use_statevector=True)
    assert np.max(np.abs(r1["v"] - r2["v"])) < 1e-12
    assert sum(st["swap_updates"] for st in r1["stats"]) > 0      # ring routing exercised


# ---------------------------------------------------------------- P7
def test_trotter_mode_mps_equals_statevector_and_conserves_magnetisation():
    prob = W.spin_ring(8, 1.0, seed=0)
    par = W.Params(T=1.0, n_steps=100, delta=math.pi / 256, n_samples=1, chi_max=16,
                   cutoff=0.0, n_snapshots=5, variant=planner.TROTTER)
    r1 = R.run(prob, par)
    r2 = R.run(prob, par, use_statevector=True)
    assert np.max(np.abs(r1["v"] - r2["v"])) < 1e-12
    assert np.max(np.abs(r1["v"].sum(axis=2))) < 1e-12


# ---------------------------------------------------------------- P8
def test_tepai_mean_converges_to_trotter_and_exact():
    prob = W.spin_ring(4, 1.0, seed=3)
    T, N, delta = 1.0, 100, math.pi / 16
    par = W.Params(T=T, n_steps=N, delta=delta, n_samples=1500, chi_max=4, cutoff=0.0,
                   n_snapshots=4, seed=9)
    r = R.run(prob, par, use_statevector=True)
    tpar = W.Params(T=T, n_steps=N, delta=delta, n_samples=1, chi_max=4, cutoff=0.0,
                    n_snapshots=4, variant=planner.TROTTER)
    zt = R.run(prob, tpar, use_statevector=True)["v"][0]
    dev = np.abs(r["mean"] - zt)
    assert np.all(dev <= 4 * r["stderr"] + 1e-12)
    # Statement 2: Var[v] <= 1 for the signed per-configuration values
    assert np.all(np.var(r["sign"][:, :, None] * r["v"], axis=0) <= 1.0)
    times = [T * j / N for j in r["snaps"]]
    ze = sv.exact_z(prob, times)
    # exact evolution within the statistical band plus the first-order Trotter error
    assert np.all(np.abs(r["mean"] - ze) <= 4 * r["stderr"] + np.abs(zt - ze) + 1e-12)


# ---------------------------------------------------------------- P9
def test_two_site_heisenberg_closed_form():
    J = 0.7
    prob = W.Problem(n=2, periodic=False, Jx=np.array([J]), Jy=np.array([J]),
                     Jz=np.array([J]), h=np.zeros(2), init_bits=np.array([0, 1], np.uint8))
    ts = np.linspace(0, 2, 9)
    z = sv.exact_z(prob, ts)
    assert np.allclose(z[:, 0], np.cos(4 * J * ts), atol=1e-12)
    assert np.allclose(z[:, 1], -np.cos(4 * J * ts), atol=1e-12)


def test_single_qubit_rotation_expectation():
    psi = sv.basis_state([0])
    for phi in (0.2, 1.3, 2.9):
        out = sv.apply_1(psi, gates.rotation('X', phi) if False else
                         np.array([[math.cos(phi / 2), -1j * math.sin(phi / 2)],
                                   [-1j * math.sin(phi / 2), math.cos(phi / 2)]]), 0)
        assert abs(sv.expect_z(out)[0] - math.cos(phi)) < 1e-14


# ---------------------------------------------------------------- P10
def test_no_pi_variant():
    prob = W.spin_ring(6, 1.0, seed=1)
    T, N, delta = 1.0, 200, math.pi / 64
    plan = planner.make_plan(prob, T, N, delta, planner.NO_PI)
    assert abs(plan.gnorm_step - 1.0) < 1e-15
    assert np.allclose(plan.q, np.abs(plan.theta) / delta, atol=1e-15)
    for s in range(20):
        ev = sampler.sample_events(plan, 1, s, N)
        assert not np.any(ev[:, 2] == sampler.EV_C)
        assert sampler.sign_after(ev, N) == 1


# ---------------------------------------------------------------- estimator
def test_neumaier_against_fsum():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(1000) * 1e16, rng.standard_normal(1000),
                        -rng.standard_normal(1000) * 1e16])
    rng.shuffle(x)
    s, c = estimator.neumaier(x)
    assert abs((s + c) - math.fsum(x)) <= 2.0


def test_estimate_matches_plain_mean_and_std():
    rng = np.random.default_rng(1)
    v = rng.uniform(-1, 1, (500, 3, 4))
    sg = rng.choice([-1, 1], (500, 3)).astype(np.int8)
    gn = np.array([1.0, 1.5, 2.0])
    mean, se, part = estimator.estimate(v, sg, gn)
    x = sg[:, :, None] * v
    assert np.allclose(mean, gn[:, None] * x.mean(axis=0), atol=1e-15)
    assert np.allclose(se, gn[:, None] * x.std(axis=0, ddof=1) / math.sqrt(500), atol=1e-14)


# ---------------------------------------------------------------- truncation / MPS
def _keep_brute(s, chi, cut, floor_rel, gap_rel):
    """The keep rule by exhaustive search over cut positions: the target is the
    largest kk that is at most chi, at most the number of values above the
    floor, and at most the first kk whose discarded tail is within the cutoff.
    When the value right after the target is above the floor, the cut must sit
    at a clear gap (s_{kk-1} - s_kk > gap_rel s_0): the largest such kk at or
    below the target wins, and without one the target stays."""
    n = len(s)
    tot = float(np.sum(s ** 2))
    tails = [float(np.sum(s[kk:] ** 2)) for kk in range(n + 1)]
    k_cut = next(kk for kk in range(1, n + 1) if tails[kk] <= cut * tot or kk == n)
    above = [j for j in range(n) if s[j] > floor_rel * s[0]]
    target = max(1, min([chi, len(above), k_cut, n]))
    if target == n or not (s[target] > floor_rel * s[0]):
        return target
    clear = [kk for kk in range(1, target + 1) if s[kk - 1] - s[kk] > gap_rel * s[0]]
    return max(clear) if clear else target


@pytest.mark.parametrize("floor_rel,gap_rel", [(1e-14, 1e-12), (1e-14, 1e-4), (4e-6, 1e-4), (4e-6, 1e-12)])
def test_keep_count_brute_force(floor_rel, gap_rel):
    """keep_count against the brute-force rule, with planted exact ties, near
    ties inside and outside the band (gaps of 0.5 and 2 band widths measured
    against s_0, so a band taken relative to s_k instead of s_0 fails), and
    values planted just below and above the floor."""
    rng = np.random.default_rng(2)
    planted = {"tie": 0, "in": 0, "out": 0, "floor": 0}
    for _ in range(1500):
        s = np.sort(rng.exponential(1.0, rng.integers(1, 14)) ** 3)[::-1]
        if len(s) > 2:
            i = int(rng.integers(1, len(s) - 1))
            kind = rng.choice(["tie", "in", "out", "floor", "none"])
            if kind == "tie":
                s[i + 1] = s[i]
            elif kind == "in":
                s[i + 1] = max(s[i] - 0.5 * gap_rel * s[0], 0.0)
            elif kind == "out":
                s[i + 1] = max(s[i] - 2.0 * gap_rel * s[0], 0.0)
            elif kind == "floor":
                s[i] = (0.5 if rng.random() < 0.5 else 2.0) * floor_rel * s[0]
                s[i + 1:] = np.minimum(s[i + 1:], s[i])
            s = np.sort(s)[::-1]
            if kind in planted:
                planted[kind] += 1
        chi, cut = int(rng.integers(1, 12)), float(10.0 ** rng.uniform(-14, -0.5))
        k = M.keep_count(s, chi, cut, floor_rel, gap_rel=gap_rel)
        assert k == _keep_brute(s, chi, cut, floor_rel, gap_rel), (s, chi, cut, k)
    assert min(planted.values()) > 100


def test_keep_count_default_is_the_paper_rule():
    """Default band: only equal values are held together; a gap of 1e-9 s_0
    (far above FP64 rounding) is a valid cut, and an exact tie is not."""
    s = np.array([1.0, 0.5, 0.5 - 1e-9, 0.2])
    assert M.keep_count(s, 2, 0.0, 1e-14) == 2
    s = np.array([1.0, 0.5, 0.5, 0.2])
    assert M.keep_count(s, 2, 0.0, 1e-14) == 1
    assert M.PAPER_TIE_REL == 1e-12


def test_truncated_update_discards_weight_per_eckart_young():
    rng = np.random.default_rng(3)
    ts, _ = W.random_mps_tensors(6, 8, seed=4)
    m = M.canonicalize(ts)
    before = M.expect_z(m)
    M.move_centre(m, 2)
    th = np.tensordot(m.A[2], m.A[3], axes=(2, 0))
    g = gates.rotation('XX', 0.7)
    th = np.einsum('stuv,auvb->astb', g.reshape(2, 2, 2, 2), th)
    s = np.linalg.svd(th.reshape(th.shape[0] * 2, -1), compute_uv=False)
    M.apply_two(m, 2, g, chi_max=3, cutoff=0.0, floor_rel=1e-14)
    th2 = np.tensordot(m.A[2], m.A[3], axes=(2, 0)).reshape(th.shape[0] * 2, -1)
    # rebuilt theta is the best rank-3 approximation, rescaled to unit norm
    best = np.sum(s[:3] ** 2)
    err = np.linalg.norm(th2 * math.sqrt(best) - th.reshape(th2.shape)) ** 2
    assert abs(err - np.sum(s[3:] ** 2)) < 1e-12
    assert m.stats["max_chi"] == 3
    assert before.shape == (6,)


def _dense_from_tensors(ts):
    psi = ts[0]
    for a in ts[1:]:
        psi = np.tensordot(psi, a, axes=(psi.ndim - 1, 0))
    return psi.reshape((2,) * len(ts))


def test_canonicalize_and_measure_against_dense_contraction():
    ts, _ = W.random_mps_tensors(7, 4, seed=8)
    psi = _dense_from_tensors(ts)
    want = sv.expect_z(psi)
    m = M.canonicalize(ts)
    assert np.allclose(M.expect_z(m), want, atol=1e-12)
    # right-canonical: sum_s A^s A^s^dag = I for sites > 0
    for a in m.A[1:]:
        mat = a.reshape(a.shape[0], -1)
        assert np.allclose(mat @ mat.conj().T, np.eye(a.shape[0]), atol=1e-12)


def test_oracle_does_not_import_product_package():
    here = os.path.join(os.path.dirname(os.path.dirname(__file__)), "oracle")
    for f in os.listdir(here):
        if f.endswith(".py"):
            src = open(os.path.join(here, f)).read()
            assert "paper_2604_13144_gb300" not in src
            assert "import workloads" not in src


def test_regauge_leaves_untruncated_results_unchanged():
    """The gauge change used to measure conditioning is exact: without
    truncation both gauges give the same <Z_i> to rounding."""
    prob = W.spin_ring(6, 1.0, seed=6)
    par = W.Params(T=0.5, n_steps=100, delta=math.pi / 32, n_samples=2, chi_max=8, cutoff=0.0,
                   n_snapshots=2, seed=2)
    a = R.run(prob, par)
    b = R.run(prob, par, regauge=True)
    assert np.max(np.abs(a["v"] - b["v"])) < 1e-12
    assert sum(s["qr_moves"] for s in b["stats"]) > sum(s["qr_moves"] for s in a["stats"])


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 9, 64])
def test_folded_ring_order_keeps_bonds_within_distance_two(n):
    order = M.chain_order(n, True)
    assert sorted(order) == list(range(n))
    pos = {s: p for p, s in enumerate(order)}
    for i in range(n):
        assert abs(pos[i] - pos[(i + 1) % n]) <= 2
    assert M.chain_order(n, False) == list(range(n))


# ---- general observables and product initial states ----------------------

def test_pauli_strings_mps_equal_state_vector():
    """Two independent evaluations of Pauli-string expectations (full-chain MPS
    contraction vs. operators applied to the dense state vector) agree on an
    evolved, untruncated state; ring order included."""
    from oracle import mps as M, statevector as S, planner as Pl, sampler as Sa
    n = 6
    prob = W.spin_ring(n, 1.0, seed=4)
    prob.init_bits = np.array([2, 0, 5, 1, 3, 4], dtype=np.uint8)
    plan = Pl.make_plan(prob, 0.3, 40, math.pi / 32, 0)
    ev = Sa.sample_events(plan, 7, 3, 40)
    m = M.product_state(prob.init_bits, True)
    M.run_events(m, plan, ev, [40], 64, 0.0)
    psi = S.basis_state(prob.init_bits)
    for e in ev:
        psi = S.apply_event(psi, plan, int(e[1]), int(e[2]))
    rng = np.random.default_rng(1)
    for _ in range(12):
        codes = np.zeros(n, dtype=np.int64)
        k = int(rng.integers(1, 4))
        sites = rng.choice(n, size=k, replace=False)
        codes[sites] = rng.integers(1, 4, size=k)
        assert abs(M.expect_string(m, codes) - S.expect_string(psi, codes)) <= 1e-12


def test_product_state_codes_give_single_site_values():
    from oracle import mps as M
    codes = np.array([0, 1, 2, 3, 4, 5], dtype=np.uint8)
    m = M.product_state(codes, False)
    want = {1: [0, 0, 1, -1, 0, 0], 2: [0, 0, 0, 0, 1, -1], 3: [1, -1, 0, 0, 0, 0]}
    for p, vals in want.items():
        for i, v in enumerate(vals):
            s = np.zeros(6, dtype=np.int64)
            s[i] = p
            assert abs(M.expect_string(m, s) - v) <= 1e-15
    # a string on a product state factorises: <X_2 Y_4 Z_0> = 1 * 1 * 1
    assert abs(M.expect_string(m, np.array([3, 0, 1, 0, 2, 0])) - 1.0) <= 1e-15
    assert abs(M.expect_string(m, np.array([3, 0, 1, 1, 0, 0])) + 1.0) <= 1e-15


def test_two_site_heisenberg_from_plus_minus_gives_cos4t():
    """H = XX + YY + ZZ on an open pair (no fields) from |+->: the three terms
    commute, so the Trotter product is exact, and by SU(2) symmetry
    <X_0>(t) = cos(4t), the X-basis image of the |01> case."""
    prob = W.Problem(n=2, periodic=False, Jx=np.array([1.0]), Jy=np.array([1.0]), Jz=np.array([1.0]),
                     h=np.zeros(2), init_bits=np.array([2, 3], dtype=np.uint8))
    par = W.Params(T=0.7, n_steps=7, delta=0.5, n_samples=1, chi_max=4, cutoff=0.0, n_snapshots=7,
                   seed=0, variant=2, obs_strings=np.array([[1, 0]]))
    from oracle import run as oracle_run
    r = oracle_run.run(prob, par)
    ts = 0.1 * np.arange(1, 8)
    assert np.allclose(r["v"][0, :, 0], np.cos(4 * ts), atol=1e-12, rtol=0)


# ---------------------------------------------------------------- P15
def test_continuous_rates_are_the_finite_n_limit():
    """The N -> infinity sampler's rates are the limits of the finite-N draw
    probabilities built from Eq. gammas: q_k N / T -> lam_k, r_k -> r_inf,
    ||g||_1 -> exp(2 tan(Delta/2) ||c||_1 T)."""
    prob, par, _ = W.workload(W.RING8)
    cp = planner.make_plan(prob, par.T, par.n_steps, par.delta, planner.CONTINUOUS)
    errs = []
    for N in (10 ** 4, 10 ** 5, 10 ** 6):
        fp = planner.make_plan(prob, par.T, N, par.delta)
        e_lam = np.max(np.abs(fp.q * N / par.T - cp.lam) / cp.lam)
        e_r = np.max(np.abs(fp.r - cp.r_inf)) / cp.r_inf
        e_g = abs(fp.gnorm_step ** N / planner.gnorm_time(cp, par.T) - 1)
        errs.append(max(e_lam, e_r, e_g))
        assert np.array_equal(cp.phi, fp.phi)          # setting B = R_k(sign(theta) Delta)
    # first-order convergence: the error falls tenfold per tenfold N
    assert 8 < errs[0] / errs[1] < 12 and 8 < errs[1] / errs[2] < 12 and errs[2] < 5e-4
    assert abs(np.sum(cp.lam) * par.T / planner.nu_infinity(prob, par.T, par.delta) - 1) < 1e-14


def test_continuous_sampler_counts_and_times():
    """Poisson law of the continuous sampler: per term, E[count] = lam_k t_M with
    variance equal to the mean, so the total gate count has mean nu_inf and
    standard deviation sqrt(nu_inf), the limit law App. A.5 states; the C
    fraction is r_inf; given the count, the event times are uniform on
    [0, t_M] (mean t_M / 2)."""
    prob = W.spin_ring(4, 1.0, seed=2)
    par = W.Params(T=1.0, n_steps=100, delta=math.pi / 8, n_samples=1, chi_max=4, cutoff=0.0,
                   n_snapshots=4, variant=planner.CONTINUOUS)
    plan = planner.make_plan(prob, par.T, par.n_steps, par.delta, planner.CONTINUOUS)
    ts = planner.snapshot_times(plan, par.steps_run(), par.n_snapshots)
    L = len(plan.terms)
    Ns = 1500
    cnt = np.zeros((Ns, L))
    nc, tsum, ntot = 0, 0.0, 0
    for s in range(Ns):
        ev, tt = sampler.sample_events_continuous(plan, 11, s, ts)
        assert np.all(np.diff(tt) >= 0) and np.all((tt > 0) & (tt <= ts[-1]))
        # snapshot index: first m with t <= t_m
        assert np.all(tt <= ts[ev[:, 0] - 1])
        assert np.all((ev[:, 0] == 1) | (tt > ts[np.maximum(ev[:, 0] - 2, 0)]))
        np.add.at(cnt[s], ev[:, 1], 1)
        nc += int(np.sum(ev[:, 2] == sampler.EV_C))
        tsum += float(np.sum(tt))
        ntot += len(tt)
    mu = plan.lam * ts[-1]
    assert np.all(np.abs(cnt.mean(axis=0) - mu) < 4 * np.sqrt(mu / Ns))
    tot = cnt.sum(axis=1)
    assert abs(tot.var(ddof=1) / mu.sum() - 1) < 0.15
    assert abs(nc / ntot - plan.r_inf) < 4 * math.sqrt(plan.r_inf * (1 - plan.r_inf) / ntot)
    assert abs(tsum / ntot - ts[-1] / 2) < 4 * ts[-1] / math.sqrt(12 * ntot)


def test_continuous_mean_is_unbiased_for_exact_evolution():
    """In the N -> infinity limit the sampled circuits carry no Trotter error:
    the signed, ||g||_1-weighted mean estimates <Z_i>(t) of exp(-iHt) itself."""
    prob = W.spin_ring(4, 1.0, seed=3)
    # |0>|+i>|1>|+>: a start state that is not real, so that <Z_i>(t) differs
    # from <Z_i>(-t) and a sign error in the B rotations shows
    prob.init_bits = np.array([0, 4, 1, 2])
    par = W.Params(T=0.25, n_steps=100, delta=math.pi / 8, n_samples=3000, chi_max=4,
                   cutoff=0.0, n_snapshots=4, seed=9, variant=planner.CONTINUOUS)
    r = R.run(prob, par, use_statevector=True)
    ze = sv.exact_z(prob, list(r["times"]))
    assert np.all(np.abs(r["mean"] - ze) <= 4 * r["stderr"] + 1e-12)
    # the estimate resolves the dynamics: exact values move well beyond the band
    assert np.max(np.abs(ze - ze[0])) > 10 * np.max(r["stderr"])
    assert abs(r["gnorm"][-1] - planner.gnorm_infinity(prob, par.T, par.delta)) < 1e-12


def test_continuous_mps_equals_statevector():
    prob = W.spin_ring(6, 1.0, seed=4)
    par = W.Params(T=0.6, n_steps=100, delta=math.pi / 16, n_samples=3, chi_max=8,
                   cutoff=0.0, n_snapshots=3, seed=2, variant=planner.CONTINUOUS)
    r1 = R.run(prob, par)
    r2 = R.run(prob, par, use_statevector=True)
    assert np.max(np.abs(r1["v"] - r2["v"])) < 1e-12
    assert np.array_equal(r1["sign"], r2["sign"]) and np.all(r1["nu"] > 0)


# ---------------------------------------------------------------- P16
@pytest.mark.parametrize("n", [5, 6, 7])
def test_three_site_update_untruncated_equals_statevector(n):
    """Bond-2 gates as one three-site update (no swaps) reproduce the exact
    circuit when nothing is truncated."""
    prob = W.spin_ring(n, 1.0, seed=n)
    par = W.Params(T=1.0, n_steps=60, delta=math.pi / 24, n_samples=3, chi_max=2 ** (n // 2),
                   cutoff=0.0, n_snapshots=3, seed=5)
    r1 = R.run(prob, par, three_site=True)
    r2 = R.run(prob, par, use_statevector=True)
    assert np.max(np.abs(r1["v"] - r2["v"])) < 1e-12
    assert all(st["three_site_updates"] > 0 and st["swap_updates"] == 0 for st in r1["stats"])
    # moving the centre back after each update is a change of gauge only
    r3 = R.run(prob, par, three_site=True, regauge=True)
    assert np.max(np.abs(r3["v"] - r2["v"])) < 1e-12


def test_three_site_truncation_fidelity_is_the_product_of_kept_weights():
    """Truncating the first split projects onto the kept left Schmidt vectors
    (kept weight 1 - e1); the second split's kept subspace lies inside that
    range, so the truncated state has fidelity exactly (1 - e1)(1 - e2) with
    the exact gated state. Checked against a dense contraction."""
    rng = np.random.default_rng(4)
    ts, _ = W.random_mps_tensors(8, 8, seed=11)
    m = M.canonicalize(ts)
    psi = _dense_from_tensors(m.A)
    psi = psi / np.linalg.norm(psi)
    g, _ = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))
    # dense gate on sites 2 and 4 of the open chain (basis |s_2 s_4>)
    ex = np.einsum('xysu,abscudef->abxcydef', g.reshape(2, 2, 2, 2), psi.reshape([2] * 8)).reshape(-1)
    e1, e2 = M.apply_three(m, 2, g, chi_max=5, cutoff=0.0, floor_rel=1e-14)
    assert e1 > 1e-4 and e2 > 1e-4
    got = _dense_from_tensors(m.A)
    assert abs(np.linalg.norm(got) - 1.0) < 1e-12
    fid = abs(np.vdot(ex, got)) ** 2
    assert abs(fid - (1 - e1) * (1 - e2)) < 1e-12
    # left-orthonormal sites 2 and 3, centre on 4
    for p in (2, 3):
        a = m.A[p].reshape(-1, m.A[p].shape[2])
        assert np.allclose(a.conj().T @ a, np.eye(a.shape[1]), atol=1e-12)
    assert m.c == 4


def test_three_site_truncates_less_than_swap_routing():
    """On a truncated ring (12 sites, chi = 8) the three-site update, which
    truncates twice per bond-2 gate instead of three times, stays closer to the
    exact circuit in every sample."""
    prob = W.spin_ring(12, 1.0, seed=5)
    par = W.Params(T=1.0, n_steps=100, delta=math.pi / 16, n_samples=6, chi_max=8, cutoff=0.0,
                   n_snapshots=4, seed=2)
    a = R.run(prob, par)
    b = R.run(prob, par, three_site=True)
    c = R.run(prob, par, use_statevector=True)
    ea = np.mean(np.abs(a["v"] - c["v"]), axis=(1, 2))
    eb = np.mean(np.abs(b["v"] - c["v"]), axis=(1, 2))
    assert np.all(eb < ea) and np.mean(eb) < 0.7 * np.mean(ea)


# ---------------------------------------------------------------- P4b
def test_finite_n_gaps_are_geometric():
    """Independent per-gate draws: the steps between successive events of one
    term follow Geometric(q_k) (chi-squared test over gap bins); a counter
    or key mix-up that correlated draws across steps would fail it."""
    import scipy.stats as st
    prob = W.spin_ring(4, 1.0, seed=2)
    T, N, delta = 1.0, 40, math.pi / 16
    plan = planner.make_plan(prob, T, N, delta)
    k = int(np.argmax(plan.q))
    q = float(plan.q[k])
    assert 0.2 < q < 0.8
    # from each start point (step 0 or an event of term k) with at least 6
    # steps left, the next event of term k comes 1..6 steps later or not
    # within 6 steps: fully observed categories, i.i.d. Geometric(q) by the
    # independence of the draws
    obs = np.zeros(7)
    for s in range(1500):
        ev = sampler.sample_events(plan, 3, s, N)
        j = ev[ev[:, 1] == k, 0]
        for j0 in np.concatenate([[0], j]):
            if j0 > N - 6:
                break
            nxt = j[j > j0]
            g = int(nxt[0] - j0) if len(nxt) else N + 1
            obs[min(g, 7) - 1] += 1
    p = np.array([q * (1 - q) ** (g - 1) for g in range(1, 7)] + [(1 - q) ** 6])
    exp = p * obs.sum()
    chi2 = float(np.sum((obs - exp) ** 2 / exp))
    assert st.chi2.sf(chi2, len(obs) - 1) > 1e-3, (obs, exp)


def test_continuous_gaps_are_exponential():
    """Waiting times between successive events of one term in the N -> infinity
    sampler are Exp(lam_k) (Kolmogorov-Smirnov), and C marks are independent of
    the gaps (equal mean gap before B and C events within the statistics)."""
    import scipy.stats as st
    prob = W.spin_ring(4, 1.0, seed=2)
    par = W.Params(T=1.0, n_steps=100, delta=math.pi / 4, n_samples=1, chi_max=4, cutoff=0.0,
                   n_snapshots=2, variant=planner.CONTINUOUS)
    plan = planner.make_plan(prob, par.T, par.n_steps, par.delta, planner.CONTINUOUS)
    ts = planner.snapshot_times(plan, par.steps_run(), par.n_snapshots)
    k = int(np.argmax(plan.lam))
    lam = float(plan.lam[k])
    # from each start point (t = 0 or an event of term k) at least `cut` before
    # t_M, the wait to the next event of term k is observed if it is < cut:
    # such waits follow Exp(lam) conditioned on < cut
    cut = ts[-1] / 2
    g, gaps, marks = [], [], []
    for s in range(1500):
        ev, tt = sampler.sample_events_continuous(plan, 5, s, ts)
        sel = ev[:, 1] == k
        t = tt[sel]
        gaps.extend(np.diff(np.concatenate([[0.0], t])).tolist())
        marks.extend(ev[sel, 2].tolist())
        for t0 in np.concatenate([[0.0], t]):
            if t0 > ts[-1] - cut:
                break
            nxt = t[t > t0]
            if len(nxt) and nxt[0] - t0 < cut:
                g.append(nxt[0] - t0)
    gaps = np.array(gaps)
    marks = np.array(marks)
    cdf = lambda x: (1 - np.exp(-lam * x)) / (1 - math.exp(-lam * cut))
    assert len(g) > 1000 and st.kstest(np.array(g), cdf).pvalue > 1e-3
    c = marks == sampler.EV_C
    assert c.sum() > 100
    d = gaps[c].mean() - gaps[~c].mean()
    assert abs(d) < 4 * gaps.std() * math.sqrt(1 / c.sum() + 1 / (~c).sum())
