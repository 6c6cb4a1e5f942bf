"""Host planner of the oracle: term list, angles and PAI tables in FP64.

Follows App. A.3 (Eq. productFormula, Eq. settings, Eq. gammas), App. A.4
(no-pi variant), App. A.5 (Eq. ap:eq_nu_infty) and App. A.6
(Eq. overhead-bound, Eq. overhead).

Term order inside one Trotter step: Z_0 .. Z_{n-1}, then for every bond
b = 0 .. nb-1 the three terms XX_b, YY_b, ZZ_b. On a ring, bond n-1 joins
sites n-1 and 0. The paper writes prod_{k=1}^L without fixing an order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

UNBIASED, NO_PI, TROTTER, CONTINUOUS = 0, 1, 2, 3


@dataclasses.dataclass
class Term:
    pauli: str     # 'Z' (single site) or 'XX', 'YY', 'ZZ' (bond)
    site: int      # single-site: the site; bond: the bond index b
    a: int         # first site acted on
    b: int         # second site acted on (== a for single-site terms)
    c: float       # coefficient c_k


def term_list(prob) -> list[Term]:
    """H = sum_k c_k h_k for the spin ring of Sec. III, Eq. (spinRing)."""
    terms = [Term('Z', i, i, i, float(prob.h[i])) for i in range(prob.n)]
    nb = prob.n if prob.periodic else prob.n - 1
    for bnd in range(nb):
        a, b = bnd, (bnd + 1) % prob.n
        terms.append(Term('XX', bnd, a, b, float(prob.Jx[bnd])))
        terms.append(Term('YY', bnd, a, b, float(prob.Jy[bnd])))
        terms.append(Term('ZZ', bnd, a, b, float(prob.Jz[bnd])))
    return terms


def gammas(theta: float, delta: float) -> tuple[float, float, float]:
    """PAI coefficients gamma_1, gamma_2, gamma_3 at |theta| (Eq. gammas)."""
    t = abs(theta)
    g1 = math.cos(t / 2) * math.sin(delta / 2 - t / 2) / math.sin(delta / 2)
    g2 = math.sin(t) / math.sin(delta)
    g3 = -math.sin(t / 2) * math.sin(delta / 2 - t / 2) / math.cos(delta / 2)
    return g1, g2, g3


def threshold_u64(p: float) -> int:
    """floor(p * 2^64), saturated to [0, 2^64 - 1]: a draw x (uniform u64) picks
    the event when x < threshold, so P = threshold / 2^64."""
    if not p > 0.0:
        return 0
    v = math.ldexp(p, 64)
    if v >= 2.0 ** 64:
        return (1 << 64) - 1
    return int(math.floor(v))


@dataclasses.dataclass
class Plan:
    terms: list
    theta: np.ndarray          # theta_k = 2 c_k T / N (App. A.3)
    gam: np.ndarray            # (L, 3) gamma_l(|theta_k|)
    gnorm_gate: np.ndarray     # ||gamma(|theta_k|)||_1
    q: np.ndarray              # probability that gate (j,k) is not A
    r: np.ndarray              # probability of C given not A
    thr_event: list            # floor(q * 2^64)
    thr_c: list                # floor(r * 2^64)
    phi: np.ndarray            # angle of the applied rotation for setting B
    gnorm_step: float          # prod_k ||gamma_k||_1 for one Trotter step
    variant: int
    n_steps: int
    delta: float
    lam: np.ndarray = None     # CONTINUOUS: event rate of term k per unit time
    r_inf: float = 0.0         # CONTINUOUS: probability that an event is C
    T: float = 0.0             # total time of the product formula


def make_plan(prob, T: float, n_steps: int, delta: float, variant: int = UNBIASED) -> Plan:
    terms = term_list(prob)
    L = len(terms)
    theta = np.array([2.0 * t.c * T / n_steps for t in terms])
    gam = np.zeros((L, 3))
    q = np.zeros(L)
    r = np.zeros(L)
    gn = np.zeros(L)
    phi = np.zeros(L)
    lam = np.zeros(L)
    r_inf = 0.0
    if variant == CONTINUOUS:
        # N -> infinity limit of the PAI draws (App. A.3 Eq. gammas at small
        # theta): per unit time, term k leaves A with rate
        # |c_k| (3 - cos Delta) / sin Delta (whose sum times T is nu_inf of
        # App. A.5), and a non-A event is C with probability
        # |gamma_3| / (|gamma_2| + |gamma_3|) -> (1 - cos Delta) / (3 - cos Delta).
        rate = (3.0 - math.cos(delta)) / math.sin(delta)
        r_inf = (1.0 - math.cos(delta)) / (3.0 - math.cos(delta))
        for k, t in enumerate(terms):
            lam[k] = abs(t.c) * rate
            phi[k] = math.copysign(delta, t.c) if t.c != 0.0 else delta
        return Plan(terms=terms, theta=theta, gam=gam, gnorm_gate=np.ones(L), q=q, r=np.full(L, r_inf),
                    thr_event=[0] * L, thr_c=[threshold_u64(r_inf)] * L, phi=phi, gnorm_step=1.0,
                    variant=variant, n_steps=n_steps, delta=delta, lam=lam, r_inf=r_inf, T=T)
    for k, th in enumerate(theta):
        if variant == TROTTER:
            # deterministic product formula: every gate is R_k(theta_k)
            gam[k] = (0.0, 1.0, 0.0)
            q[k], r[k], gn[k], phi[k] = 1.0, 0.0, 1.0, th
            continue
        if variant == NO_PI:
            # App. A.4: gamma~_1 = 1 - lambda, gamma~_2 = lambda, lambda = |theta|/Delta
            frac = abs(th) / delta
            gam[k] = (1.0 - frac, frac, 0.0)
        else:
            gam[k] = gammas(th, delta)
        a = np.abs(gam[k])
        gn[k] = a[0] + a[1] + a[2]
        nonid = a[1] + a[2]
        q[k] = nonid / gn[k]
        r[k] = a[2] / nonid if nonid > 0 else 0.0
        # setting B = R_k(sign(theta) Delta) (Eq. settings)
        phi[k] = math.copysign(delta, th) if th != 0.0 else delta
    gstep = 1.0
    for k in range(L):
        gstep *= gn[k]
    return Plan(terms=terms, theta=theta, gam=gam, gnorm_gate=gn, q=q, r=r,
                thr_event=[threshold_u64(x) for x in q],
                thr_c=[threshold_u64(x) for x in r],
                phi=phi, gnorm_step=gstep, variant=variant,
                n_steps=n_steps, delta=delta, lam=lam, r_inf=r_inf, T=T)


def check_theta(plan: Plan) -> bool:
    """The PAI decomposition assumes |theta_kj| <= Delta <= pi (App. A.3)."""
    if plan.variant in (TROTTER, CONTINUOUS):
        return True
    return bool(np.all(np.abs(plan.theta) <= plan.delta) and plan.delta <= math.pi)


def snapshot_steps(run_steps: int, M: int) -> list[int]:
    """Snapshot m = 1..M is taken after step j_m = m * run_steps / M."""
    return [m * run_steps // M for m in range(1, M + 1)]


def snapshot_times(plan: Plan, run_steps: int, M: int) -> np.ndarray:
    """CONTINUOUS: snapshot m = 1..M at time t_m = (T run_steps / N) m / M,
    evaluated as t_run * m / M."""
    t_run = plan.T * run_steps / plan.n_steps
    return np.array([t_run * m / M for m in range(1, M + 1)])


def gnorm_time(plan: Plan, t: float) -> float:
    """CONTINUOUS: ||g(t)||_1 = exp[2 tan(Delta/2) ||c||_1 t] (Eq. overhead)."""
    c1 = sum(abs(tm.c) for tm in plan.terms)
    return math.exp(2.0 * math.tan(plan.delta / 2) * c1 * t)


def gnorm_at(plan: Plan, j: int) -> float:
    """||g(t_j)||_1 = prod over the first j steps of prod_k ||gamma_k||_1
    (Eq. overhead-bound, time-independent case)."""
    return plan.gnorm_step ** j


def expected_nu(plan: Plan, run_steps: int) -> float:
    """E[nu] for finite N: every gate (j,k) is non-identity with prob. q_k."""
    return run_steps * float(np.sum(plan.q))


def nu_infinity(prob, T: float, delta: float) -> float:
    """nu_inf = csc(Delta) (3 - cos Delta) ||c||_1 T (Eq. ap:eq_nu_infty)."""
    c1 = sum(abs(t.c) for t in term_list(prob))
    return (3.0 - math.cos(delta)) / math.sin(delta) * c1 * T


def gnorm_infinity(prob, T: float, delta: float) -> float:
    """||g||_1^inf = exp[2 tan(Delta/2) ||c||_1 T] (Eq. overhead)."""
    c1 = sum(abs(t.c) for t in term_list(prob))
    return math.exp(2.0 * math.tan(delta / 2) * c1 * T)
