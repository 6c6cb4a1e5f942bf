"""One TE-PAI ensemble run composed from the oracle's parts.

For global samples s = offset .. offset + Ns - 1:
  1. the sampler draws the events of sample s (Sec. II.B step 2);
  2. the MPS (or the state vector, for tiny rings) applies them in gate order
     and records <Z_i> after each snapshot step j_m (Sec. II.A);
  3. sign(g_l) at j_m = (-1)^{#C events up to j_m} (App. B).
Then the estimator forms ||g(t_m)||_1 * mean_s(sign * v) (Sec. II.B).
"""
from __future__ import annotations

import numpy as np

from . import estimator, planner, sampler
from . import mps as mps_mod
from . import statevector as sv


def run(prob, par, init_tensors=None, use_statevector: bool = False,
        floor_rel: float = 1e-14, gap_rel: float = mps_mod.PAPER_TIE_REL, samples=None,
        regauge: bool = False, three_site: bool = False):
    """Return dict with v (Ns, M, n_obs), sign (Ns, M), gnorm (M,), mean,
    stderr, partials, events_total, per-sample MPS statistics and each
    sample's final MPS (site tensors in chain order; MPS runs only)."""
    plan = planner.make_plan(prob, par.T, par.n_steps, par.delta, par.variant)
    S = par.steps_run()
    cont = par.variant == planner.CONTINUOUS
    if cont:
        # snapshots are times; event rows carry their snapshot index m = 1..M
        t_snaps = planner.snapshot_times(plan, S, par.n_snapshots)
        snaps = list(range(1, par.n_snapshots + 1))
    else:
        snaps = planner.snapshot_steps(S, par.n_snapshots)
    strings = getattr(par, "obs_strings", None)
    if strings is not None:
        strings = np.asarray(strings, dtype=np.int64).reshape(-1, prob.n)
    obs = (np.arange(prob.n) if strings is None and par.obs_sites is None
           else np.arange(len(strings)) if strings is not None
           else np.asarray(par.obs_sites, dtype=np.int64))
    idx = (range(par.sample_offset, par.sample_offset + par.n_samples)
           if samples is None else samples)
    vs, signs, nus, stats, states = [], [], [], [], []
    for s in idx:
        ev = (sampler.sample_events_continuous(plan, par.seed, s, t_snaps)[0] if cont
              else sampler.sample_events(plan, par.seed, s, S))
        nus.append(len(ev))
        if use_statevector:
            z = sv.run_events(prob.init_bits, plan, ev, snaps, strings)
            stats.append({})
        else:
            m = (mps_mod.product_state(prob.init_bits, prob.periodic) if init_tensors is None
                 else mps_mod.canonicalize(init_tensors, prob.periodic))
            z = mps_mod.run_events(m, plan, ev, snaps, par.chi_max, par.cutoff, floor_rel, gap_rel,
                                   regauge, strings, three_site)
            stats.append(m.stats)
            states.append([a.copy() for a in m.A])
        vs.append(z[:, obs])
        signs.append([sampler.sign_after(ev, j) for j in snaps])
    v = np.array(vs)
    sg = np.array(signs, dtype=np.int8)
    gn = (np.array([planner.gnorm_time(plan, t) for t in t_snaps]) if cont
          else np.array([planner.gnorm_at(plan, j) for j in snaps]))
    mean, se, part = estimator.estimate(v, sg, gn)
    return {"v": v, "sign": sg, "gnorm": gn, "mean": mean, "stderr": se,
            "partials": part, "nu": np.array(nus), "stats": stats, "plan": plan,
            "snaps": snaps, "states": states,
            "times": (t_snaps if cont else np.array([par.T * j / par.n_steps for j in snaps]))}
