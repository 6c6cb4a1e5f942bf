"""Truncation-rule settings under which the oracle takes the same keep
decisions as one precision mode of the CUDA path: that precision's
singular-value floor (values at or below floor_rel * s_0 are zero to working
precision: 1e-14 in FP64, 4e-6 with FP32 tensors) and the run's tie band
(tie_rel, or the paper's rule, where only equal values are tied, when it is 0)."""
from oracle import mps

FLOOR = {0: 1e-14, 1: 4e-6}


def oracle_rule(par) -> dict:
    tie = float(getattr(par, "tie_rel", 0.0) or 0.0)
    return {"floor_rel": FLOOR[int(par.precision)], "gap_rel": tie if tie > 0 else mps.PAPER_TIE_REL}
