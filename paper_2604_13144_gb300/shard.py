"""Sample sharding across processes (one per GPU) and the one exchange step.

Samples are independent: rank r of W evolves the contiguous global range
[offset + r * per_rank, ...), which fixes its circuits through the Philox key.
The only exchange is the merge of each rank's per-(snapshot, observable)
partials (Neumaier sum, compensation, sum of squares) into the ensemble mean
and standard error of Sec. II.B / Statement 2. Partials are merged in rank
order with compensated summation, so the result does not depend on the order in
which ranks finish.
"""
from __future__ import annotations

import math

import numpy as np


def shard_range(n_total: int, rank: int, world: int, offset: int = 0) -> tuple[int, int]:
    """(sample_offset, n_samples) of `rank`: contiguous, sizes differ by <= 1."""
    base, rem = divmod(n_total, world)
    start = rank * base + min(rank, rem)
    count = base + (1 if rank < rem else 0)
    return offset + start, count


def _two_sum(a: float, b: float) -> tuple[float, float]:
    s = a + b
    bp = s - a
    return s, (a - (s - bp)) + (b - bp)


def merge_partials(partials: list[np.ndarray], counts: list[int], gnorm: np.ndarray):
    """partials[r]: (M, n_obs, 3) = (sum, compensation, sum of squares) of
    sign * v over rank r's samples; counts[r]: its sample count. Returns
    (mean, stderr) with mean = ||g(t_m)||_1 * sum / N_s."""
    M, nobs, _ = partials[0].shape
    ns = int(sum(counts))
    mean = np.zeros((M, nobs))
    se = np.zeros((M, nobs))
    for m in range(M):
        for o in range(nobs):
            s, c, q = 0.0, 0.0, 0.0
            for p in partials:
                s, e1 = _two_sum(s, float(p[m, o, 0]))
                c += e1 + float(p[m, o, 1])
                q += float(p[m, o, 2])
            mu = (s + c) / ns
            mean[m, o] = gnorm[m] * mu
            if ns > 1:
                var = max(0.0, (q - ns * mu * mu) / (ns - 1))
                se[m, o] = gnorm[m] * math.sqrt(var / ns)
    return mean, se


def allgather_merge(local_partials: np.ndarray, local_count: int, gnorm: np.ndarray, dist):
    """Gather every rank's partials over torch.distributed (any backend) and
    merge them in rank order on every rank."""
    import torch
    world = dist.get_world_size()
    t = torch.from_numpy(np.ascontiguousarray(local_partials, dtype=np.float64)).reshape(-1)
    c = torch.tensor([float(local_count)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t, c = t.cuda(), c.cuda()
    ts = [torch.zeros_like(t) for _ in range(world)]
    cs = [torch.zeros_like(c) for _ in range(world)]
    dist.all_gather(ts, t)
    dist.all_gather(cs, c)
    parts = [x.cpu().numpy().reshape(local_partials.shape) for x in ts]
    counts = [int(x.item()) for x in cs]
    return merge_partials(parts, counts, gnorm)
