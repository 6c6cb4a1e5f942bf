"""Multi-process sharding of the ensemble on CPU (gloo, world size 2): the
per-rank partials merged over torch.distributed equal the single-process
estimate over all samples."""
import os
import socket

import numpy as np
import pytest

from oracle import estimator
from paper_2604_13144_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _data(ns=101, M=3, nobs=5):
    rng = np.random.default_rng(11)
    v = rng.uniform(-1, 1, (ns, M, nobs))
    sg = rng.choice([-1, 1], (ns, M)).astype(np.int8)
    g = np.array([1.0, 1.3, 1.7])
    return v, sg, g


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    v, sg, g = _data()
    off, cnt = shard.shard_range(v.shape[0], rank, world)
    _, _, part = estimator.estimate(v[off:off + cnt], sg[off:off + cnt], g)
    mean, se = shard.allgather_merge(part, cnt, g, dist)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.stack([mean, se]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_ranges_partition_the_samples():
    for n in (1, 7, 100, 101):
        for w in (1, 2, 3, 8):
            rs = [shard.shard_range(n, r, w, offset=5) for r in range(w)]
            assert rs[0][0] == 5 and sum(c for _, c in rs) == n
            for (o1, c1), (o2, _) in zip(rs, rs[1:]):
                assert o1 + c1 == o2


def test_gloo_two_ranks_merge_equals_single_process(tmp_path):
    torch_mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    torch_mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    v, sg, g = _data()
    mean, se, _ = estimator.estimate(v, sg, g)
    for r in range(2):
        got = np.load(tmp_path / f"r{r}.npy")
        assert np.allclose(got[0], mean, rtol=0, atol=1e-15)
        assert np.allclose(got[1], se, rtol=1e-12, atol=1e-15)


def _oracle_worker(rank, world, port, out_dir):
    """Each rank runs the oracle on its own range of global sample indices of
    the N -> infinity sampler and the ranks merge their partials."""
    import math
    import torch.distributed as dist
    import workloads as W
    from oracle import run as orun
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prob = W.spin_ring(4, 1.0, seed=1)
    ns = 9
    off, cnt = shard.shard_range(ns, rank, world, offset=100)
    par = W.Params(T=0.5, n_steps=10, delta=math.pi / 8, n_samples=cnt, chi_max=4, cutoff=0.0,
                   n_snapshots=2, seed=4, sample_offset=off, variant=3)
    r = orun.run(prob, par, use_statevector=True)
    mean, se = shard.allgather_merge(r["partials"], cnt, r["gnorm"], dist)
    np.save(os.path.join(out_dir, f"c{rank}.npy"), np.stack([mean, se]))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_sharded_continuous_sampler_equals_single_process(tmp_path):
    """Circuits are keyed by the global sample index, so two ranks running
    disjoint index ranges reproduce the single-process N -> infinity estimate."""
    import math
    import workloads as W
    from oracle import run as orun
    torch_mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    torch_mp.spawn(_oracle_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    prob = W.spin_ring(4, 1.0, seed=1)
    par = W.Params(T=0.5, n_steps=10, delta=math.pi / 8, n_samples=9, chi_max=4, cutoff=0.0,
                   n_snapshots=2, seed=4, sample_offset=100, variant=3)
    ref = orun.run(prob, par, use_statevector=True)
    for r in range(2):
        got = np.load(tmp_path / f"c{r}.npy")
        assert np.allclose(got[0], ref["mean"], rtol=0, atol=1e-14)
        assert np.allclose(got[1], ref["stderr"], rtol=1e-12, atol=1e-14)
