"""Noise-parallel replicas on CPU (gloo, world size 2): disjoint noise slices
and merged level statistics equal to one process over the union of samples.
Samples come from the oracle on a tiny lattice, so no GPU is involved."""
import os

import numpy as np
import pytest

from paper_2402_00016_gb300 import replicas


def _samples(indices):
    import synth
    from oracle import krylov, noise, wilson
    dims, shape = (2, 2, 2, 4), (4, 2, 2, 2, 4, 3)
    U = synth.random_gauge(dims, 0.5, 1)
    op = lambda v: wilson.apply_M(U, 0.12, v.reshape(shape)).ravel()
    theta = np.array([1.1 + 0.1j, 0.8 - 0.2j, 1.4 + 0.0j])
    out = []
    for j in indices:
        e = noise.z4_noise(dims, 9, j, 2).ravel()
        out.append(np.vdot(e, krylov.apply_poly(op, theta, e)))
    return np.array(out)


def _worker(rank, world, port, n, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = [replicas.noise_first(s, rank, world, n) + k for s in range(steps) for k in range(n)]
    st = replicas.merge_level(_samples(idx))
    q.put((rank, idx, st))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_process():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    n, steps, world = 3, 2, 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda t: t[0])
    idx0, idx1 = set(res[0][1]), set(res[1][1])
    assert not (idx0 & idx1)
    union = sorted(idx0 | idx1)
    assert union == list(range(world * n * steps))
    ref = replicas.stats_from_moments(replicas.local_moments(_samples(union)))
    for _, _, st in res:
        assert st["n"] == ref["n"]
        assert abs(st["mean"] - ref["mean"]) < 1e-12 * abs(ref["mean"])
        assert abs(st["var_re"] - ref["var_re"]) < 1e-9 * max(1.0, abs(ref["var_re"]))
        x = _samples(union)
        assert abs(ref["var_re"] - np.var(x.real, ddof=1)) < 1e-9 * max(1.0, np.var(x.real))
