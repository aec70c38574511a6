"""Noise-parallel replicas: one process per GPU, each on its own noise indices.

Noise vectors are independent units and the Philox stream is keyed by the
noise index, so splitting the indices among ranks gives exactly the samples a
single process would draw.  The only exchange is the merge of per-level
sufficient statistics (count, sums of the real and imaginary parts and of
their squares), done once per estimate; there is no collective on the data
path.
"""
import numpy as np


def noise_first(step, rank, world, n):
    """First noise index of rank `rank` at `step` for a level of n noises per rank."""
    return (int(step) * int(world) + int(rank)) * int(n)


def local_moments(samples):
    """(n, sum re, sum im, sum re^2, sum im^2) of complex samples, FP64."""
    x = np.asarray(samples, dtype=np.complex128)
    return np.array([x.size, x.real.sum(), x.imag.sum(), (x.real ** 2).sum(), (x.imag ** 2).sum()])


def stats_from_moments(m):
    n, sr, si, qr, qi = (float(v) for v in m)
    mean = complex(sr / n, si / n)
    var_re = (qr - n * mean.real ** 2) / (n - 1) if n > 1 else 0.0
    var_im = (qi - n * mean.imag ** 2) / (n - 1) if n > 1 else 0.0
    return {"n": int(n), "mean": mean, "var_re": var_re, "var_im": var_im,
            "stderr_re": float(np.sqrt(max(var_re, 0.0) / n)), "stderr_im": float(np.sqrt(max(var_im, 0.0) / n))}


def merge_level(samples, group=None):
    """All-reduce the moments of this rank's samples (torch.distributed, any backend)."""
    import torch
    import torch.distributed as dist
    m = torch.tensor(local_moments(samples), dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        backend = dist.get_backend(group)
        if backend == "nccl":
            m = m.cuda()
        dist.all_reduce(m, op=dist.ReduceOp.SUM, group=group)
    return stats_from_moments(m.cpu().numpy())
