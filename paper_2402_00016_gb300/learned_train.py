"""Training set and training of the learned subtraction operator / preconditioner at
scale, through the library's public calls (the paper has no learned part; the
network approximates M^-1 of Sec. 1 and stays linear in its input).

make_pairs: (eta, M^-1 eta) pairs from the method's own deflated, refined solves
(mmc_solve, Sec. 8) on Z(4) noise, in batches, gathered into two FP32 fields of
n_pairs vectors (the layout mmc_net_train reads).
train: mmc_net_train over those pairs, optionally with BF16 weights and hidden
activations (mmc_net_set_precision).

python -m paper_2402_00016_gb300.learned_train --dims 16 16 16 16 --pairs 4096
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_pairs(mmc, ctx, n_pairs, batch=256, level=31, rel_tol=1e-8, precond=None, m_inner=16):
    """Two FP32 fields (eta, x) of n_pairs vectors with M x = eta to rel_tol; batch must be a
    multiple of 16 dividing n_pairs.  Returns (eta, x, matvec-free stats dict)."""
    if n_pairs % batch or batch % 16:
        raise ValueError("batch must be a multiple of 16 dividing n_pairs")
    pre = mmc.MMC_ZERO if precond is None else precond
    eta = mmc.new_field(ctx, n_pairs, mmc.MMC_F32)
    xs = mmc.new_field(ctx, n_pairs, mmc.MMC_F32)
    b = mmc.new_field(ctx, batch, mmc.MMC_F64)
    x = mmc.new_field(ctx, batch, mmc.MMC_F64)
    step = mmc.mmc_field_bytes(ctx, batch, mmc.MMC_F32)  # batch is whole rhs blocks: contiguous
    its_total, t0 = 0, time.time()
    for k in range(n_pairs // batch):
        mmc.mmc_noise(ctx, level, k * batch, mmc.MMC_TAG_NOISE, batch, mmc.MMC_F64, b)
        x.zero_()
        its, rel = mmc.mmc_solve(ctx, b, x, batch, rel_tol, pre, mmc.MMC_F32, m_inner, 400)
        its_total += its
        mmc.mmc_convert(ctx, b, mmc.MMC_F64, eta.data_ptr() + k * step, mmc.MMC_F32, batch)
        mmc.mmc_convert(ctx, x, mmc.MMC_F64, xs.data_ptr() + k * step, mmc.MMC_F32, batch)
    return eta, xs, {"seconds": time.time() - t0, "inner_iterations": its_total}


def train(mmc, ctx, eta, xs, n_pairs, iters=1500, batch=32, lr=2e-3, seed=7, bf16=True):
    """A network trained on the pairs; returns (handle, loss history)."""
    h = mmc.mmc_net_create(ctx, None, seed)
    if bf16:
        mmc.mmc_net_set_precision(ctx, h, mmc.MMC_BF16)
    hist = mmc.mmc_net_train(ctx, h, eta, xs, n_pairs, batch, iters, lr)
    return h, hist


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 16])
    ap.add_argument("--eps", type=float, default=0.25)
    ap.add_argument("--kappa", type=float, default=0.1565)
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--iters", type=int, default=1500)
    ap.add_argument("--fp32", action="store_true", help="FP32 network instead of BF16")
    a = ap.parse_args(argv)
    import synth
    from paper_2402_00016_gb300 import build
    build.build()
    from paper_2402_00016_gb300 import mmc
    ctx = mmc.mmc_create(a.dims, seed=5, device=0)
    try:
        mmc.mmc_load_gauge(ctx, synth.random_gauge(a.dims, a.eps, 2), a.kappa, 1)
        hp, _ = mmc.mmc_gmres_poly(ctx, 40)
        lam = mmc.mmc_deflate(ctx, 40, hp, 200, 1e-3)
        eta, xs, st = make_pairs(mmc, ctx, a.pairs, precond=hp)
        h, hist = train(mmc, ctx, eta, xs, a.pairs, iters=a.iters, bf16=not a.fp32)
        print(json.dumps({"dims": a.dims, "pairs": a.pairs, "deflated": len(lam), "solves": st,
                          "loss_first": float(np.mean(hist[:10])), "loss_last": float(np.mean(hist[-10:])),
                          "weights": None}), flush=True)
    finally:
        mmc.mmc_destroy(ctx)


if __name__ == "__main__":
    main()
