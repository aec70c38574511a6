"""Throughput of the fused step kernel on one configuration (a small driver for
profilers and for tuning): a polynomial level chain eta^H Theta p(M) eta on a
synthetic field, timed with CUDA events.

python -m paper_2402_00016_gb300.kernel_bench --dims 16 16 16 16 --nrhs 128 --prec bf16 --degree 8 --reps 3
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 16])
    ap.add_argument("--nrhs", type=int, default=128)
    ap.add_argument("--prec", default="bf16", choices=["f64", "f32", "bf16"])
    ap.add_argument("--degree", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--rpt", type=int, default=0)
    ap.add_argument("--minb", type=int, default=0)
    ap.add_argument("--spc", type=int, default=0)
    ap.add_argument("--blocked", type=int, default=-1, help="1: 4D-blocked site traversal, 0: lexicographic")
    ap.add_argument("--ns", type=int, default=-1, help="ring slots of the staged kernel (0: as many as fit)")
    ap.add_argument("--autotune", action="store_true", help="pick the kernel variant with mmc_autotune first")
    ap.add_argument("--graphs", type=int, default=1, help="replay step chains as CUDA graphs")
    ap.add_argument("--rmax", type=int, default=16, help="largest rhs block of the field layout (8 or 16)")
    ap.add_argument("--version", type=int, default=0, help="step-kernel version (0: keep the default)")
    ap.add_argument("--hint", type=int, default=-1, help="store hint of version 4 (1: L2 evict-first)")
    ap.add_argument("--horner-layout", type=int, default=0,
                    help="--solve: 1 runs the Horner chains in the paired-component layout")
    ap.add_argument("--sweep", default=None,
                    help="JSON list of variants {version, rpt, minb, spc, blocked, hint}: time each in turn")
    ap.add_argument("--solve", type=int, default=0,
                    help="m > 0: time nrhs refined solves (FGMRES(8)) right-preconditioned by a degree m-1 "
                         "polynomial in Horner form (the step chains of the M^-1 level) instead of a level chain")
    ap.add_argument("--apply", action="store_true",
                    help="time p(M) X as a vector (the accumulating chain, mmc_apply_poly) instead of a level "
                         "chain's bilinear")
    ap.add_argument("--solve-outer", type=int, default=2,
                    help="FP64 refinement cycles of each timed solve (the launches are timed whether or not "
                         "the solve converges in them)")
    ap.add_argument("--deflate", type=int, default=0,
                    help="k > 0: random deflation space of k vectors, levels deflated (tensor-core projections)")
    a = ap.parse_args(argv)
    import torch
    import synth
    from paper_2402_00016_gb300 import build
    build.build()
    from paper_2402_00016_gb300 import mmc
    prec = mmc.PREC[a.prec]
    ctx = mmc.mmc_create(a.dims, seed=3, device=0)
    try:
        mmc.mmc_set_rhs_block_max(ctx, a.rmax)
        mmc.mmc_load_gauge(ctx, synth.random_gauge(a.dims, 0.25, 1), 0.1565, 1)
        mmc.mmc_set_step_variant(ctx, prec, a.rpt, a.minb, a.spc)
        mmc.mmc_set_graphs(ctx, a.graphs)
        if a.blocked >= 0:
            mmc.mmc_set_step_variant(ctx, prec, 0, 200 + a.blocked, 0)
        if a.ns >= 0:
            mmc.mmc_set_step_variant(ctx, prec, 0, 300 + a.ns, 0)
        if a.version > 0:
            mmc.mmc_set_step_variant(ctx, prec, 0, 100 + a.version, 0)
        if a.hint >= 0:
            mmc.mmc_set_step_variant(ctx, prec, 0, 400 + a.hint, 0)
        mmc.mmc_set_horner_layout(ctx, a.horner_layout)
        tuned = mmc.mmc_autotune(ctx, a.nrhs, prec) if a.autotune else None
        if a.deflate > 0:
            vol12 = 12 * int(np.prod(a.dims))
            rng = np.random.default_rng(5)
            Z = rng.standard_normal((a.deflate, vol12)) + 1j * rng.standard_normal((a.deflate, vol12))
            Z /= np.linalg.norm(Z, axis=1, keepdims=True)
            lam = 0.2 + 0.1j * np.arange(a.deflate)
            mmc.mmc_set_deflation(ctx, lam, Z, Z.copy())
        # fixed Leja-ordered roots on a circle around 1 (no setup kernels before the chain)
        m = a.degree + 1
        theta = mmc.mmc_leja_order(1.0 + 0.8 * np.exp(2j * np.pi * (np.arange(m) + 0.5) / m))
        h = mmc.mmc_poly_from_roots(ctx, theta)
        h2 = mmc.mmc_poly_from_roots(ctx, theta[:2]) if a.deflate > 0 else mmc.MMC_ZERO
        defl = 1 if a.deflate > 0 else 0
        if a.solve > 0:
            hp = mmc.mmc_poly_from_roots(ctx, mmc.mmc_leja_order(
                1.0 + 0.8 * np.exp(2j * np.pi * (np.arange(a.solve) + 0.5) / a.solve)))
            b = mmc.new_field(ctx, a.nrhs, mmc.MMC_F64)
            x = mmc.new_field(ctx, a.nrhs, mmc.MMC_F64)
            mmc.mmc_noise(ctx, 2, 0, mmc.MMC_TAG_NOISE, a.nrhs, mmc.MMC_F64, b)
            for rep in range(a.reps + 1):  # the first is the warm-up
                if rep == 1:
                    mmc.mmc_profile(ctx, 1)
                x.zero_()
                try:
                    its, rel = mmc.mmc_solve(ctx, b, x, a.nrhs, 1e-8, hp, prec, 8, a.solve_outer)
                    converged = True
                except mmc.MMCError as e:
                    if e.code != mmc.MMC_ERR_NOCONV:
                        raise
                    its, converged = None, False
            p = mmc.mmc_profile_read(ctx)
            print(json.dumps({"dims": a.dims, "nrhs": a.nrhs, "prec": a.prec, "solve_degree": a.solve - 1,
                              "iterations": its, "converged": converged, "step_launches": p["step_launches"],
                              "classes": mmc.mmc_profile_classes(ctx)}), flush=True)
            return
        variants = json.loads(a.sweep) if a.sweep else [None]
        vol = int(np.prod(a.dims))
        for var in variants:
            if var is not None:
                v = {"version": 2, "rpt": 1, "minb": 4, "spc": 64, "blocked": 0, "ns": 0}
                v.update(var)
                for rc in (0, 1):
                    mmc.mmc_set_step_variant_class(ctx, prec, rc, v)
                mmc.mmc_set_step_variant(ctx, prec, 0, 400 + int(var.get("hint", 0)), 0)
            if a.apply:
                xa = mmc.new_field(ctx, a.nrhs, prec)
                ya = mmc.new_field(ctx, a.nrhs, prec)
                mmc.mmc_noise(ctx, 1, 0, mmc.MMC_TAG_NOISE, a.nrhs, prec, xa)

            def one(r):
                if a.apply:
                    mmc.mmc_apply_poly(ctx, h, xa, ya, a.nrhs, prec)
                else:
                    mmc.mmc_trace_level(ctx, h, h2, 0, defl, a.nrhs, a.nrhs * r, 1, prec)

            one(0)  # warm-up
            mmc.mmc_profile(ctx, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for r in range(a.reps):
                one(r + 1)
            e1.record()
            torch.cuda.synchronize()
            p = mmc.mmc_profile_read(ctx)
            out = {"dims": a.dims, "nrhs": a.nrhs, "prec": a.prec, "degree": a.degree, "apply": a.apply,
                   "graphs": a.graphs, "rmax": a.rmax,
                   "step_launches": p["step_launches"], "avg_launch_ms": p["step_ms"] / max(1, p["step_launches"]),
                   "algorithmic_GBps": p["step_bytes"] / p["step_ms"] / 1e6 if p["step_ms"] else 0,
                   "TFLOPs": p["step_flops"] / p["step_ms"] / 1e9 if p["step_ms"] else 0,
                   "ps_per_site_rhs": 1e9 * p["step_ms"] / max(1, p["step_launches"]) / (vol * a.nrhs),
                   "wall_ms": e0.elapsed_time(e1), "variant": var if var is not None else tuned}
            print(json.dumps(out), flush=True)
    finally:
        mmc.mmc_destroy(ctx)


if __name__ == "__main__":
    main()
