"""Benchmark: 24^4 multipolynomial Monte Carlo noise samples per second.

Workload (the batched 24^4 form): synthetic gauge field U = exp(i eps H),
eps 0.25, kappa 0.1565, antiperiodic time; levels
  Tr(M^-1 - p_dbl)     8 noises   (p_dbl: 40 inner x 8 outer, degree 319)
  Tr(p_dbl - p_128)   32 noises   deflated
  Tr(p_128 - p_32)   128 noises   deflated
  Tr(p_32 - p_8)     512 noises   deflated
  Tr(p_8)            exact, by probing (setup)
A step is one pass over all four Monte Carlo levels: 680 Z(4) samples with
fresh noise indices, FP32 spinor storage (BF16 with --storage bf16) and FP32
arithmetic, FP64 bilinear accumulation, refined FP64 solves.  The polynomials, the deflation
eigenpairs and the exact last level are set up once before timing (reported
as setup_s).  value = samples / device time (CUDA events over the timed
steps); e2e = the same through the public API with the gauge configuration
uploaded from pinned host memory and the samples read back every step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mmc|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "24^4 noise samples/s at fixed trace error vs plain FP64; Dslash HBM GB/s"
WORKLOAD = "c4_24x24x24x24"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def time_to_error(var, seconds, noises, eps):
    """Seconds for the multilevel estimate to reach standard error eps, from one measured step
    (level l: sample variance var[l], seconds[l] for its noises[l] samples).  Returned: the
    time at the step's noise proportions, (sum_l seconds_l) (sum_l var_l / N_l) / eps^2 (both
    factors scale inversely under a common change of every N_l), and the time with the counts
    re-allocated cost-optimally (N_l proportional to sqrt(var_l / c_l), c_l = seconds_l / N_l,
    the cost function Sec. 9 names), (sum_l sqrt(var_l c_l))^2 / eps^2."""
    var_over_n = sum(v / n for v, n in zip(var, noises))
    fixed = sum(seconds) * var_over_n / eps ** 2
    sv = sum(np.sqrt(max(v, 0.0) * t / n) for v, t, n in zip(var, seconds, noises))
    return fixed, sv ** 2 / eps ** 2


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, n in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def level_plan(h, top_deflated=False):
    """(hi, lo, deflate, n_noise, level id) of the four Monte Carlo levels; the top level
    M^-1 - p_dbl is deflated with the deflated double polynomial."""
    from paper_2402_00016_gb300 import mmc
    return [(mmc.MMC_INV, h["dbl"], 1 if top_deflated else 0, 8, 1), (h["dbl"], h["p128"], 1, 32, 2),
            (h["p128"], h["p32"], 1, 128, 3), (h["p32"], h["p8"], 1, 512, 4)]


# matvecs per sample of the polynomial parts of each level (the M^-1 level's solves come on top)
POLY_MATVECS_BY_LEVEL = [319, 319 + 128, 128 + 32, 32 + 8]
NOISES = [8, 32, 128, 512]
SAMPLES = sum(NOISES)
LEVELS = ["M^-1 - p_dbl(40x8)", "p_dbl - p_128", "p_128 - p_32", "p_32 - p_8"]
# Matvecs per sample of each level as the library's estimator spends them on this workload
# (its own counters, mmc_level_stats.matvecs / noises, of an earlier run of this command: the
# M^-1 level's refined, deflated, polynomial-preconditioned solves included).  The CPU legs
# charge the oracle the same work per sample, so they time the same algorithm.
MATVECS_PER_SAMPLE = [28328 / 8, 14304 / 32, 20480 / 128, 20480 / 512]
# DRAM traffic of the dominant step-kernel class, per site and right-hand side, from one ncu
# capture per kernel form (dram__bytes_read.sum + dram__bytes_write.sum of a 64-rhs degree-8
# level chain with the code bilinear at 24^4, the launch scaled to 512 rhs by site-rhs count):
# keyed by the kernel form; a form without a capture reports null.
TRAFFIC_PER_SITE_RHS = {
    # (kernel version, register cap, traversal, class kind, storage precision): bytes per site and rhs
    (2, 4, 1, "bilinear", 1): (4.671779e9 + 2.024867e9) / (331776 * 64),  # 315.4 B
    (4, 3, 2, "bilinear", 1): (3.220147e9 + 2.017138e9) / (331776 * 64),  # 246.6 B
    # the other fourth-form variants (register cap 3..6, traversal 0..2), one capture of the
    # eight launches of the timed level of each (their median)
    (4, 3, 0, "bilinear", 1): (4.801522e9 + 2.017512e9) / (331776 * 64),  # 321.1 B
    (4, 3, 1, "bilinear", 1): (4.842631e9 + 2.013644e9) / (331776 * 64),  # 322.9 B
    (4, 4, 0, "bilinear", 1): (4.308748e9 + 2.018456e9) / (331776 * 64),  # 298.0 B
    (4, 4, 1, "bilinear", 1): (4.840953e9 + 2.013706e9) / (331776 * 64),  # 322.8 B
    (4, 4, 2, "bilinear", 1): (3.468966e9 + 2.014524e9) / (331776 * 64),  # 258.2 B
    (4, 5, 0, "bilinear", 1): (4.598836e9 + 2.021913e9) / (331776 * 64),  # 311.8 B, links staged in shared memory
    (4, 5, 1, "bilinear", 1): (4.829387e9 + 2.018181e9) / (331776 * 64),  # 322.5 B, links staged in shared memory
    (4, 5, 2, "bilinear", 1): (3.576689e9 + 2.017936e9) / (331776 * 64),  # 263.5 B, links staged in shared memory
    (4, 6, 0, "bilinear", 1): (4.484482e9 + 2.016758e9) / (331776 * 64),  # 306.2 B, third link rows rebuilt
    (4, 6, 1, "bilinear", 1): (4.827532e9 + 2.014122e9) / (331776 * 64),  # 322.2 B, third link rows rebuilt
    (4, 6, 2, "bilinear", 1): (3.473146e9 + 2.012985e9) / (331776 * 64),  # 258.4 B, third link rows rebuilt
    # the Horner chains of the 8-rhs solves (one launch of the kernel_bench solve mode; minb 3
    # in the blocked layout, minb 6 in the paired-component layout the solves use by default)
    (4, 3, 0, "aux", 1): (669.179392e6 + 238.431744e6) / (331776 * 8),  # 341.9 B
    (4, 6, 0, "aux", 1): (664.114688e6 + 238.064128e6) / (331776 * 8),  # 339.9 B, third link rows rebuilt
}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_slice(U, kappa, dims, reps, first=0):
    """Time the oracle on a bounded slice: `reps` degree-2 polynomial samples
    eta^H p(M) eta at 24^4 (2 matvecs each).  Returns (seconds, matvecs)."""
    from oracle import krylov, noise, wilson
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    op = lambda v: wilson.apply_M(U, kappa, v.reshape(shape)).ravel()
    theta = np.array([1.1 + 0.2j, 0.9 - 0.1j, 1.3 + 0.0j])
    t0 = time.time()
    for r in range(reps):
        eta = noise.z4_noise(dims, 3, first + r, 4).ravel()
        np.vdot(eta, krylov.apply_poly(op, theta, eta))
    return time.time() - t0, 2 * reps


def _oracle_worker(args):
    """One process of the all-core leg: build the gauge field, then time `reps` samples."""
    reps, first = args
    import synth
    W = synth.WORKLOADS[WORKLOAD]
    U = synth.random_gauge(W.dims, W.eps, W.gauge_seed)
    return oracle_slice(U, W.kappa, W.dims, reps, first)


def cpu_oracle(reps_one, all_cores=True):
    """The oracle as it stands, on the host cores: one process (numpy single-threaded), then
    one process per core at once (spawned, one degree-2 sample each).  Seconds per oracle
    matvec of each leg, the per-level per-noise times they give with the library's matvecs
    per sample, and samples/s for the workload's noise mix."""
    import multiprocessing as mp
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"  # every oracle process single-threaded
    ctx = mp.get_context("spawn")  # never fork a process that holds a CUDA context
    with ctx.Pool(1) as pool:
        dt, mv = pool.map(_oracle_worker, [(reps_one, 0)])[0]
    legs = {"1": {"cores": 1, "s_per_matvec": dt / mv, "sample": "%d degree-2 samples (%d matvecs) in %.1f s"
                  % (reps_one, mv, dt)}}
    ncores = os.cpu_count() or 1
    if all_cores and ncores > 1:
        t0 = time.time()
        with ctx.Pool(ncores) as pool:
            res = pool.map(_oracle_worker, [(1, 100 + i) for i in range(ncores)])
        wall = time.time() - t0
        span = max(r[0] for r in res)
        mvs = sum(r[1] for r in res)
        legs["all"] = {"cores": ncores, "s_per_matvec": span / mvs,
                       "sample": "%d processes x 1 degree-2 sample (%d matvecs in all), slowest %.1f s "
                                 "(%.1f s with gauge generation)" % (ncores, mvs, span, wall)}
    for leg in legs.values():
        per_noise = [m * leg["s_per_matvec"] for m in MATVECS_PER_SAMPLE]
        leg["seconds_per_noise_by_level"] = per_noise
        leg["value"] = SAMPLES / sum(n * t for n, t in zip(NOISES, per_noise))
    return legs


def run_reference(args, rank):
    if rank != 0:
        return
    import synth
    W = synth.WORKLOADS[WORKLOAD]
    U = synth.random_gauge(W.dims, W.eps, W.gauge_seed)
    for _ in range(args.warmup):
        oracle_slice(U, W.kappa, W.dims, 1)
    t, mv = 0.0, 0
    for it in range(args.steps):
        dt, m = oracle_slice(U, W.kappa, W.dims, 1, first=it)
        t += dt
        mv += m
    per_noise = [m * t / mv for m in MATVECS_PER_SAMPLE]
    value = SAMPLES / sum(n * x for n, x in zip(NOISES, per_noise))
    line = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattice": "24^4", "eps": W.eps, "kappa": W.kappa,
                       "levels": LEVELS, "noises": NOISES, "storage": "f64 (oracle)",
                       "parallelism": "1 host core"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "samples/s", "cores": 1,
                             "cpu": cpu_model(),
                             "seconds_per_noise_by_level": per_noise,
                             "sample": "per step: one degree-2 polynomial sample (2 oracle matvecs) at 24^4; "
                                       "samples/s = the workload's noise mix at the library's matvecs per "
                                       "sample of each level (solves included) times the oracle's measured "
                                       "seconds per matvec"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mmc")
    ap.add_argument("--deflate-k", type=int, default=100)
    ap.add_argument("--arnoldi", type=int, default=200)
    ap.add_argument("--solve-m", type=int, default=8, help="inner FGMRES length of the M^-1 level solves")
    ap.add_argument("--precond", default="in", choices=["in", "dbl"],
                    help="right preconditioner of those solves: the inner GMRES polynomial (degree 39) or the "
                         "double polynomial (degree 319)")
    ap.add_argument("--horner-layout", default="paired", choices=["blocked", "paired"],
                    help="layout of the Horner preconditioner chains in the 8-rhs solves (paired: two "
                         "components of an rhs per 16-byte access, converted in and out per application)")
    ap.add_argument("--solve-storage", default="f32", choices=["f32", "bf16"],
                    help="storage of the inner FGMRES stage and its preconditioner chain in those solves (the "
                         "FP64 outer loop refines to 1e-10 either way)")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16"],
                    help="spinor storage of the polynomial chains (BF16 rounding shifts the level samples by "
                         "several standard errors on this workload: see error_vs_fp64)")
    ap.add_argument("--outer-m", type=int, default=8, help="outer GMRES length of the double polynomial")
    ap.add_argument("--dbl-deflated", action="store_true",
                    help="deflated double polynomial (outer cycle from the deflated start vector) and a deflated "
                         "top level")
    ap.add_argument("--rounding", default="nearest", choices=["nearest", "stochastic"],
                    help="rounding of BF16 chain storage (stochastic keeps the BF16 levels unbiased)")
    ap.add_argument("--learned", action="store_true",
                    help="the learned form: a BF16 network trained on 16^4 solve pairs as the M^-1 level's "
                         "preconditioner and as an extra level p_8 - N with Tr(N) exact")
    ap.add_argument("--separate", dest="merged", action="store_false",
                    help="run every polynomial level as its own chain (default: the polynomial levels in one "
                         "batch, one launch per degree over all their chains)")
    ap.add_argument("--learned-pairs", type=int, default=4096)
    ap.add_argument("--learned-iters", type=int, default=1500)
    ap.add_argument("--cpu-reps", type=int, default=4, help="degree-2 oracle samples of the one-core leg")
    ap.add_argument("--plain-samples", type=int, default=4,
                    help="FP64 single-vector samples per level for the plain form")
    ap.add_argument("--tune-file", default=None,
                    help="autotuner cache: load the kernel variants from this JSON file if it exists, else tune "
                         "and write it (a profiling run then reuses the plain run's choices)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import torch.distributed as dist
    import synth
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc, replicas

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    W = synth.WORKLOADS[WORKLOAD]
    storage = mmc.PREC[args.storage]
    t_setup = time.time()
    U = synth.random_gauge(W.dims, W.eps, W.gauge_seed)
    ctx = mmc.mmc_create(W.dims, seed=W.noise_seed, device=local)
    mmc.mmc_profile(ctx, 1)  # counts every library launch from here on (launch index of the timed region)
    mmc.mmc_load_gauge(ctx, U, W.kappa, W.t_antiperiodic)
    h = {}
    h["in"], _ = mmc.mmc_gmres_poly(ctx, 40)
    if not args.dbl_deflated:
        h["out"], _ = mmc.mmc_gmres_poly(ctx, args.outer_m, h["in"])
        h["dbl"] = mmc.mmc_poly_double(ctx, h["in"], h["out"])
    h["p128"], _ = mmc.mmc_gmres_poly(ctx, 129)
    h["p32"], _ = mmc.mmc_gmres_poly(ctx, 33)
    h["p8"], _ = mmc.mmc_gmres_poly(ctx, 9)
    if args.tune_file and (args.tune_file.lstrip().startswith("{") or os.path.exists(args.tune_file)):
        if args.tune_file.lstrip().startswith("{"):  # the choice given inline
            tune = json.loads(args.tune_file)
        else:
            with open(args.tune_file) as f:
                tune = json.load(f)
        for key, t in tune.items():
            prec = mmc.PREC[key.split("_")[0]]
            mmc.mmc_set_step_variant_class(ctx, prec, 1 if key.endswith("_512rhs") else 0, t)
    else:
        # one variant per storage precision and rhs-block class: the 512-noise batch of the
        # cheapest level (16-rhs blocks, every polynomial level) and the 8-rhs solves
        tune = {}
        for name in ("f32", "bf16"):
            tune[name + "_512rhs"] = mmc.mmc_autotune(ctx, 512, mmc.PREC[name])
            tune[name + "_8rhs"] = mmc.mmc_autotune(ctx, 8, mmc.PREC[name])
        if args.tune_file:
            with open(args.tune_file, "w") as f:
                json.dump(tune, f)
    mmc.mmc_set_rounding(ctx, mmc.MMC_ROUND_STOCHASTIC if args.rounding == "stochastic" else mmc.MMC_ROUND_NEAREST,
                         seed=W.noise_seed)
    mmc.mmc_set_solve_params(ctx, args.solve_m, 400)
    mmc.mmc_set_solve_storage(ctx, mmc.PREC[args.solve_storage])
    mmc.mmc_set_horner_layout(ctx, 1 if args.horner_layout == "paired" else 0)
    t_poly = time.time() - t_setup
    lam = mmc.mmc_deflate(ctx, args.deflate_k, h["in"], args.arnoldi, 1e-3) if args.deflate_k > 0 else []
    if args.dbl_deflated:
        # the deflated double polynomial: p_out from the start vector without the deflated
        # eigenvector components; the top level is then deflated too
        h["out"], _ = mmc.mmc_gmres_poly_deflated(ctx, args.outer_m, h["in"])
        h["dbl"] = mmc.mmc_poly_double(ctx, h["in"], h["out"])
    pre = h[args.precond]
    pre_plain = pre  # the plain FP64 form keeps the polynomial preconditioner
    t_defl = time.time() - t_setup - t_poly
    learned_info = None
    if args.learned:
        # the learned form: a network trained on (eta, M^-1 eta) pairs from 16^4 solves of
        # fields drawn with this workload's eps and kappa (BF16 weights and activations),
        # as the right preconditioner of the M^-1 level's solves and as the operand of an
        # extra Monte Carlo level p_8 - N whose exact last level Tr(N) replaces Tr(p_8)
        from paper_2402_00016_gb300 import learned_train
        t0 = time.time()
        dims16 = (16, 16, 16, 16)
        c16 = mmc.mmc_create(dims16, seed=W.noise_seed + 100, device=local)
        try:
            mmc.mmc_load_gauge(c16, synth.random_gauge(dims16, W.eps, W.gauge_seed + 1), W.kappa, 1)
            hp16, _ = mmc.mmc_gmres_poly(c16, 40)
            lam16 = mmc.mmc_deflate(c16, 40, hp16, 200, 1e-3)
            eta16, xs16, solves = learned_train.make_pairs(mmc, c16, args.learned_pairs, precond=hp16)
            hn16, hist = learned_train.train(mmc, c16, eta16, xs16, args.learned_pairs, iters=args.learned_iters)
            weights = mmc.mmc_net_get_weights(c16, hn16)
            del eta16, xs16
            torch.cuda.empty_cache()  # the 4096 training pairs (51 GB): back to the device, not torch's cache
        finally:
            mmc.mmc_destroy(c16)
        h["net"] = mmc.mmc_net_create(ctx, weights)
        mmc.mmc_net_set_precision(ctx, h["net"], mmc.MMC_BF16)
        pre = h["net"]
        learned_info = {"train_pairs": args.learned_pairs, "train_lattice": "16^4", "deflated_16": len(lam16),
                        "pair_solves": solves, "iters": args.learned_iters, "loss_first": float(np.mean(hist[:10])),
                        "loss_last": float(np.mean(hist[-10:])), "seconds": time.time() - t0,
                        "storage": "bf16 weights and activations, fp32 accumulation"}
        exact = mmc.mmc_trace_exact(ctx, h["net"], mmc.MMC_THETA_ONE, mmc.MMC_EXACT_PROBE, mmc.MMC_F32)
        ncol = mmc.mmc_probe_colours(ctx, 3)
    else:
        exact = mmc.mmc_trace_exact(ctx, h["p8"], mmc.MMC_THETA_ONE, mmc.MMC_EXACT_PROBE, mmc.MMC_F64)
        ncol = mmc.mmc_probe_colours(ctx, 8)
    t_setup = time.time() - t_setup
    plan = level_plan(h, args.dbl_deflated)
    if args.learned:
        plan.append((h["p8"], h["net"], 0, 512, 5))
    samples_per_step = sum(n for (_, _, _, n, _) in plan)

    nets = {h["net"]} if args.learned else set()

    def batchable(hi, lo):
        return hi != mmc.MMC_INV and hi not in nets and lo not in nets

    def step(it):
        out = [None] * len(plan)
        if args.merged:
            # the polynomial levels in one batch per deflation flag (one launch per degree
            # over all their chains), the solve and network levels on their own
            for defl in (0, 1):
                idx = [i for i, (hi, lo, d, _, _) in enumerate(plan) if d == defl and batchable(hi, lo)]
                if not idx:
                    continue
                res = mmc.mmc_trace_levels(ctx, [plan[i][0] for i in idx], [plan[i][1] for i in idx],
                                           mmc.MMC_THETA_ONE, defl, [plan[i][3] for i in idx],
                                           [replicas.noise_first(it, rank, world, plan[i][3]) for i in idx],
                                           [plan[i][4] for i in idx], storage)
                for i, r in zip(idx, res):
                    out[i] = r
        for i, (hi, lo, defl, n, lvl) in enumerate(plan):
            if out[i] is None:
                first = replicas.noise_first(it, rank, world, n)
                out[i] = mmc.mmc_trace_level(ctx, hi, lo, mmc.MMC_THETA_ONE, defl, n, first, lvl, storage,
                                             pre, want_samples=True)
        return out

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    for it in range(args.warmup):
        step(10_000 + it)
    barrier()
    launches_before = mmc.mmc_profile_read(ctx)["all_launches"]
    mmc.mmc_profile(ctx, 1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        results = [step(it) for it in range(args.steps)]
        ev1.record()
        barrier()
    ms = ev0.elapsed_time(ev1)
    prof = mmc.mmc_profile_read(ctx)
    classes = mmc.mmc_profile_classes(ctx)
    mmc.mmc_profile(ctx, 0)
    ms_max = ms
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    samples = samples_per_step * args.steps * world
    value = samples / (ms_max / 1e3)

    # end to end: gauge configuration from pinned host memory every step, samples read back
    Ut = torch.from_numpy(np.ascontiguousarray(U)).pin_memory()
    Upin = Ut.numpy()
    barrier()
    t0 = time.time()
    for it in range(args.steps):
        mmc.mmc_update_gauge(ctx, Upin)
        res = step(1000 + it)
        _ = [r["samples"].copy() for r in res]
    barrier()
    e2e_s = time.time() - t0
    e2e_val = samples / e2e_s if world == 1 else samples_per_step * args.steps / e2e_s * world

    # statistics of the last timed step (trace error of the estimator), merged over replicas
    last = results[-1]
    merged = [replicas.merge_level(r["samples"]) for r in last]
    est = exact.real + sum(m["mean"].real + r["corr_re"] for m, r in zip(merged, last))
    stderr = float(np.sqrt(sum(m["var_re"] / m["n"] for m in merged)))

    # The plain FP64 single-vector form on the same GPU: same polynomials, deflation and
    # preconditioner, FP64 storage and arithmetic (FP64 solves), one noise vector per call.
    # Bounded: args.plain_samples samples per level (fresh noise indices), their mean time
    # extrapolated to the 8/32/128/512 mix; the spread is reported.
    plain = None
    if rank == 0:
        per_sample, spread = [], []
        for (hi, lo, defl, n, lvl) in plan:
            ts = []
            for q in range(args.plain_samples):
                torch.cuda.synchronize()
                t0 = time.time()
                mmc.mmc_trace_level(ctx, hi, lo, mmc.MMC_THETA_ONE, defl, 1, 900_000 + q, lvl, mmc.MMC_F64,
                                    pre_plain, want_samples=False)
                torch.cuda.synchronize()
                ts.append(time.time() - t0)
            per_sample.append(float(np.mean(ts)))
            spread.append([float(np.min(ts)), float(np.max(ts))])
        t_step = sum(n * t for (_, _, _, n, _), t in zip(plan, per_sample))
        plain = {"value": samples_per_step / t_step, "unit": "samples/s", "seconds_per_sample_by_level": per_sample,
                 "min_max_seconds_by_level": spread,
                 "sample": "%d FP64 single-vector samples per level (host wall time each), their mean "
                           "extrapolated to the 8/32/128/512 mix" % args.plain_samples,
                 "speedup_of_value": value / (samples_per_step / t_step)}

    # Error of the reduced-precision form against the FP64 form (which the parity tests pin
    # to the oracle): the same noises through both, per level; bias in units of the level's
    # standard error for its configured noise count.
    err_vs_fp64 = None
    if rank == 0:
        err_vs_fp64 = []
        for (hi, lo, defl, n, lvl), r in zip(plan, last):
            q = 1 if hi == mmc.MMC_INV else min(n, 4)  # the FP64 solves are the costly part
            a = mmc.mmc_trace_level(ctx, hi, lo, mmc.MMC_THETA_ONE, defl, q, 800_000, lvl, storage, pre)
            b = mmc.mmc_trace_level(ctx, hi, lo, mmc.MMC_THETA_ONE, defl, q, 800_000, lvl, mmc.MMC_F64, pre_plain)
            d = a["samples"] - b["samples"]
            se = float(np.sqrt(r["var_re"] / n)) if r["var_re"] > 0 else float("nan")
            err_vs_fp64.append({"noises": q, "max_abs_sample_diff": float(np.abs(d).max()),
                                "mean_diff_re": float(d.real.mean()),
                                "mean_diff_over_stderr": float(d.real.mean() / se) if se == se else None,
                                "correction_diff": a["corr_re"] - b["corr_re"]})

    # CPU baseline: the oracle on bounded slices of the same workload (rank 0 only), on one
    # host core and on all of them
    cpu = None
    if rank == 0 and world == 1:
        legs = cpu_oracle(args.cpu_reps, all_cores=True)
        best = legs.get("all", legs["1"])
        cpu = {"value": best["value"], "unit": "samples/s", "cores": best["cores"], "kind": "oracle",
               "cpu": cpu_model(), "legs": legs,
               "sample": "oracle seconds per matvec at 24^4 from degree-2 polynomial samples (%s); samples/s = "
                         "the 8/32/128/512 noise mix at the library's matvecs per sample of each level, the "
                         "M^-1 level's solves included" % best["sample"]}

    # Roofline of the dominant step-kernel class (the launch class with the most device time in
    # the timed steps): its algorithmic bytes (mmc_profile_classes: every operand element once,
    # links once per launch, nothing for the noise codes) over its CUDA-event time.
    peak, peak_kind = measured_peaks()
    dom = max(classes, key=lambda c: c["ms"]) if classes else None
    if dom and dom["ms"] > 0:
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        # site-rhs per launch, averaged over the class's launches (a merged chain's launches
        # shrink as its shorter polynomials finish): 1368 + 48 flops per site-rhs of a hop step
        units = dom["flops"] / max(1, dom["launches"]) / (1368.0 + 48.0)
        rc = 1 if dom["nrhs_padded"] >= 16 else 0
        tkey = "%s_%s" % (("f64", "f32", "bf16")[dom["prec"]], "512rhs" if rc else "8rhs")
        form = tune.get(tkey, {}) if isinstance(tune, dict) else {}
        tps = TRAFFIC_PER_SITE_RHS.get((form.get("version"), form.get("minb"), form.get("blocked"), dom["kind"],
                                        dom["prec"]))
        traffic = tps * units if tps else None
    else:
        achieved, traffic, units, form = 0.0, None, 0, {}
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": "24^4", "eps": W.eps, "kappa": W.kappa,
                   "levels": LEVELS + (["p_8 - N (learned)"] if args.learned else []), "double": {"m_in": 40, "m_out": args.outer_m, "deflated": args.dbl_deflated},
                   "noises": [n for (_, _, _, n, _) in plan], "storage": args.storage, "rounding": args.rounding, "arithmetic": "fp32, fp64 bilinears",
                   "deflated": len(lam), "probe_colours": ncol,
                   "batch": "polynomial levels merged (one launch per degree)" if args.merged else "per level",
                   "solves": {"fgmres_m": args.solve_m, "precond": "p_in (degree 39)" if args.precond == "in"
                              else "p_dbl (degree 319)", "tol": 1e-10, "inner_storage": args.solve_storage,
                              "horner_layout": args.horner_layout}, "l2": "inputs larger than L2 (GB-sized fields)",
                   "parallelism": "replicas" if world > 1 else "1 gpu"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_basis": ("DRAM bytes read and written per launch of this class's kernel form, "
                                       "from one ncu capture of the same form (a 64-rhs level chain, or an "
                                       "8-rhs Horner chain), scaled by site-rhs to this launch" if traffic else
                                       "no DRAM counters were taken for this kernel form"),
                     "kernel": "step kernel (fused Wilson stencil + Leja step + epilogue), class %s, %s storage, "
                               "%d rhs per launch" % (dom["kind"], ("f64", "f32", "bf16")[dom["prec"]],
                                                      dom["nrhs_padded"]) if dom else None,
                     "form": form,
                     "algorithmic_bytes_per_launch": dom["bytes"] / max(1, dom["launches"]) if dom else None,
                     "site_rhs_per_launch": units,
                     "peak_kind": peak_kind, "launches": dom["launches"] if dom else 0,
                     "avg_launch_ms": dom["ms"] / max(1, dom["launches"]) if dom else None,
                     "share_of_step": dom["ms"] / ms if (dom and ms > 0) else None,
                     "tflops": dom["flops"] / (dom["ms"] / 1e3) / 1e12 if (dom and dom["ms"]) else 0,
                     "all_step_launches": {"launches": prof["step_launches"], "ms": prof["step_ms"],
                                           "achieved_GBps": prof["step_bytes"] / (prof["step_ms"] / 1e3) / 1e9
                                           if prof["step_ms"] else 0.0,
                                           "share_of_step": prof["step_ms"] / ms if ms > 0 else None},
                     "classes": classes},
        "gpu_launches": prof["all_launches"],
        "graphs": {"chain_graph_replays": prof["graph_launches"], "note": mmc.mmc_graph_note(ctx)},
        "launch_index_timed_start": launches_before,
        "e2e": {"value": e2e_val, "unit": "samples/s",
                "h2d_bytes_per_step": int(U.nbytes),
                "d2h_bytes_per_step": int(samples_per_step * 16)},
        "clocks": clk.summary(),
        "setup_s": {"total": t_setup, "polynomials_and_tuning": t_poly, "deflation": t_defl},
        "learned": learned_info,
        "autotune": tune,
        "estimate": {"trace_re": est, "stderr": stderr, "exact_last_level": exact.real,
                     "per_level_var": [r["var_re"] for r in last],
                     "per_level_seconds": [r["seconds"] for r in last],
                     "per_level_matvecs": [r["matvecs"] for r in last]},
    }
    # time to a target error eps at the step's noise proportions and with the counts
    # re-allocated cost-optimally; the plain FP64 form shares the variances (same estimator)
    eps_target = 0.0005 * float(np.prod(W.dims))
    noises = [n for (_, _, _, n, _) in plan]
    var_over_n = sum(r["var_re"] / n for r, n in zip(last, noises))
    t_opt = sum(r["seconds"] for r in last)
    line["estimate"]["time_x_var"] = t_opt * var_over_n
    line["estimate"]["eps_target"] = eps_target
    (line["estimate"]["seconds_to_eps"],
     line["estimate"]["seconds_to_eps_cost_optimal"]) = time_to_error([r["var_re"] for r in last],
                                                                      [r["seconds"] for r in last], noises,
                                                                      eps_target)
    if plain:
        t_plain = sum(n * t for (_, _, _, n, _), t in zip(plan, plain["seconds_per_sample_by_level"]))
        plain["time_x_var"] = t_plain * var_over_n
        plain["seconds_to_eps"] = t_plain * var_over_n / eps_target ** 2
        plain["speedup_at_equal_error"] = t_plain / t_opt
    if cpu:
        line["cpu_baseline"] = cpu
    if plain:
        line["plain_fp64_single_vector"] = plain
    if err_vs_fp64:
        line["error_vs_fp64"] = err_vs_fp64
    if rank == 0:
        print(json.dumps(line), flush=True)
    mmc.mmc_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
