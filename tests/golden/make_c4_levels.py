"""Write tests/golden/c4_24x24x24x24_levels.json: expected level samples of the
24^4 near-critical workload (eps 0.25, kappa 0.1565, antiperiodic time), computed
by the oracle alone (FP64 numpy, oracle/ and synth/ only).

Contents:
* the Leja-ordered GMRES roots (Sec. 3) of the workload's polynomials from the
  Z(4) start vector (noise index 0, level 0, tag 'GMRS'): p_8, p_32, p_128 (m = 9,
  33, 129) and the double polynomial 40 inner x 8 outer (Sec. 5);
* for a few noise indices of three Monte Carlo levels (Eq. 2, Sec. 6) the samples
  eta_j^H (p_hi(M) - p_lo(M)) eta_j and the Cauchy-Schwarz scales
  ||eta_j|| (||p_hi(M) eta_j|| + ||p_lo(M) eta_j||) that bound a normwise error;
* M eta_j and p_hi(M) eta_j element statistics for element-wise checks are not
  stored (the vectors are 4M entries); the GPU tests check those at sampled sites.

Run once on a CPU (about 35 minutes on 8 cores):
    python tests/golden/make_c4_levels.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_24x24x24x24_levels.json")
WORKLOAD = "c4_24x24x24x24"
# (level id, hi, lo, noise count of the level, sampled noise indices)
LEVELS = [(4, "p32", "p8", 512, (0, 300, 511)),
          (3, "p128", "p32", 128, (0, 127)),
          (2, "dbl", "p128", 32, (0, 31))]


def _setup():
    import synth
    from oracle import wilson
    W = synth.WORKLOADS[WORKLOAD]
    U = synth.random_gauge(W.dims, W.eps, W.gauge_seed)
    shape = (W.dims[3], W.dims[2], W.dims[1], W.dims[0], 4, 3)
    op = lambda v: wilson.apply_M(U, W.kappa, v.reshape(shape), bool(W.t_antiperiodic)).ravel()
    return W, op


def _roots(job):
    from oracle import krylov, noise
    W, op = _setup()
    b = noise.z4_noise(W.dims, W.noise_seed, 0, 0, noise.TAG_GMRES).ravel()
    if job == "dbl":
        tin, tout = krylov.double_poly_roots(op, b, 40, 8)
        return {"in": tin, "out": tout}
    m = {"p8": 9, "p32": 33, "p128": 129}[job]
    return {job: krylov.gmres_poly_roots(op, b, m)}


def _sample(args):
    level, hi, lo, j, roots = args
    from oracle import krylov, noise
    W, op = _setup()
    eta = noise.z4_noise(W.dims, W.noise_seed, j, level).ravel()

    def apply(name, v):
        if name == "dbl":
            return krylov.apply_double(op, roots["in"], roots["out"], v)
        return krylov.apply_poly(op, roots[name], v)

    ph = apply(hi, eta)
    pl = apply(lo, eta)
    x = np.vdot(eta, ph - pl)
    ne = np.linalg.norm(eta)
    return {"level": level, "j": j, "sample": [x.real, x.imag],
            "hi_bilinear": [np.vdot(eta, ph).real, np.vdot(eta, ph).imag],
            "scale": ne * (np.linalg.norm(ph) + np.linalg.norm(pl))}


def main():
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(4) as pool:
        parts = pool.map(_roots, ["dbl", "p128", "p32", "p8"])
    roots = {}
    for p in parts:
        roots.update(p)
    print("roots %.0f s" % (time.time() - t0), flush=True)
    jobs = [(lvl, hi, lo, j, roots) for (lvl, hi, lo, n, js) in LEVELS for j in js]
    with ctx.Pool(min(8, len(jobs))) as pool:
        samples = pool.map(_sample, jobs)
    print("samples %.0f s" % (time.time() - t0), flush=True)
    cx = lambda a: [[float(z.real), float(z.imag)] for z in a]
    out = {"workload": WORKLOAD,
           "source": "oracle (FP64 numpy): krylov.gmres_poly_roots, krylov.double_poly_roots, krylov.apply_poly, "
                     "krylov.apply_double on synth.random_gauge and noise.z4_noise",
           "roots": {k: cx(v) for k, v in roots.items()},
           "levels": [{"level": lvl, "hi": hi, "lo": lo, "n_noise": n, "samples": [s for s in samples
                                                                                  if s["level"] == lvl]}
                      for (lvl, hi, lo, n, js) in LEVELS]}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT, flush=True)


if __name__ == "__main__":
    main()
