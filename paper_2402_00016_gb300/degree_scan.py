"""Relative variance of polynomial subtraction against the polynomial degree (Sec. 4,
Eq. 3, Eq. 4, Fig. 1), through the library's public calls.

For each gauge configuration (seed) and degree d the subtraction level
Tr(Theta (M^-1 - p_d(M))) is sampled with the same Z(4) noise vectors as the
unsubtracted estimator Tr(Theta M^-1) ("no subtraction", NS):

    x_NS(eta)  = eta^H Theta M^-1 eta          (refined solves, mmc_trace_level(MMC_INV, MMC_ZERO))
    x_d(eta)   = x_NS(eta) - eta^H Theta p_d(M) eta    (mmc_trace_level(p_d, MMC_ZERO))

p_d the GMRES polynomial of degree d (Sec. 3, GMRES(d + 1)).  Per configuration the
variances sigma^2_A (of x_d) and sigma^2_NS (of x_NS) are the unbiased sample
variances of the real part; over configurations the relative variance (Eq. 3) is
mean(sigma^2_A) / mean(sigma^2_NS) and the log-averaged one (Eq. 4) is
10^(mean log10 sigma^2_A - mean log10 sigma^2_NS).

The paper measures this on quenched beta = 6.0 configurations at kappa = 0.1570,
which are not available here; the synthetic fields U = exp(i eps H) at the
near-critical kappa of the workloads stand in for them.

python -m paper_2402_00016_gb300.degree_scan --dims 8 8 8 8 --seeds 1 2 3 4 5 --degrees 5 10 20 50 100 200
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def config_variances(mmc, ctx, degrees, n_noise, level=7, theta_op=0, roots=None, precond_m=16):
    """Sample variances (real part) of the NS estimator and of each degree's subtraction
    level on one configuration loaded in ctx; also returns the samples.  ``roots``:
    optional {degree: Leja-ordered roots} to use instead of the library's GMRES cycle."""
    handles = {}
    for d in degrees:
        if roots is not None:
            handles[d] = mmc.mmc_poly_from_roots(ctx, roots[d])
        else:
            handles[d], _ = mmc.mmc_gmres_poly(ctx, d + 1)
    pre, _ = mmc.mmc_gmres_poly(ctx, precond_m)
    ns = mmc.mmc_trace_level(ctx, mmc.MMC_INV, mmc.MMC_ZERO, theta_op, 0, n_noise, 0, level, mmc.MMC_F64,
                             precond=pre)
    out = {"ns": {"var": ns["var_re"], "samples": ns["samples"]}, "levels": {}}
    for d in degrees:
        st = mmc.mmc_trace_level(ctx, handles[d], mmc.MMC_ZERO, theta_op, 0, n_noise, 0, level, mmc.MMC_F64)
        x = ns["samples"] - st["samples"]
        out["levels"][d] = {"var": float(np.var(x.real, ddof=1)), "samples": x}
    return out


def relative_variances(per_config, degrees):
    """Eq. 3 and Eq. 4 over configurations for every degree."""
    vns = np.array([c["ns"]["var"] for c in per_config])
    res = {}
    for d in degrees:
        va = np.array([c["levels"][d]["var"] for c in per_config])
        res[d] = {"relative": float(va.mean() / vns.mean()),
                  "log_averaged": float(10.0 ** (np.mean(np.log10(va)) - np.mean(np.log10(vns))))}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[8, 8, 8, 8])
    ap.add_argument("--eps", type=float, default=0.3)
    ap.add_argument("--kappa", type=float, default=0.155)
    ap.add_argument("--seeds", type=int, nargs="+", default=[1, 2, 3, 4, 5])
    ap.add_argument("--degrees", type=int, nargs="+", default=[5, 10, 20, 50, 100, 200])
    ap.add_argument("--noises", type=int, default=32)
    a = ap.parse_args(argv)
    import synth
    from paper_2402_00016_gb300 import build
    build.build()
    from paper_2402_00016_gb300 import mmc
    per_config = []
    for seed in a.seeds:
        ctx = mmc.mmc_create(a.dims, seed=seed, device=0)
        try:
            mmc.mmc_load_gauge(ctx, synth.random_gauge(a.dims, a.eps, seed), a.kappa, 1)
            per_config.append(config_variances(mmc, ctx, a.degrees, a.noises))
        finally:
            mmc.mmc_destroy(ctx)
    rv = relative_variances(per_config, a.degrees)
    print(json.dumps({"dims": a.dims, "eps": a.eps, "kappa": a.kappa, "seeds": a.seeds, "noises": a.noises,
                      "ns_var": [c["ns"]["var"] for c in per_config],
                      "relative_variance": {str(d): rv[d] for d in a.degrees}}), flush=True)


if __name__ == "__main__":
    main()
