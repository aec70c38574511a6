"""Trace estimators: Hutchinson with subtraction (Sec. 1-2), multipolynomial
levels (Sec. 6), level deflation with its exact correction (Sec. 7), exact
traces of low-degree polynomials (Sec. 6, probing) and statistics (Sec. 4,
Sec. 8).

A level is a pair (hi, lo) of linear maps on flat vectors; its sample for
noise eta is x = eta^H Theta (A_hi - A_lo) eta.  With deflation data
(lambda, Z, U) and scalar functions c(lambda) = p_hi(lambda) - p_lo(lambda),
x -= sum_i c_i (eta^H Theta z_i)(u_i^H eta) and the level value is
mean(x) + sum_i c_i u_i^H Theta z_i (the trace of the deflated part).

Reading taken for "variance" and "standard error" (Sec. 4, Sec. 8): the
unbiased sample variance of the real part for a Hermitian-like insertion
(Theta = 1) and of the imaginary part for Theta = gamma_4, standard error
s / sqrt(N); the complex variance mean |x - mean|^2 is reported too.
"""
import numpy as np


def level_samples(hi, lo, theta_apply, etas, defl=None, c=None):
    """Samples x_n = eta_n^H Theta (hi - lo) eta_n (Eq. 2, Sec. 6), optionally deflated (Sec. 7).

    ``hi``, ``lo``: maps on flat vectors (lo may be None for zero);
    ``theta_apply``: the site-local insertion Theta on flat vectors;
    ``etas``: list of flat noise vectors; ``defl`` = (Z, U); ``c`` = c_i.
    Returns (samples, correction).
    """
    xs = []
    for eta in etas:
        v = hi(eta)
        if lo is not None:
            v = v - lo(eta)
        x = np.vdot(eta, theta_apply(v))
        if defl is not None and c is not None and len(c):
            Z, U = defl
            a = np.array([np.vdot(eta, theta_apply(Z[:, i])) for i in range(Z.shape[1])])
            bb = U.conj().T @ eta
            x = x - np.sum(c * a * bb)
        xs.append(x)
    corr = 0.0 + 0.0j
    if defl is not None and c is not None and len(c):
        Z, U = defl
        corr = sum(c[i] * np.vdot(U[:, i], theta_apply(Z[:, i])) for i in range(Z.shape[1]))
    return np.array(xs, dtype=np.complex128), corr


def stats(samples, part="re"):
    """Mean, unbiased sample variance of the chosen part, standard error, complex variance."""
    x = np.asarray(samples, dtype=np.complex128)
    n = x.size
    mean = x.mean()
    comp = x.real if part == "re" else x.imag
    var = comp.var(ddof=1) if n > 1 else 0.0
    cvar = np.sum(np.abs(x - mean) ** 2) / (n - 1) if n > 1 else 0.0
    return {"n": n, "mean": mean, "var": var, "stderr": np.sqrt(var / n) if n else 0.0,
            "cvar": cvar}


def exact_trace_unit(apply_map, theta_apply, n, batch=256):
    """Tr(Theta A) = sum_j e_j^H Theta A e_j over all n unit vectors (Sec. 6, last level).

    ``apply_map`` maps an n x B block of columns to A times it."""
    total = 0.0 + 0.0j
    for s in range(0, n, batch):
        cols = np.arange(s, min(n, s + batch))
        E = np.zeros((n, cols.size), dtype=np.complex128)
        E[cols, np.arange(cols.size)] = 1.0
        Y = theta_apply(apply_map(E))
        total += np.sum(Y[cols, np.arange(cols.size)])
    return total


def exact_trace_probing(apply_map, theta_apply, colour, n_colours, n_site_dofs=12):
    """Tr(Theta A) by probing (Sec. 6): probe vectors e_{c,a} = sum_{x: colour(x)=c} e_{x,a}.

    Exact when A couples no two distinct sites of equal colour.  ``colour`` is
    an integer array over sites (canonical site order); dofs are 12 per site.
    """
    vol = colour.size
    n = vol * n_site_dofs
    total = 0.0 + 0.0j
    for c in range(n_colours):
        sites = np.nonzero(colour == c)[0]
        E = np.zeros((n, n_site_dofs), dtype=np.complex128)
        for a in range(n_site_dofs):
            E[sites * n_site_dofs + a, a] = 1.0
        Y = theta_apply(apply_map(E))
        total += np.sum(np.conj(E) * Y)
    return total


def log_averaged_relative_variance(var_method, var_ns):
    """10^(mean log10 var_A - mean log10 var_NS) over configurations (Sec. 4, Eq. 4)."""
    return 10.0 ** (np.mean(np.log10(var_method)) - np.mean(np.log10(var_ns)))


def relative_variance(var_method, var_ns):
    """Ratio of configuration-averaged variances (Sec. 4, Eq. 3)."""
    return np.mean(var_method) / np.mean(var_ns)


# ------------------------------------------------------------ noise counts
# Sec. 8 checks each level's standard error after a first batch of noises and
# then after every further few; the paper states the total target
# eps = 0.0005 V but not how it is split between levels.  Reading taken: with
# L Monte Carlo levels each level stops at the first check where its standard
# error is at most eps / sqrt(L), so the levels' errors combined in quadrature
# meet eps.  Sec. 9 names cost-optimal allocation (Giles) as future work; it is
# the alternative rule below.

def equal_split_counts(streams, eps, n_first, n_check, n_max, part="re"):
    """Noises used per level under the check-every-few stopping rule.

    ``streams[l]``: that level's samples in noise order (at least n_max[l] of
    them, or as many as the rule can use); ``n_first``, ``n_check``, ``n_max``:
    per-level lists.  Level l stops at the first n in n_first, n_first +
    n_check, ... (capped at n_max) where stderr(streams[l][:n]) <= eps/sqrt(L).
    """
    L = len(streams)
    target = eps / np.sqrt(L)
    counts = []
    for l, x in enumerate(streams):
        n = min(n_first[l], n_max[l])
        while True:
            se = stats(x[:n], part)["stderr"]
            if se <= target or n >= n_max[l]:
                break
            n = min(n + n_check[l], n_max[l])
        counts.append(n)
    return counts


def giles_allocation(var, cost, eps):
    """Real noise counts N_l = eps^-2 sqrt(V_l / C_l) sum_k sqrt(V_k C_k).

    They minimise the total cost sum_l C_l N_l subject to sum_l V_l / N_l =
    eps^2 (Lagrange multiplier: C_l N_l^2 / V_l is the same for every level).
    """
    var = np.asarray(var, dtype=np.float64)
    cost = np.asarray(cost, dtype=np.float64)
    s = np.sum(np.sqrt(var * cost))
    return np.sqrt(var / cost) * s / eps**2


def cost_optimal_counts(streams, costs, eps, n_first, n_check, n_max, part="re"):
    """Noises used per level when the counts follow the cost-optimal allocation.

    Pilot: n_first[l] noises per level.  Then repeatedly: sample variances V_l
    from the samples so far, targets N_l = ceil(giles_allocation(V, C, eps));
    each level below its target gets the shortfall rounded up to a multiple of
    n_check[l], capped at n_max[l]; stop when no level gets more.  ``costs``:
    cost of one sample per level (fixed).
    """
    counts = [min(f, m) for f, m in zip(n_first, n_max)]
    while True:
        var = [stats(x[:n], part)["var"] for x, n in zip(streams, counts)]
        target = np.ceil(giles_allocation(var, costs, eps))
        grew = False
        for l in range(len(streams)):
            short = int(target[l]) - counts[l]
            if short > 0 and counts[l] < n_max[l]:
                add = -(-short // n_check[l]) * n_check[l]
                counts[l] = min(counts[l] + add, n_max[l])
                grew = True
        if not grew:
            return counts
