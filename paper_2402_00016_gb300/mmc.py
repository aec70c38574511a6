"""Thin Python binding of the C ABI in include/mmc.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Device fields are
torch uint8 tensors on the context's device (see ``new_field``); host arrays
are numpy complex128 in the canonical order.  There is no CPU fallback: if
libmmc.so cannot be loaded, importing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmmc.so")

MMC_OK = 0
MMC_F64, MMC_F32, MMC_BF16 = 0, 1, 2
MMC_THETA_ONE, MMC_THETA_G4, MMC_THETA_G5 = 0, 1, 2
MMC_EXACT_UNIT, MMC_EXACT_PROBE = 0, 1
MMC_OP_M = -1
MMC_ZERO = -1
MMC_INV = -2
MMC_TAG_NOISE = 0x4E4F4953
MMC_TAG_GMRES = 0x474D5253
MMC_TAG_ARNOLDI = 0x4445464C
MMC_NET_BASE = 0x100000
MMC_ROUND_NEAREST, MMC_ROUND_STOCHASTIC = 0, 1
MMC_NET_WEIGHTS = 1152
PREC = {"f64": MMC_F64, "f32": MMC_F32, "bf16": MMC_BF16}
THETA = {"1": MMC_THETA_ONE, "g4": MMC_THETA_G4, "g5": MMC_THETA_G5}
ERRORS = {-1: "MMC_ERR_ARG", -2: "MMC_ERR_NOMEM", -3: "MMC_ERR_CUDA", -4: "MMC_ERR_BREAKDOWN",
          -5: "MMC_ERR_NOCONV", -6: "MMC_ERR_TIMEOUT", -7: "MMC_ERR_NAN", -8: "MMC_ERR_STATE"}
(MMC_ERR_ARG, MMC_ERR_NOMEM, MMC_ERR_CUDA, MMC_ERR_BREAKDOWN, MMC_ERR_NOCONV, MMC_ERR_TIMEOUT, MMC_ERR_NAN,
 MMC_ERR_STATE) = range(-1, -9, -1)

if not os.path.exists(_LIB_PATH):
    raise ImportError("libmmc.so is not built (run __graft_entry__.build() or paper_2402_00016_gb300/build.py)")
lib = ctypes.CDLL(_LIB_PATH)

_vp, _i, _d, _u32, _u64, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint32,
                                ctypes.c_uint64, ctypes.c_size_t)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class mmc_level_stats(ctypes.Structure):
    _fields_ = [("n", _i), ("k_deflated", _i), ("mean_re", _d), ("mean_im", _d), ("var_re", _d),
                ("var_im", _d), ("cvar", _d), ("stderr_re", _d), ("stderr_im", _d), ("corr_re", _d),
                ("corr_im", _d), ("value_re", _d), ("value_im", _d), ("seconds", _d),
                ("matvecs", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mmc_level_spec(ctypes.Structure):
    _fields_ = [("hi", _i), ("lo", _i), ("deflate", _i), ("level", ctypes.c_uint32), ("n_first", _i),
                ("n_check", _i), ("n_max", _i)]


MMC_ALLOC_EQUAL, MMC_ALLOC_COST = 0, 1


class mmc_profile_stats(ctypes.Structure):
    _fields_ = [("step_launches", ctypes.c_longlong), ("step_ms", _d), ("step_bytes", _d), ("step_flops", _d),
                ("all_launches", ctypes.c_longlong), ("graph_launches", ctypes.c_longlong),
                ("graph_captures", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mmc_profile_class(ctypes.Structure):
    _fields_ = [("kind", _i), ("prec", _i), ("nrhs_padded", _i), ("launches", ctypes.c_longlong), ("ms", _d),
                ("bytes", _d), ("flops", _d)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PROF_KINDS = {0: "plain", 1: "bilinear", 2: "accumulate", 3: "aux"}

_SIGS = {
    "mmc_create": (_i, [ctypes.POINTER(_vp), _ip, _u64, _i]),
    "mmc_destroy": (_i, [_vp]),
    "mmc_last_error": (ctypes.c_char_p, [_vp]),
    "mmc_set_seed": (_i, [_vp, _u64]),
    "mmc_rhs_block": (_i, [_i]),
    "mmc_field_bytes": (_sz, [_vp, _i, _i]),
    "mmc_load_gauge": (_i, [_vp, _dp, _d, _i]),
    "mmc_pack": (_i, [_vp, _dp, _i, _i, _vp]),
    "mmc_unpack": (_i, [_vp, _vp, _i, _i, _dp]),
    "mmc_apply_M": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "mmc_noise": (_i, [_vp, _u32, _u32, _u32, _i, _i, _vp, _vp]),
    "mmc_noise_noalloc": (_i, [_vp, _u32, _u32, _u32, _i, _i, _vp, _vp]),
    "mmc_gmres_poly": (_i, [_vp, _i, _i, _dp, _ip]),
    "mmc_poly_from_roots": (_i, [_vp, _i, _dp, _ip]),
    "mmc_poly_double": (_i, [_vp, _i, _i, _ip]),
    "mmc_poly_degree": (_i, [_vp, _i]),
    "mmc_poly_eval": (_i, [_vp, _i, _i, _dp, _dp]),
    "mmc_apply_poly": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp]),
    "mmc_deflate": (_i, [_vp, _i, _i, _i, _d, _dp, _ip]),
    "mmc_solve": (_i, [_vp, _vp, _vp, _i, _d, _i, _i, _i, _i, _ip, _dp]),
    "mmc_set_deflation": (_i, [_vp, _i, _dp, _dp, _dp]),
    "mmc_get_deflation": (_i, [_vp, _ip, _dp, _dp, _dp]),
    "mmc_set_tensor_projections": (_i, [_vp, _i]),
    "mmc_trace_level": (_i, [_vp, _i, _i, _i, _i, _i, _u32, _u32, _i, _i,
                             ctypes.POINTER(mmc_level_stats), _dp]),
    "mmc_trace_levels": (_i, [_vp, _i, _ip, _ip, _ip, ctypes.POINTER(_u32), ctypes.POINTER(_u32), _i, _i, _i,
                              ctypes.POINTER(mmc_level_stats), ctypes.POINTER(_dp)]),
    "mmc_trace_exact": (_i, [_vp, _i, _i, _i, _i, _dp]),
    "mmc_estimate": (_i, [_vp, _i, ctypes.POINTER(mmc_level_spec), _i, _i, _i, _d, _i, _dp, _u32,
                          ctypes.POINTER(mmc_level_stats), _dp]),
    "mmc_probe_colours": (_i, [_vp, _i, _ip]),
    "mmc_net_create": (_i, [_vp, _dp, _u64, _ip]),
    "mmc_net_set_weights": (_i, [_vp, _i, _dp]),
    "mmc_net_get_weights": (_i, [_vp, _i, _dp]),
    "mmc_net_apply": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "mmc_net_loss_grad": (_i, [_vp, _i, _vp, _vp, _i, _dp, _dp]),
    "mmc_net_train": (_i, [_vp, _i, _vp, _vp, _i, _i, _i, _d, _dp]),
    "mmc_profile": (_i, [_vp, _i]),
    "mmc_profile_read": (_i, [_vp, ctypes.POINTER(mmc_profile_stats)]),
    "mmc_profile_classes": (_i, [_vp, _i, ctypes.POINTER(mmc_profile_class), _ip]),
    "mmc_update_gauge": (_i, [_vp, _dp]),
    "mmc_set_step_variant": (_i, [_vp, _i, _i, _i, _i]),
    "mmc_set_step_variant_class": (_i, [_vp, _i, _i, _i, _i, _i, _i, _i, _i]),
    "mmc_set_graphs": (_i, [_vp, _i]),
    "mmc_set_solve_storage": (_i, [_vp, _i]),
    "mmc_set_rhs_block_max": (_i, [_vp, _i]),
    "mmc_test_stall_staged": (_i, [_vp, _i, ctypes.c_longlong]),
    "mmc_graph_note": (ctypes.c_char_p, [_vp]),
    "mmc_set_solve_params": (_i, [_vp, _i, _i]),
    "mmc_set_solve_refinement": (_i, [_vp, _d, _i]),
    "mmc_set_gram_schmidt": (_i, [_vp, _i]),
    "mmc_set_horner_layout": (_i, [_vp, _i]),
    "mmc_autotune": (_i, [_vp, _i, _i, _ip, _dp]),
    "mmc_harmonic_ritz": (_i, [_i, _dp, _i, _dp]),
    "mmc_leja_order": (_i, [_i, _dp, _dp]),
    "mmc_eig": (_i, [_i, _dp, _i, _dp, _dp]),
    "mmc_deflation_pairs": (_i, [_i, _dp, _dp, _d, _i, _ip, _ip, _ip]),
    "mmc_set_deflation_bound": (_i, [_vp, _d]),
    "mmc_set_rounding": (_i, [_vp, _i, _u64]),
    "mmc_net_set_precision": (_i, [_vp, _i, _i]),
    "mmc_convert": (_i, [_vp, _vp, _i, _vp, _i, _i, _vp]),
    "mmc_gmres_poly_deflated": (_i, [_vp, _i, _i, _dp, _ip]),
    "mmc_probe_colouring": (_i, [_ip, _i, _ip, _ip]),
    "mmc_deflation_condition": (_i, [_i, _dp, _i, _ip, _d, _ip, _ip]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class MMCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "error"), code, msg))
        self.code = code


def _check(code, ctx=None):
    if code != MMC_OK:
        msg = lib.mmc_last_error(ctx).decode() if ctx else ""
        raise MMCError(code, msg)


def _cplx(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data_as(_dp)


def _stream(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------------ context
def mmc_create(dims, seed=0, device=0):
    ctx = _vp()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    _check(lib.mmc_create(ctypes.byref(ctx), d, int(seed), int(device)))
    return ctx


def mmc_destroy(ctx):
    _check(lib.mmc_destroy(ctx))


def mmc_last_error(ctx):
    return lib.mmc_last_error(ctx).decode()


def mmc_set_seed(ctx, seed):
    _check(lib.mmc_set_seed(ctx, int(seed)), ctx)


def mmc_rhs_block(nrhs):
    return lib.mmc_rhs_block(int(nrhs))


def mmc_field_bytes(ctx, nrhs, prec):
    return lib.mmc_field_bytes(ctx, int(nrhs), int(prec))


def new_field(ctx, nrhs, prec, device="cuda"):
    """A zeroed device field (torch uint8 tensor) for nrhs vectors of precision prec."""
    import torch
    return torch.zeros(mmc_field_bytes(ctx, nrhs, prec), dtype=torch.uint8, device=device)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if hasattr(t, "data_ptr") else ctypes.c_void_p(int(t))


# ----------------------------------------------------------------- operator
def mmc_load_gauge(ctx, U, kappa, t_antiperiodic=1):
    U, p = _cplx(U)
    _check(lib.mmc_load_gauge(ctx, p, float(kappa), int(t_antiperiodic)), ctx)


def mmc_pack(ctx, host, nrhs, prec, field):
    host, p = _cplx(host)
    _check(lib.mmc_pack(ctx, p, int(nrhs), int(prec), _ptr(field)), ctx)


def mmc_unpack(ctx, field, nrhs, prec, vol):
    out = np.empty(int(nrhs) * int(vol) * 12, dtype=np.complex128)
    _check(lib.mmc_unpack(ctx, _ptr(field), int(nrhs), int(prec), out.ctypes.data_as(_dp)), ctx)
    return out.reshape(int(nrhs), int(vol) * 12)


def mmc_apply_M(ctx, x, y, nrhs, prec, dagger=0, stream=None):
    _check(lib.mmc_apply_M(ctx, _ptr(x), _ptr(y), int(nrhs), int(prec), int(dagger), _stream(stream)), ctx)


def mmc_noise(ctx, level, first, tag, nrhs, prec, field, stream=None):
    _check(lib.mmc_noise(ctx, int(level), int(first), int(tag), int(nrhs), int(prec), _ptr(field),
                         _stream(stream)), ctx)


def mmc_noise_noalloc(ctx, level, first, tag, nrhs, prec, field, stream=None):
    """mmc_noise for callers that cannot allocate device memory (static id table, <= 4096 rhs)."""
    _check(lib.mmc_noise_noalloc(ctx, int(level), int(first), int(tag), int(nrhs), int(prec), _ptr(field),
                                 _stream(stream)), ctx)


# --------------------------------------------------------------- polynomials
def mmc_gmres_poly(ctx, m, op_handle=MMC_OP_M):
    theta = np.zeros(2 * int(m))
    h = ctypes.c_int()
    _check(lib.mmc_gmres_poly(ctx, int(m), int(op_handle), theta.ctypes.data_as(_dp), ctypes.byref(h)), ctx)
    return h.value, theta[0::2] + 1j * theta[1::2]


def mmc_poly_from_roots(ctx, theta):
    theta, p = _cplx(theta)
    h = ctypes.c_int()
    _check(lib.mmc_poly_from_roots(ctx, int(theta.size), p, ctypes.byref(h)), ctx)
    return h.value


def mmc_poly_double(ctx, h_in, h_out):
    h = ctypes.c_int()
    _check(lib.mmc_poly_double(ctx, int(h_in), int(h_out), ctypes.byref(h)), ctx)
    return h.value


def mmc_poly_degree(ctx, handle):
    d = lib.mmc_poly_degree(ctx, int(handle))
    if d < 0:
        _check(d, ctx)
    return d


def mmc_poly_eval(ctx, handle, alpha):
    alpha, p = _cplx(np.atleast_1d(alpha))
    out = np.zeros(alpha.size, dtype=np.complex128)
    _check(lib.mmc_poly_eval(ctx, int(handle), int(alpha.size), p, out.ctypes.data_as(_dp)), ctx)
    return out


def mmc_apply_poly(ctx, handle, x, y, nrhs, prec, stream=None):
    _check(lib.mmc_apply_poly(ctx, int(handle), _ptr(x), _ptr(y), int(nrhs), int(prec), _stream(stream)), ctx)


# -------------------------------------------------------- deflation / solves
def mmc_deflate(ctx, k, poly_handle, m_arnoldi, tol_accept=1e-3):
    lam = np.zeros(2 * int(k))
    ka = ctypes.c_int()
    _check(lib.mmc_deflate(ctx, int(k), int(poly_handle), int(m_arnoldi), float(tol_accept),
                           lam.ctypes.data_as(_dp), ctypes.byref(ka)), ctx)
    return (lam[0::2] + 1j * lam[1::2])[: ka.value]


def mmc_set_deflation(ctx, lam, Z, U):
    """Z, U: arrays (k, 12V) complex in canonical order; lam: k complex."""
    lam, pl = _cplx(np.atleast_1d(lam))
    Z, pz = _cplx(Z)
    U, pu = _cplx(U)
    _check(lib.mmc_set_deflation(ctx, int(lam.size), pl, pz, pu), ctx)


def mmc_get_deflation(ctx, vol):
    k = ctypes.c_int()
    _check(lib.mmc_get_deflation(ctx, ctypes.byref(k), None, None, None), ctx)
    lam = np.zeros(2 * k.value)
    Z = np.zeros(2 * k.value * 12 * int(vol))
    U = np.zeros(2 * k.value * 12 * int(vol))
    _check(lib.mmc_get_deflation(ctx, ctypes.byref(k), lam.ctypes.data_as(_dp), Z.ctypes.data_as(_dp),
                                 U.ctypes.data_as(_dp)), ctx)
    c = lambda a: (a[0::2] + 1j * a[1::2])
    return c(lam), c(Z).reshape(k.value, -1), c(U).reshape(k.value, -1)


def mmc_set_tensor_projections(ctx, enable):
    _check(lib.mmc_set_tensor_projections(ctx, int(enable)), ctx)


def mmc_solve(ctx, b, x, nrhs, rel_tol=1e-10, precond_handle=MMC_ZERO, prec_inner=MMC_F32, m_inner=48,
              max_outer=400):
    its = ctypes.c_int()
    rel = np.zeros(int(nrhs))
    _check(lib.mmc_solve(ctx, _ptr(b), _ptr(x), int(nrhs), float(rel_tol), int(precond_handle), int(prec_inner),
                         int(m_inner), int(max_outer), ctypes.byref(its), rel.ctypes.data_as(_dp)), ctx)
    return its.value, rel


# --------------------------------------------------------------- estimators
def mmc_trace_level(ctx, hi, lo, theta_op, deflate, n_noise, first_noise, level, prec, precond=MMC_ZERO,
                    want_samples=True):
    st = mmc_level_stats()
    samples = np.zeros(2 * int(n_noise)) if want_samples else None
    _check(lib.mmc_trace_level(ctx, int(hi), int(lo), int(theta_op), int(deflate), int(n_noise),
                               int(first_noise), int(level), int(prec), int(precond), ctypes.byref(st),
                               samples.ctypes.data_as(_dp) if want_samples else None), ctx)
    s = st.as_dict()
    if want_samples:
        s["samples"] = samples[0::2] + 1j * samples[1::2]
    return s


def mmc_trace_levels(ctx, his, los, theta_op, deflate, n_noises, first_noises, levels, prec, want_samples=True):
    """Several polynomial levels in one batch; a list of per-level dicts as mmc_trace_level's."""
    n = len(his)
    if not (len(los) == len(n_noises) == len(first_noises) == len(levels) == n):
        raise ValueError("per-level arguments must have the same length")
    ia = lambda v: (ctypes.c_int * n)(*[int(x) for x in v])
    ua = lambda v: (ctypes.c_uint32 * n)(*[int(x) for x in v])
    st = (mmc_level_stats * n)()
    bufs = [np.zeros(2 * int(k)) for k in n_noises] if want_samples else None
    ptrs = (_dp * n)(*[b.ctypes.data_as(_dp) for b in bufs]) if want_samples else None
    _check(lib.mmc_trace_levels(ctx, n, ia(his), ia(los), ia(n_noises), ua(first_noises), ua(levels),
                                int(theta_op), int(deflate), int(prec), st, ptrs), ctx)
    out = []
    for l in range(n):
        d = st[l].as_dict()
        if want_samples:
            d["samples"] = bufs[l][0::2] + 1j * bufs[l][1::2]
        out.append(d)
    return out


def mmc_trace_exact(ctx, handle, theta_op, method, prec=MMC_F64):
    out = np.zeros(2)
    _check(lib.mmc_trace_exact(ctx, int(handle), int(theta_op), int(method), int(prec), out.ctypes.data_as(_dp)),
           ctx)
    return out[0] + 1j * out[1]


def mmc_probe_colours(ctx, reach):
    n = ctypes.c_int()
    _check(lib.mmc_probe_colours(ctx, int(reach), ctypes.byref(n)), ctx)
    return n.value


# ----------------------------------------------------------- learned network
def _weights_in(weights):
    """Accept a list of three (9, C_out, C_in) complex arrays or a flat complex array."""
    if isinstance(weights, (list, tuple)):
        weights = np.concatenate([np.asarray(w, dtype=np.complex128).ravel() for w in weights])
    w = np.ascontiguousarray(weights, dtype=np.complex128).ravel()
    if w.size != MMC_NET_WEIGHTS:
        raise ValueError("expected %d complex weights" % MMC_NET_WEIGHTS)
    return w


def _weights_out(flat):
    shapes = [(9, 8, 4), (9, 8, 8), (9, 4, 8)]
    out, off = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(flat[off:off + n].reshape(sh))
        off += n
    return out


def mmc_net_create(ctx, weights=None, seed=0):
    h = ctypes.c_int()
    if weights is None:
        _check(lib.mmc_net_create(ctx, None, int(seed), ctypes.byref(h)), ctx)
    else:
        w = _weights_in(weights)
        _check(lib.mmc_net_create(ctx, w.ctypes.data_as(_dp), int(seed), ctypes.byref(h)), ctx)
    return h.value


def mmc_net_set_weights(ctx, handle, weights):
    w = _weights_in(weights)
    _check(lib.mmc_net_set_weights(ctx, int(handle), w.ctypes.data_as(_dp)), ctx)


def mmc_net_get_weights(ctx, handle):
    out = np.zeros(2 * MMC_NET_WEIGHTS)
    _check(lib.mmc_net_get_weights(ctx, int(handle), out.ctypes.data_as(_dp)), ctx)
    return _weights_out(out[0::2] + 1j * out[1::2])


def mmc_net_apply(ctx, handle, x, y, nrhs, stream=None):
    _check(lib.mmc_net_apply(ctx, int(handle), _ptr(x), _ptr(y), int(nrhs), _stream(stream)), ctx)


def mmc_net_loss_grad(ctx, handle, eta, xs, nrhs):
    loss = ctypes.c_double()
    g = np.zeros(2 * MMC_NET_WEIGHTS)
    _check(lib.mmc_net_loss_grad(ctx, int(handle), _ptr(eta), _ptr(xs), int(nrhs), ctypes.byref(loss),
                                 g.ctypes.data_as(_dp)), ctx)
    return loss.value, _weights_out(g[0::2] + 1j * g[1::2])


def mmc_net_train(ctx, handle, eta, xs, npairs, batch, iters, lr):
    hist = np.zeros(max(1, int(iters)))
    _check(lib.mmc_net_train(ctx, int(handle), _ptr(eta), _ptr(xs), int(npairs), int(batch), int(iters),
                             float(lr), hist.ctypes.data_as(_dp)), ctx)
    return hist[: int(iters)]


# ---------------------------------------------------------------- profiling
def mmc_profile(ctx, enable):
    _check(lib.mmc_profile(ctx, int(enable)), ctx)


def mmc_profile_read(ctx):
    st = mmc_profile_stats()
    _check(lib.mmc_profile_read(ctx, ctypes.byref(st)), ctx)
    return st.as_dict()


def mmc_test_stall_staged(ctx, enable, wait_iters=0):
    """Fault injection for tests: the staged step kernel's bounded waits run out."""
    _check(lib.mmc_test_stall_staged(ctx, int(bool(enable)), int(wait_iters)), ctx)


def mmc_set_rhs_block_max(ctx, rmax):
    _check(lib.mmc_set_rhs_block_max(ctx, int(rmax)), ctx)


def mmc_set_solve_storage(ctx, prec_inner):
    _check(lib.mmc_set_solve_storage(ctx, int(prec_inner)), ctx)


def mmc_set_solve_params(ctx, m_inner=0, max_outer=0):
    _check(lib.mmc_set_solve_params(ctx, int(m_inner), int(max_outer)), ctx)


def mmc_set_solve_refinement(ctx, inner_reduction, inner_cycles):
    _check(lib.mmc_set_solve_refinement(ctx, float(inner_reduction), int(inner_cycles)), ctx)


def mmc_set_gram_schmidt(ctx, passes):
    _check(lib.mmc_set_gram_schmidt(ctx, int(passes)), ctx)


def mmc_set_horner_layout(ctx, paired):
    _check(lib.mmc_set_horner_layout(ctx, int(paired)), ctx)


def mmc_set_step_variant(ctx, prec, rpt=0, minb=0, spc=0):
    _check(lib.mmc_set_step_variant(ctx, int(prec), int(rpt), int(minb), int(spc)), ctx)


def mmc_set_graphs(ctx, enable):
    _check(lib.mmc_set_graphs(ctx, int(bool(enable))), ctx)


def mmc_graph_note(ctx):
    return lib.mmc_graph_note(ctx).decode()


def mmc_set_step_variant_class(ctx, prec, rhs_class, v):
    """v: a dict as returned by mmc_autotune (rpt, minb, spc, version, blocked, ns)."""
    _check(lib.mmc_set_step_variant_class(ctx, int(prec), int(rhs_class), int(v["version"]), int(v["rpt"]),
                                          int(v["minb"]), int(v["spc"]), int(v.get("blocked", 0)),
                                          int(v.get("ns", 0))), ctx)


def mmc_estimate(ctx, levels, theta_op, prec, precond, eps, alloc=MMC_ALLOC_EQUAL, cost=None, first_noise=0):
    """levels: list of dicts with hi, lo, deflate, level, n_first, n_check, n_max.
    Returns (per-level stats dicts, total value, total stderr)."""
    L = len(levels)
    specs = (mmc_level_spec * L)(*[mmc_level_spec(int(v["hi"]), int(v["lo"]), int(v.get("deflate", 0)),
                                                  int(v["level"]), int(v["n_first"]), int(v["n_check"]),
                                                  int(v["n_max"])) for v in levels])
    out = (mmc_level_stats * L)()
    tot = np.zeros(2)
    c = None
    if cost is not None:
        c = np.ascontiguousarray(cost, dtype=np.float64)
        assert c.size == L
    _check(lib.mmc_estimate(ctx, L, specs, int(theta_op), int(prec), int(precond), float(eps), int(alloc),
                            c.ctypes.data_as(_dp) if c is not None else None, int(first_noise), out,
                            tot.ctypes.data_as(_dp)), ctx)
    return [o.as_dict() for o in out], float(tot[0]), float(tot[1])


def mmc_autotune(ctx, nrhs, prec):
    best = (ctypes.c_int * 6)()
    ms = ctypes.c_double()
    _check(lib.mmc_autotune(ctx, int(nrhs), int(prec), best, ctypes.byref(ms)), ctx)
    return {"rpt": best[0], "minb": best[1], "spc": best[2], "version": best[3], "blocked": best[4],
            "ns": best[5], "ms": ms.value}


def mmc_update_gauge(ctx, U):
    U, p = _cplx(U)
    _check(lib.mmc_update_gauge(ctx, p), ctx)


# ---------------------------------------------------------- host-only helpers
def mmc_harmonic_ritz(H):
    H = np.asfortranarray(H, dtype=np.complex128)
    m = H.shape[1]
    out = np.zeros(2 * m)
    _check(lib.mmc_harmonic_ritz(int(m), H.ctypes.data_as(_dp), int(H.shape[0]), out.ctypes.data_as(_dp)))
    return out[0::2] + 1j * out[1::2]


def mmc_leja_order(theta):
    theta, p = _cplx(theta)
    out = np.zeros(2 * theta.size)
    _check(lib.mmc_leja_order(int(theta.size), p, out.ctypes.data_as(_dp)))
    return out[0::2] + 1j * out[1::2]


def mmc_eig(A, vectors=False):
    A = np.asfortranarray(A, dtype=np.complex128)
    n = A.shape[0]
    w = np.zeros(2 * n)
    vr = np.zeros(2 * n * n) if vectors else None
    _check(lib.mmc_eig(int(n), A.ctypes.data_as(_dp), int(n), w.ctypes.data_as(_dp),
                       vr.ctypes.data_as(_dp) if vectors else None))
    ev = w[0::2] + 1j * w[1::2]
    if not vectors:
        return ev
    V = (vr[0::2] + 1j * vr[1::2]).reshape(n, n, order="F")
    return ev, V


def mmc_deflation_pairs(lam, res, tol_accept, k):
    """(keep, partner): candidate indices of the kept eigenpairs and their gamma_5 partners."""
    lam, p = _cplx(lam)
    res = np.ascontiguousarray(res, dtype=np.float64)
    m = lam.size
    keep = np.zeros(max(1, m), dtype=np.int32)
    partner = np.zeros(max(1, m), dtype=np.int32)
    n = ctypes.c_int(0)
    _check(lib.mmc_deflation_pairs(int(m), p, res.ctypes.data_as(_dp), float(tol_accept), int(k),
                                   keep.ctypes.data_as(_ip), partner.ctypes.data_as(_ip), ctypes.byref(n)))
    return [int(v) for v in keep[: n.value]], [int(v) for v in partner[: n.value]]


def mmc_deflation_condition(S, mates, max_u=100.0):
    """Kept positions of the pairs after the overlap drop rules."""
    S = np.asfortranarray(S, dtype=np.complex128)
    q = S.shape[0]
    mates = np.ascontiguousarray(mates, dtype=np.int32)
    sel = np.zeros(max(1, q), dtype=np.int32)
    n = ctypes.c_int(0)
    _check(lib.mmc_deflation_condition(int(q), S.ctypes.data_as(_dp), int(q), mates.ctypes.data_as(_ip),
                                       float(max_u), sel.ctypes.data_as(_ip), ctypes.byref(n)))
    return [int(v) for v in sel[: n.value]]


def mmc_set_deflation_bound(ctx, max_u):
    _check(lib.mmc_set_deflation_bound(ctx, float(max_u)), ctx)


def mmc_probe_colouring(dims, reach):
    """(colour per site, number of colours) of the probing colouring; pure host."""
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    V = int(np.prod(dims))
    colour = np.zeros(V, dtype=np.int32)
    n = ctypes.c_int(0)
    _check(lib.mmc_probe_colouring(d, int(reach), colour.ctypes.data_as(_ip), ctypes.byref(n)))
    return colour, n.value


def mmc_profile_classes(ctx):
    """Per-class step-kernel counters (list of dicts; kind named by PROF_KINDS)."""
    n = ctypes.c_int(0)
    _check(lib.mmc_profile_classes(ctx, 0, None, ctypes.byref(n)), ctx)
    arr = (mmc_profile_class * max(1, n.value))()
    _check(lib.mmc_profile_classes(ctx, n.value, arr, ctypes.byref(n)), ctx)
    out = []
    for i in range(n.value):
        d = arr[i].as_dict()
        d["kind"] = PROF_KINDS.get(d["kind"], str(d["kind"]))
        out.append(d)
    return out


def mmc_gmres_poly_deflated(ctx, m, op_handle=MMC_OP_M):
    """(handle, theta): GMRES(m) polynomial from the start vector with the deflated eigenvectors removed."""
    theta = np.zeros(2 * int(m))
    h = ctypes.c_int()
    _check(lib.mmc_gmres_poly_deflated(ctx, int(m), int(op_handle), theta.ctypes.data_as(_dp), ctypes.byref(h)), ctx)
    return h.value, theta[0::2] + 1j * theta[1::2]


def mmc_set_rounding(ctx, mode, seed=0):
    """BF16 chain storage: MMC_ROUND_NEAREST or MMC_ROUND_STOCHASTIC (salt sequence from seed)."""
    _check(lib.mmc_set_rounding(ctx, int(mode), int(seed) & 0xFFFFFFFFFFFFFFFF), ctx)


def mmc_net_set_precision(ctx, handle, prec):
    _check(lib.mmc_net_set_precision(ctx, int(handle), int(prec)), ctx)


def mmc_convert(ctx, src, src_prec, dst, dst_prec, nrhs, stream=None):
    _check(lib.mmc_convert(ctx, _ptr(src), int(src_prec), _ptr(dst), int(dst_prec), int(nrhs), _stream(stream)), ctx)
