"""Gauge-covariant linear stencil network (a learned subtraction operator and
preconditioner; the paper has no learned part, so nothing here is cited to
it beyond the operator it approximates, M^-1 of Sec. 1).

Architecture: feature maps of C_0 = 4, C_1 = 8, C_2 = 8, C_3 = 4 channels per
site, each channel a colour 3-vector (so 12 -> 24 -> 24 -> 12 complex numbers
per site); three linear stencil layers

  out[x, o] = sum_i W0[o, i] in[x, i]
            + sum_mu sum_i ( Wf[mu][o, i] U_mu(x) in[x+mu, i]
                           + Wb[mu][o, i] U_mu(x-mu)^+ in[x-mu, i] )

with the same antiperiodic sign on time hops as M.  No nonlinearity: the
network is a fixed linear operator N, gauge covariant (U_mu(x) ->
g(x) U_mu(x) g(x+mu)^+, in -> g in gives out -> g out), so Tr(Theta N) is
well defined and a subtraction with N keeps the estimator unbiased.

Weights of a layer: array (9, C_out, C_in) complex, index 0 = W0,
1 + mu = Wf[mu], 5 + mu = Wb[mu].

Loss on pairs (eta_b, x_b = M^-1 eta_b): L = (1/B) sum_b ||N eta_b - x_b||^2 / ||x_b||^2.
Gradients use the convention G = dL/dRe(W) + i dL/dIm(W) = 2 dL/dconj(W).
"""
import numpy as np

CHANNELS = (4, 8, 8, 4)
_AXIS = (3, 2, 1, 0)


def _to_channels(psi):
    """canonical [t][z][y][x][spin][colour](,B) -> same array (spin is the channel)."""
    return psi


def _shift(f, mu, forward):
    ax = _AXIS[mu]
    out = np.roll(f, -1 if forward else 1, axis=ax)
    if mu == 3:
        out = out.copy()
        if forward:
            out[-1] *= -1.0
        else:
            out[0] *= -1.0
    return out


def _colour(Umat, f):
    """(U f)[x, i, a] = sum_b U(x)_{ab} f[x, i, b]; f shape [t,z,y,x,C,3,...]."""
    if f.ndim == 7:
        return np.matmul(Umat[:, :, :, :, None, :, :], f)
    return np.matmul(Umat[:, :, :, :, None, :, :], f[..., None])[..., 0]


def _mix(W, f):
    """(W f)[x, o, a] = sum_i W[o, i] f[x, i, a]."""
    sh = f.shape
    flat = f.reshape(sh[:4] + (sh[4], -1))
    out = np.matmul(W, flat)
    return out.reshape(sh[:4] + (W.shape[0],) + sh[5:])


def hop_features(U, f):
    """The 9 features of a layer input: f, U_mu(x) f(x+mu), U_mu(x-mu)^+ f(x-mu)."""
    feats = [f]
    back = [np.conj(np.swapaxes(np.roll(U[mu], 1, axis=_AXIS[mu]), -1, -2)) for mu in range(4)]
    for mu in range(4):
        feats.append(_colour(U[mu], _shift(f, mu, True)))
    for mu in range(4):
        feats.append(_colour(back[mu], _shift(f, mu, False)))
    return feats


def layer_forward(U, W, f):
    feats = hop_features(U, f)
    out = None
    for w in range(9):
        t = _mix(W[w], feats[w])
        out = t if out is None else out + t
    return out


def forward(U, weights, eta):
    """N eta for eta in canonical layout (optionally with a trailing batch axis)."""
    f = eta
    for W in weights:
        f = layer_forward(U, W, f)
    return f


def _adjoint_hops(U, g, w):
    """Adjoint of feature w applied to g: F_mu^+ g (w = 1+mu), B_mu^+ g (w = 5+mu)."""
    if w == 0:
        return g
    mu = (w - 1) % 4
    if w <= 4:
        # (F f)(x) = s U(x) f(x+mu)  ->  (F^+ g)(y) = s U(y-mu)^+ g(y-mu)
        Ub = np.conj(np.swapaxes(np.roll(U[mu], 1, axis=_AXIS[mu]), -1, -2))
        return _colour(Ub, _shift(g, mu, False))
    # (B f)(x) = s U(x-mu)^+ f(x-mu)  ->  (B^+ g)(y) = s U(y) g(y+mu)
    return _colour(U[mu], _shift(g, mu, True))


def loss_and_grad(U, weights, etas, xs):
    """Loss and complex gradients (2 dL/dconj W) for a batch (trailing axis B)."""
    acts = [etas]
    for W in weights:
        acts.append(layer_forward(U, W, acts[-1]))
    out = acts[-1]
    B = etas.shape[-1]
    r = out - xs
    xn = np.sum(np.abs(xs) ** 2, axis=tuple(range(6)))
    L = float(np.mean(np.sum(np.abs(r) ** 2, axis=tuple(range(6))) / xn))
    delta = 2.0 * r / (B * xn)          # 2 dL/dconj(out)
    grads = [None] * len(weights)
    for l in range(len(weights) - 1, -1, -1):
        W = weights[l]
        feats = hop_features(U, acts[l])
        G = np.zeros_like(W)
        for w in range(9):
            # G[w][o, i] = sum over sites, colour, batch of delta[x, o, a] conj(feat[x, i, a])
            G[w] = np.einsum("tzyxoab,tzyxiab->oi", delta, np.conj(feats[w]))
        grads[l] = G
        if l > 0:
            dprev = None
            for w in range(9):
                t = _adjoint_hops(U, _mix(W[w].conj().T, delta), w)
                dprev = t if dprev is None else dprev + t
            delta = dprev
    return L, grads


def init_weights(seed, scale=0.05):
    """Seeded initial weights: W0 near a channel-embedding identity, small hop weights."""
    rng = np.random.default_rng(seed)
    ws = []
    for l in range(3):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        W = scale * (rng.standard_normal((9, co, ci)) + 1j * rng.standard_normal((9, co, ci)))
        for k in range(min(ci, co)):
            W[0, k, k] += 1.0
        ws.append(W)
    return ws


def adam_step(weights, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update on complex weights (real and imaginary parts as separate parameters)."""
    t = state.get("t", 0) + 1
    state["t"] = t
    out = []
    for l, (W, G) in enumerate(zip(weights, grads)):
        m = state.setdefault(("m", l), np.zeros_like(W))
        v = state.setdefault(("v", l), np.zeros(W.shape + (2,)))
        m = beta1 * m + (1 - beta1) * G
        g2 = np.stack([G.real ** 2, G.imag ** 2], axis=-1)
        v = beta2 * v + (1 - beta2) * g2
        state[("m", l)], state[("v", l)] = m, v
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        step = mh.real / (np.sqrt(vh[..., 0]) + eps) + 1j * mh.imag / (np.sqrt(vh[..., 1]) + eps)
        out.append(W - lr * step)
    return out
