"""Pins for the oracle's learned gauge-covariant stencil network: finite-difference
gradients, linearity, gauge covariance and the per-site closed form."""
import numpy as np

import synth
from oracle import learned, wilson

DIMS = (4, 2, 2, 4)
SHAPE = (4, 2, 2, 4, 4, 3)


def _batch(seed, B):
    return synth.random_spinor(DIMS, seed, B)


def test_finite_difference_gradients():
    U = synth.random_gauge(DIMS, 0.5, 1)
    ws = learned.init_weights(3, scale=0.2)
    etas = _batch(4, 3)
    xs = _batch(5, 3)
    L, grads = learned.loss_and_grad(U, ws, etas, xs)
    rng = np.random.default_rng(0)
    for trial in range(4):
        d = [rng.standard_normal(W.shape) + 1j * rng.standard_normal(W.shape) for W in ws]
        h = 1e-6
        lp = learned.loss_and_grad(U, [W + h * dw for W, dw in zip(ws, d)], etas, xs)[0]
        lm = learned.loss_and_grad(U, [W - h * dw for W, dw in zip(ws, d)], etas, xs)[0]
        fd = (lp - lm) / (2 * h)
        an = sum(np.sum((np.conj(G) * dw).real) for G, dw in zip(grads, d))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_linearity_and_covariance():
    U = synth.random_gauge(DIMS, 0.5, 2)
    ws = learned.init_weights(7, scale=0.3)
    a, b = _batch(8, 1)[..., 0], _batch(9, 1)[..., 0]
    lhs = learned.forward(U, ws, 0.7 * a - 2.1j * b)
    rhs = 0.7 * learned.forward(U, ws, a) - 2.1j * learned.forward(U, ws, b)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()
    g = synth.gauge_transform_matrices(DIMS, 11)
    axes = (3, 2, 1, 0)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[mu] = np.einsum("...ab,...bc,...dc->...ad", g, U[mu], np.roll(g, -1, axis=axes[mu]).conj())
    ga = np.einsum("tzyxab,tzyxsb->tzyxsa", g, a)
    out1 = learned.forward(Ug, ws, ga)
    out2 = np.einsum("tzyxab,tzyxsb->tzyxsa", g, learned.forward(U, ws, a))
    assert np.abs(out1 - out2).max() < 1e-12 * np.abs(out2).max()


def test_site_local_closed_form():
    """With every hop weight zero the network is the per-site matrix W0_3 W0_2 W0_1 on the spin index."""
    U = synth.random_gauge(DIMS, 0.5, 3)
    ws = learned.init_weights(5, scale=0.3)
    for W in ws:
        W[1:] = 0
    a = _batch(6, 1)[..., 0]
    P = ws[2][0] @ ws[1][0] @ ws[0][0]
    want = np.einsum("su,tzyxua->tzyxsa", P, a)
    assert np.abs(learned.forward(U, ws, a) - want).max() < 1e-13


def test_hop_features_rebuild_wilson_hop():
    """The spin-projected sum of the 8 hop features is the Wilson hop D of M = 1 - kappa D
    (an independent construction of the same links, boundary signs and daggers)."""
    from oracle import gamma
    U = synth.random_gauge(DIMS, 0.5, 4)
    a = _batch(7, 1)[..., 0]
    feats = learned.hop_features(U, a)
    Dp = sum(np.einsum("su,tzyxua->tzyxsa", np.eye(4) - gamma.GAMMA[m], feats[1 + m]) +
             np.einsum("su,tzyxua->tzyxsa", np.eye(4) + gamma.GAMMA[m], feats[5 + m]) for m in range(4))
    D = a - wilson.apply_M(U, 1.0, a)
    assert np.abs(Dp - D).max() < 1e-12
    # a single forward-t hop weight reproduces that feature through the network
    ws = [np.zeros((9, 4, 4), complex) for _ in range(3)]
    ws[0][1 + 3] = np.eye(4)
    ws[1][0] = np.eye(4)
    ws[2][0] = np.eye(4)
    assert np.abs(learned.forward(U, ws, a) - feats[4]).max() < 1e-14


def test_adam_closed_form_for_constant_gradient():
    """Adam's bias corrections make m_hat = g and v_hat = g^2 exactly for a gradient that
    does not change, so every step moves each real parameter by -lr * g / (|g| + eps);
    real and imaginary parts are separate parameters."""
    rng = np.random.default_rng(3)
    W = [rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))]
    G = [rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))]
    G[0][0, 0] = 0.5 - 2.0j
    lr, eps = 0.01, 1e-8
    state = {}
    cur = W
    for t in range(1, 6):
        cur = learned.adam_step(cur, G, state, lr, eps=eps)
        step = lr * (G[0].real / (np.abs(G[0].real) + eps) + 1j * G[0].imag / (np.abs(G[0].imag) + eps))
        assert np.allclose(cur[0], W[0] - t * step, rtol=0, atol=1e-12)
    assert state["t"] == 5
