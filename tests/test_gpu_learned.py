"""GPU parity of the learned gauge-covariant stencil network against the oracle
(forward pass and Wirtinger gradients), its training, and what it gains: as
the right preconditioner of the refined solves it cuts the inner iterations
against the unpreconditioned method; as a level operand and in the exact
trace it matches the oracle.  FP32 kernels: tolerance 1e-5 relative for the
forward pass, 1e-4 for gradients (sums over every site and colour)."""
import numpy as np
import pytest

import synth
from oracle import learned, wilson, gamma

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 2, 6)
SHAPE = (6, 2, 4, 4, 4, 3)


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


@pytest.fixture(scope="module")
def env(mmc):
    U = synth.random_gauge(DIMS, 0.5, 1)
    ctx = mmc.mmc_create(DIMS, seed=4, device=0)
    mmc.mmc_load_gauge(ctx, U, 0.13, 1)
    yield U, ctx
    mmc.mmc_destroy(ctx)


def _batch_canon(seed, B):
    return synth.random_spinor(DIMS, seed, B)  # [t,z,y,x,4,3,B]


def _to_rows(a):
    return a.transpose(6, 0, 1, 2, 3, 4, 5).reshape(a.shape[-1], -1)


def test_forward_matches_oracle(mmc, env):
    U, ctx = env
    ws = learned.init_weights(3, scale=0.2)
    h = mmc.mmc_net_create(ctx, ws)
    B = 21
    xin = _batch_canon(5, B)
    x = mmc.new_field(ctx, B, mmc.MMC_F32)
    y = mmc.new_field(ctx, B, mmc.MMC_F32)
    mmc.mmc_pack(ctx, _to_rows(xin), B, mmc.MMC_F32, x)
    xr = mmc.mmc_unpack(ctx, x, B, mmc.MMC_F32, 192)
    mmc.mmc_net_apply(ctx, h, x, y, B)
    got = mmc.mmc_unpack(ctx, y, B, mmc.MMC_F32, 192)
    for j in range(B):
        want = learned.forward(U, ws, xr[j].reshape(SHAPE)).ravel()
        assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < 1e-5


def test_loss_and_gradients_match_oracle(mmc, env):
    U, ctx = env
    ws = learned.init_weights(8, scale=0.2)
    h = mmc.mmc_net_create(ctx, ws)
    B = 16
    e = _batch_canon(11, B)
    t = _batch_canon(12, B)
    ef = mmc.new_field(ctx, B, mmc.MMC_F32)
    tf = mmc.new_field(ctx, B, mmc.MMC_F32)
    mmc.mmc_pack(ctx, _to_rows(e), B, mmc.MMC_F32, ef)
    mmc.mmc_pack(ctx, _to_rows(t), B, mmc.MMC_F32, tf)
    e32 = mmc.mmc_unpack(ctx, ef, B, mmc.MMC_F32, 192).T.reshape(SHAPE + (B,))
    t32 = mmc.mmc_unpack(ctx, tf, B, mmc.MMC_F32, 192).T.reshape(SHAPE + (B,))
    L_ref, g_ref = learned.loss_and_grad(U, ws, e32, t32)
    L, g = mmc.mmc_net_loss_grad(ctx, h, ef, tf, B)
    assert abs(L - L_ref) < 1e-5 * abs(L_ref)
    for G, Gr in zip(g, g_ref):
        assert np.linalg.norm(G - Gr) < 1e-4 * np.linalg.norm(Gr)


def _solve_pairs(mmc, ctx, n, level):
    b = mmc.new_field(ctx, n, mmc.MMC_F64)
    x = mmc.new_field(ctx, n, mmc.MMC_F64)
    mmc.mmc_noise(ctx, level, 0, mmc.MMC_TAG_NOISE, n, mmc.MMC_F64, b)
    its, rel = mmc.mmc_solve(ctx, b, x, n, 1e-8, mmc.MMC_ZERO, mmc.MMC_F32, 24, 200)
    b32 = mmc.new_field(ctx, n, mmc.MMC_F32)
    x32 = mmc.new_field(ctx, n, mmc.MMC_F32)
    mmc.mmc_pack(ctx, mmc.mmc_unpack(ctx, b, n, mmc.MMC_F64, 192), n, mmc.MMC_F32, b32)
    mmc.mmc_pack(ctx, mmc.mmc_unpack(ctx, x, n, mmc.MMC_F64, 192), n, mmc.MMC_F32, x32)
    return b, b32, x32


def test_training_and_preconditioner_gain(mmc, env):
    U, ctx = env
    h = mmc.mmc_net_create(ctx, None, 7)
    _, eta, xs = _solve_pairs(mmc, ctx, 64, 21)
    hist = mmc.mmc_net_train(ctx, h, eta, xs, 64, 16, 300, 3e-3)
    assert hist[-10:].mean() < 0.5 * hist[:4].mean(), (hist[:4], hist[-10:])
    # what the trained network gains: fewer inner FGMRES iterations at the same 1e-10 target
    b = mmc.new_field(ctx, 4, mmc.MMC_F64)
    mmc.mmc_noise(ctx, 33, 0, mmc.MMC_TAG_NOISE, 4, mmc.MMC_F64, b)
    x0 = mmc.new_field(ctx, 4, mmc.MMC_F64)
    its_plain, _ = mmc.mmc_solve(ctx, b, x0, 4, 1e-10, mmc.MMC_ZERO, mmc.MMC_F32, 8, 400)
    x1 = mmc.new_field(ctx, 4, mmc.MMC_F64)
    its_net, rel = mmc.mmc_solve(ctx, b, x1, 4, 1e-10, h, mmc.MMC_F32, 8, 400)
    assert rel.max() <= 1e-10
    assert its_net < its_plain, (its_net, its_plain)


def test_level_and_exact_trace_with_network(mmc, env):
    U, ctx = env
    ws = learned.init_weights(9, scale=0.2)
    h = mmc.mmc_net_create(ctx, ws)
    n = 5
    st = mmc.mmc_trace_level(ctx, h, mmc.MMC_ZERO, mmc.MMC_THETA_ONE, 0, n, 0, 6, mmc.MMC_BF16)
    from oracle import noise
    for j in range(n):
        e = noise.z4_noise(DIMS, 4, j, 6)
        want = np.vdot(e.ravel(), learned.forward(U, ws, e).ravel())
        assert abs(st["samples"][j] - want) < 1e-5 * np.linalg.norm(e) ** 2
    # exact Tr(N) and Tr(gamma4 N): unit vectors and probing (reach 3) against the oracle
    E = np.eye(12 * 192).reshape(SHAPE + (12 * 192,))
    NE = learned.forward(U, ws, E).reshape(12 * 192, 12 * 192)
    ref1 = np.trace(NE)
    G4 = np.kron(np.eye(192), np.kron(gamma.GAMMA[3], np.eye(3)))
    ref4 = np.trace(G4 @ NE)
    for method in (mmc.MMC_EXACT_UNIT, mmc.MMC_EXACT_PROBE):
        got1 = mmc.mmc_trace_exact(ctx, h, mmc.MMC_THETA_ONE, method)
        got4 = mmc.mmc_trace_exact(ctx, h, mmc.MMC_THETA_G4, method)
        assert abs(got1 - ref1) < 1e-5 * abs(ref1)
        assert abs(got4 - ref4) < 1e-5 * abs(ref1)


BF16_UNIT = 2.0 ** -8


def test_bf16_network_forward_matches_oracle(mmc, env):
    """BF16 weights and hidden activations, FP32 arithmetic: against the FP64 oracle with the
    same (unrounded) weights.  Each weight and each stored hidden activation carries a
    relative rounding error of at most 2^-9; through three layers of norm about 1 that
    leaves a normwise relative error of a few times 2^-8: the bound is 4 x 2^-8."""
    U, ctx = env
    ws = learned.init_weights(3, scale=0.2)
    h = mmc.mmc_net_create(ctx, ws)
    mmc.mmc_net_set_precision(ctx, h, mmc.MMC_BF16)
    B = 21
    xin = _batch_canon(5, B)
    x = mmc.new_field(ctx, B, mmc.MMC_F32)
    y = mmc.new_field(ctx, B, mmc.MMC_F32)
    mmc.mmc_pack(ctx, _to_rows(xin), B, mmc.MMC_F32, x)
    xr = mmc.mmc_unpack(ctx, x, B, mmc.MMC_F32, 192)
    mmc.mmc_net_apply(ctx, h, x, y, B)
    got = mmc.mmc_unpack(ctx, y, B, mmc.MMC_F32, 192)
    worst = 0.0
    for j in range(B):
        want = learned.forward(U, ws, xr[j].reshape(SHAPE)).ravel()
        worst = max(worst, np.linalg.norm(got[j] - want) / np.linalg.norm(want))
    assert worst < 4 * BF16_UNIT, worst
    assert worst > 1e-5  # the BF16 path is really taken (FP32 gives ~1e-7)


def test_bf16_network_gradients_and_training(mmc, env):
    """Gradients of the BF16 forward pass against the oracle's FP64 gradients (bound 8 x 2^-8
    normwise: the rounding of weights and stored activations enters the gradient through
    both factors of every weight's sum), and BF16 training lowers the loss."""
    U, ctx = env
    ws = learned.init_weights(8, scale=0.2)
    h = mmc.mmc_net_create(ctx, ws)
    mmc.mmc_net_set_precision(ctx, h, mmc.MMC_BF16)
    B = 16
    e = _batch_canon(11, B)
    t = _batch_canon(12, B)
    ef = mmc.new_field(ctx, B, mmc.MMC_F32)
    tf = mmc.new_field(ctx, B, mmc.MMC_F32)
    mmc.mmc_pack(ctx, _to_rows(e), B, mmc.MMC_F32, ef)
    mmc.mmc_pack(ctx, _to_rows(t), B, mmc.MMC_F32, tf)
    e32 = mmc.mmc_unpack(ctx, ef, B, mmc.MMC_F32, 192).T.reshape(SHAPE + (B,))
    t32 = mmc.mmc_unpack(ctx, tf, B, mmc.MMC_F32, 192).T.reshape(SHAPE + (B,))
    L_ref, g_ref = learned.loss_and_grad(U, ws, e32, t32)
    L, g = mmc.mmc_net_loss_grad(ctx, h, ef, tf, B)
    assert abs(L - L_ref) < 8 * BF16_UNIT * abs(L_ref)
    for G, Gr in zip(g, g_ref):
        assert np.linalg.norm(G - Gr) < 8 * BF16_UNIT * np.linalg.norm(Gr)
    h2 = mmc.mmc_net_create(ctx, None, 7)
    mmc.mmc_net_set_precision(ctx, h2, mmc.MMC_BF16)
    _, eta, xs = _solve_pairs(mmc, ctx, 64, 22)
    hist = mmc.mmc_net_train(ctx, h2, eta, xs, 64, 16, 300, 3e-3)
    assert hist[-10:].mean() < 0.5 * hist[:4].mean(), (hist[:4], hist[-10:])
