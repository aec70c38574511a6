"""GPU parity of the core kernels against the oracle, through the C ABI:
Z(4) noise (bit-exact), layout round trips, M and M^+ (Sec. 1's Wilson-Dirac
matrix) in FP64 / FP32 / BF16 storage, GMRES polynomials (Sec. 3) and the
double polynomial (Sec. 5).

Tolerances: FP64 1e-12 relative; FP32 1e-5 relative; BF16 storage: the
input is fed exactly (Z(4) entries are representable) or compared against
the oracle applied to the BF16-rounded input, so the only error left is the
FP32 arithmetic plus one rounding of the output to BF16's 8-bit significand:
normwise relative error <= 2^-8 (plus 1e-6 for the FP32 arithmetic)."""
import numpy as np
import pytest

import synth
from oracle import krylov, noise, wilson

pytestmark = pytest.mark.gpu

BF16_BOUND = 2.0 ** -8 + 1e-6


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


def _shape(dims):
    return (dims[3], dims[2], dims[1], dims[0], 4, 3)


def _bf16_round(a):
    """Round complex128 values to bfloat16 (round to nearest even) on both parts."""
    def r(x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        b = x.view(np.uint32).astype(np.uint64)
        b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
        return b.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(a.real) + 1j * r(a.imag)


class Lattice:
    def __init__(self, mmc, dims, eps=0.5, kappa=0.13, tap=1, seed=11):
        self.dims, self.kappa, self.tap = dims, kappa, tap
        self.U = synth.random_gauge(dims, eps, seed)
        self.V = int(np.prod(dims))
        self.shape = _shape(dims)
        self.ctx = mmc.mmc_create(dims, seed=5, device=0)
        mmc.mmc_load_gauge(self.ctx, self.U, kappa, tap)

    def op(self, v):
        return wilson.apply_M(self.U, self.kappa, v.reshape(self.shape), bool(self.tap)).ravel()

    def opdag(self, v):
        return wilson.apply_Mdag(self.U, self.kappa, v.reshape(self.shape), bool(self.tap)).ravel()


@pytest.fixture(scope="module")
def lat(mmc):
    L = Lattice(mmc, (6, 4, 2, 6))  # V = 288: several CTAs and a ragged tail
    yield L
    mmc.mmc_destroy(L.ctx)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("nrhs", [1, 3, 16, 21])
def test_noise_bit_exact(mmc, lat, prec, nrhs):
    f = mmc.new_field(lat.ctx, nrhs, prec)
    mmc.mmc_noise(lat.ctx, 3, 10, mmc.MMC_TAG_NOISE, nrhs, prec, f)
    got = mmc.mmc_unpack(lat.ctx, f, nrhs, prec, lat.V)
    for j in range(nrhs):
        want = noise.z4_noise(lat.dims, 5, 10 + j, 3).ravel()
        assert np.array_equal(got[j], want)


@pytest.mark.parametrize("prec", [0, 1])
def test_pack_roundtrip(mmc, lat, prec):
    x = synth.random_spinor(lat.dims, 1, 5).transpose(6, 0, 1, 2, 3, 4, 5).reshape(5, -1)
    f = mmc.new_field(lat.ctx, 5, prec)
    mmc.mmc_pack(lat.ctx, x, 5, prec, f)
    got = mmc.mmc_unpack(lat.ctx, f, 5, prec, lat.V)
    tol = 0 if prec == 0 else 1e-7
    assert np.abs(got - x).max() <= tol * np.abs(x).max() + 0.0


@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("prec,nrhs", [(0, 1), (0, 3), (0, 21), (1, 1), (1, 5), (1, 16), (1, 21), (2, 2), (2, 19)])
def test_apply_M(mmc, lat, prec, nrhs, dagger):
    rng_x = synth.random_spinor(lat.dims, 7, nrhs).transpose(6, 0, 1, 2, 3, 4, 5).reshape(nrhs, -1)
    x = mmc.new_field(lat.ctx, nrhs, prec)
    y = mmc.new_field(lat.ctx, nrhs, prec)
    mmc.mmc_pack(lat.ctx, rng_x, nrhs, prec, x)
    xin = mmc.mmc_unpack(lat.ctx, x, nrhs, prec, lat.V)  # what the kernel actually sees
    mmc.mmc_apply_M(lat.ctx, x, y, nrhs, prec, dagger)
    got = mmc.mmc_unpack(lat.ctx, y, nrhs, prec, lat.V)
    tol = {0: 1e-12, 1: 1e-5, 2: BF16_BOUND}[prec]
    f = lat.opdag if dagger else lat.op
    for j in range(nrhs):
        want = f(xin[j])
        err = np.linalg.norm(got[j] - want) / np.linalg.norm(want)
        assert err < tol, (j, err)


def test_apply_M_free_field_periodic(mmc):
    """Periodic time and the unit gauge: plane waves are eigenvectors (closed form)."""
    dims = (4, 2, 2, 4)
    ctx = mmc.mmc_create(dims, 0, 0)
    try:
        kappa = 0.1
        mmc.mmc_load_gauge(ctx, synth.unit_gauge(dims), kappa, 0)
        t, z, y, xg = np.meshgrid(*[np.arange(d) for d in (4, 2, 2, 4)], indexing="ij")
        p = (2 * np.pi / 4, np.pi, 0.0, 2 * np.pi * 3 / 4)
        phase = np.exp(1j * (p[0] * xg + p[1] * y + p[2] * z + p[3] * t))
        from oracle import gamma
        S = sum(gamma.GAMMA[m] * np.sin(p[m]) for m in range(4))
        w, chis = np.linalg.eigh(S)
        psi = (phase[..., None, None] * chis[:, 0][:, None] * np.array([1.0, 2.0, -1.0])[None, :]).ravel()
        lam = 1 - 2 * kappa * sum(np.cos(q) for q in p) + 2j * kappa * w[0]
        f = mmc.new_field(ctx, 1, 0)
        g = mmc.new_field(ctx, 1, 0)
        mmc.mmc_pack(ctx, psi[None, :], 1, 0, f)
        mmc.mmc_apply_M(ctx, f, g, 1, 0, 0)
        got = mmc.mmc_unpack(ctx, g, 1, 0, 64)[0]
        assert np.abs(got - lam * psi).max() < 1e-13
    finally:
        mmc.mmc_destroy(ctx)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_apply_poly_oracle_roots(mmc, lat, prec, tol):
    """p(M) with the oracle's Ritz values fed to the GPU (Sec. 3 recurrence)."""
    b = noise.z4_noise(lat.dims, 5, 0, 0, noise.TAG_GMRES).ravel()
    theta = krylov.gmres_poly_roots(lat.op, b, 12)
    h = mmc.mmc_poly_from_roots(lat.ctx, theta)
    assert mmc.mmc_poly_degree(lat.ctx, h) == 11
    nrhs = 5
    x = mmc.new_field(lat.ctx, nrhs, prec)
    y = mmc.new_field(lat.ctx, nrhs, prec)
    mmc.mmc_noise(lat.ctx, 2, 0, mmc.MMC_TAG_NOISE, nrhs, prec, x)
    mmc.mmc_apply_poly(lat.ctx, h, x, y, nrhs, prec)
    got = mmc.mmc_unpack(lat.ctx, y, nrhs, prec, lat.V)
    for j in range(nrhs):
        eta = noise.z4_noise(lat.dims, 5, j, 2).ravel()
        want = krylov.apply_poly(lat.op, theta, eta)
        assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < tol


def test_gmres_poly_ritz_values(mmc, lat):
    """GPU CGS2 Arnoldi + host harmonic Ritz/Leja vs the oracle (MGS) for small m."""
    b = noise.z4_noise(lat.dims, 5, 0, 0, noise.TAG_GMRES).ravel()
    for m in (1, 4, 10):
        h, theta = mmc.mmc_gmres_poly(lat.ctx, m)
        ref = krylov.gmres_poly_roots(lat.op, b, m)
        assert np.abs(theta - ref).max() < 1e-9 * np.abs(ref).max()
        # the residual-polynomial identity on the GPU's own roots
        x = synth.random_spinor(lat.dims, 3).ravel()
        lhs = x - lat.op(krylov.apply_poly(lat.op, theta, x))
        assert np.linalg.norm(lhs - krylov.apply_pi(lat.op, theta, x)) < 1e-12 * np.linalg.norm(x)


def test_double_poly(mmc, lat):
    """p_double = p_in(M) p_out(phi_in(M)) (Sec. 5): Ritz values and application in FP64."""
    b = noise.z4_noise(lat.dims, 5, 0, 0, noise.TAG_GMRES).ravel()
    h_in, th_in = mmc.mmc_gmres_poly(lat.ctx, 5)
    h_out, th_out = mmc.mmc_gmres_poly(lat.ctx, 4, h_in)
    ref_in, ref_out = krylov.double_poly_roots(lat.op, b, 5, 4)
    assert np.abs(th_in - ref_in).max() < 1e-9 * np.abs(ref_in).max()
    assert np.abs(th_out - ref_out).max() < 1e-8 * np.abs(ref_out).max()
    h = mmc.mmc_poly_double(lat.ctx, h_in, h_out)
    assert mmc.mmc_poly_degree(lat.ctx, h) == 19
    a = np.array([0.5 + 0.1j, 1.3 - 0.2j])
    assert np.allclose(mmc.mmc_poly_eval(lat.ctx, h, a), krylov.double_scalar(th_in, th_out, a), rtol=1e-13)
    nrhs = 3
    x = mmc.new_field(lat.ctx, nrhs, 0)
    y = mmc.new_field(lat.ctx, nrhs, 0)
    mmc.mmc_noise(lat.ctx, 4, 0, mmc.MMC_TAG_NOISE, nrhs, 0, x)
    mmc.mmc_apply_poly(lat.ctx, h, x, y, nrhs, 0)
    got = mmc.mmc_unpack(lat.ctx, y, nrhs, 0, lat.V)
    for j in range(nrhs):
        eta = noise.z4_noise(lat.dims, 5, j, 4).ravel()
        want = krylov.apply_double(lat.op, th_in, th_out, eta)
        assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < 1e-12


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("ver,rpt,minb", [(1, 1, 1), (1, 2, 3), (2, 1, 4), (2, 1, 6), (2, 2, 3),
                                          (3, 1, 300), (3, 1, 302), (3, 2, 300),
                                          (4, 1, 4), (4, 1, 3), (4, 1, 5), (4, 1, 6), (4, 1, 401), (5, 1, 303),
                                          (5, 1, 304),
                                          (5, 1, 306)])
@pytest.mark.parametrize("nrhs", [5, 21])
def test_step_kernel_variants(mmc, lat, prec, ver, rpt, minb, nrhs):
    """Every step-kernel version (generic, compile-time rhs block, rows staged by bulk
    copies with the deepest and the shallowest ring, one or two rhs per lane, the
    persistent pipelined form with either register cap, with its links staged in shared
    memory or rebuilt from two rows, and with evict-first stores, the
    form with operands staged by asynchronous copies at each pipeline depth), lane widths
    and register caps give M x, and M^+ x for the staged and persistent forms."""
    mmc.mmc_set_step_variant(lat.ctx, prec, rpt, 100 + ver, 0)
    mmc.mmc_set_step_variant(lat.ctx, prec, 0, minb, 0)
    try:
        if ver in (3, 4, 5):
            rng_x = synth.random_spinor(lat.dims, 10, nrhs).transpose(6, 0, 1, 2, 3, 4, 5).reshape(nrhs, -1)
            x = mmc.new_field(lat.ctx, nrhs, prec)
            y = mmc.new_field(lat.ctx, nrhs, prec)
            mmc.mmc_pack(lat.ctx, rng_x, nrhs, prec, x)
            xin = mmc.mmc_unpack(lat.ctx, x, nrhs, prec, lat.V)
            mmc.mmc_apply_M(lat.ctx, x, y, nrhs, prec, 1)
            got = mmc.mmc_unpack(lat.ctx, y, nrhs, prec, lat.V)
            tol = 1e-5 if prec == 1 else BF16_BOUND
            for j in range(nrhs):
                want = lat.opdag(xin[j])
                assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < tol
        rng_x = synth.random_spinor(lat.dims, 9, nrhs).transpose(6, 0, 1, 2, 3, 4, 5).reshape(nrhs, -1)
        x = mmc.new_field(lat.ctx, nrhs, prec)
        y = mmc.new_field(lat.ctx, nrhs, prec)
        mmc.mmc_pack(lat.ctx, rng_x, nrhs, prec, x)
        xin = mmc.mmc_unpack(lat.ctx, x, nrhs, prec, lat.V)
        mmc.mmc_apply_M(lat.ctx, x, y, nrhs, prec, 0)
        got = mmc.mmc_unpack(lat.ctx, y, nrhs, prec, lat.V)
        tol = 1e-5 if prec == 1 else BF16_BOUND
        for j in range(nrhs):
            want = lat.op(xin[j])
            assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < tol
    finally:
        mmc.mmc_set_step_variant(lat.ctx, prec, 1, 102, 0)
        mmc.mmc_set_step_variant(lat.ctx, prec, 0, 4, 0)
        mmc.mmc_set_step_variant(lat.ctx, prec, 0, 300, 0)
        mmc.mmc_set_step_variant(lat.ctx, prec, 0, 400, 0)


@pytest.mark.parametrize("prec", [1, 2])
def test_step_variant_per_rhs_class(mmc, lat, prec):
    """The 8-rhs class and the 16-rhs class keep separate variants: a batch of each runs
    with its own kernel form and both give M x; out-of-range settings are rejected."""
    staged = {"version": 3, "rpt": 2, "minb": 1, "spc": 64, "blocked": 0, "ns": 0}
    plain = {"version": 2, "rpt": 1, "minb": 4, "spc": 32, "blocked": 0, "ns": 0}
    try:
        mmc.mmc_set_step_variant_class(lat.ctx, prec, 0, staged)
        mmc.mmc_set_step_variant_class(lat.ctx, prec, 1, plain)
        for nrhs in (6, 19):
            rng_x = synth.random_spinor(lat.dims, 12, nrhs).transpose(6, 0, 1, 2, 3, 4, 5).reshape(nrhs, -1)
            x = mmc.new_field(lat.ctx, nrhs, prec)
            y = mmc.new_field(lat.ctx, nrhs, prec)
            mmc.mmc_pack(lat.ctx, rng_x, nrhs, prec, x)
            xin = mmc.mmc_unpack(lat.ctx, x, nrhs, prec, lat.V)
            mmc.mmc_apply_M(lat.ctx, x, y, nrhs, prec, 0)
            got = mmc.mmc_unpack(lat.ctx, y, nrhs, prec, lat.V)
            tol = 1e-5 if prec == 1 else BF16_BOUND
            for j in range(nrhs):
                want = lat.op(xin[j])
                assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < tol
        for bad in ({"rpt": 3}, {"version": 6}, {"ns": 7}, {"spc": 48}, {"blocked": 3}):
            with pytest.raises(mmc.MMCError):
                mmc.mmc_set_step_variant_class(lat.ctx, prec, 0, dict(staged, **bad))
    finally:
        mmc.mmc_set_step_variant(lat.ctx, prec, 1, 102, 0)
        mmc.mmc_set_step_variant(lat.ctx, prec, 0, 4, 0)
        mmc.mmc_set_step_variant(lat.ctx, prec, 0, 300, 0)


@pytest.mark.parametrize("prec", [1, 2])
def test_rebuilt_link_rows_need_special_unitary_links(mmc, prec):
    """The form that rebuilds each link's third row (minb 6, 8- and 16-rhs blocks) on a
    gauge field with one link that is not special unitary: the library detects it at load
    time and runs the form that loads whole links, so M x still matches the oracle; on the
    special unitary field (antiperiodic time, the negated boundary links included) the
    rebuilt rows match it too."""
    dims = (4, 4, 2, 6)
    shape = (6, 2, 4, 4, 4, 3)
    U = synth.random_gauge(dims, 0.5, 4)
    bad = U.copy()
    bad[3, 5, 1, 2, 3] *= 1.25  # one time link at t = Lt - 1, scaled
    for field, nrhs in ((U, 6), (bad, 6), (U, 21), (bad, 21)):
        ctx = mmc.mmc_create(dims, seed=3, device=0)
        try:
            mmc.mmc_load_gauge(ctx, field, 0.13, 1)
            for rc in (0, 1):
                mmc.mmc_set_step_variant_class(ctx, prec, rc, {"version": 4, "rpt": 1, "minb": 6, "spc": 64,
                                                               "blocked": 0, "ns": 0})
            xs = synth.random_spinor(dims, 12, nrhs).transpose(6, 0, 1, 2, 3, 4, 5).reshape(nrhs, -1)
            x = mmc.new_field(ctx, nrhs, prec)
            y = mmc.new_field(ctx, nrhs, prec)
            mmc.mmc_pack(ctx, xs, nrhs, prec, x)
            xin = mmc.mmc_unpack(ctx, x, nrhs, prec, int(np.prod(dims)))
            tol = 1e-5 if prec == 1 else BF16_BOUND
            for dag in (0, 1):
                mmc.mmc_apply_M(ctx, x, y, nrhs, prec, dag)
                got = mmc.mmc_unpack(ctx, y, nrhs, prec, int(np.prod(dims)))
                for j in range(nrhs):
                    v = xin[j].reshape(shape)
                    want = (wilson.apply_Mdag(field, 0.13, v) if dag else wilson.apply_M(field, 0.13, v)).ravel()
                    assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < tol, (dag, j)
        finally:
            mmc.mmc_destroy(ctx)


@pytest.mark.parametrize("prec,ver", [(0, 1), (1, 2), (2, 2), (1, 4), (2, 4), (1, 5), (2, 5)])
def test_chain_graphs_replay_identical(mmc, lat, prec, ver):
    """A step chain replayed from its captured CUDA graph gives the same bits as the
    chain launched degree by degree, for p(M) X and for the level samples (whose
    partial sums the persistent form accumulates per CTA over its work items)."""
    import torch
    mmc.mmc_set_step_variant(lat.ctx, prec, 1 if ver >= 4 else 0, 100 + ver, 0)
    theta = mmc.mmc_leja_order(1.0 + 0.7 * np.exp(2j * np.pi * (np.arange(6) + 0.5) / 6))
    h = mmc.mmc_poly_from_roots(lat.ctx, theta)
    h2 = mmc.mmc_poly_from_roots(lat.ctx, theta[:3])
    nrhs = 19
    x = mmc.new_field(lat.ctx, nrhs, prec)
    mmc.mmc_noise(lat.ctx, 2, 0, mmc.MMC_TAG_NOISE, nrhs, prec, x)
    outs, samples = [], []
    y = mmc.new_field(lat.ctx, nrhs, prec)  # the same operands: the second call replays the graph
    try:
        for on in (True, True, False):  # capture, replay, direct
            mmc.mmc_set_graphs(lat.ctx, on)
            mmc.mmc_profile(lat.ctx, 1)
            y.zero_()
            mmc.mmc_apply_poly(lat.ctx, h, x, y, nrhs, prec)
            outs.append(y.clone())
            st = mmc.mmc_trace_level(lat.ctx, h, h2, mmc.MMC_THETA_ONE, 0, nrhs, 40, 3, prec)
            samples.append(st["samples"])
            replays = mmc.mmc_profile_read(lat.ctx)["graph_launches"]
            mmc.mmc_profile(lat.ctx, 0)
            assert (replays > 0) == on, (on, replays, mmc.mmc_graph_note(lat.ctx))
        torch.cuda.synchronize()
        for k in range(1, 3):
            assert torch.equal(outs[0], outs[k]), k
            assert np.array_equal(samples[0], samples[k]), k
    finally:
        mmc.mmc_set_graphs(lat.ctx, True)
        if prec != 0:
            mmc.mmc_set_step_variant(lat.ctx, prec, 2, 102, 0)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_rhs_block_max_8(mmc, prec):
    """A context whose blocked layout holds at most 8 rhs per block gives the same M x
    (several blocks and a ragged last one) and the same p(M) x as the oracle."""
    dims = (6, 4, 2, 6)
    U = synth.random_gauge(dims, 0.5, 11)
    ctx = mmc.mmc_create(dims, seed=5, device=0)
    try:
        mmc.mmc_set_rhs_block_max(ctx, 8)
        mmc.mmc_load_gauge(ctx, U, 0.13, 1)
        with pytest.raises(mmc.MMCError):
            mmc.mmc_set_rhs_block_max(ctx, 4)
        V = int(np.prod(dims))
        nrhs = 21
        assert mmc.mmc_field_bytes(ctx, nrhs, prec) == 24 * V * 12 * (16, 8, 4)[prec]
        x = mmc.new_field(ctx, nrhs, prec)
        y = mmc.new_field(ctx, nrhs, prec)
        mmc.mmc_noise(ctx, 2, 0, mmc.MMC_TAG_NOISE, nrhs, prec, x)
        mmc.mmc_apply_M(ctx, x, y, nrhs, prec, 0)
        got = mmc.mmc_unpack(ctx, y, nrhs, prec, V)
        theta = np.array([1.0 + 0.5j, 1.0 - 0.5j, 0.6 + 0.0j])
        h = mmc.mmc_poly_from_roots(ctx, theta)
        mmc.mmc_apply_poly(ctx, h, x, y, nrhs, prec)
        gotp = mmc.mmc_unpack(ctx, y, nrhs, prec, V)
        shape = _shape(dims)
        op = lambda v: wilson.apply_M(U, 0.13, v.reshape(shape), True).ravel()
        tol = (1e-12, 1e-5, BF16_BOUND)[prec]
        for j in (0, 7, 8, 20):
            eta = noise.z4_noise(dims, 5, j, 2).ravel()
            want = op(eta)
            assert np.linalg.norm(got[j] - want) / np.linalg.norm(want) < tol, j
            wantp = krylov.apply_poly(op, theta, eta)
            assert np.linalg.norm(gotp[j] - wantp) / np.linalg.norm(wantp) < 3 * tol, j
    finally:
        mmc.mmc_destroy(ctx)
