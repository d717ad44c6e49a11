"""Per-kernel parity: each step of the hot path on the GPU (through the C ABI)
against the oracle's step with the same semantics, FP64.

Tolerances: the GPU and the oracle evaluate the same formula in FP64 with a
different summation order, so per-cell results agree to a few ulps of the
largest term; 1e-13 relative (max norm) leaves room for that and catches any
dropped term, sign or index.
"""
import numpy as np
import pytest

import oracle
import workload
from tests.gpu_common import ctx_fixture, dev, host, nominal

pytestmark = pytest.mark.gpu

SIZES = [4, 8, 16, 34, 48]   # 34: not a multiple of the warp / tile widths


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    c.close()


def _field(n, seed):
    return workload.smooth_periodic_field(n, 1e-6, seed) + 2e-7 * workload.lognormal_delta(n, 1.5, seed + 7)


def _maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n", SIZES)
def test_operator(ctx, n):
    alpha, s, h = nominal()
    phi = _field(n, 1)
    got = host(ctx.step_operator(dev(phi), h, alpha))
    assert _maxrel(got, oracle.operator(phi, h, alpha)) < 1e-13


@pytest.mark.parametrize("n", SIZES)
def test_residual(ctx, n):
    alpha, s, h = nominal()
    phi = _field(n, 2)
    f = s * workload.lognormal_delta(n, 1.0, 3)
    c = 3e-11
    got = host(ctx.step_residual(dev(phi), dev(f), c, h, alpha))
    ref = oracle.residual(phi, f, c, h, alpha)
    assert _maxrel(got, ref) < 1e-13


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("scale", [1.0, 30.0])
def test_sweep(ctx, n, scale):
    alpha, s, h = nominal()
    phi = _field(n, 4)
    f = s * scale * workload.lognormal_delta(n, 1.0, 5)
    c = 1e-10
    got = host(ctx.step_sweep(dev(phi), dev(f), c, h, alpha))
    ref = oracle.sweep(phi, f, c, h, alpha)
    assert _maxrel(got, ref) < 1e-13


def test_sweep_repeated_matches(ctx):
    """Ten sweeps in a row stay on the oracle's trajectory."""
    alpha, s, h = nominal()
    n = 16
    phi = _field(n, 6)
    f = s * workload.lognormal_delta(n, 1.0, 8)
    g, r = dev(phi), phi
    for _ in range(10):
        g = ctx.step_sweep(g, dev(f), 0.0, h, alpha)
        r = oracle.sweep(r, f, 0.0, h, alpha)
    assert _maxrel(host(g), r) < 1e-12


@pytest.mark.parametrize("n", [4, 8, 16, 34, 48])
def test_restrict(ctx, n):
    x = _field(n, 9)
    got = host(ctx.step_restrict(dev(x)))
    assert _maxrel(got, oracle.restrict(x)) < 1e-15


@pytest.mark.parametrize("nc", [2, 4, 8, 17, 24])
def test_prolong_add(ctx, nc):
    c = _field(nc, 10)
    f = _field(2 * nc, 11)
    got = host(ctx.step_prolong_add(dev(c), dev(f)))
    assert _maxrel(got, oracle.prolong_add(c, f)) < 1e-14


@pytest.mark.parametrize("n", [8, 16, 34])
def test_force_periodic(ctx, n):
    h = 0.37
    phi = _field(n, 12)
    got = host(ctx.force(dev(phi), h))
    assert _maxrel(got, oracle.force(phi, h)) < 1e-13


@pytest.mark.parametrize("dims,g", [((10, 12, 14), 1), ((9, 8, 7), 2), ((66, 66, 66), 1)])
def test_force_box(ctx, dims, g):
    h = 0.25
    rng = np.random.default_rng(1)
    phi = rng.standard_normal(dims)
    got = host(ctx.force(dev(phi), h, ghost=g, periodic=False))
    assert _maxrel(got, oracle.force(phi, h, ghost=g, periodic=False)) < 1e-14


@pytest.mark.parametrize("nc,o,pn,g", [
    (16, (0, 0, 0), (16, 16, 16), 0),
    (16, (3, 5, 7), (4, 6, 8), 1),
    (16, (14, 15, 0), (5, 3, 4), 1),      # wraps across the periodic boundary
    (12, (11, 0, 6), (12, 2, 3), 2),
    (32, (20, 9, 31), (8, 8, 8), 1),
])
def test_refine_interpolate(ctx, nc, o, pn, g):
    phic = _field(nc, 13)
    got = host(ctx.refine_interpolate(dev(phic), o, pn, g))
    assert _maxrel(got, oracle.refine_interpolate(phic, o, pn, g)) < 1e-15


# ---------------------------------------------------------------- fused and FP32 sweeps

FUSED_SIZES = [4, 8, 16, 32, 34, 48, 64, 80]   # 34, 48, 80: ragged tiles (tile 16 x 32)


@pytest.mark.parametrize("n", FUSED_SIZES)
def test_sweep_fused_fp64(ctx, n):
    """The fused plane-marching kernel is the same snapshot red-black sweep."""
    alpha, s, h = nominal()
    phi = _field(n, 21)
    f = s * 10.0 * workload.lognormal_delta(n, 1.5, 22)
    c = 2e-10
    got = host(ctx.step_sweep_fused(dev(phi), dev(f), c, h, alpha))
    ref = oracle.sweep(phi, f, c, h, alpha)
    assert _maxrel(got, ref) < 1e-13


def _f32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("n", [8, 16, 34, 64])
@pytest.mark.parametrize("fused", [False, True])
def test_sweep_fp32_plain(ctx, n, fused):
    """Without a base the FP32 sweep is the oracle's sweep to FP32 rounding."""
    alpha, s, h = nominal()
    phi = _field(n, 23)
    f = s * 5.0 * workload.lognormal_delta(n, 1.0, 24)
    c = 1e-10
    got = host(ctx.step_sweep_f32(_f32(phi), _f32(f), c, h, alpha, fused=fused)).astype(np.float64)
    ref = oracle.sweep(phi, f, c, h, alpha)
    # phi - h^2 L / 6: the FP32 error is a few ulps of phi
    assert np.abs(got - ref).max() < 2e-6 * np.abs(ref).max()


def _base_field(n, seed, rough):
    """A physical base: the linear (alpha = 0) potential of s delta, for which
    1 + (4 alpha / 3) L_B = 1 + (4/3) eps delta stays positive (the physical branch)."""
    from tests import _pins
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(n, 1.0 + 0.5 * rough, seed)
    B = _pins.fft_poisson(s * delta, h)
    beta = 1 + 4 * alpha / 3 * _pins_lap(B, h)
    assert beta.min() > 0.2, beta.min()
    return B


def _pins_lap(phi, h):
    out = -6.0 * phi
    for a in range(3):
        out += np.roll(phi, 1, axis=a) + np.roll(phi, -1, axis=a)
    return out / h ** 2


@pytest.mark.parametrize("n", [8, 34, 64])
@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("rough", [0.0, 1.0])
def test_sweep_fp32_correction_form(ctx, n, fused, rough):
    """With a base B, the FP32 sweep relaxes e in op(B + e) - op(B) = f + c: it must
    equal the oracle's FP64 sweep of u = B + e with right-hand side op(B) + f, minus B."""
    alpha, s, h = nominal()
    B = _base_field(n, 25, rough)
    e = 1e-3 * B * (1.0 + 0.1 * workload.lognormal_delta(n, 1.0, 26))
    rhs = 1e-3 * s * 5.0 * workload.lognormal_delta(n, 1.0, 27)
    c = 3e-13
    got = host(ctx.step_sweep_f32(_f32(e), _f32(rhs), c, h, alpha, base=_f32(B),
                                  fused=fused)).astype(np.float64)
    Bq = np.asarray(B, dtype=np.float32).astype(np.float64)   # the base the kernel sees
    eq = np.asarray(e, dtype=np.float32).astype(np.float64)
    fq = np.asarray(rhs, dtype=np.float32).astype(np.float64)
    u = oracle.sweep(Bq + eq, oracle.operator(Bq, h, alpha) + fq, c, h, alpha)
    ref = u - Bq
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("n", [32, 48, 64, 96])
def test_fused_matches_two_pass_fp32(ctx, n):
    alpha, s, h = nominal()
    B = _base_field(n, 28, 1.0)
    e = 1e-2 * B * (1.0 + 0.1 * workload.lognormal_delta(n, 1.0, 29))
    rhs = 1e-2 * s * workload.lognormal_delta(n, 1.0, 30)
    a = host(ctx.step_sweep_f32(_f32(e), _f32(rhs), 0.0, h, alpha, base=_f32(B), fused=False))
    b = host(ctx.step_sweep_f32(_f32(e), _f32(rhs), 0.0, h, alpha, base=_f32(B), fused=True))
    assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()


@pytest.mark.parametrize("n", [32, 64, 96, 160])
@pytest.mark.parametrize("rough", [0.0, 1.0])
def test_march_equals_fused_fp32(ctx, n, rough):
    """The column-march FP32 sweep applies the same update to the same operands in the same
    order as the gather-based fused and two-pass kernels: equal to the bit (fused), and to
    FP32 rounding (two-pass); and it is the oracle's sweep of B + e (correction form)."""
    alpha, s, h = nominal()
    B = _base_field(n, 31, rough)
    e = 1e-2 * B * (1.0 + 0.1 * workload.lognormal_delta(n, 1.0, 32))
    rhs = 1e-2 * s * workload.lognormal_delta(n, 1.0, 33)
    c = 2e-12
    args = (_f32(e), _f32(rhs), c, h, alpha)
    m = host(ctx.step_sweep_f32(*args, base=_f32(B), fused=2))
    f1 = host(ctx.step_sweep_f32(*args, base=_f32(B), fused=1))
    f0 = host(ctx.step_sweep_f32(*args, base=_f32(B), fused=0))
    assert np.array_equal(m, f1), (float(np.abs(m - f1).max() / np.abs(f1).max()),
                                   int((m != f1).sum()), np.argwhere(m != f1)[:8].tolist())
    assert np.abs(m - f0).max() <= 1e-6 * np.abs(f0).max()
    if n <= 64:
        Bq = np.asarray(B, dtype=np.float32).astype(np.float64)
        eq = np.asarray(e, dtype=np.float32).astype(np.float64)
        fq = np.asarray(rhs, dtype=np.float32).astype(np.float64)
        u = oracle.sweep(Bq + eq, oracle.operator(Bq, h, alpha) + fq, c, h, alpha)
        ref = u - Bq
        assert np.abs(m.astype(np.float64) - ref).max() < 1e-4 * np.abs(ref).max()


def test_march_refuses_sizes_it_does_not_tile(ctx):
    import torch
    import paper_1511_08200_gb300 as mg
    alpha, s, h = nominal()
    for n in (16, 48):
        z = torch.zeros((n,) * 3, dtype=torch.float32, device="cuda")
        with pytest.raises(mg.MG5Error) as e:
            ctx.step_sweep_f32(z, z, 0.0, h, alpha, base=z, fused=2)
        assert e.value.code == mg.E_ARG
    z = torch.zeros((32,) * 3, dtype=torch.float32, device="cuda")
    with pytest.raises(mg.MG5Error):
        ctx.step_sweep_f32(z, z, 0.0, h, alpha, fused=2)   # no base


@pytest.mark.parametrize("n", [32, 64, 96, 128, 160])
def test_resid_restrict_march_equals_gather_fp32(ctx, n):
    """The column-march residual + restriction of the FP32 correction equation gives the gather
    kernel's coarse e and coarse r to the bit, the residual statistics to FP32 summation order;
    and the coarse residual is the 8-child mean of the oracle's residual of B + e.  At 128 and
    160 the CTAs' shares of (tile, plane pair) units cross tile boundaries."""
    alpha, s, h = nominal()
    B = _base_field(n, 34, 1.0)
    e = 1e-2 * B * (1.0 + 0.1 * workload.lognormal_delta(n, 1.0, 35))
    rhs = 1e-2 * s * workload.lognormal_delta(n, 1.0, 36)
    c = 3e-12
    args = (_f32(e), _f32(rhs), _f32(B), c, h, alpha)
    ec0, rc0, st0 = ctx.step_resid_restrict_f32(*args, march=False)
    ec1, rc1, st1 = ctx.step_resid_restrict_f32(*args, march=True)
    assert np.array_equal(host(ec0), host(ec1)) and np.array_equal(host(rc0), host(rc1))
    assert st1[0] == pytest.approx(st0[0], rel=1e-5, abs=1e-6 * st0[1] / n ** 1.5)
    assert st1[1] == pytest.approx(st0[1], rel=1e-5)
    Bq = np.asarray(B, dtype=np.float32).astype(np.float64)
    eq = np.asarray(e, dtype=np.float32).astype(np.float64)
    fq = np.asarray(rhs, dtype=np.float32).astype(np.float64)
    r = oracle.residual(Bq + eq, oracle.operator(Bq, h, alpha) + fq, c, h, alpha)
    rref = oracle.restrict(r)
    got = host(rc1).astype(np.float64)
    assert np.abs(got - rref).max() <= 2e-3 * np.abs(rref).max()
    assert np.abs(host(ec1) - oracle.restrict(eq)).max() <= 1e-6 * np.abs(eq).max()
