"""Position-dependent truncation (Sec. 3.3) through the C ABI against the oracle:
the parent-force mask (bit-exact: both sides decide |F5| > theta |F_GR| in FP64 with
every product and sum rounded as written) and the masked patch relaxation (the same
discrete solution on the masked cells, the other cells bit-identical to the entry box).

Bars: the relaxed phi within relative L2 1e-10 (1e-9 at 64^3, tol 1e-11) of the
oracle's Gauss-Seidel relaxation of the same masked problem, as for the unmasked patch."""
import numpy as np
import pytest

import oracle
import workload
from tests.gpu_common import ctx_fixture, dev, host, nominal, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    c.close()


def _mg():
    import paper_1511_08200_gb300 as mg
    return mg


def _u8(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def _parent_forces(coarse, h, tol=1e-12):
    """Oracle fifth-force and GR solves on the parent grid and their gradients (Sec. 3.2:
    F5 = grad(phi)/2; Psi_GR solves the alpha = 0 equation with source (3 beta/2) s delta)."""
    beta, alpha, s = oracle.ndgp_coefficients(1.0, 0.3, 1.0)
    phi, info = oracle.solve(coarse, alpha, s, h, tol=tol)
    psi, _ = oracle.solve(coarse, 0.0, 1.5 * beta * s, h, tol=tol)
    return phi, info, oracle.force(phi, h), oracle.force(psi, h), (beta, alpha, s)


def _ratio_quantile(gphi, ggr, q, o=None, pn=None):
    """q-quantile of the parent F5/F_GR, over the whole grid or the parents [o, o + pn)."""
    r = 0.5 * np.sqrt((gphi ** 2).sum(0)) / np.sqrt((ggr ** 2).sum(0))
    if o is not None:
        n = r.shape[0]
        r = r[np.ix_(*[(o[a] + np.arange(pn[a])) % n for a in range(3)])]
    return float(np.quantile(r, q))


@pytest.mark.parametrize("o,pn", [((3, 5, 7), (8, 8, 8)), ((28, 30, 1), (6, 4, 10)),
                                  ((0, 0, 0), (32, 32, 32))])
def test_parent_force_mask_matches_oracle(ctx, o, pn):
    _, _, h = nominal()
    coarse = workload.lognormal_delta(32, 1.5, 21)
    _, _, gphi, ggr, _ = _parent_forces(coarse, h)
    for q in (0.0, 0.3, 0.7, 1.0):
        theta = _ratio_quantile(gphi, ggr, q)
        want = oracle.parent_force_mask(gphi, ggr, o, pn, theta)
        got, count = ctx.parent_force_mask(dev(gphi), dev(ggr), o, pn, theta, count=True)
        got = host(got)
        assert got.shape == want.shape and got.dtype == np.uint8
        assert np.array_equal(got, want)
        assert count == int(want.sum())


@pytest.mark.parametrize("pd,o,pn", [((10, 12, 14), (2, 3, 4), (4, 4, 5)),
                                     ((32, 32, 32), (0, 8, 16), (16, 12, 8))])
def test_parent_force_mask_box_parent_matches_oracle(ctx, pd, o, pn):
    """A refinement's interior as the parent (no wrap), gradients as mg5_force writes them."""
    rng = np.random.default_rng(sum(pd))
    gphi = 0.24 * rng.standard_normal((3,) + pd)
    ggr = rng.standard_normal((3,) + pd)
    for theta in (0.0, 0.1, 0.12, 0.3):
        want = oracle.parent_force_mask(gphi, ggr, o, pn, theta, periodic=False)
        got, count = ctx.parent_force_mask(dev(gphi), dev(ggr), o, pn, theta, periodic=False,
                                           count=True)
        assert np.array_equal(host(got), want) and count == int(want.sum())


def test_parent_force_mask_zero_gravity_and_threshold_zero(ctx):
    n = 8
    gphi = np.zeros((3, n, n, n))
    gphi[1, 2, 3, 4] = 1e-3
    ggr = np.zeros_like(gphi)
    got = host(ctx.parent_force_mask(dev(gphi), dev(ggr), (2, 3, 4), (1, 1, 2), 0.0))
    want = oracle.parent_force_mask(gphi, ggr, (2, 3, 4), (1, 1, 2), 0.0)
    assert np.array_equal(got, want) and got[:, :, :2].all() and not got[:, :, 2:].any()


def _masked_patch(nc=32, pn=8, q=0.5, seed=7):
    """A refinement of the densest pn^3 window of a lognormal parent grid; the mask is the
    parent criterion at the q-quantile of the parent's F5/F_GR."""
    _, _, h = nominal()
    fine = workload.lognormal_delta(2 * nc, 1.5, seed)
    coarse = workload.block_mean(fine, 2)
    o = workload.densest_window(coarse, pn)
    idx = [(2 * o[a] + np.arange(2 * pn)) % (2 * nc) for a in range(3)]
    dpatch = np.ascontiguousarray(fine[np.ix_(*idx)])
    phi, info, gphi, ggr, (beta, alpha, s) = _parent_forces(coarse, h)
    theta = _ratio_quantile(gphi, ggr, q, o, (pn, pn, pn))
    mask = oracle.parent_force_mask(gphi, ggr, o, (pn, pn, pn), theta)
    box = oracle.refine_interpolate(phi, o, (pn, pn, pn), 1)
    return dpatch, mask, box, info.compat_c, alpha, s, h / 2


@pytest.mark.parametrize("q", [0.2, 0.6, 0.95])
def test_relax_patch_masked_matches_oracle(ctx, q):
    mg = _mg()
    dpatch, mask, box, c, alpha, s, hf = _masked_patch(q=q)
    assert 0 < mask.sum() < mask.size
    p = mg.default_params(alpha=alpha, s=s, h=hf, tol=1e-12, max_cycles=200)
    got, info = ctx.relax_patch_masked(dev(dpatch), _u8(mask), p, c, dev(box))
    assert info.status == 0 and info.rel_residual <= 1e-12
    ref, nsw, rel = oracle.relax_patch_masked(dpatch, box, mask, alpha, s, hf, c, tol=1e-12)
    assert rel <= 1e-12
    got = host(got)
    on = np.zeros(box.shape, bool)
    on[1:-1, 1:-1, 1:-1] = mask != 0
    assert rel_l2(got[on], ref[on]) <= 1e-10
    assert np.array_equal(got[~on], box[~on])


def test_relax_patch_masked_all_ones_equals_unmasked(ctx):
    """An all-ones mask runs the unmasked V-cycle."""
    mg = _mg()
    dpatch, mask, box, c, alpha, s, hf = _masked_patch(q=0.5)
    p = mg.default_params(alpha=alpha, s=s, h=hf, tol=1e-11)
    a, ia = ctx.relax_patch(dev(dpatch), p, c, dev(box))
    b, ib = ctx.relax_patch_masked(dev(dpatch), _u8(np.ones_like(mask)), p, c, dev(box))
    # the same iteration; the masked kernels are separate instantiations, so the compiler may
    # round a few products differently (fused or not): equal up to rounding, not bit for bit
    assert ia.cycles == ib.cycles
    assert ib.rel_residual == pytest.approx(ia.rel_residual, rel=1e-4)
    assert rel_l2(host(b), host(a)) <= 1e-13


def test_relax_patch_masked_empty_mask(ctx):
    mg = _mg()
    dpatch, mask, box, c, alpha, s, hf = _masked_patch(q=0.5)
    p = mg.default_params(alpha=alpha, s=s, h=hf, tol=1e-11)
    got, info = ctx.relax_patch_masked(dev(dpatch), _u8(np.zeros_like(mask)), p, c, dev(box))
    assert info.status == 0 and info.cycles == 0
    assert np.array_equal(host(got), box)


@pytest.mark.parametrize("pf,seed", [((12, 16, 20), 31), ((8, 6, 10), 32), ((2, 4, 2), 33)])
def test_relax_patch_masked_ragged_random_parent_mask(ctx, pf, seed):
    """Non-cubic patches (two grids, one grid) with a random mask at parent granularity."""
    mg = _mg()
    alpha, s, h = nominal()
    rng = np.random.default_rng(seed)
    dims = tuple(x + 2 for x in pf)
    hf = h / 2
    box = s * hf * hf * rng.standard_normal(dims)        # phi on the scale s delta h^2
    delta = np.exp(rng.standard_normal(pf)) - 1.0
    par = rng.random(tuple(x // 2 for x in pf)) < 0.5
    par.flat[0] = True
    mask = np.repeat(np.repeat(np.repeat(par, 2, 0), 2, 1), 2, 2).astype(np.uint8)
    c = 0.01 * s
    p = mg.default_params(alpha=alpha, s=s, h=hf, tol=1e-12, max_cycles=200)
    got, info = ctx.relax_patch_masked(dev(delta), _u8(mask), p, c, dev(box))
    assert info.status == 0
    ref, nsw, rel = oracle.relax_patch_masked(delta, box, mask, alpha, s, hf, c, tol=1e-12)
    assert rel <= 1e-12
    got = host(got)
    on = np.zeros(dims, bool)
    on[1:-1, 1:-1, 1:-1] = mask != 0
    assert rel_l2(got[on], ref[on]) <= 1e-10
    assert np.array_equal(got[~on], box[~on])


def test_relax_patch_masked_full_size_64(ctx):
    """The 64^3 patch of the refinement workload (128^3 parent grid), mask at the median
    parent F5/F_GR, against the oracle's masked Gauss-Seidel relaxation, both to 1e-11."""
    mg = _mg()
    beta, alpha, s = oracle.ndgp_coefficients(1.0, 0.3, 1.0)
    coarse, dpatch, o = workload.patch_workload(256, 1.5, 2, 32)
    hc = 250.0 / 128
    phi, info, gphi, ggr, _ = _parent_forces(coarse, hc, tol=1e-13)
    theta = _ratio_quantile(gphi, ggr, 0.5, o, (32, 32, 32))
    mask = oracle.parent_force_mask(gphi, ggr, o, (32, 32, 32), theta)
    gmask = host(ctx.parent_force_mask(dev(gphi), dev(ggr), o, (32, 32, 32), theta))
    assert np.array_equal(gmask, mask) and 0 < mask.sum() < mask.size
    box = oracle.refine_interpolate(phi, o, (32, 32, 32), 1)
    p = mg.default_params(alpha=alpha, s=s, h=hc / 2, tol=1e-11)
    got, pinfo = ctx.relax_patch_masked(dev(dpatch), _u8(mask), p, info.compat_c, dev(box))
    assert pinfo.status == 0 and pinfo.cycles < 40
    ref, nsw, rel = oracle.relax_patch_masked(dpatch, box, mask, alpha, s, hc / 2, info.compat_c,
                                              tol=1e-11)
    assert rel <= 1e-11
    got = host(got)
    on = np.zeros(box.shape, bool)
    on[1:-1, 1:-1, 1:-1] = mask != 0
    assert rel_l2(got[on], ref[on]) <= 1e-9
    assert np.array_equal(got[~on], box[~on])


@pytest.mark.parametrize("frac", [0.002, 0.03, 0.08])
def test_relax_patch_masked_sparse_mask(ctx, frac):
    """Masks of a few percent of the cells (the deep levels of Sec. 3.3's criterion) go through
    masked sweeps first: the same solution as the oracle's masked relaxation, and for the
    sparsest mask without a V-cycle."""
    mg = _mg()
    alpha, s, h = nominal()
    pf = (32, 32, 32)
    rng = np.random.default_rng(int(frac * 1000) + 40)
    hf = h / 2
    dims = tuple(x + 2 for x in pf)
    box = s * hf * hf * rng.standard_normal(dims)
    delta = np.exp(rng.standard_normal(pf)) - 1.0
    par = rng.random(tuple(x // 2 for x in pf)) < frac
    par.flat[int(rng.integers(par.size))] = True
    mask = np.repeat(np.repeat(np.repeat(par, 2, 0), 2, 1), 2, 2).astype(np.uint8)
    c = 0.01 * s
    p = mg.default_params(alpha=alpha, s=s, h=hf, tol=1e-12, max_cycles=200)
    got, info = ctx.relax_patch_masked(dev(delta), _u8(mask), p, c, dev(box))
    assert info.status == 0 and info.rel_residual <= 1e-12
    if frac < 0.01:
        assert info.cycles == 0
    ref, nsw, rel = oracle.relax_patch_masked(delta, box, mask, alpha, s, hf, c, tol=1e-12)
    assert rel <= 1e-12
    got = host(got)
    on = np.zeros(dims, bool)
    on[1:-1, 1:-1, 1:-1] = mask != 0
    assert rel_l2(got[on], ref[on]) <= 1e-10
    assert np.array_equal(got[~on], box[~on])
