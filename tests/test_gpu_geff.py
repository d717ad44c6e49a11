"""GR force and G_eff (Eq. modpoisson, Eq. errors2) from the same engine: the GR
potential is the alpha = 0 solve with source (3 beta / 2) s delta, on the domain
grid and relaxed on the patch like the fifth force (F5 = grad(phi) / 2)."""
import numpy as np
import pytest

import workload
from tests.gpu_common import ctx_fixture, dev, host, nominal

pytestmark = pytest.mark.gpu


def _mag(g):
    return np.sqrt((g ** 2).sum(axis=0))


def _field_pair(ctx, mg, coarse, dpatch, o, pn, a, src, h):
    p = mg.default_params(alpha=a, s=src, h=h, tol=1e-12)
    phi, _, info = ctx.solve_fifth_force(dev(coarse), p)
    g = ctx.force(phi, h)
    box = ctx.refine_interpolate(phi, o, pn, 1)
    pp = mg.default_params(alpha=a, s=src, h=h / 2, tol=1e-12, max_cycles=100000)
    relaxed, _ = ctx.relax_patch(dev(dpatch), pp, info.compat_c, box.clone())
    gp = ctx.force(relaxed, h / 2, ghost=1, periodic=False)
    return host(g), host(gp)


def test_force_ratio_linear_limit_is_one_over_3beta():
    """alpha -> 0: phi = (2 / 3 beta) Psi, so F5/F_GR = 1/(3 beta) in every cell (Sec. 2)."""
    import paper_1511_08200_gb300 as mg
    ctx = ctx_fixture()
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    h = 250.0 / 512
    coarse, dpatch, o = workload.patch_workload(64, 1.0, 4, 8)
    pn = (8, 8, 8)
    g5, g5p = _field_pair(ctx, mg, coarse, dpatch, o, pn, 0.0, s, h)
    ggr, ggrp = _field_pair(ctx, mg, coarse, dpatch, o, pn, 0.0, 1.5 * beta * s, h)
    for f5, fgr in ((g5, ggr), (g5p, ggrp)):
        m = _mag(fgr)
        keep = m > 0.1 * m.max()
        ratio = 0.5 * _mag(f5)[keep] / m[keep]
        assert np.abs(ratio * 3.0 * beta - 1.0).max() <= 1e-8
    ctx.close()


def test_screening_lowers_the_ratio_in_the_dense_patch():
    """Nominal alpha: the Vainshtein mechanism suppresses F5/F_GR where the density is
    high (Eq. eomvarphi_sph2 in the spherical case), so the median ratio on the densest
    patch is below the linear value 1/(3 beta) and below the domain median (the domain is
    mostly underdense, where the normal branch leaves the ratio near or above linear)."""
    import paper_1511_08200_gb300 as mg
    ctx = ctx_fixture()
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    h = 250.0 / 512
    coarse, dpatch, o = workload.patch_workload(128, 1.5, 2, 16)
    pn = (16, 16, 16)
    g5, g5p = _field_pair(ctx, mg, coarse, dpatch, o, pn, alpha, s, h)
    ggr, ggrp = _field_pair(ctx, mg, coarse, dpatch, o, pn, 0.0, 1.5 * beta * s, h)
    r_dom = np.median(0.5 * _mag(g5) / _mag(ggr))
    r_patch = np.median(0.5 * _mag(g5p) / _mag(ggrp))
    assert r_patch < 1.0 / (3.0 * beta) and r_patch < r_dom
    ctx.close()
