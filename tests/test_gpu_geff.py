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


def _oracle_geff(coarse, dpatch, o, pn, alpha, s, beta, h):
    """The Eq. (errors2) quantities from the oracle's fields, in numpy: the fifth force (solve,
    force) and the GR force (alpha = 0, source (3 beta / 2) s delta) on the domain; on the
    patch the truncated level (trilinear phi interpolated, then differenced), the relaxed level
    (interpolant as Dirichlet ghosts, relaxed), the tricubic variant and the coarse force
    interpolated directly."""
    import oracle
    hp = h / 2
    phi, info = oracle.solve(coarse, alpha, s, h, tol=1e-13)
    psi, ginfo = oracle.solve(coarse, 0.0, 1.5 * beta * s, h, tol=1e-13)
    grad, g_psi = oracle.force(phi, h), oracle.force(psi, h)
    box = oracle.refine_interpolate(phi, o, pn, 1)
    g_tr = oracle.force(box, hp, ghost=1, periodic=False)
    full, _, _ = oracle.relax_patch(dpatch, box, alpha, s, hp, info.compat_c, tol=1e-13)
    g_full = oracle.force(full, hp, ghost=1, periodic=False)
    gbox = oracle.refine_interpolate(psi, o, pn, 1)
    gfull, _, _ = oracle.relax_patch(dpatch, gbox, 0.0, 1.5 * beta * s, hp, ginfo.compat_c,
                                     tol=1e-13)
    g_gr = oracle.force(gfull, hp, ghost=1, periodic=False)
    g_cub = oracle.force(oracle.refine_cubic(phi, o, pn, 1), hp, ghost=1, periodic=False)
    g_fi = np.stack([oracle.refine_interpolate(np.ascontiguousarray(grad[a]), o, pn, 0)
                     for a in range(3)])
    q = lambda t: list(np.quantile(t.ravel(), [0.5, 0.99]))   # noqa: E731
    rl2 = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))   # noqa: E731
    d5 = 0.5 * _mag(g_tr - g_full)
    return {"eps_trunc_rel_l2_by_interpolant": {"phi_trilinear": rl2(g_tr, g_full),
                                                "phi_tricubic": rl2(g_cub, g_full),
                                                "force_trilinear": rl2(g_fi, g_full)},
            "f5_over_fgr_domain_p50_p99": q(0.5 * _mag(grad) / _mag(g_psi)),
            "f5_over_fgr_patch_p50_p99": q(0.5 * _mag(g_full) / _mag(g_gr)),
            "f5_over_fgr_patch_trunc_p50_p99": q(0.5 * _mag(g_tr) / _mag(g_gr)),
            "eps_trunc_rel_l2": rl2(g_tr, g_full),
            "eps_trunc_p50_p99": q(d5 / (0.5 * _mag(g_full))),
            "geff_error_p50_p99": q(d5 / _mag(g_gr))}


def test_geff_report_matches_oracle():
    """The bench's Eq. (errors2) report (F5/F_GR on the domain and the patch, eps_trunc and the
    G_eff error quantiles, eps_trunc per interpolant), computed by the bench's own functions
    from the GPU fields of a 16^3 patch in a 32^3 domain, against the same quantities from
    the oracle's fields."""
    import torch
    import bench
    import paper_1511_08200_gb300 as mg
    ctx = ctx_fixture()
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    h = 250.0 / 128
    coarse, dpatch, o = workload.patch_workload(64, 1.5, 2, 8)
    pn = (8, 8, 8)
    d_c, d_p = dev(coarse), dev(dpatch)
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-12)
    grad = torch.empty((3, 32, 32, 32), dtype=torch.float64, device="cuda")
    phi, _, info = ctx.solve_fifth_force(d_c, p, grad=grad)
    box = ctx.refine_interpolate(phi, o, pn, 1)
    g_tr = ctx.force(box, h / 2, ghost=1, periodic=False)
    pp = mg.default_params(alpha=alpha, s=s, h=h / 2, tol=1e-12, max_cycles=1000)
    full, _ = ctx.relax_patch(d_p, pp, info.compat_c, box.clone())
    g_full = ctx.force(full, h / 2, ghost=1, periodic=False)
    f = bench.geff_fields(mg, torch, ctx, d_c, d_p, phi, grad, o, pn, h, beta, s, tol=1e-12)
    got = bench.geff_numbers(torch, beta, grad, f["g_psi"], g_tr, g_full, f["g_gr"], f["g_cub"],
                             f["g_fi"])
    want = _oracle_geff(coarse, dpatch, o, pn, alpha, s, beta, h)
    for k, v in want.items():
        g = got[k]
        if isinstance(v, dict):
            for kk in v:
                assert g[kk] == pytest.approx(v[kk], rel=1e-8), (k, kk)
        else:
            assert g == pytest.approx(v, rel=1e-8), k
    ctx.close()
