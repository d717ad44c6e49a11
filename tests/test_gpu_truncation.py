"""Nested refinements (Sec. 3.1, Fig. amr) and truncation at several levels (Sec. 3.2,
Table 1): the box-sourced coarse-to-fine interpolation, and the properties of a nested
hierarchy around a halo — screening deepens with the level, and the truncation error on the
finest level vanishes when nothing is truncated and is largest when most is."""
import numpy as np
import pytest

import oracle
import workload
from tests.gpu_common import ctx_fixture, dev, host, nominal

pytestmark = pytest.mark.gpu


def test_refine_from_box_equals_refine_from_domain():
    """A parent box cut out of a periodic grid (with its ghost shell) interpolates to the
    same fine values as the periodic grid itself, and both match the oracle."""
    import paper_1511_08200_gb300 as mg
    ctx = ctx_fixture()
    n = 32
    phi = workload.smooth_periodic_field(n, 1.0, 9) + 0.01 * workload.lognormal_delta(n, 1.0, 10)
    o1, p1 = (5, 9, 3), (12, 12, 12)                 # parent window (with a 1-cell ghost shell)
    idx = [np.arange(o1[a] - 1, o1[a] + p1[a] + 1) % n for a in range(3)]
    box = dev(phi[np.ix_(*idx)])
    for o2, p2, g in (((2, 3, 4), (4, 6, 5), 1), ((0, 0, 0), (12, 12, 12), 1), ((1, 1, 1), (3, 2, 4), 2)):
        got = host(ctx.refine_interpolate_box(box, 1, o2, p2, g))
        ref = host(ctx.refine_interpolate(dev(phi), tuple(o1[a] + o2[a] for a in range(3)), p2, g))
        assert np.array_equal(got, ref)
        assert np.abs(got - oracle.refine_interpolate(phi, tuple(o1[a] + o2[a] for a in range(3)),
                                                       p2, g)).max() <= 1e-15
    # a window whose stencil leaves the box is refused
    with pytest.raises(mg.MG5Error):
        ctx.refine_interpolate_box(box, 1, (0, 0, 0), (12, 12, 12), 2)
    with pytest.raises(mg.MG5Error):
        ctx.refine_interpolate_box(box, 1, (6, 0, 0), (7, 4, 4), 1)
    ctx.close()


def test_nested_truncation_properties():
    import paper_1511_08200_gb300 as mg
    import torch
    import bench
    ctx = ctx_fixture()
    levels = 3
    deltas, origins, spacings = workload.nested_halo_workload(64, 125.0, levels, 8)
    d = [dev(x) for x in deltas]
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    tol = 1e-9
    phi, _, i5 = ctx.solve_fifth_force(d[0], mg.default_params(alpha=alpha, s=s, h=spacings[0], tol=tol))
    s_gr = 1.5 * beta * s
    psi, _, ig = ctx.solve_fifth_force(d[0], mg.default_params(alpha=0.0, s=s_gr, h=spacings[0], tol=tol))
    mag = lambda g: np.sqrt((g ** 2).sum(axis=0))
    frc = lambda b, h: host(ctx.force(b, h, ghost=1, periodic=False))
    gr = bench.nested_chain(ctx, mg, torch, d, origins, spacings, psi, 0.0, s_gr, ig.compat_c,
                            levels + 1, tol)
    fgr = [None] + [mag(frc(gr[l], spacings[l])) for l in range(1, levels + 1)]
    g = {}
    for T in (1, 2, 3, levels + 1):
        b = bench.nested_chain(ctx, mg, torch, d, origins, spacings, phi, alpha, s, i5.compat_c, T, tol)
        g[T] = [None] + [0.5 * frc(b[l], spacings[l]) for l in range(1, levels + 1)]
    full = g[levels + 1]
    ratio = [np.median(mag(full[l]) / fgr[l]) for l in range(1, levels + 1)]
    # screening deepens towards the halo: F5/F_GR falls level by level, below 1/(3 beta)
    assert all(a > b for a, b in zip(ratio, ratio[1:])), ratio
    assert ratio[0] < 1.0 / (3.0 * beta)
    eps = {T: np.linalg.norm(g[T][levels] - full[levels]) / np.linalg.norm(full[levels]) for T in g}
    assert eps[levels + 1] == 0.0
    assert eps[1] > eps[levels] > 0.0
    # Eq. errors2: the G_eff error is eps_trunc damped by F5/F_GR
    dgeff = np.median(mag(g[1][levels] - full[levels]) / fgr[levels])
    eps_med = np.median(mag(g[1][levels] - full[levels]) / mag(full[levels]))
    assert dgeff < eps_med
    ctx.close()


def test_refine_cubic_matches_oracle():
    """The tricubic variant on the GPU equals the oracle's (fixed-order sums: to rounding)."""
    ctx = ctx_fixture()
    n = 24
    phi = workload.smooth_periodic_field(n, 1.0, 12) + 0.02 * workload.lognormal_delta(n, 1.0, 13)
    for o, pn, g in (((3, 20, 7), (6, 5, 8), 1), ((0, 0, 0), (24, 24, 24), 0), ((23, 1, 12), (4, 4, 4), 3)):
        got = host(ctx.refine_interpolate_cubic(dev(phi), o, pn, g))
        ref = oracle.refine_cubic(phi, o, pn, g)
        assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    ctx.close()
