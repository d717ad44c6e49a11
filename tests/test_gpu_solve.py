"""Solve-level parity: mg5_solve_fifth_force (FP64 and mixed), the force, the
coarse->fine interpolation and the patch relaxation against the FP64 oracle.

Bars (from the specification of the hot path): FP64 phi and force within
relative L2 1e-10 of the oracle's converged discrete solution; mixed
precision within 1e-6.  A residual tolerance of 1e-10 leaves phi about
1.5e-10 from the exact discrete solution (the error / residual ratio of the
V-cycle's last smooth modes), so the 1e-10 phi checks solve to 1e-12; the
1e-10 runs are checked against the bound they imply.
"""
import numpy as np
import pytest

import oracle
import workload
from tests.gpu_common import ctx_fixture, dev, host, need_gpu, nominal, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ctx_fixture()
    yield c
    c.close()


def _mg():
    import paper_1511_08200_gb300 as mg
    return mg


def _solve(ctx, delta, alpha, s, h, tol, precision="fp64", grad=True, **kw):
    import torch
    mg = _mg()
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision=precision, **kw)
    d = dev(delta)
    g = torch.empty((3,) + delta.shape, dtype=torch.float64, device="cuda") if grad else None
    phi, g, info = ctx.solve_fifth_force(d, p, grad=g)
    return host(phi), (host(g) if grad else None), info


@pytest.mark.parametrize("n,sigma,seed", [(8, 1.0, 1), (16, 1.0, 2), (32, 1.0, 1), (48, 1.5, 3),
                                          (64, 1.5, 4), (80, 1.0, 5)])
def test_fp64_solve_matches_oracle(ctx, n, sigma, seed):
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(n, sigma, seed)
    phi, g, info = _solve(ctx, delta, alpha, s, h, 1e-12)
    ref, rinfo = oracle.solve(delta, alpha, s, h, tol=1e-13)
    assert info.status == 0, info
    assert rel_l2(phi, ref) <= 1e-10
    assert rel_l2(g, oracle.force(ref, h)) <= 1e-10
    assert info.compat_c == pytest.approx(rinfo.compat_c, rel=1e-8, abs=1e-12 * abs(s))
    assert info.levels == rinfo.levels and info.coarsest_n == rinfo.coarsest_n
    assert abs(phi.mean()) <= 1e-14 * np.abs(phi).max()


@pytest.mark.parametrize("n,sigma", [(32, 1.0), (48, 1.5), (128, 1.5)])
def test_fp64_fmg_start_matches_oracle(ctx, n, sigma):
    """The full-multigrid start reaches the same discrete solution in no more cycles (with the
    default over-relaxed smoother a V-cycle is strong enough that it often saves none)."""
    mg = _mg()
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(n, sigma, 11)
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-12)
    phi, _, info = ctx.solve_fifth_force(dev(delta), p, fmg=True)
    _, _, plain = ctx.solve_fifth_force(dev(delta), p)
    ref, _ = oracle.solve(delta, alpha, s, h, tol=1e-13)
    assert info.status == 0
    assert rel_l2(host(phi), ref) <= 1e-10
    assert info.cycles <= plain.cycles


def test_fp64_config_32_tol_1e10(ctx):
    """The 32^3 sigma = 1 workload at the stated tolerance: the oracle, recomputing
    the residual of the GPU's phi, finds it below 1e-10; phi and the force lie
    within the bound that residual implies, and the cycle count is the oracle's."""
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(32, 1.0, 1)
    phi, g, info = _solve(ctx, delta, alpha, s, h, 1e-10, omega=1.0)   # the oracle's smoother
    ref_tight, _ = oracle.solve(delta, alpha, s, h, tol=1e-13)
    ref_same, rinfo = oracle.solve(delta, alpha, s, h, tol=1e-10)
    r = oracle.residual(phi, s * delta, info.compat_c, h, alpha)
    assert np.linalg.norm(r) / np.linalg.norm(s * delta) <= 1e-10
    assert info.cycles == rinfo.cycles
    assert rel_l2(phi, ref_same) <= 1e-12        # same algorithm, same stopping point
    assert rel_l2(phi, ref_tight) <= 5e-10
    assert rel_l2(g, oracle.force(ref_tight, h)) <= 5e-10


def test_fp64_full_size_128(ctx):
    """The 128^3 sigma = 1.5 coarse grid of the refinement workload, element by element."""
    alpha, s, h = nominal()
    coarse, patch, o = workload.patch_workload(256, 1.5, 2, 32)
    h2 = 2 * (250.0 / 512)
    phi, g, info = _solve(ctx, coarse, alpha, s, h2, 1e-12)
    ref, _ = oracle.solve(coarse, alpha, s, h2, tol=1e-13)
    assert info.status == 0
    assert rel_l2(phi, ref) <= 1e-10
    assert rel_l2(g, oracle.force(ref, h2)) <= 1e-10


def test_linear_limit_alpha_zero(ctx):
    alpha, s, h = 0.0, 1.0, 1.0
    delta = workload.lognormal_delta(32, 1.0, 9)
    phi, _, info = _solve(ctx, delta, alpha, s, h, 1e-12, grad=False)
    ref, _ = oracle.solve(delta, alpha, s, h, tol=1e-13)
    assert rel_l2(phi, ref) <= 1e-10
    assert abs(info.compat_c) < 1e-13


@pytest.mark.parametrize("n,sigma", [(32, 1.0), (64, 2.0), (96, 2.0)])
def test_mixed_matches_fp64_oracle(ctx, n, sigma):
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(n, sigma, 3)
    phi, g, info = _solve(ctx, delta, alpha, s, h, 1e-8, precision="mixed")
    ref, _ = oracle.solve(delta, alpha, s, h, tol=1e-13)
    assert info.status == 0, info
    assert info.rel_residual <= 1e-8
    r = oracle.residual(phi, s * delta, info.compat_c, h, alpha)
    assert np.linalg.norm(r) / np.linalg.norm(s * delta) <= 1e-8
    assert rel_l2(phi, ref) <= 1e-6
    assert rel_l2(g, oracle.force(ref, h)) <= 1e-6


def test_warm_start_converges_at_once(ctx):
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(16, 1.0, 4)
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-10)
    d = dev(delta)
    phi, _, info = ctx.solve_fifth_force(d, p)
    phi2, _, info2 = ctx.solve_fifth_force(d, p, phi=phi.clone(), warm=True)
    assert info2.cycles == 0 and info2.status == 0
    assert torch.allclose(phi2, phi, rtol=0, atol=1e-12 * float(phi.abs().max()))


def test_host_io_equals_device_path(ctx):
    mg = _mg()
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(32, 1.0, 6)
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-10)
    phi_d, _, _ = ctx.solve_fifth_force(dev(delta), p)
    phi_h = np.zeros_like(delta)
    grad_h = np.zeros((3,) + delta.shape)
    ctx.solve_fifth_force_host(delta, p, phi=phi_h, grad=grad_h)
    assert np.array_equal(phi_h, host(phi_d))
    assert rel_l2(grad_h, oracle.force(phi_h, h)) < 1e-13
    # host buffers around a graph replay (FP64 and mixed): the device path's values
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-8)):
        q = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision=prec)
        ref, _, iref = ctx.solve_fifth_force(dev(delta), q, fmg=prec == "fp64")
        for _ in range(2):
            ph = np.zeros_like(delta)
            gh = np.zeros((3,) + delta.shape)
            _, _, ig = ctx.solve_fifth_force_host(delta, q, phi=ph, grad=gh, fmg=prec == "fp64",
                                                  graph=True)
            assert np.array_equal(ph, host(ref)) and ig.cycles == iref.cycles
            assert rel_l2(gh, oracle.force(ph, h)) < 1e-13


def test_status_codes(ctx):
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-10)
    d = dev(workload.lognormal_delta(16, 1.0, 1))
    # not converged within the cap: phi is the last iterate, status reported
    q = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-14, max_cycles=2)
    _, _, info = ctx.solve_fifth_force(d, q, raise_on_status=False)
    assert info.status == mg.E_NOT_CONVERGED and info.cycles == 2
    # non-finite input
    bad = d.clone()
    bad[3, 4, 5] = float("nan")
    _, _, info = ctx.solve_fifth_force(bad, p, raise_on_status=False)
    assert info.status == mg.E_NONFINITE
    # odd size and too-large coarsest grid
    for n in (15, 66):
        with pytest.raises(mg.MG5Error) as e:
            ctx.solve_fifth_force(torch.zeros((n,) * 3, dtype=torch.float64, device="cuda"), p)
        assert e.value.code == mg.E_ARG
    # the context is still usable
    _, _, info = ctx.solve_fifth_force(d, p)
    assert info.status == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stopping_norm_when_the_mean_dominates(ctx, precision):
    """The stopping test's ||r - mean r|| / ||s delta|| when the residual's mean is a million
    times its spread (a source whose mean is far from zero, checked before any smoothing: the
    FP64 solve's warm-start check of phi = 0, the mixed solve's first FP64 residual).  The
    first entry of the residual history against the oracle's residual reduced in two passes
    (numpy: mean first, then the norm of r - mean)."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    n = 64
    d0 = workload.lognormal_delta(n, 1.0, 7)
    delta = d0 + 1e6 * d0.std()
    r = oracle.residual(np.zeros_like(delta), s * delta, 0.0, h, alpha)
    m = r.mean()
    assert abs(m) >= 0.99e6 * r.std()
    want = float(np.linalg.norm(r - m) / np.linalg.norm(s * delta))
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-30, max_cycles=0, precision=precision)
    phi = torch.zeros((n,) * 3, dtype=torch.float64, device="cuda")
    _, _, info = ctx.solve_fifth_force(dev(delta), p, phi=phi, warm=(precision == "fp64"),
                                       raise_on_status=False)
    assert info.status == mg.E_NOT_CONVERGED and len(info.history) >= 1
    got = info.history[0]
    assert abs(got - want) <= 1e-12 * want, (got, want)


def test_budget_is_enforced():
    need_gpu()
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    small = mg.Context(0, hbm_budget_bytes=1 << 20)
    p = mg.default_params(alpha=alpha, s=s, h=h)
    with pytest.raises(mg.MG5Error) as e:
        small.solve_fifth_force(torch.zeros((64,) * 3, dtype=torch.float64, device="cuda"), p)
    assert e.value.code == mg.E_OOM
    assert small.bytes_held() <= 1 << 20
    small.close()


def test_zero_source_gives_zero(ctx):
    import torch
    mg = _mg()
    p = mg.default_params(alpha=0.1, s=1.0, h=1.0)
    phi, _, info = ctx.solve_fifth_force(torch.zeros((8,) * 3, dtype=torch.float64, device="cuda"), p)
    assert info.status == 0 and info.cycles == 0
    assert float(phi.abs().max()) == 0.0


def _patch_case(nc=32, pn=8, sigma=1.5, seed=7):
    fine = workload.lognormal_delta(2 * nc, sigma, seed)
    coarse = workload.block_mean(fine, 2)
    o = workload.densest_window(coarse, pn)
    idx = [(2 * o[a] + np.arange(2 * pn)) % (2 * nc) for a in range(3)]
    return coarse, np.ascontiguousarray(fine[np.ix_(*idx)]), o


def test_refine_and_relax_patch_match_oracle(ctx):
    """Truncated (interpolated) vs relaxed fine phi on a 16^3 patch of a 32^3 grid."""
    mg = _mg()
    alpha, s, h = nominal()
    coarse, dpatch, o = _patch_case()
    pn = (8, 8, 8)
    phic, _, info = _solve(ctx, coarse, alpha, s, h, 1e-12, grad=False)
    ref_c, rinfo = oracle.solve(coarse, alpha, s, h, tol=1e-13)
    box = ctx.refine_interpolate(dev(phic), o, pn, 1)
    box_ref = oracle.refine_interpolate(ref_c, o, pn, 1)
    assert rel_l2(host(box), box_ref) <= 1e-10
    hf = h / 2
    p = mg.default_params(alpha=alpha, s=s, h=hf, tol=1e-12, max_cycles=100000)
    relaxed, pinfo = ctx.relax_patch(dev(dpatch), p, info.compat_c, box.clone())
    ref_relaxed, nsw, rel = oracle.relax_patch(dpatch, box_ref, alpha, s, hf, rinfo.compat_c,
                                               tol=1e-12)
    assert pinfo.status == 0 and pinfo.rel_residual <= 1e-12
    got = host(relaxed)
    assert rel_l2(got, ref_relaxed) <= 1e-10
    # ghosts untouched
    assert np.array_equal(got[0], host(box)[0]) and np.array_equal(got[:, :, -1], host(box)[:, :, -1])
    # forces on the patch interior: truncated (interpolated) vs full (relaxed)
    g_tr = host(ctx.force(box, hf, ghost=1, periodic=False))
    g_full = host(ctx.force(relaxed, hf, ghost=1, periodic=False))
    assert rel_l2(g_tr, oracle.force(box_ref, hf, ghost=1, periodic=False)) <= 1e-10
    assert rel_l2(g_full, oracle.force(ref_relaxed, hf, ghost=1, periodic=False)) <= 1e-10
    assert 0 < rel_l2(g_tr, g_full) < 1.0


def test_relax_patch_full_size_64(ctx):
    """The 64^3 patch of the refinement workload (128^3 coarse grid), relaxed by the
    patch multigrid, against the oracle's Gauss-Seidel relaxation of the same
    Dirichlet problem, both to 1e-11."""
    mg = _mg()
    alpha, s, h = nominal()
    coarse, dpatch, o = workload.patch_workload(256, 1.5, 2, 32)
    hc = 250.0 / 128
    ref_c, rinfo = oracle.solve(coarse, alpha, s, hc, tol=1e-13)
    box_ref = oracle.refine_interpolate(ref_c, o, (32, 32, 32), 1)
    box = dev(box_ref)
    p = mg.default_params(alpha=alpha, s=s, h=hc / 2, tol=1e-11)
    relaxed, pinfo = ctx.relax_patch(dev(dpatch), p, rinfo.compat_c, box)
    assert pinfo.status == 0 and pinfo.cycles < 30
    ref_relaxed, nsw, rel = oracle.relax_patch(dpatch, box_ref, alpha, s, hc / 2, rinfo.compat_c,
                                               tol=1e-11)
    assert rel <= 1e-11
    got = host(relaxed)
    assert rel_l2(got[1:-1, 1:-1, 1:-1], ref_relaxed[1:-1, 1:-1, 1:-1]) <= 1e-9
    g = host(ctx.force(relaxed, hc / 2, ghost=1, periodic=False))
    gref = oracle.force(ref_relaxed, hc / 2, ghost=1, periodic=False)
    assert rel_l2(g, gref) <= 1e-9


def _batch_boxes(nbox, seed0=1000):
    """A small version of the batched workload: sizes from {32, 48, 64}, alpha log-uniform."""
    rng = np.random.Generator(np.random.PCG64(seed0))
    alpha, s, h = nominal()
    out = []
    for b in range(nbox):
        n = int(rng.choice([32, 48, 64]))
        a = alpha * 10 ** rng.uniform(-1, 1)
        out.append((n, workload.lognormal_delta(n, 1.0, seed0 + b), a))
    return out, s, h


def test_batch_equals_alone_and_oracle(ctx):
    """Every box solved inside the batch graph gives the same result as the box
    solved alone (same kernels, same order: bit-identical), and matches the FP64
    oracle within 1e-6."""
    import torch
    mg = _mg()
    boxes, s, h = _batch_boxes(6)
    deltas = [dev(d) for _, d, _ in boxes]
    params = [mg.default_params(alpha=a, s=s, h=h, tol=1e-8, precision="mixed") for _, _, a in boxes]
    grads = [torch.empty((3,) + d.shape, dtype=torch.float64, device="cuda") for d in deltas]
    phis, grads, infos = ctx.solve_batch(deltas, params, grads=grads)
    for i, (n, d, a) in enumerate(boxes):
        assert infos[i].status == 0, infos[i]
        alone, g_alone, ia = ctx.solve_fifth_force(deltas[i], params[i],
                                                   grad=torch.empty_like(grads[i]))
        assert torch.equal(phis[i], alone)
        assert torch.equal(grads[i], g_alone)
        assert infos[i].outer_iters == ia.outer_iters and infos[i].cell_updates == ia.cell_updates
        ref, _ = oracle.solve(d, a, s, h, tol=1e-13)
        assert rel_l2(host(phis[i]), ref) <= 1e-6
    # the same call again reuses the resident graph and gives the same answer
    phis2, _, infos2 = ctx.solve_batch(deltas, params, phis=[torch.empty_like(x) for x in phis],
                                       grads=grads)
    for a, b in zip(phis, phis2):
        assert torch.equal(a, b)


def test_batch_mixed_status_per_box(ctx):
    """A box that cannot converge within its cap reports it; the others are unaffected."""
    import torch
    mg = _mg()
    boxes, s, h = _batch_boxes(3, seed0=2000)
    deltas = [dev(d) for _, d, _ in boxes]
    params = [mg.default_params(alpha=a, s=s, h=h, tol=1e-8, precision="mixed") for _, _, a in boxes]
    params[1] = mg.default_params(alpha=boxes[1][2], s=s, h=h, tol=1e-14, max_cycles=1,
                                  precision="mixed")
    phis, _, infos = ctx.solve_batch(deltas, params, raise_on_status=False)
    assert infos[0].status == 0 and infos[2].status == 0
    assert infos[1].status == mg.E_NOT_CONVERGED and infos[1].outer_iters == 1


def _window(a, o, w):
    """The periodic w^3 window of a (leading three axes) with corner o."""
    n = a.shape[-1]
    ix = [(int(q) + np.arange(w)) % n for q in o]
    return a[..., ix[0][:, None, None], ix[1][None, :, None], ix[2][None, None, :]]


@pytest.fixture(scope="module")
def oracle512():
    """The 512^3 sigma = 2 input of the mixed512 / fp64_512 records and the FP64 oracle's own
    solve of it (tolerance 1e-11, on the host cores; a few minutes), shared by the tests below."""
    need_gpu()
    import torch
    alpha, s, h = nominal()
    n = 512
    d = workload.lognormal_delta_torch(n, 2.0, 3, torch.device("cuda"))   # bench.py's field
    delta = host(d)
    del d
    torch.cuda.empty_cache()
    ref, rinfo = oracle.solve(delta, alpha, s, h, tol=1e-11)
    assert rinfo.rel_residual <= 1e-11
    return delta, ref, oracle.force(ref, h), workload.densest_window(delta, 128)


def test_mixed_512_full_size(oracle512):
    """The 512^3 sigma = 2 mixed-precision workload as bench.py runs it (the same input field,
    tuned sweep schedules) against the FP64 oracle's own 512^3 solve (tolerance 1e-11, on the
    host cores): phi and the force within relative L2 1e-6 on the 128^3 subvolume at the
    origin, on the densest 128^3 window and over the whole grid; the oracle also recomputes
    the residual of the GPU result cell by cell (<= 1e-8)."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    n = 512
    delta, ref, ref_g, dense = oracle512
    ctx = mg.Context(0)
    d = dev(delta)
    ctx.autotune(n, "mixed")
    pm = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-8, precision="mixed")
    grad = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    phim, _, im = ctx.solve_fifth_force(d, pm, grad=grad)
    assert im.status == 0 and im.rel_residual <= 1e-8
    got, got_g = host(phim), host(grad)
    ctx.close()
    del phim, grad, d
    torch.cuda.empty_cache()
    r = oracle.residual(got, s * delta, im.compat_c, h, alpha)
    assert np.linalg.norm(r) / np.linalg.norm(s * delta) <= 1e-8
    del r
    for o in ((0, 0, 0), dense):
        assert rel_l2(_window(got, o, 128), _window(ref, o, 128)) <= 1e-6, o
        assert rel_l2(_window(got_g, o, 128), _window(ref_g, o, 128)) <= 1e-6, o
    assert rel_l2(got, ref) <= 1e-6
    assert rel_l2(got_g, ref_g) <= 1e-6


def test_fp64_512_full_size(oracle512):
    """The fp64_512 record's configuration (the same 512^3 input, FP64 mode, full-multigrid
    start, graph replay) solved to 1e-12 against the oracle's 512^3 solution: phi and the force
    within relative L2 1e-10 over the whole grid and on the densest 128^3 window."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    n = 512
    delta, ref, ref_g, dense = oracle512
    ctx = mg.Context(0)
    d = dev(delta)
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-12)
    grad = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    phi, _, info = ctx.solve_fifth_force(d, p, grad=grad, fmg=True, graph=True)
    assert info.status == 0 and info.rel_residual <= 1e-12
    got, got_g = host(phi), host(grad)
    ctx.close()
    del phi, grad, d
    torch.cuda.empty_cache()
    assert rel_l2(got, ref) <= 1e-10
    assert rel_l2(got_g, ref_g) <= 1e-10
    assert rel_l2(_window(got, dense, 128), _window(ref, dense, 128)) <= 1e-10
    assert rel_l2(_window(got_g, dense, 128), _window(ref_g, dense, 128)) <= 1e-10


def test_graph_solve_equals_host_driven(ctx):
    """MG5_GRAPH replays a captured solve: bit-identical to the host-driven mixed solve,
    on the first call (capture) and on cache hits; other parameters make a new entry."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    for n, sigma, tol in ((32, 1.0, 1e-8), (48, 2.0, 1e-6), (96, 1.5, 1e-8)):
        d = dev(workload.lognormal_delta(n, sigma, 21))
        p = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision="mixed")
        ref, gref, iref = ctx.solve_fifth_force(d, p, grad=torch.empty((3,) + d.shape, dtype=torch.float64, device="cuda"))
        for _ in range(2):
            phi, g, info = ctx.solve_fifth_force(d, p, graph=True,
                                                 grad=torch.empty((3,) + d.shape, dtype=torch.float64, device="cuda"))
            assert torch.equal(phi, ref) and torch.equal(g, gref)
            assert info.outer_iters == iref.outer_iters and info.cell_updates == iref.cell_updates
            assert info.rel_residual == iref.rel_residual and info.status == 0
    # a different input through a cached graph
    d2 = dev(workload.lognormal_delta(32, 1.0, 22))
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-8, precision="mixed")
    ref2, _, _ = ctx.solve_fifth_force(d2, p)
    phi2, _, _ = ctx.solve_fifth_force(d2, p, graph=True,
                                       grad=torch.empty((3,) + d2.shape, dtype=torch.float64, device="cuda"))
    assert torch.equal(phi2, ref2)
    with pytest.raises(mg.MG5Error):   # FP64 needs nu1 + nu2 even (the loop body's buffer swaps)
        ctx.solve_fifth_force(d2, mg.default_params(alpha=alpha, s=s, h=h, nu1=1), graph=True)


def test_graph_recaptured_after_schedule_change(ctx):
    """A captured solve follows the sweep schedules of its capture; after the schedule table
    changes, the next graph call captures again, so replay and host-driven solve stay
    bit-identical (for mixed and FP64, and for a batch)."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    d = dev(workload.lognormal_delta(64, 1.0, 23))
    for prec, tol in (("mixed", 1e-8), ("fp64", 1e-10)):
        p = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision=prec)
        old, tuned = mg.schedule_get(0, prec, 64)
        try:
            other = mg.SWEEP_TWO_PASS if old.form != mg.SWEEP_TWO_PASS else mg.SWEEP_FUSED
            for form in (old.form, other):
                mg.schedule_set(0, prec, 64, form)
                ref, _, _ = ctx.solve_fifth_force(d, p, fmg=(prec == "fp64"))
                got, _, _ = ctx.solve_fifth_force(d, p, fmg=(prec == "fp64"), graph=True)
                assert torch.equal(got, ref), (prec, form)
        finally:
            mg.schedule_set(0, prec, 64, old.form, old.block, old.chunk)
    # a batch captured under one table and relaunched under another
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-8, precision="mixed")
    old, _ = mg.schedule_get(0, "mixed", 64)
    outs = [torch.zeros_like(d), torch.zeros_like(d)]   # the same pointers: the cached batch
    try:
        other = mg.SWEEP_TWO_PASS if old.form != mg.SWEEP_TWO_PASS else mg.SWEEP_FUSED
        for form in (old.form, other):
            mg.schedule_set(0, "mixed", 64, form)
            phis, _, _ = ctx.solve_batch([d, d], [p, p], phis=outs)
            ref, _, _ = ctx.solve_fifth_force(d, p)
            assert torch.equal(phis[0], ref) and torch.equal(phis[1], ref), form
    finally:
        mg.schedule_set(0, "mixed", 64, old.form, old.block, old.chunk)


@pytest.mark.parametrize("n,fmg", [(32, False), (64, True), (128, True)])
def test_fp64_graph_solve_equals_host_driven(ctx, n, fmg):
    """The FP64 solve captured with its V-cycle loop as a WHILE node runs the same kernels as
    the host-driven solve: bit-identical phi and force, cycles and cell updates, on the
    capture and on a cache hit, and it matches the oracle."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(n, 1.5, 31)
    d = dev(delta)
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-10)
    g0 = torch.empty((3,) + d.shape, dtype=torch.float64, device="cuda")
    ref, gref, iref = ctx.solve_fifth_force(d, p, grad=g0, fmg=fmg)
    for _ in range(2):
        g1 = torch.empty_like(g0)
        phi, g, info = ctx.solve_fifth_force(d, p, graph=True, fmg=fmg, grad=g1)
        assert torch.equal(phi, ref) and torch.equal(g, gref)
        assert (info.cycles, info.cell_updates, info.coarse_sweeps) == \
            (iref.cycles, iref.cell_updates, iref.coarse_sweeps)
        assert info.rel_residual == iref.rel_residual and info.status == 0
    if n <= 64:
        oref, _ = oracle.solve(delta, alpha, s, h, tol=1e-12)
        assert rel_l2(host(phi), oref) <= 1e-9


def test_relax_patch_graph_equals_host_driven(ctx):
    """mg5_relax_patch_graph replays the captured patch relaxation: bit-identical to
    mg5_relax_patch, on the capture and on cache hits with a new compat_c and a new box."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    coarse, dpatch, o = _patch_case()
    phic, _, info = _solve(ctx, coarse, alpha, s, h, 1e-12, grad=False)
    pn = (8, 8, 8)
    box = ctx.refine_interpolate(dev(phic), o, pn, 1)
    p = mg.default_params(alpha=alpha, s=s, h=h / 2, tol=1e-12, max_cycles=200)
    d = dev(dpatch)
    for c, scale in ((info.compat_c, 1.0), (info.compat_c, 1.0), (1.5 * info.compat_c, 1.01)):
        b0 = (box * scale).contiguous()
        ref, iref = ctx.relax_patch(d, p, c, b0.clone())
        got, ig = ctx.relax_patch(d, p, c, b0.clone(), graph=True)
        assert torch.equal(ref, got)
        assert (ig.cycles, ig.cell_updates, ig.coarse_sweeps, ig.status) == \
            (iref.cycles, iref.cell_updates, iref.coarse_sweeps, iref.status)
        assert ig.rel_residual == iref.rel_residual
    with pytest.raises(mg.MG5Error):   # nu1 + nu2 odd
        ctx.relax_patch(d, mg.default_params(alpha=alpha, s=s, h=h / 2, nu2=1), info.compat_c,
                        box.clone(), graph=True)


@pytest.mark.parametrize("prec,w,tol,bar", [("fp64", 0.0, 1e-11, 1e-9), ("mixed", 1.3, 1e-8, 1e-6)])
def test_relaxation_weight_same_solution(ctx, prec, w, tol, bar):
    """The smoother's weight changes the iteration, not the discrete problem: an over-relaxed
    smoother (the FP64 default 1.3; 1.3 set by hand in the mixed mode) reaches the plain
    update's (omega = 1) solution; in FP64 it takes fewer V-cycles."""
    mg = _mg()
    alpha, s, h = nominal()
    d = dev(workload.lognormal_delta(64, 1.5, 41))
    p1 = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision=prec, omega=1.0)
    p2 = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision=prec, omega=w)
    a, _, ia = ctx.solve_fifth_force(d, p1)
    b, _, ib = ctx.solve_fifth_force(d, p2)
    assert ia.status == 0 and ib.status == 0
    assert rel_l2(host(b), host(a)) <= bar
    if prec == "fp64":
        assert ib.cycles < ia.cycles
    with pytest.raises(mg.MG5Error):
        ctx.solve_fifth_force(d, mg.default_params(alpha=alpha, s=s, h=h, omega=2.0))


@pytest.mark.parametrize("n,prec,tol,bar", [(144, "fp64", 1e-10, 1e-9), (176, "mixed", 1e-8, 1e-6)])
def test_spectral_coarsest_grid(ctx, n, prec, tol, bar):
    """Sides 16 x odd stop halving at a coarsest grid of (2 x odd)^3 (here 18^3 and 22^3), which
    the coarsest solve handles with its DFT-preconditioned iteration: the solve converges in a
    V-cycle count like the power-of-two sizes' and matches the oracle."""
    alpha, s, h = nominal()
    delta = workload.lognormal_delta(n, 1.5, 51)
    phi, _, info = _solve(ctx, delta, alpha, s, h, tol, precision=prec, grad=False)
    assert info.status == 0
    assert info.coarsest_n == 2 * (n // 16) > 6
    assert info.rel_residual <= tol
    assert info.cycles <= (10 if prec == "fp64" else 12)
    ref, _ = oracle.solve(delta, alpha, s, h, tol=1e-11)
    assert rel_l2(phi, ref) <= bar


def test_bench_step_configuration_matches_oracle(ctx):
    """The refinement step in the launch configuration bench.py times: the 128^3 FP64 solve
    (full-multigrid start, V(3,1), coarsest capped at 4 sweeps a visit) and the 64^3 patch
    relaxation (same cap), both as graph replays, plus the mixed 128^3 solve, against the
    oracle's converged solutions.  The FP64 runs stop at 1e-10, which leaves phi within a few
    1e-10 of the discrete solution; the mixed run at 1e-8 within the 1e-6 bar."""
    import bench
    mg = _mg()
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    coarse, patch, o = workload.patch_workload(bench.N_FINE, bench.SIGMA, bench.SEED, bench.PN)
    h = bench.H_COARSE
    p64, pmix, ppatch = bench.step_params(mg, alpha, s)
    import torch
    grad = torch.empty((3,) + coarse.shape, dtype=torch.float64, device="cuda")
    phi, grad, info = ctx.solve_fifth_force(dev(coarse), p64, grad=grad, fmg=True, graph=True)
    assert info.status == 0 and info.rel_residual <= 1e-10 and info.cycles <= 6
    ref, rinfo = oracle.solve(coarse, alpha, s, h, tol=1e-13)
    assert rel_l2(host(phi), ref) <= 5e-10
    assert rel_l2(host(grad), oracle.force(ref, h)) <= 5e-10
    pn = (bench.PN,) * 3
    box = ctx.refine_interpolate(phi, o, pn, 1)
    box_ref = oracle.refine_interpolate(ref, o, pn, 1)
    assert rel_l2(host(box), box_ref) <= 5e-10
    relaxed, pinfo = ctx.relax_patch(dev(patch), ppatch, info.compat_c, box.clone(), graph=True)
    assert pinfo.status == 0 and pinfo.rel_residual <= 1e-10 and pinfo.cycles <= 8
    ref_relaxed, nsw, rel = oracle.relax_patch(patch, box_ref, alpha, s, h / 2, rinfo.compat_c,
                                               tol=1e-11)
    assert rel <= 1e-11
    got = host(relaxed)
    assert rel_l2(got[1:-1, 1:-1, 1:-1], ref_relaxed[1:-1, 1:-1, 1:-1]) <= 1e-9
    phim, gm, im = ctx.solve_fifth_force(dev(coarse), pmix)
    assert im.status == 0 and im.rel_residual <= 1e-8
    assert rel_l2(host(phim), ref) <= 1e-6


def test_bench_batch_configuration_matches_oracle(ctx):
    """The 96-box batched workload as bench.py runs it (tuned schedules, one graph launch):
    every box converges, and for every grid size the boxes with the smallest and the largest
    alpha match the FP64 oracle within the mixed-precision bar 1e-6."""
    import torch
    import bench
    mg = _mg()
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    sizes, scales, deltas, params = bench.batch_boxes(mg, torch.device("cuda"), alpha, s)
    for n in sorted(set(int(x) for x in sizes)):
        ctx.autotune(n, "mixed")
    phis, _, infos = ctx.solve_batch(deltas, params)
    assert all(i.status == 0 and i.rel_residual <= 1e-8 for i in infos)
    h = bench.L_BOX / 512
    for n in sorted(set(int(x) for x in sizes)):
        idx = [b for b in range(len(sizes)) if int(sizes[b]) == n]
        for b in {min(idx, key=lambda q: scales[q]), max(idx, key=lambda q: scales[q])}:
            d = host(deltas[b])
            ref, rinfo = oracle.solve(d, params[b].alpha, s, h, tol=1e-12)
            assert rinfo.status == 0
            assert rel_l2(host(phis[b]), ref) <= 1e-6, (n, b, scales[b])


@pytest.mark.parametrize("alpha_scale", [0.0, 1.0, 10.0])
def test_vcycle_reduction_factor(ctx, alpha_scale):
    """The GPU FP64 V-cycle reduces the residual by a factor <= 0.2 per cycle (Sec. 3.1: the
    coarse grids remove the long-wavelength error that relaxation alone reduces slowly), in the
    Poisson limit and at the nominal nonlinearity; at 10 x the
    nominal one the first cycle is a nonlinear transient (measured 0.31), every later one
    <= 0.2."""
    mg = _mg()
    alpha, s, h = nominal()
    d = dev(workload.lognormal_delta(64, 1.5, 9))
    p = mg.default_params(alpha=alpha * alpha_scale, s=s, h=h, tol=1e-12)
    _, _, info = ctx.solve_fifth_force(d, p)
    hist = list(info.history)
    assert info.status == 0 and len(hist) >= 4
    ratios = [b / a for a, b in zip(hist, hist[1:])]
    if alpha_scale > 1.0:
        assert ratios[0] <= 0.5, ratios
        ratios = ratios[1:]
    assert max(ratios) <= 0.2, ratios
