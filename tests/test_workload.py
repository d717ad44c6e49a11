"""The seeded synthetic inputs have the statistics their recipe states (the stand-in for the
paper's N-body densities): the Gaussian field's sample std, zero mean and k^-2 spectrum cut at
the Nyquist sphere, and the lognormal contrast's mean zero and delta > -1."""
import numpy as np

import workload


def test_gaussian_field_spectrum_and_moments():
    n, sigma = 48, 1.3
    g = workload.gaussian_random_field(n, sigma, 11)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - sigma) < 1e-12
    gk = np.abs(np.fft.fftn(g)) ** 2
    f = np.fft.fftfreq(n) * n
    kk = 2 * np.pi * np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2) / n
    assert gk[0, 0, 0] < 1e-20 * gk.sum()
    assert gk[kk > np.pi * 1.0001].max() < 1e-20 * gk.sum()       # nothing beyond Nyquist
    # shell-averaged power against k: slope -2 (white noise filtered by 1/k)
    edges = np.linspace(0.2, 2.5, 12)
    kc, pk = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        sel = (kk >= a) & (kk < b)
        kc.append(kk[sel].mean())
        pk.append(gk[sel].mean())
    slope = np.polyfit(np.log(kc), np.log(pk), 1)[0]
    assert -2.2 < slope < -1.8, slope


def test_lognormal_delta_recipe():
    a = workload.lognormal_delta(32, 1.5, 3)
    b = workload.lognormal_delta(32, 1.5, 3)
    c = workload.lognormal_delta(32, 1.5, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)      # seeded
    assert abs(a.mean()) < 1e-12 and a.min() > -1.0
    g = workload.gaussian_random_field(32, 1.5, 3)
    # 1 + delta is exp(g - sigma^2/2) up to the renormalising constant
    r = (1.0 + a) / np.exp(g - 0.5 * 1.5 ** 2)
    assert np.ptp(r) < 1e-12 * r.mean()


def test_block_mean_conserves_mass():
    f = workload.lognormal_delta(16, 1.0, 5)
    c = workload.block_mean(f, 2)
    assert c.shape == (8, 8, 8)
    assert abs(c.sum() * 8 - f.sum()) < 1e-9
    assert np.isclose(c[1, 2, 3], f[2:4, 4:6, 6:8].mean())


def test_densest_window_brute_force():
    """The FFT box filter finds the periodic window a direct scan finds (wrapping windows
    included), and the refinement workload's patch is the fine block under it."""
    n, w = 12, 4
    d = workload.lognormal_delta(n, 1.5, 8)
    best, arg = -np.inf, None
    for i in range(n):
        for j in range(n):
            for k in range(n):
                idx = [(np.arange(w) + o) % n for o in (i, j, k)]
                v = d[np.ix_(*idx)].sum()
                if v > best + 1e-9:
                    best, arg = v, (i, j, k)
    assert workload.densest_window(d, w) == arg
    coarse, patch, o = workload.patch_workload(24, 1.5, 2, 4)
    fine = workload.lognormal_delta(24, 1.5, 2)
    assert np.array_equal(coarse, workload.block_mean(fine, 2))
    assert o == workload.densest_window(coarse, 4)
    idx = [(2 * o[a] + np.arange(8)) % 24 for a in range(3)]
    assert np.array_equal(patch, fine[np.ix_(*idx)])
    assert np.isclose(workload.block_mean(patch, 2).sum(),
                      coarse[np.ix_(*[(o[a] + np.arange(4)) % 12 for a in range(3)])].sum())


def test_nested_halo_workload_geometry():
    """The nested refinements halve the spacing per level, sit inside their parents, keep the
    domain's mean density contrast at zero, and zoom into the halo: each level's mean density
    contrast is above its parent's."""
    deltas, origins, spacings = workload.nested_halo_workload(n_dom=32, levels=3, pn=8)
    assert len(deltas) == 4 and origins[0] is None
    assert abs(deltas[0].mean()) < 1e-12 and deltas[0].shape == (32, 32, 32)
    for lev in range(1, 4):
        assert deltas[lev].shape == (16, 16, 16)
        assert np.isclose(spacings[lev], spacings[0] / 2 ** lev)
        o = origins[lev]
        assert all(0 <= x for x in o)
        if lev >= 2:                      # inside the parent's interior (no wrap)
            assert all(x + 8 <= 16 for x in o)
        assert deltas[lev].min() > -1.0
    means = [float(d.mean()) for d in deltas]
    assert all(b > a for a, b in zip(means, means[1:])), means


def test_serving_stream_recipe():
    """The serving stream's requests: Poisson arrivals at the offered rate, sides
    16 round(10^U(log 32, log 256)/16), sigma ~ U(0.5, 2), tolerance 1e-6 or 1e-8 with p = 1/2
    (the same draws for every run: one generator, seed 5)."""
    import bench
    gaps, sizes, sigmas, tols = bench.serving_stream(12000, rate=200.0)
    assert abs(gaps.mean() - 1 / 200.0) < 0.03 / 200.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05          # exponential: cv = 1
    assert sizes.min() >= 32 and sizes.max() <= 256 and np.all(sizes % 16 == 0)
    # log-uniform sides: the median side near sqrt(32 * 256) = 90.5
    assert 80 <= np.median(sizes) <= 100
    assert sigmas.min() >= 0.5 and sigmas.max() <= 2.0
    assert set(np.unique(tols)) == {1e-6, 1e-8} and abs((tols == 1e-6).mean() - 0.5) < 0.02
    again = bench.serving_stream(12000, rate=200.0)
    assert all(np.array_equal(a, b) for a, b in zip((gaps, sizes, sigmas, tols), again))
