"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module builds input fields only; it holds none of the solver's
arithmetic.  The paper's simulations (Sec. 4.1: L = 250 Mpc/h, 512^3
particles, domain cell 0.48 Mpc/h, CIC densities on an AMR mesh) are not
available, so a lognormal transform of a Gaussian random field stands in for
the density contrast delta of Eq. (eomvarphi).

Recipe (every reading of the short specification is stated here):
  * white noise w ~ N(0, 1) from numpy ``PCG64(seed)``, shape N^3, C order;
  * Fourier filter sqrt(P(k)) with P(k) ~ k^-2, k = 2 pi |n| / N; the k = 0
    mode and every mode with |k| > pi (beyond the Nyquist sphere) are zeroed;
  * g = IFFT, minus its mean, rescaled to sample standard deviation sigma;
  * 1 + delta = exp(g - sigma^2 / 2), renormalised so that mean(delta) = 0;
    delta > -1 everywhere.
"""
from __future__ import annotations

import numpy as np


def gaussian_random_field(n: int, sigma: float, seed: int) -> np.ndarray:
    """Zero-mean GRF with P(k) ~ k^-2 truncated at the Nyquist sphere, std sigma."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(w)
    fi = np.fft.fftfreq(n) * n
    fk = np.fft.rfftfreq(n) * n
    n2 = fi[:, None, None] ** 2 + fi[None, :, None] ** 2 + fk[None, None, :] ** 2
    k = 2.0 * np.pi * np.sqrt(n2) / n
    amp = np.zeros_like(k)
    keep = (k > 0) & (k <= np.pi)
    amp[keep] = 1.0 / k[keep]          # sqrt(k^-2)
    g = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g *= sigma / sd
    return g


def lognormal_delta(n: int, sigma: float, seed: int) -> np.ndarray:
    """delta = exp(g - sigma^2/2) - 1, renormalised to zero mean (FP64, C order)."""
    g = gaussian_random_field(n, sigma, seed)
    one_plus = np.exp(g - 0.5 * sigma * sigma)
    one_plus /= one_plus.mean()
    return np.ascontiguousarray(one_plus - 1.0)


def block_mean(fine: np.ndarray, factor: int = 2) -> np.ndarray:
    """Mass-conserving coarse density: mean over factor^3 blocks (CIC-like deposit)."""
    n0, n1, n2 = fine.shape
    return fine.reshape(n0 // factor, factor, n1 // factor, factor, n2 // factor,
                        factor).mean(axis=(1, 3, 5))


def densest_window(delta: np.ndarray, w: int):
    """Origin of the periodic w^3 window with the largest sum of delta.

    Box filter by FFT; ties go to the lexicographically smallest origin.
    """
    n = delta.shape[0]
    box = np.zeros_like(delta)
    box[:w, :w, :w] = 1.0
    # sum over [o, o+w) for every origin o: correlation of delta with the box
    s = np.fft.irfftn(np.fft.rfftn(delta) * np.conj(np.fft.rfftn(box)), s=delta.shape,
                     axes=(0, 1, 2))
    s = np.round(s, 9)
    flat = int(np.argmax(s))     # first maximum in C order = lexicographically smallest
    return tuple(int(x) for x in np.unravel_index(flat, delta.shape))


def patch_workload(n_fine: int = 256, sigma: float = 1.5, seed: int = 2, pn: int = 32):
    """The refinement workload: coarse (n_fine/2)^3 delta plus a 2x-refined patch.

    Returns (delta_coarse, delta_fine_patch, origin) where the patch covers the
    pn^3 coarse cells with the largest summed delta, and delta_fine_patch is the
    (2 pn)^3 block of the n_fine^3 field under it (periodic wrap).
    """
    fine = lognormal_delta(n_fine, sigma, seed)
    coarse = block_mean(fine, 2)
    o = densest_window(coarse, pn)
    idx = [(2 * o[a] + np.arange(2 * pn)) % n_fine for a in range(3)]
    patch = fine[np.ix_(idx[0], idx[1], idx[2])]
    return np.ascontiguousarray(coarse), np.ascontiguousarray(patch), o


def gaussian_blob(n: int, amp: float, radius: float, centre=None) -> np.ndarray:
    """delta = amp exp(-r^2 / 2R^2) minus its mean, centred at cell centre `centre`."""
    c = (n / 2.0 - 0.5) if centre is None else centre
    x = np.arange(n) - c
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    d = amp * np.exp(-r2 / (2.0 * radius * radius))
    return np.ascontiguousarray(d - d.mean())


def smooth_periodic_field(n: int, amp: float, seed: int, modes: int = 4) -> np.ndarray:
    """Sum of a few random low-order Fourier modes (a smooth periodic test field)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = 2.0 * np.pi * np.arange(n) / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    out = np.zeros((n, n, n))
    for _ in range(modes):
        kx, ky, kz = rng.integers(-2, 3, size=3)
        if kx == 0 and ky == 0 and kz == 0:
            kx = 1
        ph = rng.uniform(0, 2 * np.pi)
        out += rng.uniform(0.5, 1.0) * np.cos(kx * X + ky * Y + kz * Z + ph)
    return np.ascontiguousarray(amp * out)


def batch_workload(nbox: int = 96, seed0: int = 1000, sizes=(32, 48, 64, 96, 128),
                   sigma: float = 1.0, alpha_nominal: float = 1.0, size_seed: int = 4):
    """The batched workload: per-box sizes uniform from `sizes`, per-box seeds
    seed0 + b, and alpha = nominal x 10^U(-1, 1) (log-uniform in [0.1, 10])."""
    rng = np.random.Generator(np.random.PCG64(size_seed))
    ns = rng.choice(np.asarray(sizes), size=nbox)
    scales = 10.0 ** rng.uniform(-1.0, 1.0, size=nbox)
    boxes = []
    for b in range(nbox):
        n = int(ns[b])
        boxes.append((n, lognormal_delta(n, sigma, seed0 + b), alpha_nominal * float(scales[b])))
    return boxes


def lognormal_delta_torch(n: int, sigma: float, seed: int, device="cuda"):
    """The same recipe on the GPU with torch's seeded generator (for large batched and
    serving inputs; its numbers differ from the numpy generator's)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    w = torch.randn((n, n, n), generator=g, device=device, dtype=torch.float64)
    wk = torch.fft.rfftn(w)
    fi = torch.fft.fftfreq(n, device=device, dtype=torch.float64) * n
    fk = torch.fft.rfftfreq(n, device=device, dtype=torch.float64) * n
    n2 = fi[:, None, None] ** 2 + fi[None, :, None] ** 2 + fk[None, None, :] ** 2
    k = 2.0 * torch.pi * torch.sqrt(n2) / n
    amp = torch.where((k > 0) & (k <= torch.pi), 1.0 / torch.clamp(k, min=1e-30), torch.zeros_like(k))
    gr = torch.fft.irfftn(wk * amp, s=(n, n, n))
    gr -= gr.mean()
    sd = gr.std(unbiased=False)
    if float(sd) > 0:
        gr *= sigma / sd
    one_plus = torch.exp(gr - 0.5 * sigma * sigma)
    one_plus /= one_plus.mean()
    return (one_plus - 1.0).contiguous()


def serving_sizes(rng, count: int):
    """Grid sides for the serving stream: 16 round(10^U(log10 32, log10 256) / 16)."""
    u = rng.uniform(np.log10(32.0), np.log10(256.0), size=count)
    return (16 * np.round(10.0 ** u / 16.0)).astype(int)


# ---------------------------------------------------------------------------
# Nested refinements around one halo (the multi-level truncation workload).
#
# The paper's refinement levels follow collapsed haloes (Sec. 4.1, Table 1:
# truncation at l_d + 1 .. l_d + 4).  Stand-in: a lognormal background (as
# above, generated at twice the domain resolution and block-averaged, then
# trilinearly interpolated below that scale) plus one NFW halo (Navarro, Frenk
# & White profile; M200 from R200 = (3 M / (4 pi 200 rho_crit))^(1/3),
# concentration c) placed at the densest window of the background.  Every level
# gets delta as the average over ss^3 sub-points of each cell; one constant
# (minus the halo's mean over the box) keeps mean(delta) = 0 on the domain.
# ---------------------------------------------------------------------------
RHO_CRIT = 2.775e11   # h^2 M_sun / Mpc^3


def nfw_delta(r: np.ndarray, m200: float, conc: float, omega_m: float = 0.3) -> np.ndarray:
    """rho_NFW(r) / rho_bar (Mpc/h, M_sun/h); the cusp is capped at r = r_s / 50, zero beyond R200."""
    r200 = (3.0 * m200 / (4.0 * np.pi * 200.0 * RHO_CRIT)) ** (1.0 / 3.0)
    rs = r200 / conc
    rho_s = (200.0 / 3.0) * RHO_CRIT * conc ** 3 / (np.log1p(conc) - conc / (1.0 + conc))
    x = np.maximum(r, rs / 50.0) / rs
    rho = rho_s / (x * (1.0 + x) ** 2)
    return np.where(r < r200, rho, 0.0) / (omega_m * RHO_CRIT)


def _trilinear_periodic(field: np.ndarray, pts: np.ndarray, cell: float) -> np.ndarray:
    """Periodic trilinear interpolation of a cell-centred cube at points (..., 3)."""
    n = field.shape[0]
    u = pts / cell - 0.5
    i0 = np.floor(u).astype(np.int64)
    w = u - i0
    out = np.zeros(pts.shape[:-1])
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                wt = ((w[..., 0] if a else 1 - w[..., 0]) * (w[..., 1] if b else 1 - w[..., 1])
                      * (w[..., 2] if c else 1 - w[..., 2]))
                out += wt * field[(i0[..., 0] + a) % n, (i0[..., 1] + b) % n, (i0[..., 2] + c) % n]
    return out


def _cell_average(f, x0: np.ndarray, h: float, dims, ss: int) -> np.ndarray:
    """Mean of f over ss^3 sub-points of each cell of a box with corner x0, spacing h."""
    acc = np.zeros(dims)
    offs = (np.arange(ss) + 0.5) / ss
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), axis=-1)
    for ox in offs:
        for oy in offs:
            for oz in offs:
                acc += f(x0 + h * (idx + np.array([ox, oy, oz])))
    return acc / ss ** 3


def nested_halo_workload(n_dom: int = 128, box: float = 250.0, levels: int = 4, pn: int = 16,
                         m200: float = 1e14, conc: float = 5.0, sigma: float = 1.5, seed: int = 2,
                         ss: int = 2):
    """Domain delta (n_dom^3, periodic) and `levels` nested refinements around one halo.

    Level l >= 1 is a (2 pn)^3 box at spacing box / n_dom / 2^l covering parent interior
    cells [o_l, o_l + pn) of level l - 1 (the domain window may wrap), centred on the
    halo.  Returns (deltas, origins, spacings): deltas[0] the domain, deltas[l] the
    level-l interior, origins[l] the window of level l in its parent (origins[0] = None).
    """
    bg = block_mean(lognormal_delta(2 * n_dom, sigma, seed), 2)
    h0 = box / n_dom
    r200 = (3.0 * m200 / (4.0 * np.pi * 200.0 * RHO_CRIT)) ** (1.0 / 3.0)
    o = densest_window(bg, 8)
    centre = (np.asarray(o, dtype=np.float64) + 4.0) * h0

    def halo(p):
        d = ((p - centre + box / 2) % box) - box / 2          # minimum image
        return nfw_delta(np.linalg.norm(d, axis=-1), m200, conc)

    def halo_on(corner, h, dims, wrap):
        """Cell averages of the halo on a grid, evaluated only on cells near it."""
        out = np.zeros(dims)
        reach = int(np.ceil(r200 / h)) + 2
        c = np.floor((centre - corner) / h).astype(np.int64)
        rng = [np.arange(c[a] - reach, c[a] + reach + 1) for a in range(3)]
        if not wrap:
            rng = [r[(r >= 0) & (r < dims[a])] for a, r in enumerate(rng)]
        if any(len(r) == 0 for r in rng):
            return out
        sub = _cell_average(halo, corner + h * np.array([r[0] for r in rng]), h,
                            tuple(len(r) for r in rng), ss)
        ix = np.ix_(*[r % dims[a] if wrap else r for a, r in enumerate(rng)])
        out[ix] += sub
        return out

    halo_dom = halo_on(np.zeros(3), h0, (n_dom,) * 3, True)
    offset = -halo_dom.mean()
    deltas, origins, spacings = [np.ascontiguousarray(bg + halo_dom + offset)], [None], [h0]
    corner, h = np.zeros(3), h0
    for lev in range(1, levels + 1):
        # the window of pn parent cells whose centre is nearest the halo centre
        oc = np.round((centre - corner) / h - pn / 2.0).astype(np.int64)
        if lev == 1:
            oc = oc % n_dom
        else:
            oc = np.clip(oc, 0, 2 * pn - pn)
        corner = corner + oc * h
        h = h / 2.0
        dims = (2 * pn,) * 3
        idx = np.stack(np.meshgrid(*[np.arange(2 * pn)] * 3, indexing="ij"), axis=-1)
        bgf = _trilinear_periodic(bg, (corner + h * (idx + 0.5)) % box, h0)
        d = bgf + halo_on(corner, h, dims, False) + offset
        deltas.append(np.ascontiguousarray(d))
        origins.append(tuple(int(x) for x in oc))
        spacings.append(h)
    return deltas, origins, spacings
