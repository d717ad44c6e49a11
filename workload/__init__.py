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
