"""Independent checks that pin the oracle to the paper and to mathematics.

Nothing here calls the oracle: these are second, differently written
statements of the same discrete problem (a Hessian-matrix form of the
operator, Fourier symbols, a dense Newton solve, an FFT Poisson solve, the
spherical closed form of Eq. (eomvarphi_sph2)).
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# the operator of Eq. (eomvarphi) as a 3x3 Hessian matrix
# --------------------------------------------------------------------------

def _shift(a, d, axis, periodic):
    if periodic:
        return np.roll(a, -d, axis=axis)
    raise ValueError


def hessian_matrix(phi: np.ndarray, h: float) -> np.ndarray:
    """Central-difference Hessian as a (3, 3, *shape) array on a periodic cube."""
    H = np.empty((3, 3) + phi.shape)
    for a in range(3):
        p = np.roll(phi, -1, axis=a)
        m = np.roll(phi, 1, axis=a)
        H[a, a] = (p + m - 2.0 * phi) / h ** 2
        for b in range(a + 1, 3):
            pp = np.roll(np.roll(phi, -1, axis=a), -1, axis=b)
            pm = np.roll(np.roll(phi, -1, axis=a), 1, axis=b)
            mp = np.roll(np.roll(phi, 1, axis=a), -1, axis=b)
            mm = np.roll(np.roll(phi, 1, axis=a), 1, axis=b)
            H[a, b] = H[b, a] = (pp - pm - mp + mm) / (4.0 * h ** 2)
    return H


def op_matrix(phi: np.ndarray, h: float, alpha: float) -> np.ndarray:
    """tr(H) + alpha (tr(H)^2 - tr(H H)) on a periodic cube."""
    H = hessian_matrix(phi, h)
    tr = H[0, 0] + H[1, 1] + H[2, 2]
    trHH = np.einsum("ab...,ba...->...", H, H)
    return tr + alpha * (tr * tr - trHH)


def op_matrix_box(phi_box: np.ndarray, h: float, alpha: float) -> np.ndarray:
    """Same operator on the interior of a box with a one-cell ghost shell."""
    H = np.empty((3, 3) + tuple(s - 2 for s in phi_box.shape))

    def sl(di, dj, dk):
        n0, n1, n2 = phi_box.shape
        return phi_box[1 + di:n0 - 1 + di, 1 + dj:n1 - 1 + dj, 1 + dk:n2 - 1 + dk]

    e = np.eye(3, dtype=int)
    c = sl(0, 0, 0)
    for a in range(3):
        H[a, a] = (sl(*e[a]) + sl(*(-e[a])) - 2.0 * c) / h ** 2
        for b in range(a + 1, 3):
            H[a, b] = H[b, a] = (sl(*(e[a] + e[b])) - sl(*(e[a] - e[b]))
                                 - sl(*(-e[a] + e[b])) + sl(*(-e[a] - e[b]))) / (4.0 * h ** 2)
    tr = H[0, 0] + H[1, 1] + H[2, 2]
    trHH = np.einsum("ab...,ba...->...", H, H)
    return tr + alpha * (tr * tr - trHH)


# --------------------------------------------------------------------------
# Fourier symbols (single cosine mode)
# --------------------------------------------------------------------------

def cos_mode(n: int, nvec, h: float, phase: float = 0.3):
    """phi = cos(theta), theta = 2 pi n.x / N + phase, on cell index x."""
    i = np.arange(n)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    th = 2.0 * np.pi * (nvec[0] * I + nvec[1] * J + nvec[2] * K) / n + phase
    return th


def op_symbol_cos(n: int, nvec, h: float, alpha: float, amp: float, phase: float = 0.3):
    """Closed form of the discrete operator applied to amp cos(theta)."""
    th = cos_mode(n, nvec, h, phase)
    kh = [2.0 * np.pi * v / n for v in nvec]
    d = [-(4.0 / h ** 2) * np.sin(x / 2) ** 2 for x in kh]              # D_aa symbol
    o = {(a, b): -(np.sin(kh[a]) * np.sin(kh[b])) / h ** 2 for a in range(3) for b in range(3)}
    L = sum(d) * amp * np.cos(th)
    hh = (sum(x * x for x in d) + 2.0 * (o[0, 1] ** 2 + o[0, 2] ** 2 + o[1, 2] ** 2)) \
        * (amp * np.cos(th)) ** 2
    return L + alpha * (L * L - hh)


# --------------------------------------------------------------------------
# linear limit: FFT Poisson with the discrete eigenvalues
# --------------------------------------------------------------------------

def fft_poisson(f: np.ndarray, h: float) -> np.ndarray:
    """Solve the 7-point periodic Poisson problem lap(phi) = f - mean(f), mean(phi) = 0."""
    n = f.shape[0]
    fk = np.fft.fftn(f)
    q = np.fft.fftfreq(n) * n
    s2 = np.sin(np.pi * q / n) ** 2
    lam = -(4.0 / h ** 2) * (s2[:, None, None] + s2[None, :, None] + s2[None, None, :])
    lam[0, 0, 0] = 1.0
    pk = fk / lam
    pk[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(pk))


# --------------------------------------------------------------------------
# brute force: dense Newton on the whole discrete system with unknown c
# --------------------------------------------------------------------------

def dense_newton(f: np.ndarray, h: float, alpha: float, steps: int = 6, iters: int = 30):
    """Solve op(phi) - c = f, mean(phi) = 0 by Newton with a dense Jacobian.

    Jacobian columns of the operator come from central differences, which
    are exact for a quadratic operator.  Cells whose indices agree modulo 4
    are perturbed together: their 3x3x3 stencils never overlap, so each row
    of a group's directional derivative belongs to exactly one perturbed
    cell.  The unknown c and the mean constraint enter linearly.
    Continuation in alpha from 0 selects the physical branch.
    Returns (phi, c).
    """
    n = f.shape[0]
    assert n % 4 == 0
    m = n ** 3
    idx = np.arange(m).reshape(f.shape)
    i = np.arange(n)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")

    def F(phi, c, al):
        return (op_matrix(phi, h, al) - f - c).ravel()

    phi = np.zeros(f.shape)
    c = 0.0
    for st in range(1, steps + 1):
        al = alpha * st / steps
        for _ in range(iters):
            r = np.concatenate([F(phi, c, al), [phi.mean()]])
            if np.max(np.abs(r)) < 1e-15 * max(1.0, np.max(np.abs(f))):
                break
            Jm = np.zeros((m + 1, m + 1))
            eps = 1.0
            for g in range(64):
                sel = (I % 4 == g // 16) & (J % 4 == (g // 4) % 4) & (K % 4 == g % 4)
                if not sel.any():
                    continue
                e = np.where(sel, eps, 0.0)
                dF = (F(phi + e, c, al) - F(phi - e, c, al)) / (2 * eps)
                # owner of each row: the perturbed cell within distance 1 of it
                for di in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        for dk in (-1, 0, 1):
                            q = idx[sel]
                            qi, qj, qk = I[sel], J[sel], K[sel]
                            p = idx[(qi + di) % n, (qj + dj) % n, (qk + dk) % n]
                            Jm[p, q] = dF[p]
            Jm[:m, m] = -1.0
            Jm[m, :m] = 1.0 / m
            dx = np.linalg.solve(Jm, -r)
            phi = phi + dx[:m].reshape(f.shape)
            c = c + dx[m]
            if np.max(np.abs(dx)) < 1e-15 * max(1.0, np.max(np.abs(phi))):
                break
    return phi, c


# --------------------------------------------------------------------------
# spherical symmetry: Eq. (eomvarphi_sph) / (eomvarphi_sph2)
# --------------------------------------------------------------------------

def gaussian_enclosed(r, amp, R, background):
    """m(r) = int_0^r delta(x) x^2 dx for delta = amp exp(-x^2/2R^2) - background."""
    from scipy.special import erf
    r = np.asarray(r, dtype=float)
    m = amp * R ** 3 * (np.sqrt(np.pi / 2) * erf(r / (np.sqrt(2) * R))
                        - (r / R) * np.exp(-r ** 2 / (2 * R ** 2)))
    return m - background * r ** 3 / 3.0


def spherical_dphi_dr(r, m, alpha, s):
    """phi_r from integrating Eq. (eomvarphi) over a sphere: y = phi_r / r solves
    2 alpha y^2 + y = s m(r) / r^3; physical root."""
    q = s * m / r ** 3
    if alpha == 0:
        return r * q
    return r * (-1.0 + np.sqrt(1.0 + 8.0 * alpha * q)) / (4.0 * alpha)
