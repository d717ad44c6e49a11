"""FP64 CPU oracle for the nDGP scalar-field multigrid (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The GPU library never
imports this package and this package never imports the GPU library.

The arithmetic lives in ``mg_oracle.c`` (plain C, FP64, OpenMP over the outer
loop only); this module compiles it with gcc and wraps it with ctypes and
numpy.  Paper: arXiv:1511.08200, Eq. (eomvarphi), Eq. (newton), Sec. 3.1-3.2.

Parity status per function (what pins it is in ``tests/test_oracle_pins.py``):
  ndgp_coefficients  pinned: closed form of Eq. (beta) at a = 1, finite differences
  operator           pinned: independent Hessian-matrix form, Fourier symbol
  cell_update        pinned: Newton iteration of Eq. (newton), back-substitution
  sweep              pinned: snapshot invariant (every cell of the colour solves its
                     own equation against the start-of-half-sweep state)
  restrict/prolong   pinned: closed forms on Fourier modes, constants
  solve              pinned: FFT Poisson (alpha = 0), dense Newton on 4^3 and 8^3,
                     manufactured solutions, spherical Vainshtein profile, V-cycle
                     reduction factor <= 0.2 at alpha = 0
  force              pinned: closed form on Fourier modes
  refine_interpolate pinned: constants, linear fields, 1-D closed form
  relax_patch        pinned: manufactured Dirichlet solution
  relax_patch_masked pinned: all-ones mask = relax_patch, empty mask = identity, a box
                     mask = relax_patch of the sub-box, alpha = 0 = sparse direct solve
  parent_force_mask  pinned: hand-placed parents (wrap included), constant ratios
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.%s.so" % platform.machine())
_lib = None


def build(force: bool = False) -> str:
    """Compile mg_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP).  No contraction
    into fused multiply-adds: every product and sum is rounded as written, the same on
    x86 (no FMA at the default target) and on Arm (FMA by default)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o",
             tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d, i, ll = ctypes.c_double, ctypes.c_int, ctypes.c_longlong
    P = ctypes.c_void_p
    lib.or_ndgp_coefficients.argtypes = [d, d, d, P, P, P]
    lib.or_operator.argtypes = [P, i, d, d, P]
    lib.or_cell_update.argtypes = [P, i, i, i, i, d, d, d]
    lib.or_cell_update.restype = d
    lib.or_sweep.argtypes = [P, P, d, i, d, d]
    lib.or_residual.argtypes = [P, P, d, i, d, d, P]
    lib.or_restrict.argtypes = [P, i, P]
    lib.or_prolong_add.argtypes = [P, i, P]
    lib.or_num_levels.argtypes = [i]
    lib.or_num_levels.restype = i
    lib.or_solve.argtypes = [P, i, P, P, P]
    lib.or_solve.restype = i
    lib.or_force.argtypes = [P, P, i, d, i, P]
    lib.or_refine_interpolate.argtypes = [P, i, P, P, i, P]
    lib.or_refine_cubic.argtypes = [P, i, P, P, i, P]
    lib.or_patch_residual.argtypes = [P, P, d, P, d, d, P]
    lib.or_relax_patch.argtypes = [P, P, d, d, d, d, d, i, i, P, P]
    lib.or_relax_patch.restype = i
    lib.or_patch_sweep.argtypes = [P, P, d, P, d, d]
    lib.or_parent_force_mask.argtypes = [P, P, P, i, P, P, d, P]
    lib.or_relax_patch_masked.argtypes = [P, P, d, d, d, d, P, d, i, i, P, P]
    lib.or_relax_patch_masked.restype = i
    lib.or_clamped.restype = ll
    _lib = lib
    return lib


def _p(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i3(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))


class _Params(ctypes.Structure):
    _fields_ = [
        ("alpha", ctypes.c_double),
        ("s", ctypes.c_double),
        ("h", ctypes.c_double),
        ("tol", ctypes.c_double),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("nu_coarse", ctypes.c_int),
        ("max_cycles", ctypes.c_int),
    ]


class _Info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("cycles", ctypes.c_int),
        ("levels", ctypes.c_int),
        ("coarsest_n", ctypes.c_int),
        ("rel_residual", ctypes.c_double),
        ("compat_c", ctypes.c_double),
        ("phi_mean_removed", ctypes.c_double),
        ("clamped", ctypes.c_longlong),
        ("cell_updates", ctypes.c_longlong),
        ("history", ctypes.c_double * 128),
    ]


@dataclass
class SolveInfo:
    status: int
    cycles: int
    levels: int
    coarsest_n: int
    rel_residual: float
    compat_c: float
    phi_mean_removed: float
    clamped: int
    cell_updates: int = 0
    history: list = field(default_factory=list)


def ndgp_coefficients(a: float, omega_m0: float, h0rc: float):
    """(beta, alpha, s) of Eq. (beta) and Eq. (eomvarphi); alpha in (Mpc/h)^2, s in (h/Mpc)^2."""
    lib = _load()
    out = np.zeros(3)
    base = out.ctypes.data
    lib.or_ndgp_coefficients(a, omega_m0, h0rc, base, base + 8, base + 16)
    return float(out[0]), float(out[1]), float(out[2])


def operator(phi: np.ndarray, h: float, alpha: float) -> np.ndarray:
    """LHS of Eq. (eomvarphi) on a periodic cube, from the definition."""
    phi = _f64(phi)
    n = phi.shape[0]
    out = np.empty_like(phi)
    _load().or_operator(_p(phi), n, h, alpha, _p(out))
    return out


def cell_update(phi: np.ndarray, idx, h: float, alpha: float, rhs: float) -> float:
    phi = _f64(phi)
    i, j, k = idx
    return float(_load().or_cell_update(_p(phi), phi.shape[0], i, j, k, h, alpha, rhs))


def sweep(phi: np.ndarray, f: np.ndarray, c: float, h: float, alpha: float) -> np.ndarray:
    """One snapshot red-black sweep (red first); returns the new field."""
    out = _f64(phi).copy()
    f = _f64(f)
    _load().or_sweep(_p(out), _p(f), c, out.shape[0], h, alpha)
    return out


def residual(phi, f, c, h, alpha) -> np.ndarray:
    phi, f = _f64(phi), _f64(f)
    r = np.empty_like(phi)
    _load().or_residual(_p(phi), _p(f), c, phi.shape[0], h, alpha, _p(r))
    return r


def restrict(fine: np.ndarray) -> np.ndarray:
    fine = _f64(fine)
    n = fine.shape[0]
    out = np.empty((n // 2,) * 3)
    _load().or_restrict(_p(fine), n, _p(out))
    return out


def prolong_add(coarse: np.ndarray, fine: np.ndarray) -> np.ndarray:
    coarse = _f64(coarse)
    out = _f64(fine).copy()
    _load().or_prolong_add(_p(coarse), coarse.shape[0], _p(out))
    return out


def num_levels(n: int) -> int:
    return int(_load().or_num_levels(n))


def solve(delta, alpha, s, h, tol=1e-10, nu1=2, nu2=2, nu_coarse=500, max_cycles=100,
          phi0=None):
    """FAS V-cycle solve of Eq. (eomvarphi) on the periodic cube; returns (phi, SolveInfo)."""
    delta = _f64(delta)
    n = delta.shape[0]
    phi = np.zeros_like(delta) if phi0 is None else _f64(phi0).copy()
    prm = _Params(alpha, s, h, tol, nu1, nu2, nu_coarse, max_cycles)
    info = _Info()
    _load().or_solve(_p(delta), n, ctypes.byref(prm), _p(phi), ctypes.byref(info))
    hist = [info.history[q] for q in range(min(info.cycles + 1, 128))]
    return phi, SolveInfo(info.status, info.cycles, info.levels, info.coarsest_n,
                          info.rel_residual, info.compat_c, info.phi_mean_removed,
                          info.clamped, info.cell_updates, hist)


def force(phi, h, ghost=0, periodic=True) -> np.ndarray:
    """Central-difference gradient, shape (3, *interior)."""
    phi = _f64(phi)
    d = _i3(phi.shape)
    inner = tuple(int(x) - 2 * ghost for x in phi.shape)
    out = np.empty((3,) + inner)
    _load().or_force(_p(phi), _p(d), ghost, h, 1 if periodic else 0, _p(out))
    return out


def refine_interpolate(phic, origin, pn, ghost) -> np.ndarray:
    phic = _f64(phic)
    o, pn_ = _i3(origin), _i3(pn)
    dims = tuple(2 * int(x) + 2 * ghost for x in pn_)
    out = np.empty(dims)
    _load().or_refine_interpolate(_p(phic), phic.shape[0], _p(o), _p(pn_), ghost, _p(out))
    return out


def refine_cubic(phic, origin, pn, ghost) -> np.ndarray:
    """Tricubic (4-point Lagrange per axis) variant of refine_interpolate (an extension)."""
    phic = _f64(phic)
    o, pn_ = _i3(origin), _i3(pn)
    dims = tuple(2 * int(x) + 2 * ghost for x in pn_)
    out = np.empty(dims)
    _load().or_refine_cubic(_p(phic), phic.shape[0], _p(o), _p(pn_), ghost, _p(out))
    return out


def patch_residual(phi_box, f_interior, c, h, alpha) -> np.ndarray:
    phi_box, f_interior = _f64(phi_box), _f64(f_interior)
    pf = _i3(f_interior.shape)
    r = np.empty_like(f_interior)
    _load().or_patch_residual(_p(phi_box), _p(f_interior), c, _p(pf), h, alpha, _p(r))
    return r


def patch_sweep(phi_box, f_interior, c, h, alpha) -> np.ndarray:
    out = _f64(phi_box).copy()
    f_interior = _f64(f_interior)
    pf = _i3(f_interior.shape)
    _load().or_patch_sweep(_p(out), _p(f_interior), c, _p(pf), h, alpha)
    return out


def relax_patch(delta_f, phi_box, alpha, s, h, c, tol=1e-10, max_sweeps=200000, check=10):
    """Sweep the Dirichlet patch problem to tolerance; returns (phi_box, sweeps, rel)."""
    delta_f = _f64(delta_f)
    out = _f64(phi_box).copy()
    pf = _i3(delta_f.shape)
    rel = np.zeros(1)
    nsw = _load().or_relax_patch(_p(delta_f), _p(pf), alpha, s, h, c, tol, max_sweeps, check,
                                 _p(out), _p(rel))
    return out, int(nsw), float(rel[0])


def parent_force_mask(grad_phi, grad_gr, origin, pn, theta, periodic=True) -> np.ndarray:
    """Sec. 3.3 parent criterion: uint8 mask of the (2 pn) fine interior, 1 where
    |grad(phi)/2| > theta |grad(Psi_GR)| at the parent cell.  Gradients SoA (3, *pd) on the
    periodic domain (periodic=True) or on a refinement's interior (no wrap)."""
    grad_phi, grad_gr = _f64(grad_phi), _f64(grad_gr)
    pd = _i3(grad_phi.shape[1:])
    o, pn_ = _i3(origin), _i3(pn)
    assert grad_gr.shape == grad_phi.shape and grad_phi.shape[0] == 3
    assert all(0 <= o[a] and 1 <= pn_[a] for a in range(3))
    if not periodic:
        assert all(o[a] + pn_[a] <= pd[a] for a in range(3)), "window outside the parent"
    out = np.empty(tuple(2 * int(x) for x in pn_), dtype=np.uint8)
    _load().or_parent_force_mask(_p(grad_phi), _p(grad_gr), _p(pd), 1 if periodic else 0, _p(o),
                                 _p(pn_), theta, _p(out))
    return out


def relax_patch_masked(delta_f, phi_box, mask, alpha, s, h, c, tol=1e-10, max_sweeps=200000,
                       check=10):
    """relax_patch iterating only the cells with mask != 0; returns (phi_box, sweeps, rel)."""
    delta_f = _f64(delta_f)
    out = _f64(phi_box).copy()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    assert m.shape == delta_f.shape and out.shape == tuple(x + 2 for x in delta_f.shape)
    pf = _i3(delta_f.shape)
    rel = np.zeros(1)
    nsw = _load().or_relax_patch_masked(_p(delta_f), _p(pf), alpha, s, h, c, _p(m), tol,
                                        max_sweeps, check, _p(out), _p(rel))
    return out, int(nsw), float(rel[0])


def clamped() -> int:
    return int(_load().or_clamped())
