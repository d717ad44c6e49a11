"""GB300-native nonlinear multigrid for the nDGP fifth force (arXiv:1511.08200).

Thin ctypes binding of ``libmg5.so`` (C ABI declared in ``include/mg5.h``).
The functions keep the C names without the ``mg5_`` prefix and only marshal
arguments: every step of the solve runs in the library's CUDA kernels.
Device fields are torch CUDA tensors (float64, C-contiguous); PyTorch is used
for device memory and streams only.  There is no CPU fallback: if the
library has not been built, importing this package raises.

With MG5_BOUNDS=1 in the environment the range-checked build libmg5_bounds.so
is loaded instead (``python -m paper_1511_08200_gb300._build --bounds``); every
tensor handed to it is noted as a buffer its kernels may touch, and
``bounds_check()`` reports the first out-of-range access since the last call.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
_BOUNDS = os.environ.get("MG5_BOUNDS", "0") == "1"
_LIB_PATH = os.path.join(_HERE, "libmg5_bounds.so" if _BOUNDS else "libmg5.so")

if not os.path.exists(_LIB_PATH):
    raise ImportError(
        "%s is not built; run %s (nvcc, sm_103a) before importing paper_1511_08200_gb300"
        % (os.path.basename(_LIB_PATH),
           "`python -m paper_1511_08200_gb300._build --bounds`" if _BOUNDS
           else "`python -c 'import __graft_entry__ as g; g.build()'`"))

_lib = ctypes.CDLL(_LIB_PATH)

OK, W_DISC_CLAMP, W_UNTUNED = 0, 1, 2
SWEEP_TWO_PASS, SWEEP_FUSED, SWEEP_MARCH = 0, 1, 2
E_ARG, E_OOM, E_CUDA, E_NOT_CONVERGED, E_DIVERGED, E_NONFINITE, E_TOO_LARGE = -1, -2, -3, -4, -5, -6, -7
FP64, MIXED = 0, 1
WARM, HOST_IO, FMG_START, GRAPH = 1, 2, 4, 8

_c_int, _c_double, _c_void_p, _c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_c_uint = ctypes.c_uint


class Params(ctypes.Structure):
    _fields_ = [("alpha", _c_double), ("s", _c_double), ("h", _c_double), ("tol", _c_double),
                ("nu1", _c_int), ("nu2", _c_int), ("nu_coarse", _c_int), ("max_cycles", _c_int),
                ("precision", _c_int), ("inner_cycles", _c_int), ("omega", _c_double)]


class _Info(ctypes.Structure):
    _fields_ = [("status", _c_int), ("cycles", _c_int), ("outer_iters", _c_int),
                ("levels", _c_int), ("coarsest_n", _c_int), ("n_history", _c_int),
                ("rel_residual", _c_double), ("compat_c", _c_double),
                ("phi_mean_removed", _c_double), ("disc_clamped", ctypes.c_longlong),
                ("cell_updates", ctypes.c_longlong), ("ms_total", _c_double),
                ("coarse_sweeps", ctypes.c_longlong), ("history", _c_double * 64)]


@dataclass
class Info:
    status: int
    cycles: int
    outer_iters: int
    levels: int
    coarsest_n: int
    rel_residual: float
    compat_c: float
    phi_mean_removed: float
    disc_clamped: int
    cell_updates: int
    ms_total: float
    coarse_sweeps: int = 0
    history: list = field(default_factory=list)

    @classmethod
    def _from(cls, i: _Info) -> "Info":
        return cls(i.status, i.cycles, i.outer_iters, i.levels, i.coarsest_n, i.rel_residual,
                   i.compat_c, i.phi_mean_removed, i.disc_clamped, i.cell_updates, i.ms_total,
                   i.coarse_sweeps, [i.history[q] for q in range(min(i.n_history, 64))])


class _Request(ctypes.Structure):
    _fields_ = [("delta", _c_void_p), ("N", _c_int), ("params", Params), ("phi", _c_void_p),
                ("grad", _c_void_p), ("tag", ctypes.c_ulonglong)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("builds", ctypes.c_longlong), ("evictions", ctypes.c_longlong),
                ("fallbacks", ctypes.c_longlong), ("memory_waits", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("build_seconds", _c_double)]


class _Completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_ulonglong), ("status", _c_int), ("pad", _c_int),
                ("t_submit", _c_double), ("t_admit", _c_double), ("t_done", _c_double),
                ("info", _Info)]


class Schedule(ctypes.Structure):
    """mg5_schedule: how one grid side is swept (form, two-pass block, fused chunk, tuned ms)."""
    _fields_ = [("form", _c_int), ("block", _c_int), ("chunk", _c_int), ("ms", ctypes.c_float)]


_P = _c_void_p
_I3 = ctypes.c_int * 3
_sigs = {
    "mg5_version": ([], _c_int),
    "mg5_kernel_launches": ([], ctypes.c_longlong),
    "mg5_status_string": ([_c_int], ctypes.c_char_p),
    "mg5_default_params": ([_P], _c_int),
    "mg5_ndgp_coefficients": ([_c_double, _c_double, _c_double, _P, _P, _P], _c_int),
    "mg5_workspace_bytes": ([_c_int, _c_int, _P], _c_int),
    "mg5_create": ([_P, _c_int, _c_size_t], _c_int),
    "mg5_destroy": ([_P], _c_int),
    "mg5_last_error": ([_P], ctypes.c_char_p),
    "mg5_bytes_held": ([_P], _c_size_t),
    "mg5_release": ([_P], _c_int),
    "mg5_solve_fifth_force": ([_P, _P, _c_int, _P, _c_uint, _P, _P, _P, _P], _c_int),
    "mg5_force": ([_P, _P, _I3, _c_int, _c_double, _c_int, _P, _P], _c_int),
    "mg5_refine_interpolate": ([_P, _P, _c_int, _I3, _I3, _c_int, _P, _P], _c_int),
    "mg5_refine_interpolate_cubic": ([_P, _P, _c_int, _I3, _I3, _c_int, _P, _P], _c_int),
    "mg5_refine_interpolate_box": ([_P, _P, _I3, _c_int, _I3, _I3, _c_int, _P, _P], _c_int),
    "mg5_relax_patch": ([_P, _P, _I3, _P, _c_double, _P, _P, _P], _c_int),
    "mg5_relax_patch_graph": ([_P, _P, _I3, _P, _c_double, _P, _P, _P], _c_int),
    "mg5_relax_patch_masked": ([_P, _P, _I3, _P, _P, _c_double, _P, _P, _P], _c_int),
    "mg5_parent_force_mask": ([_P, _P, _P, _I3, _c_int, _I3, _I3, _c_double, _P,
                               ctypes.POINTER(ctypes.c_longlong), _P], _c_int),
    "mg5_solve_batch": ([_P, _c_int, _P, _P, _P, _P, _P, _P, _P], _c_int),
    "mg5_cached_bytes": ([_P, _c_int, _c_int, _P], _c_int),
    "mg5_graph_cached_bytes": ([_P, _c_int, _P, _c_int, _P], _c_int),
    "mg5_graph_workspace_bytes": ([_c_int, _c_int, _P], _c_int),
    "mg5_server_create": ([_P, _c_int, _c_int, _c_size_t], _c_int),
    "mg5_server_submit": ([_P, _P], _c_int),
    "mg5_server_poll": ([_P, _P, _c_int, _c_int], _c_int),
    "mg5_server_pending": ([_P, _P, _P], _c_int),
    "mg5_server_clock": ([_P], _c_double),
    "mg5_server_bytes_held": ([_P], _c_size_t),
    "mg5_server_destroy": ([_P], _c_int),
    "mg5_server_get_stats": ([_P, _P], _c_int),
    "mg5_set_blocking_wait": ([_P, _c_int], _c_int),
    "mg5_set_autotune": ([_P, _c_int], _c_int),
    "mg5_autotune": ([_P, _c_int, _c_int, _P], _c_int),
    "mg5_schedule_get": ([_c_int, _c_int, _c_int, _P], _c_int),
    "mg5_schedule_set": ([_c_int, _c_int, _c_int, _P], _c_int),
    "mg5_tune_clear": ([], _c_int),
    "mg5_tune_save": ([ctypes.c_char_p], _c_int),
    "mg5_tune_load": ([ctypes.c_char_p], _c_int),
    "mg5_residual_norm_noalloc": ([_P, _P, _c_double, _c_int, _c_double, _c_double, _P, _P], _c_int),
    "mg5_residual_norm_noalloc_max_cells": ([], ctypes.c_longlong),
    "mg5_bounds_build": ([], _c_int),
    "mg5_bounds_note": ([_P], _c_int),
    "mg5_bounds_check": ([ctypes.c_char_p, _c_int], _c_int),
    "mg5_profile_enable": ([_P, _c_int], _c_int),
    "mg5_profile_read": ([_P, _P, _P, _c_int], _c_int),
    "mg5_profile_name": ([_c_int], ctypes.c_char_p),
    "mg5_profile_units": ([_P, _P, _c_int], _c_int),
    "mg5_step_sweep": ([_P, _P, _P, _P, _c_double, _c_int, _c_double, _c_double, _P], _c_int),
    "mg5_step_sweep_fused": ([_P, _P, _P, _P, _c_double, _c_int, _c_double, _c_double, _P], _c_int),
    "mg5_step_sweep_f32": ([_P, _P, _P, _P, _P, _c_double, _c_int, _c_double, _c_double, _c_int, _P],
                           _c_int),
    "mg5_step_operator": ([_P, _P, _c_int, _c_double, _c_double, _P, _P], _c_int),
    "mg5_step_resid_restrict_f32": ([_P, _P, _P, _P, _c_double, _c_int, _c_double, _c_double, _c_int,
                                     _P, _P, _P, _P], _c_int),
    "mg5_step_residual": ([_P, _P, _P, _c_double, _c_int, _c_double, _c_double, _P, _P], _c_int),
    "mg5_step_restrict": ([_P, _P, _c_int, _P, _P], _c_int),
    "mg5_step_prolong_add": ([_P, _P, _c_int, _P, _P], _c_int),
}
for _name, (_args, _res) in _sigs.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


class MG5Error(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("mg5 status %d (%s): %s" % (code, status_string(code), msg))
        self.code = code


def version() -> int:
    return _lib.mg5_version()


def kernel_launches() -> int:
    """Kernel launches the library has enqueued in this process."""
    return _lib.mg5_kernel_launches()


def status_string(code: int) -> str:
    return _lib.mg5_status_string(code).decode()


def default_params(**kw) -> Params:
    p = Params()
    _lib.mg5_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": FP64, "mixed": MIXED}[v]
        setattr(p, k, v)
    return p


def ndgp_coefficients(a: float, omega_m0: float, h0rc: float):
    """(beta, alpha, s) of Eq. (beta) / Eq. (eomvarphi) for the LCDM-matched nDGP background."""
    b, al, s = _c_double(), _c_double(), _c_double()
    rc = _lib.mg5_ndgp_coefficients(a, omega_m0, h0rc, ctypes.byref(b), ctypes.byref(al),
                                    ctypes.byref(s))
    if rc != OK:
        raise MG5Error(rc, "bad cosmology")
    return b.value, al.value, s.value


def graph_workspace_bytes(n: int, with_grad: bool = False) -> int:
    """Device bytes one cached MG5_GRAPH solve of side n holds."""
    out = _c_size_t()
    rc = _lib.mg5_graph_workspace_bytes(n, 1 if with_grad else 0, ctypes.byref(out))
    if rc != OK:
        raise MG5Error(rc, "bad size")
    return out.value


def _prec(precision) -> int:
    if isinstance(precision, str):
        return {"fp64": FP64, "mixed": MIXED}[precision]
    return int(precision)


def schedule_get(device: int, precision, n: int):
    """mg5_schedule_get: (Schedule, tuned?) of (device, precision, n)."""
    out = Schedule()
    rc = _lib.mg5_schedule_get(device, _prec(precision), n, ctypes.byref(out))
    if rc not in (OK, W_UNTUNED):
        raise MG5Error(rc, "schedule_get")
    return out, rc == OK


def schedule_set(device: int, precision, n: int, form: int, block: int = 256, chunk: int = 0):
    s = Schedule(form, block, chunk, 0.0)
    rc = _lib.mg5_schedule_set(device, _prec(precision), n, ctypes.byref(s))
    if rc != OK:
        raise MG5Error(rc, "schedule_set")


def tune_clear():
    _lib.mg5_tune_clear()


def tune_save(path: str):
    rc = _lib.mg5_tune_save(str(path).encode())
    if rc != OK:
        raise MG5Error(rc, "tune_save %s" % path)


def tune_load(path: str) -> int:
    """Applies a saved table; returns the number of entries that matched a visible GPU."""
    rc = _lib.mg5_tune_load(str(path).encode())
    if rc < 0:
        raise MG5Error(rc, "tune_load %s" % path)
    return rc


def workspace_bytes(n: int, precision=FP64) -> int:
    if isinstance(precision, str):
        precision = {"fp64": FP64, "mixed": MIXED}[precision]
    out = _c_size_t()
    rc = _lib.mg5_workspace_bytes(n, precision, ctypes.byref(out))
    if rc != OK:
        raise MG5Error(rc, "bad size")
    return out.value


def _ptr(t, dtype="float64", device=None) -> int:
    """Device pointer of a contiguous torch CUDA tensor of the given dtype (on `device`
    when given), or None."""
    if t is None:
        return None
    import torch
    want = getattr(torch, dtype)
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == want and t.is_contiguous()):
        raise TypeError("expected a contiguous %s CUDA tensor" % dtype)
    if device is not None and (t.device.index or 0) != device:
        raise MG5Error(E_ARG, "tensor on cuda:%d, the context is on cuda:%d"
                       % (t.device.index or 0, device))
    if _BOUNDS:
        _lib.mg5_bounds_note(t.data_ptr())
    return t.data_ptr()


def bounds_build() -> bool:
    """True when the loaded library is the range-checked build."""
    return bool(_lib.mg5_bounds_build())


def bounds_check():
    """The first out-of-range access the range-checked build recorded since the last call
    ("file: line L: kind out of range"), or None; clears the record.  Synchronise the device
    first.  Always None in the ordinary build."""
    buf = ctypes.create_string_buffer(256)
    return buf.value.decode() if _lib.mg5_bounds_check(buf, 256) else None


# Shape checks, made before any pointer reaches the library: a buffer of the wrong size
# would make the kernels read or write past its end.
def _dims(t) -> tuple:
    return tuple(int(x) for x in t.shape)


def _want(t, shape, name: str):
    """MG5Error(E_ARG) unless t (tensor or array; None passes) has exactly `shape`."""
    if t is not None and _dims(t) != tuple(int(x) for x in shape):
        raise MG5Error(E_ARG, "%s has shape %s, expected %s" % (name, _dims(t), tuple(shape)))


def _cube(t, name: str) -> int:
    """Side N of an N x N x N tensor or array; MG5Error(E_ARG) otherwise."""
    d = _dims(t)
    if len(d) != 3 or d[0] != d[1] or d[1] != d[2]:
        raise MG5Error(E_ARG, "%s must be a cube N x N x N, got shape %s" % (name, d))
    return d[0]


def _box(t, name: str) -> tuple:
    """Dims of a 3-D tensor or array; MG5Error(E_ARG) otherwise."""
    d = _dims(t)
    if len(d) != 3:
        raise MG5Error(E_ARG, "%s must be 3-D, got shape %s" % (name, d))
    return d


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Context:
    """Owns the device hierarchy (mg5_ctx); one per thread."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._h = _c_void_p()
        rc = _lib.mg5_create(ctypes.byref(self._h), device, hbm_budget_bytes)
        if rc != OK:
            raise MG5Error(rc, "mg5_create failed")
        self.device = device

    def close(self):
        if self._h:
            _lib.mg5_destroy(self._h)
            self._h = _c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return _lib.mg5_last_error(self._h).decode()

    def bytes_held(self) -> int:
        return _lib.mg5_bytes_held(self._h)

    def cached_bytes(self, n: int, precision=FP64) -> int:
        if isinstance(precision, str):
            precision = {"fp64": FP64, "mixed": MIXED}[precision]
        out = _c_size_t()
        self._check(_lib.mg5_cached_bytes(self._h, n, precision, ctypes.byref(out)))
        return out.value

    def release(self):
        _lib.mg5_release(self._h)

    def set_autotune(self, on: bool = True):
        """mg5_set_autotune: tune untuned grid sides before each solve / batch capture."""
        self._check(_lib.mg5_set_autotune(self._h, 1 if on else 0))

    def autotune(self, n: int, precision="fp64", stream=None):
        """mg5_autotune: time the sweep schedules of every grid side of n's hierarchy."""
        self._check(_lib.mg5_autotune(self._h, n, _prec(precision), _stream(stream)))

    def set_blocking_wait(self, on: bool = True):
        """mg5_set_blocking_wait: sleep (True) or spin (False, default) while waiting for the GPU."""
        self._check(_lib.mg5_set_blocking_wait(self._h, 1 if on else 0))

    def _check(self, rc: int, allow=(OK,)):
        if rc not in allow:
            raise MG5Error(rc, self.last_error())
        return rc

    # ------------------------------------------------------------ tracing
    def profile_enable(self, on: bool = True):
        self._check(_lib.mg5_profile_enable(self._h, 1 if on else 0))

    def profile_read(self) -> dict:
        """{kernel class: (total ms, launches, cells)} from CUDA events on the launching stream."""
        n = 32
        ms = (_c_double * n)()
        calls = (ctypes.c_longlong * n)()
        units = (_c_double * n)()
        k = _lib.mg5_profile_read(self._h, ms, calls, n)
        if k < 0:
            self._check(k)
        _lib.mg5_profile_units(self._h, units, n)
        return {_lib.mg5_profile_name(i).decode(): (ms[i], calls[i], units[i]) for i in range(k)}

    # ------------------------------------------------------------ hot path
    def solve_fifth_force(self, delta, params: Params, phi=None, grad=None, warm=False,
                          stream=None, raise_on_status=True, fmg=False, graph=False):
        """mg5_solve_fifth_force on device tensors.  phi (out, N^3) and grad
        (out, 3 x N^3, optional) are allocated if not given.  Returns (phi, grad, Info)."""
        import torch
        n = _cube(delta, "delta")
        _want(phi, (n, n, n), "phi")
        _want(grad, (3, n, n, n), "grad")
        if phi is None:
            phi = torch.zeros_like(delta)
        info = _Info()
        flags = (WARM if warm else 0) | (FMG_START if fmg else 0) | (GRAPH if graph else 0)
        dv = self.device
        rc = _lib.mg5_solve_fifth_force(self._h, _ptr(delta, device=dv), n, ctypes.byref(params),
                                        flags, _ptr(phi, device=dv), _ptr(grad, device=dv),
                                        ctypes.byref(info), _stream(stream))
        if raise_on_status:
            self._check(rc, (OK, W_DISC_CLAMP))
        elif rc in (E_ARG, E_OOM, E_CUDA):
            self._check(rc)
        return phi, grad, Info._from(info)

    def solve_fifth_force_host(self, delta, params: Params, phi=None, grad=None, warm=False,
                               stream=None, raise_on_status=True, fmg=False, graph=False):
        """Same call with HOST buffers (numpy float64 or pinned CPU tensors): the
        library copies delta in and phi / grad out (MG5_HOST_IO); graph=True replays
        the captured solve between the copies (MG5_GRAPH)."""
        n = _cube(delta, "delta")
        if phi is None:
            raise MG5Error(E_ARG, "phi (host, N^3) is required with host buffers")
        _want(phi, (n, n, n), "phi")
        _want(grad, (3, n, n, n), "grad")
        info = _Info()
        flags = HOST_IO | (WARM if warm else 0) | (FMG_START if fmg else 0) | (GRAPH if graph else 0)
        rc = _lib.mg5_solve_fifth_force(self._h, _host_ptr(delta), n, ctypes.byref(params), flags,
                                        _host_ptr(phi), _host_ptr(grad), ctypes.byref(info),
                                        _stream(stream))
        if raise_on_status:
            self._check(rc, (OK, W_DISC_CLAMP))
        return phi, grad, Info._from(info)

    def solve_batch(self, deltas, params, phis=None, grads=None, stream=None, raise_on_status=True):
        """mg5_solve_batch: deltas / params / phis / grads are per-box lists (device
        tensors; params a list of Params or one Params for all).  Returns (phis, grads, infos)."""
        import torch
        nb = len(deltas)
        if isinstance(params, Params):
            params = [params] * nb
        ns = [_cube(d, "deltas[%d]" % b) for b, d in enumerate(deltas)]
        for name, lst in (("params", params), ("phis", phis), ("grads", grads)):
            if lst is not None and len(lst) != nb:
                raise MG5Error(E_ARG, "%s has %d entries for %d boxes" % (name, len(lst), nb))
        for b, n in enumerate(ns):
            _want(phis[b] if phis is not None else None, (n, n, n), "phis[%d]" % b)
            _want(grads[b] if grads is not None else None, (3, n, n, n), "grads[%d]" % b)
        if phis is None:
            phis = [torch.zeros_like(d) for d in deltas]
        dv = self.device
        P = ctypes.c_void_p * nb
        parr = (Params * nb)(*params)
        narr = (_c_int * nb)(*ns)
        garr = P(*[_ptr(g, device=dv) for g in grads]) if grads is not None else None
        infos = (_Info * nb)()
        rc = _lib.mg5_solve_batch(self._h, nb, P(*[_ptr(d, device=dv) for d in deltas]), narr, parr,
                                  P(*[_ptr(x, device=dv) for x in phis]), garr, infos,
                                  _stream(stream))
        if raise_on_status:
            self._check(rc, (OK, W_DISC_CLAMP))
        elif rc in (E_ARG, E_OOM, E_CUDA):
            self._check(rc)
        return phis, grads, [Info._from(i) for i in infos]

    def force(self, phi, h: float, ghost: int = 0, periodic: bool = True, grad=None, stream=None):
        import torch
        dims = list(_box(phi, "phi"))
        inner = [d - 2 * ghost for d in dims]
        if ghost < 0 or min(inner) < 1:
            raise MG5Error(E_ARG, "ghost %d leaves no interior in %s" % (ghost, tuple(dims)))
        _want(grad, [3] + inner, "grad")
        if grad is None:
            grad = torch.empty([3] + inner, dtype=phi.dtype, device=phi.device)
        dv = self.device
        self._check(_lib.mg5_force(self._h, _ptr(phi, device=dv), _I3(*dims), ghost, h,
                                   1 if periodic else 0, _ptr(grad, device=dv), _stream(stream)))
        return grad

    def refine_interpolate(self, phi_coarse, origin, pn, ghost: int, out=None, stream=None):
        import torch
        nc = _cube(phi_coarse, "phi_coarse")
        dims = [2 * int(p) + 2 * ghost for p in pn]
        _want(out, dims, "out")
        if out is None:
            out = torch.empty(dims, dtype=phi_coarse.dtype, device=phi_coarse.device)
        _ptr(out, device=self.device)
        self._check(_lib.mg5_refine_interpolate(self._h, _ptr(phi_coarse, device=self.device), nc, _I3(*origin),
                                                _I3(*pn), ghost, _ptr(out), _stream(stream)))
        return out

    def refine_interpolate_cubic(self, phi_coarse, origin, pn, ghost: int, out=None, stream=None):
        """mg5_refine_interpolate_cubic: the tricubic variant of refine_interpolate."""
        import torch
        nc = _cube(phi_coarse, "phi_coarse")
        dims = [2 * int(p) + 2 * ghost for p in pn]
        _want(out, dims, "out")
        if out is None:
            out = torch.empty(dims, dtype=phi_coarse.dtype, device=phi_coarse.device)
        _ptr(out, device=self.device)
        self._check(_lib.mg5_refine_interpolate_cubic(self._h, _ptr(phi_coarse, device=self.device), nc, _I3(*origin),
                                                      _I3(*pn), ghost, _ptr(out), _stream(stream)))
        return out

    def refine_interpolate_box(self, box, pg: int, origin, pn, ghost: int, out=None, stream=None):
        """mg5_refine_interpolate_box: child window [origin, origin + pn) of a parent box
        (dims box.shape, interior offset pg) -> fine box (2 pn + 2 ghost per axis)."""
        import torch
        bd = _box(box, "box")
        dims = [2 * int(p) + 2 * ghost for p in pn]
        _want(out, dims, "out")
        if out is None:
            out = torch.empty(dims, dtype=box.dtype, device=box.device)
        _ptr(out, device=self.device)
        self._check(_lib.mg5_refine_interpolate_box(self._h, _ptr(box, device=self.device), _I3(*bd),
                                                    pg, _I3(*origin), _I3(*pn), ghost, _ptr(out),
                                                    _stream(stream)))
        return out

    def relax_patch(self, delta_fine, params: Params, compat_c: float, phi_box, stream=None,
                    raise_on_status=True, graph=False):
        """mg5_relax_patch (graph=True: mg5_relax_patch_graph): phi_box ((pf + 2)^3, ghosts
        fixed) is relaxed in place."""
        pf = list(_box(delta_fine, "delta_fine"))
        if phi_box is None:
            raise MG5Error(E_ARG, "phi_box is required")
        _want(phi_box, [x + 2 for x in pf], "phi_box")
        info = _Info()
        fn = _lib.mg5_relax_patch_graph if graph else _lib.mg5_relax_patch
        dv = self.device
        rc = fn(self._h, _ptr(delta_fine, device=dv), _I3(*pf), ctypes.byref(params),
                compat_c, _ptr(phi_box, device=dv), ctypes.byref(info), _stream(stream))
        if raise_on_status:
            self._check(rc, (OK, W_DISC_CLAMP))
        return phi_box, Info._from(info)

    def relax_patch_masked(self, delta_fine, mask, params: Params, compat_c: float, phi_box,
                           stream=None, raise_on_status=True):
        """mg5_relax_patch_masked: relax only the cells of `mask` (uint8, shape of delta_fine);
        the others keep their values (Sec. 3.3)."""
        pf = list(_box(delta_fine, "delta_fine"))
        if mask is None or phi_box is None:
            raise MG5Error(E_ARG, "mask and phi_box are required")
        _want(mask, pf, "mask")
        _want(phi_box, [x + 2 for x in pf], "phi_box")
        info = _Info()
        dv = self.device
        rc = _lib.mg5_relax_patch_masked(self._h, _ptr(delta_fine, device=dv), _I3(*pf),
                                         _ptr(mask, "uint8", device=dv), ctypes.byref(params),
                                         compat_c, _ptr(phi_box, device=dv), ctypes.byref(info),
                                         _stream(stream))
        if raise_on_status:
            self._check(rc, (OK, W_DISC_CLAMP))
        return phi_box, Info._from(info)

    def parent_force_mask(self, grad_phi, grad_gr, origin, pn, theta: float, periodic=True,
                          out=None, count=False, stream=None):
        """mg5_parent_force_mask: uint8 mask of the (2 pn) fine interior, 1 where
        |grad(phi)/2| > theta |grad(Psi_GR)| at the parent cell (gradients (3, *pd) on the
        periodic domain, or on a refinement's interior with periodic=False).  Returns the
        mask, or (mask, number of ones) with count=True."""
        import torch
        gd = _dims(grad_phi)
        if len(gd) != 4 or gd[0] != 3:
            raise MG5Error(E_ARG, "grad_phi must have shape (3, d0, d1, d2), got %s" % (gd,))
        _want(grad_gr, gd, "grad_gr")
        pd = list(gd[1:])
        dims = [2 * int(p) for p in pn]
        _want(out, dims, "out")
        if out is None:
            out = torch.empty(dims, dtype=torch.uint8, device=grad_phi.device)
        n = ctypes.c_longlong(0)
        dv = self.device
        self._check(_lib.mg5_parent_force_mask(self._h, _ptr(grad_phi, device=dv),
                                               _ptr(grad_gr, device=dv), _I3(*pd),
                                               1 if periodic else 0, _I3(*origin), _I3(*pn),
                                               theta, _ptr(out, "uint8", device=dv),
                                               ctypes.byref(n) if count else None,
                                               _stream(stream)))
        return (out, int(n.value)) if count else out

    # ------------------------------------------------------------ single steps
    def _cubes(self, n, **tensors):
        """Every given tensor (None passes) must be n x n x n."""
        for name, t in tensors.items():
            _want(t, (n, n, n), name)

    def step_sweep(self, phi_in, f, c: float, h: float, alpha: float, out=None, stream=None):
        import torch
        n = _cube(phi_in, "phi_in")
        self._cubes(n, f=f, out=out)
        out = torch.empty_like(phi_in) if out is None else out
        dv = self.device
        self._check(_lib.mg5_step_sweep(self._h, _ptr(phi_in, device=dv), _ptr(out, device=dv),
                                        _ptr(f, device=dv), c, n, h, alpha, _stream(stream)))
        return out

    def step_sweep_fused(self, phi_in, f, c: float, h: float, alpha: float, out=None, stream=None):
        import torch
        n = _cube(phi_in, "phi_in")
        self._cubes(n, f=f, out=out)
        out = torch.empty_like(phi_in) if out is None else out
        dv = self.device
        self._check(_lib.mg5_step_sweep_fused(self._h, _ptr(phi_in, device=dv),
                                              _ptr(out, device=dv), _ptr(f, device=dv), c, n, h,
                                              alpha, _stream(stream)))
        return out

    def step_sweep_f32(self, e_in, f, c: float, h: float, alpha: float, base=None, fused=False,
                       out=None, stream=None):
        """mg5_step_sweep_f32; fused: False/0 two-pass, True/1 fused, 2 column march."""
        import torch
        n = _cube(e_in, "e_in")
        self._cubes(n, f=f, base=base, out=out)
        out = torch.empty_like(e_in) if out is None else out
        dv = self.device
        self._check(_lib.mg5_step_sweep_f32(self._h, _ptr(e_in, "float32", dv),
                                            _ptr(out, "float32", dv), _ptr(f, "float32", dv),
                                            _ptr(base, "float32", dv), c, n, h, alpha,
                                            int(fused), _stream(stream)))
        return out

    def step_resid_restrict_f32(self, e, f, base, c: float, h: float, alpha: float, march=False,
                                stream=None):
        """mg5_step_resid_restrict_f32: (R e, R r, (mean r, ||r - mean r||)) of the FP32
        correction equation's residual r = f + c - (op(B + e) - op(B))."""
        import torch
        n = _cube(e, "e")
        self._cubes(n, f=f, base=base)
        if base is None:
            raise MG5Error(E_ARG, "base is required")
        ec = torch.empty((n // 2,) * 3, dtype=torch.float32, device=e.device)
        rc = torch.empty_like(ec)
        st = (_c_double * 2)()
        dv = self.device
        self._check(_lib.mg5_step_resid_restrict_f32(
            self._h, _ptr(e, "float32", dv), _ptr(f, "float32", dv), _ptr(base, "float32", dv), c,
            n, h, alpha, 1 if march else 0, _ptr(ec, "float32", dv), _ptr(rc, "float32", dv), st,
            _stream(stream)))
        return ec, rc, (st[0], st[1])

    def step_operator(self, phi, h: float, alpha: float, out=None, stream=None):
        import torch
        n = _cube(phi, "phi")
        self._cubes(n, out=out)
        out = torch.empty_like(phi) if out is None else out
        dv = self.device
        self._check(_lib.mg5_step_operator(self._h, _ptr(phi, device=dv), n, h, alpha,
                                           _ptr(out, device=dv), _stream(stream)))
        return out

    def step_residual(self, phi, f, c: float, h: float, alpha: float, out=None, stream=None):
        import torch
        n = _cube(phi, "phi")
        self._cubes(n, f=f, out=out)
        out = torch.empty_like(phi) if out is None else out
        dv = self.device
        self._check(_lib.mg5_step_residual(self._h, _ptr(phi, device=dv), _ptr(f, device=dv), c, n,
                                           h, alpha, _ptr(out, device=dv), _stream(stream)))
        return out

    def step_restrict(self, fine, out=None, stream=None):
        import torch
        n = _cube(fine, "fine")
        if n % 2:
            raise MG5Error(E_ARG, "fine grid side %d is odd" % n)
        self._cubes(n // 2, out=out)
        out = torch.empty((n // 2,) * 3, dtype=fine.dtype, device=fine.device) if out is None else out
        dv = self.device
        self._check(_lib.mg5_step_restrict(self._h, _ptr(fine, device=dv), n, _ptr(out, device=dv),
                                           _stream(stream)))
        return out

    def step_prolong_add(self, coarse, fine, stream=None):
        nc = _cube(coarse, "coarse")
        self._cubes(2 * nc, fine=fine)
        dv = self.device
        self._check(_lib.mg5_step_prolong_add(self._h, _ptr(coarse, device=dv), nc,
                                              _ptr(fine, device=dv), _stream(stream)))
        return fine


@dataclass
class Completion:
    tag: int
    status: int
    t_submit: float
    t_admit: float
    t_done: float
    info: Info


class Server:
    """mg5_server: continuous-batching solves on `slots` workers (own context + stream
    each), admitted in arrival order by HBM footprint.  Tensors passed to submit()
    must stay alive until their completion is polled."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget_bytes: int = 0):
        self._h = _c_void_p()
        rc = _lib.mg5_server_create(ctypes.byref(self._h), device, slots, hbm_budget_bytes)
        if rc != OK:
            raise MG5Error(rc, "mg5_server_create failed")
        self.device = device
        self._keep = {}

    def submit(self, delta, params: Params, phi, grad=None, tag: int = 0):
        n = _cube(delta, "delta")
        if phi is None:
            raise MG5Error(E_ARG, "phi is required")
        _want(phi, (n, n, n), "phi")
        _want(grad, (3, n, n, n), "grad")
        dv = self.device
        req = _Request(_ptr(delta, device=dv), n, params, _ptr(phi, device=dv),
                       _ptr(grad, device=dv), tag)
        rc = _lib.mg5_server_submit(self._h, ctypes.byref(req))
        if rc != OK:
            raise MG5Error(rc, "submit rejected")
        self._keep[tag] = (delta, phi, grad)

    def poll(self, max_n: int = 64, wait_ms: int = 0):
        buf = (_Completion * max_n)()
        n = _lib.mg5_server_poll(self._h, buf, max_n, wait_ms)
        if n < 0:
            raise MG5Error(n, "poll failed")
        out = []
        for c in buf[:n]:
            self._keep.pop(c.tag, None)
            out.append(Completion(c.tag, c.status, c.t_submit, c.t_admit, c.t_done, Info._from(c.info)))
        return out

    def pending(self):
        q, r = _c_int(), _c_int()
        _lib.mg5_server_pending(self._h, ctypes.byref(q), ctypes.byref(r))
        return q.value, r.value

    def clock(self) -> float:
        return _lib.mg5_server_clock(self._h)

    def bytes_held(self) -> int:
        return _lib.mg5_server_bytes_held(self._h)

    def stats(self) -> dict:
        """mg5_server_get_stats: builds, evictions, fallbacks, memory waits, completed, build seconds."""
        st = _ServerStats()
        rc = _lib.mg5_server_get_stats(self._h, ctypes.byref(st))
        if rc != OK:
            raise MG5Error(rc, "server stats")
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def close(self):
        if self._h:
            _lib.mg5_server_destroy(self._h)
            self._h = _c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def residual_norm_noalloc(phi, f, c: float, h: float, alpha: float, out=None, stream=None):
    """mg5_residual_norm_noalloc: (mean r, ||r - mean r||, ||r||) of r = f + c - op(phi) into a
    3-element float64 device tensor, with no device allocation by the library (its partial
    sums live in a fixed device array; N^3 <= residual_norm_noalloc_max_cells())."""
    import torch
    n = _cube(phi, "phi")
    _want(f, (n, n, n), "f")
    _want(out, (3,), "out")
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=phi.device)
    dv = phi.device.index or 0
    rc = _lib.mg5_residual_norm_noalloc(_ptr(phi), _ptr(f, device=dv), c, n, h, alpha,
                                        _ptr(out, device=dv), _stream(stream))
    if rc != OK:
        raise MG5Error(rc, "residual_norm_noalloc")
    return out


def residual_norm_noalloc_max_cells() -> int:
    return _lib.mg5_residual_norm_noalloc_max_cells()


def _host_ptr(a):
    """Host pointer of a C-contiguous float64 numpy array or CPU tensor (None -> NULL)."""
    if a is None:
        return None
    try:
        import numpy as np
        if isinstance(a, np.ndarray):
            if not (a.dtype == np.float64 and a.flags.c_contiguous):
                raise TypeError("expected a C-contiguous float64 array")
            return a.ctypes.data
    except ImportError:
        pass
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous():
        return a.data_ptr()
    raise TypeError("expected a host float64 buffer")


__all__ = ["Context", "Server", "Completion", "Params", "Info", "MG5Error", "default_params",
           "ndgp_coefficients",
           "workspace_bytes", "status_string", "version", "FP64", "MIXED"]
