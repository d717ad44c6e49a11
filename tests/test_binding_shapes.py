"""The Python binding refuses tensors of the wrong shape before any pointer reaches the
library (a buffer smaller than the kernels assume would be read or written past its end).
No GPU: the checks run on CPU tensors, ahead of the device-pointer marshalling."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__ as g
    g.build()
    import paper_1511_08200_gb300 as m
    return m


@pytest.fixture()
def ctx(mg):
    c = mg.Context.__new__(mg.Context)   # no mg5_create: nothing below reaches the library
    c._h = ctypes.c_void_p()
    c.device = 0
    return c


def z(*shape, dtype=torch.float64):
    return torch.zeros(shape, dtype=dtype)


def _arg_error(mg, fn, *a, **kw):
    with pytest.raises(mg.MG5Error) as e:
        fn(*a, **kw)
    assert e.value.code == mg.E_ARG
    return str(e.value)


def test_solve_shapes(mg, ctx):
    p = mg.default_params()
    assert "cube" in _arg_error(mg, ctx.solve_fifth_force, z(8, 8, 6), p)
    assert "cube" in _arg_error(mg, ctx.solve_fifth_force, z(8, 8), p)
    assert "phi" in _arg_error(mg, ctx.solve_fifth_force, z(8, 8, 8), p, phi=z(8, 8, 4))
    assert "grad" in _arg_error(mg, ctx.solve_fifth_force, z(8, 8, 8), p, grad=z(8, 8, 8))
    assert "grad" in _arg_error(mg, ctx.solve_fifth_force, z(8, 8, 8), p, grad=z(3, 8, 8, 6))
    d = np.zeros((8, 8, 8))
    assert "phi" in _arg_error(mg, ctx.solve_fifth_force_host, d, p, phi=np.zeros((8, 8, 7)))
    assert "phi" in _arg_error(mg, ctx.solve_fifth_force_host, d, p)
    assert "grad" in _arg_error(mg, ctx.solve_fifth_force_host, d, p, phi=np.zeros((8, 8, 8)),
                                grad=np.zeros((3, 8, 8)))


def test_batch_shapes(mg, ctx):
    p = mg.default_params()
    ds = [z(8, 8, 8), z(16, 16, 16)]
    _arg_error(mg, ctx.solve_batch, [z(8, 8, 8), z(16, 16, 8)], p)
    assert "phis[1]" in _arg_error(mg, ctx.solve_batch, ds, p, phis=[z(8, 8, 8), z(8, 8, 8)])
    assert "grads[0]" in _arg_error(mg, ctx.solve_batch, ds, p,
                                    phis=[z(8, 8, 8), z(16, 16, 16)],
                                    grads=[z(3, 8, 8, 7), z(3, 16, 16, 16)])
    assert "entries" in _arg_error(mg, ctx.solve_batch, ds, [p])


def test_force_and_refine_shapes(mg, ctx):
    assert "grad" in _arg_error(mg, ctx.force, z(10, 10, 10), 1.0, ghost=1, grad=z(3, 10, 10, 10))
    assert "interior" in _arg_error(mg, ctx.force, z(2, 4, 4), 1.0, ghost=1)
    _arg_error(mg, ctx.force, z(4, 4), 1.0)
    for fn in (ctx.refine_interpolate, ctx.refine_interpolate_cubic):
        _arg_error(mg, fn, z(16, 16, 8), (0, 0, 0), (4, 4, 4), 1)
        assert "out" in _arg_error(mg, fn, z(16, 16, 16), (0, 0, 0), (4, 4, 4), 1, out=z(8, 8, 8))
    assert "out" in _arg_error(mg, ctx.refine_interpolate_box, z(10, 10, 10), 1, (0, 0, 0),
                               (4, 4, 4), 1, out=z(10, 10, 9))
    _arg_error(mg, ctx.refine_interpolate_box, z(10, 10), 1, (0, 0, 0), (4, 4, 4), 1)


def test_patch_shapes(mg, ctx):
    p = mg.default_params()
    assert "phi_box" in _arg_error(mg, ctx.relax_patch, z(8, 8, 8), p, 0.0, z(9, 10, 10))
    assert "phi_box" in _arg_error(mg, ctx.relax_patch, z(8, 8, 8), p, 0.0, None)
    assert "mask" in _arg_error(mg, ctx.relax_patch_masked, z(8, 8, 8), z(8, 8, 4, dtype=torch.uint8),
                                p, 0.0, z(10, 10, 10))
    assert "phi_box" in _arg_error(mg, ctx.relax_patch_masked, z(8, 8, 8),
                                   z(8, 8, 8, dtype=torch.uint8), p, 0.0, z(10, 10, 8))
    g = z(3, 16, 16, 16)
    assert "grad_gr" in _arg_error(mg, ctx.parent_force_mask, g, z(3, 16, 16, 8), (0, 0, 0),
                                   (4, 4, 4), 0.1)
    assert "grad_phi" in _arg_error(mg, ctx.parent_force_mask, z(16, 16, 16), z(16, 16, 16),
                                    (0, 0, 0), (4, 4, 4), 0.1)
    assert "out" in _arg_error(mg, ctx.parent_force_mask, g, g, (0, 0, 0), (4, 4, 4), 0.1,
                               out=z(8, 8, 4, dtype=torch.uint8))


def test_single_step_shapes(mg, ctx):
    a, b = z(8, 8, 8), z(8, 8, 4)
    assert "f" in _arg_error(mg, ctx.step_sweep, a, b, 0.0, 1.0, 0.1)
    assert "out" in _arg_error(mg, ctx.step_sweep_fused, a, a, 0.0, 1.0, 0.1, out=b)
    f32 = lambda *s: z(*s, dtype=torch.float32)   # noqa: E731
    assert "base" in _arg_error(mg, ctx.step_sweep_f32, f32(8, 8, 8), f32(8, 8, 8), 0.0, 1.0, 0.1,
                                base=f32(8, 8, 6))
    assert "out" in _arg_error(mg, ctx.step_operator, a, 1.0, 0.1, out=b)
    assert "f" in _arg_error(mg, ctx.step_residual, a, b, 0.0, 1.0, 0.1)
    assert "out" in _arg_error(mg, ctx.step_restrict, a, out=z(8, 8, 8))
    assert "odd" in _arg_error(mg, ctx.step_restrict, z(7, 7, 7))
    assert "fine" in _arg_error(mg, ctx.step_prolong_add, z(4, 4, 4), z(4, 4, 4))


def test_noalloc_and_server_shapes(mg):
    a = z(8, 8, 8)
    assert "f" in _arg_error(mg, mg.residual_norm_noalloc, a, z(8, 8, 4), 0.0, 1.0, 0.1)
    assert "out" in _arg_error(mg, mg.residual_norm_noalloc, a, a, 0.0, 1.0, 0.1, out=z(2))
    _arg_error(mg, mg.residual_norm_noalloc, z(8, 4, 8), a, 0.0, 1.0, 0.1)
    srv = mg.Server.__new__(mg.Server)
    srv._h = ctypes.c_void_p()
    srv.device = 0
    srv._keep = {}
    p = mg.default_params()
    assert "phi" in _arg_error(mg, srv.submit, a, p, z(8, 8, 6))
    assert "grad" in _arg_error(mg, srv.submit, a, p, a, grad=z(3, 8, 8))
    assert "cube" in _arg_error(mg, srv.submit, z(8, 8, 6), p, a)
