"""The sweep-schedule autotuner on the GPU: it records a timed schedule for every
grid side of a hierarchy, and every schedule gives the same solution."""
import numpy as np
import pytest

import workload
from tests.gpu_common import ctx_fixture, dev, host, nominal

pytestmark = pytest.mark.gpu


@pytest.fixture
def mg():
    import paper_1511_08200_gb300 as m
    m.tune_clear()
    yield m
    m.tune_clear()


def _sides(n):
    out = []
    while n % 2 == 0 and n // 2 >= 4:
        out.append(n)
        n //= 2
    return out   # every side but the coarsest


def test_autotune_records_every_side(mg, tmp_path):
    ctx = ctx_fixture()
    for prec in ("fp64", "mixed"):
        ctx.autotune(64, prec)
        for n in _sides(64):
            s, tuned = mg.schedule_get(0, prec, n)
            assert tuned and s.ms > 0, (prec, n)
    path = tmp_path / "t.jsonl"
    mg.tune_save(path)
    kept = {(p, n): mg.schedule_get(0, p, n)[0] for p in ("fp64", "mixed") for n in _sides(64)}
    mg.tune_clear()
    assert mg.tune_load(path) == len(kept)
    for (p, n), s in kept.items():
        t, tuned = mg.schedule_get(0, p, n)
        assert tuned and (t.form, t.block, t.chunk) == (s.form, s.block, s.chunk)
    ctx.close()


def _solve(ctx, mg, d, prec, tol):
    alpha, s, h = nominal()
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision=prec)
    phi, _, info = ctx.solve_fifth_force(d, p)
    return host(phi), info


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-11, 1e-12), ("mixed", 1e-8, 1e-7)])
def test_every_schedule_gives_the_same_solution(mg, prec, tol, bar):
    ctx = ctx_fixture()
    n = 64
    d = dev(workload.lognormal_delta(n, 1.0, 21))
    ref, iref = _solve(ctx, mg, d, prec, tol)
    scale = np.abs(ref).max()
    schedules = [dict(form=mg.SWEEP_TWO_PASS, block=b) for b in (64, 128, 512)]
    schedules += [dict(form=mg.SWEEP_FUSED, chunk=c) for c in (8, 16, 32)]
    schedules += [dict(form=mg.SWEEP_MARCH, chunk=c) for c in (0, 7, 20, 64)]
    for sch in schedules:
        mg.tune_clear()
        for m in _sides(n):
            mg.schedule_set(0, prec, m, **sch)
        got, info = _solve(ctx, mg, d, prec, tol)
        assert info.status in (0, 1)
        assert np.abs(got - ref).max() <= bar * scale, (sch, np.abs(got - ref).max() / scale)
        assert abs(info.cycles - iref.cycles) <= 1
    ctx.close()


def test_autotune_on_first_use_and_in_batch(mg):
    ctx = ctx_fixture()
    ctx.set_autotune(True)
    alpha, s, h = nominal()
    d = dev(workload.lognormal_delta(48, 1.0, 5))
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-8, precision="mixed")
    phi, _, info = ctx.solve_fifth_force(d, p)
    assert info.status in (0, 1)
    assert all(mg.schedule_get(0, "mixed", m)[1] for m in _sides(48))
    # a batch capture tunes the sides of its boxes before capturing
    boxes = [dev(workload.lognormal_delta(m, 1.0, 6 + m)) for m in (32, 64)]
    _, _, infos = ctx.solve_batch(boxes, p)
    assert all(i.status in (0, 1) for i in infos)
    assert all(mg.schedule_get(0, "mixed", m)[1] for m in _sides(32) + _sides(64))
    assert not mg.schedule_get(0, "fp64", 64)[1]     # only the precision that ran
    ctx.close()


@pytest.mark.parametrize("n", [64, 96])
def test_march_schedule_solve_is_bit_identical(mg, n):
    """A mixed solve whose FP32 sweeps run as column marches (chunks of 7, 20 and 64 planes,
    and the automatic one) equals, to the bit, the same solve with the fused sweep."""
    ctx = ctx_fixture()
    d = dev(workload.lognormal_delta(n, 1.5, 41))
    for m in _sides(n):
        mg.schedule_set(0, "mixed", m, form=mg.SWEEP_FUSED, chunk=16)
    ref, iref = _solve(ctx, mg, d, "mixed", 1e-8)
    for c in (0, 7, 20, 64):
        mg.tune_clear()
        for m in _sides(n):
            mg.schedule_set(0, "mixed", m, form=mg.SWEEP_MARCH, chunk=c)
        got, info = _solve(ctx, mg, d, "mixed", 1e-8)
        assert np.array_equal(got, ref) and info.cycles == iref.cycles, c
    ctx.close()
