"""The residual-norm entry point that allocates no device memory, for callers that
cannot call cudaMalloc (memory pools they do not own, regions where an allocation
would synchronise or break a capture, hosts that only lend their own buffers).

Collected last on purpose: it checks the fixed-array variant against the existing
residual entry point (mg5_step_residual, whose r is reduced here with torch), on
two calls in a row, with the same 1e-13 relative tolerance as the other residual
tests; and that a grid beyond the fixed array is refused.
"""
import numpy as np
import pytest

import workload
from tests.gpu_common import dev, need_gpu, nominal

pytestmark = pytest.mark.gpu


def _reference(ctx, phi, f, c, h, alpha):
    r = ctx.step_residual(phi, f, c, h, alpha)
    m = r.mean()
    return np.array([float(m), float((r - m).norm()), float(r.norm())])


def test_residual_norm_noalloc_matches_existing_entry_point():
    need_gpu()
    import torch
    import paper_1511_08200_gb300 as mg
    alpha, s, h = nominal()
    ctx = mg.Context(0)
    for n in (16, 48, 128):
        phi = dev(workload.smooth_periodic_field(n, 1e-6, 3) + 1e-7 * workload.lognormal_delta(n, 1.0, 4))
        f = dev(s * workload.lognormal_delta(n, 1.0, 5))
        c = 2e-11
        ref = _reference(ctx, phi, f, c, h, alpha)
        out = torch.empty(3, dtype=torch.float64, device="cuda")
        for _ in range(2):   # two calls in a row share the fixed array
            out.fill_(float("nan"))
            mg.residual_norm_noalloc(phi, f, c, h, alpha, out=out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref).max()), (n, got, ref)
    ctx.close()


def test_residual_norm_noalloc_rejects_too_large():
    need_gpu()
    import torch
    import paper_1511_08200_gb300 as mg
    assert mg.residual_norm_noalloc_max_cells() == 8192 * 256
    n = 130                                   # 130^3 > 2,097,152
    z = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MG5Error) as e:
        mg.residual_norm_noalloc(z, z, 0.0, 1.0, 0.1)
    assert e.value.code == mg.E_TOO_LARGE
