"""The range-checked build (-DMG5_BOUNDS): under MG5_BOUNDS=1 the binding loads
libmg5_bounds.so, and every GPU test ends by reading its record of out-of-range element
accesses (tests/conftest.py).  This file checks that the loaded library is the one asked
for and that a small solve through every kernel family of the FP64 and mixed paths leaves
no record."""
import os

import numpy as np
import pytest

import workload
from tests.gpu_common import ctx_fixture, dev, nominal

pytestmark = pytest.mark.gpu


def test_loaded_library_matches_the_request():
    import torch
    import paper_1511_08200_gb300 as mg
    want = os.environ.get("MG5_BOUNDS", "0") == "1"
    assert mg.bounds_build() == want
    alpha, s, h = nominal()
    ctx = ctx_fixture()
    d = dev(workload.lognormal_delta(32, 1.0, 11))
    for prec in ("fp64", "mixed"):
        p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-8, precision=prec)
        grad = torch.empty((3, 32, 32, 32), dtype=torch.float64, device="cuda")
        phi, _, info = ctx.solve_fifth_force(d, p, grad=grad)
        assert info.status == 0 and np.isfinite(info.rel_residual)
    torch.cuda.synchronize()
    assert mg.bounds_check() is None
    ctx.close()
