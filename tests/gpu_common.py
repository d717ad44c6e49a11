"""Shared fixtures for the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def ctx_fixture():
    need_gpu()
    import paper_1511_08200_gb300 as mg
    return mg.Context(0)


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_l2(a, b) -> float:
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


# nominal nDGP coefficients at a = 1, Omega_m = 0.3, H0 r_c = 1 (eps = alpha s = 0.0137)
def nominal():
    import oracle
    beta, alpha, s = oracle.ndgp_coefficients(1.0, 0.3, 1.0)
    return alpha, s, 250.0 / 512
