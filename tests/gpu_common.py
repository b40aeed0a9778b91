"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import numpy as np
import pytest


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="session")
def slrf_mod():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__ as ge

    ge.build()
    from paper_2510_17334_gb300 import slrf

    return slrf


def cluster_projector_error(X, Y, B, lam, rtol=1e-8):
    """Max over eigenvalue clusters of || X_c X_c^T B - Y_c Y_c^T B ||, applied to random
    probes: compares eigenvectors up to sign and rotation inside degenerate clusters."""
    lam = np.asarray(lam)
    rng = np.random.default_rng(0)
    probe = rng.standard_normal((X.shape[0], 4))
    worst = 0.0
    i = 0
    while i < len(lam):
        j = i + 1
        while j < len(lam) and abs(lam[j] - lam[i]) <= rtol * abs(lam[i]):
            j += 1
        Px = X[:, i:j] @ (X[:, i:j].T @ (B @ probe))
        Py = Y[:, i:j] @ (Y[:, i:j].T @ (B @ probe))
        worst = max(worst, float(np.abs(Px - Py).max() / np.abs(Py).max()))
        i = j
    return worst
