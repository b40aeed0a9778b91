"""slrf_apply: A X and B X with a context's matrices, in FP64 and in FP32.

The FP32 products go through the grouped-row records of a mixed-precision context (the
same records the COCG SpMM reads, Jacobi-scaled when the preconditioner is on and scaled
back by D^1/2 on both sides) or through the CSR values rounded to FP32.  Reference: the
plain sparse products A @ X, B @ X in FP64 on the host.  Bounds, elementwise:
  FP64: |Y - A X| <= 1e-13 (|A| |X|)
  FP32: |Y - A X| <= 2e-5 (|A| |X|)   (FP32 sums of up to 81 products plus the rounding of
                                        X, the values and the scales to FP32)
Cases: a 3-dof elasticity box with groups of 3 (one node each), with and without the
preconditioner; a scalar Q1 Laplacian on 21^3 nodes (n = 9,261, odd) with groups of 2 and
4, so that the last group is ragged; plain CSR; block widths that leave a ragged column
tile.
"""
import numpy as np
import pytest
import torch

import slrf_inputs as si
from gpu_common import slrf_mod  # noqa: F401
from slrf_inputs import elastic as se

pytestmark = pytest.mark.gpu


def _check(slrf_mod, p, gamma, L, k, precision, precond, group, fp32):
    opts = slrf_mod.slrf_opts_default(it_max=4, precision=precision, precond=precond, group=group)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, opts)
    rng = np.random.default_rng(5 + k)
    X = rng.standard_normal((p.n, k))
    AX, BX = ctx.apply(torch.from_numpy(X), fp32=fp32)
    A_only, _ = ctx.apply(torch.from_numpy(X), fp32=fp32, want_b=False)
    _, B_only = ctx.apply(torch.from_numpy(X), fp32=fp32, want_a=False)
    torch.cuda.synchronize()
    ctx.close()
    tol = 2e-5 if fp32 else 1e-13
    A, B = p.A(), p.B()
    absX = np.abs(X)
    for Y, M in ((AX, A), (BX, B), (A_only, A), (B_only, B)):
        Y = Y.cpu().numpy()
        ref = M @ X
        bound = abs(M) @ absX
        assert np.all(np.abs(Y - ref) <= tol * bound + 1e-300), (np.abs(Y - ref) / bound).max()


@pytest.fixture(scope="module")
def elast():
    p = se.pencil("elast_32")
    gamma, _ = se.gamma("elast_32")
    return p, gamma


@pytest.fixture(scope="module")
def lap21():
    wl = si.q1_lap(21)
    return wl.pencil, wl.gamma


@pytest.mark.parametrize("precond", [1, 0])
@pytest.mark.parametrize("k", [96, 37])
def test_fp32_through_elasticity_records(slrf_mod, elast, precond, k):
    p, gamma = elast
    _check(slrf_mod, p, gamma, 96, k, 1, precond, 3, True)


@pytest.mark.parametrize("group", [2, 4])
def test_fp32_through_ragged_groups(slrf_mod, lap21, group):
    p, gamma = lap21
    assert p.n % group != 0
    _check(slrf_mod, p, gamma, 149, 149, 1, 0, group, True)


def test_fp32_plain_csr(slrf_mod, lap21):
    p, gamma = lap21
    _check(slrf_mod, p, gamma, 149, 70, 1, 0, 1, True)


@pytest.mark.parametrize("precision", [0, 1])
def test_fp64_products(slrf_mod, elast, precision):
    p, gamma = elast
    _check(slrf_mod, p, gamma, 96, 61, precision, 1, 0, False)


def test_argument_errors(slrf_mod, lap21):
    p, gamma = lap21
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, 16, slrf_mod.slrf_opts_default())
    X = torch.ones((p.n, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(slrf_mod.SlrfError) as e:
        ctx.apply(X, want_a=False, want_b=False)
    assert e.value.status == slrf_mod.SLRF_EINVAL
    with pytest.raises(slrf_mod.SlrfError) as e:
        ctx.apply(torch.ones((p.n, 17), dtype=torch.float64, device="cuda"))  # k > L
    assert e.value.status == slrf_mod.SLRF_EINVAL
    ctx.close()
