"""Tall-skinny products of the outer update through the C ABI (slrf_tsgram, slrf_tsgemm).

The reference is the definition of the product, C = X^T Y and Z = alpha X S + beta Z, taken
in FP64 by numpy on the host.  The split-bf16 tensor-core path (mode 1) writes each entry
against the exponent E of its row as 7 base-256 digits (56 bits): the representation error
of x is below 2^(E-57) <= 2^-56 max|x_row|, the digit-level sums of the five leading levels
are exact, so every entry of the product is within n 2^-53 max|x_a| max|y_b| (well inside
the bound asserted below) -- and exactly equal when all inputs are small integers.
"""
import numpy as np
import pytest
import torch

from gpu_common import slrf_mod  # noqa: F401

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _bound(X, Y):
    n = X.shape[0]
    return 4.0 * max(n, 1) * 2.0 ** -53 * np.outer(np.abs(X).max(axis=0, initial=0), np.abs(Y).max(axis=0, initial=0))


def _rand(rng, n, k, spread=0.0):
    X = rng.standard_normal((n, k))
    if spread:
        X *= 10.0 ** rng.uniform(-spread, spread, k)[None, :]
    return X


@pytest.mark.parametrize("n,k1,k2", [(1, 1, 1), (37, 7, 33), (300, 32, 32), (4097, 105, 160), (68921, 160, 160),
                                     (20000, 257, 96)])
def test_tsgram_random_within_fp64_bound(slrf_mod, n, k1, k2):
    rng = np.random.default_rng(n + k1 + k2)
    X, Y = _rand(rng, n, k1, 40), _rand(rng, n, k2, 40)
    ref = X.T @ Y
    for mode in (1, 0):
        C = slrf_mod.tsgram(torch.from_numpy(X).to(DEV), torch.from_numpy(Y).to(DEV), mode=mode).cpu().numpy()
        err = np.abs(C - ref)
        assert np.all(err <= _bound(X, Y)), (mode, float((err / np.maximum(_bound(X, Y), 1e-300)).max()))
        # typical accuracy: relative to |X|^T |Y| the error is at rounding level
        assert float((err / (np.abs(X).T @ np.abs(Y))).max()) < 1e-13, mode


def test_tsgram_same_operand_is_symmetric_and_exact_on_integers(slrf_mod):
    rng = np.random.default_rng(5)
    n, k = 5000, 150
    X = rng.integers(-1000, 1001, size=(n, k)).astype(np.float64)
    X[:, 3] = 0.0  # an all-zero column
    Xd = torch.from_numpy(X).to(DEV)
    C = slrf_mod.tsgram(Xd, Xd, mode=1).cpu().numpy()
    assert np.array_equal(C, X.T @ X)  # integers below 2^31: every step is exact
    Y = rng.integers(-(2 ** 20), 2 ** 20, size=(n, 40)).astype(np.float64)
    C = slrf_mod.tsgram(Xd, torch.from_numpy(Y).to(DEV), mode=1).cpu().numpy()
    assert np.array_equal(C, X.T @ Y)


def test_tsgram_empty_and_nonfinite(slrf_mod):
    X = torch.zeros(0, 5, dtype=torch.float64, device=DEV)
    C = slrf_mod.tsgram(X, X, mode=1).cpu().numpy()
    assert C.shape == (5, 5) and np.all(C == 0)
    rng = np.random.default_rng(1)
    Xh = rng.standard_normal((300, 6))
    Xh[17, 2] = np.nan
    Yh = rng.standard_normal((300, 4))
    C = slrf_mod.tsgram(torch.from_numpy(Xh).to(DEV), torch.from_numpy(Yh).to(DEV), mode=1).cpu().numpy()
    assert np.all(np.isnan(C[2])) and np.all(np.isfinite(np.delete(C, 2, axis=0)))


@pytest.mark.parametrize("n,k1,k2", [(1, 1, 1), (300, 33, 17), (68921, 160, 160), (10000, 512, 40)])
def test_tsgemm_random_within_fp64_bound(slrf_mod, n, k1, k2):
    rng = np.random.default_rng(n * 3 + k1)
    X = rng.standard_normal((n, k1)) * 10.0 ** rng.uniform(-30, 30, n)[:, None]
    S = _rand(rng, k1, k2, 30)
    Z0 = rng.standard_normal((n, k2))
    for alpha, beta in ((1.0, 0.0), (-1.0, 1.0), (0.5, -2.0)):
        ref = alpha * (X @ S) + beta * Z0
        bnd = abs(alpha) * 4.0 * k1 * 2.0 ** -53 * np.outer(np.abs(X).max(axis=1), np.abs(S).max(axis=0)) \
            + 4 * 2.0 ** -53 * np.abs(ref)
        for mode in (1, 0):
            Z = torch.from_numpy(Z0.copy()).to(DEV)
            slrf_mod.tsgemm(torch.from_numpy(X).to(DEV), torch.from_numpy(S).to(DEV), Z, alpha, beta, mode=mode)
            err = np.abs(Z.cpu().numpy() - ref)
            assert np.all(err <= bnd), (mode, alpha, beta)


def test_tsgemm_exact_on_integers(slrf_mod):
    rng = np.random.default_rng(9)
    X = rng.integers(-3000, 3001, size=(70001, 160)).astype(np.float64)
    S = rng.integers(-3000, 3001, size=(160, 160)).astype(np.float64)
    Z = slrf_mod.tsgemm(torch.from_numpy(X).to(DEV), torch.from_numpy(S).to(DEV), mode=1)
    assert np.array_equal(Z.cpu().numpy(), X @ S)
