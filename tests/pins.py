"""Independent references that pin the oracle: closed-form FEM spectra and Sylvester
inertia counts.  Nothing here calls the oracle or the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def bar1d_eigs(n: int) -> np.ndarray:
    """Eigenvalues of the Dirichlet 1D linear-FEM bar with n interior nodes, h = 1/(n+1):
    lambda_k = 6 (1 - cos k pi h) / (h^2 (2 + cos k pi h)), eigenvector sin(k pi x_i)."""
    h = 1.0 / (n + 1)
    k = np.arange(1, n + 1)
    c = np.cos(k * np.pi * h)
    return 6.0 * (1.0 - c) / (h * h * (2.0 + c))


def neumann1d_eigs(nodes: int, length: float = 1.0) -> np.ndarray:
    """Eigenvalues of the Neumann 1D linear-FEM pencil on ``nodes`` nodes (k = 0..nodes-1)."""
    ne = nodes - 1
    h = length / ne
    c = np.cos(np.arange(nodes) * np.pi / ne)
    return 6.0 * (1.0 - c) / (h * h * (2.0 + c))


def q1_neumann_eigs(nodes, shift: float = 0.0) -> np.ndarray:
    """Tensor-product spectrum of the Q1 Neumann Laplacian pencil (+ shift), sorted."""
    ev = np.zeros(1)
    for s in nodes:
        ev = (ev[:, None] + neumann1d_eigs(s)[None, :]).ravel()
    return np.sort(ev) + shift


def sturm_count(d, e, gamma, db, eb) -> int:
    """Number of eigenvalues < gamma of the symmetric tridiagonal pencil (T_A, T_B) with
    diagonals d, db and off-diagonals e, eb: negative pivots of LDL^T of T_A - gamma T_B."""
    a = np.asarray(d) - gamma * np.asarray(db)
    o = np.asarray(e) - gamma * np.asarray(eb)
    cnt = 0
    piv = a[0]
    cnt += piv < 0
    for i in range(1, len(a)):
        piv = a[i] - o[i - 1] ** 2 / piv
        cnt += piv < 0
    return int(cnt)


def dense_inertia_count(A, B, gamma) -> int:
    """Negative eigenvalues of D in the Bunch-Kaufman LDL^T of A - gamma B (Sylvester)."""
    M = np.asarray(A.toarray() if hasattr(A, "toarray") else A) - gamma * np.asarray(
        B.toarray() if hasattr(B, "toarray") else B)
    _, D, _ = sla.ldl(M)
    return int(np.sum(np.linalg.eigvalsh(D) < 0))


def gap_gamma(evals: np.ndarray, want: int, rel_gap: float = 1e-6):
    """Midpoint gamma between the cluster closest to ``want`` eigenvalues and the next one."""
    lam = np.sort(evals)
    gaps = np.nonzero(np.diff(lam) > rel_gap * lam[1:])[0]
    g = gaps[np.argmin(np.abs(gaps + 1 - want))]
    return 0.5 * (lam[g] + lam[g + 1]), int(g + 1)
