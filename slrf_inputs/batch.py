"""The batched workload: many independent, uneven scalar Q1 pencils.

64 problems (seed 4): each a 2D or 3D (coin flip) Q1 Laplacian + consistent mass on a
unit box, Dirichlet on the x = 0 face, per-element stiffness coefficients lognormal(0, 0.3),
size n drawn log-uniform in [5k, 200k] (grid nodes per axis from n), a wanted count
K ~ U{10..60}, block L = ceil(1.5 K), m = 8 poles.

gamma of each problem is the midpoint of the spectral gap after its K-th eigenvalue;
the eigenvalues come from scipy's shift-invert Lanczos (library routine, run once by
`python -m slrf_inputs.batch` and stored in batch_gammas.json next to this file).
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass

import numpy as np

from . import fem

HERE = os.path.dirname(os.path.abspath(__file__))
GAMMA_FILE = os.path.join(HERE, "batch_gammas.json")


@dataclass
class BatchSpec:
    index: int
    dim: int
    nodes: tuple
    K: int
    L: int
    seed: int


def batch_specs(P: int = 64, seed: int = 4, n_lo: float = 5e3, n_hi: float = 2e5):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(P):
        dim = 2 if rng.random() < 0.5 else 3
        n_target = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        K = int(rng.integers(10, 61))
        side = int(round(n_target ** (1.0 / dim)))
        # Dirichlet on one face removes one layer of nodes
        nodes = (side + 1,) + (side,) * (dim - 1)
        specs.append(BatchSpec(i, dim, nodes, K, int(np.ceil(1.5 * K)), seed * 1000 + i))
    return specs


def batch_pencil(spec: BatchSpec) -> fem.CsrPair:
    ne = int(np.prod([s - 1 for s in spec.nodes]))
    coef = np.exp(np.random.default_rng(spec.seed).normal(0.0, 0.3, ne))
    return fem.q1_scalar(spec.nodes, coef=coef, dirichlet_face=(0, 0))


def batch_gammas():
    """gamma and count per problem from the stored table (raises if it was not generated)."""
    with open(GAMMA_FILE) as fh:
        tab = json.load(fh)
    return [(t["gamma"], t["count"]) for t in tab["problems"]]


def _one_gamma(spec: BatchSpec):
    import scipy.sparse.linalg as spla

    p = batch_pencil(spec)
    A, B = p.A().tocsc(), p.B().tocsc()
    k = min(spec.K + 14, 74)
    # shift-invert at 0 with a symmetric minimum-degree ordering of A's factorisation
    lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))
    opinv = spla.LinearOperator(A.shape, matvec=lu.solve, dtype=np.float64)
    vals = spla.eigsh(A, k=k, M=B, sigma=0.0, which="LM", OPinv=opinv, return_eigenvectors=False, tol=1e-12)
    lam = np.sort(vals)
    # gamma in the clear gap (>= 0.5 % of the upper eigenvalue) nearest to K eigenvalues, the
    # count kept within 10..60
    rel = np.diff(lam) / lam[1:]
    cand = [g for g in range(9, min(len(lam) - 1, 60)) if rel[g] >= 5e-3]
    if not cand:
        cand = [int(np.argmax(rel[9:60])) + 9]
    g = min(cand, key=lambda c: abs(c + 1 - spec.K))
    return {"index": spec.index, "dim": spec.dim, "nodes": list(spec.nodes), "n": p.n, "nnz": p.nnz,
            "K": spec.K, "count": int(g + 1), "gamma": float(0.5 * (lam[g] + lam[g + 1])),
            "rel_gap": float(rel[g]), "L": spec.L, "lambda": [float(x) for x in lam]}


def _compute_gammas(P: int = 64, seed: int = 4, workers: int = 6):
    import multiprocessing as mp

    specs = batch_specs(P, seed)
    with mp.get_context("spawn").Pool(workers) as pool:
        out = pool.map(_one_gamma, specs, chunksize=1)
    for o in out:
        print({k: v for k, v in o.items() if k != "lambda"}, flush=True)
    return out


if __name__ == "__main__":
    probs = _compute_gammas()
    with open(GAMMA_FILE, "w") as fh:
        json.dump({"source": "scipy.sparse.linalg.eigsh shift-invert (sigma = 0, SuperLU MMD_AT_PLUS_A), tol 1e-12; "
                             "gamma in the nearest gap of at least 0.5 %",
                   "problems": probs}, fh, indent=1)
