"""Q1 linear-elasticity workloads (3 dof/node, z = 0 face clamped, Young's modulus
lognormal per element, nu = 0.3, rho = 1) with gamma placed in a spectral gap.

* elast_32: 32 x 32 x 16 nodes (n = 46,080), 60 eigenvalues, block 96, E ~ lognormal(0, 0.5),
  seed 3 -- a reduced instance of the 64 x 64 x 32 box.
* elast_48: 48 x 48 x 48 nodes (n = 324,864), 50 eigenvalues, block 80, element
  stiffness parameters p_e ~ lognormal(0, 0.5), seed 5 -- the sensitivity workload.
* elast_64: 64 x 64 x 32 nodes (n = 380,928, nnz = 29.6M), 300 eigenvalues, block 480,
  E ~ lognormal(0, 0.5), seed 3 -- the full-size elasticity box.

gamma: midpoint of a gap after about the K-th eigenvalue of a shift-invert Lanczos
spectrum (scipy, run once by `python -m slrf_inputs.elastic NAME`, stored in
elastic_gammas.json): for K < 100 the gap nearest to K of relative width >= 1e-4, for
larger K the widest relative gap with a count in K - 5 .. K + 5.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

from . import fem

HERE = os.path.dirname(os.path.abspath(__file__))
GAMMA_FILE = os.path.join(HERE, "elastic_gammas.json")

SPECS = {
    "elast_32": {"nodes": (32, 32, 16), "K": 60, "block": 96, "seed": 3},
    "elast_48": {"nodes": (48, 48, 48), "K": 50, "block": 80, "seed": 5},
    "elast_64": {"nodes": (64, 64, 32), "K": 300, "block": 480, "seed": 3},
}


def element_params(name: str) -> np.ndarray:
    s = SPECS[name]
    ne = int(np.prod([x - 1 for x in s["nodes"]]))
    return np.exp(np.random.default_rng(s["seed"]).normal(0.0, 0.5, ne))


def pencil(name: str, params: np.ndarray | None = None) -> fem.CsrPair:
    s = SPECS[name]
    E = element_params(name) if params is None else params
    return fem.q1_elasticity(s["nodes"], E=E, nu=0.3, rho=1.0, clamp_face=(2, 0))


def gamma(name: str):
    with open(GAMMA_FILE) as fh:
        t = json.load(fh)[name]
    return t["gamma"], t["count"]


def _compute(name: str):
    import scipy.sparse.linalg as spla

    s = SPECS[name]
    p = pencil(name)
    A, B = p.A().tocsc(), p.B().tocsc()
    lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))
    opinv = spla.LinearOperator(A.shape, matvec=lu.solve, dtype=np.float64)
    K = s["K"]
    vals = spla.eigsh(A, k=K + max(8, K // 10), M=B, sigma=0.0, which="LM", OPinv=opinv,
                      return_eigenvectors=False, tol=1e-12)
    lam = np.sort(vals)
    rel = np.diff(lam) / lam[1:]
    if K < 100:
        gaps = np.nonzero(rel > 1e-4)[0]
        g = gaps[np.argmin(np.abs(gaps + 1 - K))]
    else:
        cand = np.arange(K - 6, K + 5)  # gap after eigenvalue g + 1, count g + 1 in K - 5 .. K + 5
        g = cand[np.argmax(rel[cand])]
    out = {"n": p.n, "nnz": p.nnz, "count": int(g + 1), "gamma": float(0.5 * (lam[g] + lam[g + 1])),
           "rel_gap": float((lam[g + 1] - lam[g]) / lam[g + 1]), "lambda_min": float(lam[0]),
           "source": "scipy eigsh shift-invert (SuperLU MMD_AT_PLUS_A), tol 1e-12"}
    if K >= 100:
        out["lambdas"] = [float(v) for v in lam]
    return out


if __name__ == "__main__":
    names = sys.argv[1:] or list(SPECS)
    tab = {}
    if os.path.exists(GAMMA_FILE):
        with open(GAMMA_FILE) as fh:
            tab = json.load(fh)
    for nm in names:
        tab[nm] = _compute(nm)
        print(nm, tab[nm], flush=True)
        with open(GAMMA_FILE, "w") as fh:
            json.dump(tab, fh, indent=1)
