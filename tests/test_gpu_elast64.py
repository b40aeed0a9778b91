"""The 64 x 64 x 32 Q1 elasticity box (n = 380,928, 29.6M entries, 3 dof/node, lognormal
modulus), the bench workload, at the settings its bench line uses.

Reference values come from oracle/ only (tests/golden/make_elast64.py): the 330 lowest
eigenvalues by shift-invert Lanczos and the count below gamma by Sylvester's law of inertia
(a symmetric sparse LU of A - gamma B).  Checks:
  * mixed path (complex-FP32 inner solves, Jacobi-preconditioned, It_max 23): the count
    equals the inertia count, every eigenvalue within 1e-8 of the reference, residuals
    <= 1e-8, B-orthonormal vectors;
  * FP64 filter apply of the whole 480-column block, compared on sampled columns with the
    oracle's filter (same preconditioned systems, It_max 4), element by element at the
    1e-8 of the other FP64 parity tests.
"""
import json
import os

import numpy as np
import pytest
import torch

import slrf_inputs as si
from gpu_common import rel, slrf_mod  # noqa: F401
from oracle import slrf_oracle as orc
from slrf_inputs import elastic as se

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def box():
    p = se.pencil("elast_64")
    gamma, _ = se.gamma("elast_64")
    with open(os.path.join(GOLD, "elast_64_spectrum.json")) as fh:
        lam = np.array(json.load(fh)["lambdas"])
    return p, gamma, lam


@pytest.fixture(scope="module")
def count(box):
    _, gamma, _ = box
    with open(os.path.join(GOLD, "elast_64_count.json")) as fh:
        cnt = json.load(fh)
    assert cnt["inertia_symmetric_ordering"] and abs(cnt["gamma"] - gamma) == 0.0
    return cnt["inertia_count"]


def test_reference_count_agrees_with_the_reference_spectrum(box, count):
    p, gamma, lam = box
    assert count == int(np.sum(lam <= gamma))


def test_mixed_solve_at_the_benched_settings(slrf_mod, box, count):
    p, gamma, lam = box
    L = se.SPECS["elast_64"]["block"]
    opts = slrf_mod.slrf_opts_default(it_max=23, precision=1, precond=1)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, opts)
    rc, nf, ev, X, rs, st = ctx.solve(torch.from_numpy(si.start_block(p.n, L, 3)), check=False)
    ctx.close()
    assert rc == 0 and nf == count
    ev = ev.cpu().numpy()
    assert np.max(np.abs(ev - lam[:count]) / lam[:count]) <= 1e-8
    assert rs.max().item() <= 1e-8
    Xh = X.cpu().numpy()
    del X
    G = Xh.T @ (p.B() @ Xh)
    assert np.abs(G - np.eye(count)).max() <= 1e-10


def test_fp64_filter_full_width_sampled_columns(slrf_mod, box):
    p, gamma, lam = box
    L = se.SPECS["elast_64"]["block"]
    it = 4
    opts = slrf_mod.slrf_opts_default(it_max=it, precision=0, precond=1)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, opts)
    V1 = si.start_block(p.n, L, 3)
    U = ctx.filter_apply(torch.from_numpy(V1)).cpu().numpy()
    ctx.close()
    A, B = p.A(), p.B()
    so, wo = orc.slrf_poles(8, gamma)
    cols = [0, 239, 479]
    Uo, fo = orc.filter_apply(A, B, V1[:, cols], None, so, wo, it, 1e-10, A.diagonal())
    assert rel(U[:, cols], Uo) <= 1e-8
