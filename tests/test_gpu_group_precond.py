"""Grouped-row COCG SpMM and Jacobi-preconditioned inner solves, through the C ABI.

Grouped rows (slrf_opts.group): the records of a group hold the union column list of its
rows in ascending order, with exact zeros where a row lacks a column; a zero product adds
an exact zero, so every row's SpMM sum runs over its own entries in the same order as the
plain CSR path (the packed FP32 FMA rounds each half like fmaf).  Rows map to warps
differently, though (a warp takes G consecutive rows), so the block sums of mu = p^T q
add the same terms in another order: the filtered blocks agree to rounding amplified over
the It_max steps -- FP64 within 1e-11 of max |U|, FP32 within 1e-5 -- with identical
COCG update counts.  Against the FP64 oracle the grouped path keeps the CSR path's parity:
1e-8 of max |U| on the Laplacian, 3e-8 on the lognormal-modulus elasticity pencil (whose
COCG amplifies rounding more; the CSR path measured 1.18e-8 there at It_max 9).

B-diagonal records (slrf_opts.bdiag): bitwise equal to the general records (exact zeros).

Jacobi preconditioner (slrf_opts.precond, D = diag(A) applied on both sides): compared with the oracle's
preconditioned COCG on the same scaled systems (D = diag(A)); the tolerances are those of
the unpreconditioned parity tests (U to 1e-8 of max |U|, update counts identical).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import pins
import slrf_inputs as si
from gpu_common import rel, slrf_mod  # noqa: F401
from oracle import slrf_oracle as orc

pytestmark = pytest.mark.gpu


def _elast(nodes=(7, 5, 4), seed=31):
    ne = int(np.prod([s - 1 for s in nodes]))
    E = np.exp(np.random.default_rng(seed).normal(0.0, 0.5, ne))
    return si.q1_elasticity(nodes, E=E)


@pytest.fixture(scope="module")
def elast():
    p = _elast()
    lam = sla.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 12)
    return p, lam, gamma, cnt


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("G", [2, 3, 4])
@pytest.mark.parametrize("family", ["elast", "lap"])
def test_grouped_spmm_matches_the_csr_path(slrf_mod, elast, precision, G, family):
    """n = 315 (elasticity, 7 x 5 x 3 free nodes: a ragged last group for G = 2, 4) or
    10 x 7 x 7 = 490 nodes (Laplacian: ragged for G = 3, 4); 21 columns x 8 poles: 20 and
    more row blocks, three FP32 tiles."""
    if family == "elast":
        p, _, gamma, _ = elast
    else:
        p = si.q1_scalar((10, 7, 7), shift=1e-3)
        gamma = 60.0
    k = 21
    V1 = si.start_block(p.n, k, 8)
    th = np.linspace(0.2, 1.4, k) * gamma
    it = 9
    out = {}
    for g in (1, G):
        opts = slrf_mod.slrf_opts_default(it_max=it, precision=precision, group=g)
        ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, k, opts)
        U0 = ctx.filter_apply(torch.from_numpy(V1)).cpu().numpy()
        U1 = ctx.filter_apply(torch.from_numpy(V1), torch.from_numpy(th)).cpu().numpy()
        its, rr, bk = ctx.filter_stats(k)
        out[g] = (U0, U1, its)
        ctx.close()
    tol = 1e-11 if precision == 0 else 1e-5
    assert rel(out[G][0], out[1][0]) <= tol
    assert rel(out[G][1], out[1][1]) <= tol
    assert np.array_equal(out[1][2], out[G][2])
    if precision == 0:
        so, wo = orc.slrf_poles(8, gamma)
        Uo, fo = orc.filter_apply(p.A(), p.B(), V1, th, so, wo, it, 1e-10)
        assert rel(out[G][1], Uo) <= (3e-8 if family == "elast" else 1e-8)
        assert np.array_equal(out[G][2], fo.iters)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("precond", [0, 1])
def test_b_diagonal_records_match_the_general_records(slrf_mod, elast, precision, precond):
    """3-row groups of the elasticity pencil (B = M (x) I_3, node-major dofs) take B-diagonal
    records (one B value per record, the row c mod 3); slrf_opts.bdiag = 0 keeps the general
    records.  A general record's other two B values are exact zeros, and fma(0, x, s) = s, so
    the COCG SpMM and the FP32 products agree bitwise (the FP32 A X, B X below).  The FP64
    real products of the filter start run through FP64 B-diagonal records in one case and
    the CSR kernel in the other (another summation order), so the filtered blocks agree to
    rounding amplified over the It_max steps: 1e-12 of max |U| in FP64, 1e-6 in FP32, with
    identical update counts.  The scalar Laplacian's 3-row groups never qualify (its B
    couples every row of a group)."""
    p, _, gamma, _ = elast
    k = 21
    V1 = si.start_block(p.n, k, 8)
    th = np.linspace(0.2, 1.4, k) * gamma
    out = {}
    for bd in (1, 0):
        opts = slrf_mod.slrf_opts_default(it_max=9, precision=precision, group=3, bdiag=bd, precond=precond)
        ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, k, opts)
        g, used, lw = ctx.format()
        assert g == 3 and used == bd and lw == (4 if precision == 1 else 1)
        U0 = ctx.filter_apply(torch.from_numpy(V1))
        U1 = ctx.filter_apply(torch.from_numpy(V1), torch.from_numpy(th))
        its, _, _ = ctx.filter_stats(k)
        AX, BX = ctx.apply(torch.from_numpy(V1), fp32=True)
        out[bd] = (U0, U1, its, AX, BX)
        ctx.close()
    tol = 1e-12 if precision == 0 else 1e-6
    for a, b in zip(out[1][:2], out[0][:2]):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= tol
    for a, b in zip(out[1][3:], out[0][3:]):
        assert torch.equal(a, b)
    assert np.array_equal(out[1][2], out[0][2])
    lap = si.q1_scalar((10, 7, 7), shift=1e-3)
    ctx = slrf_mod.Context(lap.rowptr, lap.col, lap.valA, lap.valB, 60.0, k,
                           slrf_mod.slrf_opts_default(precision=precision, group=3))
    assert ctx.format()[:2] == (3, 0)
    ctx.close()


@pytest.mark.parametrize("warm", [False, True])
def test_preconditioned_filter_matches_oracle(slrf_mod, elast, warm):
    p, lam, gamma, _ = elast
    k, it = 17, 25
    opts = slrf_mod.slrf_opts_default(it_max=it, precond=1)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, k, opts)
    V1 = si.start_block(p.n, k, 9)
    th = np.linspace(0.1, 1.5, k) * gamma if warm else None
    U = ctx.filter_apply(torch.from_numpy(V1), None if th is None else torch.from_numpy(th)).cpu().numpy()
    its, rr, bk = ctx.filter_stats(k)
    ctx.close()
    A, B = p.A(), p.B()
    so, wo = orc.slrf_poles(8, gamma)
    Uo, fo = orc.filter_apply(A, B, V1, th, so, wo, it, 1e-10, A.diagonal())
    assert rel(U, Uo) <= 1e-8
    assert np.array_equal(its, fo.iters)
    assert np.abs(rr - fo.relres).max() <= 1e-8
    assert not bk.any()
    # the preconditioner changes the iterates: the unpreconditioned oracle differs
    Un, _ = orc.filter_apply(A, B, V1, th, so, wo, it, 1e-10)
    assert rel(Un, Uo) > 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_preconditioned_solve_against_dense_eigh(slrf_mod, elast, precision):
    p, lam, gamma, cnt = elast
    L = int(np.ceil(1.5 * cnt))
    opts = slrf_mod.slrf_opts_default(it_max=12, precision=precision, precond=1)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, opts)
    rc, nf, ev, X, rs, st = ctx.solve(torch.from_numpy(si.start_block(p.n, L, 4)))
    ctx.close()
    ev = ev.cpu().numpy()
    X = X.cpu().numpy()
    assert rc == 0 and nf == cnt
    assert np.max(np.abs(ev - lam[:cnt]) / lam[:cnt]) <= (1e-10 if precision == 0 else 1e-8)
    assert rs.max().item() <= 1e-8
    assert np.abs(X.T @ (p.B() @ X) - np.eye(cnt)).max() <= 1e-10


def test_precond_rejects_a_nonpositive_diagonal(slrf_mod):
    p = si.q1_scalar((4, 4, 3), shift=1e-3)
    valA = p.valA.copy()
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    valA[np.nonzero((rows == 5) & (p.col == 5))[0]] = -1.0
    with pytest.raises(slrf_mod.SlrfError) as ei:
        slrf_mod.Context(p.rowptr, p.col, valA, p.valB, 100.0, 8, slrf_mod.slrf_opts_default(precond=1))
    assert ei.value.status == slrf_mod.SLRF_EINVAL
