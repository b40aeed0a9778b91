"""Parity of the CUDA Rayleigh-Ritz step (a6-a9) and of whole solves (Alg. 2) with the oracle
and with the closed-form / dense references that pin the oracle.

Eigenvalue tolerances follow the method's accuracy targets: relative error <= 1e-10 on
the FP64 path, <= 1e-8 on the mixed path, exact count, residuals <= 1e-8.  For the Q1
Neumann Laplacian the closed form itself is only accurate to ~5e-10 for the 1e-3
constant mode (assembly rounding, |K 1| ~ 1e-17), so the closed-form check there uses
max(1e-10 lambda, 1e-9 lambda_min), and the oracle-consistent check is the tight one.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import torch

import pins
import slrf_inputs as si
from gpu_common import cluster_projector_error, rel, slrf_mod  # noqa: F401
from oracle import slrf_oracle as orc

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _solve(slrf, p, gamma, L, seed, **kw):
    ctx = slrf.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, slrf.slrf_opts_default(**kw))
    V = torch.from_numpy(si.start_block(p.n, L, seed))
    rc, nf, ev, X, rs, st = ctx.solve(V, check=False)
    out = (rc, nf, ev.cpu().numpy(), X.cpu().numpy(), rs.cpu().numpy(), st)
    ctx.close()
    return out


@pytest.mark.parametrize("dense", [1, 0])
def test_rayleigh_ritz_step_parity(slrf_mod, dense):
    n, L = 500, 13
    p = si.bar1d_pencil(n)
    A, B = p.A(), p.B()
    lam, Xe = sla.eigh(A.toarray(), B.toarray())
    gamma = 0.5 * (lam[7] + lam[8])
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, slrf_mod.slrf_opts_default(dense=dense))
    so, wo = orc.slrf_poles(8, gamma)
    Uo, _ = orc.filter_apply(A, B, si.start_block(n, L, 5), None, so, wo, 60, 1e-10)
    # without locked vectors
    Ug, Vg, thg, rsg = ctx.rayleigh_ritz(torch.from_numpy(Uo))
    Uq, st = orc.cholqr2(Uo.copy(), B)
    tho, Vo = orc.rayleigh_ritz(Uq, A)
    Vo = orc.sign_normalise(Vo)
    reso, _, _ = orc.ritz_residuals(A, B, Vo, tho)
    assert rel(Ug.cpu().numpy(), Uq) <= 1e-12
    assert rel(thg.cpu().numpy(), tho) <= 1e-13
    assert rel(Vg.cpu().numpy(), Vo) <= 1e-10
    assert np.allclose(rsg.cpu().numpy(), reso, rtol=1e-6, atol=1e-15)
    # with locked exact eigenvectors X (CGS2 in the B-inner product first)
    X = np.ascontiguousarray(Xe[:, 20:23])
    BX = B @ X
    Ub = orc.b_orth(Uo.copy(), X, BX)
    Uq, st = orc.cholqr2(Ub, B)
    tho, Vo = orc.rayleigh_ritz(Uq, A)
    Ug, Vg, thg, rsg = ctx.rayleigh_ritz(torch.from_numpy(Uo), torch.from_numpy(X), torch.from_numpy(BX))
    assert rel(Ug.cpu().numpy(), Uq) <= 1e-11
    assert rel(thg.cpu().numpy(), tho) <= 1e-12
    assert np.abs(X.T @ (B @ Ug.cpu().numpy())).max() <= 1e-12
    ctx.close()


@pytest.mark.parametrize("k", [1, 2, 39, 97, 160, 255, 480])
def test_rayleigh_ritz_on_an_invariant_subspace_with_multiplicities(slrf_mod, k):
    """Projected eigenproblem (cooperative Jacobi) on a block that spans k exact eigenvectors
    of the 9^3 Q1 cube Laplacian, whose cube symmetry gives exactly repeated eigenvalues
    (30 triples and 26 sextets among the lowest 255): the Ritz values are the eigenvalues,
    the Ritz vectors satisfy the pencil to rounding level and are B-orthonormal.  Odd k
    exercises the padded index of the round-robin ordering; k = 255 two row entries per
    thread.  From k = 96 on the Cholesky factors come from the blocked multi-CTA kernels
    (97: one column past a panel; 255: ragged last panel and column block; 480: the
    benched block width)."""
    from slrf_inputs import fem

    p = fem.q1_scalar((9, 9, 9), shift=1e-3)
    A, B = p.A().toarray(), p.B().toarray()
    lam, Xe = sla.eigh(A, B)
    rng = np.random.default_rng(k)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    U = np.ascontiguousarray(Xe[:, :k] @ (Q * np.logspace(0, 1, k)[None, :]))  # condition 10
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, 1.01 * lam[k - 1], k, slrf_mod.slrf_opts_default())
    _, Vg, thg, rsg = ctx.rayleigh_ritz(torch.from_numpy(U))
    th, V = thg.cpu().numpy(), Vg.cpu().numpy()
    ctx.close()
    # (the 1e-3 constant mode carries the assembly rounding of A 1: its relative residual is
    # ~5e-10 and its eigenvalue moves by ~1e-13 even for the oracle's own Rayleigh-Ritz step)
    assert np.abs(th - lam[:k]).max() <= 1e-12 * max(lam[k - 1], 1.0)
    AV = A @ V
    res = np.linalg.norm(AV - (B @ V) * th[None, :], axis=0) / np.linalg.norm(AV, axis=0)
    assert res.max() <= 2e-9 and rsg.cpu().numpy().max() <= 2e-9
    assert np.abs(V.T @ B @ V - np.eye(k)).max() <= 1e-12


@pytest.mark.parametrize("k", [4, 128])
def test_rayleigh_ritz_reports_a_singular_gram(slrf_mod, k):
    n = 200
    p = si.bar1d_pencil(n)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, 100.0, k, slrf_mod.slrf_opts_default())
    U = torch.ones(n, k, dtype=torch.float64)  # rank one
    with pytest.raises(slrf_mod.SlrfError) as e:
        ctx.rayleigh_ritz(U)
    assert e.value.status == slrf_mod.SLRF_ECHOL
    ctx.close()


def test_solve_bar1d_2000_matches_closed_form_and_oracle(slrf_mod):
    gold = json.load(open(os.path.join(GOLD, "bar1d_2000_solve.json")))
    wl = si.bar1d(2000)
    rc, nf, ev, X, rs, st = _solve(slrf_mod, wl.pencil, wl.gamma, wl.block, wl.seed, it_max=gold["it_max"])
    lam = pins.bar1d_eigs(2000)
    assert rc == 0 and nf == 20 == len(gold["evals"])
    assert np.max(np.abs(ev - lam[:20]) / lam[:20]) <= 1e-10
    assert np.max(np.abs(ev - np.array(gold["evals"])) / ev) <= 1e-10
    assert rs.max() <= 1e-8
    B = wl.pencil.B()
    assert np.abs(X.T @ (B @ X) - np.eye(20)).max() <= 1e-12
    assert abs(st["outer_iters"] - gold["outer_iters"]) <= 1
    # eigenvectors: sin(k pi x_i) up to sign
    h = 1.0 / 2001
    xg = np.arange(1, 2001) * h
    for k in range(20):
        s = np.sin((k + 1) * np.pi * xg)
        s /= np.sqrt(s @ (B @ s))
        assert abs(abs(s @ (B @ X[:, k])) - 1.0) <= 1e-9


@pytest.mark.parametrize("dense", [1, 0])
@pytest.mark.parametrize("precision", [0, 1])
def test_solve_q1_small(slrf_mod, precision, dense):
    nodes = (13, 13, 13)
    p = si.q1_scalar(nodes, shift=1e-3)
    lam = pins.q1_neumann_eigs(nodes, 1e-3)
    gamma, cnt = pins.gap_gamma(lam, 40)
    L = int(np.ceil(1.5 * cnt))
    rc, nf, ev, X, rs, st = _solve(slrf_mod, p, gamma, L, 2, it_max=30, precision=precision, dense=dense)
    assert rc == 0 and nf == cnt
    tol = 1e-10 if precision == 0 else 1e-8
    assert np.all(np.abs(ev - lam[:cnt]) <= np.maximum(tol * lam[:cnt], 1e-9 * lam[0]))
    assert rs.max() <= 1e-8
    B = p.B()
    assert np.abs(X.T @ (B @ X) - np.eye(cnt)).max() <= 1e-11
    lam_d, Xd = sla.eigh(p.A().toarray(), B.toarray(), subset_by_index=[0, cnt - 1])
    assert cluster_projector_error(X, Xd, B, lam_d) <= 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_elasticity_small(slrf_mod, precision):
    E = np.exp(np.random.default_rng(3).normal(0, 0.5, 7 * 7 * 5))
    p = si.q1_elasticity((8, 8, 6), E=E)
    lam = sla.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 30)
    assert pins.dense_inertia_count(p.A(), p.B(), gamma) == cnt
    L = int(np.ceil(1.5 * cnt))
    rc, nf, ev, X, rs, st = _solve(slrf_mod, p, gamma, L, 4, it_max=60, precision=precision)
    assert rc == 0 and nf == cnt
    tol = 1e-10 if precision == 0 else 1e-8
    assert np.max(np.abs(ev - lam[:cnt]) / lam[:cnt]) <= tol
    assert rs.max() <= 1e-8


def test_basic_method(slrf_mod):
    """Alg. 1: no locking, zero initial guesses, near-exact inner solves."""
    nodes = (6, 6, 5)
    p = si.q1_scalar(nodes, shift=1e-3)
    lam = pins.q1_neumann_eigs(nodes, 1e-3)
    gamma, cnt = pins.gap_gamma(lam, 12)
    L = int(np.ceil(1.5 * cnt))
    rc, nf, ev, X, rs, st = _solve(slrf_mod, p, gamma, L, 7, it_max=400, tol_inner=1e-14, lock=0, warm_start=0,
                                   outer_max=30)
    assert rc == 0 and nf == cnt
    assert np.max(np.abs(ev - lam[:cnt]) / np.maximum(lam[:cnt], 1e-2)) <= 1e-9


def test_deterministic_and_graph_equivalent(slrf_mod):
    """Fixed-order reductions: two solves, with and without the CUDA graph, agree bitwise."""
    wl = si.bar1d(2000)
    r1 = _solve(slrf_mod, wl.pencil, wl.gamma, wl.block, 1, it_max=200)
    r2 = _solve(slrf_mod, wl.pencil, wl.gamma, wl.block, 1, it_max=200, use_graph=0)
    r3 = _solve(slrf_mod, wl.pencil, wl.gamma, wl.block, 1, it_max=200)
    assert np.array_equal(r1[2], r2[2]) and np.array_equal(r1[2], r3[2])
    assert np.array_equal(r1[3], r3[3])


def test_solve_host_entry_point(slrf_mod):
    n = 400
    p = si.bar1d_pencil(n)
    lam = pins.bar1d_eigs(n)
    gamma = 0.5 * (lam[9] + lam[10])
    V0 = si.start_block(n, 16, 9)
    ev, X, rs, st = slrf_mod.slrf_solve_host(p.rowptr, p.col, p.valA, p.valB, gamma, 16,
                                             slrf_mod.slrf_opts_default(it_max=80), V0)
    assert len(ev) == 10 and np.max(np.abs(ev - lam[:10]) / lam[:10]) <= 1e-10
    rc, nf, ev2, X2, rs2, st2 = _solve(slrf_mod, p, gamma, 16, 9, it_max=80)
    assert np.array_equal(ev, ev2)


def test_status_codes(slrf_mod):
    n = 300
    p = si.bar1d_pencil(n)
    lam = pins.bar1d_eigs(n)
    gamma = 0.5 * (lam[9] + lam[10])
    mod = slrf_mod
    # capacity smaller than the count: ETRUNC with the true count and the first pairs
    ctx = mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, 16, mod.slrf_opts_default(it_max=80))
    V = torch.from_numpy(si.start_block(n, 16, 2))
    rc, nf, ev, X, rs, st = ctx.solve(V, cap=4, check=False)
    assert rc == mod.SLRF_ETRUNC and nf == 10 and np.allclose(ev.cpu().numpy(), lam[:4], rtol=1e-10)
    # non-finite start block
    Vn = V.clone()
    Vn[3, 2] = float("nan")
    rc, *_ = ctx.solve(Vn, check=False)
    assert rc == mod.SLRF_ENAN
    # outer iteration cap
    ctx2 = mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, 16, mod.slrf_opts_default(it_max=80, outer_max=1))
    rc, *_ = ctx2.solve(V, check=False)
    assert rc == mod.SLRF_ENOCONV
    # an interval below the spectrum holds nothing
    ctx3 = mod.Context(p.rowptr, p.col, p.valA, p.valB, 0.5 * lam[0], 8, mod.slrf_opts_default(it_max=80))
    rc, nf, *_ = ctx3.solve(torch.from_numpy(si.start_block(n, 8, 3)), check=False)
    assert rc == 0 and nf == 0
    for c in (ctx, ctx2, ctx3):
        c.close()
    # a malformed pattern is rejected at setup
    bad = p.col.copy()
    bad[5] = n + 7
    with pytest.raises(mod.SlrfError) as e:
        mod.Context(p.rowptr, bad, p.valA, p.valB, gamma, 8)
    assert e.value.status == mod.SLRF_EINVAL


def test_solve_q1_41_full_size(slrf_mod):
    """The 41^3 workload: all 105 eigenpairs of (0, 259.0666], against the tensor-product
    closed form, B-orthonormal, residuals <= 1e-8."""
    wl = si.q1_lap(41)
    rc, nf, ev, X, rs, st = _solve(slrf_mod, wl.pencil, wl.gamma, wl.block, wl.seed, it_max=40)
    lam = pins.q1_neumann_eigs((41, 41, 41), 1e-3)
    assert rc == 0 and nf == 105 == int(np.sum(lam <= wl.gamma))
    assert np.all(np.abs(ev - lam[:105]) <= np.maximum(1e-10 * lam[:105], 1e-9 * lam[0]))
    assert rs.max() <= 1e-8
    B = wl.pencil.B()
    assert np.abs(X.T @ (B @ X) - np.eye(105)).max() <= 1e-11


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_q1_41_at_the_benched_settings(slrf_mod, precision):
    """The 41^3 workload at It_max 8, the inner-solve length its bench line uses, in FP64 and
    in the mixed path: all 105 eigenpairs against the tensor-product closed form (1e-10 FP64,
    1e-8 mixed, with the constant-mode floor), residuals <= 1e-8, B-orthonormal vectors."""
    wl = si.q1_lap(41)
    rc, nf, ev, X, rs, st = _solve(slrf_mod, wl.pencil, wl.gamma, wl.block, wl.seed, it_max=8, precision=precision)
    lam = pins.q1_neumann_eigs((41, 41, 41), 1e-3)
    tol = 1e-10 if precision == 0 else 1e-8
    assert rc == 0 and nf == 105 == int(np.sum(lam <= wl.gamma))
    assert np.all(np.abs(ev - lam[:105]) <= np.maximum(tol * lam[:105], 1e-9 * lam[0]))
    assert rs.max() <= 1e-8
    B = wl.pencil.B()
    assert np.abs(X.T @ (B @ X) - np.eye(105)).max() <= 1e-10


def test_solve_with_refinement_steps(slrf_mod):
    """Mixed path with two FP64 refinement steps per filter apply: same eigenpairs."""
    nodes = (9, 9, 9)
    p = si.q1_scalar(nodes, shift=1e-3)
    lam = pins.q1_neumann_eigs(nodes, 1e-3)
    gamma, cnt = pins.gap_gamma(lam, 25)
    L = int(np.ceil(1.5 * cnt))
    rc, nf, ev, X, rs, st = _solve(slrf_mod, p, gamma, L, 5, it_max=20, precision=1, refine_max=2)
    assert rc == 0 and nf == cnt
    assert np.all(np.abs(ev - lam[:cnt]) <= np.maximum(1e-8 * lam[:cnt], 1e-9 * lam[0]))
    assert rs.max() <= 1e-8


def test_stop_rule_needs_a_resolved_subspace(slrf_mod):
    """The oracle pin of the stopping rule on the GPU: with It_max = 2 on a 31 x 30 Q1 mesh
    the block stays unresolved and the solve must not report success (without the resolution
    guard it returned status OK with 0 of 10 pairs); with It_max = 5 it finds all 10, in the
    oracle's 33 outer steps (+-1 for rounding)."""
    p = si.q1_scalar((31, 30), dirichlet_face=(0, 0))
    lam = sla.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 10)
    L = int(np.ceil(1.5 * cnt))
    rc, nf, ev, X, rs, st = _solve(slrf_mod, p, gamma, L, 3, it_max=2, outer_max=30)
    assert rc == slrf_mod.SLRF_ENOCONV
    rc, nf, ev, X, rs, st = _solve(slrf_mod, p, gamma, L, 3, it_max=5, outer_max=60)
    assert rc == 0 and nf == cnt
    assert np.max(np.abs(ev - lam[:cnt]) / lam[:cnt]) <= 1e-10
    assert abs(st["outer_iters"] - 33) <= 1


def test_adaptive_it_max_resolves_short_inner_solves(slrf_mod):
    """opts.it_adapt: the same 31 x 30 mesh from It_max = 2, which alone ends unresolved;
    the problem's It_max doubles while its lowest active Ritz pair stays unresolved, and the
    solve finds all 10 pairs."""
    p = si.q1_scalar((31, 30), dirichlet_face=(0, 0))
    lam = sla.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 10)
    L = int(np.ceil(1.5 * cnt))
    rc, nf, ev, X, rs, st = _solve(slrf_mod, p, gamma, L, 3, it_max=2, it_adapt=1, outer_max=100)
    assert rc == 0 and nf == cnt
    assert np.max(np.abs(ev - lam[:cnt]) / lam[:cnt]) <= 1e-10
    assert rs.max() <= 1e-8


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_waits_report_a_timeout_and_leave_the_device_usable(slrf_mod, kind):
    """Failure detection without a fault: a wait that nothing can complete (kind 0: the
    Rayleigh-Ritz grid barrier expecting one block more than the launch has; kind 1: an
    mbarrier phase nobody arrives at) gives up at its limit and the call returns
    SLRF_ETIMEOUT; a filter apply afterwards still runs and matches the oracle."""
    import time

    t0 = time.time()
    assert slrf_mod.lib().slrf_wait_selftest(kind, None) == slrf_mod.SLRF_ETIMEOUT
    assert time.time() - t0 < 30.0
    assert slrf_mod.lib().slrf_wait_selftest(2, None) == slrf_mod.SLRF_EINVAL
    p = si.bar1d_pencil(300)
    lam = pins.bar1d_eigs(300)
    gamma = 0.5 * (lam[5] + lam[6])
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, 8, slrf_mod.slrf_opts_default(it_max=40))
    V1 = si.start_block(300, 8, 2)
    U = ctx.filter_apply(torch.from_numpy(V1)).cpu().numpy()
    ctx.close()
    so, wo = orc.slrf_poles(8, gamma)
    Uo, _ = orc.filter_apply(p.A(), p.B(), V1, None, so, wo, 40, 1e-10)
    assert rel(U, Uo) <= 1e-8
