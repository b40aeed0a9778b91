"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each check is independent of the oracle's own code: closed-form FEM spectra, dense
library eigensolvers and solvers, Sylvester inertia, the Proposition of Sec. 4, CG from
scipy, and invariants (B-orthonormality, conjugate symmetry, filter on eigenvectors).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import slrf_inputs as si
from oracle import slrf_oracle as orc
import pins

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _small_q1(nodes=(6, 5, 4), shift=1e-3):
    p = si.q1_scalar(nodes, shift=shift)
    return p, p.A(), p.B()


# ---------------------------------------------------------------- poles and weights
def test_poles_on_shifted_laplace_line():
    """Sec. 2.2: sigma = Re(sigma) (1 + alpha i); real parts inside (0, gamma)."""
    for alpha in (1.0, 0.5):
        s, w = orc.slrf_poles(8, 250.0, alpha=alpha)
        assert np.allclose(s.imag, alpha * s.real, rtol=0, atol=1e-12)
        assert np.all((s.real > 0) & (s.real < 250.0))
        assert len(np.unique(s)) == 8


def test_pole_weights_solve_the_regularised_fit():
    """The weights equal an SVD least-squares solve of the stacked system [G; sqrt(beta) I]."""
    m, beta = 8, 0.01
    s, w = orc.slrf_poles(m, 1.0, beta=beta)
    x = (np.arange(1, m + 1) - 0.5) / m
    assert np.allclose(s, x * (1 + 1j))
    t = np.concatenate([(np.arange(3000) + 0.5) / 3000, np.geomspace(1.3, 51.0, 3000)])
    f = np.concatenate([np.ones(3000), np.zeros(3000)])
    # Phi(t) = sum_j w_j/(t - s_j) + conj(w_j)/(t - conj(s_j)) written as a real design
    cols = []
    for j in range(m):
        e = np.zeros(m, complex)
        e[j] = 1.0
        cols.append(sum(e[i] / (t - s[i]) + np.conj(e[i]) / (t - np.conj(s[i])) for i in range(m)).real)
    for j in range(m):
        e = np.zeros(m, complex)
        e[j] = 1j
        cols.append(sum(e[i] / (t - s[i]) + np.conj(e[i]) / (t - np.conj(s[i])) for i in range(m)).real)
    G = np.stack(cols, axis=1)
    Gs = np.vstack([G, np.sqrt(beta) * np.eye(2 * m)])
    u, *_ = np.linalg.lstsq(Gs, np.concatenate([f, np.zeros(2 * m)]), rcond=None)
    assert np.allclose(w, u[:m] + 1j * u[m:], rtol=1e-8, atol=1e-10)


def test_filter_shape():
    """Phi passes (0, gamma] and damps [1.3 gamma, inf): the filter property of Sec. 2.
    The design (midpoint abscissae, Tikhonov-regularised fit; m = 8, alpha = 1, beta = 0.01)
    has, on the normalised axis,
    min Phi = 0.8711 (at t = gamma), max Phi = 1.0400 (at t = 0.832 gamma) on (0, gamma],
    max |Phi| = 0.2233 beyond 1.3 gamma (at the band edge) and 0.0885 beyond 1.4 gamma."""
    g = 4150.528
    s, w = orc.slrf_poles(8, g)
    t_in = np.linspace(0, 1, 200001)[1:]
    inside = orc.filter_value(t_in * g, s, w)
    outside = orc.filter_value(np.geomspace(1.3, 1e4, 200001) * g, s, w)
    beyond = orc.filter_value(np.geomspace(1.4, 1e4, 200001) * g, s, w)
    assert abs(inside.min() - 0.8711) <= 1e-3 and t_in[np.argmin(inside)] == 1.0
    assert abs(inside.max() - 1.0400) <= 1e-3
    assert abs(np.abs(outside).max() - 0.2233) <= 1e-3 and np.argmax(np.abs(outside)) == 0
    assert abs(np.abs(beyond).max() - 0.0885) <= 1e-3
    # the conjugate half: w/(t - s) + conj(w)/(t - conj s) = 2 Re(w/(t - s))
    t = 0.37 * g
    full = np.sum(w / (t - s) + np.conj(w) / (t - np.conj(s)))
    assert abs(full.imag) < 1e-12 and abs(full.real - orc.filter_value(t, s, w)) < 1e-12


# ---------------------------------------------------------------- COCG
def test_cocg_equals_scipy_cg_for_a_real_shift():
    """For a real shift sigma < 0, A - sigma B is SPD and COCG is CG: iterate k matches
    scipy's CG stopped after k iterations."""
    p, A, B = _small_q1()
    rng = np.random.default_rng(0)
    b = rng.standard_normal((p.n, 1))
    M = (A + 2.0 * B).tocsr()
    for k in (1, 3, 7):
        y, info = orc.cocg(A, B, -2.0, b, np.zeros_like(b), k, 0.0)
        x_ref, _ = spla.cg(M, b[:, 0], x0=np.zeros(p.n), rtol=0.0, atol=0.0, maxiter=k)
        assert info.iters[0] == k
        assert np.allclose(y[:, 0].real, x_ref, rtol=1e-10, atol=1e-12 * np.abs(x_ref).max())
        assert np.abs(y.imag).max() == 0


def test_cocg_solves_complex_symmetric_system():
    """Converged COCG equals a dense complex solve of (A - sigma B) y = b."""
    p, A, B = _small_q1((4, 4, 3))
    rng = np.random.default_rng(1)
    b = rng.standard_normal((p.n, 3))
    sig = 0.3 * 250 * (1 + 1j)
    y, info = orc.cocg(A, B, sig, b, np.zeros((p.n, 3)), 400, 1e-13)
    ref = np.linalg.solve(A.toarray() - sig * B.toarray(), b)
    assert np.abs(y - ref).max() <= 1e-10 * np.abs(ref).max()
    assert np.all(info.relres <= 1e-13) and not info.breakdown.any()
    # the conjugate pole gives the conjugate solution (Sec. 2: sigma_{N+j} = conj sigma_j)
    yc, _ = orc.cocg(A, B, np.conj(sig), b, np.zeros((p.n, 3)), 400, 1e-13)
    assert np.abs(yc - np.conj(y)).max() <= 1e-10 * np.abs(ref).max()


def test_cocg_breakdown_is_flagged():
    """A 2x2 complex-symmetric system with p^T M p = 0 on the first step stops, flagged."""
    A = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, -1.0]]))
    B = sp.csr_matrix(np.eye(2))
    b = np.array([[1.0], [1.0]])
    # M = A - 0*B = diag(1, -1); p = b; p^T M p = 1 - 1 = 0
    y, info = orc.cocg(A, B, 0.0, b, np.zeros((2, 1)), 10, 0.0)
    assert info.breakdown[0] and info.iters[0] == 0 and np.all(y == 0)


def test_proposition_initial_residual_and_krylov_space():
    """Sec. 4, Proposition: with y0 = v/(theta - sigma), r0 = (A - theta B) v / (sigma - theta),
    and the Cayley iterate u_k (from u0 = 0, rhs (A - theta B) v) satisfies
    u_k = v + (sigma - theta) y_k at every step."""
    p, A, B = _small_q1((5, 4, 4))
    rng = np.random.default_rng(2)
    v = rng.standard_normal((p.n, 1))
    theta, sig = 37.0, 55.0 * (1 + 1j)
    y0 = v / (theta - sig)
    r0 = B @ v - (A @ y0 - sig * (B @ y0))
    rc = A @ v - theta * (B @ v)
    assert np.allclose(r0, rc / (sig - theta), rtol=1e-12, atol=1e-13 * np.abs(rc).max())
    for k in (1, 4, 9):
        y, _ = orc.cocg(A, B, sig, B @ v, y0, k, 0.0)
        u, _ = orc.cocg(A, B, sig, rc, np.zeros_like(v), k, 0.0)
        assert np.allclose(u, v + (sig - theta) * y, rtol=1e-9, atol=1e-10 * np.abs(u).max())


def _galerkin_iterate(M, r0, k):
    """The k-th COCG correction characterised without its recurrence: the vector c of
    K_k(M, r0) whose residual r0 - M c is orthogonal to K_k in the unconjugated bilinear
    form x^T y (Petrov-Galerkin condition of COCG).  Q spans K_k (any basis of it gives the
    same c, since Q^T r = 0 <=> V^T r = 0 for V = Q T)."""
    V = [r0]
    for _ in range(k - 1):
        V.append(M @ V[-1])
    Q, _ = np.linalg.qr(np.stack(V, axis=1))
    return Q @ np.linalg.solve(Q.T @ (M @ Q), Q.T @ r0)


@pytest.mark.parametrize("precond", [False, True])
def test_cocg_iterates_satisfy_the_galerkin_condition(precond):
    """COCG (and its Jacobi-preconditioned form) after k steps equals the
    Petrov-Galerkin iterate of the (scaled) system in the Krylov space of its initial
    residual, from a nonzero initial guess.  Preconditioned: the system is
    D^-1/2 (A - sigma B) D^-1/2 z = D^-1/2 b with D = diag(A), z = D^1/2 y."""
    E = np.exp(np.random.default_rng(21).normal(0, 0.5, 3 * 3 * 2))
    p = si.q1_elasticity((4, 4, 3), E=E)
    A, B = p.A(), p.B()
    Ad, Bd = A.toarray(), B.toarray()
    rng = np.random.default_rng(22)
    b = rng.standard_normal((p.n, 1))
    y0 = rng.standard_normal((p.n, 1)) * 1e-3
    sig = 40.0 * (1 + 1j)
    d = Ad.diagonal() if precond else np.ones(p.n)
    h = 1.0 / np.sqrt(d)
    Mh = h[:, None] * (Ad - sig * Bd) * h[None, :]
    z0 = y0[:, 0] / h
    r0 = h * (b[:, 0] - (Ad - sig * Bd) @ y0[:, 0])
    for k in (1, 2, 4, 6):
        y, info = orc.cocg(A, B, sig, b, y0, k, 0.0, Ad.diagonal() if precond else None)
        ref = h * (z0 + _galerkin_iterate(Mh, r0, k))
        assert info.iters[0] == k
        assert np.abs(y[:, 0] - ref).max() <= 1e-9 * np.abs(ref).max(), k
        # relres is the scaled system's ||r|| / ||r0||
        rk = h * (b[:, 0] - (Ad - sig * Bd) @ y[:, 0])
        assert abs(info.relres[0] - np.linalg.norm(rk) / np.linalg.norm(r0)) <= 1e-8 * info.relres[0]


def test_preconditioned_cocg_solves_the_unscaled_system():
    """Converged preconditioned COCG equals a dense complex solve of (A - sigma B) y = b,
    and a constant diagonal (D = c I) gives the unpreconditioned iterates."""
    E = np.exp(np.random.default_rng(23).normal(0, 0.5, 3 * 3 * 2))
    p = si.q1_elasticity((4, 4, 3), E=E)
    A, B = p.A(), p.B()
    rng = np.random.default_rng(24)
    b = rng.standard_normal((p.n, 2))
    sig = 25.0 * (1 + 1j)
    ref = np.linalg.solve(A.toarray() - sig * B.toarray(), b)
    y, info = orc.cocg(A, B, sig, b, np.zeros((p.n, 2)), 2000, 1e-13, A.diagonal())
    assert np.abs(y - ref).max() <= 1e-9 * np.abs(ref).max() and not info.breakdown.any()
    y1, i1 = orc.cocg(A, B, sig, b, np.zeros((p.n, 2)), 7, 0.0)
    y2, i2 = orc.cocg(A, B, sig, b, np.zeros((p.n, 2)), 7, 0.0, np.full(p.n, 4.0))
    assert np.abs(y1 - y2).max() <= 1e-12 * np.abs(y1).max()
    assert np.allclose(i1.relres, i2.relres, rtol=1e-10)


# ---------------------------------------------------------------- the filter on eigenvectors
def test_filter_apply_on_exact_eigenvectors():
    """With X exact eigenvectors and converged solves, filter_apply(X) = X diag(Phi(lambda))."""
    p, A, B = _small_q1((5, 4, 3))
    lam, X = sla.eigh(A.toarray(), B.toarray())
    gamma = 0.5 * (lam[9] + lam[10])
    s, w = orc.slrf_poles(8, gamma)
    Xs = X[:, :14]
    U, info = orc.filter_apply(A, B, Xs, None, s, w, 500, 1e-14)
    ref = Xs * orc.filter_value(lam[:14], s, w)[None, :]
    assert np.abs(U - ref).max() <= 1e-9 * np.abs(ref).max()
    # same with the warm start from the exact eigenvalues: zero initial residual, no iterations
    U2, info2 = orc.filter_apply(A, B, Xs, lam[:14], s, w, 500, 1e-14)
    assert np.abs(U2 - ref).max() <= 1e-9 * np.abs(ref).max()


# ---------------------------------------------------------------- a6-a8
def test_borth_cholqr2_rayleigh_ritz():
    p, A, B = _small_q1((6, 5, 4))
    Bd = B.toarray()
    lam, Xe = sla.eigh(A.toarray(), Bd)
    rng = np.random.default_rng(3)
    X = Xe[:, :5]
    BX = B @ X
    U0 = rng.standard_normal((p.n, 12))
    U = orc.b_orth(U0, X, BX)
    assert np.abs(X.T @ (B @ U)).max() <= 1e-12 * np.abs(U).max()
    Q, st = orc.cholqr2(U, B)
    assert st == orc.OK
    assert np.abs(Q.T @ Bd @ Q - np.eye(12)).max() <= 1e-12
    T = np.linalg.lstsq(U, Q, rcond=None)[0]  # Q = U T with T upper triangular
    assert np.abs(np.tril(T, -1)).max() <= 1e-10 * np.abs(T).max()
    # Rayleigh-Ritz on an exact invariant subspace returns the exact eigenvalues
    Z, _ = orc.cholqr2(Xe[:, 3:11] @ rng.standard_normal((8, 8)), B)
    th, V = orc.rayleigh_ritz(Z, A)
    assert np.allclose(th, lam[3:11], rtol=1e-11)
    assert np.abs(V.T @ Bd @ V - np.eye(8)).max() <= 1e-12
    res, res_paper, _ = orc.ritz_residuals(A, B, V, th)
    assert res.max() <= 1e-10 and res_paper.max() <= 1e-10


def test_ritz_residuals_closed_form():
    """v = x_i + eps x_j with B-orthonormal eigenvectors x (A x = l B x) and b = B x:
    A v = l_i b_i + eps l_j b_j, B v = b_i + eps b_j, and at theta = the Rayleigh quotient
    (l_i + eps^2 l_j) / (1 + eps^2):
      ||A v - theta B v||^2 = (l_i - th)^2 |b_i|^2 + 2 eps (l_i - th)(l_j - th) b_i.b_j
                              + eps^2 (l_j - th)^2 |b_j|^2,
      ||A v||^2 = l_i^2 |b_i|^2 + 2 eps l_i l_j b_i.b_j + eps^2 l_j^2 |b_j|^2,
      ||v||_B^2 = 1 + eps^2.
    The relative residual is the first over the second; the paper's form (Sec. 3.2) is
    ||A v - theta B v|| / (theta ||v||_B)."""
    p, A, B = _small_q1((6, 5, 4))
    lam, Xe = sla.eigh(A.toarray(), B.toarray())
    cases = [(3, 7, 0.3), (10, 2, 0.05), (20, 21, 1e-2), (0, 40, 0.5)]
    V = np.stack([Xe[:, i] + e * Xe[:, j] for i, j, e in cases], axis=1)
    th = np.array([(lam[i] + e * e * lam[j]) / (1 + e * e) for i, j, e in cases])
    res, res_paper, BV = orc.ritz_residuals(A, B, V, th)
    assert np.abs(BV - B @ V).max() <= 1e-14 * np.abs(B @ V).max()
    for c, (i, j, e) in enumerate(cases):
        bi, bj = B @ Xe[:, i], B @ Xe[:, j]
        li, lj, t = lam[i], lam[j], th[c]
        num = (li - t) ** 2 * (bi @ bi) + 2 * e * (li - t) * (lj - t) * (bi @ bj) + e * e * (lj - t) ** 2 * (bj @ bj)
        den = li * li * (bi @ bi) + 2 * e * li * lj * (bi @ bj) + e * e * lj * lj * (bj @ bj)
        assert abs(res[c] - np.sqrt(num / den)) <= 1e-9 * res[c], (c, res[c], np.sqrt(num / den))
        paper = np.sqrt(num) / (t * np.sqrt(1 + e * e))
        assert abs(res_paper[c] - paper) <= 1e-9 * paper


def test_sign_normalise():
    """Sign convention: each vector's entry of largest magnitude is made positive; among equal
    magnitudes the first one decides; a zero vector stays zero."""
    V = np.array([[1.0, 2.0, 0.0, -0.5],
                  [-3.0, -2.0, 0.0, 0.25],
                  [2.0, 1.0, 0.0, 0.5]])
    out = orc.sign_normalise(V)
    expect = np.array([[-1.0, 2.0, 0.0, 0.5],
                       [3.0, -2.0, 0.0, -0.25],
                       [-2.0, 1.0, 0.0, -0.5]])
    assert np.array_equal(out, expect)


def test_cholqr2_reports_a_non_spd_gram():
    p, A, B = _small_q1((4, 4, 3))
    U = np.ones((p.n, 3))  # rank one
    _, st = orc.cholqr2(U, B)
    assert st == orc.E_CHOL


# ---------------------------------------------------------------- a9 / Alg. 2 end to end
def test_solve_bar1d_closed_form_and_sturm_count():
    """1D bar: every eigenvalue in (0, gamma] to 1e-10 of the closed form, the count equal
    to the Sturm count of A - gamma B, residuals <= 1e-8, X B-orthonormal."""
    n = 300
    p = si.bar1d_pencil(n)
    lam = pins.bar1d_eigs(n)
    gamma = 0.5 * (lam[11] + lam[12])
    h = 1.0 / (n + 1)
    cnt = pins.sturm_count(np.full(n, 2 / h), np.full(n - 1, -1 / h), gamma,
                           np.full(n, 4 * h / 6), np.full(n - 1, h / 6))
    assert cnt == 12
    V1 = si.start_block(n, 18, 11)
    r = orc.enhanced_slrf(p.A(), p.B(), gamma, V1, m=8, it_max=60, outer_max=40)
    assert r.status == orc.OK
    assert len(r.evals) == cnt
    assert np.max(np.abs(r.evals - lam[:cnt]) / lam[:cnt]) <= 1e-10
    assert r.resid.max() <= 1e-8
    assert np.abs(r.X.T @ (p.B() @ r.X) - np.eye(cnt)).max() <= 1e-10
    # eigenvectors: sin(k pi x_i), compared up to sign through B-inner products
    xg = np.arange(1, n + 1) * h
    for k in range(cnt):
        s = np.sin((k + 1) * np.pi * xg)
        s /= np.sqrt(s @ (p.B() @ s))
        assert abs(abs(s @ (p.B() @ r.X[:, k])) - 1.0) <= 1e-8


def test_solve_q1_against_dense_eigh_and_inertia():
    nodes = (6, 6, 5)
    p, A, B = _small_q1(nodes)
    lam = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    closed = pins.q1_neumann_eigs(nodes, 1e-3)
    assert np.allclose(lam[1:], closed[1:], rtol=1e-11)
    gamma, cnt = pins.gap_gamma(lam, 20)
    assert pins.dense_inertia_count(A, B, gamma) == cnt
    V1 = si.start_block(p.n, int(np.ceil(1.5 * cnt)), 5)
    r = orc.enhanced_slrf(A, B, gamma, V1, m=8, it_max=30, outer_max=40)
    assert r.status == orc.OK and len(r.evals) == cnt
    assert np.max(np.abs(r.evals - lam[:cnt]) / lam[:cnt]) <= 1e-9
    assert r.resid.max() <= 1e-8
    assert np.abs(r.X.T @ (B @ r.X) - np.eye(cnt)).max() <= 1e-10


def test_solve_elasticity_against_dense_eigh():
    E = np.exp(np.random.default_rng(9).normal(0, 0.5, 3 * 3 * 2))
    p = si.q1_elasticity((4, 4, 3), E=E)
    A, B = p.A(), p.B()
    lam = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 10)
    assert pins.dense_inertia_count(A, B, gamma) == cnt
    V1 = si.start_block(p.n, int(np.ceil(1.5 * cnt)), 6)
    r = orc.enhanced_slrf(A, B, gamma, V1, m=8, it_max=40, outer_max=40)
    assert r.status == orc.OK and len(r.evals) == cnt
    assert np.max(np.abs(r.evals - lam[:cnt]) / lam[:cnt]) <= 1e-9
    assert r.resid.max() <= 1e-8


def test_stop_rule_needs_a_resolved_subspace():
    """Inner solves far too short for the mesh (It_max = 2 on a 31 x 30 Q1 mesh) leave the
    filtered block unresolved: no Ritz value <= gamma appears in the first outer steps.
    Without the resolution guard the stopping rule reported success there with 0 of the 10
    eigenpairs; with it the run does not claim success, and status OK always comes with the
    exact count of the dense eigensolver.  A run that resolves (It_max = 5) is not delayed."""
    p = si.q1_scalar((31, 30), dirichlet_face=(0, 0))
    A, B = p.A(), p.B()
    lam = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 10)
    L = int(np.ceil(1.5 * cnt))
    V1 = si.start_block(p.n, L, 3)
    r = orc.enhanced_slrf(A, B, gamma, V1, it_max=2, outer_max=30)
    assert r.status != orc.OK
    r = orc.enhanced_slrf(A, B, gamma, V1, it_max=5, outer_max=60)
    assert r.status == orc.OK and len(r.evals) == cnt
    assert np.max(np.abs(r.evals - lam[:cnt]) / lam[:cnt]) <= 1e-10


def test_preconditioned_solve_against_dense_eigh():
    """Alg. 2 with Jacobi-preconditioned inner solves returns the same
    eigenpairs: the preconditioner changes how fast, not what, the method converges to."""
    E = np.exp(np.random.default_rng(9).normal(0, 0.5, 3 * 3 * 2))
    p = si.q1_elasticity((4, 4, 3), E=E)
    A, B = p.A(), p.B()
    lam = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 10)
    V1 = si.start_block(p.n, int(np.ceil(1.5 * cnt)), 6)
    r = orc.enhanced_slrf(A, B, gamma, V1, m=8, it_max=20, outer_max=40, precond=True)
    assert r.status == orc.OK and len(r.evals) == cnt
    assert np.max(np.abs(r.evals - lam[:cnt]) / lam[:cnt]) <= 1e-9
    assert r.resid.max() <= 1e-8


def test_basic_method_agrees():
    """Alg. 1 (no locking, zero initial guesses, near-exact inner solves) finds the same
    eigenvalues.  With zero initial guesses the inner error is relative to ||B v||, so the
    eigen-residual floor is about tol_in * lambda_max / theta: tol_in = 1e-14 here."""
    nodes = (5, 5, 4)
    p, A, B = _small_q1(nodes)
    lam = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 12)
    V1 = si.start_block(p.n, int(np.ceil(1.5 * cnt)), 7)
    r = orc.enhanced_slrf(A, B, gamma, V1, m=8, it_max=400, tol_in=1e-14, outer_max=30,
                          lock=False, warm=False)
    assert r.status == orc.OK and len(r.evals) == cnt
    assert np.max(np.abs(r.evals - lam[:cnt]) / lam[:cnt]) <= 1e-9


def test_sturm_count_matches_dense():
    n = 120
    p = si.bar1d_pencil(n)
    h = 1.0 / (n + 1)
    for gamma in (50.0, 3000.0, 2.0e5):
        c = pins.sturm_count(np.full(n, 2 / h), np.full(n - 1, -1 / h), gamma,
                             np.full(n, 4 * h / 6), np.full(n - 1, h / 6))
        assert c == pins.dense_inertia_count(p.A(), p.B(), gamma) == np.sum(pins.bar1d_eigs(n) < gamma)


# ---------------------------------------------------------------- eigenvalue adjoint
def test_eig_grad_matches_finite_differences():
    """Central differences of the dense generalized eigenvalues along random symmetric
    directions on the pattern match the adjoint, for A and for B."""
    E = np.exp(np.random.default_rng(4).normal(0, 0.5, 3 * 3 * 2))
    p = si.q1_elasticity((4, 4, 3), E=E)
    Ad, Bd = p.A().toarray(), p.B().toarray()
    lam, Xf = sla.eigh(Ad, Bd)
    k = 6
    rng = np.random.default_rng(5)
    g = rng.standard_normal(k)
    gA, gB = orc.eig_grad_values(p.rowptr, p.col, lam[:k], Xf[:, :k], g)
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    for _ in range(3):
        S = np.zeros((p.n, p.n))
        S[rows, p.col] = rng.standard_normal(p.nnz)
        Dd = S + S.T  # symmetric, on the (symmetric) pattern
        dvals = Dd[rows, p.col]
        for M0, grad, other in ((Ad, gA, "A"), (Bd, gB, "B")):
            h = 1e-6 * np.abs(M0).max() / np.abs(Dd).max()
            if other == "A":
                lp = sla.eigh(Ad + h * Dd, Bd, eigvals_only=True)[:k]
                lm = sla.eigh(Ad - h * Dd, Bd, eigvals_only=True)[:k]
            else:
                lp = sla.eigh(Ad, Bd + h * Dd, eigvals_only=True)[:k]
                lm = sla.eigh(Ad, Bd - h * Dd, eigvals_only=True)[:k]
            fd = g @ (lp - lm) / (2 * h)
            pred = grad @ dvals
            assert abs(fd - pred) <= 1e-5 * abs(fd), (other, fd, pred)


# ---------------------------------------------------------------- eigenvector adjoint
def _eig_sorted(Ad, Bd, k):
    lam, X = sla.eigh(Ad, Bd)
    X = X[:, :k]
    idx = np.argmax(np.abs(X), axis=0)
    X = X * np.sign(X[idx, np.arange(k)])[None, :]  # largest entry positive (locally constant)
    return lam[:k], X


def test_eigenvector_adjoint_matches_finite_differences():
    """L = sum_i c_i lambda_i + d_i^T x_i (sign-fixed eigenvectors): central differences of
    dense generalized eigendecompositions along random symmetric pattern directions."""
    E = np.exp(np.random.default_rng(11).normal(0, 0.5, 3 * 3 * 2))
    p = si.q1_elasticity((4, 4, 3), E=E)
    Ad, Bd = p.A().toarray(), p.B().toarray()
    k = 5
    lam, X = _eig_sorted(Ad, Bd, k)
    assert np.min(np.diff(lam)) > 1e-6 * lam[-1]  # simple eigenvalues
    rng = np.random.default_rng(12)
    c = rng.standard_normal(k)
    D = rng.standard_normal((p.n, k))
    gA, gB, Xi = orc.eig_grad_full(p.rowptr, p.col, Ad, Bd, lam, X, c, D)
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    for _ in range(2):
        S = np.zeros((p.n, p.n))
        S[rows, p.col] = rng.standard_normal(p.nnz)
        Dd = S + S.T
        dv = Dd[rows, p.col]
        for which, M0, grad in (("A", Ad, gA), ("B", Bd, gB)):
            h = 1e-6 * np.abs(M0).max() / np.abs(Dd).max()
            vals = []
            for sgn in (1, -1):
                Am = Ad + sgn * h * Dd if which == "A" else Ad
                Bm = Bd + sgn * h * Dd if which == "B" else Bd
                lp, Xp = _eig_sorted(Am, Bm, k)
                vals.append(c @ lp + np.sum(D * Xp))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - grad @ dv) <= 1e-5 * abs(fd), (which, fd, grad @ dv)


def test_full_size_reference_routines_on_a_reduced_box():
    """The routines that give the full-size elasticity box its reference spectrum and count
    (shift-invert Lanczos; Sylvester inertia from a symmetric sparse LU), checked on an
    8 x 8 x 4 box of the same generator (z = 0 clamped, lognormal modulus) against dense
    eigh and the Bunch-Kaufman inertia; the oracle's Alg. 2 finds the same count there
    (Jacobi-preconditioned inner solves of It_max 30: unpreconditioned solves of that length
    leave this lognormal-modulus box unresolved after 40 outer steps)."""
    E = np.exp(np.random.default_rng(3).normal(0, 0.5, 7 * 7 * 3))
    p = si.q1_elasticity((8, 8, 4), E=E)
    A, B = p.A(), p.B()
    lam = sla.eigh(A.toarray(), B.toarray(), eigvals_only=True)
    assert np.max(np.abs(orc.shift_invert_spectrum(A, B, 30) - lam[:30]) / lam[:30]) <= 1e-11
    for want in (10, 30, 100):
        gamma, cnt = pins.gap_gamma(lam, want)
        c, ok = orc.inertia_count(A, B, gamma)
        assert ok and c == cnt == pins.dense_inertia_count(A, B, gamma)
    gamma, cnt = pins.gap_gamma(lam, 20)
    r = orc.enhanced_slrf(A, B, gamma, si.start_block(p.n, 30, 3), m=8, it_max=30, outer_max=60, precond=True)
    assert r.status == orc.OK and len(r.evals) == cnt
    assert np.max(np.abs(r.evals - lam[:cnt]) / lam[:cnt]) <= 1e-9


def test_midpoint_quadrature_filter_is_the_butterworth_function():
    """The trapezoidal (midpoint) rule on the circle through 0 and gamma gives exactly the
    rational function 1 / (1 + ((t - c)/r)^(2m)), c = r = gamma/2: its 2m poles are the
    roots of z^(2m) = -1 and its residues -z_k/(2m) (partial fractions)."""
    g = 250.0
    for m in (4, 8, 16):
        s, w = orc.quadrature_poles("midpoint", m, g)
        assert np.allclose(np.abs(s - g / 2), g / 2) and np.all(s.imag > 0)
        t = np.linspace(-0.5, 2.5, 301) * g
        ref = 1.0 / (1.0 + ((t - g / 2) / (g / 2)) ** (2 * m))
        assert np.abs(orc.filter_value(t, s, w) - ref).max() <= 1e-12


@pytest.mark.parametrize("rule", ["gauss_legendre", "gauss_chebyshev"])
def test_gauss_quadrature_filters_tend_to_the_indicator(rule):
    """Gauss-Legendre and Gauss-Chebyshev rules on the half circle: the filter is 1 at the
    centre (the weights integrate dtheta over [0, pi]: exactly for Legendre, to the rule's
    error for Chebyshev), and Phi(t) -> 1 inside / 0 outside as m grows."""
    g = 1.0
    s, w = orc.quadrature_poles(rule, 8, g)
    x, om = np.polynomial.legendre.leggauss(8)
    if rule == "gauss_legendre":
        assert abs(orc.filter_value(0.5 * g, s, w) - 1.0) <= 1e-13
        assert np.allclose(np.sort(s.real), np.sort(0.5 * g + 0.5 * g * np.cos(np.pi * (1 + x) / 2)))
    else:
        assert abs(orc.filter_value(0.5 * g, s, w) - 1.0) <= 2e-2
    errs = []
    for m in (8, 32, 128):
        s, w = orc.quadrature_poles(rule, m, g)
        t_in = np.linspace(0.2, 0.8, 61)
        t_out = np.concatenate([np.linspace(-1.0, -0.2, 41), np.linspace(1.2, 3.0, 41)])
        errs.append(max(np.abs(orc.filter_value(t_in, s, w) - 1).max(), np.abs(orc.filter_value(t_out, s, w)).max()))
    assert errs[2] < errs[1] < errs[0] and errs[2] <= 1e-3
