"""Plain FP64 CPU oracle of the enhanced shifted-Laplace rational filter (ParaSLRF).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  It shares no code with the CUDA
library and is deliberately slow and literal: numpy/scipy in float64/complex128, each
function following one step of the method in the paper's order.

Sources (arXiv 2510.17334):
  * rational filter Phi(lambda) = sum_j w_j/(lambda - sigma_j)         -- Sec. 2, eq. (3)
  * conjugate poles sigma_{N+j} = conj(sigma_j), w_{N+j} = conj(w_j);
    filtered block U = sum_j 2 Re(w_j Y_j)                              -- Sec. 2, Alg. 1
  * shifted systems (A - sigma_j B) Y = B V                             -- Sec. 1, eq. (2)
  * poles on the lines y = x(1 +- alpha i), alpha = 1, beta = 0.01      -- Sec. 2.2, Sec. 3.2
  * enhanced method: locking, B-orthogonalisation against locked X,
    warm start Y_init = v/(theta - sigma), fixed It_max                  -- Sec. 4, Alg. 2
  * Cayley equivalence of the warm start                                -- Sec. 4, Proposition
  * eigen-residual stopping test, inner tolerance 1e-10                 -- Sec. 3.2

Readings where the paper is silent (each listed in the design notes):
  * pole/weight design: sigma_j = gamma x_j (1 + alpha i), x_j = (j - 1/2)/m; weights
    minimise sum_t (Phi(t) - 1[t <= gamma])^2 + beta ||w/gamma||^2 over 3000 uniform
    samples on (0, gamma] and 3000 geometric samples on [1.3 gamma, 51 gamma]
    (beta read as a Tikhonov weight; the band (gamma, 1.3 gamma) is not fitted).
  * inner solver: COCG (unconjugated bilinear form), stop per column at
    ||r||/||r0|| <= tol_in or It_max updates (r0 the warm-started initial residual,
    i.e. the Cayley system's own right-hand side by the Proposition).
  * locking test: ||A v - theta B v|| / ||A v|| <= tol_eig and 0 < theta <= gamma.
  * orthogonalisation: CGS2 in the B-inner product; B-orthonormalisation: Cholesky-QR2;
    Rayleigh-Ritz on the standard problem U^T A U (U B-orthonormal).
  * stopping: no active Ritz value <= gamma left after locking, two outer steps in a row,
    each with the lowest active Ritz pair resolved (relative residual <= GUARD_RES = 1e-2):
    the paper stops once the NEV wanted pairs converged; without NEV, an unresolved
    subspace (short inner solves on a large mesh) can show no Ritz value <= gamma yet.
  * start block: standard Gaussian (PCG64); first-step initial guess y0 = 0.
  * eigenvector sign: the entry of largest magnitude is made positive.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

# status codes mirrored by the library's documented semantics (not shared code)
OK = 0
E_CHOL = -6
GUARD_RES = 1e-2  # lowest active Ritz pair must be this well resolved before the stop test counts
E_NOCONV = -7


# ----------------------------------------------------------------------------------------
# Poles and weights (Sec. 2.2 takes the formula from a companion paper: midpoint abscissae,
# weights fitted to the indicator of (0, gamma] with a Tikhonov term)
# ----------------------------------------------------------------------------------------
def slrf_poles(m: int, gamma: float, alpha: float = 1.0, beta: float = 0.01, band: float = 1.3,
               n_in: int = 3000, n_out: int = 3000, t_max: float = 51.0):
    """Upper-half-plane poles sigma_j and weights w_j (j = 1..m) of the SLRF filter.

    Poles lie on the line Im = alpha * Re (Sec. 2.2, sigma = Re(sigma)(1 + alpha i)).
    Weights are the Tikhonov-regularised least-squares fit of the interval indicator.
    Everything is designed on the normalised axis t/gamma and then scaled by gamma.
    """
    x = (np.arange(1, m + 1) - 0.5) / m
    sig_hat = x * (1.0 + 1j * alpha)
    t_in = (np.arange(n_in) + 0.5) / n_in
    t_out = np.geomspace(band, t_max, n_out)
    t = np.concatenate([t_in, t_out])
    f = np.concatenate([np.ones(n_in), np.zeros(n_out)])
    C = 1.0 / (t[:, None] - sig_hat[None, :])
    # Phi(t) = sum_j 2 Re(w_j C_j(t)) = sum_j 2 (Re w_j Re C_j - Im w_j Im C_j)
    G = np.hstack([2.0 * C.real, -2.0 * C.imag])
    lhs = G.T @ G + beta * np.eye(2 * m)
    rhs = G.T @ f
    u = np.linalg.solve(lhs, rhs)
    w_hat = u[:m] + 1j * u[m:]
    return gamma * sig_hat, gamma * w_hat


def quadrature_poles(rule: str, m: int, gamma: float):
    """Upper-half poles and weights of the classical contour-integral filters the paper
    compares with (Sec. 1, Table 1): the indicator of the interval written as the Cauchy
    integral -(1/2 pi i) int dz/(t - z) over the circle z = c + r e^{i theta} through 0 and
    gamma (c = r = gamma/2), with a quadrature rule on the upper half theta in [0, pi]; the
    lower half is the conjugate, so Phi(t) = sum_j 2 Re(w_j/(t - sigma_j)) as for SLRF.
      midpoint:        theta_j = pi (j - 1/2)/m,            w_j = -r e^{i theta_j} / (2m)
      gauss_legendre:  theta_j = pi (1 + x_j)/2, x_j, omega_j the Gauss-Legendre rule on
                       [-1, 1],                               w_j = -r e^{i theta_j} omega_j / 4
      gauss_chebyshev: x_j = cos((2j - 1) pi/(2m)), omega_j = (pi/m) sqrt(1 - x_j^2) (the
                       Chebyshev rule applied to int f(x) dx), theta_j as above,
                                                              w_j = -r e^{i theta_j} omega_j / 4
    """
    c = r = 0.5 * gamma
    j = np.arange(1, m + 1)
    if rule == "midpoint":
        th = np.pi * (j - 0.5) / m
        om = np.full(m, 2.0 / m)  # so that w = -r e^{i theta} om / 4 = -r e^{i theta}/(2m)
    elif rule == "gauss_legendre":
        x, om = np.polynomial.legendre.leggauss(m)
        th = np.pi * (1.0 + x) / 2.0
    elif rule == "gauss_chebyshev":
        x = np.cos((2 * j - 1) * np.pi / (2 * m))
        om = (np.pi / m) * np.sqrt(1.0 - x * x)
        th = np.pi * (1.0 + x) / 2.0
    else:
        raise ValueError(rule)
    e = np.exp(1j * th)
    return c + r * e, -r * e * om / 4.0


def filter_value(t, sigma, w):
    """Phi(t) for real t with the conjugate half implied: sum_j 2 Re(w_j / (t - sigma_j))."""
    t = np.asarray(t, dtype=np.float64)
    return np.sum(2.0 * np.real(w[None, :] / (t.reshape(-1, 1) - sigma[None, :])), axis=1).reshape(t.shape)


# ----------------------------------------------------------------------------------------
# COCG on (A - sigma B) y = b, columns independent
# ----------------------------------------------------------------------------------------
@dataclass
class CocgInfo:
    iters: np.ndarray  # updates performed per column
    relres: np.ndarray  # final recurrence ||r|| / ||b||
    breakdown: np.ndarray  # bool per column


def cocg(A: sp.csr_matrix, B: sp.csr_matrix, sigma, b: np.ndarray, y0: np.ndarray,
         it_max: int, tol: float, d: np.ndarray | None = None):
    """Conjugate orthogonal CG for the complex-symmetric M = A - sigma B, one RHS per column.

    ``sigma`` is a scalar or one shift per column (columns are independent systems).
    Textbook COCG (van der Vorst & Melissen): CG with the unconjugated form x^T y.
      r = b - M y0, p = r, rho = r^T r
      repeat: q = M p; mu = p^T q; alpha = rho/mu; y += alpha p; r -= alpha q;
              stop if ||r|| <= tol ||r0|| or It_max updates; rho' = r^T r;
              beta = rho'/rho; p = r + beta p.
    The tolerance is relative to the initial residual r0 = b - M y0.  With the warm start
    y0 = v/(theta - sigma) this is the relative residual of the equivalent Cayley system
    (A - sigma B) u = (A - theta B) v solved from u0 = 0 (Sec. 4, Proposition (i)); with
    y0 = 0 it is the usual ||r||/||b||.
    A column whose mu or rho vanishes (or is not finite) stops and is flagged.

    Jacobi preconditioning (the paper preconditions its inner solver, Sec. 3.2; here the
    diagonal of A, applied on both sides so that the system stays complex symmetric):
    with ``d`` (the positive diagonal of D) the same iteration runs on the symmetrically
    scaled system  (D^-1/2 M D^-1/2) z = D^-1/2 b  from z0 = D^1/2 y0, and y = D^-1/2 z.
    The scaled matrix is still complex symmetric, so COCG applies unchanged; residuals,
    the stopping test and the returned relres are those of the scaled system.  d = None
    is the unpreconditioned method (the scale is exactly 1).
    """
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.complex128), (b.shape[1],))
    s = np.ones(b.shape[0]) if d is None else 1.0 / np.sqrt(np.asarray(d, dtype=np.float64))
    s = s[:, None]

    def M(X):
        # D^-1/2 (A - sigma B) D^-1/2 X
        return s * ((A @ (s * X)) - (B @ (s * X)) * sig[None, :])

    y = y0.astype(np.complex128, copy=True) / s  # z0 = D^1/2 y0 (the loop works on z)
    r = s * b.astype(np.complex128) - M(y)
    rn = np.linalg.norm(r, axis=0)
    bn = rn.copy()  # ||r0||
    active = rn > 0
    iters = np.zeros(b.shape[1], dtype=np.int64)
    brk = np.zeros(b.shape[1], dtype=bool)
    p = r.copy()
    rho = np.sum(r * r, axis=0)
    for _ in range(it_max):
        if not active.any():
            break
        q = M(p)
        mu = np.sum(p * q, axis=0)
        bad = active & ((mu == 0) | ~np.isfinite(mu))
        brk |= bad
        active &= ~bad
        alpha = np.where(active, rho / np.where(mu == 0, 1, mu), 0)
        y += alpha[None, :] * p
        r -= alpha[None, :] * q
        iters += active
        rn = np.linalg.norm(r, axis=0)
        active &= ~(rn <= tol * bn)
        rho_new = np.sum(r * r, axis=0)
        bad = active & ((rho == 0) | ~np.isfinite(rho_new))
        brk |= bad
        active &= ~bad
        beta = np.where(active, rho_new / np.where(rho == 0, 1, rho), 0)
        rho = rho_new
        p = r + beta[None, :] * p
    relres = np.where(bn > 0, rn / np.where(bn > 0, bn, 1), 0.0)  # ||r|| / ||r0||
    return s * y, CocgInfo(iters, relres, brk)  # y = D^-1/2 z


# ----------------------------------------------------------------------------------------
# Filter apply  U = sum_j 2 Re(w_j Y_j),  (A - sigma_j B) Y_j = B V
# ----------------------------------------------------------------------------------------
@dataclass
class FilterInfo:
    iters: np.ndarray  # (m, k)
    relres: np.ndarray  # (m, k)
    breakdown: np.ndarray  # (m, k)


def filter_apply(A, B, V, theta, sigma, w, it_max, tol, d=None):
    """Apply the rational filter to the real block V (n x k), the filter step of Alg. 2.

    ``theta`` = None gives the zero initial guess; otherwise column c starts from
    y0 = v_c / (theta_c - sigma_j) (the warm start of Alg. 2).  All m x k systems are solved
    side by side as independent columns, pole-major: column j*k + c is pole j, vector c.
    ``d``: diagonal of the Jacobi preconditioner of every shifted system (None: none).
    """
    n, k = V.shape
    m = len(sigma)
    b = B @ V
    bb = np.tile(b, (1, m))
    sig_cols = np.repeat(np.asarray(sigma), k)
    if theta is None:
        y0 = np.zeros((n, m * k), dtype=np.complex128)
    else:
        th = np.tile(np.asarray(theta, dtype=np.float64), m)
        y0 = np.tile(V, (1, m)) / (th[None, :] - sig_cols[None, :])
    Y, info = cocg(A, B, sig_cols, bb, y0, it_max, tol, d)
    U = np.zeros((n, k))
    for j in range(m):
        U += 2.0 * np.real(w[j] * Y[:, j * k:(j + 1) * k])
    return U, FilterInfo(info.iters.reshape(m, k), info.relres.reshape(m, k),
                         info.breakdown.reshape(m, k))


# ----------------------------------------------------------------------------------------
# B-orthogonalise against the locked vectors (first step of the outer update of Alg. 2), CGS2
# ----------------------------------------------------------------------------------------
def b_orth(U, X, BX):
    """U <- U - X (X^T B U), twice, using the stored B X."""
    for _ in range(2):
        U = U - X @ (BX.T @ U)
    return U


# ----------------------------------------------------------------------------------------
# Cholesky-QR2 in the B-inner product
# ----------------------------------------------------------------------------------------
def cholqr2(U, B):
    """Two passes of G = U^T B U, G = R^T R, U <- U R^{-1}.  Returns (U, status)."""
    for _ in range(2):
        G = U.T @ (B @ U)
        try:
            Lc = np.linalg.cholesky(G)
        except np.linalg.LinAlgError:
            return U, E_CHOL
        R = Lc.T
        U = sla.solve_triangular(R, U.T, trans="T", lower=False).T
    return U, OK


# ----------------------------------------------------------------------------------------
# Rayleigh-Ritz on the B-orthonormal basis (Alg. 2)
# ----------------------------------------------------------------------------------------
def rayleigh_ritz(U, A):
    """theta ascending and V = U S from the eigenpairs of H = U^T A U."""
    H = U.T @ (A @ U)
    theta, S = np.linalg.eigh(H)
    V = U @ S
    return theta, V


def sign_normalise(V):
    """Flip each column so that its entry of largest magnitude is positive."""
    idx = np.argmax(np.abs(V), axis=0)
    s = np.sign(V[idx, np.arange(V.shape[1])])
    s[s == 0] = 1
    return V * s[None, :]


# ----------------------------------------------------------------------------------------
# Residuals, convergence, locking
# ----------------------------------------------------------------------------------------
def ritz_residuals(A, B, V, theta):
    """Relative residual ||A v - theta B v||_2 / ||A v||_2 per column, and the paper's
    form ||(A - theta B) v||_2 / (theta ||v||_B) (Sec. 3.2)."""
    AV = A @ V
    BV = B @ V
    R = AV - BV * theta[None, :]
    rn = np.linalg.norm(R, axis=0)
    res = rn / np.linalg.norm(AV, axis=0)
    vb = np.sqrt(np.sum(V * BV, axis=0))
    res_paper = rn / (np.abs(theta) * vb)
    return res, res_paper, BV


@dataclass
class SolveResult:
    status: int
    evals: np.ndarray
    X: np.ndarray
    resid: np.ndarray
    outer_iters: int
    trace: list = field(default_factory=list)


def enhanced_slrf(A, B, gamma, V1, m=8, it_max=40, tol_in=1e-10, tol_eig=1e-8, outer_max=100,
                  alpha=1.0, beta=0.01, lock=True, warm=True, poles=None, keep_trace=False, precond=False):
    """Enhanced ParaSLRF, Alg. 2, on one address space.

    Returns the locked eigenpairs sorted ascending.  ``lock`` = False / ``warm`` = False
    give the basic method of Alg. 1 (no locking, zero initial guesses).  ``precond`` = True
    solves every shifted system with the Jacobi preconditioner D = diag(A) (see ``cocg``).
    """
    A = sp.csr_matrix(A)
    B = sp.csr_matrix(B)
    d = A.diagonal() if precond else None
    n, L = V1.shape
    sigma, w = slrf_poles(m, gamma, alpha, beta) if poles is None else poles
    V = np.array(V1, dtype=np.float64)
    theta = None
    X = np.zeros((n, 0))
    BX = np.zeros((n, 0))
    Theta = np.zeros(0)
    Res = np.zeros(0)
    quiet = 0
    trace = []
    status = E_NOCONV
    k = 0
    for k in range(1, outer_max + 1):
        U, finfo = filter_apply(A, B, V, theta if warm else None, sigma, w, it_max, tol_in, d)
        if X.shape[1] > 0:
            U = b_orth(U, X, BX)
        U, st = cholqr2(U, B)
        if st != OK:
            status = st
            break
        th, V = rayleigh_ritz(U, A)
        V = sign_normalise(V)
        res, res_paper, BV = ritz_residuals(A, B, V, th)
        conv = (res <= tol_eig) & (th > 0) & (th <= gamma)
        if keep_trace:
            trace.append(dict(k=k, n_act=V.shape[1], theta=th.copy(), res=res.copy(),
                              n_lock=int(conv.sum()), inner_iters=finfo.iters.copy()))
        if lock:
            X = np.hstack([X, V[:, conv]])
            BX = np.hstack([BX, BV[:, conv]])
            Theta = np.concatenate([Theta, th[conv]])
            Res = np.concatenate([Res, res[conv]])
            V = V[:, ~conv]
            theta = th[~conv]
            # the stop claim ("no eigenvalue <= gamma left") holds only once the subspace
            # resolves the spectrum next to gamma: the lowest active Ritz pair must have a
            # relative residual <= GUARD_RES (reading of the stopping rule, see module doc)
            res_act = res[~conv]
            unresolved = theta.size > 0 and not res_act[np.argmin(theta)] <= GUARD_RES
            pending = bool(np.any(theta <= gamma)) or unresolved
        else:
            # Alg. 1: nothing is locked; the wanted Ritz pairs are the result once all converge
            want = (th > 0) & (th <= gamma)
            pending = not np.all(conv[want]) or not want.any()
            Xout, Theta, Res = V[:, want], th[want], res[want]
            theta = th
        quiet = 0 if pending else quiet + 1
        if quiet >= 2:
            status = OK
            break
    if not lock:
        X = Xout
    order = np.argsort(Theta, kind="stable")
    return SolveResult(status, Theta[order], X[:, order], Res[order], k, trace)


# ----------------------------------------------------------------------------------------
# Eigenvalue adjoint on the pattern
# ----------------------------------------------------------------------------------------
def eig_grad_values(rowptr, col, evals, X, g_eval):
    """dL/dA_e and dL/dB_e for L with dL/dlambda_i = g_i, every stored entry e = (r, c) an
    independent parameter:  d lambda_i = x_i^T (dA - lambda_i dB) x_i  for B-normalised x_i
    (first-order perturbation of a simple eigenvalue of a symmetric-definite pencil)."""
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    # per entry: sum_i g_i x_i[r] x_i[c] and sum_i g_i lambda_i x_i[r] x_i[c]
    prod = X[rows, :] * X[np.asarray(col), :]
    gA = prod @ np.asarray(g_eval)
    gB = -(prod @ (np.asarray(g_eval) * np.asarray(evals)))
    return gA, gB


# ----------------------------------------------------------------------------------------
# Eigenvector adjoint on the pattern (dense reference for small pencils)
# ----------------------------------------------------------------------------------------
def eig_grad_full(rowptr, col, A, B, evals, X, g_eval, g_X):
    """dL/dA_e, dL/dB_e for a loss with dL/dlambda_i = g_i and dL/dx_i = g_x_i (x_i
    B-normalised, simple eigenvalues).  First-order perturbation:
      (A - lambda_i B) dx_i = -(dA - lambda_i dB - dlambda_i B) x_i,  x_i^T B dx_i = -1/2 x_i^T dB x_i.
    With xi_i solving (A - lambda_i B) xi_i = -(I - B x_i x_i^T) g_x_i, x_i^T B xi_i = 0:
      dL = sum_i [g_i x_i^T (dA - l_i dB) x_i + xi_i^T (dA - l_i dB) x_i - 1/2 (g_x_i^T x_i) x_i^T dB x_i].
    Dense: xi_i is the least-squares solution of the singular system projected B-orthogonally."""
    A = np.asarray(A.toarray() if hasattr(A, "toarray") else A)
    B = np.asarray(B.toarray() if hasattr(B, "toarray") else B)
    n, k = X.shape
    Xi = np.zeros((n, k))
    for i in range(k):
        x = X[:, i]
        rhs = -(g_X[:, i] - B @ x * (x @ g_X[:, i]))
        xi, *_ = np.linalg.lstsq(A - evals[i] * B, rhs, rcond=None)
        Xi[:, i] = xi - x * (x @ (B @ xi))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    cols = np.asarray(col)
    gA = (X[rows, :] * X[cols, :]) @ np.asarray(g_eval) + np.sum(Xi[rows, :] * X[cols, :], axis=1)
    half = 0.5 * np.sum(g_X * X, axis=0)
    gB = -((X[rows, :] * X[cols, :]) @ (np.asarray(g_eval) * evals + half)
           + (Xi[rows, :] * X[cols, :]) @ np.asarray(evals))
    return gA, gB, Xi


# ----------------------------------------------------------------------------------------
# O-result at full size: the plain definition of the answer (the eigenpairs in (0, gamma]),
# from library routines rather than from the method (used to pin large workloads)
# ----------------------------------------------------------------------------------------
def shift_invert_spectrum(A, B, k: int, tol: float = 1e-12):
    """The k smallest eigenvalues of A x = lambda B x (A, B sparse SPD), ascending, by
    shift-invert Lanczos at sigma = 0 (ARPACK through scipy.sparse.linalg.eigsh, with a
    sparse LU of A from SuperLU)."""
    import scipy.sparse.linalg as spla

    A = sp.csc_matrix(A)
    B = sp.csc_matrix(B)
    lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))
    op = spla.LinearOperator(A.shape, matvec=lu.solve, dtype=np.float64)
    vals = spla.eigsh(A, k=k, M=B, sigma=0.0, which="LM", OPinv=op, return_eigenvectors=False, tol=tol)
    return np.sort(vals)


def inertia_count(A, B, gamma: float):
    """Number of eigenvalues below gamma of the pencil (A, B) by Sylvester's law of inertia:
    the negative pivots of a symmetric factorisation P (A - gamma B) P^T = L D L^T.  SuperLU
    in symmetric mode with diagonal pivoting only (diag_pivot_thresh = 0) factors
    P M P^T = L U with U = D L^T for the symmetric M, so the signs of U's diagonal are those
    of D.  Returns (count, ok): ok is False when the row and column orderings differ (the
    factorisation is then not congruent and the count is not trusted)."""
    import scipy.sparse.linalg as spla

    M = sp.csc_matrix(A - gamma * B)
    lu = spla.splu(M, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                   options=dict(SymmetricMode=True))
    ok = bool(np.array_equal(lu.perm_r, lu.perm_c))
    d = lu.U.diagonal()
    return int(np.sum(d < 0)), ok
