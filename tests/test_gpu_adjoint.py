"""Eigenvalue adjoint on the GPU against the oracle's adjoint and, through the
autograd wrapper, against finite differences of whole GPU solves."""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import pins
import slrf_inputs as si
from gpu_common import rel, slrf_mod  # noqa: F401
from oracle import slrf_oracle as orc

pytestmark = pytest.mark.gpu


def _dense_pairs(p, k):
    """Independent eigenpairs (scipy dense eigh, B-normalised, largest entry positive)."""
    lam, X = sla.eigh(p.A().toarray(), p.B().toarray())
    X = X[:, :k]
    idx = np.argmax(np.abs(X), axis=0)
    X = np.ascontiguousarray(X * np.sign(X[idx, np.arange(k)])[None, :])
    return lam[:k].copy(), X


def test_eig_grad_matches_oracle(slrf_mod):
    """Eigenvalue adjoint (SDDMM on the pattern) vs the oracle's, both fed the same
    eigenpairs from a dense eigensolver; plus the closed form x_i^T (dA - l_i dB) x_i."""
    E = np.exp(np.random.default_rng(3).normal(0, 0.5, 5 * 5 * 4))
    p = si.q1_elasticity((6, 6, 5), E=E)
    lam, X = _dense_pairs(p, 12)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, 1.5 * lam[-1], 18, slrf_mod.slrf_opts_default())
    g = np.random.default_rng(6).standard_normal(12)
    gA, gB = ctx.eig_grad(torch.from_numpy(lam), torch.from_numpy(X), torch.from_numpy(g))
    oA, oB = orc.eig_grad_values(p.rowptr, p.col, lam, X, g)
    assert rel(gA.cpu().numpy(), oA) <= 1e-12
    assert rel(gB.cpu().numpy(), oB) <= 1e-12
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    S = np.zeros((p.n, p.n))
    S[rows, p.col] = np.random.default_rng(7).standard_normal(p.nnz)
    D = S + S.T
    dlam = np.einsum("ij,ik,kj->j", X, D, X)
    assert abs(gA.cpu().numpy() @ D[rows, p.col] - g @ dlam) <= 1e-10 * np.abs(g @ dlam)
    ctx.close()


def test_eigenvector_adjoint_matches_oracle(slrf_mod):
    """Eigenvector terms (block MINRES on the singular shifted systems) vs the oracle's
    dense least-squares reference, same independent eigenpairs on both sides."""
    E = np.exp(np.random.default_rng(11).normal(0, 0.5, 3 * 3 * 2))
    p = si.q1_elasticity((4, 4, 3), E=E)
    k = 5
    lam, X = _dense_pairs(p, k)
    rng = np.random.default_rng(12)
    c = rng.standard_normal(k)
    Dg = np.ascontiguousarray(rng.standard_normal((p.n, k)))
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, 1.5 * lam[-1], 8,
                           slrf_mod.slrf_opts_default(tol_inner=1e-13))
    gA, gB = ctx.eig_grad(torch.from_numpy(lam), torch.from_numpy(X), torch.from_numpy(c), torch.from_numpy(Dg))
    oA, oB, _ = orc.eig_grad_full(p.rowptr, p.col, p.A(), p.B(), lam, X, c, Dg)
    assert rel(gA.cpu().numpy(), oA) <= 1e-8
    assert rel(gB.cpu().numpy(), oB) <= 1e-8
    ctx.close()


def test_autograd_wrapper_against_finite_differences(slrf_mod):
    """d(sum_i c_i lambda_i)/d valA along a random symmetric direction, by central
    differences of two GPU solves (step 1e-6 relative) vs the backward pass."""
    n = 400
    p = si.bar1d_pencil(n)
    lam = pins.bar1d_eigs(n)
    gamma = 0.5 * (lam[7] + lam[8])
    L = 12
    opts = slrf_mod.slrf_opts_default(it_max=80)
    V0 = torch.from_numpy(si.start_block(n, L, 4))
    valA = torch.from_numpy(p.valA.copy()).requires_grad_(True)
    valB = torch.from_numpy(p.valB.copy()).requires_grad_(True)
    c = torch.from_numpy(np.random.default_rng(8).standard_normal(8))
    ev, X = slrf_mod.SlrfEigsh.apply(valA, valB, p.rowptr, p.col, gamma, L, opts, V0)
    loss = (c.cuda() * ev).sum()
    loss.backward()
    rows = np.repeat(np.arange(n), np.diff(p.rowptr))
    S = np.zeros((n, n))
    S[rows, p.col] = np.random.default_rng(9).standard_normal(p.nnz)
    d = (S + S.T)[rows, p.col]
    for which, base, grad in (("A", p.valA, valA.grad), ("B", p.valB, valB.grad)):
        h = 1e-6 * np.abs(base).max() / np.abs(d).max()
        vals = []
        for sgn in (1, -1):
            va = p.valA + sgn * h * d if which == "A" else p.valA
            vb = p.valB + sgn * h * d if which == "B" else p.valB
            ctx = slrf_mod.Context(p.rowptr, p.col, va, vb, gamma, L, opts)
            _, nf, e, *_ = ctx.solve(V0)
            vals.append(e.cpu().numpy())
            ctx.close()
        fd = c.numpy() @ (vals[0] - vals[1]) / (2 * h)
        pred = grad.cpu().numpy() @ d
        assert abs(fd - pred) <= 1e-5 * abs(fd), (which, fd, pred)


def test_autograd_wrapper_carries_eigenvector_gradients(slrf_mod):
    """A loss on eigenvalues and eigenvectors: the wrapper's backward equals slrf_eig_grad
    with the same eigenpairs and loss gradients (eigenvector terms included)."""
    n = 300
    p = si.bar1d_pencil(n)
    lam = pins.bar1d_eigs(n)
    gamma = 0.5 * (lam[5] + lam[6])
    L = 10
    opts = slrf_mod.slrf_opts_default(it_max=80)
    V0 = torch.from_numpy(si.start_block(n, L, 3))
    valA = torch.from_numpy(p.valA.copy()).requires_grad_(True)
    valB = torch.from_numpy(p.valB.copy()).requires_grad_(True)
    ev, X = slrf_mod.SlrfEigsh.apply(valA, valB, p.rowptr, p.col, gamma, L, opts, V0)
    c = torch.from_numpy(np.random.default_rng(1).standard_normal(6)).cuda()
    D = torch.from_numpy(np.random.default_rng(2).standard_normal((n, 6))).cuda()
    loss = (c * ev).sum() + (D * X).sum()
    loss.backward()
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, opts)
    gA, gB = ctx.eig_grad(ev.detach(), X.detach(), c, D)
    assert torch.allclose(valA.grad.cuda(), gA, rtol=1e-12, atol=0)
    assert torch.allclose(valB.grad.cuda(), gB, rtol=1e-12, atol=0)
    ctx.close()
