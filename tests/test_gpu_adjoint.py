"""Eigenvalue adjoint (a12) on the GPU against the oracle's adjoint and, through the
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


def test_eig_grad_matches_oracle(slrf_mod):
    E = np.exp(np.random.default_rng(3).normal(0, 0.5, 5 * 5 * 4))
    p = si.q1_elasticity((6, 6, 5), E=E)
    lam = sla.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 12)
    L = int(np.ceil(1.5 * cnt))
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, slrf_mod.slrf_opts_default(it_max=60))
    rc, nf, ev, X, rs, st = ctx.solve(torch.from_numpy(si.start_block(p.n, L, 2)))
    assert nf == cnt
    g = np.random.default_rng(6).standard_normal(nf)
    gA, gB = ctx.eig_grad(ev, X, torch.from_numpy(g))
    oA, oB = orc.eig_grad_values(p.rowptr, p.col, ev.cpu().numpy(), X.cpu().numpy(), g)
    assert rel(gA.cpu().numpy(), oA) <= 1e-12
    assert rel(gB.cpu().numpy(), oB) <= 1e-12
    # closed form x_i^T (dA - lambda_i dB) x_i along a random symmetric direction
    rows = np.repeat(np.arange(p.n), np.diff(p.rowptr))
    S = np.zeros((p.n, p.n))
    S[rows, p.col] = np.random.default_rng(7).standard_normal(p.nnz)
    D = S + S.T
    Xn = X.cpu().numpy()
    dlam = np.einsum("ij,ik,kj->j", Xn, D, Xn)
    assert abs(gA.cpu().numpy() @ D[rows, p.col] - g @ dlam) <= 1e-10 * np.abs(g @ dlam)
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
