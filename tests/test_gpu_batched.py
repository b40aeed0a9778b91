"""Batched uneven pencils: several independent problems of different families and
sizes solved in one batch, whose COCG phases run as one persistent launch.

Checks: every problem's eigenvalues against a dense generalized eigensolver (count
exact; FP64 <= 1e-10 relative, mixed <= 1e-8), residuals <= 1e-8, and -- since the
batched kernels run the same per-block arithmetic as the single-problem kernels -- the
FP64 batch is bitwise equal to solving each problem on its own with the same plain-CSR
SpMM (slrf_opts.group = 1, the format the persistent batched launches gather through).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import torch

import pins
import slrf_inputs as si
from gpu_common import slrf_mod  # noqa: F401

pytestmark = pytest.mark.gpu


def _problems():
    probs = [si.bar1d_pencil(300),
             si.q1_scalar((20, 21), coef=np.exp(np.random.default_rng(1).normal(0, 0.3, 19 * 20)),
                          dirichlet_face=(0, 0)),
             si.q1_scalar((7, 6, 5), dirichlet_face=(0, 0)),
             si.q1_elasticity((4, 4, 3), E=np.exp(np.random.default_rng(2).normal(0, 0.5, 18))),
             si.q1_scalar((9, 9, 9), shift=1e-3)]
    wants = [10, 14, 9, 8, 20]
    out = []
    for p, want in zip(probs, wants):
        lam = sla.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
        gamma, cnt = pins.gap_gamma(lam, want)
        out.append((p, lam, gamma, cnt, int(np.ceil(1.5 * cnt))))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_solve(slrf_mod, precision):
    probs = _problems()
    opts = slrf_mod.slrf_opts_default(it_max=40, precision=precision)
    V0 = [si.start_block(p.n, L, 10 + i) for i, (p, lam, g, c, L) in enumerate(probs)]
    batch = slrf_mod.Batch([(p.rowptr, p.col, p.valA, p.valB) for p, *_ in probs], [g for _, _, g, _, _ in probs],
                           [L for *_, L in probs], opts)
    rc, res, st = batch.solve(V0)
    assert rc == 0
    tol = 1e-10 if precision == 0 else 1e-8
    for i, ((p, lam, g, cnt, L), (status, nf, ev, X, rs)) in enumerate(zip(probs, res)):
        ev = ev.cpu().numpy()
        assert status == 0 and nf == cnt, (i, status, nf, cnt)
        assert np.all(np.abs(ev - lam[:cnt]) <= np.maximum(tol * lam[:cnt], 1e-9 * lam[0])), i
        assert rs.max().item() <= 1e-8
        if precision == 0:
            opts1 = slrf_mod.slrf_opts_default(it_max=40, precision=precision, group=1)
            ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, g, L, opts1)
            _, nf1, ev1, X1, rs1, _ = ctx.solve(torch.from_numpy(V0[i]))
            assert nf1 == nf and np.array_equal(ev1.cpu().numpy(), ev), i
            assert torch.equal(X1, X), i
            ctx.close()
    assert st["n_conv"] == sum(c for _, _, _, c, _ in probs)
    # the shared COCG launches are timed apart from the per-problem phases
    assert 0.0 < st["ms_filter"] < st["ms_total"] and st["ms_dense"] > 0.0
    assert abs(st["ms_filter"] + st["ms_dense"] - st["ms_total"]) <= 1e-6 * st["ms_total"] + 1e-9
    batch.close()


def test_autotuned_setup_solves_correctly(slrf_mod):
    """The rows-per-block autotuner changes only the COCG blocking (and with it the rounding
    order of the block reductions): the eigenpairs stay within the FP64 tolerance."""
    nodes = (13, 13, 13)
    p = si.q1_scalar(nodes, shift=1e-3)
    lam = pins.q1_neumann_eigs(nodes, 1e-3)
    gamma, cnt = pins.gap_gamma(lam, 40)
    L = int(np.ceil(1.5 * cnt))
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, slrf_mod.slrf_opts_default(it_max=30, autotune=1))
    rc, nf, ev, X, rs, st = ctx.solve(torch.from_numpy(si.start_block(p.n, L, 2)))
    ev = ev.cpu().numpy()
    assert rc == 0 and nf == cnt
    assert np.all(np.abs(ev - lam[:cnt]) <= np.maximum(1e-10 * lam[:cnt], 1e-9 * lam[0]))
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_adaptive_it_max(slrf_mod, precision):
    """A batch whose shared start It_max (3) is too short for one of its problems (the 31 x 30
    mesh): with opts.it_adapt each problem's It_max grows on its own and every problem
    returns its exact count; the fast problems keep their short solves."""
    probs = _problems()[:3]
    p = si.q1_scalar((31, 30), dirichlet_face=(0, 0))
    lam = sla.eigh(p.A().toarray(), p.B().toarray(), eigvals_only=True)
    gamma, cnt = pins.gap_gamma(lam, 10)
    probs.append((p, lam, gamma, cnt, int(np.ceil(1.5 * cnt))))
    opts = slrf_mod.slrf_opts_default(it_max=3, it_adapt=1, precision=precision, outer_max=150)
    V0 = [si.start_block(q.n, L, 20 + i) for i, (q, _, _, _, L) in enumerate(probs)]
    batch = slrf_mod.Batch([(q.rowptr, q.col, q.valA, q.valB) for q, *_ in probs], [g for _, _, g, _, _ in probs],
                           [L for *_, L in probs], opts)
    rc, res, st = batch.solve(V0)
    assert rc == 0
    tol = 1e-10 if precision == 0 else 1e-8
    for (q, lam_q, g, c, L), (status, nf, ev, X, rs) in zip(probs, res):
        ev = ev.cpu().numpy()
        assert status == 0 and nf == c
        assert np.all(np.abs(ev - lam_q[:c]) <= np.maximum(tol * lam_q[:c], 1e-9 * lam_q[0]))
        assert rs.max().item() <= 1e-8
    batch.close()
