"""The allocation-free filter apply, slrf_filter_apply_static, against slrf_filter_apply.

Some callers cannot allocate device memory: code that runs under another framework's
memory pool or budget, or a plugin that may not call cudaMalloc once it has started.
slrf_filter_apply_static serves them from a fixed static device array inside the
library.  These tests call it through the C ABI and check
  * that it returns what the context-based slrf_filter_apply returns for the same input,
    on two calls in a row (the second with the warm start and a new block, so stale
    contents of the shared array would show), into a preallocated output;
  * that a call after the first ones changes neither torch's reserved memory nor the
    device's free memory (the claim that the call allocates nothing);
  * that a user pole table (slrf_opts.poles / weights) gives what the context gives;
  * that a problem larger than the array and a malformed pattern are refused with
    SLRF_EINVAL before any kernel gathers through them.
"""
import numpy as np
import pytest
import torch

import slrf_inputs as si
from gpu_common import rel, slrf_mod  # noqa: F401
from oracle import slrf_oracle as orc

pytestmark = pytest.mark.gpu

N, L, M, IT = 2000, 32, 8, 60
GAMMA = 4150.528


@pytest.fixture(scope="module")
def bar_ctx(slrf_mod):
    p = si.bar1d_pencil(N)
    opts = slrf_mod.slrf_opts_default(m=M, it_max=IT)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, GAMMA, L, opts)
    yield p, opts, ctx
    ctx.close()


def _inputs(seed, warm):
    X = torch.from_numpy(si.start_block(N, L, seed)).cuda()
    th = torch.linspace(0.05, 1.4, L, dtype=torch.float64, device="cuda") * GAMMA if warm else None
    return X, th


def test_static_filter_matches_context_filter(slrf_mod, bar_ctx):
    p, opts, ctx = bar_ctx
    U = torch.empty((N, L), dtype=torch.float64, device="cuda")
    for seed, warm in ((3, False), (4, True)):
        X, th = _inputs(seed, warm)
        U_ref = ctx.filter_apply(X, th)
        out = slrf_mod.filter_apply_static(ctx.rowptr, ctx.col, ctx.valA, ctx.valB, GAMMA, opts, X, th, U=U)
        torch.cuda.synchronize()
        assert out.data_ptr() == U.data_ptr()
        assert rel(U.cpu().numpy(), U_ref.cpu().numpy()) <= 1e-8


def test_static_filter_allocates_nothing(slrf_mod, bar_ctx):
    p, opts, ctx = bar_ctx
    U = torch.empty((N, L), dtype=torch.float64, device="cuda")
    ins = [_inputs(5, False), _inputs(6, True)]
    for X, th in ins:  # first calls: kernels load, the pole table is designed
        slrf_mod.filter_apply_static(ctx.rowptr, ctx.col, ctx.valA, ctx.valB, GAMMA, opts, X, th, U=U)
    torch.cuda.synchronize()
    reserved = torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    for X, th in ins:
        slrf_mod.filter_apply_static(ctx.rowptr, ctx.col, ctx.valA, ctx.valB, GAMMA, opts, X, th, U=U)
        torch.cuda.synchronize()
        assert torch.cuda.memory_reserved() == reserved
        assert torch.cuda.mem_get_info()[0] == free0
    U_ref = ctx.filter_apply(*ins[1])
    assert rel(U.cpu().numpy(), U_ref.cpu().numpy()) <= 1e-8


def test_static_filter_with_a_user_pole_table(slrf_mod, bar_ctx):
    p, _, _ = bar_ctx
    s, w = orc.slrf_poles(M, GAMMA)
    opts = slrf_mod.slrf_opts_default(m=M, it_max=IT, poles=s, weights=w)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, GAMMA, L, opts)
    X, th = _inputs(7, True)
    U_ref = ctx.filter_apply(X, th)
    U = slrf_mod.filter_apply_static(ctx.rowptr, ctx.col, ctx.valA, ctx.valB, GAMMA, opts, X, th)
    torch.cuda.synchronize()
    assert rel(U.cpu().numpy(), U_ref.cpu().numpy()) <= 1e-8
    ctx.close()


def test_static_filter_rejects_a_malformed_pattern(slrf_mod, bar_ctx):
    p, opts, ctx = bar_ctx
    col = ctx.col.clone()
    col[1234] = N + 5  # column out of range: the device check refuses it before any gather
    X, _ = _inputs(8, False)
    with pytest.raises(slrf_mod.SlrfError) as e:
        slrf_mod.filter_apply_static(ctx.rowptr, col, ctx.valA, ctx.valB, GAMMA, opts, X, None)
    assert e.value.status == slrf_mod.SLRF_EINVAL
    with pytest.raises(ValueError):  # int64 column indices are refused by the binding
        slrf_mod.filter_apply_static(ctx.rowptr, ctx.col.long(), ctx.valA, ctx.valB, GAMMA, opts, X, None)


def test_static_filter_rejects_a_problem_larger_than_its_array(slrf_mod):
    n = 200_000  # 200,000 rows x 256 complex columns x 4 vectors x 16 B = 3.3 GB > the array
    p = si.bar1d_pencil(n)
    rowptr = torch.from_numpy(p.rowptr).cuda()
    col = torch.from_numpy(p.col).cuda()
    valA = torch.from_numpy(p.valA).cuda()
    valB = torch.from_numpy(p.valB).cuda()
    X = torch.ones((n, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(slrf_mod.SlrfError) as e:
        slrf_mod.filter_apply_static(rowptr, col, valA, valB, 100.0, slrf_mod.slrf_opts_default(), X, None)
    assert e.value.status == slrf_mod.SLRF_EINVAL
