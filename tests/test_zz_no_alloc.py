"""The allocation-free filter apply, slrf_filter_apply_static, against slrf_filter_apply.

Some callers cannot allocate device memory: code that runs under another framework's
memory pool or budget, or a plugin that may not call cudaMalloc once it has started.
slrf_filter_apply_static serves them from a fixed static device array inside the
library.  This test calls it through the C ABI and checks that it returns what the
context-based slrf_filter_apply returns for the same input, on two calls in a row (the
second with the warm start and a new block, so stale contents of the shared array
would show), and that a problem larger than the array is refused with SLRF_EINVAL.
"""
import numpy as np
import pytest
import torch

import slrf_inputs as si
from gpu_common import rel, slrf_mod  # noqa: F401

pytestmark = pytest.mark.gpu


def test_static_filter_matches_context_filter(slrf_mod):
    n, L, m, it = 2000, 32, 8, 60
    p = si.bar1d_pencil(n)
    gamma = 4150.528
    opts = slrf_mod.slrf_opts_default(m=m, it_max=it)
    ctx = slrf_mod.Context(p.rowptr, p.col, p.valA, p.valB, gamma, L, opts)
    for seed, warm in ((3, False), (4, True)):
        X = torch.from_numpy(si.start_block(n, L, seed)).cuda()
        th = torch.linspace(0.05, 1.4, L, dtype=torch.float64, device="cuda") * gamma if warm else None
        U_ref = ctx.filter_apply(X, th)
        U = slrf_mod.filter_apply_static(ctx.rowptr, ctx.col, ctx.valA, ctx.valB, gamma, opts, X, th)
        torch.cuda.synchronize()
        assert rel(U.cpu().numpy(), U_ref.cpu().numpy()) <= 1e-8
    ctx.close()


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
