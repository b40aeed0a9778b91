"""GB300-native shifted-Laplace rational-filter eigensolver (ParaSLRF hot path).

The compute path is ``libslrf.so`` (CUDA for sm_103a behind the C ABI in
``include/slrf.h``); ``slrf`` is its marshalling-only binding.
"""
from .slrf import (Batch, Context, Opts, SlrfEigsh, SlrfError, Stats, filter_apply_static, lib,  # noqa: F401
                   slrf_opts_default, slrf_solve_host, strerror, tsgemm, tsgram)
