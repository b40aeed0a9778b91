"""The C-ABI library builds, loads and exports every symbol that include/slrf.h declares.
Host-only entry points are exercised; nothing here launches GPU work."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_17334_gb300 import build

    build.build()
    from paper_2510_17334_gb300 import slrf

    return slrf.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "slrf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(slrf_\w+)\s*\(", txt, re.M)))


def test_header_declarations_are_exported(lib):
    names = _declared()
    assert "slrf_solve" in names and "slrf_setup" in names and "slrf_filter_apply" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_2510_17334_gb300 import slrf

    assert set(_declared()) <= set(slrf.SYMBOLS)


def test_opts_default_and_strerror(lib):
    from paper_2510_17334_gb300 import slrf

    o = slrf.slrf_opts_default()
    assert (o.m, o.alpha, o.beta, o.it_max, o.tol_inner, o.tol_eig) == (8, 1.0, 0.01, 40, 1e-10, 1e-8)
    assert o.warm_start == 1 and o.lock == 1 and o.precision == 0
    assert slrf.strerror(0) == "ok"
    assert "Cholesky" in slrf.strerror(slrf.SLRF_ECHOL)
    assert lib.slrf_opts_default(None) == slrf.SLRF_EINVAL


def test_setup_rejects_invalid_arguments_before_touching_the_device(lib):
    from paper_2510_17334_gb300 import slrf

    h = ct.c_void_p(123)
    assert lib.slrf_setup(ct.byref(h), None, 1.0, 4, None, None) == slrf.SLRF_EINVAL
    assert h.value is None
    pair = slrf.CsrPair(10, 28, None, None, None, None)
    assert lib.slrf_setup(ct.byref(h), ct.byref(pair), 1.0, 4, None, None) == slrf.SLRF_EINVAL
    assert lib.slrf_filter_apply(None, None, 1, None, None) == slrf.SLRF_EINVAL
    assert lib.slrf_solve(None, None, 0, None, None, None, None, None) == slrf.SLRF_EINVAL
    lib.slrf_destroy(None)
