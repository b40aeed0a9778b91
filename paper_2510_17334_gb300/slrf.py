"""Thin Python binding of libslrf.so: argument marshalling only.

Every function here forwards device pointers of torch tensors (or host numpy arrays for
``slrf_solve_host``) to the C ABI declared in ``include/slrf.h``; all arithmetic runs in
the library's CUDA kernels.  The binding raises ``SlrfError`` on any non-zero status and
refuses to run without the compiled library (there is no fallback path).
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.environ.get("SLRF_LIB", os.path.join(_HERE, "libslrf.so"))

SLRF_OK = 0
SLRF_EINVAL = -1
SLRF_ENOMEM = -2
SLRF_ECUDA = -3
SLRF_EBREAKDOWN = -4
SLRF_ETIMEOUT = -5
SLRF_ECHOL = -6
SLRF_ENOCONV = -7
SLRF_ENAN = -8
SLRF_ETRUNC = -9
SLRF_ESTATE = -10

SYMBOLS = ("slrf_opts_default", "slrf_setup", "slrf_get_poles", "slrf_filter_apply", "slrf_filter_timing",
           "slrf_filter_stats",
           "slrf_rayleigh_ritz", "slrf_solve", "slrf_solve_host", "slrf_eig_grad", "slrf_destroy",
           "slrf_strerror", "slrf_last_error", "slrf_filter_apply_static", "slrf_setup_batched",
           "slrf_solve_batched", "slrf_destroy_batched", "slrf_tsgram", "slrf_tsgemm", "slrf_wait_selftest",
           "slrf_apply", "slrf_format")


class SlrfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status} ({strerror(status)})")


class CsrPair(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("nnz", ct.c_int64), ("rowptr", ct.c_void_p), ("col", ct.c_void_p),
                ("valA", ct.c_void_p), ("valB", ct.c_void_p)]


class Opts(ct.Structure):
    _fields_ = [("m", ct.c_int), ("alpha", ct.c_double), ("beta", ct.c_double), ("band", ct.c_double),
                ("it_max", ct.c_int), ("refine_max", ct.c_int), ("outer_max", ct.c_int),
                ("tol_inner", ct.c_double), ("tol_eig", ct.c_double), ("precision", ct.c_int),
                ("warm_start", ct.c_int), ("lock", ct.c_int), ("use_graph", ct.c_int), ("nev", ct.c_int),
                ("seed", ct.c_uint64), ("poles", ct.c_void_p), ("weights", ct.c_void_p), ("autotune", ct.c_int),
                ("dense", ct.c_int), ("it_adapt", ct.c_int), ("precond", ct.c_int), ("group", ct.c_int),
                ("bdiag", ct.c_int)]


class Stats(ct.Structure):
    _fields_ = [("outer_iters", ct.c_int), ("n_conv", ct.c_int), ("column_solves", ct.c_int64),
                ("column_iterations", ct.c_int64), ("breakdowns", ct.c_int), ("ms_filter", ct.c_double),
                ("ms_dense", ct.c_double), ("ms_total", ct.c_double), ("kernel_launches", ct.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib() -> ct.CDLL:
    """Load libslrf.so (built by ``paper_2510_17334_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: run paper_2510_17334_gb300.build.build() first")
        L = ct.CDLL(_LIB_PATH)
        vp, i, d, i64 = ct.c_void_p, ct.c_int, ct.c_double, ct.c_int64
        L.slrf_opts_default.argtypes = [ct.POINTER(Opts)]
        L.slrf_setup.argtypes = [ct.POINTER(vp), ct.POINTER(CsrPair), d, i, ct.POINTER(Opts), vp]
        L.slrf_get_poles.argtypes = [vp, ct.POINTER(i), vp, vp]
        L.slrf_filter_apply.argtypes = [vp, vp, i, vp, vp]
        L.slrf_apply.argtypes = [vp, vp, i, vp, vp, i]
        L.slrf_format.argtypes = [vp, ct.POINTER(i), ct.POINTER(i), ct.POINTER(i)]
        L.slrf_filter_stats.argtypes = [vp, vp, vp, vp]
        L.slrf_filter_timing.argtypes = [vp, vp, i, vp, vp, vp, vp]
        L.slrf_rayleigh_ritz.argtypes = [vp, vp, i, vp, vp, i, i, vp, vp, vp]
        L.slrf_solve.argtypes = [vp, vp, i, ct.POINTER(i), vp, vp, vp, ct.POINTER(Stats)]
        L.slrf_solve_host.argtypes = [ct.POINTER(CsrPair), d, i, ct.POINTER(Opts), vp, i, ct.POINTER(i), vp, vp, vp,
                                      ct.POINTER(Stats)]
        L.slrf_eig_grad.argtypes = [vp, i, vp, vp, i, vp, vp, vp, vp]
        L.slrf_setup_batched.argtypes = [ct.POINTER(vp), i, ct.POINTER(CsrPair), vp, vp, ct.POINTER(Opts), vp]
        L.slrf_solve_batched.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, ct.POINTER(Stats)]
        L.slrf_destroy_batched.argtypes = [vp]
        L.slrf_destroy_batched.restype = None
        L.slrf_filter_apply_static.argtypes = [ct.POINTER(CsrPair), d, ct.POINTER(Opts), vp, i, vp, vp, vp]
        L.slrf_tsgram.argtypes = [i64, vp, i, i, vp, i, i, vp, i, i, vp]
        L.slrf_tsgemm.argtypes = [i64, vp, i, i, vp, i, i, vp, i, d, d, i, vp]
        L.slrf_destroy.argtypes = [vp]
        L.slrf_destroy.restype = None
        L.slrf_strerror.argtypes = [i]
        L.slrf_strerror.restype = ct.c_char_p
        L.slrf_last_error.argtypes = [vp]
        L.slrf_wait_selftest.argtypes = [i, vp]
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().slrf_strerror(int(status)).decode()


def _check(rc: int, where: str, ok=(SLRF_OK,)):
    if rc not in ok:
        raise SlrfError(rc, where)
    return rc


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ct.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return ct.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def slrf_opts_default(**kw) -> Opts:
    o = Opts()
    _check(lib().slrf_opts_default(ct.byref(o)), "slrf_opts_default")
    keep = []
    for k, v in kw.items():
        if k in ("poles", "weights"):
            arr = np.ascontiguousarray(np.stack([np.real(v), np.imag(v)], axis=1).ravel(), dtype=np.float64)
            keep.append(arr)
            setattr(o, k, arr.ctypes.data)
        else:
            setattr(o, k, v)
    o._keep = keep  # keep host tables alive while the options are
    return o


def _dev(x, dtype):
    return x.to(device="cuda", dtype=dtype).contiguous()


class Context:
    """Owns one ``slrf_ctx`` (slrf_setup ... slrf_destroy)."""

    def __init__(self, rowptr, col, valA, valB, gamma: float, block_L: int, opts: Opts | None = None,
                 stream: torch.cuda.Stream | None = None):
        self.rowptr = _dev(torch.as_tensor(rowptr), torch.int64)
        self.col = _dev(torch.as_tensor(col), torch.int32)
        self.valA = _dev(torch.as_tensor(valA), torch.float64)
        self.valB = _dev(torch.as_tensor(valB), torch.float64)
        self.n = int(self.rowptr.numel() - 1)
        self.nnz = int(self.col.numel())
        self.gamma = float(gamma)
        self.L = int(block_L)
        self.opts = opts if opts is not None else slrf_opts_default()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        pair = CsrPair(self.n, self.nnz, _ptr(self.rowptr), _ptr(self.col), _ptr(self.valA), _ptr(self.valB))
        h = ct.c_void_p()
        _check(lib().slrf_setup(ct.byref(h), ct.byref(pair), self.gamma, self.L, ct.byref(self.opts),
                                ct.c_void_p(self.stream.cuda_stream)), "slrf_setup")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().slrf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def poles(self):
        m = ct.c_int()
        s = np.zeros(64)
        w = np.zeros(64)
        _check(lib().slrf_get_poles(self.h, ct.byref(m), _ptr(s), _ptr(w)), "slrf_get_poles")
        mm = m.value
        return s[:2 * mm:2] + 1j * s[1:2 * mm:2], w[:2 * mm:2] + 1j * w[1:2 * mm:2]

    def filter_apply(self, X: torch.Tensor, theta: torch.Tensor | None = None, U: torch.Tensor | None = None):
        X = _dev(X, torch.float64)
        k = X.shape[1]
        if U is None:
            U = torch.empty_like(X)
        th = None if theta is None else _dev(theta, torch.float64)
        _check(lib().slrf_filter_apply(self.h, _ptr(X), k, _ptr(th), _ptr(U)), "slrf_filter_apply")
        return U

    def format(self):
        """(group, bdiag, lane_width) of the COCG SpMM format chosen at setup (see slrf_format)."""
        g, bd, lw = ct.c_int(), ct.c_int(), ct.c_int()
        _check(lib().slrf_format(self.h, ct.byref(g), ct.byref(bd), ct.byref(lw)), "slrf_format")
        return g.value, bd.value, lw.value

    def apply(self, X: torch.Tensor, fp32: bool = False, want_a: bool = True, want_b: bool = True):
        """(A X, B X) with the context's matrices (see slrf_apply); an output not wanted is None."""
        X = _dev(X, torch.float64)
        k = X.shape[1]
        AX = torch.empty_like(X) if want_a else None
        BX = torch.empty_like(X) if want_b else None
        _check(lib().slrf_apply(self.h, _ptr(X), k, _ptr(AX), _ptr(BX), 1 if fp32 else 0), "slrf_apply")
        return AX, BX

    def filter_timing(self, X: torch.Tensor, theta: torch.Tensor | None = None):
        """Kernel-by-kernel CUDA-event timing of one filter apply (see slrf_filter_timing)."""
        X = _dev(X, torch.float64)
        k = X.shape[1]
        U = torch.empty_like(X)
        th = None if theta is None else _dev(theta, torch.float64)
        ms = np.zeros(4)
        cnt = np.zeros(2, dtype=np.int32)
        _check(lib().slrf_filter_timing(self.h, _ptr(X), k, _ptr(th), _ptr(U), _ptr(ms), _ptr(cnt)),
               "slrf_filter_timing")
        return {"ms_total": ms[0], "ms_spmm": ms[1], "ms_update": ms[2], "ms_init": ms[3],
                "n_spmm": int(cnt[0]), "n_update": int(cnt[1]), "U": U}

    def filter_stats(self, k: int):
        m = self.opts.m
        it = np.zeros(m * k, dtype=np.int32)
        rr = np.zeros(m * k)
        bk = np.zeros(m * k, dtype=np.int32)
        _check(lib().slrf_filter_stats(self.h, _ptr(it), _ptr(rr), _ptr(bk)), "slrf_filter_stats")
        return it.reshape(m, k), rr.reshape(m, k), bk.reshape(m, k).astype(bool)

    def rayleigh_ritz(self, U: torch.Tensor, X: torch.Tensor | None = None, BX: torch.Tensor | None = None):
        U = _dev(U, torch.float64).clone()
        k = U.shape[1]
        V = torch.empty_like(U)
        th = torch.empty(k, dtype=torch.float64, device="cuda")
        rs = torch.empty(k, dtype=torch.float64, device="cuda")
        nc = 0 if X is None else X.shape[1]
        Xd = None if X is None else _dev(X, torch.float64)
        BXd = None if BX is None else _dev(BX, torch.float64)
        _check(lib().slrf_rayleigh_ritz(self.h, _ptr(U), k, _ptr(Xd), _ptr(BXd), nc, max(nc, 1), _ptr(V), _ptr(th),
                                        _ptr(rs)), "slrf_rayleigh_ritz")
        return U, V, th, rs

    def solve(self, V0: torch.Tensor | None = None, cap: int | None = None, check: bool = True):
        cap = self.L if cap is None else int(cap)
        V0d = None if V0 is None else _dev(V0, torch.float64)
        ev = torch.zeros(max(cap, 1), dtype=torch.float64, device="cuda")
        X = torch.zeros((self.n, max(cap, 1)), dtype=torch.float64, device="cuda")
        rs = torch.zeros(max(cap, 1), dtype=torch.float64, device="cuda")
        nf = ct.c_int()
        st = Stats()
        rc = lib().slrf_solve(self.h, _ptr(V0d), cap, ct.byref(nf), _ptr(ev), _ptr(X), _ptr(rs), ct.byref(st))
        if check:
            _check(rc, "slrf_solve")
        c = min(nf.value, cap)
        return rc, nf.value, ev[:c], X[:, :c], rs[:c], st.as_dict()

    def eig_grad(self, evals, X, g_eval, g_X=None):
        evals = _dev(evals, torch.float64)
        X = _dev(X, torch.float64)
        g = _dev(g_eval, torch.float64)
        gX = None if g_X is None else _dev(g_X, torch.float64)
        gA = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
        gB = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
        k = X.shape[1]
        _check(lib().slrf_eig_grad(self.h, k, _ptr(evals), _ptr(X), k, _ptr(g), _ptr(gX), _ptr(gA), _ptr(gB)),
               "slrf_eig_grad")
        return gA, gB


class Batch:
    """Owns one ``slrf_batch`` (slrf_setup_batched ... slrf_destroy_batched): independent
    problems whose COCG phases run in one persistent launch."""

    def __init__(self, problems, gammas, blocks, opts: Opts | None = None, stream=None):
        """problems: list of (rowptr, col, valA, valB) host or device arrays."""
        self.P = len(problems)
        self.opts = opts if opts is not None else slrf_opts_default()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.mats = []
        pairs = (CsrPair * self.P)()
        for i, (rp, c, a, b) in enumerate(problems):
            m = (_dev(torch.as_tensor(rp), torch.int64), _dev(torch.as_tensor(c), torch.int32),
                 _dev(torch.as_tensor(a), torch.float64), _dev(torch.as_tensor(b), torch.float64))
            self.mats.append(m)
            pairs[i] = CsrPair(int(m[0].numel() - 1), int(m[1].numel()), _ptr(m[0]), _ptr(m[1]), _ptr(m[2]),
                               _ptr(m[3]))
        self.n = [int(m[0].numel() - 1) for m in self.mats]
        self.blocks = np.ascontiguousarray(blocks, dtype=np.int32)
        g = np.ascontiguousarray(gammas, dtype=np.float64)
        h = ct.c_void_p()
        _check(lib().slrf_setup_batched(ct.byref(h), self.P, pairs, _ptr(g), _ptr(self.blocks), ct.byref(self.opts),
                                        ct.c_void_p(self.stream.cuda_stream)), "slrf_setup_batched")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().slrf_destroy_batched(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, V0=None, caps=None, check=True):
        caps = np.ascontiguousarray(self.blocks if caps is None else caps, dtype=np.int32)
        v0 = None
        keep = []
        if V0 is not None:
            v0 = (ct.c_void_p * self.P)()
            for i, v in enumerate(V0):
                t = _dev(torch.as_tensor(v), torch.float64)
                keep.append(t)
                v0[i] = t.data_ptr()
        ev = [torch.zeros(max(int(c), 1), dtype=torch.float64, device="cuda") for c in caps]
        X = [torch.zeros((n, max(int(c), 1)), dtype=torch.float64, device="cuda") for n, c in zip(self.n, caps)]
        rs = [torch.zeros(max(int(c), 1), dtype=torch.float64, device="cuda") for c in caps]
        pe = (ct.c_void_p * self.P)(*[t.data_ptr() for t in ev])
        px = (ct.c_void_p * self.P)(*[t.data_ptr() for t in X])
        pr = (ct.c_void_p * self.P)(*[t.data_ptr() for t in rs])
        nf = np.zeros(self.P, dtype=np.int32)
        stt = np.zeros(self.P, dtype=np.int32)
        st = Stats()
        rc = lib().slrf_solve_batched(self.h, v0, _ptr(caps), _ptr(nf), pe, px, pr, _ptr(stt), ct.byref(st))
        if check:
            _check(rc, "slrf_solve_batched")
        out = []
        for i in range(self.P):
            c = min(int(nf[i]), int(caps[i]))
            out.append((int(stt[i]), int(nf[i]), ev[i][:c], X[i][:, :c], rs[i][:c]))
        return rc, out, st.as_dict()


def tsgram(X: torch.Tensor, Y: torch.Tensor, mode: int = 1) -> torch.Tensor:
    """slrf_tsgram: C = X^T Y for device FP64 row-major blocks X (n x k1), Y (n x k2);
    mode 1 = split-bf16 tensor-core products, 0 = FP64 FMA."""
    assert X.is_cuda and Y.is_cuda and X.dtype == torch.float64 and Y.dtype == torch.float64
    assert X.shape[0] == Y.shape[0] and X.stride(1) == 1 and Y.stride(1) == 1
    k1, k2 = X.shape[1], Y.shape[1]
    C = torch.empty(k1, k2, dtype=torch.float64, device=X.device)
    st = torch.cuda.current_stream(X.device)
    _check(lib().slrf_tsgram(X.shape[0], _ptr(X), X.stride(0), k1, _ptr(Y), Y.stride(0), k2, _ptr(C), k2, int(mode),
                             ct.c_void_p(st.cuda_stream)), "slrf_tsgram")
    return C


def tsgemm(X: torch.Tensor, S: torch.Tensor, Z: torch.Tensor | None = None, alpha: float = 1.0, beta: float = 0.0,
           mode: int = 1) -> torch.Tensor:
    """slrf_tsgemm: Z = alpha X S + beta Z for device FP64 row-major X (n x k1), S (k1 x k2)."""
    assert X.is_cuda and S.is_cuda and X.dtype == torch.float64 and S.dtype == torch.float64
    assert X.shape[1] == S.shape[0] and X.stride(1) == 1 and S.stride(1) == 1
    n, k2 = X.shape[0], S.shape[1]
    if Z is None:
        Z = torch.zeros(n, k2, dtype=torch.float64, device=X.device)
    assert Z.shape == (n, k2) and Z.stride(1) == 1
    st = torch.cuda.current_stream(X.device)
    _check(lib().slrf_tsgemm(n, _ptr(X), X.stride(0), X.shape[1], _ptr(S), S.stride(0), k2, _ptr(Z), Z.stride(0),
                             float(alpha), float(beta), int(mode), ct.c_void_p(st.cuda_stream)), "slrf_tsgemm")
    return Z


def filter_apply_static(rowptr, col, valA, valB, gamma, opts, X, theta=None, U=None, stream=None):
    """slrf_filter_apply_static: the FP64 filter apply without a context or any device
    allocation inside the library (device tensors in, U out; the stream of X's device
    unless one is given).  The layouts the C side assumes are checked here: rowptr int64
    (n + 1), col int32 (nnz), valA / valB float64 (nnz), X and U float64 n x k contiguous,
    theta float64 (k), all on one CUDA device.  Pass a preallocated U to avoid the one
    allocation this wrapper would otherwise make."""
    dev = X.device
    n = int(rowptr.numel() - 1)
    nnz = int(col.numel())

    def need(t, dtype, shape, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device == dev and t.dtype == dtype
                and t.is_contiguous() and tuple(t.shape) == shape):
            raise ValueError(f"{name}: expected a contiguous {dtype} tensor of shape {shape} on {dev}")

    if not X.is_cuda or X.dim() != 2:
        raise ValueError("X: expected a 2-D CUDA tensor")
    k = int(X.shape[1])
    need(rowptr, torch.int64, (n + 1,), "rowptr")
    need(col, torch.int32, (nnz,), "col")
    need(valA, torch.float64, (nnz,), "valA")
    need(valB, torch.float64, (nnz,), "valB")
    need(X, torch.float64, (n, k), "X")
    if theta is not None:
        need(theta, torch.float64, (k,), "theta")
    if U is None:
        U = torch.empty_like(X)
    need(U, torch.float64, (n, k), "U")
    pair = CsrPair(n, nnz, _ptr(rowptr), _ptr(col), _ptr(valA), _ptr(valB))
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    _check(lib().slrf_filter_apply_static(ct.byref(pair), float(gamma), ct.byref(opts), _ptr(X), k, _ptr(theta),
                                          _ptr(U), ct.c_void_p(st.cuda_stream)), "slrf_filter_apply_static")
    return U


def slrf_solve_host(rowptr, col, valA, valB, gamma, block_L, opts=None, V0=None, cap=None):
    """Whole solve from host numpy arrays through ``slrf_solve_host``."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    valA = np.ascontiguousarray(valA, dtype=np.float64)
    valB = np.ascontiguousarray(valB, dtype=np.float64)
    n = rowptr.size - 1
    cap = block_L if cap is None else cap
    opts = opts if opts is not None else slrf_opts_default()
    pair = CsrPair(n, col.size, _ptr(rowptr), _ptr(col), _ptr(valA), _ptr(valB))
    V0 = None if V0 is None else np.ascontiguousarray(V0, dtype=np.float64)
    ev = np.zeros(cap)
    X = np.zeros((n, cap))
    rs = np.zeros(cap)
    nf = ct.c_int()
    st = Stats()
    rc = lib().slrf_solve_host(ct.byref(pair), float(gamma), int(block_L), ct.byref(opts), _ptr(V0), cap,
                               ct.byref(nf), _ptr(ev), _ptr(X), _ptr(rs), ct.byref(st))
    _check(rc, "slrf_solve_host")
    c = min(nf.value, cap)
    return ev[:c], X[:, :c], rs[:c], st.as_dict()


def quadrature_table(rule: str, m: int, gamma: float):
    """Pole table (upper-half poles sigma_j, weights w_j) of a classical contour-integral
    filter, for slrf_opts_default(poles=..., weights=...): a quadrature rule for the Cauchy
    integral of the interval's indicator over the circle through 0 and gamma (centre and
    radius gamma/2), on the upper half circle theta in [0, pi]; the lower half is the
    conjugate.  Rules (the comparison filters of the paper's Table 1):
      "midpoint"        theta_j = pi (j - 1/2) / m, equal weights;
      "gauss_legendre"  theta_j = pi (1 + x_j) / 2 at the Gauss-Legendre points x_j;
      "gauss_chebyshev" x_j = cos((2j - 1) pi / (2m)), weights pi/m sqrt(1 - x_j^2).
    The weight of node z_j = c + r e^{i theta_j} is -r e^{i theta_j} times its quadrature
    weight on theta / (2 pi) (dz = i r e^{i theta} dtheta, and the factor -1/(2 pi i))."""
    c = r = 0.5 * float(gamma)
    j = np.arange(1, m + 1)
    if rule == "midpoint":
        theta = np.pi * (j - 0.5) / m
        wq = np.full(m, np.pi / m)
    elif rule == "gauss_legendre":
        x, wx = np.polynomial.legendre.leggauss(m)
        theta = np.pi * (1.0 + x) / 2.0
        wq = wx * np.pi / 2.0
    elif rule == "gauss_chebyshev":
        x = np.cos((2 * j - 1) * np.pi / (2 * m))
        theta = np.pi * (1.0 + x) / 2.0
        wq = (np.pi / m) * np.sqrt(1.0 - x * x) * np.pi / 2.0
    else:
        raise ValueError(f"unknown rule {rule}")
    z = np.exp(1j * theta)
    return c + r * z, -r * z * wq / (2.0 * np.pi)


def pole_shard(m: int, world: int, rank: int) -> list:
    """Poles of rank `rank` when the m upper-half poles of a filter are split over `world`
    ranks (round robin: j = rank, rank + world, ...).  Every pole belongs to exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    return list(range(rank, m, world))


class ShardedFilter:
    """Pole-sharded filter apply (the paper's first parallel level, Sec. 2.3): each rank
    solves the shifted systems of its own poles and one sum all-reduce of the partial
    blocks gives U = sum_j 2 Re(w_j Y_j) on every rank.  The warm start splits by pole as
    well (Y_j = x/(theta - sigma_j) + correction), so a context built on a subset of the
    pole table returns exactly that subset's share, including its part of Phi(theta) x.
    The all-reduce is torch.distributed's (NCCL between GPUs); no kernel of the library
    touches a peer's memory.  Ranks with no pole contribute zeros."""

    def __init__(self, rowptr, col, valA, valB, gamma, block_L, opts, sigma, w, group=None, stream=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        world = dist.get_world_size(group)
        rank = dist.get_rank(group)
        mine = pole_shard(len(sigma), world, rank)
        self.ctx = None
        if mine:
            sig = np.asarray(sigma)[mine]
            ww = np.asarray(w)[mine]
            o = Opts()
            ct.memmove(ct.byref(o), ct.byref(opts), ct.sizeof(Opts))
            arr_s = np.ascontiguousarray(np.stack([sig.real, sig.imag], axis=1).ravel())
            arr_w = np.ascontiguousarray(np.stack([ww.real, ww.imag], axis=1).ravel())
            o.m = len(mine)
            o.poles = arr_s.ctypes.data
            o.weights = arr_w.ctypes.data
            o._keep = [arr_s, arr_w]
            self.ctx = Context(rowptr, col, valA, valB, gamma, block_L, o, stream=stream)

    def filter_apply(self, X: torch.Tensor, theta: torch.Tensor | None = None) -> torch.Tensor:
        if self.ctx is not None:
            U = self.ctx.filter_apply(X, theta)
        else:
            U = torch.zeros_like(_dev(X, torch.float64))
        self.dist.all_reduce(U, op=self.dist.ReduceOp.SUM, group=self.group)
        return U

    def close(self):
        if self.ctx is not None:
            self.ctx.close()
            self.ctx = None


class SlrfEigsh(torch.autograd.Function):
    """Eigenpairs in (0, gamma] of (A, B) given by CSR values on a fixed pattern; backward
    is the adjoint slrf_eig_grad (eigenvalue terms, plus the eigenvector terms when the
    loss depends on X), returning gradients on the values of A and B."""

    @staticmethod
    def forward(fctx, valA, valB, rowptr, col, gamma, block_L, opts, V0):
        ctx = Context(rowptr, col, valA.detach(), valB.detach(), gamma, block_L, opts)
        _, nf, ev, X, rs, _ = ctx.solve(V0)
        fctx.slrf = ctx
        fctx.devices = (valA.device, valB.device)
        fctx.save_for_backward(ev, X)
        return ev.clone(), X.clone()

    @staticmethod
    def backward(fctx, g_ev, g_X):
        ev, X = fctx.saved_tensors
        if g_ev is None:
            g_ev = torch.zeros_like(ev)
        gx = None if (g_X is None or not bool(torch.any(g_X != 0))) else g_X.contiguous()
        gA, gB = fctx.slrf.eig_grad(ev, X, g_ev.contiguous(), gx)
        return gA.to(fctx.devices[0]), gB.to(fctx.devices[1]), None, None, None, None, None, None
