"""GB300 accelerated cyclic reduction (ACR) -- thin Python binding of the C ABI.

Every function here only marshals arguments to ``_lib/libacr.so`` (built by
``build.py`` from ``csrc/``); all arithmetic runs in the library's CUDA
kernels.  There is no CPU fallback: if the library is missing or a call fails
the functions raise.

Arrays: right-hand sides / solutions are FP64 CUDA tensors holding an
``N x nrhs`` column-major block (``N = n^3``, lexicographic ``i + n j + n^2 k``):
either a 1-D tensor of length ``N`` (one column) or a 2-D tensor of shape
``(N, nrhs)`` with ``stride(0) == 1`` (e.g. ``t.T`` of a contiguous
``(nrhs, N)`` tensor); the leading dimension is ``stride(1)``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libacr.so")

ACR_OK = 0
ACR_ERR_ARG = 1
ACR_ERR_OOM = 2
ACR_ERR_BREAKDOWN = 3
ACR_ERR_RANK_CAP = 4
ACR_ERR_CUDA = 5
ACR_ERR_NOT_CONVERGED = 6
ACR_FP64 = 0
ACR_FP32 = 1
KERNEL_CLASSES = ("gemm", "splitk_reduce", "householder_qr", "pivoted_cholesky", "core_truncation", "rebuild_coef",
                  "gauss_jordan", "copy", "assemble", "permute", "stencil_fp64", "gemm_tcgen05", "hodlr_expand",
                  "tf32_split")


class AcrOpts(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("shift", C.c_double),
        ("max_rank", C.c_int),
        ("mem_budget", C.c_size_t),
        ("autotune", C.c_int),
        ("nrhs_max", C.c_int),
        ("cuda_stream", C.c_void_p),
        ("profile", C.c_int),
        ("inverse_fp64", C.c_int),
        ("tensor_cores", C.c_int),
        ("core_svd", C.c_int),
        ("coarse_dense_max", C.c_int),
        ("graphs", C.c_int),
        ("velocity", C.c_void_p),
        ("chol_passes", C.c_int),
    ]


class AcrStats(C.Structure):
    _fields_ = [
        ("n", C.c_int),
        ("leaf", C.c_int),
        ("levels_cr", C.c_int),
        ("levels_h", C.c_int),
        ("precision", C.c_int),
        ("tol", C.c_double),
        ("max_rank", (C.c_int * 16) * 16),
        ("max_rank_d", (C.c_int * 16) * 16),
        ("factor_bytes", C.c_size_t),
        ("peak_bytes", C.c_size_t),
        ("t_factor_ms", C.c_double),
        ("t_level_ms", C.c_double * 16),
        ("gemm_flops", C.c_longlong),
        ("kernel_launches", C.c_longlong),
        ("kc_ms", C.c_double * 16),
        ("kc_flops", C.c_double * 16),
        ("kc_bytes", C.c_double * 16),
        ("kc_launches", C.c_longlong * 16),
        ("jacobi_sweeps_max", C.c_int),
        ("graphs_captured", C.c_int),
        ("coarse_dense", C.c_int),
        ("levels_stored", C.c_int),
        ("tail_recomputes", C.c_longlong),
    ]


class AcrError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s: %s (status %d)" % (what, error_string(status), status))
        self.status = status


_lib = None


def load_library():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("ACR CUDA library not built (%s); run paper_1701_00182_gb300/build.py" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    H = C.c_void_p
    P = C.c_void_p
    sig = {
        "acr_default_opts": (None, [C.POINTER(AcrOpts)]),
        "acr_factor": (C.c_int, [C.c_int, P, C.c_double, C.c_int, C.POINTER(AcrOpts), C.POINTER(H)]),
        "acr_solve": (C.c_int, [H, P, P, C.c_int, C.c_long]),
        "acr_solve_transpose": (C.c_int, [H, P, P, C.c_int, C.c_long]),
        "acr_residual": (C.c_int, [H, P, P, P, C.c_int, C.c_long, C.POINTER(C.c_double)]),
        "acr_residual_noalloc": (C.c_int, [H, P, P, P, C.c_int, C.c_long, C.POINTER(C.c_double)]),
        "acr_solve_ir": (C.c_int, [H, P, P, C.c_int, C.c_long, C.c_double, C.c_int, C.POINTER(C.c_int),
                                   C.POINTER(C.c_double)]),
        "acr_solve_ir_transpose": (C.c_int, [H, P, P, C.c_int, C.c_long, C.c_double, C.c_int, C.POINTER(C.c_int),
                                             C.POINTER(C.c_double)]),
        "acr_grad_logkappa": (C.c_int, [H, P, P, P, C.c_int, C.c_long]),
        "acr_solve_fgmres": (C.c_int, [H, P, P, C.c_int, C.c_long, C.c_double, C.c_int, C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "acr_get_factor_block": (C.c_int, [H, C.c_int, C.c_int, C.c_int, P]),
        "acr_get_stats": (C.c_int, [H, C.POINTER(AcrStats)]),
        "acr_destroy": (None, [H]),
        "acr_error_string": (C.c_char_p, [C.c_int]),
        "acr_plane_ordering": (C.c_int, [C.c_int, C.c_int, P, P]),
        "acr_plan_blocks": (C.c_int, [C.c_int, C.c_int, C.c_double, P, C.c_long, C.POINTER(C.c_long)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def error_string(status: int) -> str:
    return load_library().acr_error_string(int(status)).decode()


def _check(status: int, what: str, allow=(ACR_OK,)):
    if status not in allow:
        raise AcrError(status, what)
    return status


def _cols(t, n: int):
    """(ptr, nrhs, ld) of an FP64 CUDA tensor holding an N x nrhs column-major block."""
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError("expected a float64 CUDA tensor")
    N = n ** 3
    if t.dim() == 1:
        if t.numel() != N or t.stride(0) != 1:
            raise ValueError("1-D tensor must be contiguous with n^3 entries")
        return t.data_ptr(), 1, N
    if t.dim() != 2 or t.shape[0] != N or t.stride(0) != 1:
        raise ValueError("2-D tensor must be (N, nrhs) column major (stride(0) == 1)")
    return t.data_ptr(), t.shape[1], max(t.stride(1), N)


def acr_default_opts() -> AcrOpts:
    o = AcrOpts()
    load_library().acr_default_opts(C.byref(o))
    return o


class Handle:
    """Owns an ``acr_handle``; ``close()`` (or garbage collection) calls ``acr_destroy``."""

    def __init__(self, ptr, n: int, opts: AcrOpts):
        self._p = C.c_void_p(ptr)
        self.n = n
        self.opts = opts

    @property
    def ptr(self):
        if not self._p:
            raise ValueError("handle already destroyed")
        return self._p

    def close(self):
        if self._p:
            load_library().acr_destroy(self._p)
            self._p = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f64_buffer(a, count: int, what: str):
    """(owner, pointer) of a contiguous float64 numpy array / tensor (host or CUDA) of `count` values."""
    try:
        import torch

        is_t = isinstance(a, torch.Tensor)
    except ImportError:
        is_t = False
    if is_t:
        if a.dtype != torch.float64 or a.numel() != count or not a.is_contiguous():
            raise ValueError("%s tensor must be contiguous float64 with %d entries" % (what, count))
        return a, a.data_ptr()
    keep = np.ascontiguousarray(a, dtype=np.float64)
    if keep.size != count:
        raise ValueError("%s must have %d entries" % (what, count))
    return keep, keep.ctypes.data


def acr_factor(n: int, log_kappa, tol: float, leaf: int, opts: AcrOpts | None = None, **kw) -> Handle:
    """ACR elimination; ``log_kappa`` is a float64 numpy array / tensor (host or CUDA) of n^3 values or None.

    Keyword overrides of the options: precision, shift, max_rank, mem_budget, autotune, nrhs_max, stream,
    velocity (3 x n^3 float64, planar beta_x, beta_y, beta_z: the convection velocity), and the other
    acr_opts fields by name.
    """
    lib = load_library()
    o = opts if opts is not None else acr_default_opts()
    keep_v = None
    for k, v in kw.items():
        if k == "stream":
            o.cuda_stream = C.c_void_p(v)
        elif k == "velocity":
            if v is None:
                o.velocity = None
            else:
                keep_v, pv = _f64_buffer(v, 3 * n ** 3, "velocity")
                o.velocity = C.c_void_p(pv)
        else:
            setattr(o, k, v)
    keep = None
    ptr = None
    if log_kappa is not None:
        keep, ptr = _f64_buffer(log_kappa, n ** 3, "log_kappa")
    h = C.c_void_p()
    st = lib.acr_factor(int(n), ptr, float(tol), int(leaf), C.byref(o), C.byref(h))
    del keep, keep_v
    o.velocity = None  # the library copied it; do not keep a pointer to a released buffer
    _check(st, "acr_factor")
    return Handle(h.value, n, o)


def acr_solve(h: Handle, rhs, x) -> None:
    p_b, nrhs, ld = _cols(rhs, h.n)
    p_x, nrhs2, ld2 = _cols(x, h.n)
    if nrhs != nrhs2 or ld != ld2:
        raise ValueError("rhs and x must have the same shape and leading dimension")
    _check(load_library().acr_solve(h.ptr, p_b, p_x, nrhs, ld), "acr_solve")


def acr_solve_transpose(h: Handle, rhs, x) -> None:
    p_b, nrhs, ld = _cols(rhs, h.n)
    p_x, nrhs2, ld2 = _cols(x, h.n)
    if nrhs != nrhs2 or ld != ld2:
        raise ValueError("rhs and x must have the same shape and leading dimension")
    _check(load_library().acr_solve_transpose(h.ptr, p_b, p_x, nrhs, ld), "acr_solve_transpose")


def acr_residual(h: Handle, b, x, r) -> np.ndarray:
    p_b, nrhs, ld = _cols(b, h.n)
    p_x, _, _ = _cols(x, h.n)
    p_r, _, _ = _cols(r, h.n)
    rel = (C.c_double * nrhs)()
    _check(load_library().acr_residual(h.ptr, p_b, p_x, p_r, nrhs, ld, rel), "acr_residual")
    return np.array(rel[:])


def acr_residual_noalloc(h: Handle, b, x, r) -> np.ndarray:
    """acr_residual without any device allocation in the call (fixed scratch; nrhs <= 64)."""
    p_b, nrhs, ld = _cols(b, h.n)
    p_x, _, _ = _cols(x, h.n)
    p_r, _, _ = _cols(r, h.n)
    rel = (C.c_double * nrhs)()
    _check(load_library().acr_residual_noalloc(h.ptr, p_b, p_x, p_r, nrhs, ld, rel), "acr_residual_noalloc")
    return np.array(rel[:])


def acr_solve_ir(h: Handle, b, x, rtol: float = 1e-10, maxit: int = 50, check: bool = True):
    """FP64 iterative refinement with ACR; returns (iterations, relative residuals, status)."""
    p_b, nrhs, ld = _cols(b, h.n)
    p_x, _, _ = _cols(x, h.n)
    it = C.c_int(0)
    rel = (C.c_double * nrhs)()
    st = load_library().acr_solve_ir(h.ptr, p_b, p_x, nrhs, ld, float(rtol), int(maxit), C.byref(it), rel)
    if check:
        _check(st, "acr_solve_ir")
    return it.value, np.array(rel[:]), st


def acr_solve_ir_transpose(h: Handle, b, x, rtol: float = 1e-10, maxit: int = 50, check: bool = True):
    """Refinement with the transpose solve; returns (iterations, relative residuals, status)."""
    p_b, nrhs, ld = _cols(b, h.n)
    p_x, _, _ = _cols(x, h.n)
    it = C.c_int(0)
    rel = (C.c_double * nrhs)()
    st = load_library().acr_solve_ir_transpose(h.ptr, p_b, p_x, nrhs, ld, float(rtol), int(maxit), C.byref(it), rel)
    if check:
        _check(st, "acr_solve_ir_transpose")
    return it.value, np.array(rel[:]), st


def acr_grad_logkappa(h: Handle, u, lam, grad) -> None:
    """grad (float64 CUDA, N) = -kappa * sum_columns lam^T (dA/dkappa) u."""
    p_u, nrhs, ld = _cols(u, h.n)
    p_l, nrhs2, ld2 = _cols(lam, h.n)
    if nrhs != nrhs2 or ld != ld2:
        raise ValueError("u and lam must have the same shape and leading dimension")
    p_g, _, _ = _cols(grad, h.n)
    _check(load_library().acr_grad_logkappa(h.ptr, p_u, p_l, p_g, nrhs, ld), "acr_grad_logkappa")


def acr_solve_fgmres(h: Handle, b, x, rtol: float = 1e-10, restart: int = 50, maxit: int = 500, check: bool = True):
    """FP64 right-preconditioned FGMRES with ACR; returns (preconditioner applications, rel. residuals, status)."""
    p_b, nrhs, ld = _cols(b, h.n)
    p_x, _, _ = _cols(x, h.n)
    it = C.c_int(0)
    rel = (C.c_double * nrhs)()
    st = load_library().acr_solve_fgmres(h.ptr, p_b, p_x, nrhs, ld, float(rtol), int(restart), int(maxit),
                                         C.byref(it), rel)
    if check:
        _check(st, "acr_solve_fgmres")
    return it.value, np.array(rel[:]), st


def acr_get_factor_block(h: Handle, which: int, level: int, index: int) -> np.ndarray:
    m = h.n * h.n
    out = np.empty((m, m), dtype=np.float64)
    _check(load_library().acr_get_factor_block(h.ptr, int(which), int(level), int(index), out.ctypes.data),
           "acr_get_factor_block")
    return out


def acr_get_stats(h: Handle) -> dict:
    s = AcrStats()
    _check(load_library().acr_get_stats(h.ptr, C.byref(s)), "acr_get_stats")
    q, L = s.levels_cr, s.levels_h
    return {
        "n": s.n, "leaf": s.leaf, "levels_cr": q, "levels_h": L, "precision": s.precision, "tol": s.tol,
        "max_rank": [[s.max_rank[r][l] for l in range(L)] for r in range(q + 1)],
        "max_rank_d": [[s.max_rank_d[r][l] for l in range(L)] for r in range(q + 1)],
        "factor_bytes": s.factor_bytes, "peak_bytes": s.peak_bytes, "t_factor_ms": s.t_factor_ms,
        "t_level_ms": [s.t_level_ms[r] for r in range(min(q, 16))], "gemm_flops": s.gemm_flops,
        "kernel_launches": s.kernel_launches,
        "jacobi_sweeps_max": s.jacobi_sweeps_max,
        "graphs_captured": s.graphs_captured,
        "coarse_dense": s.coarse_dense,
        "levels_stored": s.levels_stored,
        "tail_recomputes": s.tail_recomputes,
        "kernels": {nm: {"ms": s.kc_ms[i], "flops": s.kc_flops[i], "bytes": s.kc_bytes[i],
                         "launches": s.kc_launches[i]} for i, nm in enumerate(KERNEL_CLASSES)},
    }


def acr_destroy(h: Handle) -> None:
    h.close()


def acr_error_string(status: int) -> str:
    return error_string(status)


def acr_plane_ordering(n: int, leaf: int):
    """Host-only planner query: (perm, ncut) of the plane cluster tree."""
    perm = np.empty(n * n, dtype=np.int32)
    ncut = np.zeros(32, dtype=np.int32)
    L = load_library().acr_plane_ordering(int(n), int(leaf), perm.ctypes.data, ncut.ctypes.data)
    if L < 0:
        raise AcrError(-L, "acr_plane_ordering")
    return perm, ncut[:L].copy()


def acr_plan_blocks(n: int, leaf: int, eta=None):
    """Host-only planner query: the block cluster tree of one plane as an
    (nblocks, 4) int array of (level, t, s, low rank); eta None = weak."""
    lib = load_library()
    e = -1.0 if eta is None else float(eta)
    cnt = C.c_long(0)
    st = lib.acr_plan_blocks(int(n), int(leaf), e, None, 0, C.byref(cnt))
    if st != ACR_OK:
        raise AcrError(st, "acr_plan_blocks")
    out = np.empty((cnt.value, 4), dtype=np.int32)
    st = lib.acr_plan_blocks(int(n), int(leaf), e, out.ctypes.data, cnt.value, C.byref(cnt))
    if st != ACR_OK:
        raise AcrError(st, "acr_plan_blocks")
    return out


def _colmajor(t):
    """Same values as an (N,) / (N, r) column-major CUDA tensor."""
    if t.dim() == 1:
        return t.contiguous()
    return t.t().contiguous().t()


def _autograd_function():
    import torch

    class ACRSolve(torch.autograd.Function):
        """u = A(exp(log_kappa))^{-1} f through ACR; backward by the transpose solve.

        forward: acr_factor + acr_solve (or refinement to rtol); backward:
        lambda = A^{-T} grad_u (acr_solve_transpose, or transpose refinement),
        grad_f = lambda, grad_log_kappa = acr_grad_logkappa(u, lambda).  The
        factorisation of the forward pass is kept for the backward pass; with
        mem_budget > 0 it keeps only the CR levels that fit in that many bytes,
        and the forward and backward solves recompute the others.
        """

        @staticmethod
        def forward(ctx, log_kappa, f, n, tol, leaf, precision, rtol, mem_budget):
            h = acr_factor(n, log_kappa.detach().contiguous(), tol, leaf, precision=precision,
                           nrhs_max=1 if f.dim() == 1 else f.shape[1], mem_budget=int(mem_budget or 0))
            fb = _colmajor(f.detach())
            x = _colmajor(torch.zeros_like(fb))
            if rtol:
                acr_solve_ir(h, fb, x, rtol=rtol, maxit=80)
            else:
                acr_solve(h, fb, x)
            ctx.h, ctx.rtol, ctx.n = h, rtol, n
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, gu):
            (u,) = ctx.saved_tensors
            h = ctx.h
            g = _colmajor(gu.detach())
            lam = _colmajor(torch.zeros_like(g))
            if ctx.rtol:
                acr_solve_ir_transpose(h, g, lam, rtol=ctx.rtol, maxit=80)
            else:
                acr_solve_transpose(h, g, lam)
            grad = torch.zeros(ctx.n ** 3, dtype=torch.float64, device=u.device)
            acr_grad_logkappa(h, u, lam, grad)
            return grad, lam, None, None, None, None, None, None

    return ACRSolve


_ACRSolve = None


def acr_solve_autograd(log_kappa, f, n: int, tol: float, leaf: int, precision: int = ACR_FP64, rtol=None,
                       mem_budget: int = 0):
    """Differentiable solve u(log_kappa, f) on CUDA float64 tensors (see ACRSolve)."""
    global _ACRSolve
    if _ACRSolve is None:
        _ACRSolve = _autograd_function()
    return _ACRSolve.apply(log_kappa, f, n, tol, leaf, precision, rtol, mem_budget)
