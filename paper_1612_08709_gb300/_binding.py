"""ctypes marshalling of torch tensors into the C ABI of libtssvd.so.

Argument marshalling only: every computation happens in the library's CUDA
kernels.  Functions keep the C names (ts_svd, lowrank_svd, ts_svd_backward)
and raise TsSvdError on a negative (invalid argument) or hard-failure
status; soft statuses (non-convergence, rank deficiency) are returned in the
info dictionary.
"""
import ctypes
import math
import os

import torch

from . import build as _build

TSSVD_OK = 0
TSSVD_ENOCONV = 1
TSSVD_RANKDEF = 2
TSSVD_ETIMEOUT = 3
TSSVD_ECUDA = 4
TSSVD_ENOMEM = 5
TSSVD_ECOMM = 6

_MODES = {"fp64": 0, "bf16x3": 1, "bf16x6": 2, "fp64_tc": 3, "auto": 4}
_MODE_NAMES = {v: k for k, v in _MODES.items()}

# Square root of the paper's example working precision 1e-11 (Remark "working").
PAPER_DROP_TOL = math.sqrt(1e-11)


class TsSvdError(RuntimeError):
    pass


class _Opts(ctypes.Structure):
    _fields_ = [
        ("passes", ctypes.c_int),
        ("scale", ctypes.c_int),
        ("drop_tol", ctypes.c_double),
        ("mode", ctypes.c_int),
        ("max_sweeps", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("out_rank", ctypes.c_int64),
        ("sweeps", ctypes.c_int * 4),
        ("ranks", ctypes.c_int * 2),
    ]


class _Desc(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
        ("lda", ctypes.c_int64), ("U", ctypes.c_void_p), ("S", ctypes.c_void_p),
        ("V", ctypes.c_void_p), ("out_rank", ctypes.c_int64), ("status", ctypes.c_int),
        ("mode", ctypes.c_int), ("sweeps", ctypes.c_int * 3),
    ]


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Loads libtssvd.so (building it first if its sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if _build._stale():
        _build.build()
    if not os.path.exists(path):
        raise ImportError("libtssvd.so is missing (%s); run build()" % path)
    L = ctypes.CDLL(path)
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    op = ctypes.POINTER(_Opts)
    L.tssvd_default_opts.argtypes = [op]
    L.tssvd_default_opts.restype = None
    L.tssvd_status_string.argtypes = [ctypes.c_int]
    L.tssvd_status_string.restype = ctypes.c_char_p
    L.ts_svd_workspace_size.argtypes = [i64, i64, ctypes.c_int, op]
    L.ts_svd_workspace_size.restype = ctypes.c_size_t
    L.lowrank_svd_workspace_size.argtypes = [i64, i64, i64, op]
    L.lowrank_svd_workspace_size.restype = ctypes.c_size_t
    for name in ("ts_svd", "ts_svd_f32"):
        f = getattr(L, name)
        f.argtypes = [vp, i64, i64, i64, vp, vp, vp, op]
        f.restype = ctypes.c_int
    L.ts_pca_workspace_size.argtypes = [i64, i64, ctypes.c_int, op]
    L.ts_pca_workspace_size.restype = ctypes.c_size_t
    for name in ("ts_pca", "ts_pca_f32"):
        f = getattr(L, name)
        f.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, op]
        f.restype = ctypes.c_int
    L.lowrank_svd.argtypes = [vp, i64, i64, i64, i64, i64, ctypes.c_int, vp, vp, vp, vp, op]
    L.lowrank_svd.restype = ctypes.c_int
    for name in ("ts_svd_backward", "ts_svd_backward_f32"):
        f = getattr(L, name)
        f.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, vp, vp, op]
        f.restype = ctypes.c_int
    L.ts_svd_tsqr_workspace_size.argtypes = [i64, i64, op]
    L.ts_svd_tsqr_workspace_size.restype = ctypes.c_size_t
    L.lowrank_svd_tsqr.argtypes = [vp, i64, i64, i64, i64, i64, ctypes.c_int, vp, vp, vp, vp, vp,
                                   vp, op]
    L.lowrank_svd_tsqr.restype = ctypes.c_int
    L.ts_svd_tsqr.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, vp, op]
    L.ts_svd_tsqr.restype = ctypes.c_int
    L.lowrank_svd_backward.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, op]
    L.lowrank_svd_backward.restype = ctypes.c_int
    L.ts_gram_workspace_size.argtypes = [i64, i64]
    L.ts_gram_workspace_size.restype = ctypes.c_size_t
    L.ts_gram.argtypes = [vp, i64, i64, i64, vp, op]
    L.ts_gram.restype = ctypes.c_int
    L.ts_matmul_workspace_size.argtypes = [i64, i64, i64]
    L.ts_matmul_workspace_size.restype = ctypes.c_size_t
    L.ts_matmul.argtypes = [vp, i64, i64, i64, vp, i64, i64, vp, i64, op]
    L.ts_matmul.restype = ctypes.c_int
    L.ts_svd_batched.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int, ctypes.c_int, op]
    L.ts_svd_batched.restype = ctypes.c_int
    L.ts_svd_batched_workspace_size.argtypes = [ctypes.POINTER(_Desc), ctypes.c_int,
                                                ctypes.c_int, op]
    L.ts_svd_batched_workspace_size.restype = ctypes.c_size_t
    L.tssvd_launch_count.argtypes = []
    L.tssvd_launch_count.restype = ctypes.c_longlong
    L.tssvd_profile_enable.argtypes = [ctypes.c_int]
    L.tssvd_profile_enable.restype = ctypes.c_int
    L.tssvd_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    L.tssvd_profile_report.restype = ctypes.c_size_t
    L.tssvd_fp64_fma_rate.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    L.tssvd_fp64_fma_rate.restype = ctypes.c_int
    L.ts_svd_rowshard.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, op]
    L.ts_svd_rowshard.restype = ctypes.c_int
    L.ts_svd_host.argtypes = [vp, i64, i64, i64, vp, vp, vp, op]
    L.ts_svd_host.restype = ctypes.c_int
    L.ts_svd_host_workspace_size.argtypes = [i64, i64, op]
    L.ts_svd_host_workspace_size.restype = ctypes.c_size_t
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points the binding expects the library to export."""
    return ["tssvd_default_opts", "tssvd_status_string", "ts_svd_workspace_size", "ts_svd",
            "ts_svd_f32", "lowrank_svd_workspace_size", "lowrank_svd", "ts_svd_backward",
            "tssvd_launch_count", "tssvd_profile_enable", "tssvd_profile_report",
            "ts_gram_workspace_size", "ts_gram", "ts_matmul_workspace_size", "ts_matmul",
            "ts_svd_backward_f32", "ts_svd_batched", "ts_svd_batched_workspace_size",
            "ts_pca_workspace_size", "ts_pca", "ts_pca_f32", "lowrank_svd_backward",
            "ts_svd_tsqr_workspace_size", "ts_svd_tsqr", "lowrank_svd_tsqr",
            "tssvd_fp64_fma_rate", "ts_svd_rowshard", "ts_svd_host",
            "ts_svd_host_workspace_size"]


def _opts(passes=2, scale=True, drop_tol=PAPER_DROP_TOL, mode="fp64", max_sweeps=50,
          stream=None, workspace=None):
    o = _Opts()
    lib().tssvd_default_opts(ctypes.byref(o))
    o.passes = int(passes)
    o.scale = int(bool(scale))
    o.drop_tol = float(drop_tol)
    o.mode = _MODES[mode]
    o.max_sweeps = int(max_sweeps)
    if stream is None:
        stream = torch.cuda.current_stream()
    o.stream = ctypes.c_void_p(stream.cuda_stream)
    if workspace is not None:
        assert workspace.is_cuda and workspace.is_contiguous()
        o.workspace = ctypes.c_void_p(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check(rc, name):
    if rc < 0:
        raise TsSvdError("%s: invalid argument %d" % (name, -rc))
    if rc in (TSSVD_ETIMEOUT, TSSVD_ECUDA, TSSVD_ENOMEM, TSSVD_ECOMM):
        raise TsSvdError("%s: %s" % (name, lib().tssvd_status_string(rc).decode()))
    return rc


def _info(o, rc):
    return {"status": rc, "rank": int(o.out_rank), "sweeps": list(o.sweeps)[:3],
            "sweeps_fp32": int(o.sweeps[3]), "ranks": list(o.ranks)}


def _as_matrix(A):
    if not (isinstance(A, torch.Tensor) and A.is_cuda and A.dim() == 2):
        raise TsSvdError("expected a 2-D CUDA tensor")
    if A.stride(1) != 1:
        raise TsSvdError("A must be row-major (unit column stride)")
    return A


def ts_svd_workspace_size(m, n, dtype=torch.float64, **kw):
    o = _opts(**kw) if torch.cuda.is_available() else None
    if o is None:
        o = _Opts()
        lib().tssvd_default_opts(ctypes.byref(o))
    return int(lib().ts_svd_workspace_size(m, n, 4 if dtype == torch.float32 else 8,
                                           ctypes.byref(o)))


def lowrank_svd_workspace_size(m, n, l, mode="fp64"):
    o = _opts(2, False, PAPER_DROP_TOL, mode, 50, None, None)
    return int(lib().lowrank_svd_workspace_size(m, n, l, ctypes.byref(o)))


def ts_svd(A, passes=2, scale=True, drop_tol=PAPER_DROP_TOL, mode="fp64", max_sweeps=50,
           stream=None, workspace=None, out=None):
    """Thin SVD of a tall-skinny CUDA tensor A (m x n, float64 or float32).

    Returns (U m x n, S n, V n x n, info).  See include/tssvd.h (ts_svd).
    """
    A = _as_matrix(A)
    m, n = A.shape
    dt = A.dtype
    if dt not in (torch.float64, torch.float32):
        raise TsSvdError("A must be float64 or float32")
    if out is None:
        U = torch.empty((m, n), dtype=dt, device=A.device)
        S = torch.empty((n,), dtype=dt, device=A.device)
        V = torch.empty((n, n), dtype=dt, device=A.device)
    else:
        U, S, V = out
    o = _opts(passes, scale, drop_tol, mode, max_sweeps, stream, workspace)
    f = lib().ts_svd if dt == torch.float64 else lib().ts_svd_f32
    with torch.cuda.device(A.device):
        rc = f(_ptr(A), m, n, A.stride(0), _ptr(U), _ptr(S), _ptr(V), ctypes.byref(o))
    _check(rc, "ts_svd")
    return U, S, V, _info(o, rc)


def ts_svd_host(A, passes=2, scale=True, drop_tol=PAPER_DROP_TOL, mode="fp64", max_sweeps=50,
                stream=None, workspace=None, out=None, device=None):
    """Thin SVD of a float64 CPU tensor A (m x n, row-major rows; pin it with
    A.pin_memory() for the copies to overlap the compute) computed on the
    current (or given) CUDA device; returns CPU tensors (U, S, V, info).
    See include/tssvd.h (ts_svd_host)."""
    if not (isinstance(A, torch.Tensor) and not A.is_cuda and A.dim() == 2 and
            A.dtype == torch.float64 and A.stride(1) == 1):
        raise TsSvdError("ts_svd_host: A must be a float64 CPU matrix with unit column stride")
    m, n = A.shape
    if out is None:
        pin = A.is_pinned()
        U = torch.empty((m, n), dtype=torch.float64, pin_memory=pin)
        S = torch.empty((n,), dtype=torch.float64, pin_memory=pin)
        V = torch.empty((n, n), dtype=torch.float64, pin_memory=pin)
    else:
        U, S, V = out
    for x in (U, S, V):
        if x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise TsSvdError("ts_svd_host: outputs must be contiguous float64 CPU tensors")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    with torch.cuda.device(dev):
        o = _opts(passes, scale, drop_tol, mode, max_sweeps, stream, workspace)
        rc = lib().ts_svd_host(_ptr(A), m, n, A.stride(0), _ptr(U), _ptr(S), _ptr(V),
                               ctypes.byref(o))
    _check(rc, "ts_svd_host")
    return U, S, V, _info(o, rc)


def ts_svd_host_workspace_size(m, n, **kw):
    o = _opts(**kw) if torch.cuda.is_available() else None
    if o is None:
        o = _Opts()
        lib().tssvd_default_opts(ctypes.byref(o))
    return int(lib().ts_svd_host_workspace_size(m, n, ctypes.byref(o)))


def ts_pca_workspace_size(m, n, dtype=torch.float64, **kw):
    o = _opts(**kw) if torch.cuda.is_available() else None
    if o is None:
        o = _Opts()
        lib().tssvd_default_opts(ctypes.byref(o))
    return int(lib().ts_pca_workspace_size(m, n, 4 if dtype == torch.float32 else 8,
                                           ctypes.byref(o)))


def ts_pca(A, passes=2, scale=True, drop_tol=PAPER_DROP_TOL, mode="fp64", max_sweeps=50,
           stream=None, workspace=None, out=None):
    """PCA of the rows of a CUDA tensor A (m x n, float64 or float32): the thin
    SVD of A - 1 mu^T.  Returns (mu n, U m x n, S n, V n x n, info).  See
    include/tssvd.h (ts_pca)."""
    A = _as_matrix(A)
    m, n = A.shape
    dt = A.dtype
    if dt not in (torch.float64, torch.float32):
        raise TsSvdError("A must be float64 or float32")
    if out is None:
        mu = torch.empty((n,), dtype=dt, device=A.device)
        U = torch.empty((m, n), dtype=dt, device=A.device)
        S = torch.empty((n,), dtype=dt, device=A.device)
        V = torch.empty((n, n), dtype=dt, device=A.device)
    else:
        mu, U, S, V = out
    o = _opts(passes, scale, drop_tol, mode, max_sweeps, stream, workspace)
    f = lib().ts_pca if dt == torch.float64 else lib().ts_pca_f32
    with torch.cuda.device(A.device):
        rc = f(_ptr(A), m, n, A.stride(0), _ptr(mu), _ptr(U), _ptr(S), _ptr(V),
               ctypes.byref(o))
    _check(rc, "ts_pca")
    return mu, U, S, V, _info(o, rc)


def lowrank_svd(A, k, l, iters, Omega, drop_tol=PAPER_DROP_TOL, mode="fp64", max_sweeps=50,
                stream=None, workspace=None):
    """Rank-k SVD by Algorithm 8.  A (m x n) and Omega (n x l) float64 CUDA
    tensors.  Returns (U m x k, S k, V n x k, info)."""
    A = _as_matrix(A)
    m, n = A.shape
    Omega = Omega.contiguous()
    U = torch.empty((m, k), dtype=torch.float64, device=A.device)
    S = torch.empty((k,), dtype=torch.float64, device=A.device)
    V = torch.empty((n, k), dtype=torch.float64, device=A.device)
    o = _opts(2, False, drop_tol, mode, max_sweeps, stream, workspace)
    with torch.cuda.device(A.device):
        rc = lib().lowrank_svd(_ptr(A), m, n, A.stride(0), int(k), int(l), int(iters),
                               _ptr(Omega), _ptr(U), _ptr(S), _ptr(V), ctypes.byref(o))
    _check(rc, "lowrank_svd")
    return U, S, V, _info(o, rc)


def ts_gram(A, mode="fp64", stream=None, workspace=None):
    """B = A^T A (n x n, FP64) of a float64 CUDA tensor A (m x n)."""
    A = _as_matrix(A)
    m, n = A.shape
    B = torch.empty((n, n), dtype=torch.float64, device=A.device)
    o = _opts(mode=mode, stream=stream, workspace=workspace)
    with torch.cuda.device(A.device):
        rc = lib().ts_gram(_ptr(A), m, n, A.stride(0), _ptr(B), ctypes.byref(o))
    _check(rc, "ts_gram")
    return B


def ts_matmul(A, M, mode="fp64", stream=None, workspace=None):
    """C = A M for float64 CUDA tensors A (m x k) and M (k x n)."""
    A = _as_matrix(A)
    M = _as_matrix(M)
    m, k = A.shape
    n = M.shape[1]
    C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    o = _opts(mode=mode, stream=stream, workspace=workspace)
    with torch.cuda.device(A.device):
        rc = lib().ts_matmul(_ptr(A), m, k, A.stride(0), _ptr(M), n, M.stride(0), _ptr(C), n,
                             ctypes.byref(o))
    _check(rc, "ts_matmul")
    return C


def ts_svd_batched(As, passes=2, scale=True, drop_tol=PAPER_DROP_TOL, mode="fp64",
                   max_sweeps=50, stream=None, workspace=None, outs=None):
    """Many TS-SVDs in one graph launch.  As: list of 2-D CUDA tensors of one
    dtype (float64 or float32), row-major.  Returns (list of (U, S, V),
    list of info dicts, call status).  Passing the same tensors (and `outs`)
    again replays the cached graph."""
    if not As:
        raise TsSvdError("empty batch")
    dt = As[0].dtype
    descs = (_Desc * len(As))()
    res = []
    for i, A in enumerate(As):
        A = _as_matrix(A)
        if A.dtype != dt:
            raise TsSvdError("all members must have the same dtype")
        m, n = A.shape
        if outs is None:
            U = torch.empty((m, n), dtype=dt, device=A.device)
            S = torch.empty((n,), dtype=dt, device=A.device)
            V = torch.empty((n, n), dtype=dt, device=A.device)
        else:
            U, S, V = outs[i]
        res.append((U, S, V))
        descs[i].A = A.data_ptr()
        descs[i].m, descs[i].n, descs[i].lda = m, n, A.stride(0)
        descs[i].U, descs[i].S, descs[i].V = U.data_ptr(), S.data_ptr(), V.data_ptr()
    o = _opts(passes, scale, drop_tol, mode, max_sweeps, stream, workspace)
    eb = 8 if dt == torch.float64 else 4
    with torch.cuda.device(As[0].device):
        rc = lib().ts_svd_batched(descs, len(As), eb, ctypes.byref(o))
    if rc < 0:
        raise TsSvdError("ts_svd_batched: invalid argument %d" % (-rc))
    if rc in (TSSVD_ETIMEOUT, TSSVD_ECUDA, TSSVD_ENOMEM, TSSVD_ECOMM):
        raise TsSvdError("ts_svd_batched: %s" % lib().tssvd_status_string(rc).decode())
    infos = [{"status": descs[i].status, "rank": int(descs[i].out_rank),
              "mode": _MODE_NAMES.get(descs[i].mode, descs[i].mode),
              "sweeps": list(descs[i].sweeps)} for i in range(len(As))]
    return res, infos, rc


def ts_svd_batched_workspace_size(shapes, dtype=torch.float64, passes=2, scale=True,
                                  drop_tol=PAPER_DROP_TOL, mode="fp64", max_sweeps=50):
    descs = (_Desc * len(shapes))()
    for i, (m, n) in enumerate(shapes):
        descs[i].m, descs[i].n, descs[i].lda = m, n, n
    o = _Opts()
    lib().tssvd_default_opts(ctypes.byref(o))
    o.passes, o.scale, o.drop_tol = passes, int(bool(scale)), float(drop_tol)
    o.mode, o.max_sweeps = _MODES[mode], max_sweeps
    return int(lib().ts_svd_batched_workspace_size(descs, len(shapes),
                                                   8 if dtype == torch.float64 else 4,
                                                   ctypes.byref(o)))


def ts_svd_backward(A, S, V, dU=None, dS=None, dV=None, mode="fp64", stream=None, workspace=None):
    """dA of the thin SVD (see include/tssvd.h, ts_svd_backward); FP64 or
    FP32 storage (all tensors of A's dtype); mode "fp64" or "fp64_tc" for
    the tall products."""
    A = _as_matrix(A)
    m, n = A.shape
    dt = A.dtype
    dA = torch.empty((m, n), dtype=dt, device=A.device)
    c = [x.contiguous() if x is not None else None for x in (S, V, dU, dS, dV)]
    for x in c:
        if x is not None and x.dtype != dt:
            raise TsSvdError("ts_svd_backward: all tensors must have A's dtype")
    o = _opts(mode=mode, stream=stream, workspace=workspace)
    f = lib().ts_svd_backward if dt == torch.float64 else lib().ts_svd_backward_f32
    with torch.cuda.device(A.device):
        rc = f(_ptr(A), m, n, A.stride(0), *[_ptr(x) for x in c], _ptr(dA), ctypes.byref(o))
    _check(rc, "ts_svd_backward")
    return dA


class TSSVD(torch.autograd.Function):
    """Differentiable thin SVD: forward by ts_svd, backward by ts_svd_backward
    (U is recomputed from A, V and S rather than stored)."""

    @staticmethod
    def forward(ctx, A, passes=2, scale=True, drop_tol=0.0, mode="fp64"):
        U, S, V, info = ts_svd(A, passes=passes, scale=scale, drop_tol=drop_tol, mode=mode)
        ctx.save_for_backward(A, S, V)
        ctx.mode = "fp64_tc" if mode == "fp64_tc" else "fp64"
        return U, S, V

    @staticmethod
    def backward(ctx, gU, gS, gV):
        A, S, V = ctx.saved_tensors
        dA = ts_svd_backward(A, S, V, dU=gU, dS=gS, dV=gV, mode=ctx.mode)
        return dA, None, None, None, None


def lowrank_svd_backward(U, S, V, dU=None, dS=None, dV=None, mode="fp64", stream=None,
                         workspace=None):
    """dA (m x n) of the rank-k SVD (U m x k, S k, V n x k, float64 CUDA
    tensors); see include/tssvd.h (lowrank_svd_backward)."""
    if not (isinstance(U, torch.Tensor) and U.is_cuda and U.dim() == 2):
        raise TsSvdError("expected 2-D CUDA tensors")
    m, k = U.shape
    n = V.shape[0]
    c = [x.contiguous() if x is not None else None for x in (U, S, V, dU, dS, dV)]
    for x in c:
        if x is not None and x.dtype != torch.float64:
            raise TsSvdError("lowrank_svd_backward: float64 tensors only")
    if V.shape != (n, k) or S.shape != (k,):
        raise TsSvdError("lowrank_svd_backward: U m x k, S k, V n x k")
    dA = torch.empty((m, n), dtype=torch.float64, device=U.device)
    o = _opts(mode=mode, stream=stream, workspace=workspace)
    with torch.cuda.device(U.device):
        rc = lib().lowrank_svd_backward(m, n, k, *[_ptr(x) for x in c], _ptr(dA),
                                        ctypes.byref(o))
    _check(rc, "lowrank_svd_backward")
    return dA


class LowRankSVD(torch.autograd.Function):
    """Differentiable rank-k SVD: forward by lowrank_svd (Algorithm 8),
    backward by lowrank_svd_backward (exact for A of rank k).  Omega (the
    random starting matrix) takes no gradient."""

    @staticmethod
    def forward(ctx, A, k, l, iters, Omega, drop_tol=0.0, mode="fp64"):
        U, S, V, info = lowrank_svd(A, k, l, iters, Omega, drop_tol=drop_tol, mode=mode)
        ctx.save_for_backward(U, S, V)
        ctx.mode = "fp64_tc" if mode == "fp64_tc" else "fp64"
        return U, S, V

    @staticmethod
    def backward(ctx, gU, gS, gV):
        U, S, V = ctx.saved_tensors
        dA = lowrank_svd_backward(U, S, V, dU=gU, dS=gS, dV=gV, mode=ctx.mode)
        return dA, None, None, None, None, None, None


def ts_svd_tsqr(A, theta, perm, passes=2, drop_tol=PAPER_DROP_TOL, max_sweeps=50, stream=None,
                workspace=None, mode="fp64"):
    """Algorithm 1 (passes=1) or 2 (passes=2) on a float64 CUDA tensor A
    (m x n).  theta: 2h phases, perm: 2h int64 indices (h = ceil(n / 2)),
    both CUDA tensors: the random mixing of Remark "randomness".  mode
    "fp64" or "fp64_tc": the engine of the two tall products.  Returns
    (U, S, V, info).  See include/tssvd.h (ts_svd_tsqr)."""
    A = _as_matrix(A)
    m, n = A.shape
    if A.dtype != torch.float64:
        raise TsSvdError("ts_svd_tsqr: float64 only")
    h = (n + 1) // 2
    theta = theta.contiguous()
    perm = perm.contiguous()
    if theta.dtype != torch.float64 or perm.dtype != torch.int64 or theta.numel() != 2 * h \
            or perm.numel() != 2 * h:
        raise TsSvdError("ts_svd_tsqr: theta float64 and perm int64, 2 * ceil(n / 2) each")
    U = torch.empty((m, n), dtype=torch.float64, device=A.device)
    S = torch.empty((n,), dtype=torch.float64, device=A.device)
    V = torch.empty((n, n), dtype=torch.float64, device=A.device)
    o = _opts(passes, False, drop_tol, mode, max_sweeps, stream, workspace)
    with torch.cuda.device(A.device):
        rc = lib().ts_svd_tsqr(_ptr(A), m, n, A.stride(0), _ptr(theta), _ptr(perm), _ptr(U),
                               _ptr(S), _ptr(V), ctypes.byref(o))
    _check(rc, "ts_svd_tsqr")
    return U, S, V, _info(o, rc)


def lowrank_svd_tsqr(A, k, l, iters, Omega, theta, perm, drop_tol=PAPER_DROP_TOL, max_sweeps=50,
                     stream=None, workspace=None, mode="fp64"):
    """Algorithm 7 (float64 CUDA tensors): returns (U m x k, S k, V n x k,
    info).  theta, perm: the mixing draw for l columns (2 ceil(l/2) each);
    mode "fp64" or "fp64_tc" (the engine of the tall products).  See
    include/tssvd.h (lowrank_svd_tsqr)."""
    A = _as_matrix(A)
    m, n = A.shape
    Omega = Omega.contiguous()
    theta = theta.contiguous()
    perm = perm.contiguous()
    h = (l + 1) // 2
    if theta.numel() != 2 * h or perm.numel() != 2 * h or perm.dtype != torch.int64:
        raise TsSvdError("lowrank_svd_tsqr: theta and perm of 2 * ceil(l / 2) entries")
    U = torch.empty((m, k), dtype=torch.float64, device=A.device)
    S = torch.empty((k,), dtype=torch.float64, device=A.device)
    V = torch.empty((n, k), dtype=torch.float64, device=A.device)
    o = _opts(2, False, drop_tol, mode, max_sweeps, stream, workspace)
    with torch.cuda.device(A.device):
        rc = lib().lowrank_svd_tsqr(_ptr(A), m, n, A.stride(0), int(k), int(l), int(iters),
                                    _ptr(Omega), _ptr(theta), _ptr(perm), _ptr(U), _ptr(S),
                                    _ptr(V), ctypes.byref(o))
    _check(rc, "lowrank_svd_tsqr")
    return U, S, V, _info(o, rc)
