"""Row-sharded TS-SVD (ts_svd_rowshard) and the collectives it calls back.

Each rank holds a block of A's rows.  The library makes every exchange of
the method through the caller's all-reduce (include/tssvd.h, tssvd_comm):
the MaxEntry column maxima, each Gram matrix (the per-partition Gram
matrices the paper's Section 2 aggregates) and each step's column sums of
squares.  Everything else runs in the library's kernels; this module only
marshals tensors and adapts a torch.distributed process group to the C
callback.
"""
import ctypes

import torch

from ._binding import PAPER_DROP_TOL, TsSvdError, _as_matrix, _check, _info, _opts, _ptr, lib

DT_F64, DT_U64 = 0, 1
OP_SUM, OP_MAX = 0, 1

_ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


class _Comm(ctypes.Structure):
    _fields_ = [("allreduce", _ALLREDUCE_FN), ("ctx", ctypes.c_void_p), ("rank", ctypes.c_int),
                ("size", ctypes.c_int)]


class _DeviceArray:
    """A device pointer seen as a 1-D array (CUDA array interface), so that
    torch can wrap the library's buffer without a copy."""

    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr), False), "strides": None,
                                         "version": 3}


def device_view(ptr, count, dtype, device):
    """The library's device buffer as a torch tensor (float64, or int64 for
    the unsigned 64-bit column maxima: they are bit patterns of |x|, below
    2^63, so signed and unsigned maxima agree)."""
    arr = _DeviceArray(ptr, count, "<f8" if dtype == DT_F64 else "<i8")
    return torch.as_tensor(arr, device=device)


def reduce_fixed_order(t, op, group=None):
    """All-reduce of tensor t in place that every rank finishes with the
    same bits whatever the backend: the ranks' arrays are gathered and
    combined in rank order (sum or maximum)."""
    import torch.distributed as dist
    size = dist.get_world_size(group)
    if size == 1:
        return t
    parts = [torch.empty_like(t) for _ in range(size)]
    dist.all_gather(parts, t, group=group)
    acc = parts[0].clone()
    for p in parts[1:]:
        if op == OP_SUM:
            acc += p
        else:
            torch.maximum(acc, p, out=acc)
    t.copy_(acc)
    return t


def row_block(m, rank, size):
    """Rows [lo, hi) of an m-row matrix held by `rank` of `size`: blocks as
    equal as possible, the first m % size ranks one row longer."""
    if not (0 <= rank < size) or m < size:
        raise ValueError("need 0 <= rank < size <= m")
    q, r = divmod(m, size)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


class DistComm:
    """tssvd_comm over a torch.distributed process group: the library's
    device buffers are reduced with reduce_fixed_order on the call's stream
    (NCCL for CUDA tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)
        self.failures = 0
        self._cb = _ALLREDUCE_FN(self._allreduce)
        self.c = _Comm(self._cb, None, self.rank, self.size)

    def _allreduce(self, buf, count, dtype, op, stream, ctx):
        try:
            dev = torch.cuda.current_device()
            t = device_view(buf, count, dtype, dev)
            st = (torch.cuda.ExternalStream(stream, device=dev) if stream
                  else torch.cuda.default_stream(dev))
            with torch.cuda.stream(st):
                reduce_fixed_order(t, op, self.group)
            return 0
        except Exception:  # reported to the library as a failed exchange
            self.failures += 1
            return 1


def ts_svd_rowshard(A_local, comm, passes=2, scale=True, drop_tol=PAPER_DROP_TOL, mode="fp64",
                    max_sweeps=50, stream=None, workspace=None, out=None):
    """Thin SVD of the matrix whose rows are spread over the ranks of
    `comm` (a DistComm or any object with a ctypes tssvd_comm in `.c`);
    A_local is this rank's block (m_local x n CUDA float64 tensor).

    Returns (U_local m_local x n, S n, V n x n, info); S and V are the same
    on every rank.  See include/tssvd.h (ts_svd_rowshard).
    """
    A = _as_matrix(A_local)
    if A.dtype != torch.float64:
        raise TsSvdError("ts_svd_rowshard takes float64")
    m, n = A.shape
    if out is None:
        U = torch.empty((m, n), dtype=A.dtype, device=A.device)
        S = torch.empty((n,), dtype=A.dtype, device=A.device)
        V = torch.empty((n, n), dtype=A.dtype, device=A.device)
    else:
        U, S, V = out
    o = _opts(passes, scale, drop_tol, mode, max_sweeps, stream, workspace)
    with torch.cuda.device(A.device):
        rc = lib().ts_svd_rowshard(_ptr(A), m, n, A.stride(0), _ptr(U), _ptr(S), _ptr(V),
                                   ctypes.byref(comm.c), ctypes.byref(o))
    _check(rc, "ts_svd_rowshard")
    return U, S, V, _info(o, rc)
