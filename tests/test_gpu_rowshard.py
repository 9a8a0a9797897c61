"""ts_svd_rowshard through the C ABI on one GPU.

- One rank (a NULL all-reduce): the same bits as ts_svd.
- Two and three ranks in one process: each rank a thread with its own CUDA
  stream and workspace, calling the library on its row block; their
  all-reduce (host-side, rank order) runs when every rank has contributed.
  A token lets one rank's GPU work run at a time (a rank finishes its
  stream before it hands the token on), so no two ranks' kernels are on
  the GPU together and no kernel waits for another rank.  S and V must be
  the same bits on every rank; the stacked U, S and V must match the FP64
  oracle's SVD of the whole matrix at the usual tolerances.
- A failing all-reduce gives TSSVD_ECOMM.
"""
import threading

import numpy as np
import pytest

import workloads
from test_gpu_parity import col_err_up_to_sign, gaps, orth

gpu = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class _Shared:
    def __init__(self, size):
        self.size = size
        self.token = threading.Lock()
        self.cv = threading.Condition()
        self.rounds = {}

    def exchange(self, rnd, rank, arr, op):
        with self.cv:
            parts = self.rounds.setdefault(rnd, {})
            parts[rank] = arr
            self.cv.notify_all()
            ok = self.cv.wait_for(lambda: len(self.rounds[rnd]) == self.size, timeout=120)
            if not ok:
                raise RuntimeError("exchange timed out")
            allp = [self.rounds[rnd][r] for r in range(self.size)]
        acc = allp[0].copy()
        for p in allp[1:]:
            acc = acc + p if op == 0 else np.maximum(acc, p)
        return acc


class _ThreadComm:
    def __init__(self, shared, rank, fail=False):
        import torch
        from paper_1612_08709_gb300 import _rowshard as rs
        self.torch, self.rs = torch, rs
        self.shared, self.rank, self.fail = shared, rank, fail
        self.rnd = 0
        self.calls = 0
        self._cb = rs._ALLREDUCE_FN(self._allreduce)
        self.c = rs._Comm(self._cb, None, rank, shared.size)

    def _allreduce(self, buf, count, dtype, op, stream, ctx):
        torch = self.torch
        self.calls += 1
        if self.fail:
            return 1
        try:
            st = torch.cuda.ExternalStream(stream)
            st.synchronize()
            t = self.rs.device_view(buf, count, dtype, torch.cuda.current_device())
            host = t.cpu().numpy().copy()
            self.shared.token.release()
            try:
                res = self.shared.exchange(self.rnd, self.rank, host, op)
            finally:
                self.shared.token.acquire()
            self.rnd += 1
            with torch.cuda.stream(st):
                t.copy_(torch.from_numpy(res).to(t.device))
            st.synchronize()
            return 0
        except Exception:
            return 1


def _run_ranks(A, size, **kw):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n = A.shape
    shared = _Shared(size)
    out = [None] * size
    errs = []

    def rank_main(r):
        try:
            lo, hi = pkg.row_block(m, r, size)
            st = torch.cuda.Stream()
            Ad = torch.as_tensor(A[lo:hi], device="cuda")
            ws = torch.empty((pkg.ts_svd_workspace_size(hi - lo, n, **kw),), dtype=torch.uint8,
                             device="cuda")
            torch.cuda.synchronize()
            comm = _ThreadComm(shared, r)
            with shared.token:
                U, S, V, info = pkg.ts_svd_rowshard(Ad, comm, stream=st, workspace=ws, **kw)
                st.synchronize()
            out[r] = (U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), info, comm.calls)
        except Exception as e:  # reported below
            errs.append((r, repr(e)))

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(size)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=600)
    assert not errs, errs
    return out


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_rowshard_single_rank_equals_ts_svd(mode):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300 import _rowshard as rs
    m, n = 5000, 60
    A, _, _, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-7), 71)
    Ad = torch.as_tensor(A, device="cuda")

    class One:
        c = rs._Comm(rs._ALLREDUCE_FN(), None, 0, 1)
    U1, S1, V1, i1 = pkg.ts_svd_rowshard(Ad, One(), drop_tol=0.0, mode=mode)
    U0, S0, V0, i0 = pkg.ts_svd(Ad, drop_tol=0.0, mode=mode)
    torch.cuda.synchronize()
    assert torch.equal(U0, U1) and torch.equal(S0, S1) and torch.equal(V0, V1)
    assert i0["rank"] == i1["rank"] and i0["sweeps"] == i1["sweeps"]


@gpu
@pytest.mark.parametrize("size,mode,passes,scale",
                         [(2, "fp64", 2, True), (2, "fp64_tc", 2, True), (3, "fp64_tc", 2, False),
                          (3, "fp64", 1, False)])
def test_rowshard_ranks_match_oracle(orc, size, mode, passes, scale):
    m, n = 9001, 96
    A, _, s0, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-6), 72)
    out = _run_ranks(A, size, passes=passes, scale=scale, drop_tol=0.0, mode=mode)
    for r in range(1, size):
        assert np.array_equal(out[r][1], out[0][1]) and np.array_equal(out[r][2], out[0][2])
        assert out[r][4] == out[0][4] > 0
    U = np.vstack([o[0] for o in out])
    S, V = out[0][1], out[0][2]
    Ur, Sr, Vr, rr, st = orc.ts_svd(A, passes=passes, scale=scale, drop_tol=0.0)
    assert out[0][3]["rank"] == rr
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
    if passes == 2:
        assert orth(U) <= 1e-12 and orth(V) <= 1e-12
        tolv = np.clip(1e-10 * Sr[0] / gaps(Sr), 1e-13, 1.0)
        assert np.all(col_err_up_to_sign(V, Vr) <= tolv)
        assert np.all(col_err_up_to_sign(U, Ur) <= tolv)
    else:
        assert orth(U) <= max(1e-12, 100 * orth(Ur))


@gpu
def test_rowshard_failed_allreduce_reports_ecomm():
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n = 2000, 20
    A = torch.as_tensor(np.random.default_rng(73).standard_normal((m, n)), device="cuda")
    shared = _Shared(1)
    comm = _ThreadComm(shared, 0, fail=True)
    with pytest.raises(pkg.TsSvdError, match="all-reduce"):
        pkg.ts_svd_rowshard(A, comm, drop_tol=0.0)
    assert comm.calls == 1
    # the library is usable afterwards
    U, S, V, info = pkg.ts_svd(A, drop_tol=0.0)
    assert info["rank"] == n
