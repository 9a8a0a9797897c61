"""The row-sharded form on the CPU (no GPU): world_size-2 gloo process
groups exercise the collective that ts_svd_rowshard calls back
(reduce_fixed_order) and the decomposition it implements, with the FP64
oracle's steps standing in for the kernels on each rank:

- the row split (row_block) covers every row once;
- the per-rank Gram matrices (the per-partition Gram matrices of the
  paper's Section 2), summed in rank order, equal the whole matrix's Gram
  bit for bit on integer data (every sum exact) and to rounding otherwise,
  with every rank holding the same bits;
- Algorithm 4 carried out with per-rank tall steps and all-reduced Gram
  matrices, column maxima and sums of squares (the exchanges the library
  makes) gives the oracle's SVD of the whole matrix.
"""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_row_block_partition():
    import sys
    sys.path.insert(0, ROOT)
    from paper_1612_08709_gb300._rowshard import row_block
    for m, size in [(10, 3), (7, 7), (1000, 4), (1001, 8)]:
        got = [row_block(m, r, size) for r in range(size)]
        assert got[0][0] == 0 and got[-1][1] == m
        for (a, b), (c, d) in zip(got, got[1:]):
            assert b == c
        lens = [b - a for a, b in got]
        assert max(lens) - min(lens) <= 1
    with pytest.raises(ValueError):
        row_block(3, 0, 4)


def _sharded_alg4(A_local, reduce):
    """Algorithm 4 with MaxEntry scaling on row blocks: tall steps on the
    local rows (oracle kernels), exchanges through reduce(array, op)."""
    import oracle
    n = A_local.shape[1]
    # MaxEntry column scaling: column maxima over all rows (op 1 = max)
    cmax = reduce(np.abs(A_local).max(axis=0), 1)
    d = np.where(cmax > 0, 2.0 ** np.ceil(np.log2(np.where(cmax > 0, cmax, 1.0))), 1.0)
    As = A_local / d
    B = reduce(oracle.gram(As), 0)
    lam, Vt, _, _ = oracle.jacobi_eig(B)
    Yt = oracle.matmul(As, Vt)
    sig = np.sqrt(reduce(oracle.col_norms(Yt) ** 2, 0))
    Y = Yt / sig
    Z = reduce(oracle.gram(Y), 0)
    mu, W, _, _ = oracle.jacobi_eig(Z)
    Qt = oracle.matmul(Y, W)
    T = np.sqrt(reduce(oracle.col_norms(Qt) ** 2, 0))
    Q = Qt / T
    R = (T[:, None] * W.T * sig[None, :]) @ Vt.T * d[None, :]
    X, P, s, _ = oracle.jacobi(np.ascontiguousarray(R.T))
    V = X / s
    U = oracle.matmul(Q, P)
    return U, s, V


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import workloads
        from paper_1612_08709_gb300._rowshard import reduce_fixed_order, row_block

        def reduce(a, op):
            t = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64))
            return reduce_fixed_order(t, op).numpy().copy()

        out = {}
        # integer data: every partial and total Gram entry is exact
        m, n = 3001, 17
        Ai = np.random.default_rng(5).integers(-50, 51, size=(m, n)).astype(np.float64)
        lo, hi = row_block(m, rank, world)
        Bi = reduce(oracle.gram(Ai[lo:hi]), 0)
        out["int_exact"] = bool(np.array_equal(Bi, oracle.gram(Ai)))
        out["int_bytes"] = Bi.tobytes()
        # general data: to rounding, same bits on every rank
        Ag = np.random.default_rng(6).standard_normal((m, n))
        Bg = reduce(oracle.gram(Ag[lo:hi]), 0)
        ref = oracle.gram(Ag)
        out["gen_err"] = float(np.abs(Bg - ref).max() / np.abs(ref).max())
        out["gen_bytes"] = Bg.tobytes()
        # maximum
        mx = reduce(np.abs(Ag[lo:hi]).max(axis=0), 1)
        out["max_ok"] = bool(np.array_equal(mx, np.abs(Ag).max(axis=0)))
        # the sharded two-pass TS-SVD against the oracle on the whole matrix
        m2, n2 = 4000, 40
        A, _, s0, _ = workloads.known_spectrum(m2, n2, workloads.sigma_geometric(n2, 1e-7), 7)
        lo2, hi2 = row_block(m2, rank, world)
        U, S, V = _sharded_alg4(A[lo2:hi2], reduce)
        out["block"] = (lo2, hi2)
        out["U"], out["S"], out["V"] = U, S, V
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_rank_gram_reduction_and_sharded_svd():
    mp = pytest.importorskip("torch.multiprocessing")
    import oracle
    import workloads
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r0, r1 = res[0], res[1]
    assert r0["int_exact"] and r1["int_exact"]
    assert r0["int_bytes"] == r1["int_bytes"]
    assert r0["gen_err"] <= 1e-15 and r0["gen_bytes"] == r1["gen_bytes"]
    assert r0["max_ok"] and r1["max_ok"]
    # replicated results are identical on both ranks
    assert np.array_equal(r0["S"], r1["S"]) and np.array_equal(r0["V"], r1["V"])
    m2, n2 = 4000, 40
    A, _, s0, _ = workloads.known_spectrum(m2, n2, workloads.sigma_geometric(n2, 1e-7), 7)
    Ur, Sr, Vr, rr, st = oracle.ts_svd(A, passes=2, scale=True, drop_tol=0.0)
    U = np.vstack([r0["U"], r1["U"]])
    assert np.abs(r0["S"] - Sr).max() <= 1e-11 * Sr[0]
    assert np.abs(r0["S"] - s0).max() <= 1e-11 * s0[0]
    assert np.abs(U.T @ U - np.eye(n2)).max() <= 1e-12
    for j in range(n2):  # vectors up to sign (distinct singular values)
        sg = np.sign(Vr[:, j] @ r0["V"][:, j])
        assert np.abs(r0["V"][:, j] * sg - Vr[:, j]).max() <= 1e-9
        assert np.abs(U[:, j] * sg - Ur[:, j]).max() <= 1e-9
