"""FP64-accurate tensor-core mode (TSSVD_FP64_TC): digit-sliced products on
tcgen05 against FP64 references, and the full TS-SVD held to the same
oracle tolerances as the plain FP64 path.

Error bounds: each value keeps 49 bits below its row's power-of-two scale
(truncated digits), products of digit pairs are exact, level sums are exact
in FP32 and combined in double-FP32 (about 2^-47).  Gram entries are held
to 2e-13 * sqrt(B_ii B_jj) and product entries to 2e-13 * (|A| |M|)_rj.
"""
import numpy as np
import pytest

import workloads

gpu = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@gpu
@pytest.mark.parametrize("m,n,seed", [(64, 16, 1), (1000, 37, 2), (5003, 128, 3), (20000, 200, 4),
                                      (3001, 300, 5), (130, 129, 6), (700, 1, 7)])
def test_fp64tc_gram(m, n, seed):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    A = np.random.default_rng(seed).standard_normal((m, n)) * np.logspace(0, -3, n)
    B = pkg.ts_gram(torch.as_tensor(A, device="cuda"), mode="fp64_tc").cpu().numpy()
    ref = A.T @ A
    d = np.sqrt(np.diag(ref))
    err = np.abs(B - ref) / np.outer(d, d)
    assert err.max() <= 2e-13, err.max()


@gpu
@pytest.mark.parametrize("m,k,n,seed", [(128, 16, 16, 1), (1000, 50, 50, 2), (777, 200, 200, 3),
                                        (4099, 65, 256, 4), (300, 333, 7, 5), (129, 129, 130, 6)])
def test_fp64tc_matmul(m, k, n, seed):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, k)) * rng.uniform(0.5, 2.0, size=(m, 1))
    M = rng.standard_normal((k, n))
    C = pkg.ts_matmul(torch.as_tensor(A, device="cuda"), torch.as_tensor(M, device="cuda"),
                      mode="fp64_tc").cpu().numpy()
    ref = A @ M
    scale = np.abs(A) @ np.abs(M)
    err = np.abs(C - ref) / scale
    assert err.max() <= 2e-13, err.max()


def _col_err(X, Y):
    return np.array([min(np.abs(X[:, j] - Y[:, j]).max(), np.abs(X[:, j] + Y[:, j]).max())
                     for j in range(X.shape[1])])


@gpu
@pytest.mark.parametrize("m,n,lo,seed", [(20000, 50, 1e-6, 1), (20000, 50, 1e-8, 2),
                                         (3001, 130, 1e-6, 3), (200, 200, 1e-6, 4),
                                         (4099, 65, 1e-4, 6), (1000, 1, 1.0, 5)])
@pytest.mark.parametrize("passes,scale", [(2, True), (2, False), (1, False)])
def test_fp64tc_ts_svd_matches_oracle(orc, m, n, lo, seed, passes, scale):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    s = workloads.sigma_geometric(n, lo) if n > 1 else np.ones(1)
    A, _, _, _ = workloads.known_spectrum(m, n, s, seed)
    Ur, Sr, Vr, rr, st = orc.ts_svd(A, passes=passes, scale=scale, drop_tol=0.0)
    U, S, V, info = pkg.ts_svd(torch.as_tensor(A, device="cuda"), passes=passes, scale=scale,
                               drop_tol=0.0, mode="fp64_tc")
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    assert info["rank"] == rr
    # Algorithm 3 takes sigma from the Gram matrix, which resolves sigma_j
    # only to about eps * sigma_1^2 / sigma_j (1e-8 at condition 1e8), for
    # the oracle and the GPU alike
    s_tol = 1e-11 if (passes == 2 or lo >= 1e-6) else 1e-7
    assert np.abs(S - Sr).max() <= s_tol * Sr[0]
    if passes == 2:
        assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
        g = np.full(n, np.inf)
        for j in range(n):
            if j > 0:
                g[j] = min(g[j], Sr[j - 1] - Sr[j])
            if j + 1 < n:
                g[j] = min(g[j], Sr[j] - Sr[j + 1])
        tolv = np.clip(1e-10 * Sr[0] / g, 1e-13, 1.0)
        assert np.all(_col_err(V, Vr) <= tolv)
        assert np.all(_col_err(U, Ur) <= tolv)
    else:
        o_ref = np.abs(Ur.T @ Ur - np.eye(n)).max()
        assert np.abs(U.T @ U - np.eye(n)).max() <= max(1e-12, 100 * o_ref)
    assert np.abs(A @ V - U * S).max() <= 1e-10 * Sr[0]


@gpu
def test_fp64tc_fp32_storage(orc):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n = 5000, 40
    A, _, _, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-3), 13)
    A32 = A.astype(np.float32)
    ref = orc.ts_svd(A32.astype(np.float64), drop_tol=0.0)
    U, S, V, info = pkg.ts_svd(torch.as_tensor(A32, device="cuda"), drop_tol=0.0, mode="fp64_tc")
    S = S.double().cpu().numpy()
    U = U.double().cpu().numpy()
    assert np.abs(S - ref[1]).max() <= 1e-6 * ref[1][0]
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-5


@gpu
@pytest.mark.parametrize("mode", ["fp64_tc", "fp64"])
@pytest.mark.parametrize("m,n,lo,seed,rank", [(20000, 50, 1e-8, 11, 50), (3001, 130, 1e-6, 12, 130),
                                              (5000, 60, 1e-4, 13, 40)])
def test_three_passes_match_oracle(orc, mode, m, n, lo, seed, rank):
    """passes = 3 (the second pass of Algorithm 4 run once more on Q):
    the same SVD as the oracle's two passes, to the two-pass tolerances;
    columns dropped by the second pass stay dropped (rank 40 of 60: the
    trailing singular values are exact zeros)."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    s = workloads.sigma_geometric(n, lo)
    s[rank:] = 0.0
    A, _, _, _ = workloads.known_spectrum(m, n, s, seed)
    tol = 0.0 if rank == n else 1e-6
    Ur, Sr, Vr, rr, st = orc.ts_svd(A, passes=2, scale=True, drop_tol=tol)
    U, S, V, info = pkg.ts_svd(torch.as_tensor(A, device="cuda"), passes=3, scale=True,
                               drop_tol=tol, mode=mode)
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    assert info["rank"] == rr == rank
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
    r = rr
    assert np.abs(U[:, :r].T @ U[:, :r] - np.eye(r)).max() <= 1e-12
    assert np.abs(V[:, :r].T @ V[:, :r] - np.eye(r)).max() <= 1e-12
    g = np.full(r, np.inf)
    for j in range(r):
        if j > 0:
            g[j] = min(g[j], Sr[j - 1] - Sr[j])
        if j + 1 < r:
            g[j] = min(g[j], Sr[j] - Sr[j + 1])
    tolv = np.clip(1e-10 * Sr[0] / g, 1e-13, 1.0)
    assert np.all(_col_err(V[:, :r], Vr[:, :r]) <= tolv)
    assert np.all(_col_err(U[:, :r], Ur[:, :r]) <= tolv)
    assert np.all(S[r:] == 0) and np.all(U[:, r:] == 0) and np.all(V[:, r:] == 0)
    assert np.abs(A @ V - U * S).max() <= 1e-10 * Sr[0]
