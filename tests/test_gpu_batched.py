"""Batched TS-SVD (one CUDA-graph launch for many uneven members) against
the one-call-per-member path and the oracle."""
import numpy as np
import pytest

import workloads

gpu = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _members(count, seed, m_range=(300, 20000), n_range=(1, 64)):
    shapes = workloads.batch_shapes(count, seed, m_range, n_range)
    mats = [workloads.batch_instance(m, n, seed * 1000 + i)[0] for i, (m, n) in enumerate(shapes)]
    return shapes, mats


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_batched_equals_per_member_calls(mode):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    shapes, mats = _members(24, 3)
    As = [torch.as_tensor(A, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As, drop_tol=0.0, mode=mode)
    for A, (U, S, V), info in zip(As, outs, infos):
        U1, S1, V1, i1 = pkg.ts_svd(A, drop_tol=0.0, mode=mode)
        assert info["rank"] == i1["rank"] and info["status"] == i1["status"]
        if mode == "fp64":
            # same kernels, same launch shapes: identical results
            assert torch.equal(S, S1) and torch.equal(U, U1) and torch.equal(V, V1)
        else:
            # the phased batch (one-CTA Jacobi solves, one-sided second
            # eigensolve): the same SVD to rounding
            n = A.shape[1]
            eye = torch.eye(n, dtype=A.dtype, device=A.device)
            assert (S - S1).abs().max() <= 1e-12 * S1[0]
            assert (U.T @ U - eye).abs().max() <= 1e-12
            assert (V.T @ V - eye).abs().max() <= 1e-12
            assert (A @ V - U * S).abs().max() <= 1e-11 * S1[0]


@gpu
def test_batched_wide_members_match_oracle(orc):
    """Members with n from 100 to 256: the batch gives the oracle's SVD,
    member by member."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    shapes, mats = _members(6, 9, m_range=(2000, 30000), n_range=(100, 256))
    As = [torch.as_tensor(A, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As, drop_tol=0.0, mode="fp64_tc")
    for A, (U, S, V), info in zip(mats, outs, infos):
        Ur, Sr, Vr, rr, st = orc.ts_svd(A, drop_tol=0.0)
        n = A.shape[1]
        S, U, V = S.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()
        assert info["rank"] == rr == n
        assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
        assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
        assert np.abs(A @ V - U * S).max() <= 1e-10 * Sr[0]


@gpu
def test_batched_replay_and_oracle(orc):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    shapes, mats = _members(12, 5)
    As = [torch.as_tensor(A, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As, drop_tol=0.0)
    first = [o[1].clone() for o in outs]
    L = pkg.lib()
    n0 = L.tssvd_launch_count()
    outs2, infos2, rc2 = pkg.ts_svd_batched(As, drop_tol=0.0, outs=outs)
    assert L.tssvd_launch_count() > n0  # replayed graph kernels are counted
    for a, b in zip(first, outs2):
        assert torch.equal(a, b[1])
    for A, (U, S, V), info in list(zip(mats, outs2, infos2))[:4]:
        Ur, Sr, Vr, rr, st = orc.ts_svd(A, drop_tol=0.0)
        assert info["rank"] == rr
        assert np.abs(S.cpu().numpy() - Sr).max() <= 1e-11 * Sr[0]
        Uh = U.cpu().numpy()
        assert np.abs(Uh.T @ Uh - np.eye(A.shape[1])).max() <= 1e-12


@gpu
def test_batched_fp32_and_autotuned(orc):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    shapes, mats = _members(10, 7, n_range=(8, 48))
    As32 = [torch.as_tensor(A, dtype=torch.float32, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As32, drop_tol=0.0)
    for A, (U, S, V) in zip(mats, outs):
        Sr = np.linalg.svd(A.astype(np.float32).astype(np.float64), compute_uv=False)
        assert np.abs(S.double().cpu().numpy() - Sr).max() <= 1e-5 * Sr[0]
    As = [torch.as_tensor(A, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As, drop_tol=0.0, mode="auto")
    assert all(i["mode"] in ("fp64", "fp64_tc") for i in infos)
    for A, (U, S, V) in zip(mats, outs):
        Sr = orc.ts_svd(A, drop_tol=0.0)[1]
        assert np.abs(S.cpu().numpy() - Sr).max() <= 1e-11 * Sr[0]


_FULL_REF = {}


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_batched_full_ranges_every_member_vs_oracle(orc, mode):
    """Members drawn from the 512-member workload's ranges (m in [1,000,
    200,000], n in [16, 256], sigma log-uniform in [1e-6, 1]); every member
    of the batch is compared with the oracle: sigma, both factors' columns
    (Davis-Kahan scale), orthonormality, rank.  Several digit-product column
    tiles per member and Jacobi solves of up to 128 pairs run concurrently
    on the worker streams."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    from test_gpu_parity import col_err_up_to_sign, gaps
    shapes = workloads.batch_shapes(8, 17)
    shapes[0] = (200000, 256)   # the ranges' corners
    shapes[1] = (1000, 16)
    mats = [workloads.batch_instance(m, n, 1700 + i)[0] for i, (m, n) in enumerate(shapes)]
    As = [torch.as_tensor(A, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As, drop_tol=0.0, mode=mode)
    for i, (A, (U, S, V), info) in enumerate(zip(mats, outs, infos)):
        n = A.shape[1]
        if i not in _FULL_REF:
            _FULL_REF[i] = orc.ts_svd(A, drop_tol=0.0)
        Ur, Sr, Vr, rr, st = _FULL_REF[i]
        U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
        assert info["rank"] == rr == n and info["status"] == st
        assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
        assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
        tolv = np.clip(1e-10 * Sr[0] / gaps(Sr), 1e-13, 1.0)
        assert np.all(col_err_up_to_sign(V, Vr) <= tolv)
        assert np.all(col_err_up_to_sign(U, Ur) <= tolv)


@gpu
def test_phased_batch_fp32_storage_and_rank_deficiency(orc):
    """The phased executor (mode auto, n <= 256) with FP32 storage, and with
    FP64 storage on members whose trailing singular values are exactly
    zero (the discard steps drop those columns: exact zeros in S, U, V)."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    shapes = [(6000, 40), (3000, 120), (9000, 7), (2500, 200)]
    mats, ranks = [], []
    for i, (m, n) in enumerate(shapes):
        s = workloads.sigma_geometric(n, 1e-4)
        r = max(1, n - 1 - n // 4)
        s[r:] = 0.0
        A, _, _, _ = workloads.known_spectrum(m, n, s, 4100 + i)
        mats.append(A)
        ranks.append(r)
    As = [torch.as_tensor(A, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As, drop_tol=1e-6, mode="auto")
    for A, r, (U, S, V), info in zip(mats, ranks, outs, infos):
        Ur, Sr, Vr, rr, st = orc.ts_svd(A, drop_tol=1e-6)
        assert info["mode"] == "fp64_tc" and info["rank"] == rr == r
        U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
        assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
        assert np.all(S[r:] == 0) and np.all(U[:, r:] == 0) and np.all(V[:, r:] == 0)
        assert np.abs(U[:, :r].T @ U[:, :r] - np.eye(r)).max() <= 1e-12
        assert np.abs(V[:, :r].T @ V[:, :r] - np.eye(r)).max() <= 1e-12
    As32 = [torch.as_tensor(A, dtype=torch.float32, device="cuda") for A in mats]
    outs, infos, rc = pkg.ts_svd_batched(As32, drop_tol=1e-6, mode="auto")
    for A, (U, S, V), info in zip(mats, outs, infos):
        Sr = np.linalg.svd(A.astype(np.float32).astype(np.float64), compute_uv=False)
        r = info["rank"]
        assert info["mode"] == "fp64_tc"
        assert np.abs(S.double().cpu().numpy()[:r] - Sr[:r]).max() <= 1e-5 * Sr[0]
        Ud = U.double().cpu().numpy()[:, :r]
        assert np.abs(Ud.T @ Ud - np.eye(r)).max() <= 1e-5
