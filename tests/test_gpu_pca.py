"""GPU parity of the PCA entry point (abstract, problem 1: the SVD of the
column-centred matrix) against the oracle, through the C ABI.

Tolerances: the means within 4 units of rounding of max |A| (FP64 sums of
up to 200,000 terms in a different order); the SVD of the centred matrix
as in test_gpu_parity (singular values 1e-11 sigma_1, vectors 1e-10
sigma_1 / gap, orthonormality 1e-12), since both sides factor centred
matrices that agree to the rounding of one subtraction.
"""
import numpy as np
import pytest

import workloads
from test_gpu_parity import compare_svd, orth

gpu = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run_pca(A, dtype=None, lda_pad=0, **kw):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    dt = dtype or torch.float64
    m, n = A.shape
    if lda_pad:
        buf = torch.zeros((m, n + lda_pad), dtype=dt, device="cuda")
        buf[:, :n] = torch.as_tensor(A, dtype=dt)
        Ad = buf[:, :n]
    else:
        Ad = torch.as_tensor(A, dtype=dt, device="cuda")
    mu, U, S, V, info = pkg.ts_pca(Ad, **kw)
    torch.cuda.synchronize()
    f = lambda t: t.double().cpu().numpy()
    return f(mu), (f(U), f(S), f(V)), info


CASES = [(20000, 50, 61, 2), (3001, 130, 62, 2), (777, 13, 63, 1), (200000, 200, 64, 2)]


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("m,n,seed,passes", CASES)
def test_pca_matches_oracle(orc, m, n, seed, passes, mode):
    sigma = workloads.sigma_geometric(n, 1e-8)
    A, c, Q, s0, V0 = workloads.pca_data(m, n, sigma, seed)
    mu, got, info = run_pca(A, passes=passes, mode=mode, drop_tol=0.0)
    rmu, U, S, V, r, st = orc.pca(A, passes=passes, drop_tol=0.0)
    assert np.abs(mu - rmu).max() <= 4 * np.finfo(float).eps * np.abs(A).max()
    assert info["rank"] == r and info["status"] == st
    # Algorithm 3 is orthonormal only to ~eps * kappa^2: hold the GPU to the
    # oracle's own level there
    o_tol = 1e-12 if passes == 2 else max(1e-12, 100 * orth(U[:, :r]))
    compare_svd(A - rmu, got, (U, S, V, r), o_tol=o_tol, check_vectors=(passes == 2))


@gpu
def test_pca_leading_dimension_and_fp32(orc):
    torch = _torch()
    A, c, Q, s0, V0 = workloads.pca_data(5000, 40, np.linspace(3.0, 1.0, 40), 65)
    mu, got, info = run_pca(A, lda_pad=3, drop_tol=0.0)
    rmu, U, S, V, r, st = orc.pca(A, drop_tol=0.0)
    assert np.abs(mu - rmu).max() <= 4 * np.finfo(float).eps * np.abs(A).max()
    compare_svd(A - rmu, got, (U, S, V, r))
    # FP32 storage: means and centred values carry FP32 rounding of |A| ~ 1e3
    mu32, (U32, S32, V32), info32 = run_pca(A, dtype=torch.float32, drop_tol=0.0)
    assert np.abs(mu32 - rmu).max() <= 1e-6 * np.abs(A).max()
    assert np.abs(S32 - S).max() <= 2e-3 * S[0]
    assert np.abs(U32.T @ U32 - np.eye(40)).max() <= 1e-4


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_pca_rank_limits(orc, mode):
    """All rows equal: rank 0 and zero outputs.  m = n: rank m - 1."""
    A = np.tile(np.array([1.5, -2.0, 8.0, 0.25, 3e5]), (4096, 1))
    mu, (U, S, V), info = run_pca(A, mode=mode)
    assert np.array_equal(mu, A[0])
    assert info["rank"] == 0 and info["status"] == 2
    assert not S.any() and not U.any() and not V.any()
    B = np.random.default_rng(66).standard_normal((48, 48))
    mu, got, info = run_pca(B, mode=mode)
    rmu, U, S, V, r, st = orc.pca(B)
    assert r == 47 and info["rank"] == 47 and info["status"] == st
    compare_svd(B - rmu, got, (U, S, V, r))
