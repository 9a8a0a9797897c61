"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances (FP64 path): singular values within 1e-11 * sigma_1 (normwise,
the stated bound for the FP64-accurate path); singular vectors within
1e-10 * sigma_1 / gap_j per column (the Davis-Kahan scale of FP64 rounding);
orthonormality of U and V <= 1e-12; ranks and statuses identical.
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


def col_err_up_to_sign(X, Y):
    e = np.zeros(X.shape[1])
    for j in range(X.shape[1]):
        e[j] = min(np.abs(X[:, j] - Y[:, j]).max(), np.abs(X[:, j] + Y[:, j]).max())
    return e


def gaps(s):
    g = np.full(len(s), np.inf)
    for j in range(len(s)):
        if j > 0:
            g[j] = min(g[j], abs(s[j - 1] - s[j]))
        if j + 1 < len(s):
            g[j] = min(g[j], abs(s[j] - s[j + 1]))
    return g


def orth(U):
    return np.abs(U.T @ U - np.eye(U.shape[1])).max()


def compare_svd(A, got, ref, s_tol=1e-11, v_tol=1e-10, o_tol=1e-12, check_vectors=True):
    U, S, V = got
    Ur, Sr, Vr, rr = ref
    s1 = Sr[0]
    assert np.abs(S - Sr).max() <= s_tol * s1, (np.abs(S - Sr).max() / s1)
    r = rr
    if r == 0:
        return
    assert orth(U[:, :r]) <= o_tol
    assert orth(V[:, :r]) <= o_tol
    assert np.abs(A @ V[:, :r] - U[:, :r] * S[:r]).max() <= 10 * s_tol * s1
    if check_vectors:
        g = gaps(Sr[:r])
        tolv = np.clip(v_tol * s1 / g, 1e-13, 1.0)
        ev = col_err_up_to_sign(V[:, :r], Vr[:, :r])
        eu = col_err_up_to_sign(U[:, :r], Ur[:, :r])
        assert np.all(ev <= tolv), (ev / tolv).max()
        assert np.all(eu <= tolv), (eu / tolv).max()
    # discarded columns are exactly zero
    assert np.all(S[r:] == 0) and np.all(U[:, r:] == 0) and np.all(V[:, r:] == 0)


def run_gpu(A, dtype=None, lda_pad=0, **kw):
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
    U, S, V, info = pkg.ts_svd(Ad, **kw)
    torch.cuda.synchronize()
    return (U.double().cpu().numpy(), S.double().cpu().numpy(), V.double().cpu().numpy()), info


SHAPES = [(20000, 50, 1), (777, 13, 2), (3001, 130, 3), (200, 200, 4), (1000, 1, 5),
          (4099, 65, 6), (64, 64, 7)]


@gpu
@pytest.mark.parametrize("m,n,seed", SHAPES)
@pytest.mark.parametrize("passes,scale", [(2, True), (2, False), (1, False)])
def test_ts_svd_fp64_matches_oracle(orc, m, n, seed, passes, scale):
    s = workloads.sigma_geometric(n, 1e-6) if n > 1 else np.ones(1)
    A, _, _, _ = workloads.known_spectrum(m, n, s, seed)
    ref = orc.ts_svd(A, passes=passes, scale=scale, drop_tol=0.0)
    got, info = run_gpu(A, passes=passes, scale=scale, drop_tol=0.0)
    assert info["rank"] == ref[3] and info["status"] == ref[4]
    # Algorithm 3 is orthonormal only to ~eps * kappa^2; hold the GPU to the
    # oracle's own level there.
    o_tol = 1e-12 if passes == 2 else max(1e-12, 100 * orth(ref[0][:, :ref[3]]))
    compare_svd(A, got, ref[:4], o_tol=o_tol, check_vectors=(passes == 2))


@gpu
def test_ts_svd_small_tall_workload_error_report(orc):
    """The 20,000 x 50 workload: sigma_j = 10^(-6 (j-1)/49), two passes,
    MaxEntry scaling; sigma error, orthonormality and residual against the
    oracle and against the known spectrum."""
    m, n = 20000, 50
    s = workloads.sigma_small_tall(n)
    A, U0, s0, V0 = workloads.known_spectrum(m, n, s, 1)
    ref = orc.ts_svd(A, passes=2, scale=True, drop_tol=0.0)
    (U, S, V), info = run_gpu(A, passes=2, scale=True, drop_tol=0.0)
    assert np.abs(S - ref[1]).max() <= 1e-11
    assert np.abs(S - s0).max() <= 1e-11
    assert orth(U) <= 1e-12 and orth(V) <= 1e-12
    assert np.linalg.norm(A @ V - U * S) / np.linalg.norm(A) <= 1e-12


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_ts_svd_leading_dimension(orc, mode):
    m, n = 1500, 37
    A, _, _, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-4), 11)
    ref = orc.ts_svd(A, drop_tol=0.0)
    got, info = run_gpu(A, lda_pad=5, drop_tol=0.0, mode=mode)
    compare_svd(A, got, ref[:4])


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_ts_svd_rank_deficient(orc, mode):
    rng = np.random.default_rng(12)
    A = rng.standard_normal((2000, 24))
    A[:, 5] = 0.0
    A[:, 17] = 2.0 * A[:, 3]
    for passes in (1, 2):
        ref = orc.ts_svd(A, passes=passes)
        got, info = run_gpu(A, passes=passes, mode=mode)
        assert info["rank"] == ref[3] == 22
        assert info["status"] == ref[4] == 2
        compare_svd(A, got, ref[:4],
                    o_tol=1e-12 if passes == 2 else max(1e-12, 100 * orth(ref[0][:, :22])),
                    check_vectors=(passes == 2))


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_ts_svd_paper_matrix_discard(orc, mode):
    """The paper's DCT test matrix with the default discard threshold
    sqrt(1e-11): the GPU keeps the same columns as the oracle."""
    A, _, s0, _ = workloads.paper_dct_matrix(3000, 120, 120)
    for passes in (1, 2):
        ref = orc.ts_svd(A, passes=passes, scale=False)
        got, info = run_gpu(A, passes=passes, scale=False, mode=mode)
        assert info["rank"] == ref[3]
        r = ref[3]
        assert np.abs(got[1][:r] - ref[1][:r]).max() <= 1e-11


@gpu
def test_ts_svd_fp32_storage(orc):
    torch = _torch()
    m, n = 5000, 40
    A, _, s0, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-3), 13)
    A32 = A.astype(np.float32)
    ref = orc.ts_svd(A32.astype(np.float64), drop_tol=0.0)
    (U, S, V), info = run_gpu(A32.astype(np.float64), dtype=torch.float32, drop_tol=0.0)
    assert np.abs(S - ref[1]).max() <= 1e-6 * ref[1][0]
    assert orth(U) <= 1e-5 and orth(V) <= 1e-5


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_lowrank_paper_pin_on_gpu(orc, mode):
    """Algorithm 8 on the GPU reproduces the paper's printed error (sigma_7
    for l = 20, i = 2) and matches the oracle run with the same Omega, with
    the products in FP64 FMA or in FP64-accurate tensor-core digits."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n, l = 1500, 400, 20
    A, _, s0, _ = workloads.paper_dct_matrix(m, n, l)
    Om = workloads.gaussian(n, l, 4)
    Ur, Sr, Vr, rr, st = orc.lowrank_svd(A, l, l, 2, Om)
    U, S, V, info = pkg.lowrank_svd(torch.as_tensor(A, device="cuda"), l, l, 2,
                                    torch.as_tensor(Om, device="cuda"), mode=mode)
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    assert info["rank"] == rr == 6
    err = orc.spectral_error(A, U[:, :rr], S[:rr], V[:, :rr])
    assert abs(err - 4.83e-7) < 0.006 * 4.83e-7
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("m,n,k,l,iters,seed", [(3000, 700, 10, 16, 2, 21), (1200, 900, 5, 8, 0, 22),
                                                (2049, 1000, 30, 40, 1, 23),
                                                (1000, 2500, 20, 70, 1, 24)])
def test_lowrank_matches_oracle(orc, m, n, k, l, iters, seed, mode):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    A, _, _, _ = workloads.lowrank_plus_noise(m, n, 60, seed)
    Om = workloads.gaussian(n, l, seed + 100)
    Ur, Sr, Vr, rr, st = orc.lowrank_svd(A, k, l, iters, Om, drop_tol=0.0)
    U, S, V, info = pkg.lowrank_svd(torch.as_tensor(A, device="cuda"), k, l, iters,
                                    torch.as_tensor(Om, device="cuda"), drop_tol=0.0, mode=mode)
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    assert info["rank"] == rr
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
    assert orth(U) <= 1e-12 and orth(V) <= 1e-12
    g = gaps(Sr)
    tolv = np.clip(1e-9 * Sr[0] / g, 1e-13, 1.0)
    assert np.all(col_err_up_to_sign(V, Vr) <= tolv)
    assert np.all(col_err_up_to_sign(U, Ur) <= tolv)


@gpu
def test_backward_matches_oracle(orc):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n, k = 3000, 32, 4
    s = workloads.sigma_distinct_gaps(n)
    A, _, _, _ = workloads.known_spectrum(m, n, s, 31)
    rng = np.random.default_rng(32)
    w = rng.standard_normal(n)
    Bm = rng.standard_normal((m, 8))
    Ad = torch.as_tensor(A, device="cuda")
    U, S, V, info = pkg.ts_svd(Ad, drop_tol=0.0)
    Uh = U.cpu().numpy()
    dU = np.zeros((m, n))
    dU[:, :k] = 2.0 * Bm @ (Bm.T @ Uh[:, :k])
    dV = rng.standard_normal((n, n))
    dA = pkg.ts_svd_backward(Ad, S, V, dU=torch.as_tensor(dU, device="cuda"),
                             dS=torch.as_tensor(w, device="cuda"),
                             dV=torch.as_tensor(dV, device="cuda")).cpu().numpy()
    ref = orc.ts_svd_backward(A, S.cpu().numpy(), V.cpu().numpy(), dU=dU, dS=w, dV=dV)
    assert np.abs(dA - ref).max() <= 1e-10 * np.abs(ref).max()


@gpu
def test_invalid_argument_raises():
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    A = torch.zeros((3, 5), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.TsSvdError):
        pkg.ts_svd(A)


@gpu
@pytest.mark.parametrize("m,n,seed", [(5003, 77, 41), (20000, 200, 42), (300, 300, 43), (100, 1, 44)])
def test_gram_matches_oracle(orc, m, n, seed):
    """Step a2 on its own: B = A^T A against the oracle's Gram."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    A = np.random.default_rng(seed).standard_normal((m, n))
    B = pkg.ts_gram(torch.as_tensor(A, device="cuda")).cpu().numpy()
    Br = orc.gram(A)
    assert np.abs(B - Br).max() <= 1e-13 * np.abs(Br).max()
    assert np.array_equal(B, B.T)


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_repeated_singular_values_match_oracle(orc, mode):
    """Appendix B's spectrum (many repeated singular values and a zero): the
    GPU matches the oracle in the values and, for each repeated value, in
    the column subspace of U and V (individual vectors are not defined)."""
    n = 96
    s = workloads.sigma_devils_staircase(n)
    A, _, s0, _ = workloads.known_spectrum(5000, n, s, 43)
    Ur, Sr, Vr, rr, st = orc.ts_svd(A, drop_tol=0.0)
    (U, S, V), info = run_gpu(A, drop_tol=0.0, mode=mode)
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
    k = int((s0 > 0).sum())
    assert orth(U[:, :k]) <= 1e-12 and orth(V[:, :k]) <= 1e-12
    for X, Y in ((U, Ur), (V, Vr)):
        for v in np.unique(s0[:k]):
            idx = np.where(s0[:k] == v)[0]
            d = np.abs(X[:, idx] @ X[:, idx].T - Y[:, idx] @ Y[:, idx].T).max()
            assert d <= 1e-10, (v, d)


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_ts_svd_badly_scaled_columns(orc, mode):
    """Columns scaled from 1e-150 to 1e150 (MaxEntry scaling, Remark
    "working"'s motivation for scale-aware processing; per-column digit
    exponents far apart): the two-pass result matches the oracle's relative
    to each column's scale."""
    m, n = 3000, 24
    A, _, _, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-2), 61)
    colscale = 10.0 ** np.linspace(-150, 150, n)
    A = A * colscale
    Ur, Sr, Vr, rr, st = orc.ts_svd(A, drop_tol=0.0)
    (U, S, V), info = run_gpu(A, drop_tol=0.0, mode=mode)
    assert info["rank"] == rr and info["status"] == st == 0
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
    assert orth(U[:, :rr]) <= 1e-12 and orth(V[:, :rr]) <= 1e-12
    # residual column by column relative to the column's own scale
    R = A @ V[:, :rr] - U[:, :rr] * S[:rr]
    assert np.abs(R).max() <= 1e-10 * Sr[0]


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_ts_svd_three_hundred_columns(orc, mode):
    """n = 300: several Gram tiles (digit path: 3 row blocks of 128), 150
    Jacobi pairs over more than one CTA per pair index range."""
    m, n = 6000, 300
    A, _, _, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-6), 62)
    ref = orc.ts_svd(A, drop_tol=0.0)
    got, info = run_gpu(A, drop_tol=0.0, mode=mode)
    compare_svd(A, got, ref[:4])
