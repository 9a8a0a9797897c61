"""GPU parity of Algorithms 1 and 2 (randomized TS-SVD via TSQR, with the
random mixing of Remark "randomness") against the oracle, through the C
ABI, on the same mixing draws.

Tolerances as in test_gpu_parity: singular values within 1e-11 sigma_1,
vectors within 1e-10 sigma_1 / gap, orthonormality 1e-12; the GPU's TSQR
tree and the oracle's flat Householder QR give the same R up to the signs
of its rows, so the SVDs agree to rounding.
"""
import numpy as np
import pytest

import workloads
from test_gpu_parity import compare_svd

gpu = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run_tsqr(A, mix, **kw):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    t1, t2, p1, p2 = mix
    theta = torch.as_tensor(np.concatenate([t1, t2]), device="cuda")
    perm = torch.as_tensor(np.concatenate([p1, p2]).astype(np.int64), device="cuda")
    Ad = torch.as_tensor(A, device="cuda")
    U, S, V, info = pkg.ts_svd_tsqr(Ad, theta, perm, **kw)
    torch.cuda.synchronize()
    f = lambda t: t.cpu().numpy()
    return (f(U), f(S), f(V)), info


# tree shapes: one block (300 x 300), two to six levels (50,000 x 100),
# panel width 8 (3,000 x 700: blocks of 1,400 rows)
CASES = [(3000, 24, 90), (2001, 13, 91), (20000, 50, 92), (777, 9, 93), (50000, 100, 94),
         (300, 300, 95), (3000, 700, 96)]


@gpu
@pytest.mark.parametrize("passes", [1, 2])
@pytest.mark.parametrize("m,n,seed", CASES)
def test_tsqr_matches_oracle(orc, m, n, seed, passes):
    s = workloads.sigma_geometric(n, 1e-6)
    A, _, _, _ = workloads.known_spectrum(m, n, s, seed)
    mix = workloads.mixing_draws(n, seed)
    ref = orc.ts_svd_tsqr(A, mix, passes=passes, wp=0.0)
    got, info = run_tsqr(A, mix, passes=passes, drop_tol=0.0)
    assert info["rank"] == ref[3] and info["status"] == ref[4]
    compare_svd(A, got, ref[:4])


@gpu
@pytest.mark.parametrize("m,n,seed", CASES[:6])
def test_tsqr_fp64_tc_products_match_oracle(orc, m, n, seed):
    """Algorithm 2 with the two tall products on the FP64-accurate digit
    kernels: the same bar as the FP64 path."""
    s = workloads.sigma_geometric(n, 1e-6)
    A, _, _, _ = workloads.known_spectrum(m, n, s, seed)
    mix = workloads.mixing_draws(n, seed)
    ref = orc.ts_svd_tsqr(A, mix, passes=2, wp=0.0)
    got, info = run_tsqr(A, mix, passes=2, drop_tol=0.0, mode="fp64_tc")
    assert info["rank"] == ref[3] and info["status"] == ref[4]
    compare_svd(A, got, ref[:4])


@gpu
@pytest.mark.parametrize("passes", [1, 2])
def test_tsqr_paper_matrix_discard(orc, passes):
    """The paper's matrix with the working precision 1e-11 (drop_tol =
    sqrt(1e-11)): same discards (rank) and singular values as the oracle."""
    m, n = 4000, 120
    A, _, _, _ = workloads.paper_dct_matrix(m, n, n)
    mix = workloads.mixing_draws(n, 96)
    ref = orc.ts_svd_tsqr(A, mix, passes=passes, wp=1e-11)
    got, info = run_tsqr(A, mix, passes=passes, drop_tol=1e-11 ** 0.5)
    assert info["rank"] == ref[3] and info["status"] == ref[4] == 2
    compare_svd(A, got, ref[:4], check_vectors=False)


@gpu
def test_tsqr_rank_deficient_and_invalid_permutation(orc):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    A = np.random.default_rng(97).standard_normal((5000, 16))
    A[:, 5] = 0.0
    mix = workloads.mixing_draws(16, 98)
    ref = orc.ts_svd_tsqr(A, mix, passes=2)
    got, info = run_tsqr(A, mix, passes=2)
    assert ref[3] == 15 and info["rank"] == 15 and info["status"] == 2
    compare_svd(A, got, ref[:4])
    # a permutation entry out of range is reported as invalid argument 6
    t1, t2, p1, p2 = mix
    p1 = p1.copy()
    p1[3] = 99
    with pytest.raises(pkg.TsSvdError, match="argument 6"):
        run_tsqr(A, (t1, t2, p1, p2))


def run_lowrank_tsqr(A, k, l, iters, Om, mix, **kw):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    t1, t2, p1, p2 = mix
    theta = torch.as_tensor(np.concatenate([t1, t2]), device="cuda")
    perm = torch.as_tensor(np.concatenate([p1, p2]).astype(np.int64), device="cuda")
    U, S, V, info = pkg.lowrank_svd_tsqr(torch.as_tensor(A, device="cuda"), k, l, iters,
                                         torch.as_tensor(Om, device="cuda"), theta, perm, **kw)
    torch.cuda.synchronize()
    return U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy(), info


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("m,n,k,l,iters,seed", [(3000, 800, 10, 16, 2, 100),
                                                (2000, 1500, 20, 25, 1, 101),
                                                (5000, 600, 8, 8, 0, 102)])
def test_lowrank_tsqr_matches_oracle(orc, m, n, k, l, iters, seed, mode):
    """Algorithm 7 on a low-rank-plus-noise matrix: S, U, V against the
    oracle with the same Omega and mixing draw, with the tall products in
    FP64 FMA or FP64-accurate digit products."""
    A, _, _, _ = workloads.lowrank_plus_noise(m, n, 40, seed)
    Om = workloads.gaussian(n, l, seed + 1)
    mix = workloads.mixing_draws(l, seed + 2)
    Ur, Sr, Vr, rr, st = orc.lowrank_svd_tsqr(A, k, l, iters, Om, mix)
    U, S, V, info = run_lowrank_tsqr(A, k, l, iters, Om, mix, mode=mode)
    assert info["rank"] == rr and info["status"] == st
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-12
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-12
    g = np.full(k, np.inf)
    for j in range(k):
        if j > 0: g[j] = min(g[j], Sr[j - 1] - Sr[j])
        if j + 1 < k: g[j] = min(g[j], Sr[j] - Sr[j + 1])
    tol = np.clip(1e-10 * Sr[0] / g, 1e-13, 1.0)
    for j in range(k):
        eu = min(np.abs(U[:, j] - Ur[:, j]).max(), np.abs(U[:, j] + Ur[:, j]).max())
        ev = min(np.abs(V[:, j] - Vr[:, j]).max(), np.abs(V[:, j] + Vr[:, j]).max())
        assert eu <= tol[j] and ev <= tol[j], (j, eu, ev, tol[j])


@gpu
def test_lowrank_tsqr_paper_pin_on_gpu(orc):
    """The paper's matrix for l = 20, i = 2: spectral error sigma_12 =
    2.64e-12 (Algorithm 7's printed value), ranks as the oracle's."""
    l = 20
    m, n = 1500, 400
    A, U0, s0, V0 = workloads.paper_dct_matrix(m, n, l)
    Om = workloads.gaussian(n, l, 4)
    mix = workloads.mixing_draws(l, 11)
    U, S, V, info = run_lowrank_tsqr(A, l, l, 2, Om, mix)
    r = info["rank"]
    ref = orc.lowrank_svd_tsqr(A, l, l, 2, Om, mix)
    assert r == ref[3] == 11
    err = orc.spectral_error(A, U[:, :r], S[:r], V[:, :r])
    assert abs(err - 2.64e-12) < 0.006 * 2.64e-12
    assert orc.orth_error(U[:, :r]) < 1e-13
