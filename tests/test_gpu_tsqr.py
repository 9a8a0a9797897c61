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


CASES = [(3000, 24, 90), (2001, 13, 91), (20000, 50, 92), (777, 9, 93), (50000, 100, 94),
         (300, 300, 95)]


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
