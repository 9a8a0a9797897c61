"""The differentiable TS-SVD: TSSVD (torch.autograd.Function over ts_svd and
ts_svd_backward) against FP64 central finite differences, and the FP32
forward/backward against the oracle's FP64 analytic gradient.

Loss of the differentiable workload: L = sum_j w_j sigma_j + ||U_k^T B||_F^2
(sign-invariant), sigma_j = 1 + (n - j)/n (distinct, gaps 1/n).
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


def _setup(m, n, k, nb, seed, dtype):
    torch = _torch()
    s = workloads.sigma_distinct_gaps(n)
    A, _, _, _ = workloads.known_spectrum(m, n, s, seed)
    rng = np.random.default_rng(seed + 1)
    w = rng.standard_normal(n)
    Bm = rng.standard_normal((m, nb))
    dev = "cuda"
    return (torch.as_tensor(A, dtype=dtype, device=dev), torch.as_tensor(w, dtype=dtype, device=dev),
            torch.as_tensor(Bm, dtype=dtype, device=dev), A, w, Bm)


def _loss(torch, pkg, A, w, Bm, k):
    U, S, V = pkg.TSSVD.apply(A, 2, True, 0.0)
    return (w * S).sum() + ((U[:, :k].T @ Bm) ** 2).sum()


@gpu
def test_autograd_matches_finite_differences():
    """2,000 x 32, k = 4, B 2,000 x 8: the analytic adjoint against central
    differences of the GPU forward, relative error <= 1e-6."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n, k = 2000, 32, 4
    A, w, Bm, _, _, _ = _setup(m, n, k, 8, 41, torch.float64)
    Ag = A.clone().requires_grad_(True)
    L = _loss(torch, pkg, Ag, w, Bm, k)
    L.backward()
    G = Ag.grad
    rng = np.random.default_rng(7)
    for t in range(3):
        E = torch.as_tensor(rng.standard_normal((m, n)), device="cuda")
        h = 1e-6
        with torch.no_grad():
            lp = _loss(torch, pkg, A + h * E, w, Bm, k)
            lm = _loss(torch, pkg, A - h * E, w, Bm, k)
        fd = float((lp - lm) / (2 * h))
        an = float((G * E).sum())
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (fd, an)


@gpu
def test_backward_fp64_and_fp32_match_oracle_gradient(orc):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n, k = 5000, 64, 8
    A, w, Bm, A_h, w_h, B_h = _setup(m, n, k, 8, 43, torch.float64)
    U, S, V, info = pkg.ts_svd(A, drop_tol=0.0)
    Uh = U.cpu().numpy()
    dU = np.zeros((m, n))
    dU[:, :k] = 2.0 * B_h @ (B_h.T @ Uh[:, :k])
    ref = orc.ts_svd_backward(A_h, S.cpu().numpy(), V.cpu().numpy(), dU=dU, dS=w_h)
    g64 = pkg.ts_svd_backward(A, S, V, dU=torch.as_tensor(dU, device="cuda"), dS=w).cpu().numpy()
    assert np.abs(g64 - ref).max() <= 1e-10 * np.abs(ref).max()
    # FP32 storage: forward in ts_svd_f32, adjoint evaluated in FP64
    A32 = A.float()
    U32, S32, V32, info = pkg.ts_svd(A32, drop_tol=0.0)
    dU32 = torch.as_tensor(dU, dtype=torch.float32, device="cuda")
    g32 = pkg.ts_svd_backward(A32, S32, V32, dU=dU32, dS=w.float()).double().cpu().numpy()
    assert np.abs(g32 - ref).max() <= 1e-3 * np.abs(ref).max()


@gpu
def test_fp32_forward_autograd_runs_on_the_workload_loss():
    """FP32 forward (FP64 eigensolves) and backward through autograd on a
    reduced copy of the 500,000 x 512 workload: the gradient agrees with the
    FP64 path's to FP32 accuracy."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n, k = 20000, 128, 16
    A64, w64, B64, _, _, _ = _setup(m, n, k, 8, 47, torch.float64)
    Ag = A64.clone().requires_grad_(True)
    _loss(torch, pkg, Ag, w64, B64, k).backward()
    A32 = A64.float().requires_grad_(True)
    _loss(torch, pkg, A32, w64.float(), B64.float(), k).backward()
    g64, g32 = Ag.grad, A32.grad.double()
    assert float((g32 - g64).abs().max()) <= 1e-3 * float(g64.abs().max())


@gpu
def test_backward_fp64_tc_matches_oracle_gradient(orc):
    """The adjoint with its three tall products on the FP64-accurate
    digit-sliced tensor-core kernels: FP64 storage within 1e-10 of the
    oracle's analytic gradient (as the FP64 FMA path), FP32 storage within
    FP32 accuracy; autograd through TSSVD in that mode matches FP64's."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n, k = 6000, 96, 8
    A, w, Bm, A_h, w_h, B_h = _setup(m, n, k, 8, 53, torch.float64)
    U, S, V, info = pkg.ts_svd(A, drop_tol=0.0, mode="fp64_tc")
    Uh = U.cpu().numpy()
    dU = np.zeros((m, n))
    dU[:, :k] = 2.0 * B_h @ (B_h.T @ Uh[:, :k])
    dV = np.random.default_rng(54).standard_normal((n, n))
    ref = orc.ts_svd_backward(A_h, S.cpu().numpy(), V.cpu().numpy(), dU=dU, dS=w_h, dV=dV)
    g = pkg.ts_svd_backward(A, S, V, dU=torch.as_tensor(dU, device="cuda"), dS=w,
                            dV=torch.as_tensor(dV, device="cuda"), mode="fp64_tc").cpu().numpy()
    assert np.abs(g - ref).max() <= 1e-10 * np.abs(ref).max()
    A32 = A.float()
    U32, S32, V32, info = pkg.ts_svd(A32, drop_tol=0.0, mode="fp64_tc")
    g32 = pkg.ts_svd_backward(A32, S32, V32, dU=torch.as_tensor(dU, dtype=torch.float32, device="cuda"),
                              dS=w.float(), mode="fp64_tc").double().cpu().numpy()
    ref32 = orc.ts_svd_backward(A_h, S.cpu().numpy(), V.cpu().numpy(), dU=dU, dS=w_h)
    assert np.abs(g32 - ref32).max() <= 1e-3 * np.abs(ref32).max()
    Ag = A.clone().requires_grad_(True)
    U2, S2, V2 = pkg.TSSVD.apply(Ag, 2, True, 0.0, "fp64_tc")
    ((w * S2).sum() + ((U2[:, :k].T @ Bm) ** 2).sum()).backward()
    Af = A.clone().requires_grad_(True)
    _loss(torch, pkg, Af, w, Bm, k).backward()
    assert float((Ag.grad - Af.grad).abs().max()) <= 1e-9 * float(Af.grad.abs().max())


# --------------------------------------------------------------------------
# Rank-k adjoint (lowrank_svd_backward) and the LowRankSVD autograd function
# --------------------------------------------------------------------------


def _factors(m, n, k, seed):
    rng = np.random.default_rng(seed)
    U = workloads.orthonormal(m, k, rng)
    V = workloads.orthonormal(n, k, rng)
    S = np.linspace(4.0, 1.0, k) + 0.1 * rng.random(k)
    S = np.sort(S)[::-1].copy()
    return U, S, V, rng


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("m,n,k,which", [(3000, 700, 20, "all"), (777, 131, 9, "all"),
                                         (2000, 300, 16, "dU"), (2000, 300, 16, "dV"),
                                         (20000, 2000, 50, "all")])
def test_lowrank_backward_matches_oracle(orc, m, n, k, which, mode):
    """Element by element against the oracle's adjoint; tolerance 1e-11 of
    max |dA| (both sides evaluate the same formula in FP64, the GPU with
    the projections folded into one m x 2k by 2k x n product)."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    U, S, V, rng = _factors(m, n, k, 90 + m % 7)
    dU = rng.standard_normal((m, k)) if which in ("all", "dU") else None
    dS = rng.standard_normal(k) if which == "all" else None
    dV = rng.standard_normal((n, k)) if which in ("all", "dV") else None
    ref = orc.lowrank_svd_backward(U, S, V, dU=dU, dS=dS, dV=dV)
    t = lambda x: torch.as_tensor(x, device="cuda") if x is not None else None
    got = pkg.lowrank_svd_backward(t(U), t(S), t(V), dU=t(dU), dS=t(dS), dV=t(dV), mode=mode)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@gpu
@pytest.mark.parametrize("mode", ["fp64", "fp64_tc"])
def test_lowrank_autograd_finite_differences(mode):
    """LowRankSVD on A of rank exactly k: autograd's dA against central
    differences of L = sum_j w_j sigma_j + ||U^T B||_F^2 + ||V^T C||_F^2
    through LAPACK's truncated SVD, along random directions."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n, k, l = 400, 120, 6, 10
    U0, S0, V0, rng = _factors(m, n, k, 95)
    A = (U0 * S0) @ V0.T
    w = rng.standard_normal(k)
    Bm = rng.standard_normal((m, 2))
    Cm = rng.standard_normal((n, 2))
    Omega = rng.standard_normal((n, l))
    Ad = torch.tensor(A, device="cuda", requires_grad=True)
    U, S, V = pkg.LowRankSVD.apply(Ad, k, l, 2, torch.as_tensor(Omega, device="cuda"), 0.0, mode)
    wd, Bd, Cd = (torch.as_tensor(x, device="cuda") for x in (w, Bm, Cm))
    L = (wd * S).sum() + ((U.T @ Bd) ** 2).sum() + ((V.T @ Cd) ** 2).sum()
    L.backward()
    dA = Ad.grad.cpu().numpy()

    def loss(X):
        Ux, sx, Vtx = np.linalg.svd(X, full_matrices=False)
        return float(w @ sx[:k] + np.sum((Ux[:, :k].T @ Bm) ** 2) +
                     np.sum((Vtx[:k] @ Cm) ** 2))

    for _ in range(3):
        E = rng.standard_normal((m, n))
        h = 1e-6
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        an = float(np.sum(dA * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (fd, an)
