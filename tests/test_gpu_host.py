"""ts_svd_host: the TS-SVD on host buffers, with the copies of A and U
overlapped with the compute in row chunks (FP64_TC, two passes) or run
before and after it (other modes).  Checked against the oracle on small
shapes and against the device-buffer call and the known spectrum on shapes
of several chunks (the chunked first Gram takes per-chunk digit scales, so
its bits differ from the one-shot Gram while both are FP64-accurate)."""
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
@pytest.mark.parametrize("mode,passes", [("fp64_tc", 2), ("fp64", 2), ("fp64_tc", 3)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_call_matches_oracle(orc, mode, passes, pinned):
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    m, n = 20011, 48
    A, _, s0, _ = workloads.known_spectrum(m, n, workloads.sigma_geometric(n, 1e-7), 31)
    Ah = torch.as_tensor(A)
    if pinned:
        Ah = Ah.pin_memory()
    U, S, V, info = pkg.ts_svd_host(Ah, passes=passes, drop_tol=0.0, mode=mode)
    assert not U.is_cuda and info["rank"] == n
    Ur, Sr, Vr, rr, st = orc.ts_svd(A, drop_tol=0.0)
    U, S, V = U.numpy(), S.numpy(), V.numpy()
    assert np.abs(S - Sr).max() <= 1e-11 * Sr[0]
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-12
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-12
    assert np.abs(A @ V - U * S).max() <= 1e-10 * Sr[0]


@gpu
@pytest.mark.parametrize("m", [100000, 100003])
def test_host_call_several_chunks(m):
    """n = 1000: chunks of 33,536 rows (about 256 MB), the last one ragged
    for m = 100,003; the same SVD as the device call to the FP64-accurate
    tolerances, and the known spectrum."""
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    n = 1000
    sig = workloads.sigma_geometric(n, 1e-6)
    A, _, s0, _ = workloads.known_spectrum_torch(m, n, sig, 32, torch.device("cuda", 0))
    Ah = A.cpu().pin_memory()
    U, S, V, info = pkg.ts_svd_host(Ah, drop_tol=0.0, mode="fp64_tc")
    U1, S1, V1, i1 = pkg.ts_svd(A, drop_tol=0.0, mode="fp64_tc")
    assert info["rank"] == i1["rank"] == n
    s0 = torch.as_tensor(s0).cpu()
    assert (S - s0).abs().max() <= 1e-11 * s0[0]
    assert (S - S1.cpu()).abs().max() <= 1e-12 * s0[0]
    Ud, Vd, Sd = U.cuda(), V.cuda(), S.cuda()
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert (Ud.T @ Ud - eye).abs().max() <= 1e-12
    assert (Vd.T @ Vd - eye).abs().max() <= 1e-12
    assert (A @ Vd - Ud * Sd).abs().max() <= 1e-10 * s0[0]
    # the two calls' singular vectors agree column by column up to sign
    # where the spectrum is well separated (geometric: gaps about 1.4% of
    # each value)
    dots = (Vd * V1).sum(0).abs()
    assert (1.0 - dots).abs().max() <= 1e-8


@gpu
def test_host_call_rejects_bad_arguments():
    torch = _torch()
    import paper_1612_08709_gb300 as pkg
    with pytest.raises(pkg.TsSvdError):
        pkg.ts_svd_host(torch.zeros((10, 20), dtype=torch.float64))  # m < n
    with pytest.raises(pkg.TsSvdError):
        pkg.ts_svd_host(torch.zeros((10, 2), dtype=torch.float32))
