"""ts_gram_noalloc (the Gram step for callers that cannot let the library
allocate device memory) against the allocating ts_gram, through the C ABI,
and against the FP64 CPU oracle's Gram matrix (an independent check: ts_gram
runs the same kernels).

Two calls in a row with different shapes, so the second call must not be
affected by what the first left in the shared fixed scratch.  Same
tolerance as the other Gram parity tests (1e-13 relative to max |B|).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest


@pytest.mark.gpu
def test_gram_noalloc_matches_allocating_gram_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1612_08709_gb300 as pkg
    from paper_1612_08709_gb300._binding import _Opts

    L = pkg.lib()
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.ts_gram_noalloc.argtypes = [vp, i64, i64, i64, vp, vp]
    L.ts_gram_noalloc.restype = ctypes.c_int
    stream = torch.cuda.current_stream()

    for (m, n, seed) in [(30011, 300, 1), (4099, 61, 2)]:
        A = torch.as_tensor(np.random.default_rng(seed).standard_normal((m, n)), device="cuda")
        B_ref = torch.empty((n, n), dtype=torch.float64, device="cuda")
        B_na = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        o = _Opts()
        L.tssvd_default_opts(ctypes.byref(o))
        o.stream = vp(stream.cuda_stream)
        assert L.ts_gram(vp(A.data_ptr()), m, n, n, vp(B_ref.data_ptr()), ctypes.byref(o)) == 0
        rc = L.ts_gram_noalloc(vp(A.data_ptr()), m, n, n, vp(B_na.data_ptr()),
                               vp(stream.cuda_stream))
        assert rc == 0
        ref = B_ref.cpu().numpy()
        got = B_na.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
        import oracle
        want = oracle.gram(A.cpu().numpy())
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max()

    # sizes beyond the fixed scratch are rejected before any work
    A = torch.zeros((800, 725), dtype=torch.float64, device="cuda")
    B = torch.zeros((725, 725), dtype=torch.float64, device="cuda")
    assert L.ts_gram_noalloc(vp(A.data_ptr()), 800, 725, 725, vp(B.data_ptr()),
                             vp(stream.cuda_stream)) == -3
