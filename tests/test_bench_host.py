"""Host logic of bench.py that needs no GPU: the reference arm's JSON line
(the oracle timed on a bounded sample) and the roofline accounting of the
kernel event totals."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload,sample", [
    (None, "2000 x 1000 rows of the same recipe: the oracle's tall products of one pass"),
    ("ts_2m_x_200", "4000 x 200 rows of the same recipe: one full two-pass TS-SVD")])
def test_reference_arm_json_line(workload, sample):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--steps", "1", "--warmup", "0", "--cpu-rows", "4000"]
    if workload:
        cmd += ["--workload", workload]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["config"]["workload"] == (workload or "ts_1m_x_1000")
    assert d["config"]["flops"].startswith("6 m n^2")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert sample in cb["sample"], cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_roofline_accounting_follows_the_first_eigensolve():
    """With the pivoted Cholesky path the one-sided kernel launches twice a
    step (first eigensolve and small SVD) and the Gram-form one once."""
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps = 2
        workload = "ts_2m_x_200"
        mode = "fp64_tc"

    m, n, sweeps = 2_000_000, 200, [10, 18, 16]
    rounds = n - 1
    kernels = {"jacobi_svd": (4, 40.0), "jacobi_eig": (2, 22.0), "pchol": (2, 6.0),
               "oz_nn": (6, 30.0)}
    dom, allr = bench.roofline(kernels, m, n, 68.0, Args, 8, sweeps)
    assert dom["kernel"] == "jacobi_svd" and dom["launches_per_step"] == 2.0
    flops_svd = (10 + 16) / 2.0 * rounds * 9.0 * n * n
    assert dom["achieved"] == pytest.approx(flops_svd / (10.0e-3) / 1e12)
    eig = next(e for e in allr if e["kernel"] == "jacobi_eig")
    assert eig["achieved"] == pytest.approx(18 * rounds * 6.0 * n * n / (11.0e-3) / 1e12)
    pc = next(e for e in allr if e["kernel"] == "pchol")
    assert pc["achieved"] == pytest.approx(2.0 * n ** 3 / 3.0 / (3.0e-3) / 1e12)
    # without the Cholesky path: both eigensolves on the Gram-form kernel
    kernels2 = {"jacobi_svd": (2, 24.0), "jacobi_eig": (4, 60.0)}
    dom2, _ = bench.roofline(kernels2, m, n, 74.0, Args, 8, [27, 19, 12])
    assert dom2["kernel"] == "jacobi_eig"
    assert dom2["achieved"] == pytest.approx((27 + 19) / 2.0 * rounds * 6.0 * n * n / 15.0e-3 / 1e12)
    for e in allr:
        assert e["frac"] == pytest.approx(e["achieved"] / e["peak"])


def test_roofline_accounting_of_the_wide_two_precision_path():
    """256 < n <= 2048: the FP64 one-sided kernel launches three times
    (first and second eigensolves without accumulation, 6 n^2 a round; SVD
    of R with it, 9 n^2), the FP32 kernel three times (sweeps[3] its summed
    sweeps, 9 n^2 FP32 flops a round against the derived FP32 peak)."""
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps = 1
        workload = "ts_1m_x_1000"
        mode = "fp64_tc"

    m, n = 1_000_000, 1000
    sweeps = [4, 19, 4, 43]
    rounds = n - 1 + (n & 1)
    kernels = {"jacobi_svd": (3, 283.0), "jacobi_svd32": (3, 191.0), "pchol_grid": (2, 17.7),
               "oz_nn": (3, 160.0)}
    mdl = bench.kernel_models(m, n, 8, sweeps, cholesky_first=True)
    assert "jacobi_eig" not in mdl
    dom, allr = bench.roofline(kernels, m, n, 755.0, Args, 8, sweeps)
    assert dom["kernel"] == "jacobi_svd"
    assert dom["achieved"] == pytest.approx((6.0 * 4 + 6.0 * 19 + 9.0 * 4) / 3.0 * rounds * n * n
                                            / (283.0 / 3 * 1e-3) / 1e12)
    f32 = next(e for e in allr if e["kernel"] == "jacobi_svd32")
    assert f32["bound"] == "alu" and f32["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS)
    assert f32["achieved"] == pytest.approx(43 / 3.0 * rounds * 9.0 * n * n
                                            / (191.0 / 3 * 1e-3) / 1e12)
