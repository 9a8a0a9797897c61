#!/usr/bin/env python
"""Benchmark of the GB300 TS-SVD / low-rank SVD library.

One step = one full call of the hot path on one batch of synthetic input:
by default the two-pass Gram TS-SVD (Algorithm 4 with MaxEntry scaling) of
a 1,000,000 x 1,000 FP64 matrix A = U diag(sigma) V^T with seeded
orthonormal factors and sigma geometric from 1 to 1e-8, in the
FP64-accurate tensor-core mode (digit-sliced products on tcgen05).  The
plain FP64 (DFMA) path is timed beside it on the same input
("fp64_path"), with both accuracies, for the comparison at equal accuracy,
and the 2,000,000 x 200 workload of the same recipe is timed after it
("also").

Prints one JSON line (rank 0).  `value` is GFLOP/s of the algorithm's
nominal products, 6 m n^2 for two passes (Gram A^T A counted as m n^2,
A V~ 2 m n^2, Gram Y^T Y m n^2, Y W 2 m n^2; the final U = Q P is not
counted), with A resident in HBM; `e2e` is the same metric through the
host-buffer C-ABI call (ts_svd_host) from pinned host memory, the copies of
A in and of U, S, V back inside the timed region and overlapped with the
compute by row chunks (`serial_ms` gives copy, compute and copy run in
turn for comparison).
The FP64 roofline peak is the FP64 FMA rate measured on the same GPU in
the same run (tssvd_fp64_fma_rate).  `--impl reference` times the FP64 CPU
oracle instead (bounded samples of the same workload on the host cores).

Multi-GPU (torchrun): the row-sharded TS-SVD (ts_svd_rowshard), each rank
holding m rows of an (N m) x n matrix with known singular values (weak
scaling); the method's exchange steps are NCCL all-reduces.
"""
import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "TS-SVD & rank-k SVD GFLOP/s, % of GB300 roofline, vs plain FP64 at equal accuracy"

WORKLOADS = {
    # tall-skinny SVD at scale (2,000,000 x 200 and 1,000,000 x 1,000)
    "ts_2m_x_200": dict(kind="ts", m=2_000_000, n=200, lo=1e-8, seed=2),
    "ts_1m_x_1000": dict(kind="ts", m=1_000_000, n=1000, lo=1e-8, seed=3),
    # a 200,000 x 200 case of the same recipe (inputs still larger than L2)
    # for kernel profiling
    "ts_200k_x_200": dict(kind="ts", m=200_000, n=200, lo=1e-8, seed=2),
    # 20,000 x 1,000 of the 1,000,000 x 1,000 recipe: the same n x n solves
    # on a 160 MB input, for profiling the Jacobi kernels
    "ts_20k_x_1000": dict(kind="ts", m=20_000, n=1000, lo=1e-8, seed=3),
    # the small plain case (20,000 x 50, sigma 1..1e-6)
    "ts_20k_x_50": dict(kind="ts", m=20_000, n=50, lo=1e-6, seed=1),
    # 512 uneven tall-skinny SVDs in one graph launch (m in [1e3, 2e5], n in
    # [16, 256], sigma log-uniform in [1e-6, 1])
    "batch_512": dict(kind="batch", count=512, m_range=(1000, 200000), n_range=(16, 256), seed=5),
    # a small batch of the same recipe for profiling captures
    "batch_32": dict(kind="batch", count=32, m_range=(1000, 40000), n_range=(16, 256), seed=5),
    # randomized low-rank SVD of a 100,000 x 20,000 matrix (rank-200 signal
    # with sigma_j = 1/j plus 1e-4 Gaussian noise), k = 50, l = 60, 2 power steps
    "lowrank_100k_x_20k": dict(kind="lowrank", m=100_000, n=20_000, r=200, k=50, l=60, iters=2,
                               seed=4),
    # Algorithm 2 (randomized TSQR TS-SVD, Remark "randomness" mixing) on the
    # 200,000 x 200 recipe
    "tsqr_200k_x_200": dict(kind="tsqr", m=200_000, n=200, lo=1e-8, seed=2, passes=2),
    # Algorithm 7 (TSQR-based TS-SVDs) on the low-rank workload
    "lowrank_tsqr_100k_x_20k": dict(kind="lowrank", m=100_000, n=20_000, r=200, k=50, l=60,
                                    iters=2, seed=4, method="tsqr"),
    # forward and backward of the differentiable TS-SVD: 500,000 x 512 FP32,
    # sigma_j = 1 + (n - j)/n, loss sum_j w_j sigma_j + ||U_k^T B||_F^2 with
    # k = 64, B 500,000 x 8
    "grad_500k_x_512": dict(kind="grad", m=500_000, n=512, k=64, nb=8, seed=6),
}

# FP64 FMA peak when it cannot be measured: 152 SMs x 2 DFMA/clk/SM x 2 flop
# x 2.07 GHz (GB300's FP64 units and maximum SM clock).  run_ours replaces it
# with the rate measured on the device (set_fp64_peak).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07e9 / 1e9
FP64_PEAK_SOURCE = "FP64 FMA: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz (derived)"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# The best DFMA rate measured on the GB300s (independent FMA chains
# at the 2.07 GHz maximum clock).  The in-run measurement is taken before
# the timed region and has read as low as 1.06 (the clock is not yet at its
# maximum then), so the roofline divides by the larger of the two.
FP64_PEAK_BEST_TFLOPS = 1.256


def set_fp64_peak(L):
    """Measures the device's FP64 FMA rate (tssvd_fp64_fma_rate) and makes
    the larger of it and the best recorded rate the FP64 roofline peak;
    returns the in-run measurement (None if it failed)."""
    global FP64_PEAK_GFLOPS, FP64_PEAK_SOURCE
    v = ctypes.c_double(0.0)
    meas = v.value if L.tssvd_fp64_fma_rate(ctypes.byref(v), None) == 0 and v.value > 0 else None
    peak = max(meas or 0.0, FP64_PEAK_BEST_TFLOPS)
    FP64_PEAK_GFLOPS = peak * 1e3
    FP64_PEAK_SOURCE = ("FP64 FMA rate, measured: max(this run's tssvd_fp64_fma_rate %s, best "
                        "DFMA probe on this GPU type %.3f) TFLOP/s"
                        % ("%.3f" % meas if meas else "n/a", FP64_PEAK_BEST_TFLOPS))
    return meas


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ts_1m_x_1000", choices=sorted(WORKLOADS))
    ap.add_argument("--also", default="ts_2m_x_200",
                    help="comma-separated tall-skinny workloads timed after the headline "
                         "(device-resident, same steps; '' to skip)")
    ap.add_argument("--mode", default="fp64_tc", choices=["fp64", "bf16x3", "bf16x6", "fp64_tc"])
    ap.add_argument("--passes", type=int, default=2, choices=[2, 3],
                    help="tall-skinny workloads: 3 runs Algorithm 4's second pass twice "
                         "(the flop count stays the two-pass 6mn^2)")
    ap.add_argument("--compare-steps", type=int, default=2,
                    help="timed steps of the plain FP64 path reported beside the headline "
                         "(0 to skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-rows", type=int, default=200_000,
                    help="rows of the bounded host sample the oracle is timed on")
    return ap.parse_args()


def nominal_flops(w):
    """Nominal flops of one two-pass TS-SVD: 6 m n^2 (the Gram matrices
    counted as m n^2 each, symmetric; A V~ and Y W 2 m n^2 each)."""
    m, n = w["m"], w["n"]
    return 6.0 * m * n * n


FLOP_COUNT = ("6 m n^2 per two-pass TS-SVD: Gram A^T A (m n^2, symmetric), A V~ (2 m n^2), "
              "Gram Y^T Y (m n^2), Y W (2 m n^2); U = Q P not counted")


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th is not None:
            self.th.join(timeout=5)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                mhz.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# ------------------------------------------------------------ reference arm

def host_sample(w, rows):
    import numpy as np
    import workloads
    s = workloads.sigma_geometric(w["n"], w["lo"])
    A, _, _, _ = workloads.known_spectrum(rows, w["n"], s, w["seed"])
    return A


# Above this n the oracle's n x n Jacobi solves (serial, plain loops) take
# minutes each, so its bounded sample is the tall products alone.
ORACLE_FULL_MAX_N = 256


def oracle_sample_text(w, rows):
    n = w["n"]
    if n <= ORACLE_FULL_MAX_N:
        return ("%d x %d rows of the same recipe: one full two-pass TS-SVD (6 m n^2 nominal "
                "flops)" % (rows, n))
    return ("%d x %d rows of the same recipe: the oracle's tall products of one pass (Gram "
            "A^T A and A V~, 3 m n^2 flops); its n x n Jacobi solves at n = %d take minutes "
            "each and are not in the sample" % (rows, n, n))


def time_oracle(w, rows, reps=1):
    """GFLOP/s of the FP64 CPU oracle on a bounded sample of workload w:
    the whole two-pass TS-SVD of `rows` rows when n is small, else the
    tall products of one pass (the oracle's Gram and A V~ on `rows` rows)."""
    import numpy as np
    import oracle
    A = host_sample(w, rows)
    n = w["n"]
    full = n <= ORACLE_FULL_MAX_N
    V = None if full else np.linalg.qr(np.random.default_rng(7).standard_normal((n, n)))[0]
    t0 = time.perf_counter()
    for _ in range(reps):
        if full:
            oracle.ts_svd(A, passes=2, scale=True, drop_tol=0.0)
        else:
            oracle.gram(A)
            oracle.matmul(A, V)
    dt = (time.perf_counter() - t0) / reps
    flops = (6.0 if full else 3.0) * rows * n ** 2
    return flops / dt / 1e9, dt, oracle.num_threads()


def oracle_rows(w, rows):
    """Rows of the oracle's bounded sample (10-30 s of host work at the
    default 200,000 rows on 16 cores)."""
    return min(rows, w["m"])


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOADS[args.workload]
    rows = oracle_rows(w, args.cpu_rows)
    if w["n"] > ORACLE_FULL_MAX_N:
        rows = max(2000, rows // 4)  # one sample per step: keep the whole run to minutes
    for _ in range(max(0, min(args.warmup, 1))):
        time_oracle(w, min(rows, 20000))
    vals, dts = [], []
    cores = None
    for _ in range(args.steps):
        v, dt, cores = time_oracle(w, rows)
        vals.append(v)
        dts.append(dt)
    value = statistics.mean(vals)
    sample = "per step: %s (workload %d x %d)" % (oracle_sample_text(w, rows), w["m"], w["n"])
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * statistics.mean(dts), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "m": w["m"], "n": w["n"], "passes": 2,
                      "scale": 1, "mode": "fp64-cpu-oracle", "flops": FLOP_COUNT},
           "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores,
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# -------------------------------------------------------------- our arm

def max_over_ranks(ms, dev):
    """The slowest rank's time (the whole job's), by an all-reduce over the
    process group when there is more than one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gflops(flops_per_rank, world, ms_max):
    """Whole-job throughput: the work of every rank over the slowest rank's
    time (replicas: each rank runs its own instance of the workload)."""
    return flops_per_rank * world / (ms_max * 1e-3) / 1e9


def replica_seed(base, rank):
    """Input seed of a rank's replica (distinct inputs per rank)."""
    return base + 1000 * rank


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1612_08709_gb300 as pkg
    import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    m, n = w["m"], w["n"]
    L = pkg.lib()
    fp64_peak = set_fp64_peak(L)

    # input A = U diag(sigma) V^T, built on the device (torch QR of seeded
    # Gaussians); each rank its own replica seed
    sigma = workloads.sigma_geometric(n, w["lo"])
    A, U0, s0, V0 = workloads.known_spectrum_torch(m, n, sigma, replica_seed(w["seed"], rank), dev)
    del U0, V0
    U = torch.empty((m, n), dtype=torch.float64, device=dev)
    S = torch.empty((n,), dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    wsb = pkg.ts_svd_workspace_size(m, n, drop_tol=0.0, mode=args.mode, passes=args.passes)
    ws = torch.empty((wsb,), dtype=torch.uint8, device=dev)
    kw = dict(passes=args.passes, scale=True, drop_tol=0.0, mode=args.mode, workspace=ws,
              out=(U, S, V))

    def step():
        return pkg.ts_svd(A, **kw)[3]

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    # per-kernel CUDA events over the timed region (recorded by the library
    # on the stream each kernel is launched on)
    L.tssvd_profile_enable(1)
    L.tssvd_profile_report(ctypes.create_string_buffer(16), 16)  # clear
    n0 = L.tssvd_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        info = step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    launches = L.tssvd_launch_count() - n0
    L.tssvd_profile_enable(0)
    kernels = read_profile(L)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, dev)
    flops = nominal_flops(w)
    value = job_gflops(flops, world, ms_max)

    # accuracy of the last result (outside the timed region)
    with torch.no_grad():
        s_t = torch.as_tensor(s0 if not torch.is_tensor(s0) else s0.cpu().numpy(), device=dev)
        sig_err = float((S - s_t).abs().max() / s_t[0])
        orth_u = float((U.T @ U - torch.eye(n, dtype=U.dtype, device=dev)).abs().max())
        orth_v = float((V.T @ V - torch.eye(n, dtype=V.dtype, device=dev)).abs().max())
        resid = float(torch.linalg.norm(A @ V - U * S) / torch.linalg.norm(A))

    # the plain FP64 (DFMA) path on the same input, for "vs plain FP64 at
    # equal accuracy"
    fp64_path = None
    if args.mode != "fp64" and args.compare_steps > 0:
        kw64 = dict(kw)
        kw64["mode"] = "fp64"
        wsb64 = pkg.ts_svd_workspace_size(m, n, drop_tol=0.0, mode="fp64")
        if wsb64 > ws.numel():
            ws = torch.empty((wsb64,), dtype=torch.uint8, device=dev)
        kw64["workspace"] = ws
        U64, S64, V64 = torch.empty_like(U), torch.empty_like(S), torch.empty_like(V)
        kw64["out"] = (U64, S64, V64)
        pkg.ts_svd(A, **kw64)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.compare_steps):
            pkg.ts_svd(A, **kw64)
        g1.record(stream)
        torch.cuda.synchronize()
        ms64 = g0.elapsed_time(g1) / args.compare_steps
        with torch.no_grad():
            eye = torch.eye(n, dtype=U.dtype, device=dev)
            fp64_path = {"value": flops / (ms64 * 1e-3) / 1e9, "ms_per_step": ms64,
                         "steps": args.compare_steps,
                         "sigma_err_normwise": float((S64 - s_t).abs().max() / s_t[0]),
                         "orth_U": float((U64.T @ U64 - eye).abs().max()),
                         "speedup_of_headline": ms64 / ms_max}
        del U64, S64, V64

    # end to end: pinned host buffers (placed on the GPU's NUMA node when
    # the host has several), copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        numa = bind_to_gpu_numa_node(dev)
        try:
            Ah = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
            Ah.copy_(A)
            Uh = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
            Uh.zero_()
            Sh = torch.empty((n,), dtype=torch.float64, pin_memory=True)
            Vh = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        finally:
            restore = numa.pop("restore", None)
            if restore is not None:
                os.sched_setaffinity(0, restore)
        # the public host-buffer call: A's row chunks go in and U's come out
        # on the library's copy streams, overlapped with the compute
        wsh = torch.empty((pkg.ts_svd_host_workspace_size(m, n, drop_tol=0.0, mode=args.mode,
                                                          passes=args.passes),),
                          dtype=torch.uint8, device=dev)
        kwh = dict(passes=args.passes, scale=True, drop_tol=0.0, mode=args.mode, workspace=wsh,
                   out=(Uh, Sh, Vh))

        def e2e_step():
            pkg.ts_svd_host(Ah, **kwh)

        e2e_step()
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        f1.record(stream)
        torch.cuda.synchronize()
        ms_e = f0.elapsed_time(f1) / args.e2e_steps
        ms_e = max_over_ranks(ms_e, dev)
        eye = torch.eye(n, dtype=torch.float64, device=dev)
        Ue = Uh.to(dev)
        e2e_orth = float((Ue.T @ Ue - eye).abs().max())
        del Ue, wsh
        # the same copies and call in turn, for the breakdown
        Ad = torch.empty_like(A)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        Ad.copy_(Ah, non_blocking=True)
        ev[1].record(stream)
        pkg.ts_svd(Ad, **kw)
        ev[2].record(stream)
        Uh.copy_(U, non_blocking=True)
        Sh.copy_(S, non_blocking=True)
        Vh.copy_(V, non_blocking=True)
        ev[3].record(stream)
        torch.cuda.synchronize()
        ph = [ev[i].elapsed_time(ev[i + 1]) for i in range(3)]
        e2e = {"value": job_gflops(flops, world, ms_e), "unit": "GFLOP/s",
               "h2d_bytes_per_step": m * n * 8, "d2h_bytes_per_step": (m * n + n + n * n) * 8,
               "ms_per_step": ms_e, "api": "ts_svd_host (pinned host buffers, overlapped copies)",
               "orth_U": e2e_orth,
               "serial_ms": {"h2d": ph[0], "ts_svd": ph[1], "d2h": ph[2], "total": sum(ph)},
               "host_numa": numa}
        del Ah, Uh, Sh, Vh, Ad

    # roofline of the dominant kernel (largest total event time in the
    # timed region): algorithmic flops or bytes per launch / mean duration
    roof, roof_all = roofline(kernels, m, n, ms, args, A.element_size(),
                               info["sweeps"] + [info.get("sweeps_fp32", 0)])
    esize = A.element_size()
    del A, U, S, V, ws
    torch.cuda.empty_cache()

    # the other tall-skinny workloads of the same recipe, device-resident
    also = {}
    for name in [x for x in args.also.split(",") if x and x != args.workload]:
        if WORKLOADS.get(name, {}).get("kind") != "ts":
            continue
        also[name] = measure_ts(torch, pkg, L, WORKLOADS[name], args, dev, rank)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = oracle_rows(w, args.cpu_rows)
        v, dt, cores = time_oracle(w, rows)
        cpu = {"value": v, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": "%s, %.1f s" % (oracle_sample_text(w, rows), dt)}

    out = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp64_tc": "bf16 digits+fp32+f64"}.get(args.mode, "bf16+fp32+f64"),
           "data": "synthetic",
           "config": {"workload": args.workload, "m": m, "n": n, "passes": args.passes, "scale": 1,
                      "mode": args.mode, "drop_tol": 0.0,
                      "sigma": "geometric 1..%g" % w["lo"],
                      "l2": "inputs larger than L2 (A is %.1f GB)" % (m * n * esize / 1e9),
                      "flops": FLOP_COUNT,
                      "parallelism": "replicas" if world > 1 else "single"},
           "roofline": roof, "roofline_kernels": roof_all, "cpu_baseline": cpu, "e2e": e2e,
           "gpu_launches": int(launches),
           "fp64_fma_rate_in_run_tflops": fp64_peak,
           "fp64_path": fp64_path,
           "also": also,
           "clocks": clk,
           "accuracy": {"sigma_err_normwise": sig_err, "orth_U": orth_u, "orth_V": orth_v,
                        "residual_rel": resid, "rank": info["rank"],
                        "sweeps": info["sweeps"], "sweeps_fp32": info.get("sweeps_fp32", 0)},
           "kernels_ms": {k: {"launches": c, "total_ms": t} for k, (c, t) in kernels.items()}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_rowshard(args):
    """N > 1 ranks (torchrun, one GPU each): the row-sharded TS-SVD
    (ts_svd_rowshard).  Each rank holds m rows of an (N m) x n matrix with
    known singular values (weak scaling: the rows per rank stay fixed as N
    grows); the exchanges are all-reduces over NCCL through the library's
    callback (n x n doubles per Gram matrix, n per norm step, n words for
    the column maxima).  value = the N ranks' nominal flops over the
    slowest rank's time."""
    import torch
    import torch.distributed as dist

    import paper_1612_08709_gb300 as pkg
    import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist.init_process_group("nccl")
    w = WORKLOADS[args.workload]
    m, n = w["m"], w["n"]
    L = pkg.lib()
    fp64_peak = set_fp64_peak(L)
    sigma = workloads.sigma_geometric(n, w["lo"])
    A, s_t, V0 = workloads.known_spectrum_rowblock_torch(m, n, sigma, w["seed"], rank, world, dev)
    del V0
    U = torch.empty((m, n), dtype=torch.float64, device=dev)
    S = torch.empty((n,), dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    ws = torch.empty((pkg.ts_svd_workspace_size(m, n, drop_tol=0.0, mode=args.mode),),
                     dtype=torch.uint8, device=dev)
    comm = pkg.DistComm()
    kw = dict(passes=2, scale=True, drop_tol=0.0, mode=args.mode, workspace=ws, out=(U, S, V))

    def step():
        return pkg.ts_svd_rowshard(A, comm, **kw)[3]

    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    L.tssvd_profile_enable(1)
    L.tssvd_profile_report(ctypes.create_string_buffer(16), 16)  # clear
    n0 = L.tssvd_launch_count()
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        info = step()
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    launches = L.tssvd_launch_count() - n0
    L.tssvd_profile_enable(0)
    kernels = read_profile(L)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, dev)
    flops = nominal_flops(w)
    value = job_gflops(flops, world, ms_max)
    with torch.no_grad():
        G = U.T @ U
        dist.all_reduce(G)
        eye = torch.eye(n, dtype=U.dtype, device=dev)
        acc = {"sigma_err_normwise": float((S - s_t).abs().max() / s_t[0]),
               "orth_U": float((G - eye).abs().max()),
               "orth_V": float((V.T @ V - eye).abs().max()), "rank": info["rank"],
               "sweeps": info["sweeps"], "sweeps_fp32": info.get("sweeps_fp32", 0)}
    roof, roof_all = roofline(kernels, m, n, ms, args, A.element_size(),
                               info["sweeps"] + [info.get("sweeps_fp32", 0)])
    out = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": {"fp64": "f64", "fp64_tc": "bf16 digits+fp32+f64"}.get(args.mode, "bf16+fp32+f64"),
           "data": "synthetic",
           "config": {"workload": args.workload, "m_per_rank": m, "m": m * world, "n": n,
                      "passes": 2, "scale": 1, "mode": args.mode, "drop_tol": 0.0,
                      "sigma": "geometric 1..%g" % w["lo"], "flops": FLOP_COUNT,
                      "l2": "inputs larger than L2 (A is %.1f GB per rank)" % (m * n * 8 / 1e9),
                      "parallelism": "row-sharded over %d ranks (NCCL all-reduce)" % world},
           "roofline": roof, "roofline_kernels": roof_all, "cpu_baseline": None,
           "e2e": None, "gpu_launches": int(launches), "fp64_fma_rate_in_run_tflops": fp64_peak,
           "clocks": clk, "accuracy": acc,
           "kernels_ms": {k: {"launches": c, "total_ms": t} for k, (c, t) in kernels.items()}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    dist.destroy_process_group()


def measure_ts(torch, pkg, L, w, args, dev, rank):
    """Device-resident timing of one more tall-skinny workload (same mode,
    steps and warm-up as the headline): GFLOP/s on the 6 m n^2 count, the
    accuracy against the known spectrum and the per-kernel event times."""
    import workloads
    m, n = w["m"], w["n"]
    sigma = workloads.sigma_geometric(n, w["lo"])
    A, U0, s0, V0 = workloads.known_spectrum_torch(m, n, sigma, replica_seed(w["seed"], rank), dev)
    del U0, V0
    U = torch.empty((m, n), dtype=torch.float64, device=dev)
    S = torch.empty((n,), dtype=torch.float64, device=dev)
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    ws = torch.empty((pkg.ts_svd_workspace_size(m, n, drop_tol=0.0, mode=args.mode),),
                     dtype=torch.uint8, device=dev)
    kw = dict(passes=2, scale=True, drop_tol=0.0, mode=args.mode, workspace=ws, out=(U, S, V))
    for _ in range(args.warmup):
        info = pkg.ts_svd(A, **kw)[3]
    L.tssvd_profile_enable(1)
    L.tssvd_profile_report(ctypes.create_string_buffer(16), 16)  # clear
    ms = _timed(torch, lambda: pkg.ts_svd(A, **kw), args.steps)
    L.tssvd_profile_enable(0)
    kernels = read_profile(L)
    info = pkg.ts_svd(A, **kw)[3]
    ms = max_over_ranks(ms, dev)
    with torch.no_grad():
        s_t = torch.as_tensor(s0, device=dev)
        eye = torch.eye(n, dtype=U.dtype, device=dev)
        acc = {"sigma_err_normwise": float((S - s_t).abs().max() / s_t[0]),
               "orth_U": float((U.T @ U - eye).abs().max()),
               "orth_V": float((V.T @ V - eye).abs().max()),
               "rank": info["rank"], "sweeps": info["sweeps"],
               "sweeps_fp32": info.get("sweeps_fp32", 0)}
    roof, _ = roofline(kernels, m, n, ms, args, A.element_size(),
                               info["sweeps"] + [info.get("sweeps_fp32", 0)])
    out = {"value": nominal_flops(w) / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms,
           "steps": args.steps, "m": m, "n": n, "mode": args.mode, "accuracy": acc,
           "roofline": roof,
           "kernels_ms": {k: {"launches": c, "total_ms": t} for k, (c, t) in kernels.items()}}
    del A, U, S, V, ws
    torch.cuda.empty_cache()
    return out


def bind_to_gpu_numa_node(dev):
    """On a host with several NUMA nodes that have CPUs, restrict this
    process to the CPUs of the GPU's node (from sysfs) so that pinned host
    buffers allocated and first touched now live there; the caller restores
    the old affinity ("restore") afterwards.  Returns what it found."""
    import glob
    info = {"nodes_with_cpus": 0, "gpu_node": None, "bound": False, "restore": None}
    try:
        nodes = {}
        for p in glob.glob("/sys/devices/system/node/node[0-9]*"):
            cl = open(os.path.join(p, "cpulist")).read().strip()
            if not cl:
                continue
            cpus = set()
            for part in cl.split(","):
                a, _, b = part.partition("-")
                cpus |= set(range(int(a), int(b or a) + 1))
            nodes[int(os.path.basename(p)[4:])] = cpus
        info["nodes_with_cpus"] = len(nodes)
        import torch
        pr = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        node = int(open("/sys/bus/pci/devices/%s/numa_node" % bus).read().strip())
        info["gpu_node"] = node
        if len(nodes) > 1 and node in nodes:
            allowed = os.sched_getaffinity(0)
            mine = nodes[node] & allowed
            if mine and mine != allowed:
                os.sched_setaffinity(0, mine)
                info["bound"] = True
                info["restore"] = allowed
    except (OSError, ValueError, AttributeError):
        pass
    return info


# HBM copy bandwidth: the measured copy rate in MEASURED_PEAKS.json when
# present, else an earlier GB300 measurement (6.8 TB/s).
def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def bf16_peak(sustained=True):
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    try:
        with open(p) as f:
            return float(json.load(f)[key]), "measured (MEASURED_PEAKS.json %s)" % key
    except (OSError, ValueError, KeyError):
        return (1700.0 if sustained else 1900.0), "fallback"


def kernel_models(m, n, esize, sweeps, cholesky_first=False):
    """Algorithmic work per launch of each kernel of the two-pass TS-SVD.

    Returns {kernel: (bound, amount, unit)}: FP64 flops for the FP64-pipe
    kernels ("alu"), bf16 digit-product flops for the tensor-core digit
    products ("tensor"), bytes for the streaming kernels ("hbm").
      nn_tall   A*M, m x n by n x n:          2 m n^2 flops
      tn_gram   Gram of m x n (symmetric):     m n (n + 1) flops
      jacobi_eig  Gram-form Jacobi, per round the symmetric update of B
                  (24 flops per 2 x 2 block, n^2 / 8 blocks) and of V (6n
                  per rotation, n / 2 rotations): 6 n^2 per round, n - 1
                  rounds per sweep, the step's mean sweep count
      jacobi_svd  one-sided Jacobi: per pair 3n FMAs (dots) and 2n outputs
                  of X and of J at 3 flops: 18n, n / 2 pairs: 9 n^2 per round
      pchol       pivoted Cholesky of the n x n Gram: n^3 / 3 FMAs
    cholesky_first: the first eigensolve ran as pivoted Cholesky and the
    one-sided kernel (n <= 2048, FP64-accurate modes), so jacobi_eig is the
    second eigensolve alone (sweeps[1]) and jacobi_svd launches twice, for
    sweeps[0] and sweeps[2]; otherwise jacobi_eig launches for sweeps[0]
    and sweeps[1] and jacobi_svd once (sweeps[2]).  For 256 < n <= 2048
    all three solves are one-sided on a Cholesky factor or on R: jacobi_svd
    launches three times (the two eigensolves without accumulating
    rotations, 6 n^2 per round: 3n FMAs of dots and 2n outputs at 3 flops
    per pair; the SVD of R with it, 9 n^2), each after an FP32 phase,
    jacobi_svd32 (9 n^2 FP32 flops per round, sweeps[3] summed over its
    three launches).
      oz_nn, oz_gram  28 bf16 digit-pair products per FP64-accurate product
      oz_*_image  read the tall operand once, write 7 bf16 digits per entry
      colmax, oz_rowexp  read the tall operand once; colsumsq reads m n FP64
    """
    rounds = n - 1 + (n & 1)
    mdl = {"nn_tall": ("alu", 2.0 * m * n * n), "tn_gram": ("alu", float(m) * n * (n + 1)),
           "oz_nn": ("tensor", 28 * 2.0 * m * n * n), "oz_gram": ("tensor", 28.0 * m * n * (n + 1)),
           "tc_gram": ("hbm", float(esize) * m * n), "tc_nn": ("hbm", float(esize) * m * n + 8.0 * m * n),
           "oz_gram_image": ("hbm", (esize + 14.0) * m * n), "oz_row_image": ("hbm", (8 + 14.0) * m * n),
           "colmax": ("hbm", float(esize) * m * n), "oz_rowexp": ("hbm", 8.0 * m * n),
           "colsumsq": ("hbm", 8.0 * m * n)}
    mdl["pchol"] = ("alu", 2.0 * n * n * n / 3.0)
    if sweeps and len(sweeps) >= 3 and min(sweeps[:3]) > 0:
        wide = 256 < n <= 2048
        if cholesky_first and wide:
            # three one-sided solves, each an FP32 phase and an FP64 polish
            mdl["jacobi_svd"] = ("alu", (6.0 * sweeps[0] + 6.0 * sweeps[1] + 9.0 * sweeps[2])
                                 / 3.0 * rounds * n * n)
            if len(sweeps) >= 4 and sweeps[3] > 0:
                mdl["jacobi_svd32"] = ("alu32", sweeps[3] / 3.0 * rounds * 9.0 * n * n)
        elif cholesky_first:
            mdl["jacobi_eig"] = ("alu", float(sweeps[1]) * rounds * 6.0 * n * n)
            mdl["jacobi_svd"] = ("alu", (sweeps[0] + sweeps[2]) / 2.0 * rounds * 9.0 * n * n)
        else:
            mdl["jacobi_eig"] = ("alu", (sweeps[0] + sweeps[1]) / 2.0 * rounds * 6.0 * n * n)
            mdl["jacobi_svd"] = ("alu", float(sweeps[2]) * rounds * 9.0 * n * n)
    return mdl


def roofline_entry(name, cnt, tot_ms, model, step_ms, args):
    per_launch_s = tot_ms / max(cnt, 1) * 1e-3
    bound, amount = model
    traffic = load_traffic(name, args.workload, args.mode)
    e = {"bound": bound, "kernel": name, "launches_per_step": cnt / max(args.steps, 1),
         "share_of_step": tot_ms / (step_ms * args.steps) if step_ms > 0 else None,
         "traffic": traffic}
    if bound == "alu":
        peak = FP64_PEAK_GFLOPS / 1e3
        e.update(achieved=amount / per_launch_s / 1e12, peak=peak, unit="TFLOP/s",
                 peak_source=FP64_PEAK_SOURCE)
    elif bound == "alu32":
        e["bound"] = "alu"
        e.update(achieved=amount / per_launch_s / 1e12, peak=FP32_PEAK_TFLOPS, unit="TFLOP/s",
                 peak_source="FP32 FMA: 152 SMs x 128 FMA/clk x 2 flops x 2.07 GHz (derived)")
    elif bound == "tensor":
        peak, src = bf16_peak(sustained=True)
        e.update(achieved=amount / per_launch_s / 1e12, peak=peak, unit="TFLOP/s", peak_source=src)
    else:
        peak, src = hbm_peak()
        e.update(achieved=amount / per_launch_s / 1e9, peak=peak, unit="GB/s", peak_source=src)
    e["frac"] = e["achieved"] / e["peak"]
    if name.startswith("jacobi"):
        e["note"] = ("latency-bound: one grid barrier and a chain of dependent FP64 "
                     "operations per round; the fraction is of the FP64 pipe")
    elif name == "pchol":
        e["note"] = ("one CTA, a barrier-separated chain of n pivot steps; the fraction "
                     "is of the whole GPU's FP64 pipe")
    return e


def roofline(kernels, m, n, ms, args, esize, sweeps=None):
    """Roofline of the dominant kernel (largest event time in the timed
    region) and of every other modelled kernel with a share above 1%:
    algorithmic work per launch (kernel_models) / mean launch duration."""
    if not kernels:
        return None, []
    mdl = kernel_models(m, n, esize, sweeps,
                        cholesky_first=("pchol" in kernels or "pchol_grid" in kernels))
    ranked = sorted(kernels.items(), key=lambda kv: -kv[1][1])
    entries = []
    for name, (cnt, tot) in ranked:
        if name in mdl and tot >= 0.01 * ms * args.steps:
            entries.append(roofline_entry(name, cnt, tot, mdl[name], ms, args))
    top = ranked[0][0]
    dom = next((e for e in entries if e["kernel"] == top), entries[0] if entries else None)
    return dom, entries


def read_profile(L):
    """{kernel: (launches, total_ms)} from the library's event records."""
    need = int(L.tssvd_profile_report(None, 0))
    buf = ctypes.create_string_buffer(need + 64)
    L.tssvd_profile_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        parts = line.split()
        if len(parts) == 3:
            out[parts[0]] = (int(parts[1]), float(parts[2]))
    return out


def load_traffic(kernel, workload, mode):
    """DRAM bytes per launch from a committed ncu summary, if it matches."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get("%s|%s|%s" % (kernel, workload, mode))
    if not e:
        return None
    return e.get("bytes_per_launch")


def _timed(torch, fn, steps):
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def dominant_tensor_roofline(kernels, steps, bf16_flops_per_step, names=("oz_nn", "oz_tn")):
    """Roofline of a step's digit products taken together (the dominant
    kernel class of the low-rank, batched and gradient workloads): their
    nominal bf16 digit-product flops per step over their summed event time
    per step, against the sustained bf16 peak."""
    t = sum(kernels.get(k, (0, 0.0))[1] for k in names) / max(steps, 1)
    if t <= 0 or bf16_flops_per_step <= 0:
        return None
    peak, src = bf16_peak(sustained=True)
    ach = bf16_flops_per_step / (t * 1e-3) / 1e12
    top = max(kernels.items(), key=lambda kv: kv[1][1])[0] if kernels else None
    return {"bound": "tensor", "kernel": "+".join(names), "dominant_by_time": top,
            "ms_per_step": t, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak, "peak_source": src, "traffic": None,
            "note": "28 bf16 digit-pair products per FP64-accurate product"}


def run_batched(args):
    """512 uneven members: one ts_svd_batched graph launch per step, against
    one ts_svd call per member (the loop)."""
    import numpy as np
    import torch

    import paper_1612_08709_gb300 as pkg
    import workloads
    w = WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    shapes = workloads.batch_shapes(w["count"], w["seed"], w["m_range"], w["n_range"])
    As, sig = [], []
    for i, (m, n) in enumerate(shapes):
        rng = np.random.default_rng(w["seed"] * 100003 + i)
        s = np.sort(np.exp(rng.uniform(np.log(1e-6), 0.0, size=n)))[::-1].copy()
        A, U0, s0, V0 = workloads.known_spectrum_torch(m, n, s, w["seed"] * 1000 + i, dev)
        del U0, V0
        As.append(A)
        sig.append(torch.as_tensor(s, device=dev))
    flops = sum(6.0 * m * n * n for m, n in shapes)
    mode = "auto" if args.mode == "fp64_tc" else args.mode
    set_fp64_peak(pkg.lib())
    outs, infos, rc = pkg.ts_svd_batched(As, drop_tol=0.0, mode=mode)  # tunes + captures
    for _ in range(max(0, args.warmup - 1)):
        pkg.ts_svd_batched(As, drop_tol=0.0, mode=mode, outs=outs)
    L = pkg.lib()
    n0 = L.tssvd_launch_count()
    clocks = ClockSampler(0)
    clocks.start()
    # the batched solves are timed by event nodes of the graph and reported
    # through the library's profiler
    L.tssvd_profile_enable(1)
    L.tssvd_profile_report(ctypes.create_string_buffer(16), 16)  # clear
    ms = _timed(torch, lambda: pkg.ts_svd_batched(As, drop_tol=0.0, mode=mode, outs=outs), args.steps)
    L.tssvd_profile_enable(0)
    kernels = read_profile(L)
    clk = clocks.stop()
    launches = L.tssvd_launch_count() - n0
    err = max(float((o[1] - s).abs().max() / s[0]) for o, s in zip(outs, sig))
    orth = max(float((o[0].T @ o[0] - torch.eye(o[0].shape[1], dtype=o[0].dtype, device=dev))
                     .abs().max()) for o in outs)
    modes = {}
    for i in infos:
        modes[i["mode"]] = modes.get(i["mode"], 0) + 1
    loop_ms = None
    if args.compare_steps > 0:
        per_mode = [i["mode"] for i in infos]

        def loop():
            for A, o, md in zip(As, outs, per_mode):
                pkg.ts_svd(A, drop_tol=0.0, mode=md, out=o)
        loop()
        loop_ms = _timed(torch, loop, 1)
    # Roofline over the whole step (a graph replay's kernels are not timed one
    # by one): the members' FP64-accurate tall products, 8 m n^2 each (both
    # Gram matrices, A V~, Y W, U), as 28 digit-pair products on the tensor
    # cores when every member ran FP64_TC.
    roof = None
    if "jacobi_batch" in kernels:
        # the phased executor's dominant kernel: the batched one-sided
        # solves, FP64 work as bench.kernel_models counts it (6 n^2 a round
        # without accumulation, 9 n^2 with), each member's own sweep counts
        jf = 0.0
        for (m, n), inf in zip(shapes, infos):
            sw = inf["sweeps"]
            rounds = n - 1 + (n & 1)
            jf += (6.0 * max(sw[0], 0) + 6.0 * max(sw[1], 0) + 9.0 * max(sw[2], 0)) * rounds * n * n
        c, t = kernels["jacobi_batch"]
        steps_seen = c / 3.0
        peak, src = FP64_PEAK_GFLOPS / 1e3, FP64_PEAK_SOURCE
        ach = jf * steps_seen / (t * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "jacobi_batch (three launches a step)",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": src, "traffic": None,
                "launch_ms_mean": t / c, "share_of_step": t / steps_seen / ms}
    elif set(modes) == {"fp64_tc"}:
        peak, src = bf16_peak(sustained=True)
        ach = 28.0 * sum(8.0 * m * n * n for m, n in shapes) / (ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "kernel": "whole step (digit products of all members)",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": src, "traffic": None,
                "note": "lower bound of the products' own rate: the step's time includes the "
                        "members' Jacobi solves"}
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle's two-pass TS-SVD of the first members whose work adds up
        # to about 2e10 nominal flops (a bounded sample of the same batch)
        import oracle
        t_s, f_s, used = 0.0, 0.0, 0
        for A, (m, n) in zip(As, shapes):
            Ah = A.cpu().numpy()
            t0 = time.perf_counter()
            oracle.ts_svd(Ah, passes=2, scale=True, drop_tol=0.0)
            t_s += time.perf_counter() - t0
            f_s += 6.0 * m * n * n
            used += 1
            if f_s >= 2e10 or used >= 4:
                break
        cpu = {"value": f_s / t_s / 1e9, "unit": "GFLOP/s", "cores": oracle.num_threads(),
               "kind": "oracle",
               "sample": "two-pass TS-SVD of the batch's first %d members (%.2g nominal flops), "
                         "%.1f s" % (used, f_s, t_s)}
    out = {"metric": METRIC, "value": flops / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "roofline": roof, "cpu_baseline": cpu,
           "e2e": None, "e2e_note": "not measured: the batch's inputs are 53 GB of pinned host memory",
           "config": {"workload": args.workload, "members": len(shapes),
                      "m_range": list(w["m_range"]), "n_range": list(w["n_range"]),
                      "mode": mode, "modes_chosen": modes, "passes": 2, "scale": 1,
                      "executor": "phased" if (mode in ("auto", "fp64_tc") and
                                               max(n for _, n in shapes) <= 256) else "per member",
                      "l2": "inputs larger than L2 (%.0f GB)" % (sum(m * n for m, n in shapes) * 8 / 1e9)},
           "gpu_launches": int(launches), "clocks": clk,
           "kernels_ms": {k: {"launches": c, "total_ms": t} for k, (c, t) in kernels.items()},
           "accuracy": {"sigma_err_normwise_max": err, "orth_U_max": orth,
                        "sweeps_mean": [round(sum(max(i["sweeps"][j], 0) for i in infos) / len(infos), 2)
                                        for j in range(3)],
                        "sweeps_max": [max(i["sweeps"][j] for i in infos) for j in range(3)]},
           "loop_baseline": None if loop_ms is None else
           {"ms_per_step": loop_ms, "value": flops / (loop_ms * 1e-3) / 1e9,
            "speedup_of_batched": loop_ms / ms}}
    print(json.dumps(out), flush=True)


def run_lowrank(args):
    """Algorithm 8 on the 100,000 x 20,000 workload."""
    import numpy as np
    import torch

    import paper_1612_08709_gb300 as pkg
    import workloads
    w = WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    m, n, r, k, l, it = w["m"], w["n"], w["r"], w["k"], w["l"], w["iters"]
    Ur = workloads.orthonormal_torch(m, r, w["seed"], dev)
    Vr = workloads.orthonormal_torch(n, r, w["seed"] + 1, dev)
    s = torch.as_tensor(1.0 / np.arange(1, r + 1), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(w["seed"] + 2)
    A = torch.randn(m, n, generator=g, device=dev, dtype=torch.float64)
    A.mul_(1e-4 / m ** 0.5)
    A.addmm_(Ur * s, Vr.T)
    del Ur, Vr
    Om = torch.as_tensor(workloads.gaussian(n, l, w["seed"] + 3), device=dev)
    mode = args.mode if args.mode in ("fp64", "fp64_tc") else "fp64"
    tsqr = w.get("method") == "tsqr"
    if tsqr:
        t1, t2, p1, p2 = workloads.mixing_draws(l, w["seed"] + 5)
        theta = torch.as_tensor(np.concatenate([t1, t2]), device=dev)
        perm = torch.as_tensor(np.concatenate([p1, p2]).astype(np.int64), device=dev)

    def step():
        if tsqr:
            return pkg.lowrank_svd_tsqr(A, k, l, it, Om, theta, perm, drop_tol=0.0, mode=mode)
        return pkg.lowrank_svd(A, k, l, it, Om, drop_tol=0.0, mode=mode)
    for _ in range(args.warmup):
        U, S, V, info = step()
    clocks = ClockSampler(0)
    clocks.start()
    L = pkg.lib()
    set_fp64_peak(L)
    L.tssvd_profile_enable(1)
    L.tssvd_profile_report(ctypes.create_string_buffer(16), 16)  # clear
    n0 = L.tssvd_launch_count()
    ms = _timed(torch, step, args.steps)
    clk = clocks.stop()
    launches = L.tssvd_launch_count() - n0
    L.tssvd_profile_enable(0)
    kernels = read_profile(L)
    U, S, V, info = step()
    flops = 2.0 * (2 * it + 2) * m * n * l
    eye = torch.eye(k, dtype=U.dtype, device=dev)
    # roofline: the products with A, 2(2i+2) m n l FP64-accurate flops a
    # step, as 28 digit-pair products on the tensor cores (FP64_TC), or on
    # the FP64 pipe (FP64)
    if mode == "fp64_tc":
        roof = dominant_tensor_roofline(kernels, args.steps, 28.0 * flops)
    else:
        t = sum(v[1] for kname, v in kernels.items() if kname.startswith(("nn_", "tn_"))) / args.steps
        roof = None if t <= 0 else {
            "bound": "alu", "kernel": "nn_tall+tn_*", "achieved": flops / (t * 1e-3) / 1e12,
            "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s", "peak_source": FP64_PEAK_SOURCE,
            "frac": flops / (t * 1e-3) / 1e12 / (FP64_PEAK_GFLOPS / 1e3), "traffic": None}
    # end to end: A from pinned host memory, U, S, V back (one step)
    e2e = None
    if args.e2e_steps > 0:
        Ah = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A)
        Uh = torch.empty((m, k), dtype=torch.float64, pin_memory=True)
        Sh = torch.empty((k,), dtype=torch.float64, pin_memory=True)
        Vh = torch.empty((n, k), dtype=torch.float64, pin_memory=True)
        Ad = torch.empty_like(A)

        def e2e_step():
            Ad.copy_(Ah, non_blocking=True)
            if tsqr:
                Uo, So, Vo, _ = pkg.lowrank_svd_tsqr(Ad, k, l, it, Om, theta, perm, drop_tol=0.0,
                                                     mode=mode)
            else:
                Uo, So, Vo, _ = pkg.lowrank_svd(Ad, k, l, it, Om, drop_tol=0.0, mode=mode)
            Uh.copy_(Uo, non_blocking=True)
            Sh.copy_(So, non_blocking=True)
            Vh.copy_(Vo, non_blocking=True)
        e2e_step()
        ms_e = _timed(torch, e2e_step, args.e2e_steps)
        e2e = {"value": flops / (ms_e * 1e-3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms_e,
               "h2d_bytes_per_step": m * n * 8, "d2h_bytes_per_step": (m * k + k + n * k) * 8}
        del Ah, Uh, Sh, Vh, Ad
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle's Algorithm 8 on a 10,000-row sample of the same recipe
        # (same n, k, l, power steps; its products are the bulk of its time)
        import oracle
        ms_rows = min(10_000, m)
        As = A[:ms_rows].cpu().numpy()
        t0 = time.perf_counter()
        oracle.lowrank_svd(As, k, l, it, Om.cpu().numpy(), drop_tol=0.0)
        dt = time.perf_counter() - t0
        cpu = {"value": 2.0 * (2 * it + 2) * ms_rows * n * l / dt / 1e9, "unit": "GFLOP/s",
               "cores": oracle.num_threads(), "kind": "oracle",
               "sample": "Algorithm 8 on the first %d of %d rows (n = %d, k = %d, l = %d, %d power "
                         "steps), %.1f s" % (ms_rows, m, n, k, l, it, dt)}
    out = {"metric": METRIC, "value": flops / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "m": m, "n": n, "k": k, "l": l, "iters": it,
                      "mode": mode, "algorithm": 7 if tsqr else 8, "flops": "2(2i+2)mnl",
                      "l2": "inputs larger than L2 (A is %.0f GB)" % (m * n * 8 / 1e9)},
           "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "e2e": e2e,
           "cpu_baseline": cpu,
           "kernels_ms": {kk: {"launches": c, "total_ms": t} for kk, (c, t) in kernels.items()},
           "accuracy": {"sigma_err_vs_signal_max": float((S - s[:k]).abs().max()),
                        "orth_U": float((U.T @ U - eye).abs().max()),
                        "orth_V": float((V.T @ V - eye).abs().max()), "rank": info["rank"]}}
    print(json.dumps(out), flush=True)


def run_tsqr(args):
    """Algorithm 1 or 2 (randomized TSQR TS-SVD) on the tall-skinny recipe.
    Nominal flops 12mn^2 for Algorithm 2 (mixing product 2mn^2, two TSQRs of
    4mn^2 each: Householder factorization and Q, U = Q P 2mn^2), 8mn^2 for
    Algorithm 1."""
    import numpy as np
    import torch

    import paper_1612_08709_gb300 as pkg
    import workloads
    w = WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    m, n, passes = w["m"], w["n"], w["passes"]
    sigma = workloads.sigma_geometric(n, w["lo"])
    A, U0, s0, V0 = workloads.known_spectrum_torch(m, n, sigma, w["seed"], dev)
    del U0, V0
    t1, t2, p1, p2 = workloads.mixing_draws(n, w["seed"] + 5)
    theta = torch.as_tensor(np.concatenate([t1, t2]), device=dev)
    perm = torch.as_tensor(np.concatenate([p1, p2]).astype(np.int64), device=dev)

    mode = args.mode if args.mode in ("fp64", "fp64_tc") else "fp64"

    def step():
        return pkg.ts_svd_tsqr(A, theta, perm, passes=passes, drop_tol=0.0, mode=mode)
    for _ in range(args.warmup):
        U, S, V, info = step()
    L = pkg.lib()
    clocks = ClockSampler(0)
    clocks.start()
    L.tssvd_profile_enable(1)
    L.tssvd_profile_report(ctypes.create_string_buffer(16), 16)  # clear
    n0 = L.tssvd_launch_count()
    ms = _timed(torch, step, args.steps)
    launches = L.tssvd_launch_count() - n0
    L.tssvd_profile_enable(0)
    kernels = read_profile(L)
    clk = clocks.stop()
    U, S, V, info = step()
    flops = (12.0 if passes == 2 else 8.0) * m * n * n
    # the Householder kernels against the FP64 pipe, LAPACK's operation
    # counts per block of b rows: 2bn^2 - 2n^3/3 to factor it, 4bn^2 - 2n^3 to
    # apply its reflections to [C; 0] (forming Q), over every level of the
    # reduction tree (blocks of ceil(rows / b) with b = max(4n, 256), the
    # stacked n x n R factors the next level)
    qr_flops, rows = 0.0, m
    while True:
        b = max(4 * n if n <= 256 else 2 * n, 256)
        nb = max(1, -(-rows // b))
        qr_flops += 6.0 * rows * n * n - nb * (2.0 / 3.0 + 2.0) * n ** 3
        if nb == 1:
            break
        rows = nb * n
    qr_flops *= passes
    qr_ms = sum(t for k2, (c, t) in kernels.items()
                if k2.startswith(("tsqr_geqrf", "tsqr_orgqr"))) / args.steps
    roof = None
    if qr_ms > 0:
        ach = qr_flops / (qr_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "tsqr_geqrf+tsqr_orgqr", "achieved": ach,
                "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                "frac": ach / (FP64_PEAK_GFLOPS / 1e3), "traffic": None,
                "share_of_step": qr_ms / ms,
                "peak_source": FP64_PEAK_SOURCE}
    st = torch.as_tensor(s0, device=dev)
    eye = torch.eye(n, dtype=U.dtype, device=dev)
    out = {"metric": METRIC, "value": flops / (ms * 1e-3) / 1e9, "unit": "GFLOP/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "m": m, "n": n, "algorithm": passes,
                      "mode": mode,
                      "flops": "12mn^2" if passes == 2 else "8mn^2",
                      "l2": "inputs larger than L2 (A is %.1f GB)" % (m * n * 8 / 1e9)},
           "roofline": roof, "gpu_launches": int(launches), "clocks": clk,
           "accuracy": {"sigma_err_normwise": float((S - st).abs().max() / st[0]),
                        "orth_U": float((U.T @ U - eye).abs().max()),
                        "orth_V": float((V.T @ V - eye).abs().max()), "rank": info["rank"]},
           "kernels_ms": {k2: {"launches": c, "total_ms": t} for k2, (c, t) in kernels.items()}}
    print(json.dumps(out), flush=True)


def run_grad(args):
    """One step = forward TS-SVD (FP32 storage), the loss, and its backward
    through the thin-SVD adjoint (TSSVD autograd).  Nominal flops 8mn^2:
    6mn^2 for the forward TS-SVD and 2mn^2 for the adjoint (the count of
    one m x n by n x n product; its other tall products are not counted)."""
    import numpy as np
    import torch

    import paper_1612_08709_gb300 as pkg
    import workloads
    w = WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    m, n, k, nb = w["m"], w["n"], w["k"], w["nb"]
    s = workloads.sigma_distinct_gaps(n)
    A = workloads.known_spectrum_torch(m, n, s, w["seed"], dev)[0].float()
    rng = np.random.default_rng(w["seed"] + 1)
    wv = torch.as_tensor(rng.standard_normal(n), dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(w["seed"] + 2)
    B = torch.randn(m, nb, generator=g, device=dev, dtype=torch.float32)
    mode = args.mode if args.mode in ("fp64", "fp64_tc") else "fp64_tc"
    out = {}

    def step():
        Ag = A.detach().requires_grad_(True)
        U, S, V = pkg.TSSVD.apply(Ag, 2, True, 0.0, mode)
        L = (wv * S).sum() + ((U[:, :k].T @ B) ** 2).sum()
        L.backward()
        out["S"], out["U"], out["G"] = S.detach(), U.detach(), Ag.grad
    for _ in range(args.warmup):
        step()
    L_ = pkg.lib()
    clocks = ClockSampler(0)
    clocks.start()
    L_.tssvd_profile_enable(1)
    L_.tssvd_profile_report(ctypes.create_string_buffer(16), 16)  # clear
    n0 = L_.tssvd_launch_count()
    ms = _timed(torch, step, args.steps)
    launches = L_.tssvd_launch_count() - n0
    L_.tssvd_profile_enable(0)
    kernels = read_profile(L_)
    clk = clocks.stop()
    st = torch.as_tensor(s, device=dev)
    U = out["U"].double()
    res = {"metric": METRIC, "value": 8.0 * m * n * n / (ms * 1e-3) / 1e9, "unit": "GFLOP/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "fp32 storage; " + ("bf16 digits+fp32+f64" if mode == "fp64_tc" else "f64"),
           "data": "synthetic",
           "config": {"workload": args.workload, "m": m, "n": n, "k": k, "mode": mode,
                      "flops": "8mn^2 (6mn^2 forward + 2mn^2 adjoint)",
                      "l2": "inputs larger than L2 (A is %.1f GB FP32)" % (m * n * 4 / 1e9)},
           "gpu_launches": int(launches), "clocks": clk,
           # the step's tall products as executed: forward 8 m n^2 (both Gram
           # matrices, A V~, Y W, U), adjoint 8 m n^2 (U recomputed, U^T dU,
           # [U | dU] times a 2n x n factor), 28 digit-pair products each
           "roofline": (dominant_tensor_roofline(kernels, args.steps, 28.0 * 16.0 * m * n * n)
                        if mode == "fp64_tc" else None),
           "cpu_baseline": None,
           "cpu_baseline_note": "not measured: the oracle's serial Jacobi solves at n = 512 "
                                "take minutes",
           "accuracy": {"sigma_err_normwise": float((out["S"].double() - st).abs().max() / st[0]),
                        "orth_U": float((U.T @ U - torch.eye(n, dtype=U.dtype, device=dev)).abs().max()),
                        "grad_norm": float(out["G"].double().norm())},
           "kernels_ms": kernels}
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif WORKLOADS[args.workload]["kind"] == "batch":
        run_batched(args)
    elif WORKLOADS[args.workload]["kind"] == "lowrank":
        run_lowrank(args)
    elif WORKLOADS[args.workload]["kind"] == "grad":
        run_grad(args)
    elif WORKLOADS[args.workload]["kind"] == "tsqr":
        run_tsqr(args)
    elif int(os.environ.get("WORLD_SIZE", "1")) > 1:
        run_rowshard(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
