"""Benchmark of the spin summation on GB300.

One step = one spin summation B = S(A) over the whole workload, FP64:
the 3D CCSDT-shaped tensor A[a,b,c,i,j,k] with a,b,c extent 48 and i,j,k
extent 16 (453M doubles, 3.6 GB), Table II row 1 applied factorized
(B = (2 - pi213)((2 - pi321 - pi132)(A))), out of place, seeded uniform
inputs. Metric: effective HBM bandwidth 2 * N * sizeof(double) / time (the
paper's Eq. 12, in GB/s rather than GiB/s).

Prints one JSON line. `value` is device-timed (CUDA events on the launching
stream, inputs resident); `e2e` times the same call through the public API
with pinned host buffers (H2D of A and D2H of B inside the timed region);
`roofline` relates the kernel to the measured HBM copy bandwidth;
`cpu_baseline` is the oracle (test infrastructure) on a bounded sample of the
same workload on the host cores. `--impl reference` times only that oracle.

Multi-GPU (torchrun, one rank per GPU): every rank runs its own copy of the
workload with no collective on the data path (weak scaling); barriers and a
max over ranks bracket the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "3d-spinsum fp64 A[48,48,48,16,16,16] Table-II-row-1 factorized out-of-place"
SHAPE = (48, 48, 48, 16, 16, 16)
D = 3

# smaller workloads of the same kernels for profiler captures (--case); the
# default case is the benchmark workload above
CASES = {
    "3d": (3, (48, 48, 48, 16, 16, 16), 1),
    "3d-small": (3, (24, 24, 24, 16, 16, 16), 1),     # 453 MB per tensor: above L2, one ncu capture
    "4d": (4, (12,) * 8, 5),
    "4d-small": (4, (8, 8, 8, 8, 12, 12, 12, 12), 5),
    # the paper's own layout: a dense N^d tensor, every index permuted (tiled kernel)
    "paper-3d": (3, (344,) * 3, 1),
    "paper-4d": (4, (80,) * 4, 5),
    # the same at the sizes of the default run's paper-layout lines (one-pass captures only)
    "paper-3d-544": (3, (544,) * 3, 1),
    "paper-4d-112": (4, (112,) * 4, 5),
    # the summation fused into a contraction with W[8, 8^3] (FP64-pipe-bound kernel)
    "contract-small": (3, (48, 48, 48, 8, 8, 8), 1),
}
CONTRACT_Y = 8


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-extra", action="store_true", help="skip the extra per-case lines")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    p.add_argument("--case", default="3d", choices=sorted(CASES),
                   help="workload: the benchmark (3d) or a smaller one for profiler captures")
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def wait_first_sample(self, timeout: float = 10.0):
        """nvidia-smi's start-up can hold the GPU for a while; time nothing
        before its first sample has arrived."""
        t0 = time.time()
        while self.proc and not self.samples and time.time() - t0 < timeout:
            time.sleep(0.05)
        time.sleep(0.2)

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ts, line in self.samples:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((ts, float(parts[1]), float(parts[2]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 - 0.1 <= r[0] <= self.t1 + 0.1]
        if not inside:  # timed region shorter than the sampling interval: nearest samples
            mid = ((self.t0 or 0) + (self.t1 or 0)) / 2
            inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in inside:
            for name, v in zip(names[1:], r[3][1:]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": sorted(reasons), "samples": len(inside)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# the sources that define each profiled kernel's code and launch (a committed
# DRAM-traffic figure is used only while these are unchanged)
KERNEL_SOURCES = {
    "k1": ("ss_internal.h", "ss_kernels.cuh", "ss_k1_d3.cu", "ss_k1_d4_exact.cu", "ss_host.cpp", "ss_status.cu"),
    "k2": ("ss_internal.h", "ss_kernels.cuh", "ss_k2.cuh", "ss_k2_d3.cu", "ss_k2_d4_exact.cu", "ss_host.cpp",
           "ss_status.cu"),
    "kc": ("ss_internal.h", "ss_kernels.cuh", "ss_contract.cuh", "ss_kc_d3.cu", "ss_host.cpp", "ss_status.cu"),
}
CASE_KERNEL = {"3d": "k1", "3d-small": "k1", "4d": "k1", "4d-small": "k1", "paper-3d": "k2", "paper-4d": "k2",
               "paper-3d-544": "k2", "paper-4d-112": "k2",
               "contract-small": "kc"}


def kernel_source_hash(kernel: str = "k1") -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1705_06661_gb300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(case: str):
    """DRAM bytes per launch from the committed ncu summary, only if the
    kernel's sources are unchanged since it was taken."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return None
    c = rec.get("cases", {}).get(case)
    if c is None or c.get("source_hash") != kernel_source_hash(CASE_KERNEL[case]):
        return None
    return c.get("dram_bytes_per_launch")


def cpu_baseline(seconds: float = 10.0):
    """The oracle as it stands on a bounded sample of the workload: the same
    operator and permuted extent with the spectator block cut from 48^3 to
    16^3 (16.8M elements), repeated for about `seconds`."""
    import oracle
    import workloads as wl
    shape = (16, 16, 16, 16, 16, 16)
    A = wl.uniform(1, shape)
    B = np.empty(shape, order="F")
    coef = wl.table2(1)
    n = A.size
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.spinsum(A, D, coef, factorized=True, B=B)
        reps += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": round(2 * n * 8 * reps / dt / 1e9, 3), "unit": "GB/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"A[16,16,16,16,16,16] ({n} doubles), same operator/mode, {reps} runs in {dt:.1f} s"}


def paper_cpu_algorithm(reps: int = 2):
    """The paper's own blocked CPU algorithm (Algorithms 5a/5b and 6, native
    host library) and the algorithm it is measured against (Algorithm 2, the
    NCC code's, expanded operator) on the host cores, on the paper-layout
    tensors of the tiled GPU lines: best of `reps` runs each."""
    import cpu_alg6
    import workloads as wl
    out = []
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    for d, n_, row in ((3, 544, 1), (4, 112, 5)):
        shp = (n_,) * d
        A = np.asfortranarray(wl.uniform(3, shp))
        B = np.empty(shp, order="F")
        coef = wl.table2(row)
        best = best2 = None
        for _ in range(reps):
            t0 = time.perf_counter()
            cpu_alg6.spinsum_alg6(A, coef, factorized=True, out=B, threads=threads)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
            t0 = time.perf_counter()
            cpu_alg6.spinsum_alg2(A, coef, out=B, threads=threads)
            dt = time.perf_counter() - t0
            best2 = dt if best2 is None else min(best2, dt)
        out.append({"case": f"paper layout {d}d N={n_} row{row} factorized out-of-place, paper's Alg. 6 on host",
                    "GB/s": round(2 * A.size * 8 / best / 1e9, 2), "ms": round(best * 1e3, 2), "threads": threads,
                    "alg2_GB/s": round(2 * A.size * 8 / best2 / 1e9, 2), "alg2_ms": round(best2 * 1e3, 2),
                    "alg6_speedup_over_alg2": round(best2 / best, 2)})
        del A, B
    return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, bytes_per_step: int, steps: int, dt_max: float) -> float:
    """Whole-job GB/s of `world` replicas that each ran `steps` steps of
    `bytes_per_step` algorithmic bytes, timed by the slowest rank."""
    return world * bytes_per_step * steps / dt_max / 1e9


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    import workloads as wl
    shape = (16, 16, 16, 16, 16, 16)      # bounded sample of the workload per step
    A = wl.uniform(1, shape)
    B = np.empty(shape, order="F")
    coef = wl.table2(1)
    for _ in range(args.warmup):
        oracle.spinsum(A, D, coef, factorized=True, B=B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.spinsum(A, D, coef, factorized=True, B=B)
    dt = time.perf_counter() - t0
    val = 2 * A.size * 8 * args.steps / dt / 1e9
    sample = f"A[16,16,16,16,16,16] ({A.size} doubles) per step, same operator and mode"
    print(json.dumps({
        "impl": "reference", "metric": "spin-summation effective HBM GB/s (2*N*bytes/time)", "value": round(val, 3),
        "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (SplitMix64 seed 1, uniform [-1,1))",
        "config": {"workload": WORKLOAD, "reference_sample": sample},
        "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(), "sample": sample, "value": round(val, 3),
                         "unit": "GB/s"},
        "e2e": {"value": round(val, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def time_steps(fn, steps, stream, world):
    import torch
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1) / 1e3


def best_of(fn, reps, stream):
    """(per-launch time of `reps` back-to-back launches, best single launch)"""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    loop = e0.elapsed_time(e1) / 1e3 / reps
    ts = []
    for _ in range(3):
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return loop, min(ts)


def extra_cases_contract(ss, wl, dev, stream, A, B, coef):
    """The summation fused into a contraction over the permuted group,
    C[s, y] = sum_t S(A)[s, t] W[y, t] on the benchmark tensor (S(A) never
    stored), against the unfused pair (the summation into B, then the
    contraction kernel alone on B) and, for context, cuBLAS DGEMM for the
    contraction alone. Both kernels are bound by the FP64 pipe (Y multiply-adds
    per element of A); the fused call saves the write and re-read of S(A)."""
    import torch
    out = []
    spec = tuple(A.shape[:3])
    S = int(np.prod(spec))
    T = int(np.prod(A.shape[3:]))
    n = A.numel()
    Braw = B.permute(*reversed(range(6))).reshape(T, S)     # B's storage as a (T, S) row-major matrix
    for Y in (4, 8, 32, 128):
        W = ss.colmajor_empty((Y, T), device=dev)
        W.copy_(torch.from_numpy(wl.uniform(7, (Y, T))).to(dev))
        C = ss.colmajor_empty(spec + (Y,), device=dev)
        reps = 5 if Y <= 32 else 2
        torch.matmul(W.permute(1, 0).t(), Braw)      # cuBLAS's first call on this shape sets up; not timed
        fused, _ = best_of(lambda: ss.contract(A, coef, W, out=C, factorized=True), reps, stream)
        summ, _ = best_of(lambda: ss.spinsum(A, coef, d=3, out=B, factorized=True), reps, stream)
        plain, _ = best_of(lambda: ss.contract(B, None, W, out=C), reps, stream)
        Wraw = W.permute(1, 0)
        cublas, _ = best_of(lambda: torch.matmul(Wraw.t(), Braw), reps, stream)
        tf = 2 * n * Y / fused / 1e12
        out.append({"case": f"fused summation+contraction Y={Y} (3d row1 factorized, A[48^3,16^3] x W[{Y},16^3])",
                    "ms": round(fused * 1e3, 3), "unfused_ms": round((summ + plain) * 1e3, 3),
                    "unfused_parts_ms": [round(summ * 1e3, 3), round(plain * 1e3, 3)],
                    "speedup_vs_unfused": round((summ + plain) / fused, 3),
                    "cublas_dgemm_contraction_only_ms": round(cublas * 1e3, 3),
                    "fp64_TFLOPs": round(tf, 3), "bound": "fp64",
                    "frac_of_nominal_fp64": round(tf / 1.25, 3)})
        del W, C
    return out


def extra_cases_batched_and_autograd(ss, wl, dev, stream, hbm_peak):
    """The batched workload (64 uneven 3D blocks, one persistent launch per
    class, replayed from a CUDA graph; FP64 and FP32 storage) and the
    differentiable 4D workload (10^8, forward + backward)."""
    import torch
    out = []
    blocks = wl.config4_blocks()
    for tdt, name in ((torch.float64, "fp64"), (torch.float32, "fp32-storage")):
        specs, nel = [], 0
        for pr in blocks:
            a = ss.colmajor_empty(pr.shape, dtype=tdt, device=dev)
            a.copy_(torch.from_numpy(wl.uniform(pr.seed, pr.shape)).to(dev))
            specs.append({"A": a, "B": ss.colmajor_like(a), "coef": pr.coef, "d": 3, "factorized": True})
            nel += a.numel()
        plan = ss.Plan(specs, tune=True)
        g = torch.cuda.CUDAGraph()
        s2 = torch.cuda.Stream(dev)
        s2.wait_stream(stream)
        with torch.cuda.stream(s2):
            with torch.cuda.graph(g, stream=s2):
                plan.execute()
        stream.wait_stream(s2)
        mn, one = best_of(g.replay, 10, stream)
        es = 8 if tdt == torch.float64 else 4
        out.append({"case": f"batched 64 uneven 3D blocks {name} (graph replay)", "elements": nel,
                    "GB/s": round(2 * nel * es / mn / 1e9, 1), "ms": round(mn * 1e3, 4),
                    "frac": round(2 * nel * es / mn / 1e9 / hbm_peak, 4), "plan": plan.describe()})
        plan.close()
        del specs, g
        torch.cuda.empty_cache()
    shape = (10,) * 8
    A = ss.colmajor_empty(shape, device=dev)
    A.copy_(torch.from_numpy(wl.uniform(4, shape)).to(dev))
    A.requires_grad_(True)
    G = ss.colmajor_empty(shape, device=dev)
    G.copy_(torch.from_numpy(wl.uniform(5, shape)).to(dev))
    coef = wl.random_coef(4, 105)

    def fwd_bwd():
        A.grad = None
        ss.spinsum_autograd(A, coef, d=4).backward(G)

    for _ in range(3):          # the first backward passes start autograd's device thread
        fwd_bwd()
    torch.cuda.synchronize()
    mn, one = best_of(fwd_bwd, 10, stream)
    n = A.numel()
    out.append({"case": "4d 10^8 random set forward+backward (autograd)", "GB/s": round(4 * n * 8 / mn / 1e9, 1),
                "ms": round(mn * 1e3, 4), "frac": round(4 * n * 8 / mn / 1e9 / hbm_peak, 4)})
    return out


def run_ours(args):
    import torch

    import paper_1705_06661_gb300 as ss
    import workloads as wl

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "of measured (MEASURED_PEAKS.json hbm_gbs, torch copy)" if hbm_peak else "of fallback"
    hbm_peak = hbm_peak or 6800.0

    # ---- inputs, resident in HBM ----
    A_host = wl.uniform(1, SHAPE)                      # column-major float64, 3.6 GB
    N = A_host.size
    A = ss.colmajor_empty(SHAPE, device=dev)
    A.copy_(torch.from_numpy(A_host).to(dev))
    B = ss.colmajor_like(A)
    coef = wl.table2(CASES[args.case][2])
    step = lambda: ss.spinsum(A, coef, d=D, out=B, factorized=True)  # noqa: E731
    if args.case.startswith("contract"):
        T = int(np.prod(SHAPE[D:]))
        Wc = ss.colmajor_empty((CONTRACT_Y, T), device=dev)
        Wc.copy_(torch.from_numpy(wl.uniform(7, (CONTRACT_Y, T))).to(dev))
        Cc = ss.colmajor_empty(tuple(SHAPE[:D]) + (CONTRACT_Y,), device=dev)
        step = lambda: ss.contract(A, coef, Wc, out=Cc, factorized=True)  # noqa: E731

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ss.spinsum_check_status(stream.cuda_stream)

    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first_sample()
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ss.spinsum_launch_count(reset=True)
    clocks.mark("t0")
    dt = time_steps(step, args.steps, stream, world)
    clocks.mark("t1")
    launches = ss.spinsum_launch_count(reset=True)
    clocks.stop()
    dt_max = allmax(world, dt)
    bytes_step = 2 * N * 8
    value = replica_throughput(world, bytes_step, args.steps, dt_max)
    ms_step = dt_max / args.steps * 1e3
    per_launch_s = dt / max(launches, 1)
    achieved = bytes_step / per_launch_s / 1e9 if launches == args.steps else bytes_step * args.steps / dt / 1e9
    ss.spinsum_check_status(stream.cuda_stream)

    # ---- end to end through the public API with pinned host buffers ----
    # spinsum_host on pinned buffers: the kernel reads A and writes B over the
    # host link (zero-copy); every step moves all of A in and all of B out
    nd = len(SHAPE)
    A_pin_cm = torch.empty(SHAPE[::-1], dtype=torch.float64).pin_memory().permute(*reversed(range(nd)))
    A_pin_cm.copy_(torch.from_numpy(A_host))
    B_pin = torch.empty(SHAPE[::-1], dtype=torch.float64).pin_memory().permute(*reversed(range(nd)))
    def e2e_step():
        ss.spinsum_host(A_pin_cm, coef, out=B_pin, d=D, factorized=True)

    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    dt_e2e = allmax(world, time_steps(e2e_step, e2e_steps, stream, world))
    e2e_val = world * bytes_step * e2e_steps / dt_e2e / 1e9
    # the result that came back is the device result (B holds it unless the
    # timed step was the contraction profiling case)
    if not args.case.startswith("contract"):
        assert torch.equal(B_pin[(slice(0, 2),) * nd], B[(slice(0, 2),) * nd].cpu())

    # ---- extra cases: other modes and the 4D workload (not the headline) ----
    extra = []
    if not args.no_extra and rank == 0:
        reps = 10
        cases = [
            # in place, repeated application grows the dominant component by the spectral radius of
            # the operator (12 for row 1); alpha = 2^-4 keeps the values bounded across repetitions
            ("3d row1 factorized in-place (alpha=2^-4)",
             lambda: ss.spinsum(A, coef, d=D, inplace=True, factorized=True, alpha=0.0625)),
            ("3d row1 expanded out-of-place", lambda: ss.spinsum(A, coef, d=D, out=B)),
            ("3d random-set expanded out-of-place", lambda: ss.spinsum(A, wl.random_coef(3, 102), d=D, out=B)),
            ("3d row1 strict-fp64 out-of-place", lambda: ss.spinsum(A, coef, d=D, out=B, factorized=True,
                                                                    strict=True)),
        ]
        for name, fn in cases:
            for _ in range(2):
                fn()
            mn, one = best_of(fn, reps, stream)
            extra.append({"case": name, "GB/s": round(bytes_step / mn / 1e9, 1), "ms": round(mn * 1e3, 4),
                          "ms_single_launch": round(one * 1e3, 4), "frac": round(bytes_step / mn / 1e9 / hbm_peak, 4)})
        del A_pin_cm, B_pin
        A32 = ss.colmajor_empty(SHAPE, dtype=torch.float32, device=dev)
        A32.copy_(A)
        B32 = ss.colmajor_like(A32)
        fn = lambda: ss.spinsum(A32, coef, d=D, out=B32, factorized=True)  # noqa: E731
        fn()
        mn, one = best_of(fn, reps, stream)
        extra.append({"case": "3d row1 factorized fp32-storage", "GB/s": round(2 * N * 4 / mn / 1e9, 1),
                      "ms": round(mn * 1e3, 4), "frac": round(2 * N * 4 / mn / 1e9 / hbm_peak, 4)})
        del A32, B32
        torch.cuda.empty_cache()
        extra += extra_cases_contract(ss, wl, dev, stream, A, B, coef)
        del A, B
        torch.cuda.empty_cache()
        shape4 = (12,) * 8
        A4 = ss.colmajor_empty(shape4, device=dev)
        A4.copy_(torch.from_numpy(wl.uniform(2, shape4)).to(dev))
        B4 = ss.colmajor_like(A4)
        n4 = A4.numel()
        for name, c4, kw in [("4d row5 factorized out-of-place", wl.table2(5), {"factorized": True}),
                             ("4d row5 factorized in-place (alpha=2^-6)", wl.table2(5),
                              {"factorized": True, "inplace": True, "alpha": 2.0 ** -6}),
                             ("4d row6 factorized out-of-place", wl.table2(6), {"factorized": True}),
                             ("4d row18 out-of-place", wl.table2(18), {}),
                             ("4d random-set expanded out-of-place", wl.random_coef(4, 103), {})]:
            if kw.get("inplace"):
                fn = lambda c4=c4, kw=kw: ss.spinsum(A4, c4, d=4, **kw)  # noqa: E731
            else:
                fn = lambda c4=c4, kw=kw: ss.spinsum(A4, c4, d=4, out=B4, **kw)  # noqa: E731
            for _ in range(2):
                fn()
            mn, one = best_of(fn, reps, stream)
            extra.append({"case": name, "GB/s": round(2 * n4 * 8 / mn / 1e9, 1), "ms": round(mn * 1e3, 4),
                          "ms_single_launch": round(one * 1e3, 4), "frac": round(2 * n4 * 8 / mn / 1e9 / hbm_peak, 4)})
        del A4, B4
        torch.cuda.empty_cache()
        # packed antisymmetric storage: the 3D tensor unpacked from its C(16, 3) = 560 values per position
        Pk = ss.colmajor_empty((48, 48, 48, 560), device=dev)
        Pk.copy_(torch.from_numpy(wl.uniform(5, (48, 48, 48, 560))).to(dev))
        Bk = ss.colmajor_empty(SHAPE, device=dev)
        for name, fn, nb in (("unpack 3d A[48^3, C(16,3)] -> A[48^3,16^3]", lambda: ss.unpack(Pk, 3, 16, out=Bk),
                              (Pk.numel() + Bk.numel()) * 8),
                             ("pack 3d A[48^3,16^3] -> A[48^3, C(16,3)]", lambda: ss.pack(Bk, 3, out=Pk),
                              2 * Pk.numel() * 8)):
            for _ in range(2):
                fn()
            mn, one = best_of(fn, reps, stream)
            extra.append({"case": name, "GB/s": round(nb / mn / 1e9, 1), "ms": round(mn * 1e3, 4),
                          "frac": round(nb / mn / 1e9 / hbm_peak, 4)})
        del Pk, Bk
        torch.cuda.empty_cache()
        # d = 2 (the CCSD pair, coefficients 2, -1): spectator layout and the N^2 matrix
        for shp2, nm in (((96, 96, 96, 96), "2d A[96^4]"), ((8192, 8192), "paper layout 2d N=8192")):
            A2 = ss.colmajor_empty(shp2, device=dev)
            A2.copy_(torch.from_numpy(wl.uniform(3, shp2)).to(dev))
            B2 = ss.colmajor_like(A2)
            c2 = np.array([[2.0, -1.0]])
            for name, fn in ((f"{nm} (2,-1) out-of-place", lambda: ss.spinsum(A2, c2, d=2, out=B2)),
                             (f"{nm} (2,-1) in-place (alpha=0.5)",
                              lambda: ss.spinsum(A2, c2, d=2, inplace=True, alpha=0.5))):
                for _ in range(2):
                    fn()
                mn, one = best_of(fn, reps, stream)
                n2 = A2.numel()
                extra.append({"case": name, "GB/s": round(2 * n2 * 8 / mn / 1e9, 1), "ms": round(mn * 1e3, 4),
                              "frac": round(2 * n2 * 8 / mn / 1e9 / hbm_peak, 4)})
            del A2, B2
            torch.cuda.empty_cache()
        # the paper's own layout: a dense N^d tensor with every index permuted (tiled kernel)
        for dp, Np, rowp in ((3, 544, 1), (4, 112, 5)):
            shp = (Np,) * dp
            Ap = ss.colmajor_empty(shp, device=dev)
            Ap.copy_(torch.from_numpy(wl.uniform(3, shp)).to(dev))
            Bp = ss.colmajor_like(Ap)
            cp = wl.table2(rowp)
            for name, kw, tgt in [(f"paper layout {dp}d N={Np} row{rowp} factorized out-of-place", {}, Bp),
                                  (f"paper layout {dp}d N={Np} row{rowp} factorized in-place (alpha=2^-6)",
                                   {"inplace": True, "alpha": 2.0 ** -6}, None)]:
                if tgt is None:
                    fn = lambda cp=cp, kw=kw: ss.spinsum(Ap, cp, d=dp, factorized=True, **kw)  # noqa: E731
                else:
                    fn = lambda cp=cp: ss.spinsum(Ap, cp, d=dp, out=Bp, factorized=True)  # noqa: E731
                for _ in range(2):
                    fn()
                mn, one = best_of(fn, reps, stream)
                npe = Ap.numel()
                extra.append({"case": name, "GB/s": round(2 * npe * 8 / mn / 1e9, 1), "ms": round(mn * 1e3, 4),
                              "frac": round(2 * npe * 8 / mn / 1e9 / hbm_peak, 4)})
            del Ap, Bp
            torch.cuda.empty_cache()
        extra += extra_cases_batched_and_autograd(ss, wl, dev, stream, hbm_peak)
        ss.spinsum_check_status(stream.cuda_stream)

    cpu = None
    host_alg = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()
        if not args.no_extra:
            host_alg = paper_cpu_algorithm()

    if rank == 0:
        out = {
            "metric": "spin-summation effective HBM GB/s (2*N*bytes/time)",
            "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(ms_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (SplitMix64 seed 1, uniform [-1,1)), inputs resident in HBM",
            "config": {"workload": WORKLOAD, "elements": N, "bytes_per_step": bytes_step,
                       "l2": "inputs larger than L2 (3.6 GB per tensor), no flush",
                       "parallelism": f"replicas x{world} (one full problem per GPU)"},
            "element_updates_per_s": round(world * N * args.steps / dt_max, 1),
            "gibps_eq12": round(world * bytes_step * args.steps / dt_max / 2 ** 30, 1),
            "frac_of_8TBps": round(value / 8000.0, 4),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(achieved / hbm_peak, 4), "peak_source": peak_src,
                         "traffic": ncu_traffic(args.case),
                         "algorithmic_bytes_per_launch": bytes_step},
            "e2e": {"value": round(e2e_val, 1), "unit": "GB/s", "h2d_bytes_per_step": N * 8,
                    "d2h_bytes_per_step": N * 8, "steps": e2e_steps},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
            "paper_cpu_algorithm": host_alg,
            "paper_context": "Alg. 6 speedups over NCC 2.4-5.5x on 2x Xeon E5-2680 v3 (FP64); no absolute numbers",
            "cases": extra,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    global D, SHAPE, WORKLOAD
    args = parse()
    if args.case != "3d":
        d, shape, row = CASES[args.case]
        D, SHAPE = d, shape
        WORKLOAD = f"{d}d-spinsum fp64 A{list(shape)} Table-II-row-{row} factorized out-of-place (profiling case)"
        args.no_extra = True
        args.no_cpu = True
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
