#!/usr/bin/env python3
"""Benchmark: transformed coefficients per second at n = 1e6 on GB300.

Workload (one "step"): the single-vector n = 1,000,000 transform in both
directions -- Legendre->Chebyshev and Chebyshev->Legendre -- of the same
vector, coefficients N(0,1) (j+1)^-1 from seed 1 (float64, host PCG64).
Inputs are resident in HBM; the L2 cache (129 MB) is flushed by writing a
256 MB buffer before every timed step (outside the step's events).

Reported (one JSON line on rank 0):
  value        2n / device time per step, for the fastest FP64-accurate tier
  e2e          same metric through the C ABI with pinned host buffers
               (host->device copy of both inputs and device->host copy of
               both outputs inside the timed region)
  accuracy     E_2 / E_inf of the timed tier on sampled output rows against
               the CPU oracle (the same rows the cpu_baseline leg computes)
  tiers        coefficients/s of every FP64-accurate tier, including the
               plain FP64 path
  roofline     the dominant kernel's achieved FP64 rate (or bytes) per launch
               over its CUDA-event duration in the timed region
  cpu_baseline the oracle (direct O(n^2) double-double sum) on the host's
               cores, on a bounded sample of the same workload's rows

--impl reference times the oracle itself (the only reference this project
has) on the same workload and prints the same line with "impl": "reference".
Multi-GPU (torchrun): every rank transforms its own copy (replicas; the
transform has no exchange step), value = all ranks' coefficients / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_COEF = 1_000_000
PAPER_COEF_PER_S = 1_000_000 / 0.020   # paper: ~20 ms per 1e6 L2C, 1 core of an M3 Pro (context only)
CPU_ROWS = 4096                         # oracle rows per direction for the CPU baseline / accuracy sample
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz
# Double-float tier: one FP64-equivalent multiply-add costs 12 FP32-pipe
# instructions (TwoProd with fma, cross terms, TwoSum accumulation); the FP32
# issue limit is 152 SMs x 128 lanes x 2070 MHz.
DF_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 12 * 2 / 1e12
try:  # measured copy bandwidth of the GB300s
    HBM_PEAK_GBS = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
except Exception:
    HBM_PEAK_GBS = 6800.0  # fallback figure for a GB300
# DRAM bytes per launch of the two largest kernels (the band k_near, kind 7,
# and the last down chunk, kind 4), dram__bytes_read.sum + dram__bytes_write.sum
# from the ncu captures summarised in profiles/df_single_n1e6.md and
# profiles/f64_single_n1e6.md (one L2C launch at n = 1e6).
TRAFFIC = {("f64_df", 7): 19.508e6, ("f64_df", 4): 17.348e6, ("f64", 7): 17.028e6, ("f64", 4): 17.365e6}
KIND_NAMES = {0: "leaf_restrict", 1: "upward", 2: "couple", 3: "downward", 4: "spread_sum_scale", 5: "prepare",
              6: "other", 7: "near_band"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tier", default="auto", help="f64 | f64_df | f64_split | auto (fastest FP64-accurate)")
    ap.add_argument("--cpu-rows", type=int, default=CPU_ROWS)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle legs (profiling runs)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workloads")
    ap.add_argument("--profile", default=None,
                    help="TIER:DIRECTION:N:BATCH[:levels] -- build one plan, run it twice, exit (a short target for ncu); "
                         "':levels' gives a split plan its per-level launches")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------ multi-rank
def replica_throughput(ms_local, coef_per_rank, device=None):
    """Whole-job throughput of N independent replicas (the transform has no
    exchange step): every rank transforms its own copy; the job time is the
    slowest rank's.  Returns (ms_max, coefficients/s over all ranks)."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    ms = float(ms_local)
    if ws > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ws * coef_per_rank / (ms / 1e3)


# ---------------------------------------------------------------- oracle leg
def oracle_leg(n, x, rows_per_dir):
    """Time the oracle on `rows_per_dir` sampled rows of each direction."""
    import numpy as np
    import oracle
    import workloads
    rows = workloads.sample_rows(n, 4096)
    rng = np.random.default_rng(12345)
    pick = np.sort(rng.choice(rows, size=min(rows_per_dir, rows.size), replace=False))
    t0 = time.perf_counter()
    ref_l2c = oracle.apply(oracle.L2C, x, rows=pick)
    ref_c2l = oracle.apply(oracle.C2L, x, rows=pick)
    dt = time.perf_counter() - t0
    return pick, ref_l2c, ref_c2l, dt, oracle.threads()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    import workloads
    n = N_COEF
    x = workloads.decaying_vector(n, seed=1, r=1.0)
    rows_all = workloads.sample_rows(n, 4096)
    per_step = max(1, args.cpu_rows // max(1, args.steps + args.warmup))
    rng = np.random.default_rng(777)
    times = []
    for k in range(args.warmup + args.steps):
        pick = np.sort(rng.choice(rows_all, size=per_step, replace=False))
        t0 = time.perf_counter()
        oracle.apply(oracle.L2C, x, rows=pick)
        oracle.apply(oracle.C2L, x, rows=pick)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = 2 * per_step / t
    line = {
        "impl": "reference", "metric": "transformed coefficients/s (n=1e6, L2C+C2L, FP64-accurate)",
        "value": value, "unit": "coefficients/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_COEF_PER_S,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "n=1e6 single vector, L2C and C2L, N(0,1)(j+1)^-1 seed 1", "n": n, "batch": 1},
        "cpu_baseline": {"value": value, "unit": "coefficients/s", "cores": oracle.threads(), "kind": "oracle",
                         "sample": "%d sampled output rows per direction per step of the n=1e6 transform "
                                   "(direct double-double row sums)" % per_step},
        "e2e": {"value": value, "unit": "coefficients/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- clock sampler
class ClockSampler:
    """SM clock and throttle reasons of one GPU, sampled while the timed
    region runs.  NVML (read-only queries through ctypes) in a background
    thread every ~1 ms, so that even a region of a few milliseconds is
    sampled; nvidia-smi at 100 ms as the fallback.  Nothing is changed on the
    GPU."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clocks-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, gpu_index: int):
        import ctypes
        import threading
        self.proc = None
        self.gpu = gpu_index
        self.samples = []
        self.max_mhz = None
        self.thread = None
        self.stop_flag = threading.Event()
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(gpu_index), ctypes.byref(h)) != 0:
                raise OSError("no NVML handle")
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
                self.max_mhz = float(mx.value)
            get_reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons

            def run():
                clk = ctypes.c_uint()
                rs = ctypes.c_ulonglong()
                while not self.stop_flag.is_set():
                    if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0:
                        r = rs.value if get_reasons(h, ctypes.byref(rs)) == 0 else 0
                        self.samples.append((float(clk.value), int(r)))
                    time.sleep(0.001)
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            time.sleep(0.005)
        except Exception:
            self.thread = None
            try:
                self.proc = subprocess.Popen(
                    ["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                     "--format=csv,noheader,nounits", "-lms", "100"],
                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            except Exception:
                self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=2)
            if not self.samples:
                return None
            reasons = set()
            for _, r in self.samples:
                for bit, nm in self.REASONS.items():
                    if r & bit:
                        reasons.add(nm)
            sm = [c for c, _ in self.samples]
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": self.max_mhz or max(sm),
                    "reasons": sorted(reasons), "samples": len(sm), "source": "nvml"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi"}


# ------------------------------------------------------------------ our leg
def near_field_nonzeros(n, L, s):
    """Nonzeros of the direct band (Step 6) for rows < n."""
    import numpy as np
    i = np.arange(n, dtype=np.int64)
    end = np.minimum(n, 2 * s * (i // (2 * s) + 2)) if L > 0 else np.full(n, n, np.int64)
    return int(((end - i + 1) // 2).sum())


def kernel_work(info, kind, direction, leaf_depth=4):
    """Algorithmic FP64 flops of one launch of a kernel kind (paper's counting, Sec. 4.2)."""
    n, L, s, M, nc, N = info["n"], info["L"], info["s"], info["M"], info["n_c"], info["N"]
    if kind == 7:
        # near-field band: 3 flops per band nonzero (mu = 4.5), scaling 1 per row
        return 3 * near_field_nonzeros(n, L, s) + n
    if kind == 4:
        # last down chunk: Step 4 on the fine levels [max(0, L-1-leaf_depth), L) (a triangular
        # M x M product, M(M+1) flops per node and parity), then the spread
        # (2M per row with a far field) and the sum with the band's part (1 per row)
        rho = max(0, L - 1 - leaf_depth)
        nodes = 0
        for g in range(rho, L):
            nodes += ((4 << g) - 4) if g > 0 else 0
        rows_far = min(n, N - 4 * s) if L > 0 else 0
        return 2 * M * (M + 1) * nodes + 2 * M * rows_far + n
    if kind == 2:  # couple: 2 M^2 per submatrix per parity
        return 4 * M * M * nc
    if kind == 0:  # leaf: 2 M s per segment per parity
        return 2 * 2 * M * s * ((2 << L) - 2)
    return None


def measured_fp32_tflops(dev):
    """FP32 FLOP/s of the CUDA cores on this GPU, measured: cuBLAS SGEMM 8192^3
    with TF32 off (best of 5, CUDA events).  The double-float ceiling is this
    rate / 12 (one FP64-equivalent multiply-add = 12 FP32-pipe instructions)."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        n = 8192
        a = torch.randn(n, n, device=dev, dtype=torch.float32)
        b = torch.randn(n, n, device=dev, dtype=torch.float32)
        c = a @ b
        torch.cuda.synchronize()
        best = None
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        del a, b, c
        return 2.0 * n ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def graph_step(fn):
    """Capture fn (library launches on the current stream) into a CUDA graph."""
    import torch
    fn()  # warm (plans, lazy module loads)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    return g.replay


def time_fn(fn, flush, steps, warmup):
    import torch
    for _ in range(warmup):
        flush.fill_(1.0)
        fn()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.fill_(float(k))
        evs[k][0].record()
        fn()
        evs[k][1].record()
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in evs)


def split_tensor_fractions(lc, dev, X, Z, n, B):
    """Executed bf16 tensor work of each split-tier kernel kind over its
    CUDA-event duration.  Every CTA takes 128 members and issues one
    tcgen05.mma (M = 128, N = 32, K = 16) per slice pair (S (S+1)/2 of them)
    and K slice of its product; counts come from the plan geometry, padding
    included."""
    plan = lc.Plan(n, "l2c", B, "f64_split", dev)
    info = plan.info
    L, s = info["L"], info["s"]
    S = 7 if n <= 100000 else 6  # the library's default slice count for this n
    pairs = S * (S + 1) // 2
    tiles = -(-B // 128)
    mma = 128 * 32 * 16 * 2
    kslices = lambda K: max(32, -(-K // 16) * 16) // 16  # K padded to 16, at least 32
    M = info["M"]
    ctas = {  # CTAs (tiles x 2 parities) per work item kind
        0: ((2 << L) - 2) * tiles * 2,
        1: sum((1 << (L - d)) - 2 for d in range(L - 1)) * tiles * 2,
        2: sum((2 << (L - d)) - 2 for d in range(L)) * tiles * 2,
        3: sum((2 << (L - d)) - 4 for d in range(L - 1)) * tiles * 2,
        4: (2 << L) * tiles * 2,  # strips of width 2s
    }
    per_cta = {0: kslices(s), 1: kslices(2 * M), 2: kslices(2 * M), 3: kslices(M), 4: kslices(2 * s) + kslices(M)}
    plan.set_split_schedule(False)  # one launch per level, timed per kind
    lc.binding.lc_plan_set_timing(plan._handle, 3)
    for _ in range(3):
        plan(X, out=Z)
    import torch
    torch.cuda.synchronize()
    tot = {}
    for slot in range(3):
        for kind, t in lc.binding.lc_plan_get_timing(plan._handle, slot):
            tot[kind] = tot.get(kind, 0.0) + t / 3
    lc.binding.lc_plan_set_timing(plan._handle, 0)
    try:
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        peak = 1900.0
    out = {}
    for kind, c in ctas.items():
        if kind in tot and tot[kind] > 0:
            fl = c * pairs * per_cta[kind] * mma
            ach = fl / (tot[kind] / 1e3) / 1e12
            out["spread_near_scale" if kind == 4 else KIND_NAMES[kind]] = {
                "bound": "tensor", "executed_tflop": fl / 1e12, "ms": tot[kind], "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak}
    del plan
    return out


def batched_leg(lc, dev, flush, args):
    """Batched workloads sharing one plan: split-precision tensor-core tier
    (one CUDA graph replay per step) against the plain FP64 tier."""
    import numpy as np
    import torch
    import workloads
    out = {}
    steps = max(3, min(10, args.steps))
    # (a) uniform batch: 256 vectors of n = 65536 (the differentiable-fit shape), L2C
    n, B = 65536, 256
    X = torch.as_tensor(workloads.decaying_vector(n, seed=5, r=1.0, batch=B), device=dev)
    Z = torch.empty_like(X)
    res = {}
    ref = None
    for tier in ("f64_split", "f64_df", "f64"):
        plan = lc.Plan(n, "l2c", B, tier, dev)
        step = graph_step(lambda: plan(X, out=Z))
        ms = time_fn(step, flush, steps, 2)
        res[tier] = {"coefficients_per_s": n * B / (ms / 1e3), "ms": ms,
                     "launches": plan.launches()}
        outs_b = locals().setdefault("outs_b", {})
        outs_b[tier] = Z.clone()
        if tier == "f64_split":  # the same plan with one launch per level
            plan.set_split_schedule(False)
            step = graph_step(lambda: plan(X, out=Z))
            ms2 = time_fn(step, flush, steps, 2)
            res[tier]["level_launches"] = {"coefficients_per_s": n * B / (ms2 / 1e3), "ms": ms2,
                                           "launches": plan.launches()}
        del plan
    # per result: every member's normwise error against the CPU oracle on
    # 128 sampled rows (the same rows for every member and tier)
    import oracle
    rows = workloads.sample_rows(n, 128, seed=10002)
    Xh = X.cpu().numpy()
    t0 = time.perf_counter()
    refs = np.stack([oracle.apply(oracle.L2C, Xh[b], rows=rows) for b in range(B)])
    oracle_s = time.perf_counter() - t0
    for t in ("f64_split", "f64_df", "f64"):
        zz = outs_b[t].cpu().numpy()[:, rows]
        per = np.linalg.norm(zz - refs, axis=1) / np.linalg.norm(refs, axis=1)
        res[t]["E2_vs_oracle_per_member"] = {"max": float(per.max()), "median": float(np.median(per)),
                                             "members": int(B), "rows_per_member": int(rows.size)}
    res["oracle_rows_s"] = oracle_s
    res["speedup_split_over_f64_batched"] = res["f64_split"]["coefficients_per_s"] / res["f64"]["coefficients_per_s"]
    res["f64_split_tensor_per_kernel"] = split_tensor_fractions(lc, dev, X, Z, n, B)
    out["uniform_65536x256_l2c"] = res
    del X, Z
    # (b) ragged batch: 4096 transforms, n log-uniform in [64, 65536]
    lengths = workloads.ragged_lengths(4096, seed=2)
    x = torch.as_tensor(workloads.ragged_batch(lengths, seed=3), device=dev)
    z = torch.empty_like(x)
    t0 = time.perf_counter()
    plan = lc.Plan(direction="l2c", dtype="f64_split", device=dev, lengths=lengths)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    # leaf tile s picked by the autotuner (plan-time, untimed like the plan itself)
    tplan, tile_s, tile_ms = lc.autotune_tile(x, "l2c", "f64_split", dev, lengths=lengths)
    if tile_ms[tile_s] < tile_ms.get(32, float("inf")):
        plan = tplan
    else:
        tile_s = 32
    step = graph_step(lambda: plan(x, out=z))
    ms = time_fn(step, flush, steps, 2)
    out["ragged_4096_l2c"] = {"coefficients_per_s": float(lengths.sum()) / (ms / 1e3), "ms": ms,
                              "coefficients": int(lengths.sum()), "plan_s": plan_s, "launches": plan.launches(),
                              "leaf_tile_s": tile_s, "autotune_ms_per_s": tile_ms}
    plan.set_split_schedule(False)  # the same plan with one launch per level
    step = graph_step(lambda: plan(x, out=z))
    ms2 = time_fn(step, flush, steps, 2)
    out["ragged_4096_l2c"]["level_launches"] = {"coefficients_per_s": float(lengths.sum()) / (ms2 / 1e3),
                                                "ms": ms2, "launches": plan.launches()}
    del tplan
    del plan, x, z
    # (b') the plain per-vector FP64 and double-float paths on a sample of 128 members
    sample = np.random.default_rng(6).choice(len(lengths), 128, replace=False)
    offs = workloads.ragged_offsets(lengths)
    xs = torch.as_tensor(workloads.ragged_batch(lengths, seed=3), device=dev)
    for tier in ("f64", "f64_df"):
        plans = [(lc.Plan(int(lengths[i]), "l2c", 1, tier, dev), int(offs[i]), int(lengths[i])) for i in sample]
        zs = torch.empty_like(xs)

        def per_vector():
            for pl_, a, m in plans:
                pl_(xs[a:a + m], out=zs[a:a + m])
        step = graph_step(per_vector)
        ms = time_fn(step, flush, max(3, steps // 2), 1)
        cnt = int(sum(m for _, _, m in plans))
        out["ragged_4096_l2c"]["per_vector_%s_sample128" % tier] = {"coefficients_per_s": cnt / (ms / 1e3), "ms": ms,
                                                                     "coefficients": cnt}
        del plans
    del xs
    # (c) 512^3 array, Legendre->Chebyshev along each axis in one call per axis
    #     (axes 0 and 2: one batch stride; axis 1: the two-level batch of
    #     lc_execute_ex); output in the array's own layout.  64 fibres per axis
    #     are checked against the oracle.
    import oracle
    N3 = 512
    cube64 = torch.as_tensor(workloads.cube(N3, seed=4), device=dev)
    fib = np.random.default_rng(8).integers(0, N3, size=(64, 2))
    for tier in ("f64_split", "f64_df", "f32"):
        cube = cube64.float() if tier == "f32" else cube64
        outc = torch.empty_like(cube)
        plan = lc.Plan(N3, "l2c", N3 * N3, tier, dev)
        res = {}
        for axis in (0, 1, 2):
            step = graph_step(lambda: plan.along_axis(cube, axis, out=outc))
            ms = time_fn(step, flush, max(3, steps // 2), 1)
            step()
            torch.cuda.synchronize()
            worst = 0.0
            for a_, b_ in fib:
                idx = [int(a_), int(b_)]
                idx.insert(axis, slice(None))
                xin = cube[tuple(idx)].double().cpu().numpy()
                zz = outc[tuple(idx)].double().cpu().numpy()
                ref = oracle.apply(oracle.L2C, xin)
                worst = max(worst, float(np.linalg.norm(zz - ref) / np.linalg.norm(ref)))
            res["axis%d" % axis] = {"coefficients_per_s": N3 ** 3 / (ms / 1e3), "ms": ms, "calls": 1,
                                    "E2_vs_oracle_max_64_fibres": worst}
        out["cube512_l2c_" + tier] = res
        del plan, outc
    # (c') Legendre synthesis on Chebyshev points along the last axis: values
    #      p(x_m) at x_m = cos((m+1/2) pi/512) of every fibre (L2C, then the
    #      cosine transform of each result vector in place)
    syn = {}
    for tier in ("f64_split", "f64_df"):
        plan = lc.Plan(N3, "l2c", N3 * N3, tier, dev, values=True)
        outc = torch.empty_like(cube64)
        step = graph_step(lambda: plan.along_axis(cube64, 2, out=outc))
        ms = time_fn(step, flush, max(3, steps // 2), 1)
        step()
        torch.cuda.synchronize()
        worst = 0.0
        for a_, b_ in fib[:16]:
            xin = cube64[int(a_), int(b_), :].cpu().numpy()
            zz = outc[int(a_), int(b_), :].cpu().numpy()
            ref = oracle.synthesis(xin)
            worst = max(worst, float(np.linalg.norm(zz - ref) / np.linalg.norm(ref)))
        syn[tier] = {"coefficients_per_s": N3 ** 3 / (ms / 1e3), "ms": ms, "launches": plan.launches(),
                     "E2_vs_oracle_max_16_fibres": worst}
        del plan, outc
    out["cube512_synthesis_axis2"] = syn
    del cube64
    # (d) differentiable least-squares fit: loss = ||leg2cheb(x) - y||^2, n = 65536, batch 256,
    #     one step = forward transform + hand-written adjoint (autograd backward)
    x0, y0 = workloads.fit_pair(65536, 256)
    fit = {}
    for tier in ("f64_df", "f64_split", "f64", "f32"):
        dt = torch.float32 if tier == "f32" else torch.float64
        xt = torch.as_tensor(x0, device=dev, dtype=dt).requires_grad_(True)
        yt = torch.as_tensor(y0, device=dev, dtype=dt)

        def fit_step():
            xt.grad = None
            loss = ((lc.leg2cheb(xt, dtype=tier) - yt) ** 2).sum()
            loss.backward()
        ms = time_fn(fit_step, flush, max(3, steps // 2), 2)
        fit[tier] = {"ms_per_step": ms, "transforms_per_step": 2,
                     "coefficients_per_s": 2 * 65536 * 256 / (ms / 1e3)}
        del xt, yt
    out["fit_65536x256_forward_backward"] = fit
    torch.cuda.synchronize()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_00033_gb300 as lc
    import workloads

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    n = N_COEF
    x_host = workloads.decaying_vector(n, seed=1, r=1.0)
    x = torch.from_numpy(x_host).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    available = ["f64", "f64_df"]  # the split tier is for batches (reported under "batched")
    tiers = {}
    tuned = {}
    plan_ms = {}
    outs = (torch.empty_like(x), torch.empty_like(x))
    for t in available:
        try:
            tiers[t] = (lc.Plan(n, "l2c", 1, t, dev), lc.Plan(n, "c2l", 1, t, dev))
        except lc.LegChebError as e:
            if e.status != 5:  # LC_ERR_UNSUPPORTED: tier not built for this request
                raise
            continue
        # plan build time (tables on the GPU, off the timed path; reported
        # separately): host clock around lc_plan_create on a workspace the caller
        # has already allocated (the C ABI never allocates), plan kernels
        # included; the median of 5 creations
        tp, tpa = [], []
        for d in ("l2c", "c2l"):
            code = lc.LC_L2C if d == "l2c" else lc.LC_C2L
            tcode = {"f64": lc.LC_F64, "f64_df": lc.LC_F64_DF}[t]
            nbytes = lc.binding.lc_plan_workspace_size(n, code, 1, tcode)
            ws_t = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            sp = torch.cuda.current_stream(dev).cuda_stream
            reps = []
            for _ in range(5):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                h = lc.binding.lc_plan_create(n, code, 1, tcode, ws_t.data_ptr(), nbytes, sp)
                torch.cuda.synchronize()
                reps.append((time.perf_counter() - t0) * 1e3)
                lc.binding.lc_destroy(h)
            tp.append(statistics.median(reps))
            del ws_t
            # the same through the Python Plan, workspace allocation included
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tmp = lc.Plan(n, d, 1, t, dev)
            torch.cuda.synchronize()
            tpa.append((time.perf_counter() - t0) * 1e3)
            del tmp
        plan_ms[t] = {"l2c": tp[0], "c2l": tp[1], "with_workspace_allocation": {"l2c": tpa[0], "c2l": tpa[1]}}
        # plan setup includes the autotuner's choice of chunk geometry (untimed, like planning)
        tuned[t] = [list(p.autotune(x, out=outs[0])[:2]) for p in tiers[t]]

    # One step: the two transforms are independent, so, as a caller would, the
    # Legendre->Chebyshev one runs on the current stream and the
    # Chebyshev->Legendre one on a second stream, joined before the step ends.
    # (The per-kernel timing pass runs them one after the other instead.)
    s2 = torch.cuda.Stream(dev)

    def step(pl, serial=False):
        if serial:
            pl[0](x, out=outs[0])
            pl[1](x, out=outs[1])
            return
        cur = torch.cuda.current_stream(dev)
        s2.wait_stream(cur)
        pl[0](x, out=outs[0])
        with torch.cuda.stream(s2):
            pl[1](x, out=outs[1])
        cur.wait_stream(s2)

    def time_tier(pl, steps, warmup, stage_timing=False, cold=True):
        for _ in range(warmup):
            flush.fill_(1.0)
            step(pl, serial=stage_timing)
        if stage_timing:
            for p in pl:
                lc.binding.lc_plan_set_timing(p._handle, steps)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(steps):
            if cold:
                flush.fill_(float(k))
            starts[k].record()
            step(pl, serial=stage_timing)
            ends[k].record()
        torch.cuda.synchronize()
        barrier()
        wall = time.perf_counter() - t0
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        stages = None
        if stage_timing:
            stages = {}
            for d, p in enumerate(pl):
                per = {}
                for k in range(steps):
                    for kind, t in lc.binding.lc_plan_get_timing(p._handle, k):
                        per.setdefault(kind, []).append(t)
                stages[d] = per
                lc.binding.lc_plan_set_timing(p._handle, 0)
        return ms, wall, stages

    # short timing of every tier to pick the fastest FP64-accurate one
    quick = {}
    for t, pl in tiers.items():
        ms, _, _ = time_tier(pl, max(5, min(20, args.steps)), args.warmup)
        quick[t] = statistics.median(ms)
    chosen = args.tier if args.tier != "auto" else min(quick, key=quick.get)
    pl = tiers[chosen]

    clocks = ClockSampler(local if ws > 1 else 0)
    ms, wall, _ = time_tier(pl, args.steps, args.warmup)
    clk = clocks.stop()
    # the same steps with the L2 cache left warm (no flush between steps): the
    # plan tables (A-hat: 85-127 MB per direction) then partly stay in L2
    ms_warm, _, _ = time_tier(pl, args.steps, 2, cold=False)
    # Per-kernel durations: the same steps again with CUDA events between the
    # library's kernels (in this mode each execution stays on one stream, so the
    # overlap of the coarse levels with the coupling is off).
    _, _, stages = time_tier(pl, args.steps, 2, stage_timing=True)
    ms_per_step, value = replica_throughput(sum(ms) / len(ms), 2 * n, dev)

    # one transform at a time on the plan's own streams (the latency a caller
    # with a single vector sees), cold L2, median
    one_ms = {}
    for d, p1, z1 in (("l2c", pl[0], outs[0]), ("c2l", pl[1], outs[1])):
        one_ms[d] = time_fn(lambda: p1(x, out=z1), flush, max(10, min(50, args.steps)), 3)

    # per-tier numbers (median of a shorter run each)
    tier_vals = {}
    for t, p2 in tiers.items():
        m2, _, _ = time_tier(p2, max(10, min(50, args.steps)), 2)
        tier_vals[t] = {"coefficients_per_s": 2 * n / (statistics.median(m2) / 1e3),
                        "ms_per_step_median": statistics.median(m2), "launches_per_step": p2[0].launches() + p2[1].launches()}

    # the nodal variant of the far field (eq:AijLag, the method the paper's
    # modal one replaces) beside the modal one, plain FP64 tier: execution
    # (same step) and planning
    nodal = {}
    if not args.no_batched:
        for nd in (0, 1):
            t0p = time.perf_counter()
            pn = (lc.Plan(n, "l2c", 1, "f64", dev, nodal=bool(nd)), lc.Plan(n, "c2l", 1, "f64", dev, nodal=bool(nd)))
            torch.cuda.synchronize()
            plan_s = time.perf_counter() - t0p
            m2, _, _ = time_tier(pn, max(10, min(50, args.steps)), 2)
            nodal["nodal" if nd else "modal"] = {
                "coefficients_per_s": 2 * n / (statistics.median(m2) / 1e3),
                "ms_per_step_median": statistics.median(m2), "plan_ms_both_directions": plan_s * 1e3}
            del pn

    # values at the Chebyshev points (option values): Legendre synthesis on the
    # n = 2^20 and n = 1e6 Chebyshev-Gauss points and its inverse, the chosen
    # tier; the same step shape (synthesis and analysis on two streams); the
    # cosine pass checked against the oracle's direct sums on 256 sampled points
    values_leg = {}
    for nv in ((1 << 20, n) if not args.no_batched else ()):
        xv = torch.from_numpy(workloads.decaying_vector(nv, seed=1, r=1.0)).to(dev)
        pv = (lc.Plan(nv, "l2c", 1, chosen, dev, values=True), lc.Plan(nv, "c2l", 1, chosen, dev, values=True))
        ov = [torch.empty_like(xv), torch.empty_like(xv)]

        def vstep():
            cur = torch.cuda.current_stream(dev)
            s2.wait_stream(cur)
            pv[0](xv, out=ov[0])
            with torch.cuda.stream(s2):
                pv[1](xv, out=ov[1])
            cur.wait_stream(s2)
        mv = time_fn(vstep, flush, max(10, min(50, args.steps)), 3)
        rec = {"coefficients_per_s": 2 * nv / (mv / 1e3), "ms_per_step": mv, "tier": chosen,
               "launches_per_step": pv[0].launches() + pv[1].launches(),
               "fft": "four-step, length n" if nv & (nv - 1) == 0 else "Bluestein, two FFTs of length 2^%d"
               % (2 * nv - 1).bit_length()}
        if rank == 0 and not args.no_cpu:
            import oracle
            c = lc.Plan(nv, "l2c", 1, chosen, dev)(xv).cpu().numpy()
            rows = workloads.sample_rows(nv, 256)
            ref = oracle.dct(0, c, rows=rows)
            got = ov[0].cpu().numpy()[rows]
            rec["cosine_pass_E2_vs_oracle_256_points"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        values_leg["n=%d" % nv] = rec
        del pv, ov, xv

    # Gegenbauer plans (coefficients of C_j^(a) <-> Chebyshev; a = 1/2 is the
    # Legendre case above): the same vector, tier and step, with the oracle's
    # error on 256 of the sampled rows per direction
    geg = {}
    if not args.no_batched:
        for a_ in (0.25, 1.5):
            pg = (lc.Plan(n, "l2c", 1, chosen, dev, alpha=a_), lc.Plan(n, "c2l", 1, chosen, dev, alpha=a_))
            m2, _, _ = time_tier(pg, max(10, min(50, args.steps)), 2)
            rec = {"coefficients_per_s": 2 * n / (statistics.median(m2) / 1e3),
                   "ms_per_step_median": statistics.median(m2), "tier": chosen}
            if rank == 0 and not args.no_cpu:
                import oracle
                rows = workloads.sample_rows(n, 4096)[::16]
                step(pg)
                torch.cuda.synchronize()
                for d_, o_ in enumerate((outs[0], outs[1])):
                    ref = oracle.apply(d_, x_host, rows=rows, alpha=a_)
                    dz = o_.cpu().numpy()[rows] - ref
                    rec[("l2c", "c2l")[d_] + "_E2_vs_oracle"] = float(np.linalg.norm(dz) / np.linalg.norm(ref))
                rec["oracle_rows"] = int(rows.size)
            geg["alpha_%g" % a_] = rec
            del pg

    # end to end through the C ABI with pinned host buffers: every step copies
    # its two inputs in from pinned host memory and its two results back.  Two
    # copy streams (host->device and device->host run at the same time), the
    # two compute streams of the device-timed step, and NQ device buffers per
    # side in a ring, so the next inputs' copies and the previous results'
    # read-backs overlap the transforms (the way a caller streams independent
    # transforms).  Transform q = 2 * step + direction uses slot q % NQ.
    NQ = 4
    h_in = (torch.from_numpy(x_host.copy()).pin_memory(), torch.from_numpy(x_host.copy()).pin_memory())
    h_out = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(NQ)]
    d_in = [torch.empty_like(x) for _ in range(NQ)]
    d_out = [torch.empty_like(x) for _ in range(NQ)]
    sc = torch.cuda.current_stream(dev)
    s_in = torch.cuda.Stream(dev)
    s_out = torch.cuda.Stream(dev)
    scs = (sc, s2)  # compute streams: one per direction, as in the device-timed step
    ev_in = [torch.cuda.Event() for _ in range(NQ)]    # input copied
    ev_done = [torch.cuda.Event() for _ in range(NQ)]  # transform done (input slot free, output ready)
    ev_out = [torch.cuda.Event() for _ in range(NQ)]   # result copied back (output slot free)

    def h2d(q):
        k = q % NQ
        with torch.cuda.stream(s_in):
            if q >= NQ:
                s_in.wait_event(ev_done[k])
            d_in[k].copy_(h_in[q % 2], non_blocking=True)
            ev_in[k].record(s_in)

    def pipeline(steps, e0=None, e1=None):
        if e0 is not None:
            e0.record(sc)
            s_in.wait_event(e0)
        total = 2 * steps
        ahead = NQ - 1
        for q in range(min(ahead, total)):
            h2d(q)
        for q in range(total):
            k, d = q % NQ, q % 2
            if q + ahead < total:
                h2d(q + ahead)
            cs = scs[d]
            cs.wait_event(ev_in[k])
            if q >= NQ:
                cs.wait_event(ev_out[k])
            with torch.cuda.stream(cs):
                pl[d](d_in[k], out=d_out[k])
            ev_done[k].record(cs)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[k])
                h_out[k].copy_(d_out[k], non_blocking=True)
                ev_out[k].record(s_out)
        sc.wait_stream(s2)
        sc.wait_stream(s_in)
        sc.wait_stream(s_out)
        if e1 is not None:
            e1.record(sc)

    e2e_steps = max(5, min(args.steps, 100))
    pipeline(2)
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    pipeline(e2e_steps, e0, e1)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_val = ws * 2 * n / (e2e_ms / 1e3)
    # the pipelined results are the device results of the chosen tier, bit for bit
    step(pl)
    torch.cuda.synchronize()
    last = 2 * e2e_steps
    e2e_same = all(bool(torch.equal(h_out[(last - 2 + d) % NQ], outs[d].cpu())) for d in range(2))

    # dominant kernel and its roofline
    info = pl[0].info
    totals = {}
    for d in stages:
        for kind, ts in stages[d].items():
            totals[kind] = totals.get(kind, 0.0) + sum(ts)
    dom = max(totals, key=totals.get)
    per_launch_ms = []
    work = 0
    for d in stages:
        if dom in stages[d]:
            per_launch_ms.extend(stages[d][dom])
    avg_ms = sum(per_launch_ms) / len(per_launch_ms)
    flops = kernel_work(info, dom, 0, (tuned.get(chosen) or [[4, 4]])[0][0])
    roofline = None
    if flops is not None and chosen in ("f64", "f64_df"):
        achieved = flops / (avg_ms / 1e3) / 1e12
        peak = FP64_PEAK_TFLOPS if chosen == "f64" else DF_PEAK_TFLOPS
        note = ("FP64 pipe: 152 SMs x 2 FMA/clk x 2 flop x 2070 MHz = 1.26 TFLOP/s (a dependent-FMA "
                "microbenchmark reached 1.01)") if chosen == "f64" else (
                "double-float on the FP32 pipe: 152 SMs x 128 lanes x 2070 MHz / 12 instructions per "
                "FP64-equivalent multiply-add x 2 flop = 6.71 TFLOP/s FP64-equivalent")
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": TRAFFIC.get((chosen, dom)),
                    "kernel": KIND_NAMES[dom], "avg_launch_ms": avg_ms, "flops_per_launch": flops,
                    "peak_kind": "derived from unit counts and the maximum SM clock (not measured)",
                    "peak_note": note}
        if chosen == "f64_df":
            # the same ceiling from a measured FP32 rate (SGEMM on the CUDA cores, TF32 off)
            f32 = measured_fp32_tflops(dev)
            roofline["measured_view"] = {"fp32_sgemm_tflops": f32, "peak": f32 / 12, "frac": achieved / (f32 / 12),
                                         "note": "double-float ceiling = measured FP32 FLOP/s / 12"}
        if TRAFFIC.get((chosen, dom)):
            # the same launch against HBM: its DRAM bytes (ncu) over its duration
            gbs = TRAFFIC[(chosen, dom)] / (avg_ms / 1e3) / 1e9
            roofline["hbm_view"] = {"achieved_gbs": gbs, "peak_gbs": HBM_PEAK_GBS, "frac": gbs / HBM_PEAK_GBS}
    # Every kernel kind: achieved rate against its own bound.  Coupling: HBM
    # (A-hat plus the w and c rows it reads and writes); the others: the ALU
    # peak of the tier, with the paper's flop counts (Sec. 4.2).
    M, s_, L_, N_, nc_ = info["M"], info["s"], info["L"], info["N"], info["n_c"]
    ld = (tuned.get(chosen) or [[4, 4]])[0][0]
    r0 = max(0, L_ - 1 - ld)
    elem = 8  # FP64 and double-float both store 8 bytes per value
    nseg_rows = sum((4 << g) - 2 for g in range(L_))
    kinds_work = {
        0: ("alu", 2 * 2 * M * s_ * ((2 << L_) - 2) + 2 * M * (M + 1) * sum((4 << g) - 4 for g in range(r0, L_ - 1))),
        1: ("alu", 2 * M * (M + 1) * sum((4 << g) - 4 for g in range(0, r0))),
        2: ("hbm", nc_ * M * M * elem + 2 * nseg_rows * 2 * M * elem),
        3: ("alu", 2 * M * (M + 1) * sum((4 << g) - 4 for g in range(1, max(1, r0)))),
        4: ("alu", kernel_work(info, 4, 0, ld)),
        7: ("alu", kernel_work(info, 7, 0, ld)),
    }
    per_kernel = {}
    alu_peak = FP64_PEAK_TFLOPS if chosen == "f64" else DF_PEAK_TFLOPS
    for kind, (bound, work) in kinds_work.items():
        if kind not in totals:
            continue
        t_s = totals[kind] / args.steps / 2 / 1e3   # seconds per direction
        if t_s <= 0:
            continue
        if bound == "hbm":
            ach = work / t_s / 1e9
            per_kernel[KIND_NAMES[kind]] = {"bound": "hbm", "achieved": ach, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                            "frac": ach / HBM_PEAK_GBS, "ms_per_direction": t_s * 1e3}
        else:
            ach = work / t_s / 1e12
            per_kernel[KIND_NAMES[kind]] = {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                                            "frac": ach / alu_peak, "ms_per_direction": t_s * 1e3}
    launches = sum(p.launches() for p in pl) * args.steps
    # Whole-step HBM fraction.  Algorithmic bytes per direction: input f and
    # output z (8 B each per coefficient), the Lambda table(s) (lambda for
    # L2C; u and v for C2L: 8 B per padded entry each) and the plan's A-hat in
    # FP64 (2592 B per submatrix) -- the FP64 plan's table bytes, whatever the
    # tier stores -- each read or written once.
    def dir_bytes(direction):
        return 16 * n + 8 * info["N"] * (1 if direction == "l2c" else 2) + info["n_c"] * info["M"] ** 2 * 8
    step_bytes = dir_bytes("l2c") + dir_bytes("c2l")
    hbm_step = {"bytes_per_step": step_bytes, "achieved_gbs": step_bytes / (ms_per_step / 1e3) / 1e9,
                "peak_gbs": HBM_PEAK_GBS, "frac": step_bytes / (ms_per_step / 1e3) / 1e9 / HBM_PEAK_GBS,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, of measured)",
                "definition": "f + z + lambda (or u, v) + FP64 A-hat, each once, both directions; / ms_per_step"}

    line = {
        "metric": "transformed coefficients/s (n=1e6, L2C+C2L, FP64-accurate)",
        "value": value, "unit": "coefficients/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_COEF_PER_S,
        "vs_baseline_note": "against the paper's one-core CPU figure (n = 1e6: 20 ms per transform, "
                            "5.0e7 coefficients/s; C2L the same): another machine's number, context only",
        "dtype": "f64_df" if chosen == "f64_df" else "f64",
        "data": "synthetic",
        "config": {"workload": "n=1e6 single vector, L2C and C2L, N(0,1)(j+1)^-1 seed 1",
                   "n": n, "batch": 1, "tier": chosen, "plan": {k: info[k] for k in ("N", "L", "s", "M", "n_c")},
                   "autotuned_chunks_l2c_c2l": tuned.get(chosen),
                   "streams": "L2C on the current stream, C2L on a second stream, joined each step",
                   "l2_flush": "256 MB write before every timed step", "parallelism": "replicas" if ws > 1 else "single"},
        "e2e": {"value": e2e_val, "unit": "coefficients/s", "h2d_bytes_per_step": 2 * 8 * n,
                "d2h_bytes_per_step": 2 * 8 * n, "matches_device_output": e2e_same, "pipelined": "host-to-device and device-to-host copy streams, two compute streams, 4-slot buffer ring",
                "note": "copies inside the timed region; consecutive steps overlap in the ring and L2 is not flushed between them, unlike the device-timed value"},
        "gpu_launches": launches,
        "tiers": tier_vals,
        "gegenbauer": geg,
        "values_at_chebyshev_points": values_leg,
        "modal_vs_nodal_f64": nodal,
        "plan_ms": plan_ms,
        "stage_ms_per_step": {KIND_NAMES[k]: v / args.steps for k, v in sorted(totals.items())},
        "ms_per_step_warm_l2": sum(ms_warm) / len(ms_warm),
        "one_transform_ms": one_ms,
        "coefficients_per_s_warm_l2": 2 * n / (sum(ms_warm) / len(ms_warm) / 1e3),
        "hbm_step": hbm_step,
        "roofline": roofline,
        "roofline_per_kernel": per_kernel,
        "clocks": clk,
        "wall_s_timed": wall,
    }

    if not args.no_batched:
        line["batched"] = batched_leg(lc, dev, flush, args)

    if rank == 0 and not args.no_cpu:
        pick, ref_l2c, ref_c2l, dt, cores = oracle_leg(n, x_host, args.cpu_rows)
        pl[0](x, out=outs[0])
        pl[1](x, out=outs[1])
        z = [outs[0].cpu().numpy()[pick], outs[1].cpu().numpy()[pick]]
        acc = {}
        for name, zz, rr in (("l2c", z[0], ref_l2c), ("c2l", z[1], ref_c2l)):
            d = zz - rr
            acc[name] = {"E_2": float(np.linalg.norm(d) / np.linalg.norm(rr)),
                         "E_inf": float(np.abs(d).max() / np.abs(rr).max()), "rows": int(pick.size)}
        line["accuracy"] = acc
        line["cpu_baseline"] = {"value": 2 * pick.size / dt, "unit": "coefficients/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "%d sampled output rows per direction of the n=1e6 transform "
                                          "(direct double-double row sums, %.1f s)" % (pick.size, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def profile_run(spec):
    """Two executions of one plan on synthetic data (a small, fixed target for profilers)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_00033_gb300 as lc
    import workloads
    parts = spec.split(":")
    tier, direction, n, batch = parts[:4]
    n, batch = int(n), int(batch)
    dev = torch.device("cuda", 0)
    dt = torch.float32 if tier == "f32" else torch.float64
    x = workloads.decaying_vector(n, seed=1, r=1.0, batch=None if batch == 1 else batch)
    xt = torch.as_tensor(x, device=dev, dtype=dt)
    plan = lc.Plan(n, direction, batch, tier, dev)
    if len(parts) > 4 and parts[4] == "levels":  # split tier: one launch per level
        plan.set_split_schedule(False)
    out = torch.empty_like(xt)
    for _ in range(2):
        plan(xt, out=out)
    torch.cuda.synchronize()
    plan.check()
    print(json.dumps({"profile": spec, "launches_per_execute": plan.launches()}))


def main():
    args = parse()
    if args.profile:
        profile_run(args.profile)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
