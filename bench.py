"""Throughput bench: one shared homogeneous support, a batch of signals.

Workload (default): N = 2^20, k = 2^12, batch 4096, complex64 samples already
resident in HBM; one step = one call of the strided transform over the whole
batch. Prints ONE JSON line (rank 0).

Legs:
  * value        device-timed coeffs/s of the batched complex64 path: the K
                 steps run back to back as one region bracketed by CUDA events
                 on the launching stream, rotating over 4 input/output pairs
                 (each step's input, larger than L2, last touched 3 steps
                 earlier: no flush); the per-step figure after a 256 MiB L2
                 write flush is reported beside it
  * e2e          the same through the public API with pinned host buffers
                 (one sdft_execute_strided_host call: H2D of the samples, the
                 transform and D2H of the coefficients, overlapped in chunks,
                 inside the timing)
  * fp64         the plain per-instance complex128 path (one call per instance),
                 the batched complex128 path on the FP64 pipe and in
                 double-float arithmetic, device-timed
  * extras       (N = 1) synthesis, a cuFFT context figure, the single-instance
                 latency, the uneven batch, the large-k plans, Shift-and-Sample
                 and the serving engine
  * roofline     algorithmic bytes / kernel time against measured HBM bandwidth
  * cpu_baseline the FP64 oracle on the host cores: its plain-C Algorithm 1
                 (OpenMP) on the whole batch, its dense k x k solve on a
                 sample, each with its relative L2 against the GPU output
`--impl reference` times only the oracle (the reference arm of this tier).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "coeffs/s batched FP32 vs plain per-instance FP64 at relL2≤1e-5; p50/p99 latency"
UNIT = "coeffs/s"
L2_FLUSH_BYTES = 256 << 20
ROTATE_SETS = 4          # input/output pairs the headline steps rotate over


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        if os.environ.get("CUDA_INJECTION64_PATH") or os.environ.get("SDFT_NO_CLOCKS"):
            return self          # under a profiler: do not poll the GPU through NVML
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(ws: int, units_per_step_per_rank: int, steps: int, seconds_this_rank: float) -> float:
    """Whole-job throughput of N independent replicas (weak scaling): the
    units all ranks processed divided by the slowest rank's time."""
    return ws * units_per_step_per_rank * steps / _max_over_ranks(ws, seconds_this_rank)


def time_device_steps(fn, steps, warmup, flush, stream):
    """Per-step CUDA-event timing on `stream`, L2 flushed (untimed) between steps."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in ev]


def run_ours(args):
    import torch
    from paper_2211_15299_gb300 import Plan

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    M, s, batch = args.log2n, args.log2k, args.batch
    inst, _ = W.workload_shared(M=M, s=s, batch=1, coeffs=False)
    k = inst.k
    plan32 = Plan(M, inst.J, "c64")
    plan64 = Plan(M, inst.J, "c128")
    n_levels = 1 + max(0, -(-(s - 12) // 8)) if s > 4 else 1

    # Synthetic samples: any vector of k samples is the sample set of exactly one
    # signal supported on J (F(J, I) is invertible), so complex Gaussian samples are
    # a valid input; seeded per rank (replicas, weak scaling).
    g = torch.Generator(device=dev)
    g.manual_seed(W.BASE_SEED + 2 + 1000 * rank)
    xs = [torch.randn((batch, k), dtype=torch.complex64, device=dev, generator=g) for _ in range(ROTATE_SETS)]
    ys = [torch.empty_like(xs[0]) for _ in range(ROTATE_SETS)]
    x32, y32 = xs[0], ys[0]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(s=None, i=0):
        plan32.execute_strided(xs[i], ys[i], stream=(s or stream).cuda_stream)

    # the tile parameters (stages per pass) chosen by the library's autotuner on
    # this workload; both choices are also timed the bench's way, below
    from paper_2211_15299_gb300 import _native as N
    N.sdft_plan_autotune(plan32.handle, batch, x32, y32, stream.cuda_stream, 5)
    tuned_spp = N.sdft_plan_get_stages_per_pass(plan32.handle)
    by_spp = {}
    for spp in (4, 3):
        N.sdft_plan_set_stages_per_pass(plan32.handle, spp)
        by_spp[spp] = 1e3 * time_rotating([lambda s=None, i=i: step(s, i) for i in range(ROTATE_SETS)],
                                          max(5, args.steps // 2), args.warmup, stream) / max(5, args.steps // 2)
    N.sdft_plan_set_stages_per_pass(plan32.handle, tuned_spp)
    tuning = {"stages_per_pass": tuned_spp, "chosen_by": "sdft_plan_autotune",
              "ms_by_stages_per_pass": {str(k): v for k, v in by_spp.items()}}

    _barrier(ws)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        _barrier(ws)
        # one step = one replay of a CUDA graph holding the strided call (the
        # host-side checks and tensor-map encoding happen once, at capture)
        region = time_rotating([lambda s=None, i=i: step(s, i) for i in range(ROTATE_SETS)],
                               args.steps, args.warmup, stream)
        _barrier(ws)
        torch.cuda.synchronize()
    total = _max_over_ranks(ws, region)
    coeffs_per_step = batch * k
    value = replica_throughput(ws, coeffs_per_step, args.steps, region)
    ms_per_step = 1e3 * total / args.steps
    # the same steps timed one by one after a 256 MiB L2 write flush (the
    # flush's dirty lines are written back inside each timed step)
    flushed = time_graph(step, args.steps, args.warmup, flush, stream)

    # roofline of the dominant kernel (the single level-0 launch per step here)
    peak, peak_kind = _peaks()
    alg_bytes = 16 * coeffs_per_step + 8 * (k - 1)
    achieved = alg_bytes / (region / args.steps) / 1e9
    traffic = _committed_traffic(M, s, batch)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "k_level<float,0,12,true>" if n_levels == 1 else "multi-level",
                "alg_bytes_per_launch": alg_bytes,
                "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                "ms_per_step_after_l2_write_flush": 1e3 * statistics.mean(flushed)}

    # context for the ridge point: the FP32 CUDA-core rate, an 8192^3 FP32 matrix
    # product with TF32 off (a cuBLAS library call on the FMA pipes, no tensor cores)
    roofline["fp32_fma_peak"] = _fp32_fma_peak(dev, stream, peak)

    if args.only_fp32:
        if rank == 0:
            print(json.dumps({"value": value, "unit": UNIT, "ms_per_step": ms_per_step, "roofline": roofline,
                              "tuning": tuning}))
        return
    # FP64: batched and plain per-instance (one call per instance), device-timed
    x64 = x32.to(torch.complex128)
    y64 = torch.empty_like(x64)

    def step64():
        plan64.execute_strided(x64, y64, stream=stream.cuda_stream)

    t64 = time_device_steps(step64, max(2, args.steps // 4), 2, flush, stream)
    fp64_batched = coeffs_per_step / statistics.mean(t64)
    n_pi = min(batch, 512)

    def step64_per_instance():
        for b in range(n_pi):
            plan64.execute(x64[b], y64[b], stream=stream.cuda_stream)

    tpi = time_device_steps(step64_per_instance, 3, 1, flush, stream)
    fp64_per_instance = n_pi * k / statistics.mean(tpi)
    # complex128 in double-float arithmetic on the FP32 pipes (SDFT_PLAN_FP64_DF)
    plan_df = Plan(M, inst.J, "c128", fp64_df=True)
    y_df = torch.empty_like(x64)

    def step_df():
        plan_df.execute_strided(x64, y_df, stream=stream.cuda_stream)

    tdf = time_device_steps(step_df, max(2, args.steps // 4), 2, flush, stream)
    fp64_df = coeffs_per_step / statistics.mean(tdf)
    step64()
    step_df()
    torch.cuda.synchronize()
    rel_df_vs_fp64 = float(torch.linalg.vector_norm(y_df - y64) / torch.linalg.vector_norm(y64))
    del y_df, plan_df
    # synthesis (the inverse map) on the same batches, graph-replayed, timed
    # like the headline (rotating over the coefficient sets)
    zs = [torch.empty_like(x32) for _ in range(ROTATE_SETS)]

    def step_syn(s=None, i=0):
        plan32.synthesize(ys[i], zs[i], stream=(s or stream).cuda_stream)

    ts, ts_fl = time_steady_and_flushed([lambda s=None, i=i: step_syn(s, i) for i in range(ROTATE_SETS)],
                                        max(3, args.steps // 4), 3, flush, stream)
    synthesis = {"coeffs_per_s": coeffs_per_step / ts, "ms_per_step": 1e3 * ts,
                 "frac_of_peak": alg_bytes / ts / 1e9 / peak, "ms_per_step_after_l2_write_flush": 1e3 * ts_fl}
    del zs
    # context only: a library batched k-point C2C FFT (cuFFT through torch.fft)
    # over the same batch moves the same bytes with a regular twiddle pattern
    yfft = torch.empty_like(x32)

    def step_fft():
        torch.fft.fft(x32, dim=1, out=yfft)

    tf = time_device_steps(step_fft, max(3, args.steps // 4), 3, flush, stream)
    fft_ceiling = {"what": f"torch.fft.fft batch {batch} x {k} complex64 (cuFFT library call)",
                   "coeffs_per_s": coeffs_per_step / statistics.mean(tf),
                   "GB_per_s": 16 * coeffs_per_step / statistics.mean(tf) / 1e9}
    del yfft
    # accuracy of the FP32 path against the FP64 path on the same input
    step()
    step64()
    torch.cuda.synchronize()
    d = (y32.to(torch.complex128) - y64)
    rel_fp32_vs_fp64 = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(y64))

    # e2e through the public API: pinned host -> device, transform, device -> host
    h_in = x32.cpu().pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty_like(x32)
    d_out = torch.empty_like(x32)

    def e2e_step():
        # one C-ABI call on host buffers: copy-in, transform and copy-out in
        # overlapped chunks (sdft_execute_strided_host)
        plan32.execute_host(h_in, h_out, d_in, d_out, stream=stream.cuda_stream)

    te = time_device_steps(e2e_step, max(3, args.steps // 4), 2, flush, stream)
    e2e_total = _max_over_ranks(ws, sum(te))
    e2e_val = ws * coeffs_per_step * len(te) / e2e_total

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(inst, x32, y32, min(args.cpu_sample, batch))
    extra = {}
    if not args.no_extra and ws == 1:      # the other workloads run at N = 1 only
        del x64, y64, h_in, h_out, d_in, d_out
        torch.cuda.empty_cache()
        extra["single"] = run_single(args)
        extra["uneven"] = run_uneven(args)
        extra["large_k"] = run_large(args)
        extra["serving"] = run_serving(args)
        extra["sas"] = run_sas(args)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(M, s, batch, ws),
        "pivots": [int(p) for p in inst.pivots],
        "tuning": tuning,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(8 * coeffs_per_step),
                "d2h_bytes_per_step": int(8 * coeffs_per_step)},
        "gpu_launches": int(args.steps * n_levels),
        "roofline": roofline,
        "fp64": {"batched_coeffs_per_s": fp64_batched, "per_instance_coeffs_per_s": fp64_per_instance,
                 "fp64_fma_peak": _fp32_fma_peak(dev, stream, peak, torch.float64, 4096),
                 "per_instance_sample": n_pi, "fp32_speedup_vs_per_instance": value / ws / fp64_per_instance,
                 "batched_double_float_coeffs_per_s": fp64_df, "rel_l2_double_float_vs_fp64": rel_df_vs_fp64},
        "rel_l2_fp32_vs_fp64": rel_fp32_vs_fp64,
        "fft_ceiling": fft_ceiling,
        "synthesis": synthesis,
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    out.update(extra)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _config(M, s, batch, ws):
    """The workload of the headline line, the same in both arms."""
    return {"workload": f"shared support N=2^{M} k=2^{s} batch {batch} complex64 (strided, one plan)",
            "log2N": M, "log2k": s, "batch": batch,
            "l2": f"inputs larger than L2, no flush: steps rotate over {ROTATE_SETS} input/output pairs, "
                  f"each step's input last touched {ROTATE_SETS - 1} steps earlier",
            "parallelism": f"replicas x{ws}"}


def _committed_traffic(M, s, batch):
    """DRAM bytes per launch from the committed ncu summary, if it still matches the kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        import hashlib
        with open(os.path.join(ROOT, "paper_2211_15299_gb300", "csrc", "kernels.cuh"), "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()[:16]
        e = d.get(f"{M}/{s}/{batch}")
        if e and e.get("kernels_cuh_sha") == h:
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def _fp32_fma_peak(dev, stream, hbm_gbs, dtype=None, n=8192):
    """Measured CUDA-core throughput (TFLOP/s) of a square matrix product in
    `dtype` (FP32 by default, TF32 disabled; FP64 for the complex128 path), and
    the ridge point it gives against the HBM peak."""
    import torch
    dtype = dtype or torch.float32
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        g = torch.Generator(device=dev)
        g.manual_seed(W.BASE_SEED + 9)
        a = torch.randn((n, n), dtype=dtype, device=dev, generator=g)
        b = torch.randn((n, n), dtype=dtype, device=dev, generator=g)
        c = torch.empty_like(a)
        for _ in range(2):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) * 1e-3 / reps
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    tflops = 2.0 * n ** 3 / sec / 1e12
    name = str(dtype).replace("torch.", "")
    return {"tflops": tflops, "how": f"torch.matmul {name} {n}^3, TF32 off (cuBLAS), mean of {reps}",
            "ridge_flop_per_byte": tflops * 1e12 / (hbm_gbs * 1e9)}


def _capture(fn):
    """A CUDA graph holding one call of `fn` (called once untimed first: it
    builds any cached work queue)."""
    import torch
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fn(s)
    torch.cuda.synchronize()
    return g


def time_graph(fn, steps, warmup, flush, stream):
    """Capture `fn` in a CUDA graph and time replays (events on `stream`, L2 flushed between)."""
    g = _capture(fn)
    return time_device_steps(lambda: g.replay(), steps, warmup, flush, stream)


def time_rotating(fns, steps, warmup, stream):
    """Steady-state timing over inputs larger than L2: one CUDA graph per buffer
    set, step i replays set i mod len(fns), and the `steps` replays run back to
    back as ONE region bracketed by CUDA events on `stream` (no flush: a set's
    input was last touched len(fns) - 1 steps earlier, with several L2
    capacities of traffic in between, and every step writes back the dirty
    output lines the step before it left in L2). Returns the region's seconds."""
    import torch
    graphs = [_capture(fn) for fn in fns]
    for i in range(warmup):
        graphs[i % len(graphs)].replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(steps):
        graphs[i % len(graphs)].replay()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) * 1e-3


def steady_sets(bytes_per_set):
    """Buffer sets a steady-state timing rotates over: enough that at least
    1 GiB (several L2 capacities) of traffic passes between two uses of a set."""
    return max(1, min(32, -(-(1 << 30) // max(1, bytes_per_set)) + 1)) if bytes_per_set < (1 << 30) else 1


def time_steady_and_flushed(fns, steps, warmup, flush, stream):
    """(steady-state seconds per step over the rotating sets `fns`, seconds per
    step of set 0 timed one by one after the 256 MiB L2 write flush)."""
    steady = time_rotating(fns, steps, warmup, stream) / steps
    flushed = statistics.mean(time_graph(fns[0], steps, warmup, flush, stream))
    return steady, flushed


def run_single(args):
    """Single-instance leg: N = 2^10, k = 2^5, complex128 (latency): one
    execute per step as a CUDA-graph replay, and the relative L2 against the
    oracle's dense solve."""
    import torch
    import oracle as O
    from paper_2211_15299_gb300 import Plan
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    inst = W.workload_single()
    plan = Plan(inst.M, inst.J, "c128")
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    I = O.sample_set(inst.M, inst.pivots)
    pos = {int(j): i for i, j in enumerate(inst.J)}
    c = np.asarray([inst.coeffs[pos[int(j)]] for j in Jc])
    f = O.synthesize(inst.M, Jc, c, I)
    x = torch.from_numpy(f).to(dev)
    y = torch.empty_like(x)

    def step(s=None):
        plan.execute_strided(x, y, stream=(s or stream).cuda_stream)

    t = time_graph(step, max(10, args.steps), args.warmup, flush, stream)
    got = y.cpu().numpy()
    return {"workload": f"N=2^{inst.M} k=2^{inst.s} complex128, one instance", "us_per_call": 1e6 * statistics.median(t),
            "rel_l2_vs_oracle": float(np.linalg.norm(got - c) / np.linalg.norm(c)), "launches_per_call": 1}


def run_large(args):
    """Large-k leg: N = 2^30, k = 2^20, batch 64, complex64, contiguous and spread pivots."""
    import torch
    from paper_2211_15299_gb300 import Plan
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for contiguous in (True, False):
        inst, _ = W.workload_large(contiguous=contiguous, batch=1, coeffs=False)
        plan = Plan(inst.M, inst.J, "c64")
        g = torch.Generator(device=dev)
        g.manual_seed(W.BASE_SEED + 3)
        x = torch.randn((args.large_batch, inst.k), dtype=torch.complex64, device=dev, generator=g)
        y = torch.empty_like(x)

        def step(s=None):
            plan.execute_strided(x, y, stream=(s or stream).cuda_stream)

        coeffs = args.large_batch * inst.k
        # both strategies x three or four stages per pass, each graph-replayed,
        # steps back to back (the input, 537 MB, is far larger than L2; the
        # queue strategy's first call builds its queue, so it runs before
        # capture); the leg reports the fastest
        from paper_2211_15299_gb300 import _native as N
        by = {}
        for name in ("levels", "queue"):
            plan.set_strategy(name)
            for spp in (4, 3):
                N.sdft_plan_set_stages_per_pass(plan.handle, spp)
                step()
                torch.cuda.synchronize()
                by[f"{name}/{spp}"] = time_rotating([step], args.steps, args.warmup, stream) / args.steps
        best = min(by, key=by.get)
        mean = by[best]
        plan.set_strategy(best.split("/")[0])
        N.sdft_plan_set_stages_per_pass(plan.handle, int(best.split("/")[1]))
        flushed = statistics.mean(time_graph(step, args.steps, args.warmup, flush, stream))
        step()
        # the oracle on the host cores: 16 of the instances (the last strategy's output)
        torch.cuda.synchronize()
        nrow = min(16, args.large_batch)
        dt, used, rel = _cpu_oracle_rows(inst.M, inst.pivots, inst.J, x[:nrow].cpu().numpy(), y[:nrow].cpu().numpy())
        cpu_oracle = {"value": nrow * inst.k / dt, "unit": UNIT, "kind": "oracle", "cores": used,
                      "sample": f"{nrow} of the {args.large_batch} instances, Algorithm 1 in the oracle's plain C "
                                "(FP64, OpenMP)", "seconds": dt, "rel_l2_gpu_vs_oracle": rel}
        res["contiguous" if contiguous else "spread"] = {
            "coeffs_per_s": coeffs / mean, "ms_per_step": 1e3 * mean, "strategy": best.split("/")[0],
            "stages_per_pass": int(best.split("/")[1]),
            "ms_by_strategy_and_stages_per_pass": {k: 1e3 * v for k, v in by.items()}, "cpu_oracle": cpu_oracle,
            "ms_per_step_after_l2_write_flush": 1e3 * flushed,
            "alg_GBps": 16 * coeffs / mean / 1e9, "frac_of_peak": 16 * coeffs / mean / 1e9 / _peaks()[0],
            "pivots": [int(p) for p in inst.pivots]}
        assert plan.device_status() == 0
    return res


def _cpu_oracle_rows(M, pivots, J, F, got, threads=None):
    """The oracle's plain-C Algorithm 1 (FP64, OpenMP over instances) on the
    rows F (B, k) of one support: (seconds, threads, relative L2 of the GPU rows
    `got` against it)."""
    threads = threads or os.cpu_count()
    import oracle as O
    from oracle import alg1
    Jc = O.canonical_support_by_key(J, pivots)
    F = np.ascontiguousarray(F, dtype=np.complex128)
    alg1.alg1_batch(M, pivots, Jc, F[:1], threads=threads)      # warm-up
    t0 = time.perf_counter()
    C, used = alg1.alg1_batch(M, pivots, Jc, F, threads=threads)
    dt = time.perf_counter() - t0
    got = np.asarray(got, dtype=np.complex128).reshape(C.shape)
    return dt, used, float(np.linalg.norm(got - C) / np.linalg.norm(C))


def run_uneven(args):
    """Uneven batch: 10,000 instances with their own supports (M in 12..24, s in 4..16),
    one persistent work-queue launch per step, complex64."""
    import torch
    from paper_2211_15299_gb300 import Batch, Plan
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    insts = W.workload_uneven(count=args.uneven_count)
    plans = [Plan(i.M, i.J, "c64") for i in insts]
    t_plan = time.perf_counter() - t0
    b = Batch(plans)
    n_items, n_ctr, grid = b.stats()
    g = torch.Generator(device=dev)
    g.manual_seed(W.BASE_SEED + 4)
    x = torch.randn(b.total, dtype=torch.complex64, device=dev, generator=g)
    y = torch.empty_like(x)

    # autotune the queue shape (item order x CTAs) on these buffers, then capture
    t0 = time.perf_counter()
    schedule, grid, ms_tuned = b.autotune(x, y, reps=3)
    t_tune = time.perf_counter() - t0
    n_items, n_ctr, grid = b.stats()
    from paper_2211_15299_gb300 import _native as N
    spp_tuned = N.sdft_batch_get_stages_per_pass(b.handle)
    staged_tuned = N.sdft_batch_get_table_staging(b.handle)
    lag_tuned = N.sdft_batch_get_lag(b.handle)

    def step(s=None):
        b.execute(x, y, stream=(s or stream).cuda_stream)

    # steps back to back (the packed input is far larger than L2)
    mean, flushed = time_steady_and_flushed([step], args.steps, args.warmup, flush, stream)
    total = b.total
    tw_bytes = sum(8 * (p.k - 1) for p in plans)
    # the oracle on the host cores: the first 64 instances, one call each
    torch.cuda.synchronize()
    xh, yh = x.cpu().numpy(), y.cpu().numpy()
    n_cpu, t_cpu, used_max, rel_max, coeffs_cpu = min(64, len(insts)), 0.0, 0, 0.0, 0
    for i in range(n_cpu):
        a, z = b.offsets[i], b.offsets[i] + plans[i].k
        dt, used, rel = _cpu_oracle_rows(insts[i].M, insts[i].pivots, insts[i].J, xh[None, a:z], yh[None, a:z],
                                         threads=1)      # one instance per call: one thread
        t_cpu += dt
        used_max = max(used_max, used)
        rel_max = max(rel_max, rel)
        coeffs_cpu += plans[i].k
    cpu_oracle = {"value": coeffs_cpu / t_cpu, "unit": UNIT, "kind": "oracle", "cores": used_max,
                  "sample": f"the first {n_cpu} instances (the largest k), one call and one thread each, "
                            "Algorithm 1 in the oracle's plain C (FP64)",
                  "seconds": t_cpu, "max_rel_l2_gpu_vs_oracle": rel_max}
    return {"instances": len(plans), "coeffs_per_step": total, "coeffs_per_s": total / mean,
            "cpu_oracle": cpu_oracle,
            "ms_per_step": 1e3 * mean, "alg_GBps": (16 * total + tw_bytes) / mean / 1e9,
            "frac_of_peak": (16 * total + tw_bytes) / mean / 1e9 / _peaks()[0],
            "ms_per_step_after_l2_write_flush": 1e3 * flushed,
            "alg_bytes_per_step": 16 * total + tw_bytes, "work_items": n_items,
            "dependency_counters": n_ctr, "grid": grid, "plan_build_s": t_plan,
            "autotune": {"schedule": schedule, "grid": grid, "stages_per_pass": spp_tuned,
                         "table_staging": staged_tuned, "lag": lag_tuned, "ms_per_run": ms_tuned,
                         "seconds": t_tune},
            "launches_per_step": 1, "graph": "one CUDA graph replay per step"}


def run_sas(args):
    """Shift-and-Sample leg: supports that are not homogeneous (N = 2^20,
    k about 3000): an arithmetic progression (complete isolation, mu* = 1), a
    random subset of a homogeneous set and a union of homogeneous sets (mu*
    shifted transforms and per-class solves); complex64, a batch of instances
    sharing the support."""
    import torch
    from paper_2211_15299_gb300 import Sas
    dev = torch.device("cuda", torch.cuda.current_device())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for kind in ("ap", "subset", "uoh"):
        J = W.workload_sas(kind)
        t0 = time.perf_counter()
        p = Sas(20, J, "c64")
        t_plan = time.perf_counter() - t0
        g = torch.Generator(device=dev)
        g.manual_seed(W.BASE_SEED + 6)
        # buffer sets (samples, workspace, coefficients) rotated over so that no
        # step finds its input in L2; set 0 is checked against the oracle
        n_sets = steady_sets(8 * args.sas_batch * (2 * p.n_samples + p.k))
        xs = [torch.randn((args.sas_batch, p.n_samples), dtype=torch.complex64, device=dev, generator=g)
              for _ in range(n_sets)]
        ws_ = [torch.empty_like(xs[0]) for _ in range(n_sets)]
        ys = [torch.empty((args.sas_batch, p.k), dtype=torch.complex64, device=dev) for _ in range(n_sets)]
        x, y = xs[0], ys[0]

        def step(s=None, i=0):
            p.execute(xs[i], ys[i], work=ws_[i], stream=(s or stream).cuda_stream)

        mean, flushed = time_steady_and_flushed([lambda s=None, i=i: step(s, i) for i in range(n_sets)],
                                                args.steps, args.warmup, flush, stream)
        coeffs = args.sas_batch * p.k
        alg = 8 * args.sas_batch * (p.n_samples + p.k)        # samples in, coefficients out
        peak, peak_kind = _peaks()
        entry = {"k": p.k, "R": p.R, "mu_star": p.mu_star, "samples_per_instance": p.n_samples,
                 "max_cond": p.max_cond, "batch": args.sas_batch, "coeffs_per_s": coeffs / mean,
                 "ms_per_step": 1e3 * mean, "plan_s": t_plan, "buffer_sets": n_sets,
                 "ms_per_step_after_l2_write_flush": 1e3 * flushed,
                 "roofline": {"bound": "hbm", "achieved": alg / mean / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": alg / mean / 1e9 / peak, "peak_kind": peak_kind,
                              "alg_bytes_per_step": alg},
                 "launches_per_step": p.launches + (1 if p.R > 12 else 0),
                 "gathered_stage_one": p.gathered}
        if not args.no_cpu:
            # the oracle's SAS (numpy FP64) on a few of the same instances
            import oracle as O
            n_cpu = 4
            order = [int(j) for j in p.support_order]
            r = [int(v) for v in p.pivots]
            f = x[:n_cpu].cpu().numpy().astype(np.complex128).reshape(n_cpu, p.mu_star, -1)
            t0 = time.perf_counter()
            ref = np.stack([O.sas_transform(20, order, r, f[b]) for b in range(n_cpu)])
            dt = time.perf_counter() - t0
            step()
            torch.cuda.synchronize()
            got = y[:n_cpu].cpu().numpy().astype(np.complex128)
            entry["cpu_oracle"] = {"value": n_cpu * p.k / dt, "unit": UNIT, "kind": "oracle",
                                   "sample": f"{n_cpu} instances, numpy FP64", "seconds": dt,
                                   "rel_l2_gpu_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}
        res[kind] = entry
    return res


def run_serving(args):
    """Serving leg: Poisson arrivals (rate, duration) of requests whose supports have
    N in 2^10..2^26 and k in 2^4..2^18; 80% reuse one of 256 resident plans, 20% bring
    a new support planned on arrival by the engine's own planner threads (the
    planning time counting in the latency); samples start in pinned host memory;
    a device-memory admission budget bounds the requests in flight."""
    import threading as th
    import torch
    from paper_2211_15299_gb300 import Plan, Server, _native as N
    rng = W.rng_for(5, 9)
    trace = W.workload_serving(rate=args.serve_rate, duration=args.serve_seconds)
    n_req = len(trace.arrivals)
    t0 = time.perf_counter()
    resident = [Plan(i.M, i.J, "c64") for i in trace.plans[:256]]
    t_resident = time.perf_counter() - t0

    def pinned(k):
        return torch.randn(k, dtype=torch.complex64).pin_memory()

    res_in = [pinned(p.k) for p in resident]
    res_out = [torch.empty(p.k, dtype=torch.complex64).pin_memory() for p in resident]
    pool = {}                                  # s -> list of free (in, out) pinned pairs
    pool_mu = th.Lock()
    late_allocs = [0]                          # pinned pairs allocated during the arrivals

    def take(s):
        with pool_mu:
            lst = pool.setdefault(s, [])
            if lst:
                return lst.pop()
            late_allocs[0] += 1
        return pinned(1 << s), torch.empty(1 << s, dtype=torch.complex64).pin_memory()

    # pinned buffers for fresh requests, allocated before the arrivals start (a
    # pinned allocation takes milliseconds and would stall the client): enough
    # per size for the most requests the engine holds in flight at this load
    for s_ in sorted(set(int(trace.plans[int(p)].s) for p in trace.plan_ids if p >= 256)):
        pool[s_] = [(pinned(1 << s_), torch.empty(1 << s_, dtype=torch.complex64).pin_memory())
                    for _ in range(32)]
    # fresh supports are planned by the engine's own planner threads (deferred
    # plans: tables built on the host, uploaded into the arena with the request)
    srv = Server("c64", budget_bytes=args.serve_budget << 20, n_slots=2, max_batch=args.serve_batch,
                 n_planners=args.serve_planners)
    h = srv.handle
    arrival = np.zeros(n_req)
    submit_t = np.zeros(n_req)
    fresh_bufs = {}
    fresh_s = {}
    fresh_J = {pid: np.ascontiguousarray(np.asarray(trace.plans[pid].J, dtype=np.uint64))
               for pid in set(int(p) for p in trace.plan_ids if p >= 256)}

    lat = np.zeros(n_req)
    done = np.zeros(n_req, dtype=bool)
    status = np.zeros(n_req, dtype=np.int32)
    stop = th.Event()

    lat_srv = np.zeros(n_req)

    def poller():
        # completions recorded with array operations (the client's own Python
        # work must not hold up the thread that submits the arrivals)
        while not stop.is_set() or not done.all():
            tags, l, st = N.sdft_server_poll(h, 8192)
            if len(tags):
                t = np.asarray(tags, dtype=np.int64)
                lat_srv[t] = l
                lat[t] = np.asarray(l) + (submit_t[t] - arrival[t])
                status[t] = st
                done[t] = True
                fr = t[is_fresh_req[t]]
                if len(fr):
                    with pool_mu:
                        for r_ in fr.tolist():
                            pool.setdefault(fresh_s.pop(r_), []).append(fresh_bufs.pop(r_))
            else:
                time.sleep(0.0002)
            if stop.is_set() and time.perf_counter() > deadline:
                break

    is_fresh_req = np.asarray(trace.plan_ids) >= 256
    deadline = float("inf")
    # the open-loop client: frequent GIL hand-offs between it and the poller,
    # and no garbage-collection pause while the arrivals run
    import gc
    switch = sys.getswitchinterval()
    sys.setswitchinterval(0.0002)
    gc_was = gc.isenabled()
    gc.disable()
    try:
        pt = th.Thread(target=poller, daemon=True)
        pt.start()
        start = time.perf_counter() + 0.05
        for r in range(n_req):
            t_arr = start + trace.arrivals[r]
            arrival[r] = t_arr
            while True:
                now = time.perf_counter()
                if now >= t_arr:
                    break
                if t_arr - now > 0.0005:
                    time.sleep(t_arr - now - 0.0003)
            pid = int(trace.plan_ids[r])
            if pid < 256:
                submit_t[r] = time.perf_counter()
                N.sdft_server_submit(h, resident[pid].handle, res_in[pid].data_ptr(), res_out[pid].data_ptr(), r)
            else:
                inst = trace.plans[pid]
                s_ = int(inst.s)
                bi, bo = take(s_)
                fresh_bufs[r] = (bi, bo)
                fresh_s[r] = s_
                submit_t[r] = time.perf_counter()
                N.sdft_server_submit_support(h, inst.M, fresh_J[pid], bi.data_ptr(), bo.data_ptr(), r)
        srv.drain(timeout_ms=600_000)
        end = time.perf_counter()
        deadline = end + 5.0
        stop.set()
        pt.join(timeout=10)
    finally:
        sys.setswitchinterval(switch)
        if gc_was:
            gc.enable()
    st = srv.stats()
    ok = status == 0
    ks = np.array([(resident[int(p)].k if p < 256 else (1 << trace.plans[int(p)].s)) for p in trace.plan_ids])
    wall = end - start
    is_fresh = np.array([p >= 256 for p in trace.plan_ids])
    split = {}
    for name, sel in (("resident", ok & ~is_fresh), ("fresh", ok & is_fresh)):
        if sel.any():
            pre = submit_t[sel] - arrival[sel]
            split[name] = {"p50_ms": float(np.percentile(lat[sel], 50) * 1e3),
                           "p99_ms": float(np.percentile(lat[sel], 99) * 1e3), "count": int(sel.sum()),
                           # arrival -> submit (client dispatch, and planning for fresh supports)
                           "client_p50_ms": float(np.percentile(pre, 50) * 1e3),
                           "client_p99_ms": float(np.percentile(pre, 99) * 1e3),
                           # submit -> completion stamp inside the server
                           "server_p50_ms": float(np.percentile(lat_srv[sel], 50) * 1e3),
                           "server_p99_ms": float(np.percentile(lat_srv[sel], 99) * 1e3)}
    out = {"requests": n_req, "offered_rate": args.serve_rate, "seconds": args.serve_seconds,
           "by_kind": split,
           "completed": int(done.sum()), "failed": int((~ok).sum()),
           "p50_ms": float(np.percentile(lat[ok], 50) * 1e3) if ok.any() else None,
           "p99_ms": float(np.percentile(lat[ok], 99) * 1e3) if ok.any() else None,
           "mean_ms": float(lat[ok].mean() * 1e3) if ok.any() else None,
           "coeffs_per_s": float(ks[ok].sum() / wall), "achieved_rate": float(ok.sum() / wall),
           "fresh_plans": int(sum(1 for p in trace.plan_ids if p >= 256)), "planned_by_server": st["planned"],
           "planner_threads": args.serve_planners,
           "micro_batches": st["micro_batches"], "max_inflight": st["max_inflight"],
           "arena_peak_MiB": st["arena_peak_bytes"] / 2**20, "budget_MiB": args.serve_budget,
           "resident_plan_build_s": t_resident, "device_status": srv.device_status(),
           "client_pinned_allocs_during_run": late_allocs[0]}
    srv.close()
    return out


def cpu_baseline(inst, x32, y32, sample):
    """The FP64 oracle on the host cores: its C restatement of Algorithm 1
    (OpenMP over instances, all cores) on the whole batch as the baseline; its
    dense solve on `sample` instances and its numpy Algorithm 1 beside it."""
    import oracle as O
    from oracle import alg1
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    I = O.sample_set(inst.M, inst.pivots)
    Fa = x32.cpu().numpy().astype(np.complex128)
    got_all = y32.cpu().numpy().astype(np.complex128)
    alg1.alg1_batch(inst.M, inst.pivots, Jc, Fa[:64], threads=os.cpu_count())      # warm-up
    # one pass over the batch takes milliseconds: repeat it for about a second
    # (at most 200 passes) and take the median pass
    runs = []
    while len(runs) < 200 and (len(runs) < 3 or sum(runs) < 1.0):
        t0 = time.perf_counter()
        Cc, used = alg1.alg1_batch(inst.M, inst.pivots, Jc, Fa, threads=os.cpu_count())
        runs.append(time.perf_counter() - t0)
    dc = statistics.median(runs)
    rel_c = float(np.linalg.norm(got_all - Cc) / np.linalg.norm(Cc))
    F = Fa[:sample]
    t0 = time.perf_counter()
    C = O.solve(inst.M, Jc, I, F)
    dt = time.perf_counter() - t0
    rel = float(np.linalg.norm(got_all[:sample] - C) / np.linalg.norm(C))
    t0 = time.perf_counter()
    Ca = O.transform_levels(inst.M, inst.pivots, Jc, Fa)
    da = time.perf_counter() - t0
    rel_a = float(np.linalg.norm(got_all - Ca) / np.linalg.norm(Ca))
    return {"value": Fa.shape[0] * inst.k / dc, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"all {Fa.shape[0]} instances, Algorithm 1 in the oracle's plain C (FP64, OpenMP), "
                      f"median of {len(runs)} passes",
            "seconds": dc, "passes": len(runs), "rel_l2_gpu_fp32_vs_oracle": rel_c,
            "dense_solve": {"value": sample * inst.k / dt, "unit": UNIT, "cores": _blas_threads(), "kind": "oracle",
                            "sample": f"{sample} instances, dense k x k LU solve (one factorisation)",
                            "seconds": dt, "rel_l2_gpu_fp32_vs_oracle": rel},
            "alg1_numpy": {"value": Fa.shape[0] * inst.k / da, "unit": UNIT, "kind": "oracle",
                           "sample": f"all {Fa.shape[0]} instances, Algorithm 1 by levels (numpy FP64, one thread)",
                           "seconds": da, "rel_l2_gpu_fp32_vs_oracle": rel_a}}


def _blas_threads():
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(v):
            return int(os.environ[v])
    return os.cpu_count()


def run_reference(args):
    """The oracle on the host cores (rank 0 only): one step = the oracle's C
    Algorithm 1 (FP64, OpenMP over instances) over the whole workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle as O
    from oracle import alg1
    M, s = args.log2n, args.log2k
    inst, _ = W.workload_shared(M=M, s=s, batch=1, coeffs=False)
    rng = W.rng_for(2, 555)
    Jc = O.canonical_support_by_key(inst.J, inst.pivots)
    F = W.complex_gaussian((args.batch, inst.k), rng)
    threads = os.cpu_count()
    for _ in range(args.warmup):
        alg1.alg1_batch(M, inst.pivots, Jc, F, threads=threads)
    times = []
    used = threads
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, used = alg1.alg1_batch(M, inst.pivots, Jc, F, threads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.batch * inst.k * args.steps / total
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": _config(M, s, args.batch, ws),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                            "sample": f"the whole workload ({args.batch} instances) per step, Algorithm 1 in the "
                                      "oracle's plain C (FP64, OpenMP over instances)"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--log2n", type=int, default=20)
    ap.add_argument("--log2k", type=int, default=12)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--cpu-sample", type=int, default=4096,
                    help="instances in the oracle dense-solve baseline (at most the batch; about 10 s of CPU work)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--only-fp32", action="store_true", help="time the complex64 leg only (profiling)")
    ap.add_argument("--large", action="store_true", help="time only the large-k leg (N=2^30, k=2^20)")
    ap.add_argument("--large-batch", type=int, default=64)
    ap.add_argument("--uneven-count", type=int, default=10000)
    ap.add_argument("--uneven", action="store_true", help="time only the uneven-batch leg")
    ap.add_argument("--sas", action="store_true", help="time only the Shift-and-Sample leg")
    ap.add_argument("--sas-batch", type=int, default=1024)
    ap.add_argument("--no-extra", action="store_true", help="skip the uneven, large-k and serving legs")
    ap.add_argument("--serve", action="store_true", help="run only the serving leg")
    ap.add_argument("--serve-rate", type=float, default=20000.0)
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-budget", type=int, default=16384, help="admission budget, MiB")
    ap.add_argument("--serve-batch", type=int, default=64)
    ap.add_argument("--serve-planners", type=int, default=8, help="the engine's planner threads")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.large:
        print(json.dumps({"large_k": run_large(args)}), flush=True)
    elif args.serve:
        print(json.dumps({"serving": run_serving(args)}), flush=True)
    elif args.uneven:
        print(json.dumps({"uneven": run_uneven(args)}), flush=True)
    elif args.sas:
        print(json.dumps({"sas": run_sas(args)}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
