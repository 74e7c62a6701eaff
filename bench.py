"""Benchmark: exact amplitudes of the n=70, d=64 brickwork workload (width 32,
32 GiB complex64 boundary, 426 T gates, 16 uniform bitstrings per step) on
one GB300 per rank.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one batch of 16 amplitudes through the whole sweep (row-0 writer,
every boundary pass, last-row reduction). ``value`` is amplitudes per second
with the bitstrings already in HBM (device API); ``e2e`` is the same metric
through the host API, including the table upload, the host->device copy of the
bitstrings from pinned memory and the device->host copy of the amplitudes.
Multi-GPU runs are independent replicas (each rank its own bitstrings; no
collective on the data path): weak scaling, value = all ranks' amplitudes /
the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle (the naive row-by-row network
contraction) on the host cores instead, on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "amplitudes/s (n=70, d=64 brickwork, width 32)"
UNIT = "amps/s"
WORKLOAD = "brickwork CZ n=70 d=64, random Cliffords, 426 T, 16 uniform bitstrings/step, width 32 (32 GiB c64 boundary)"
CPU_SAMPLE = (30, 40)  # oracle-sized slice with the same gate statistics


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def dist_setup(backend_pref):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend_pref, rank=rank, world_size=world)
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (host scalar)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# --------------------------------------------------------------------- clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.p = None
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, power = [], [], []
        names = ("active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        seen = set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], f[5:9]):
                if v.lower().startswith("active"):
                    seen.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(seen)}


# ------------------------------------------------------------ CPU baseline
def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip() + f" ({os.cpu_count()} logical CPUs)"
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return f"{platform.machine()} ({os.cpu_count()} logical CPUs)"


def cpu_sample_circuit():
    return W.random_circuit(CPU_SAMPLE[0], CPU_SAMPLE[1], None, 4, 777)


def cpu_baseline(seconds_cap: float = 30.0, threads: int = 0) -> dict:
    """FP64 oracle (naive row-by-row contraction) on the n=30, d=40 slice with
    the workload's gate statistics, scaled to the n=70, d=64 workload by the
    ratio of Algorithm 1's contraction costs of the two circuits, both counted
    by the oracle itself (no product code is loaded). threads > 0 limits the
    oracle's OpenMP threads (all host cores otherwise)."""
    import oracle
    if threads > 0:
        oracle.set_num_threads(threads)
    c = cpu_sample_circuit()
    u = oracle.circuit_gates(c)
    done = 0
    t0 = time.perf_counter()
    while done < c.bits.shape[0]:
        oracle.nb_amplitudes(c.n, c.d, u, c.bits[done:done + 1])
        done += 1
        if time.perf_counter() - t0 > seconds_cap / 2:
            break
    dt = time.perf_counter() - t0
    slice_rate = done / dt
    ratio = 2.0 ** (oracle.alg1_cost(70, 64)[1] - oracle.alg1_cost(*CPU_SAMPLE)[1])
    return {"value": slice_rate / ratio, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "cpu": _cpu_model(), "sample_amps_per_s": slice_rate, "same_config": False,
            "sample": (f"{done} amplitude(s) of an n={CPU_SAMPLE[0]}, d={CPU_SAMPLE[1]} slice (width 20) "
                       f"in {dt:.1f} s = {slice_rate:.3g} amps/s, divided by the Algorithm 1 cost ratio "
                       f"C(70,64)/C(30,40) = {ratio:.4g} (the oracle's own count of the path); the n=70, d=64 "
                       f"workload itself (2^32-entry FP64 boundary, about 9 h per amplitude) is not run")}


# --------------------------------------------------------------------- traffic
def kernel_code_hash() -> str:
    """First 16 hex digits of the SHA-256 of the pass kernel's code: the
    sources of pass_kernel.cuh and tb_internal.h (pass shapes, launch
    constants) with their comments and all white space removed, so that an
    edit of a comment keeps the key and any code change breaks it."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2608_13110_gb300", "csrc")
    src = "".join(open(os.path.join(csrc, f)).read() for f in ("pass_kernel.cuh", "tb_internal.h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", "", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def pass_traffic(h: int):
    """DRAM bytes per pass launch from the committed ncu summary, scaled to a
    2^h boundary, or None if absent or taken on other kernel sources."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = kernel_code_hash()
    kv = {}
    for line in open(path):
        if "=" in line and not line.lstrip().startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("pass_kernel_code_sha256_16") != digest:
        return None
    try:
        return float(kv["dram_bytes_per_entry"]) * float(2 ** h)
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------------- arms
def run_reference(args, rank, world):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    per_step = max(2.0, min(20.0, 150.0 / max(1, steps + warm)))
    for _ in range(warm):
        cpu_baseline(per_step, args.cpu_threads)
    vals = [cpu_baseline(per_step, args.cpu_threads) for _ in range(steps)]
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[-1])
    cb["value"] = v
    # one step of the workload is 16 amplitudes; at the oracle's rate it would take
    ms = 1e3 * 16 / v
    cb["ms_per_step_how"] = "16 amplitudes (one workload step) at the oracle's scaled rate"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "complex128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": 70, "d": 64, "n_t": 426, "bitstrings_per_step": 16,
                       "parallelism": f"replicas x{world}"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_ours(args, rank, world, local):
    import torch
    import paper_2608_13110_gb300 as tb

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nb = args.nb
    if args.shape:  # profiling aid: a smaller circuit with the same statistics
        n_, d_ = (int(v) for v in args.shape.split(","))
        c = W.random_circuit(n_, d_, None, nb, 4000 + 100 * rank + d_)
    else:
        c = W.precision_70_64(replica=rank, nb=nb)
    h_ = (c.d + 1) // 2
    if args.shape:
        metric = f"amplitudes/s (--shape n={c.n}, d={c.d}, width {h_}; profiling only, not the headline workload)"
        workload = (f"--shape profiling circuit: brickwork CZ n={c.n} d={c.d}, random Cliffords, {c.n_t} T, "
                    f"{nb} uniform bitstrings/step, width {h_}")
    else:
        metric, workload = METRIC, WORKLOAD
    sched_opts = {}
    t_tune = 0.0
    if args.schedule:
        wb, bb, tt = (int(v) for v in args.schedule.split(","))
        sched_opts = {"window_bits": wb, "bottom_bits": bb, "top_bits": tt}
    elif args.precision == "fp32" and not args.default_schedule:
        from paper_2608_13110_gb300 import autotune
        t_tune = time.perf_counter()
        sched_opts = autotune.tune((c.d + 1) // 2, nb)
        t_tune = time.perf_counter() - t_tune
    plan = tb.Plan.from_circuit(c, precision=args.precision, **sched_opts)
    info = plan.info
    h = info["boundary_bits"]
    ws = torch.empty(plan.workspace_bytes(nb), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan.upload(ws, stream)
    d_bits = torch.from_numpy(c.bits).to(dev)
    d_out = torch.empty((nb, 2), dtype=torch.float64, device=dev)

    def step():
        plan.amplitudes_device(d_bits, ws, d_out, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tb.profile_begin()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    prof = tb.profile_end()
    clk = clocks.stop()
    t_dev = e0.elapsed_time(e1) / 1e3
    amps = d_out.cpu().numpy().view(np.complex128).reshape(-1)

    barrier(world, dev)
    # end to end through the host API: pinned host bitstrings in, amplitudes out
    bits_pin = torch.from_numpy(c.bits).pin_memory()
    out_pin = torch.empty((nb, 2), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.amplitudes(bits_pin.numpy(), ws=ws, stream=stream, out=out_pin.numpy())
    t_e2e = (time.perf_counter() - t0)
    e2e_amps = out_pin.numpy().view(np.complex128).reshape(-1)

    t_dev_max = max_over_ranks(t_dev, world, dev)
    t_e2e_max = max_over_ranks(t_e2e, world, dev)
    value = world * nb * args.steps / t_dev_max
    e2e_value = world * nb * args.e2e_steps / t_e2e_max

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or 6800.0
    p = prof["pass"]
    achieved = p["bytes"] / (p["ms"] / 1e3) / 1e9 if p["ms"] > 0 else None
    n_launch = sum(v["launches"] for v in prof.values())
    traffic = pass_traffic(h) if args.precision == "fp32" else None

    line = {
        "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
        "config": {"workload": workload, "n": c.n, "d": c.d, "n_t": int(c.n_t), "bitstrings_per_step": nb,
                   "pass_arithmetic": args.precision,
                   "schedule": ({"given": sched_opts} if args.schedule else
                                ({"autotuned": sched_opts, "tune_s": round(t_tune, 1)} if sched_opts
                                 else "planner default")),
                   "width": info["width"], "passes_per_amplitude": info["n_passes"],
                   "l2": "inputs larger than L2 (32 GiB boundary, 129 MB L2)",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(c.bits.nbytes + info["table_bytes"]),
                "d2h_bytes_per_step": int(16 * nb)},
        "gpu_launches": n_launch,
        "unfused_equivalent_gbs": {
            "value": world * nb * args.steps * info["n_steps"] * 16.0 * 2.0 ** h / t_dev_max / 1e9,
            "how": "paired steps x 16 B x 2^h per amplitude / time: the bandwidth one HBM pass per step "
                   "would need for the same amps/s (secondary, not a measured bandwidth)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": (achieved / hbm_peak) if achieved else None, "traffic": traffic,
                     "traffic_over_algorithmic": (traffic / (16.0 * 2.0 ** h)) if traffic else None,
                     "kernel": "pass_kernel" if args.precision == "fp32" else "tc_pass_kernel",
                     "peak_source": f"{peak_src} copy bandwidth",
                     "pass_launches": p["launches"], "pass_ms_total": p["ms"],
                     "pass_share_of_kernel_time": p["ms"] / max(1e-9, sum(v["ms"] for v in prof.values())),
                     "fma_pipe": fma_pipe_fraction(args, info, nb, h, p, clk, dev)},
        "clocks": clk,
        "sanity": {"log_xeb": tb.log_xeb(amps, c.n), "e2e_matches_device": bool(np.array_equal(amps, e2e_amps))},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.shape:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args.cpu_threads)
        line["cpu_baseline"]["gpu_same_sample"] = gpu_rate_on_cpu_sample(tb, dev, stream, line["cpu_baseline"])
    if rank == 0:
        print(json.dumps(line))


def fma_pipe_fraction(args, info, nb, h, p, clk, dev):
    """The FP32 passes' other ceiling: the multiply-adds the pass kernels
    spend per entry (8 per paired step, 16 per row turn's 4x4 block: the
    plan's pass_madds), over the pass kernels' measured time, against SMs x
    128 FP32 lanes x the SM clock (one FMA per lane and cycle; the paired FFMA2
    issues two lanes' worth in two cycles). Secondary to the HBM roofline: the
    two floors are within 15 % of each other at width 32."""
    if args.precision != "fp32" or p["ms"] <= 0:
        return None
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_max_mhz") or 2070.0
    fma = float(nb) * args.steps * info["pass_madds"] * 2.0 ** h
    achieved = fma / (p["ms"] / 1e3) / 1e12
    peak = sms * 128 * mhz * 1e6 / 1e12
    return {"achieved": achieved, "peak": peak, "unit": "TFMA/s", "frac": achieved / peak,
            "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}


def gpu_rate_on_cpu_sample(tb, dev, stream, cb):
    """The device path on the oracle's own sample (the same n=30, d=40 circuit
    and bitstrings, each repeated 64 times per call): a like-for-like amps/s
    beside the oracle's unscaled slice rate."""
    import torch
    c = cpu_sample_circuit()
    bits = np.repeat(c.bits, 64, axis=0)
    plan = tb.Plan.from_circuit(c)
    ws = torch.empty(plan.workspace_bytes(bits.shape[0]), dtype=torch.uint8, device=dev)
    plan.upload(ws, stream)
    d_bits = torch.from_numpy(bits).to(dev)
    d_out = torch.empty((bits.shape[0], 2), dtype=torch.float64, device=dev)
    for _ in range(3):
        plan.amplitudes_device(d_bits, ws, d_out, stream)
    reps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        plan.amplitudes_device(d_bits, ws, d_out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    rate = reps * bits.shape[0] / (e0.elapsed_time(e1) / 1e3)
    got = d_out.cpu().numpy().view(np.complex128).reshape(-1)
    oracle_rate = cb.get("sample_amps_per_s")
    return {"value": rate, "unit": "amps/s on the sample circuit",
            "ratio_to_oracle_sample_rate": (rate / oracle_rate) if oracle_rate else None,
            "repeats_identical": bool(np.all(got.reshape(4, 64) == got.reshape(4, 64)[:, :1])),
            "how": f"{bits.shape[0]} bitstrings per call ({c.bits.shape[0]} distinct x 64), "
                   f"{reps} calls after 3 warm-up calls, CUDA events on the launching stream; "
                   f"256 boundaries of 8 MiB in flight (2 GiB, larger than L2), planner-default windows"}


def run_batch_workload(args, rank, world, local):
    """64 circuits of uneven size (n ~ U[20,70], d ~ U{16..48}, T density
    0.095, 32 bitstrings each = 2048 amplitudes) recorded into one CUDA graph
    with autotuned window sizes, against the plain path (one call per circuit,
    back to back on one stream)."""
    import torch
    import paper_2608_13110_gb300 as tb
    from paper_2608_13110_gb300 import autotune
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nb = 32
    circuits = W.batch_uneven(64, nb, seed0=3000 + 1000 * rank)
    t0 = time.perf_counter()
    plans = [autotune.tuned_plan(c, nb=nb) for c in circuits]
    tune_s = time.perf_counter() - t0
    d_bits = [torch.from_numpy(c.bits).to(dev) for c in circuits]
    out_b = [torch.empty((nb, 2), dtype=torch.float64, device=dev) for _ in circuits]
    out_p = [torch.empty((nb, 2), dtype=torch.float64, device=dev) for _ in circuits]
    t0 = time.perf_counter()
    batch = tb.Batch(list(zip(plans, d_bits, out_b)))
    record_s = time.perf_counter() - t0
    wss = []
    for pl in plans:
        ws = pl.alloc_workspace(nb)
        pl.upload(ws)
        wss.append(ws)
    stream = torch.cuda.current_stream(dev)

    def plain():
        for pl, db, ws, o in zip(plans, d_bits, wss, out_p):
            pl.amplitudes_device(db, ws, o, stream)

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3

    for _ in range(args.warmup):
        batch.launch(stream)
        plain()
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    clocks = ClockSampler(local)
    t_b = timed(lambda: batch.launch(stream), args.steps)
    t_p = timed(plain, args.steps)
    clk = clocks.stop()
    same = all(torch.equal(a, b) for a, b in zip(out_b, out_p))
    t_b = max_over_ranks(t_b, world, dev)
    t_p = max_over_ranks(t_p, world, dev)
    namps = 64 * nb
    line = {"metric": "amplitudes/s (64 uneven brickwork circuits, 2048 amplitudes, one graph launch)",
            "value": world * namps * args.steps / t_b, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_b / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
            "config": {"workload": "64 circuits n~U[20,70], d~U{16..48} even, T density 0.095, 32 bitstrings each",
                       "widths": sorted({(c.d + 1) // 2 for c in circuits}), "autotune_s": tune_s,
                       "graph_record_s": record_s, "parallelism": f"replicas x{world}"},
            "plain": {"value": world * namps * args.steps / t_p, "unit": UNIT, "ms_per_step": 1e3 * t_p / args.steps,
                      "how": "one tb_amplitudes_device call per circuit, back to back on one stream"},
            "identical_to_plain": bool(same), "clocks": clk}
    if rank == 0:
        print(json.dumps(line))


def _golden(name):
    """Stored FP64 amplitudes (written by the scripts in tests/golden from the
    oracle) with their circuit, or None if absent."""
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    c = W.Circuit(g["n"], g["d"], np.array(g["cliff"], np.uint8), np.array(g["tmask"], np.uint8),
                  np.array(g["bits"], np.uint8), 0)
    return c, np.array([complex(a, b) for a, b in g["amps"]])


def _errors(got, ref):
    rel = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), "max_rel": float(rel.max()),
            "n_amplitudes": int(ref.size)}


def run_precision_workload(args, rank, world, local):
    """The plain complex64 path (FP32 FMA staircase) against the split-precision
    tensor-core forms (3xTF32 and 3xBF16 dense blocks) on the n=70, d=64
    workload: amplitudes/s, the pass kernels' HBM GB/s, and each form's error
    against stored FP64 values (n=32, d=48 naive-boundary oracle; n=70, d=64
    closed form), all on the same GPU in the same run."""
    import torch
    import paper_2608_13110_gb300 as tb
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nb = args.nb_precision
    c = W.precision_70_64(replica=rank, nb=nb)
    stream = torch.cuda.current_stream(dev)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    goldens = {"n32_d48_fp64_oracle": _golden("precision_n32_d48.json"),
               "n70_d64_closed_form": _golden("closed_form_n70_d64.json")}
    forms = {}
    ref_amps = None
    clocks = ClockSampler(local)
    from paper_2608_13110_gb300 import autotune
    tuned = {} if args.default_schedule else autotune.tune((c.d + 1) // 2, 1)
    for form in ("fp32", "tf32x3", "bf16x3"):
        plan = tb.Plan.from_circuit(c, precision=form, **(tuned if form == "fp32" else {}))
        ws = torch.empty(plan.workspace_bytes(nb), dtype=torch.uint8, device=dev)
        plan.upload(ws, stream)
        d_bits = torch.from_numpy(c.bits).to(dev)
        d_out = torch.empty((nb, 2), dtype=torch.float64, device=dev)
        for _ in range(args.warmup):
            plan.amplitudes_device(d_bits, ws, d_out, stream)
        torch.cuda.synchronize(dev)
        barrier(world, dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        tb.profile_begin()
        e0.record(stream)
        for _ in range(args.steps):
            plan.amplitudes_device(d_bits, ws, d_out, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        prof = tb.profile_end()
        t = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
        amps = d_out.cpu().numpy().view(np.complex128).reshape(-1)
        del ws
        if ref_amps is None:
            ref_amps = amps
        p = prof["pass"]
        achieved = p["bytes"] / (p["ms"] / 1e3) / 1e9
        f = {"amps_per_s": world * nb * args.steps / t, "ms_per_step": 1e3 * t / args.steps,
             "passes_per_amplitude": plan.info["n_passes"],
             "pass_kernel": {"achieved_gbs": achieved, "frac_of_measured_hbm": achieved / hbm_peak,
                             "avg_ms": p["ms"] / max(1, p["launches"])},
             "rel_l2_vs_fp32_n70_d64": float(np.linalg.norm(amps - ref_amps) / np.linalg.norm(ref_amps)),
             "errors_vs_fp64": {}}
        for name, g in goldens.items():
            if g is None:
                continue
            gc, gref = g
            got = tb.Plan.from_circuit(gc, precision=form).amplitudes(gc.bits)
            f["errors_vs_fp64"][name] = _errors(got, gref)
        f["device_faults"] = tb.device_faults()
        worst = max([e["rel_l2"] for e in f["errors_vs_fp64"].values()] or [float("nan")])
        f["meets_rel_l2_1e-5"] = bool(worst <= 1e-5)
        forms[form] = f
    clk = clocks.stop()
    line = {"metric": "amplitudes/s by pass arithmetic (n=70, d=64) with error vs FP64",
            "value": forms["fp32"]["amps_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": forms["fp32"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
            "config": {"workload": f"brickwork CZ n=70 d=64, random Cliffords, 426 T, {nb} bitstrings/step, "
                                   "width 32; value = the plain FP32 form",
                       "fp32_schedule": {"autotuned": tuned} if tuned else "planner default",
                       "l2": "inputs larger than L2 (32 GiB boundary)", "parallelism": f"replicas x{world}",
                       "peak_hbm_gbs": hbm_peak},
            "forms": forms,
            "note": ("the 1e-5 relative L2 bar against FP64 is met by: " +
                     ", ".join(k for k, v in forms.items() if v.get("meets_rel_l2_1e-5")) +
                     "; not met by: " + (", ".join(k for k, v in forms.items() if not v.get("meets_rel_l2_1e-5"))
                                         or "none")),
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line))


def run_open_workload(args, rank, world, local):
    """Algorithm 2 on the n=70, d=64 workload: k = 8 open output bits, so one
    sweep of the fixed region (rows 0..61) plus the join and the late region
    returns the 256 amplitudes of a prefix. value = amplitudes/s over
    ``--nb-open`` uniform prefixes per step; compared with the plain sweep
    (one amplitude per sweep) timed in the same run."""
    import torch
    import paper_2608_13110_gb300 as tb
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    k = args.open_k
    na = args.nb_open
    if args.shape:  # profiling aid: a smaller circuit with the same statistics
        n_, d_ = (int(v) for v in args.shape.split(","))
        c = W.random_circuit(n_, d_, None, 1, 4000 + 100 * rank + d_)
    else:
        c = W.precision_70_64(replica=rank, nb=1)
    rng = np.random.default_rng(7000 + rank)
    prefixes = rng.integers(0, 2, size=(na, c.n - k), dtype=np.uint8)
    sched_opts = {}
    if args.precision == "fp32" and not args.default_schedule:
        from paper_2608_13110_gb300 import autotune
        sched_opts = autotune.tune((c.d + 1) // 2, 1)
    plan = tb.Plan.from_circuit(c, open_k=k, precision=args.precision, **sched_opts)
    info = plan.info
    stream = torch.cuda.current_stream(dev)
    ws = torch.empty(plan.workspace_bytes(na), dtype=torch.uint8, device=dev)
    plan.upload(ws, stream)
    d_pre = torch.from_numpy(prefixes).to(dev)
    d_out = torch.empty((na << k, 2), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        plan.amplitudes_device(d_pre, ws, d_out, stream)
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    clocks = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tb.profile_begin()
    e0.record(stream)
    for _ in range(args.steps):
        plan.amplitudes_device(d_pre, ws, d_out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    prof = tb.profile_end()
    clk = clocks.stop()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
    amps = d_out.cpu().numpy().view(np.complex128).reshape(na, -1)
    # end to end: host prefixes in, host amplitudes out
    pre_pin = torch.from_numpy(prefixes).pin_memory()
    out_pin = torch.empty((na << k, 2), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plan.amplitudes(pre_pin.numpy(), ws=ws, stream=stream, out=out_pin.numpy())
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    # the plain sweep on four of the same bitstrings, for the comparison and a cross-check
    ys = np.array([0, 77, 200, 255]) % (1 << k)
    bits = np.zeros((4, c.n), np.uint8)
    bits[:, : c.n - k] = prefixes[0]
    for j in range(k):
        bits[:, c.n - k + j] = (ys >> j) & 1
    pplan = tb.Plan.from_circuit(c, precision=args.precision, **sched_opts)
    pws = torch.empty(pplan.workspace_bytes(4), dtype=torch.uint8, device=dev)
    pplan.upload(pws, stream)
    d_bits = torch.from_numpy(bits).to(dev)
    p_out = torch.empty((4, 2), dtype=torch.float64, device=dev)
    pplan.amplitudes_device(d_bits, pws, p_out, stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    pplan.amplitudes_device(d_bits, pws, p_out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_plain = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
    plain_amps = p_out.cpu().numpy().view(np.complex128).reshape(-1)
    agree = float(np.linalg.norm(amps[0, ys] - plain_amps) / np.linalg.norm(plain_amps))
    b, q = tb.batched_sample(amps, rng.random(na))
    total = max(1e-9, sum(v["ms"] for v in prof.values()))
    shape = f"n={c.n}, d={c.d}" + (" (--shape, profiling)" if args.shape else "")
    line = {"metric": f"amplitudes/s ({shape}, k={k} open output bits: {1 << k} amplitudes per sweep)",
            "value": world * na * (1 << k) * args.steps / t, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
            "config": {"workload": f"brickwork CZ {shape}, random Cliffords, {c.n_t} T, k={k}, {na} uniform prefixes/step",
                       "open_k": k, "open_width": info["open_width"], "passes_per_prefix": info["n_passes"],
                       "schedule": {"autotuned": sched_opts} if sched_opts else "planner default",
                       "pass_arithmetic": args.precision, "parallelism": f"replicas x{world}"},
            "e2e": {"value": world * na * (1 << k) / t_e2e, "unit": UNIT,
                    "h2d_bytes_per_step": int(prefixes.nbytes + info["table_bytes"]),
                    "d2h_bytes_per_step": int(16 * (na << k))},
            "gpu_launches": sum(v["launches"] for v in prof.values()),
            "time_share": {c_: round(v["ms"] / total, 4) for c_, v in prof.items() if v["launches"]},
            "plain": {"value": world * 4 / t_plain, "unit": UNIT, "how": "single-amplitude sweep, same circuit"},
            "rel_l2_vs_plain_sweep": agree,
            "sampled": {"suffixes": b.tolist()[:8], "Q_a_times_A": (q * 2.0 ** (c.n - k)).tolist()[:8]},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line))


# The paper's own measurement (Sec. 5.2 and its table of full-depth results):
# n = d = 70 with T = 468, k = 8 open outputs (256 amplitudes per
# contraction), width 35 (a 256 GiB complex64 boundary), 32.16 s per
# steady-state contraction on one node of 8 H100 GPUs.
PAPER_S_PER_CONTRACTION = 32.16
PAPER_FIRST_USE_S = 54.63  # first contraction of a job (handles, plan and workspace caches)
PAPER_AMPS_PER_CONTRACTION = 256


def run_paper_workload(args, rank, world, local):
    """The paper's contraction on one GPU: n = d = 70, 468 T gates at uniform
    sites, random Cliffords (the IBM instance is not available), k = 8 open
    output bits, ``--nb-open`` uniform prefixes per step. Width 35: the plan
    works in place (one 256 GiB boundary). value = amplitudes/s; vs_baseline
    = value over the paper's 256 amplitudes per 32.16 s (8 H100 GPUs)."""
    import torch
    import paper_2608_13110_gb300 as tb
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    k = 8
    na = args.nb_open
    c = W.random_circuit(70, 70, 468, 0, 4600 + rank)
    rng = np.random.default_rng(7100 + rank)
    prefixes = rng.integers(0, 2, size=(na, c.n - k), dtype=np.uint8)
    # windows 10 / bottom 10 / top 9: the fastest of the schedules timed at width
    # 35 on a GB300 (8 absorbed rows: 3087 ms; 9 / 7 / 7: 3156 ms; the planner's
    # default 3217 ms); autotuning inside the run would time 256 GiB sweeps
    t_first = time.perf_counter()  # first use: plan, workspace, upload and the first contraction
    plan = tb.Plan.from_circuit(c, open_k=k, window_bits=10, bottom_bits=10, top_bits=9)
    info = plan.info
    need = plan.workspace_bytes(1)
    free = torch.cuda.mem_get_info(dev)[0]
    if free < need + (2 << 30):
        if rank == 0:
            print(json.dumps({"metric": "amplitudes/s (n=d=70, 468 T, k=8 open bits, width 35)", "value": None,
                              "unavailable": f"needs {need / 2**30:.1f} GiB of device memory, {free / 2**30:.1f} GiB free"}))
        return
    stream = torch.cuda.current_stream(dev)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)  # one boundary: prefixes run one after another
    plan.upload(ws, stream)
    d_pre = torch.from_numpy(prefixes).to(dev)
    d_out = torch.empty((na << k, 2), dtype=torch.float64, device=dev)
    first_use = None
    for w in range(args.warmup):
        plan.amplitudes_device(d_pre[:1] if w == 0 else d_pre, ws, d_out, stream)
        if w == 0:
            torch.cuda.synchronize(dev)
            first_use = time.perf_counter() - t_first
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    clocks = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tb.profile_begin()
    e0.record(stream)
    for _ in range(args.steps):
        plan.amplitudes_device(d_pre, ws, d_out, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    prof = tb.profile_end()
    clk = clocks.stop()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
    amps = d_out.cpu().numpy().view(np.complex128).reshape(na, -1)
    pre_pin = torch.from_numpy(prefixes).pin_memory()
    out_pin = torch.empty((na << k, 2), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plan.amplitudes(pre_pin.numpy(), ws=ws, stream=stream, out=out_pin.numpy())
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_amps = out_pin.numpy().view(np.complex128).reshape(na, -1)
    total = max(1e-9, sum(v["ms"] for v in prof.values()))
    p = prof["pass"]
    value = world * na * (1 << k) * args.steps / t
    paper_rate = PAPER_AMPS_PER_CONTRACTION / PAPER_S_PER_CONTRACTION
    line = {"metric": "amplitudes/s (n=d=70, 468 T, k=8 open output bits: 256 amplitudes per contraction, width 35)",
            "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / paper_rate, "dtype": "complex64", "data": "synthetic",
            "config": {"workload": f"brickwork CZ n=70, d=70, random Cliffords, 468 T, k=8, {na} uniform prefixes/step",
                       "open_k": k, "open_width": info["open_width"], "passes_per_prefix": info["n_passes"],
                       "in_place": True, "workspace_gib": need / 2**30,
                       "schedule": {"given": {"window_bits": 10, "bottom_bits": 10, "top_bits": 9}},
                       "pass_arithmetic": "fp32", "parallelism": f"replicas x{world}"},
            "s_per_contraction": t / (na * args.steps),
            "first_use_s": first_use,  # plan + 260 GiB workspace + upload + first contraction (wall clock)
            "baseline": {"s_per_contraction": PAPER_S_PER_CONTRACTION, "amps_per_s": paper_rate,
                         "first_use_s": PAPER_FIRST_USE_S,
                         "hardware": "one node of 8 NVIDIA H100 GPUs (cuTENSORMp, MPI)",
                         "source": "the paper's table of full-depth results (Sec. 5.2)"},
            "e2e": {"value": world * na * (1 << k) / t_e2e, "unit": UNIT,
                    "h2d_bytes_per_step": int(prefixes.nbytes + info["table_bytes"]),
                    "d2h_bytes_per_step": int(16 * (na << k))},
            "e2e_matches_device": bool(np.allclose(e2e_amps, amps, rtol=0, atol=1e-12 * np.abs(amps).max())),
            "gpu_launches": sum(v["launches"] for v in prof.values()),
            "time_share": {c_: round(v["ms"] / total, 4) for c_, v in prof.items() if v["launches"]},
            "clocks": clk}
    if p["launches"]:  # the pass kernel against the measured HBM copy bandwidth (16 B per entry per pass)
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        hbm_peak = (json.load(open(pk)).get("hbm_gbs") if os.path.exists(pk) else None) or 6800.0
        ach = 16.0 * 2.0 ** 35 / (p["ms"] / p["launches"] / 1e3) / 1e9
        line["roofline"] = {"bound": "hbm", "kernel": "pass_kernel", "achieved": ach, "peak": hbm_peak,
                            "unit": "GB/s", "frac": ach / hbm_peak, "pass_launches": p["launches"]}
    if rank == 0:
        print(json.dumps(line))


def run_serve_workload(args, rank, world, local):
    """Poisson stream (mean 20 requests/s) of amplitude requests, n ~ U[16,70],
    d even ~ U{8..44} (width <= 22: a width-33 request of 256 bitstrings alone
    needs about 35 GPU-minutes, so the full d <= 66 range cannot be served at
    20 requests/s by one GPU), 1..256 bitstrings each,
    through the serving runtime (160 GB budget, continuous admission) against
    the plain path: the same requests one at a time in arrival order."""
    import threading
    import torch
    import paper_2608_13110_gb300 as tb
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    reqs = W.serving_stream(args.requests, rate_hz=20.0, seed=5000 + 1000 * rank, max_width=22)
    plans = [tb.Plan.from_circuit(c) for _, c in reqs]
    namps = sum(c.bits.shape[0] for _, c in reqs)
    # warm the kernels and the allocator
    for pl, (_, c) in list(zip(plans, reqs))[: args.warmup]:
        pl.amplitudes(c.bits[:1])
    torch.cuda.synchronize(dev)

    srv = tb.Server(hbm_budget_bytes=160 * 10**9, slots=args.serve_slots, device=local, pinned_bytes=256 << 20)
    tickets = [None] * len(reqs)
    t0 = time.perf_counter()

    def submitter():
        for i, ((t_arr, c), pl) in enumerate(zip(reqs, plans)):
            dt = t0 + t_arr - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = srv.submit(pl, c.bits)

    clocks = ClockSampler(local)
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    res_srv = [srv.wait(t)[0] for t in tickets]
    t_srv = time.perf_counter() - t0
    st = srv.stats()
    srv.close()

    # plain path: one request at a time, in arrival order, same arrival times
    lat = []
    res_plain = []
    t0 = time.perf_counter()
    for (t_arr, c), pl in zip(reqs, plans):
        dt = t0 + t_arr - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        res_plain.append(pl.amplitudes(c.bits))
        lat.append(time.perf_counter() - (t0 + t_arr))
    t_plain = time.perf_counter() - t0
    clk = clocks.stop()
    err = max(float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)) for a, b in zip(res_srv, res_plain))
    lat.sort()
    q = lambda f: lat[min(len(lat) - 1, int(f * (len(lat) - 1) + 0.5))]
    line = {"metric": "amplitudes/s and p50/p99 latency, Poisson request stream (served)",
            "value": world * namps / max_over_ranks(t_srv, world, dev), "unit": UNIT, "n_gpus": world,
            "steps": 1, "warmup": args.warmup, "ms_per_step": 1e3 * t_srv, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
            "config": {"workload": f"{len(reqs)} requests, Poisson 20/s, n~U[16,70], d even <= 44 (width <= 22), "
                                   "1..256 bitstrings", "amplitudes": namps, "hbm_budget_bytes": 160 * 10**9,
                       "slots": args.serve_slots, "parallelism": f"replicas x{world}"},
            "latency_s": {"p50": st["p50_latency_s"], "p99": st["p99_latency_s"], "mean": st["mean_latency_s"]},
            "server": {"peak_concurrent": st["peak_concurrent"], "peak_bytes_in_use": st["peak_bytes_in_use"]},
            "plain": {"value": world * namps / max_over_ranks(t_plain, world, dev), "unit": UNIT,
                      "latency_s": {"p50": q(0.5), "p99": q(0.99), "mean": sum(lat) / len(lat)},
                      "how": "each request alone through tb_amplitudes, in arrival order"},
            "max_rel_l2_served_vs_plain": err, "clocks": clk}
    if rank == 0:
        print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--nb", type=int, default=16)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="OpenMP threads of the CPU oracle baseline (0 = every host core)")
    ap.add_argument("--workload", default="n70d64", choices=("n70d64", "batch", "serve", "precision", "open", "paper"),
                    help="n70d64: the headline metric; batch: 64 uneven circuits in one graph; "
                         "serve: Poisson request stream through the serving runtime; "
                         "precision: FP32 vs 3xTF32 / 3xBF16 tensor-core passes with errors vs FP64; "
                         "open: Algorithm 2, 256 amplitudes per sweep (k=8); "
                         "paper: the paper's own contraction (n=d=70, 468 T, k=8, width 35) on one GPU")
    ap.add_argument("--nb-open", type=int, default=2, help="prefixes per step in the open workload")
    ap.add_argument("--open-k", type=int, default=8, help="open output bits in the open workload (1..10)")
    ap.add_argument("--precision", default="fp32", choices=("fp32", "tf32x3", "bf16x3"),
                    help="pass arithmetic of the n70d64 workload")
    ap.add_argument("--default-schedule", action="store_true",
                    help="use the planner's default window schedule instead of the autotuned one")
    ap.add_argument("--schedule", default="",
                    help="window_bits,bottom_bits,top_bits of the n70d64 workload (no autotuning; profiling)")
    ap.add_argument("--nb-precision", type=int, default=4, help="bitstrings per step in the precision workload")
    ap.add_argument("--requests", type=int, default=200, help="requests in the serve workload")
    ap.add_argument("--serve-slots", type=int, default=2,
                    help="concurrent requests in the serve workload (2: best p99 on this stream)")
    ap.add_argument("--shape", default="", help="n,d of a smaller circuit (profiling only; not the reported workload)")
    args = ap.parse_args()
    if args.impl == "reference":
        rank, world, _ = dist_setup("gloo")
        run_reference(args, rank, world)
    else:
        rank, world, local = dist_setup("nccl")
        if args.workload == "batch":
            run_batch_workload(args, rank, world, local)
        elif args.workload == "serve":
            run_serve_workload(args, rank, world, local)
        elif args.workload == "precision":
            run_precision_workload(args, rank, world, local)
        elif args.workload == "open":
            run_open_workload(args, rank, world, local)
        elif args.workload == "paper":
            run_paper_workload(args, rank, world, local)
        else:
            run_ours(args, rank, world, local)
    if _env_int("WORLD_SIZE", 1) > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
