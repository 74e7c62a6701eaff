"""Autotuner for the pass schedule.

The planner groups the paired steps of every absorbed row into windows of
address bits (the step-fusion depth of one HBM pass: up to 10 bits, i.e. up
to 9 steps per window and 16 at a row turn, whose four turn steps run as one
4x4 block). Which window sizes are fastest
depends on the width, the batch of bitstrings evaluated side by side and the
GPU, so this module times candidate schedules on the device and keeps the
winner per (GPU, width, batch bucket) in a JSON cache.

    from paper_2608_13110_gb300 import autotune
    opts = autotune.tune(h=24, nb=32)      # {"window_bits": .., "bottom_bits": .., "top_bits": ..}
    plan = autotune.tuned_plan(circuit, nb=32)
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np

from . import Plan

_LOCK = threading.Lock()
NARROW_MAX_WIDTH = 12  # whole boundary in one CTA: no windows to tune


def cache_path() -> str:
    return os.environ.get("TB_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tbsweep", "autotune.json"))


def _load_cache() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(c: dict) -> None:
    """Best effort: an unwritable cache only costs re-tuning later. Each
    process writes its own temporary file, then renames it into place."""
    p = cache_path()
    tmp = f"{p}.{os.getpid()}.tmp"
    try:
        os.makedirs(os.path.dirname(p) or ".", exist_ok=True)
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        try:
            os.remove(tmp)
        except OSError:
            pass


def _bucket(nb: int) -> int:
    b = 1
    while b < nb:
        b *= 2
    return b


def candidate_options(h: int, n_rows: int = 8, limit: int = 8) -> list[dict]:
    """Feasible window choices for width h with distinct pass schedules,
    fewest passes first (ties: smallest largest pass)."""
    seen = {}
    d = 2 * h
    n = n_rows + 2
    for wb in (8, 9, 10):
        for bb in range(5, 11):
            for tt in range(5, 11):
                try:
                    p = Plan(n, d, window_bits=wb, bottom_bits=bb, top_bits=tt)
                except Exception:
                    continue
                sched = tuple(p.schedule)
                if sched in seen:
                    continue
                steps = [2 * m - 3 if s in ("top", "bot") else m for s, m, _ in sched]  # turn blocks count twice
                seen[sched] = ((len(sched), max(steps)), {"window_bits": wb, "bottom_bits": bb, "top_bits": tt})
    ranked = [v[1] for v in sorted(seen.values(), key=lambda kv: kv[0])]
    default = {"window_bits": 0, "bottom_bits": 0, "top_bits": 0}
    return [default] + ranked[: max(0, limit - 1)]


# Boundary entries the device keeps in flight per call by default (8 GiB of
# complex64): wider boundaries are evaluated one bitstring after another, so
# timing more of them measures nothing new.
BATCH_ENTRIES = 1 << 30


def measure(opts: dict, h: int, nb: int, n_rows: int = 8, reps: int = 3, seed: int = 1) -> float:
    """Milliseconds per batch of nb amplitudes of an (n_rows+2)-qubit circuit
    of width h under the given window options (median of reps). A batch
    larger than the device evaluates at once is timed on the part it runs
    concurrently and scaled."""
    import torch
    import workloads as W
    run = max(1, min(nb, BATCH_ENTRIES >> h))
    scale = nb / run
    nb = run
    c = W.random_circuit(n_rows + 2, 2 * h, None, nb, seed)
    plan = Plan.from_circuit(c, **opts)
    ws = plan.alloc_workspace(nb)
    plan.upload(ws)
    d_bits = torch.from_numpy(c.bits).cuda()
    out = torch.empty((nb, 2), dtype=torch.float64, device="cuda")
    plan.amplitudes_device(d_bits, ws, out)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.amplitudes_device(d_bits, ws, out)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times)) * scale


WIDE_LIMIT = 24  # candidates timed for boundaries of at least 2^WIDE_H entries
WIDE_H = 26


def tune(h: int, nb: int = 1, n_rows: int = 8, limit: int = 0, use_cache: bool = True) -> dict:
    """Fastest window options for width h with nb bitstrings side by side.
    limit = 0 times 8 candidates, or 24 for widths >= 26: there the address
    span of a window changes the pass time (page and DRAM locality), which the
    planner's arithmetic cost model does not see."""
    if h <= NARROW_MAX_WIDTH:
        return {"window_bits": 0, "bottom_bits": 0, "top_bits": 0}
    if limit <= 0:
        limit = WIDE_LIMIT if h >= WIDE_H else 8
    import torch
    key = f"{torch.cuda.get_device_name()}|h={h}|nb={_bucket(nb)}"
    with _LOCK:
        cache = _load_cache() if use_cache else {}
        if key in cache:
            return dict(cache[key]["opts"])
    results = []
    for opts in candidate_options(h, n_rows, limit):
        results.append((measure(opts, h, _bucket(nb), n_rows), opts))
    best_ms, best = min(results, key=lambda r: r[0])
    if use_cache:
        with _LOCK:
            cache = _load_cache()
            cache[key] = {"opts": best, "ms": best_ms, "tried": len(results)}
            _save_cache(cache)
    return dict(best)


def tuned_plan(circ, nb: int | None = None, **kw) -> Plan:
    """Plan for a circuit with autotuned window options."""
    h = (circ.d + 1) // 2
    opts = tune(h, nb if nb is not None else max(1, circ.bits.shape[0]), **kw)
    return Plan.from_circuit(circ, **opts)
