"""Host-side checks of the C-ABI library: it loads, exports every declared
symbol, and its planner reproduces the numbers the paper prints. No CUDA call
is made (the planner is host-only), so these run without a GPU."""
import ctypes
import json
import math
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_numbers.json")))


@pytest.fixture(scope="module")
def tb():
    from paper_2608_13110_gb300 import build as b
    b.build()
    import paper_2608_13110_gb300 as mod
    return mod


def test_library_exports_every_declared_symbol(tb):
    header = open(os.path.join(ROOT, "include", "tbsweep.h")).read()
    declared = set(re.findall(r"TB_API\s+[\w\s\*]+?\b(tb_\w+)\s*\(", header))
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(tb._lib, name), name
    assert declared == set(tb.EXPORTED)


def test_clifford_table_matches_oracle(tb, oracle_mod):
    ref = oracle_mod.clifford_table()
    for k in range(24):
        np.testing.assert_allclose(tb.clifford_matrix(k), ref[k], atol=1e-15)


def test_width_and_cost_at_n70_d70(tb):
    g = GOLDEN["width_cost_open_chi2_n70_d70"]
    info = tb.Plan(g["n"], g["d"]).info
    assert info["width"] == g["W"]
    assert abs(info["log2_cost"] - g["log2_C"]) < g["log2_C_tolerance"]


def test_planner_counters_equal_the_oracle_count(tb, oracle_mod):
    """The planner's W and log2 C (which the benchmark's CPU baseline does not
    use) agree with the oracle's independent count of Algorithm 1's path."""
    for n, d in [(70, 70), (70, 64), (30, 40), (70, 56), (32, 48), (12, 8), (70, 63), (5, 9), (13, 25)]:
        info = tb.Plan(n, d).info
        w, c = oracle_mod.alg1_cost(n, d)
        assert info["width"] == w and abs(info["log2_cost"] - c) < 1e-9, (n, d)


def test_constructive_width_is_ceil_d_over_2(tb):
    g = GOLDEN["constructive_width"]
    for d in g["d"]:
        assert tb.Plan(g["n"], d).info["width"] == math.ceil(d / 2), d
    for n, d in [(12, 8), (30, 40), (32, 48), (70, 56), (70, 64), (20, 16), (40, 48)]:
        info = tb.Plan(n, d).info
        assert info["width"] == d // 2 == info["boundary_bits"]
    # odd d (Proposition 1's turn case): the same width ceil(d/2)
    for n, d in [(4, 7), (12, 9), (30, 41), (70, 7), (70, 63), (70, 65), (40, 79), (9, 17)]:
        info = tb.Plan(n, d).info
        assert info["width"] == (d + 1) // 2 == info["boundary_bits"], (n, d)


def test_boundary_payload_bytes(tb):
    g = GOLDEN["boundary_payload_bytes"]
    assert tb.Plan(70, 70).info["boundary_bytes"] == g["d70_complex64"]
    assert tb.Plan(70, 60).info["boundary_bytes"] == g["d60_complex64"]


def test_cz_counts_of_the_brickwork_convention():
    g = GOLDEN["cz_counts_n70"]
    n = g["n"]
    per_layer = [len(range(l % 2, n - 1, 2)) for l in range(70)]
    assert sorted(set(per_layer)) == g["per_layer"]
    assert sum(per_layer) == g["total_d70"]


def test_plan_topology_independent_of_gate_values(tb):
    """Width, cost, step and pass counts do not depend on the one-qubit gates
    nor on how many T gates there are or where they sit (Sec. 1 contributions, Sec. 3.1)."""
    c = W.precision_70_64(nb=1)
    a = tb.Plan.from_circuit(c).info
    b = tb.Plan.from_circuit(c.clifford_twin()).info
    e = tb.Plan(70, 64).info
    for k in ("width", "log2_cost", "n_steps", "n_passes", "boundary_bytes", "table_bytes"):
        assert a[k] == b[k] == e[k], k


def test_step_and_pass_counts(tb):
    for n, d in [(70, 64), (70, 56), (30, 40), (12, 8), (2, 30), (3, 26), (70, 63), (13, 25), (5, 9)]:
        info = tb.Plan(n, d).info
        h = (d + 1) // 2
        assert info["n_steps"] == max(0, n - 2) * h
        if h <= 12 or n == 2:
            assert info["n_passes"] == 0
        else:
            # every pass advances at most 2*MAX_WINDOW-1 steps
            assert info["n_passes"] >= info["n_steps"] / 19
    # n=70, d=64: 3 passes per absorbed row plus the first window
    assert tb.Plan(70, 64).info["n_passes"] <= 68 * 3 + 1


def test_turn_steps_run_composed(tb):
    """At each row turn (a top or bottom pass) the pass kernels apply the four
    steps on the turn's two outermost window bits as one 4x4 block (16 real
    multiply-adds per entry instead of 4 x 8)."""
    for n, d, kw in [(70, 64, {}), (70, 63, {}), (30, 40, {}), (13, 26, {"window_bits": 6}),
                     (20, 50, {"bottom_bits": 7, "top_bits": 5})]:
        p = tb.Plan(n, d, **kw)
        turns = sum(1 for s, _, _ in p.schedule if s in ("top", "bot"))
        assert turns > 0
        assert p.info["pass_madds"] == 8 * p.info["n_steps"] - 16 * turns
    assert tb.Plan(12, 24).info["pass_madds"] == 0  # one-CTA kernel: no passes


def test_window_options(tb):
    for wb, bb, tt in [(9, 10, 9), (8, 0, 0), (5, 0, 0), (6, 9, 9), (9, 0, 7)]:
        info = tb.Plan(40, 60, window_bits=wb, bottom_bits=bb, top_bits=tt).info
        assert info["n_passes"] > 0
    with pytest.raises(tb.TbError):
        tb.Plan(40, 60, window_bits=11)
    with pytest.raises(tb.TbError):
        tb.Plan(40, 60, window_bits=4)


@pytest.mark.parametrize("n,d", [(1, 8), (10, 1), (10, 0), (10, 82), (10, 81), (0, 4)])
def test_domain_errors(tb, n, d):
    with pytest.raises(tb.TbError) as e:
        tb.Plan(n, d)
    assert e.value.status == tb.TB_EDOMAIN


def test_argument_errors(tb):
    n, d = 6, 8
    cl = np.zeros((d + 1, n), np.uint8)
    cl[3, 2] = 24
    with pytest.raises(tb.TbError) as e:
        tb.Plan(n, d, cl)
    assert e.value.status == tb.TB_EINVAL
    tm = np.zeros((d, n), np.uint8)
    tm[1, 1] = 2
    with pytest.raises(tb.TbError) as e:
        tb.Plan(n, d, None, tm)
    assert e.value.status == tb.TB_EINVAL
    with pytest.raises(tb.TbError) as e:
        tb.Plan(n, d, extra=[(n, 0, np.eye(2))])
    assert e.value.status == tb.TB_EINVAL


def test_bits_are_checked_before_any_device_work(tb):
    """tb_amplitudes rejects a bitstring entry outside {0,1} on the host."""
    import ctypes
    plan = tb.Plan(6, 8)
    bits = np.zeros((2, 6), np.uint8)
    bits[1, 3] = 2
    out = np.empty(4, np.float64)
    rc = tb._lib.tb_amplitudes(plan.handle, bits.ctypes.data_as(tb._u8p), 2, ctypes.c_void_p(256),
                               1 << 30, out.ctypes.data_as(tb._dp), None)
    assert rc == tb.TB_EINVAL


def test_workspace_sizes(tb):
    plan = tb.Plan(70, 64)
    one = plan.workspace_bytes(1)
    assert one >= (8 << 32)
    assert plan.workspace_min_bytes() >= (8 << 32)
    assert plan.workspace_bytes(16) >= one
    small = tb.Plan(12, 8)
    assert small.workspace_bytes(64) < (1 << 20)


def test_log_xeb_matches_oracle(tb, oracle_mod):
    rng = np.random.default_rng(2)
    amps = (rng.standard_normal(50) + 1j * rng.standard_normal(50)) * 1e-5
    assert abs(tb.log_xeb(amps, 30) - oracle_mod.log_xeb(amps, 30)) < 1e-12


def test_pass_cases_cover_every_shape(tb):
    """The GPU parity cases exercise every pass shape with every window size."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("gpu_parity", os.path.join(ROOT, "tests", "test_gpu_parity.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    seen = set()
    for n, d, wb, bb, tt in mod.PASS_CASES:
        seen |= {(s, m) for s, m, _ in tb.Plan(n, d, window_bits=wb, bottom_bits=bb, top_bits=tt).schedule}
    assert seen == {(s, m) for s in tb.Plan.PASS_SHAPES if s != "tensor" for m in range(5, 11)}


# ------------------------------------------------ split-precision tensor-core schedule

@pytest.mark.parametrize("prec,wb", [("tf32x3", 5), ("bf16x3", 6)])
def test_dense_schedule_shape(tb, prec, wb):
    """Every dense pass spans WB address bits inside the boundary; rows are
    cut into ceil((h - WB) / WB) + 1 chunks each, the first (forward) chunk
    of a row sharing the pass at address bit 0 with the previous row's last."""
    for n in (3, 4, 5, 8, 13):
        for d in range(26, 67, 2):
            h = d // 2
            p = tb.Plan(n, d, precision=prec)
            sched = p.schedule
            assert len(sched) == p.info["n_passes"] > 0
            assert all(s == "tensor" and m == wb and 0 <= lo <= h - wb for s, m, lo in sched)
            per_row = -(-(h - wb) // wb) + 1
            rows = n - 2
            assert len(sched) == rows * per_row - (rows - 1) // 2
            assert sched[0][2] == 0


def test_dense_schedule_options(tb):
    with pytest.raises(tb.TbError) as e:
        tb.Plan(8, 30, precision=3)
    assert e.value.status == tb.TB_EINVAL
    with pytest.raises(ValueError):
        tb.Plan(8, 30, precision="fp16")
    # narrow boundaries keep the single-CTA kernel: no HBM passes
    assert tb.Plan(12, 24, precision="bf16x3").info["n_passes"] == 0
    # dense matrices (hi and lo) are part of the plan's device tables
    fp32 = tb.Plan(70, 64).info
    # tables both forms share: the FP32 form's less its pass-step table (128 B
    # per entry: at most one per step plus a turn block's 8 per pass)
    base = fp32["table_bytes"] - 128 * (fp32["n_steps"] + 8 * fp32["n_passes"]) - 256
    assert tb.Plan(70, 64, precision="bf16x3").info["table_bytes"] >= base + 375 * 2 * 128 * 128 * 2
    assert tb.Plan(70, 64, precision="tf32x3").info["table_bytes"] >= base + 443 * 2 * 64 * 64 * 4


# ------------------------------------------------ open output bits (Algorithm 2)

def test_open_plan_domain_and_width(tb):
    """Algorithm 2 needs 1 <= k <= floor(d/4) (here also k <= 10, k <= n-1 and
    width >= 13); its path keeps width ceil(d/2) (Proposition 2)."""
    for n, d, k in [(16, 26, 6), (70, 64, 8), (70, 70, 10), (40, 66, 10), (13, 26, 1), (4, 26, 3)]:
        p = tb.Plan(n, d, open_k=k)
        assert p.info["open_k"] == k and p.info["open_width"] == (d + 1) // 2
        assert p.row_bytes == n - k
    for n, d, k in [(16, 26, 7), (12, 40, 12), (8, 24, 2), (70, 64, 11), (5, 40, 5)]:
        with pytest.raises(tb.TbError) as e:
            tb.Plan(n, d, open_k=k)
        assert e.value.status == tb.TB_EDOMAIN
    h = ctypes.c_void_p()
    assert tb._lib.tb_plan_create_open(16, 26, None, None, None, 0, None, 0, ctypes.byref(h)) == tb.TB_EDOMAIN


def test_open_plan_workspace_in_place_or_out_of_place(tb):
    """Open plans hold two boundaries per prefix (the tensor-core join writes
    out of place) unless the boundary is wider than 2^33 entries or the HBM
    budget cannot hold two; then one boundary plus, for k >= 4, a scratch of
    one join slice (2^-6 of the rows, at least 128 rows), or no scratch at
    all (FP32 join) when the budget cannot hold that either."""
    h, k = 20, 8
    scratch = max(128, (1 << (h - k)) >> 6) << (k + 3)
    two = tb.Plan(30, 40, open_k=k).workspace_bytes(1)
    one = tb.Plan(30, 40, open_k=k, hbm_budget_bytes=12 << 20).workspace_bytes(1)
    assert two - one == (8 << h) - scratch
    bare = tb.Plan(30, 40, open_k=k, hbm_budget_bytes=(8 << h) + (64 << 10)).workspace_bytes(1)
    assert one - bare == scratch
    assert tb.Plan(30, 40, open_k=k, hbm_budget_bytes=64 << 20).workspace_bytes(1) == two
    w35 = tb.Plan(70, 70, open_k=8)
    assert w35.info["boundary_bits"] == 35
    assert (8 << 35) + (4 << 30) < w35.workspace_bytes(1) < (8 << 35) + (5 << 30)  # + a 4 GiB join slice
    assert tb._lib.tb_workspace_bytes(tb.Plan(70, 72, open_k=8)._h, 1) == -1  # 2^36 entries: counters only


def test_open_plan_sweeps_only_the_fixed_region(tb):
    """The sweep absorbs rows 1..n-k-1 as middle rows: (n-k-1) h paired steps."""
    for n, d, k in [(16, 26, 3), (30, 40, 8), (70, 64, 8)]:
        assert tb.Plan(n, d, open_k=k).info["n_steps"] == (n - k - 1) * (d // 2)
    # the workspace holds one boundary and half a boundary per prefix
    p = tb.Plan(30, 40, open_k=8)
    assert p.workspace_min_bytes() >= p.info["table_bytes"] + 12 * 2 ** 20


def test_batched_sample_inverts_the_conditional_distribution(tb):
    """Sec. 4 batched sampler: b is the smallest suffix whose cumulative
    probability exceeds u Q_a; Q_a is the prefix's marginal mass."""
    rng = np.random.default_rng(1)
    for k in (1, 3, 8):
        amps = rng.standard_normal((5, 1 << k)) + 1j * rng.standard_normal((5, 1 << k))
        u = rng.random(5)
        b, q = tb.batched_sample(amps, u)
        p = np.abs(amps) ** 2
        np.testing.assert_allclose(q, p.sum(axis=1), rtol=1e-14)
        cdf = np.cumsum(p, axis=1)
        ref = np.array([np.searchsorted(cdf[a], u[a] * cdf[a, -1], side="right") for a in range(5)])
        np.testing.assert_array_equal(b, np.minimum(ref, (1 << k) - 1))
    # boundary variates: u = 0 picks the first suffix with mass, u -> 1 the last
    z = np.array([[0, 0, 1, 1, 0, 0, 0, 0]], np.complex128)
    assert tb.batched_sample(z, [0.0])[0][0] == 2
    assert tb.batched_sample(z, [0.999999])[0][0] == 3
    with pytest.raises(tb.TbError):
        tb.batched_sample(z, [1.0])


def test_batched_sampling_tv_identity(oracle_mod):
    """Sec. 4: with prefixes drawn uniformly, the batched sampler's output
    distribution q_k(a, b) = p(a, b) / (A Q_a) is at total variation
    distance (1/2) sum_a |Q_a - 1/A| from p. Checked exactly on the FP64 state
    vector of a small circuit (it pins the identity, not the sampler code)."""
    c = W.random_circuit(10, 12, 10, 0, 77)
    psi = oracle_mod.sv_state(c.n, c.d, oracle_mod.circuit_gates(c))
    p = np.abs(psi) ** 2
    k = 3
    A = 1 << (c.n - k)
    # state index = sum_q x_q 2^q: prefix qubits 0..n-k-1 are the low bits
    pk = p.reshape(1 << k, A)  # [b, a]
    Q = pk.sum(axis=0)
    q = pk / (A * Q[None, :])
    tv = 0.5 * np.abs(q - pk).sum()
    assert abs(tv - 0.5 * np.abs(Q - 1.0 / A).sum()) < 1e-12


def test_autotuner_measures_what_the_device_runs_at_once(tb, monkeypatch):
    """Wide boundaries are evaluated one at a time, so the tuner times the
    part of the batch the device holds and scales it; wide widths try more
    candidates (window placement matters there)."""
    from paper_2608_13110_gb300 import autotune
    seen = []

    def fake_measure(opts, h, nb, n_rows=8, reps=3, seed=1):
        seen.append((h, nb))
        return float(opts["window_bits"] or 11)

    import torch
    monkeypatch.setattr(autotune, "measure", fake_measure)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "no device (host test)")
    monkeypatch.setenv("TB_AUTOTUNE_CACHE", "/nonexistent/dir/tune.json")  # unwritable: best effort
    best = autotune.tune(32, nb=16, use_cache=False)
    assert len(seen) == autotune.WIDE_LIMIT and all(h == 32 for h, _ in seen)
    assert best["window_bits"] == min(o["window_bits"] for o in autotune.candidate_options(32, limit=24)
                                      if o["window_bits"])
    seen.clear()
    autotune.tune(20, nb=16, use_cache=False)
    assert len(seen) == 8
    assert autotune.BATCH_ENTRIES >> 32 == 0  # one width-32 boundary at a time


# ------------------------------------------------ controlled-phase entanglers

def test_cphase_plans_validate_angles_and_keep_counters(tb):
    n, d = 16, 40
    ph = W.random_phases(n, d, 5)
    a, b = tb.Plan(n, d).info, tb.Plan(n, d, cphase=ph).info
    for k in ("width", "log2_cost", "n_steps", "n_passes", "boundary_bytes", "table_bytes"):
        assert a[k] == b[k], k
    assert tb.Plan(n, d, cphase=ph, open_k=4).info["open_k"] == 4
    bad = ph.copy()
    bad[3, 1] = np.nan  # layer 3 couples (1, 2)
    with pytest.raises(tb.TbError) as e:
        tb.Plan(n, d, cphase=bad)
    assert e.value.status == tb.TB_EINVAL
    ok = ph.copy()
    ok[3, 0] = np.nan  # layer 3 does not couple (0, 1): ignored
    tb.Plan(n, d, cphase=ok)
    with pytest.raises(ValueError):
        tb.Plan(n, d, cphase=ph[:, :-1])
    with pytest.raises(tb.TbError) as e:
        tb.Plan(n, d, cphase=ph, open_k=11)
    assert e.value.status == tb.TB_EDOMAIN


def test_null_and_out_of_range_arguments_fail_without_device_work(tb):
    """Every entry point that takes host pointers or sizes refuses bad ones
    with a status (no exception crosses the ABI, no CUDA call is made)."""
    import ctypes
    L = tb._lib
    info = tb._Info()
    assert L.tb_plan_info(None, ctypes.byref(info)) == tb.TB_EINVAL
    plan = tb.Plan(8, 10)
    assert L.tb_plan_info(plan._h, None) == tb.TB_EINVAL
    assert L.tb_workspace_bytes(None, 1) == -1
    assert L.tb_workspace_bytes(plan._h, -1) == -1
    assert L.tb_plan_schedule(None, None, 0) == -1
    m = (ctypes.c_double * 8)()
    assert L.tb_clifford_matrix(24, m) == tb.TB_EINVAL
    assert L.tb_clifford_matrix(-1, m) == tb.TB_EINVAL
    out = ctypes.c_double(0.0)
    amps = np.ones(4, np.float64)
    assert L.tb_log_xeb(None, 2, 10, ctypes.byref(out)) == tb.TB_EINVAL
    assert L.tb_log_xeb(amps.ctypes.data_as(tb._dp), 0, 10, ctypes.byref(out)) == tb.TB_EINVAL
    # the device reduction checks its arguments before any device work
    assert L.tb_log_xeb_device(None, 2, 10, None, None) == tb.TB_EINVAL
    assert L.tb_log_xeb_device(ctypes.c_void_p(16), 0, 10, ctypes.c_void_p(16), None) == tb.TB_EINVAL
    assert L.tb_log_xeb_device(ctypes.c_void_p(16), 2, 0, ctypes.c_void_p(16), None) == tb.TB_EINVAL
    assert L.tb_plan_create(8, 10, None, None, None, 0, None, None) == tb.TB_EINVAL
    h = tb._vp()
    assert L.tb_plan_create(8, 10, None, None, None, -1, None, ctypes.byref(h)) == tb.TB_EINVAL
    assert L.tb_plan_create_cphase(16, 40, None, None, None, 0, None, None, -2, ctypes.byref(h)) == tb.TB_EDOMAIN
    # the sampler: variates outside [0, 1), k out of range
    z = np.zeros(2 * 4, np.float64)
    z[0] = 1.0
    u = np.array([1.0])
    b = (ctypes.c_int32 * 1)()
    assert L.tb_batched_sample(z.ctypes.data_as(tb._dp), 2, 1, u.ctypes.data_as(tb._dp), b, None) == tb.TB_EINVAL
    u = np.array([0.5])
    assert L.tb_batched_sample(z.ctypes.data_as(tb._dp), 31, 1, u.ctypes.data_as(tb._dp), b, None) == tb.TB_EINVAL
    assert L.tb_batched_sample(z.ctypes.data_as(tb._dp), 2, 1, u.ctypes.data_as(tb._dp), b, None) == tb.TB_OK
    assert b[0] == 0
    # every status has a message
    for st in range(0, 7):
        assert L.tb_status_str(st)
