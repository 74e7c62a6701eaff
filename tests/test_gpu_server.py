"""The serving runtime (tb_server_*): requests of different sizes submitted
together run concurrently, queue for memory when the budget is tight, and
every result equals the same request evaluated alone."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def tb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_13110_gb300 import build as b
    b.build()
    import paper_2608_13110_gb300 as mod
    return mod


def _mix():
    shapes = [(12, 8, 64), (30, 40, 3), (20, 34, 17), (9, 20, 128), (24, 44, 5), (16, 28, 40),
              (70, 36, 2), (18, 24, 256), (25, 30, 33), (6, 16, 7), (40, 40, 4), (14, 26, 12)]
    return [W.random_circuit(n, d, None, nb, 700 + i) for i, (n, d, nb) in enumerate(shapes)]


def test_results_alone_and_in_the_mix_agree(tb):
    circuits = _mix()
    plans = [tb.Plan.from_circuit(c) for c in circuits]
    alone = [p.amplitudes(c.bits) for p, c in zip(plans, circuits)]
    srv = tb.Server(hbm_budget_bytes=4 << 30, slots=4)
    try:
        tickets = [srv.submit(p, c.bits) for p, c in zip(plans, circuits)]
        for t, ref in zip(tickets, alone):
            got, st = srv.wait(t, timeout=120.0)
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
            assert st["latency_s"] >= st["queue_s"] >= 0.0
        stats = srv.stats()
        assert stats["completed"] == len(circuits)
        assert stats["amplitudes"] == sum(c.bits.shape[0] for c in circuits)
        assert stats["peak_concurrent"] >= 2, "requests should overlap on the device"
        assert stats["peak_bytes_in_use"] <= 4 << 30
        assert 0 < stats["p50_latency_s"] <= stats["p99_latency_s"]
    finally:
        srv.close()


def test_tight_budget_queues_instead_of_failing(tb):
    """Each request fits the budget alone but not all at once: they wait for
    memory and all complete with the same amplitudes."""
    circuits = [W.random_circuit(20, 44, None, 8, 800 + i) for i in range(5)]  # width 22: 32 MiB per boundary
    plans = [tb.Plan.from_circuit(c) for c in circuits]
    alone = [p.amplitudes(c.bits) for p, c in zip(plans, circuits)]
    srv = tb.Server(hbm_budget_bytes=96 << 20, slots=4)
    try:
        tickets = [srv.submit(p, c.bits) for p, c in zip(plans, circuits)]
        for t, ref in zip(tickets, alone):
            got, _ = srv.wait(t, timeout=120.0)
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
        assert srv.stats()["peak_bytes_in_use"] <= 96 << 20
    finally:
        srv.close()


def test_request_beyond_the_budget_is_rejected(tb):
    srv = tb.Server(hbm_budget_bytes=16 << 20, slots=2)
    try:
        c = W.random_circuit(20, 48, None, 1, 9)  # width 24: 128 MiB boundary
        with pytest.raises(tb.TbError) as e:
            srv.submit(tb.Plan.from_circuit(c), c.bits)
        assert e.value.status == tb.TB_ENOMEM
        bad = np.full((1, 6), 2, np.uint8)
        with pytest.raises(tb.TbError):
            srv.submit(tb.Plan(6, 8), bad)
    finally:
        srv.close()


def test_wait_times_out_and_the_ticket_stays_valid(tb):
    c = W.random_circuit(40, 52, None, 2, 10)  # width 26: a few hundred ms
    plan = tb.Plan.from_circuit(c)
    srv = tb.Server(hbm_budget_bytes=2 << 30, slots=1)
    try:
        t = srv.submit(plan, c.bits)
        with pytest.raises(TimeoutError):
            srv.wait(t, timeout=0.0)
        got, _ = srv.wait(t, timeout=120.0)
        ref = plan.amplitudes(c.bits)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    finally:
        srv.close()


def test_wide_requests_queue_in_arrival_order(tb):
    """Admission at realistic sizes: two width-28 requests (2 GiB boundary
    each) and small ones under a 3 GiB budget. The second wide request cannot
    start until the first has finished; the small requests submitted after it
    wait behind it (arrival order: the head of the queue is admitted first),
    while the small request submitted before it runs beside the first wide
    one. Every result equals the request evaluated alone, and the device
    memory in use never exceeds the budget."""
    budget = 3 << 30
    wide1 = W.random_circuit(30, 56, None, 2, 910)
    wide2 = W.random_circuit(32, 56, None, 1, 911)
    small = [W.random_circuit(20, 30, None, 32, 912 + i) for i in range(4)]
    order = [wide1, small[0], wide2, small[1], small[2], small[3]]
    plans = [tb.Plan.from_circuit(c) for c in order]
    assert plans[0].info["boundary_bytes"] == 2 << 30 and plans[2].info["boundary_bytes"] == 2 << 30
    alone = [p.amplitudes(c.bits) for p, c in zip(plans, order)]
    srv = tb.Server(hbm_budget_bytes=budget, slots=4)
    try:
        tickets = [srv.submit(p, c.bits) for p, c in zip(plans, order)]
        res = [srv.wait(t, timeout=300.0) for t in tickets]
        for (got, _), ref in zip(res, alone):
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
        st = [s for _, s in res]
        w1, s0, w2 = st[0], st[1], st[2]
        # the second wide request waited for the first one's memory
        assert w2["queue_s"] >= 0.5 * w1["latency_s"]
        # arrival order: nothing submitted after it was admitted before it
        for s in st[3:]:
            assert s["queue_s"] >= w2["queue_s"] - 0.05
        # the small request submitted before it ran beside the first wide one
        assert s0["queue_s"] < 0.5 * w1["latency_s"] and s0["latency_s"] < w1["latency_s"]
        stats = srv.stats()
        assert stats["peak_bytes_in_use"] <= budget
        assert stats["completed"] == len(order)
    finally:
        srv.close()
