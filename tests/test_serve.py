"""Host-side checks of the serving scheduler (admission by slots and HBM budget, FIFO,
overlap) with a fake executor: no GPU needed."""
import time

import numpy as np
import pytest

from paper_2410_02314_gb300 import serve


def make_reqs(shapes, arrivals):
    return [serve.Request(rid=k, frames=np.zeros(s, np.uint16), arrival=a) for k, (s, a) in
            enumerate(zip(shapes, arrivals))]


def test_budget_is_never_exceeded_and_all_complete():
    shapes = [(4, 64, 64), (8, 64, 64), (2, 128, 128), (6, 64, 64), (1, 256, 256), (3, 64, 64)]
    reqs = make_reqs(shapes, [0.0] * len(shapes))
    budget = max(serve.request_bytes(r) for r in reqs) + serve.request_bytes(reqs[0])
    ex = serve.FakeExecutor(4, 2e-3, time.perf_counter)
    sch = serve.Scheduler(ex, budget)
    out = sch.run(reqs)
    assert all(r.done >= r.admitted >= r.arrival for r in out)
    assert sch.peak_in_use <= budget
    assert sch.max_queue >= 1  # the budget made requests wait


def test_fifo_admission_order():
    shapes = [(2, 64, 64)] * 6
    reqs = make_reqs(shapes, [0.0, 0.001, 0.002, 0.003, 0.004, 0.005])
    ex = serve.FakeExecutor(1, 3e-3, time.perf_counter)
    out = serve.Scheduler(ex, 1 << 30).run(reqs)
    adm = [r.admitted for r in sorted(out, key=lambda r: r.arrival)]
    assert adm == sorted(adm)


def test_concurrent_slots_overlap():
    reqs = make_reqs([(5, 64, 64)] * 3, [0.0, 0.0, 0.0])
    ex = serve.FakeExecutor(3, 2e-3, time.perf_counter)
    serve.Scheduler(ex, 1 << 30).run(reqs)
    assert ex.concurrent_peak == 3


def test_request_above_budget_is_rejected():
    reqs = make_reqs([(100, 512, 512)], [0.0])
    with pytest.raises(ValueError):
        serve.Scheduler(serve.FakeExecutor(1, 1e-3, time.perf_counter), 1 << 20).run(reqs)


def test_report_percentiles():
    reqs = make_reqs([(1, 8, 8)] * 100, list(np.linspace(0, 0.99, 100)))
    for k, r in enumerate(reqs):
        r.done = r.arrival + (k + 1) * 1e-3
    rep = serve.report(reqs)
    assert abs(rep["p50_ms"] - 50.5) < 1e-6 and abs(rep["p99_ms"] - 99.01) < 1e-6


def test_record_capacity_bounds_detections():
    # detections are pairwise non-adjacent, so one per 2x2 block at most
    assert serve.record_capacity(1, 31, 50) == 16 * 25 and serve.record_capacity(2, 40, 40) == 800


def plan_cost(H, W):
    """A stand-in for the library's per-frame-size workspace: 1 MB per 4096 pixels."""
    return H * W // 4096 * (1 << 20)


def test_workspaces_count_against_the_budget():
    """A slot that runs a new frame size is charged its workspace, which stays resident: the
    budget bounds resident workspaces plus running requests at every admission, and a request
    whose workspace cannot fit next to the resident ones is refused up front."""
    shapes = [(2, 64, 64), (2, 128, 128), (2, 64, 64), (1, 256, 256), (2, 128, 128), (3, 64, 64)]
    reqs = make_reqs(shapes, [0.0] * len(shapes))
    ex = serve.FakeExecutor(2, 1e-3, time.perf_counter, plan_cost=plan_cost)
    budget = plan_cost(256, 256) + plan_cost(128, 128) + 3 * max(serve.request_bytes(r) for r in reqs)
    sch = serve.Scheduler(ex, budget)
    out = sch.run(reqs)
    assert all(r.done >= r.admitted >= r.arrival and r.error is None for r in out)
    assert sch.peak_in_use <= budget
    assert ex.resident_bytes() > 0 and sch.peak_in_use >= ex.resident_bytes()
    # the same stream under a budget that only the small sizes' workspaces fit
    small = plan_cost(128, 128) + 2 * max(serve.request_bytes(r) for r in reqs)
    ex2 = serve.FakeExecutor(2, 1e-3, time.perf_counter, plan_cost=plan_cost)
    with pytest.raises(ValueError, match="request 3"):
        serve.Scheduler(ex2, small).run(make_reqs(shapes, [0.0] * len(shapes)))


def test_resident_workspaces_make_requests_wait():
    """Two slots each holding a large workspace leave room for one more only: a request of a
    third size waits until the workspaces it would add fit (here: never on a busy slot, so it
    runs on the slot that already holds its size)."""
    shapes = [(1, 256, 256), (1, 192, 192), (1, 256, 256), (1, 192, 192)]
    reqs = make_reqs(shapes, [0.0, 0.0, 0.001, 0.001])
    ex = serve.FakeExecutor(2, 2e-3, time.perf_counter, plan_cost=plan_cost)
    budget = plan_cost(256, 256) + plan_cost(192, 192) + 2 * max(serve.request_bytes(r) for r in reqs)
    sch = serve.Scheduler(ex, budget)
    out = sch.run(reqs)
    assert sch.peak_in_use <= budget
    # each size stayed on the slot that first ran it: no slot took a second workspace
    assert all(len(p) == 1 for p in ex.plans)
    assert {r.slot for r in out if r.shape[1] == 256} != {r.slot for r in out if r.shape[1] == 192}


def test_a_device_error_fails_its_request_only():
    """A request whose kernels reported an error (the context's error word) finishes as failed,
    without records; the others complete and the report counts the failure."""
    reqs = make_reqs([(2, 64, 64)] * 5, [0.0] * 5)
    ex = serve.FakeExecutor(2, 1e-3, time.perf_counter, fail_rids={2})
    sch = serve.Scheduler(ex, 1 << 30)
    out = sch.run(reqs)
    assert [r.rid for r in out if r.error] == [2] and out[2].records is None
    assert all(r.records is not None for r in out if r.rid != 2)
    assert sch.failed == 1 and serve.report(out)["failed"] == 1
