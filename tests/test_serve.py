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
    budget = max(serve.device_bytes(r) for r in reqs) + serve.device_bytes(reqs[0])
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
