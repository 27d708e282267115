"""Admission and accounting of the serving loop, with a fake solver (no GPU)."""
import threading
import time

from paper_1703_10973_gb300.serve import Request, Server, estimate_bytes


class _Fake:
    def __init__(self, dur=0.02):
        self.dur = dur
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0
        self.order = []

    def __call__(self, d, stream):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            self.order.append(d)
        time.sleep(self.dur)
        with self.lock:
            self.active -= 1
        return dict(converged=True, obj_p=float(d), relgap=0.0, iters=1, device_bytes=0)


def _reqs(sizes, gap=0.0):
    return [Request(rid=i, data=i, arrival=i * gap, est_bytes=b) for i, b in enumerate(sizes)]


def test_budget_limits_concurrency():
    fake = _Fake()
    srv = Server(budget_bytes=300, slots=8, solver=fake, make_stream=lambda: None)
    res = srv.run(_reqs([100] * 10))
    assert all(r.ok for r in res)
    assert fake.max_active <= 3
    assert srv.stats["max_in_flight_bytes"] <= 300
    assert srv.stats["completed"] == 10


def test_slots_limit_concurrency_and_fifo_order():
    fake = _Fake()
    srv = Server(budget_bytes=10 ** 12, slots=2, solver=fake, make_stream=lambda: None)
    srv.run(_reqs([1] * 6, gap=0.001))
    assert fake.max_active <= 2
    assert fake.order == sorted(fake.order)   # first come, first served


def test_oversize_request_rejected_others_served():
    fake = _Fake(0.005)
    srv = Server(budget_bytes=100, slots=4, solver=fake, make_stream=lambda: None)
    res = srv.run(_reqs([50, 500, 50]))
    assert [r.ok for r in res] == [True, False, True]
    assert "budget" in res[1].error
    assert srv.stats["rejected"] == 1


def test_latency_includes_waiting():
    fake = _Fake(0.03)
    srv = Server(budget_bytes=10 ** 12, slots=1, solver=fake, make_stream=lambda: None)
    res = srv.run(_reqs([1, 1, 1]))
    lat = [r.latency for r in res]
    assert lat[2] >= 0.08              # waited for the two before it
    assert srv.stats["p99_ms"] >= srv.stats["p50_ms"]


def test_failed_solve_reported():
    def bad(d, stream):
        raise RuntimeError("boom")
    srv = Server(budget_bytes=10 ** 12, slots=2, solver=bad, make_stream=lambda: None)
    res = srv.run(_reqs([1, 1]))
    assert not any(r.ok for r in res) and all("boom" in r.error for r in res)


def test_estimate_grows_with_size():
    assert estimate_bytes(100, 1000, 2) < estimate_bytes(200, 1000, 2) < estimate_bytes(200, 5000, 2)
