"""The serving scheduler on the CPU (no GPU): requests are admitted in arrival order onto free
slots, never before they arrive, never beyond the slot count, and only with memory headroom."""
import threading
import time

from paper_2306_09189_gb300.serve import Request, Server, latency_stats


class FakeWorker:
    active = 0
    peak = 0
    lock = threading.Lock()

    def __init__(self, dt):
        self.dt = dt

    def run(self, m, coeffs):
        with FakeWorker.lock:
            FakeWorker.active += 1
            FakeWorker.peak = max(FakeWorker.peak, FakeWorker.active)
        time.sleep(self.dt)
        with FakeWorker.lock:
            FakeWorker.active -= 1
        return ["out-%d" % coeffs]


def test_slots_bound_concurrency_and_arrivals_are_respected():
    FakeWorker.active = FakeWorker.peak = 0
    srv = Server(None, {}, 0, reserve_bytes=0, export=False, workers=[FakeWorker(0.05) for _ in range(3)],
                 hbm_free=lambda: 1)
    reqs = [Request(i, 0.01 * i, 32, i) for i in range(9)]
    out = srv.serve(reqs)
    assert [r.rid for r in out] == list(range(9))
    assert FakeWorker.peak == 3                       # three slots used at once, never more
    for r in out:
        assert r.start >= r.arrival - 1e-3 and r.finish >= r.start + 0.045
        assert r.result == ["out-%d" % r.rid]
    st = latency_stats(out)
    assert st["p99_ms"] >= st["p50_ms"] > 40


def test_admission_waits_for_memory_headroom():
    FakeWorker.active = FakeWorker.peak = 0
    t0 = time.perf_counter()
    free = {"v": 0}

    def hbm_free():
        if time.perf_counter() - t0 > 0.1:
            free["v"] = 10
        return free["v"]

    srv = Server(None, {}, 0, reserve_bytes=5, export=False, workers=[FakeWorker(0.01)], hbm_free=hbm_free)
    out = srv.serve([Request(0, 0.0, 32, 0)])
    assert out[0].start >= 0.1                        # held back until memory freed up


def test_polynomial_depth_and_products_match_the_oracle_recursion():
    # the serving planner's level budget and the bench's key-switch count follow the
    # Paterson-Stockmeyer recursion the library runs (the oracle's cheb_ps_he pins its depth)
    from paper_2306_09189_gb300 import host
    from oracle import layers as Ly
    assert [host.ps_depth(d) for d in (5, 16, 27, 59)] == [3, 5, 5, 6]
    assert [host.ps_products(d) for d in (5, 16, 27, 59)] == [4, 8, 11, 16]
    for d in (5, 16, 27, 59):
        k, giants = Ly.cheb_ps_params(d)
        assert host.ps_products(d) >= k - 1 + len(giants) - 1
