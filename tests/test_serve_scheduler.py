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


def test_batched_steps_take_the_oldest_requests_stage_in_power_of_two_groups():
    from paper_2306_09189_gb300.serve import next_group
    sizes = [1, 2, 4, 8]
    # (arrival, rid, resolution, stage)
    waiting = [(0.0, 0, 32, 2), (0.1, 1, 32, 0), (0.2, 2, 32, 0), (0.3, 3, 64, 0), (0.4, 4, 32, 0),
               (0.5, 5, 32, 0)]
    assert next_group(waiting, sizes) == ((32, 2), [0])            # the oldest request goes first
    rest = waiting[1:]
    assert next_group(rest, sizes) == ((32, 0), [1, 2, 4, 5])      # four of its stage join it
    assert next_group(rest[:3], sizes) == ((32, 0), [1, 2])        # three waiting: a group of two
    many = [(0.01 * i, i, 32, 1) for i in range(11)]
    assert next_group(many, sizes) == ((32, 1), list(range(8)))    # capped at the largest size
    assert next_group([(0.0, 9, 64, 3)], sizes) == ((64, 3), [9])


def test_admission_refuses_to_wait_forever_for_memory():
    # nothing runs to free memory and none comes free: the server reports it instead of spinning
    import pytest
    srv = Server(None, {}, 0, reserve_bytes=5, export=False, workers=[FakeWorker(0.01)], hbm_free=lambda: 1,
                 admit_timeout=0.2)
    with pytest.raises(MemoryError):
        srv.serve([Request(0, 0.0, 32, 0)])
