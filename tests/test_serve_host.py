"""Host logic of the serving loop, on the CPU with a fake clock, a fake memory
budget and a fake engine: admission by footprint in arrival order, continuous
batching (requests join as slots free up), latency bookkeeping, sharding."""
from collections import deque

import numpy as np
import pytest

from paper_2411_04686_gb300 import serve


def test_admit_respects_slots_and_budget_in_order():
    q = deque(serve.Request(i, float(i), 10, 50, footprint=f) for i, f in enumerate([40, 30, 50, 10]))
    got = serve.admit(q, free_slots=3, free_bytes=80)
    assert [r.rid for r in got] == [0, 1]          # 40 + 30 fit, 50 does not: it blocks request 3
    assert [r.rid for r in q] == [2, 3]
    assert serve.admit(q, free_slots=0, free_bytes=10**9) == []
    assert [r.rid for r in serve.admit(q, 5, 60)] == [2, 3]


def test_footprint_grows_with_size_and_method():
    a = serve.estimate_footprint(1000, 5000)
    b = serve.estimate_footprint(100000, 500000)
    assert b > a > 5000 * 10
    assert serve.estimate_footprint(1000, 5000, method="gmres") > a
    # per extra row at fixed nnz: a row pointer plus the Krylov vectors in FP64,
    # CG r, p, q, x, b (5) and GMRES(30) its 31 basis vectors, x and b (33)
    d = 1000
    for method, vecs in (("cg", 5), ("gmres", 33)):
        grow = serve.estimate_footprint(1000 + d, 5000, method=method) - serve.estimate_footprint(1000, 5000, method=method)
        assert grow >= (8 * vecs + 4) * d, method


class FakeEngine:
    """Each submitted system finishes after `need` slots of engine time."""

    def __init__(self, capacity, need):
        self.capacity, self.need = capacity, need
        self.slots = {}
        self.t = 0

    def submit(self, M, b, x, tol, policy):
        s = next(i for i in range(self.capacity) if i not in self.slots)
        self.slots[s] = [self.need[M.rid], M.rid]
        return s

    pending = None

    def run(self, nslots, batch=8):
        self.t += nslots
        for v in self.slots.values():
            v[0] -= nslots
        return sum(1 for v in self.slots.values() if v[0] > 0)

    def launch(self, nslots, batch=8):
        # like the device engine: one launch in flight at a time, its results
        # visible only after wait()
        assert self.pending is None, "launch while the previous launch is in flight"
        self.pending = (nslots, batch)

    def wait(self):
        assert self.pending is not None, "wait without a launch"
        nslots, batch = self.pending
        self.pending = None
        return self.run(nslots, batch)

    def poll(self):
        out = [(s, {"status": 0, "rid": v[1]}) for s, v in self.slots.items() if v[0] <= 0]
        for s, _ in out:
            del self.slots[s]
        return out

    def close(self):
        pass


class FakeMatrix:
    def __init__(self, rid):
        self.rid = rid
        self.freed = False

    def free(self):
        self.freed = True


def test_continuous_batching_with_fake_engine_and_clock():
    need = {0: 30, 1: 10, 2: 10, 3: 10, 4: 5}
    eng = FakeEngine(2, need)
    clock = {"t": 0.0}
    placed = []

    def place(A, b):
        m = FakeMatrix(A)
        placed.append(m)
        return m, None, None

    srv = serve.Server(build=lambda rid: (rid, None), capacity=2, mem_budget=100, slots_per_step=10,
                       clock=lambda: clock["t"], engine=eng, place=place)
    for rid in range(5):
        srv.submit(serve.Request(rid, 0.0, 1, 1, payload=rid, footprint=40))
    order = []
    while srv.queue or srv.active:
        clock["t"] += 1.0
        srv.step()
        order = [c.rid for c in srv.done]
    # two slots and a budget for two: 0 and 1 start; 1 leaves after one launch and
    # 2 joins while 0 is still running (continuous batching), and so on; a freed
    # slot is refilled one launch later, the next request being encoded while the
    # device runs that launch
    assert order == [1, 0, 2, 3, 4]
    c = {x.rid: x for x in srv.done}
    assert c[2].admitted < c[0].finished
    assert all(m.freed for m in placed)
    assert srv.used == 0
    lat = serve.latency_stats(srv.done)
    assert lat["n"] == 5 and lat["p50_s"] > 0


def test_memory_budget_limits_concurrency():
    eng = FakeEngine(8, {i: 10 for i in range(6)})
    peak = {"v": 0}
    srv = serve.Server(build=lambda rid: (rid, None), capacity=8, mem_budget=100, slots_per_step=10,
                       clock=lambda: 0.0, engine=eng, place=lambda A, b: (FakeMatrix(A), None, None))
    for rid in range(6):
        srv.submit(serve.Request(rid, 0.0, 1, 1, payload=rid, footprint=45))
    while srv.queue or srv.active:
        srv.step()
        peak["v"] = max(peak["v"], len(srv.active))
    assert peak["v"] <= 2 and len(srv.done) == 6


def test_poisson_arrivals_and_shard():
    t = serve.poisson_arrivals(20000, rate=100.0, seed=0)
    assert np.all(np.diff(t) > 0)
    assert t[-1] / 20000 == pytest.approx(0.01, rel=0.05)
    items = list(range(11))
    parts = [serve.shard(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items and all(parts)
    # round robin, so every rank sees the whole arrival span
    assert parts == [[0, 3, 6, 9], [1, 4, 7, 10], [2, 5, 8]]


def test_latency_runs_from_arrival_to_completion():
    """Latency is finished - arrival (queueing and encoding included); p50 and
    p99 by linear interpolation between order statistics: for the latencies
    1, 2, ..., 101 they are 51 and 100."""
    done = [serve.Completion(i, arrival=10.0 * i, admitted=10.0 * i + 0.5 * (i + 1), finished=10.0 * i + i + 1,
                             info={}) for i in range(101)]
    st = serve.latency_stats(done)
    assert st["n"] == 101 and st["p50_s"] == pytest.approx(51.0) and st["p99_s"] == pytest.approx(100.0)
    assert st["mean_s"] == pytest.approx(51.0)
    assert serve.latency_stats([]) == {"n": 0}


def test_longer_steps_only_while_requests_wait():
    eng = FakeEngine(1, {0: 10, 1: 10})
    steps = []
    orig = eng.launch

    def launch(n, batch=8):
        steps.append(n)
        orig(n, batch)

    eng.launch = launch
    srv = serve.Server(build=lambda rid: (rid, None), capacity=1, mem_budget=100, slots_per_step=4,
                       clock=lambda: 0.0, engine=eng, place=lambda A, b: (FakeMatrix(A), None, None),
                       backlog_slots_per_step=8)
    for rid in range(2):
        srv.submit(serve.Request(rid, 0.0, 1, 1, payload=rid, footprint=10))
    while srv.queue or srv.active:
        srv.step()
    assert steps[0] == 8 and steps[-1] == 4          # request 1 waits at first, not at the end
    assert [c.rid for c in srv.done] == [0, 1]
