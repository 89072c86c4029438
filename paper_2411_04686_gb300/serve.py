"""Serving loop for stepped GSE-CG solves: continuous batching with admission by
HBM footprint.

Requests (a CSR matrix and a right-hand side) arrive over time.  The server
keeps one continuous-batching engine (``gse_engine_*``) running: whenever a
slot and enough device memory are free, the oldest waiting request is encoded
(``gse_encode``), its Krylov workspace allocated and the system submitted; the
engine advances every active system by a few iteration slots per step, and
finished systems leave (their memory is released), so later arrivals join
while earlier ones are still on the GPU.  Each result is independent of what
else runs (the engine's per-system partition and reduction order depend only
on the system), which the tests check bit for bit.

A step is pipelined: the engine's slots are launched without waiting
(``gse_engine_launch``), the host encodes the requests admitted into the slots
freed by the previous step while the device runs them, and only then waits
(``gse_engine_wait``), collects finished systems and submits the new ones.
Encoding thus overlaps the solves instead of alternating with them.

The admission rule (``admit``) and the footprint estimate
(``estimate_footprint``) are plain host functions, tested on the CPU with a fake
clock and a fake memory budget.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np


def estimate_footprint(n_rows: int, nnz: int, seg_bits=(16, 16, 20), group=32, method: str = "cg") -> int:
    """Device bytes a request will hold (upper estimate, before encoding):
    padded segment arrays, column indices, row metadata, Krylov workspace
    (CG: r, p, q plus x and b), reduction scratch."""
    pad = ((nnz + 1023) // 1024 + 1) * 1024
    seg_bytes = sum(2 if s <= 16 else 2 + (s - 16) / 8 for s in seg_bits) * pad
    matrix = pad * 4 + seg_bytes + pad // group * 2 + pad // 8 + 4 * (n_rows + 1) + 16 * (pad // 256) + 65536
    vectors = 8 * (n_rows + 1) * (5 if method == "cg" else 35)
    return int(matrix + vectors + (1 << 20))


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float
    n_rows: int
    nnz: int
    payload: object = None          # whatever the caller needs to build the system
    footprint: int = 0


def admit(queue: deque, free_slots: int, free_bytes: int) -> list:
    """Admission: in arrival order, take requests while a slot is free and the
    request's footprint fits in the remaining budget.  A request that does not
    fit blocks those behind it (first-come first-served, no starvation)."""
    out = []
    while queue and free_slots > 0:
        r = queue[0]
        if r.footprint > free_bytes:
            break
        queue.popleft()
        out.append(r)
        free_slots -= 1
        free_bytes -= r.footprint
    return out


@dataclasses.dataclass
class Completion:
    rid: int
    arrival: float
    admitted: float
    finished: float
    info: dict


class Server:
    """Continuous-batching CG server on the current CUDA device.

    build(payload) -> (synth.CSR, b numpy array) turns a request into a system.
    mem_budget: bytes the server may hold on the device (None: the free memory
    at start minus a 10% reserve).
    """

    def __init__(self, build, capacity: int = 64, mem_budget: int | None = None, tol: float = 1e-10,
                 policy=None, slots_per_step: int = 16, clock=time.perf_counter, engine=None, place=None,
                 backlog_slots_per_step: int | None = None):
        self.build = build
        self.capacity = capacity
        self.tol = tol
        self.slots_per_step = slots_per_step
        # longer steps while requests wait: fewer host round trips when the
        # device is the bottleneck, short steps (low latency) when it is not
        self.backlog_slots_per_step = backlog_slots_per_step or slots_per_step
        self.clock = clock
        if engine is None:                 # the real device engine
            import torch

            import paper_2411_04686_gb300 as gse
            self.policy = policy or gse.SCALED_CG
            if mem_budget is None:
                free, _ = torch.cuda.mem_get_info()
                mem_budget = int(free * 0.9)
            engine = gse.Engine(capacity)
            place = place or _place_on_device
        else:                              # host-side tests inject an engine and a placement
            self.policy = policy
        self.engine = engine
        self.place = place
        self.mem_budget = mem_budget if mem_budget is not None else 1 << 62
        self.used = 0
        self.queue: deque = deque()
        self.active = {}                # slot -> (request, admitted time, placed system)
        self.done: list[Completion] = []
        self.inflight = False           # an engine launch not yet waited for

    def submit(self, req: Request):
        if not req.footprint:
            req.footprint = estimate_footprint(req.n_rows, req.nnz)
        self.queue.append(req)

    def step(self) -> int:
        """Encode what fits while the device runs the previous launch, then
        collect finished solves, submit the encoded ones and launch the next
        slots.  Returns the number of systems still running."""
        ready = []
        for req in admit(self.queue, self.capacity - len(self.active), self.mem_budget - self.used):
            A, b = self.build(req.payload)
            ready.append((req, self.clock(), self.place(A, b)))   # (matrix handle, b, x) on the device
            self.used += req.footprint
        running = self.engine.wait() if self.inflight else 0
        self.inflight = False
        for slot, info in self.engine.poll():
            req, t_adm, sysm = self.active.pop(slot)
            self.done.append(Completion(req.rid, req.arrival, t_adm, self.clock(), info))
            self.used -= req.footprint
            sysm[0].free()
        for req, t_adm, sysm in ready:
            slot = self.engine.submit(sysm[0], sysm[1], sysm[2], self.tol, self.policy)
            self.active[slot] = (req, t_adm, sysm)
        if self.active:
            n = self.backlog_slots_per_step if self.queue else self.slots_per_step
            self.engine.launch(n, batch=n)
            self.inflight = True
        return running

    def drain(self):
        while self.queue or self.active:
            self.step()

    def close(self):
        self.engine.close()


def _place_on_device(A, b):
    """Encodes A (gse_encode) and puts b and a zero initial guess on the device."""
    import torch

    import paper_2411_04686_gb300 as gse
    M = gse.GseMatrix.from_csr(A)
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    return M, bd, x


def latency_stats(done: list) -> dict:
    lat = np.array([c.finished - c.arrival for c in done])
    if lat.size == 0:
        return {"n": 0}
    return {"n": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}


def poisson_arrivals(count: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times of a Poisson process with the given rate (requests/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def shard(items: list, rank: int, world: int) -> list:
    """Requests of one rank when N replicas split a stream (round robin)."""
    return items[rank::world]
