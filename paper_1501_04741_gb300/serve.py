"""Continuous-batching server for adjoint-LBM sensitivity requests.

A request is one unsteady sensitivity solve (primal N steps, adjoint N
steps, gradient).  The server

* admits queued requests (first come, first served) while their device
  footprint fits the HBM left: a byte model per request (populations pool,
  adjoint buffers, gradient, theta, flags, objective record) is charged
  against a capacity fixed at start (free HBM minus a reserve);
* keeps admitted requests resident as solver handles with their own state
  pool (the pool size caps the checkpoint schedule of that request);
* every tick groups the resident requests by kernel family (lattice,
  collision, scalars, storage) and phase (primal / adjoint) and advances each
  group by up to ``steps_per_tick`` steps with batched launches (one kernel
  per step for the whole group), so requests that arrive while others run
  join the next tick and their work overlaps on the device; each group
  launches on its own CUDA stream (a request moving between groups carries
  the order of its queued work along, ``Solver.set_stream``), so the
  groups' launches also overlap one another, and the tick waits for all
  group streams at its end;
* retires finished requests (J and dJ/dtheta copied out), frees their
  memory and admits from the queue again.

Per-request latency (arrival to result on the host), p50/p99 and node-update
throughput are reported.  ``run_sequential`` is the baseline: the same
requests one at a time, each solved alone in FIFO order.

Every step runs in the CUDA library; this module is scheduling only.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np
import torch

from .albm import AlbmError, Solver, batch_adjoint_step, batch_primal_step
from .inputs import Problem

Q_FLUID = {"D2Q9": 9, "D3Q19": 19}
Q_SCALAR = {"D2Q9": 9, "D3Q19": 7}
STORAGE = {"fp32": 4, "bf16": 2, "fp16": 2}
OOM = 2          # LBM_ERR_OOM


def densities(P: Problem) -> int:
    return Q_FLUID[P.lattice] + P.nscalars * Q_SCALAR[P.lattice]


# device allocations are charged in whole 2 MiB pages, the granularity of
# cudaMalloc's mappings (the library carves the pool's states out of larger
# slabs, so the pool itself costs its bytes plus at most one page)
ALLOC_GRANULE = 2 << 20


def _alloc(nbytes: float) -> int:
    return int(-(-int(nbytes) // ALLOC_GRANULE) * ALLOC_GRANULE)


def state_bytes(P: Problem) -> int:
    return densities(P) * P.n_nodes * STORAGE[P.precision]


def _stride(P: Problem) -> int:
    """Bytes one pool state occupies (its size rounded up to 256)."""
    return -(-state_bytes(P) // 256) * 256


def pool_states(P: Problem, max_states: int = 48, pool_cap_bytes: float = 0.0) -> int:
    """States the request's pool may hold: the whole trajectory when it is
    short, else the larger of ``max_states`` and what ``pool_cap_bytes``
    allows (level-1 checkpoints plus recompute slots)."""
    cap = max(int(max_states), int(pool_cap_bytes // max(_stride(P), 1)))
    return int(min(P.nsteps + 2, max(8, cap)))


def request_bytes(P: Problem, max_states: int = 48, pool_cap_bytes: float = 0.0) -> int:
    """Device bytes of one resident request (the admission byte model): the
    state pool, the two adjoint buffers, gradient, theta, flags, the
    objective record and per-block partials, each in whole allocation
    pages, plus the gradient copied out through torch at retirement."""
    N, M = P.n_nodes, densities(P)
    pool = pool_states(P, max_states, pool_cap_bytes) * _stride(P) + ALLOC_GRANULE
    lam = 2 * _alloc(M * N * 4)
    small = (_alloc(8 * N) + _alloc(4 * N) + _alloc(N) + _alloc(16 * (P.nsteps + 1))
             + _alloc(16 * (N // 64 + 1)) + 2 * ALLOC_GRANULE)
    return int(pool + lam + small + _alloc(8 * N))


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float
    P: Problem
    theta: np.ndarray
    bytes: int = 0
    solver: Solver | None = None
    admitted: float | None = None
    done: float | None = None
    J: float | None = None
    grad: np.ndarray | None = None
    error: str | None = None


@dataclasses.dataclass
class ServeStats:
    latencies: list
    p50: float
    p99: float
    makespan: float
    node_updates: float
    mlups: float
    max_resident: int
    launches: int


def _family(P: Problem):
    return (P.lattice, P.collision, P.nscalars, P.precision)


def _percentiles(lat):
    if not lat:
        return float("nan"), float("nan")
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


class Server:
    def __init__(self, reserve_bytes: float = 4 << 30, capacity_bytes: float | None = None,
                 steps_per_tick: int = 200, work_per_tick: float = 2e7, max_states: int = 48,
                 pool_fraction: float = 0.05, stream=None,
                 mem_get_info=None, keep_gradients: bool = True, solver_factory=None,
                 primal_fn=None, adjoint_fn=None):
        # the factories exist so that the scheduling can run against a fake
        # device in host-only tests
        self.solver_factory = solver_factory or Solver
        self.primal_fn = primal_fn or batch_primal_step
        self.adjoint_fn = adjoint_fn or batch_adjoint_step
        if stream is None and solver_factory is None:
            stream = torch.cuda.Stream()
        self.stream = stream
        info = mem_get_info or torch.cuda.mem_get_info
        free, _ = info()
        # the device does not hand out every byte cudaMemGetInfo reports free:
        # keep the larger of the reserve and 8 % of it back
        self.capacity = (float(capacity_bytes) if capacity_bytes is not None
                         else free - max(float(reserve_bytes), 0.08 * free))
        self.steps_per_tick = int(steps_per_tick)       # cap of steps per request per tick
        self.work_per_tick = float(work_per_tick)       # node-steps per request per tick
        self.max_states = int(max_states)
        self.pool_cap = pool_fraction * self.capacity
        self.keep_gradients = keep_gradients
        self.committed = 0
        self.queue = deque()
        self.active = []
        self.finished = []
        self.launches = 0
        self.max_resident = 0
        self.group_streams = {}      # (family, phase) -> stream of that group

    # ---- admission ------------------------------------------------------------
    def submit(self, req: Request):
        req.bytes = request_bytes(req.P, self.max_states, self.pool_cap)
        self.queue.append(req)

    def _admit(self, now: float):
        while self.queue and self.queue[0].arrival <= now:
            req = self.queue[0]
            if req.bytes > self.capacity:
                self.queue.popleft()
                req.error = "request larger than the server's device capacity"
                req.done = now
                self.finished.append(req)
                continue
            if self.committed + req.bytes > self.capacity:
                break                       # wait for memory to free up (FIFO)
            self.queue.popleft()
            try:
                budget = pool_states(req.P, self.max_states, self.pool_cap) * _stride(req.P)
                req.solver = self.solver_factory(req.P, req.theta, stream=self.stream,
                                                 mem_budget=budget)
            except (AlbmError, RuntimeError) as e:
                req.error = str(e)
                req.done = now
                self.finished.append(req)
                continue
            self.committed += req.bytes
            req.admitted = now
            self.active.append(req)
        self.max_resident = max(self.max_resident, len(self.active))

    # ---- one tick of batched work ----------------------------------------------
    def _tick(self):
        groups = {}
        for r in self.active:
            s = r.solver
            phase = "primal" if s.time < r.P.nsteps and s.adjoint_time < 0 else "adjoint"
            groups.setdefault((_family(r.P), phase), []).append(r)
        used = []
        for (fam, phase), rs in groups.items():
            st = self._group_stream((fam, phase))
            if st is not None:
                used.append(st)
                for r in rs:
                    if hasattr(r.solver, "set_stream"):
                        r.solver.set_stream(st)
            # equal node-updates per request per tick: small requests take
            # many steps while a large one takes few, so they do not wait on it
            ks = [max(1, min(self.steps_per_tick, int(self.work_per_tick / r.P.n_nodes)))
                  for r in rs]
            fn = self.primal_fn if phase == "primal" else self.adjoint_fn
            # one call per group: the library loops over the steps, each
            # launch covering the requests that still have steps this tick
            try:
                fn([r.solver for r in rs], ks)
                self.launches += max(ks) * ((len(rs) + 63) // 64)
            except AlbmError as e:
                if e.code != OOM:
                    raise
                # a state pool could not grow: finish the tick's steps of the
                # group's requests one by one, failing those that still run
                # out of memory
                for r, k in zip(rs, ks):
                    try:
                        fn([r.solver], [k])
                        self.launches += k
                    except AlbmError as e1:
                        if e1.code != OOM:
                            raise
                        self._fail(r, "out of device memory")
        for st in used:
            st.synchronize()

    def _group_stream(self, key):
        """The stream of one (family, phase) group; None on a fake device."""
        if self.stream is None:
            return None
        if key not in self.group_streams:
            self.group_streams[key] = torch.cuda.Stream()
        return self.group_streams[key]

    def _fail(self, r: Request, msg: str):
        """Retire a resident request with an error and release its memory."""
        r.error = msg
        r.done = time.perf_counter() - self._t0
        r.solver.close()
        r.solver = None
        self.committed -= r.bytes
        self.active.remove(r)
        self.finished.append(r)

    def _retire(self, now: float):
        still = []
        for r in self.active:
            s = r.solver
            if s.adjoint_time == 0:
                r.J = s.objective()
                g = s.gradient()
                g = g.cpu().numpy() if hasattr(g, "cpu") else np.asarray(g)
                if not (np.isfinite(r.J) and np.isfinite(g).all()):
                    r.error = "non-finite objective or gradient"   # watchdog
                if self.keep_gradients:
                    r.grad = g
                r.done = time.perf_counter() - self._t0
                s.close()
                r.solver = None
                self.committed -= r.bytes
                self.finished.append(r)
            else:
                still.append(r)
        self.active = still

    def cancel(self, rid: int):
        """Drop a queued or resident request; its memory is released."""
        for r in list(self.queue):
            if r.rid == rid:
                self.queue.remove(r)
                r.error = "cancelled"
                r.done = time.perf_counter() - getattr(self, "_t0", time.perf_counter())
                self.finished.append(r)
                return True
        for r in list(self.active):
            if r.rid == rid:
                r.solver.close()
                r.solver = None
                self.committed -= r.bytes
                self.active.remove(r)
                r.error = "cancelled"
                r.done = time.perf_counter() - getattr(self, "_t0", time.perf_counter())
                self.finished.append(r)
                return True
        return False

    # ---- the serving loop ------------------------------------------------------------
    def run(self, requests, on_tick=None) -> ServeStats:
        """Serve ``requests`` (arrival-ordered) in real time until all finish."""
        for r in sorted(requests, key=lambda r: r.arrival):
            self.submit(r)
        self._t0 = time.perf_counter()
        total = len(requests)
        while len(self.finished) < total:
            now = time.perf_counter() - self._t0
            self._admit(now)
            if not self.active:
                if self.queue:
                    wait = self.queue[0].arrival - (time.perf_counter() - self._t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                continue
            self._tick()
            self._retire(time.perf_counter() - self._t0)
            if on_tick is not None:
                on_tick(self)
        return self._stats(requests)

    def _stats(self, requests) -> ServeStats:
        ok = [r for r in requests if r.error is None]
        lat = [r.done - r.arrival for r in ok]
        p50, p99 = _percentiles(lat)
        makespan = max(r.done for r in requests) if requests else 0.0
        updates = float(sum(2.0 * r.P.n_nodes * r.P.nsteps for r in ok))
        return ServeStats(lat, p50, p99, makespan, updates, updates / max(makespan, 1e-9) / 1e6,
                          self.max_resident, self.launches)


def run_sequential(requests, stream=None, keep_gradients: bool = True) -> ServeStats:
    """Baseline: each request solved alone (plain FP32 path), FIFO, in real
    time with the same arrivals."""
    stream = stream if stream is not None else torch.cuda.Stream()
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        r.admitted = time.perf_counter() - t0
        try:
            with Solver(r.P, r.theta, stream=stream) as s:
                s.run()
                r.J = s.objective()
                g = s.gradient().cpu().numpy()
                if not (np.isfinite(r.J) and np.isfinite(g).all()):
                    r.error = "non-finite objective or gradient"
                if keep_gradients:
                    r.grad = g
        except (AlbmError, RuntimeError) as e:
            r.error = str(e)
        r.done = time.perf_counter() - t0
    ok = [r for r in requests if r.error is None]
    lat = [r.done - r.arrival for r in ok]
    p50, p99 = _percentiles(lat)
    makespan = max(r.done for r in requests) if requests else 0.0
    updates = float(sum(2.0 * r.P.n_nodes * r.P.nsteps for r in ok))
    return ServeStats(lat, p50, p99, makespan, updates, updates / max(makespan, 1e-9) / 1e6,
                      1, int(sum(2 * r.P.nsteps for r in ok)))
