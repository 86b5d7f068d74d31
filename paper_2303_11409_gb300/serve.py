"""Continuous-batching request loop for independent TEBD simulations on one GPU.

Requests (chain length, model, chi, step count, arrival time) come in over time.
Each admitted request keeps its MPS on the device.  Every tick merges the next
Trotter layer of every active request into one executor call, so updates of
different requests share launches (independent two-site updates processed in
parallel, arXiv:2303.11409 Sec. II).  Admission is by device-memory footprint
(the arena the request's handle will hold plus its per-layer workspace bound,
both computed from the per-bond sector-size bounds) against a budget, and by a
slot count; a request admitted mid-run joins the next tick.  Completed requests
report observables and free their memory at once, which admits waiting ones.

With lanes = 2 the active requests are dealt to two executors, each with its own
CUDA stream and workspace, and every tick runs both executor calls at once from two
host threads (the library releases the interpreter lock): one lane's host planning
and kept-count round trip overlap the other lane's kernels, and the two lanes'
kernels overlap each other.  A request stays on the lane that admitted it.
"""
from __future__ import annotations

import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import models
from ._binding import MPS, MPS_FP64, Executor, footprint_bytes
from .tebd import GateTable, strang_layers


@dataclass
class Request:
    id: int
    model: str            # "xxz" or "bh"
    L: int
    chi: int
    steps: int
    param: float          # Delta (xxz) or U (bh, J = 1)
    arrival: float = 0.0  # seconds after the start of the run
    dt: float | None = None
    cutoff: float = 1e-10
    n_max: int = 4


@dataclass
class Job:
    req: Request
    psi: MPS
    gates: GateTable
    layers: list
    bytes: int
    admitted: float
    lane: int = 0
    next_layer: int = 0
    updates: int = 0
    trunc: float = 0.0


@dataclass
class Result:
    id: int
    arrival: float
    admitted: float
    finished: float
    updates: int
    observables: np.ndarray
    trunc_err_sum: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def _setup(req: Request):
    if req.model == "xxz":
        d = 2
        occ = [1 if s % 2 == 0 else 0 for s in range(req.L)]
        dt = req.dt if req.dt is not None else 0.05
        gates = GateTable("xxz", req.L, d, dt, delta=req.param)
    elif req.model == "bh":
        d = req.n_max + 1
        occ = [1] * req.L
        dt = req.dt if req.dt is not None else 0.02
        gates = GateTable("bh", req.L, d, dt, J=1.0, U=req.param)
    else:
        raise ValueError(req.model)
    return d, occ, gates


def footprint(req: Request) -> int:
    d, occ, _ = _setup(req)
    arena, layer_ws = footprint_bytes(req.L, d, sum(occ), req.chi)
    return arena + layer_ws


def check_admissible(requests: list[Request], budget_bytes: int) -> None:
    """Refuse up front any request that could never fit in the budget, even alone."""
    for r in requests:
        if footprint(r) > budget_bytes:
            raise ValueError(f"request {r.id} needs {footprint(r)} bytes, over the {budget_bytes}-byte budget")


@dataclass
class Server:
    budget_bytes: int
    max_slots: int = 64
    stream: object = None
    clock: object = time.perf_counter
    precision: int = MPS_FP64      # sector-GEMM precision of every admitted request's MPS
    graphs: bool = False           # capture the merged update calls in CUDA graphs
    lanes: int = 1                 # executors run concurrently, each on its own stream
    executor: Executor = field(init=False)

    def __post_init__(self):
        if self.lanes not in (1, 2):
            raise ValueError("lanes must be 1 or 2")
        streams = [self.stream]
        if self.lanes == 2:
            import torch
            self._lane_stream = torch.cuda.Stream()     # kept alive with the server
            streams.append(self._lane_stream.cuda_stream)
        self.executors = []
        for st in streams:
            ex = Executor(st)
            ex.set_graphs(self.graphs)
            self.executors.append(ex)
        self.executor = self.executors[0]
        self._pool = ThreadPoolExecutor(max_workers=self.lanes) if self.lanes > 1 else None
        self.max_active_seen = 0
        self.max_bytes_seen = 0

    def run(self, requests: list[Request], deadline: float | None = None) -> list[Result]:
        """Serve every request to completion; arrivals follow req.arrival on the wall clock.
        With a deadline (seconds) the run stops at the first tick boundary after it: requests
        not finished by then are dropped (their handles freed) and counted in self.unfinished,
        their updates so far in self.unfinished_updates."""
        pending = sorted(requests, key=lambda r: (r.arrival, r.id))
        check_admissible(pending, self.budget_bytes)
        active: list[Job] = []
        done: list[Result] = []
        used = 0
        self.unfinished = 0
        self.unfinished_updates = 0
        t0 = self.clock()
        while pending or active:
            now = self.clock() - t0
            if deadline is not None and now >= deadline:
                self.unfinished = len(active) + len(pending)
                self.unfinished_updates = sum(j.updates for j in active)
                for job in active:
                    job.psi.close()
                break
            # admit arrived requests, in arrival order, while slots and memory allow
            while pending and pending[0].arrival <= now and len(active) < self.max_slots:
                need = footprint(pending[0])
                if used + need > self.budget_bytes:
                    break
                req = pending.pop(0)
                d, occ, gates = _setup(req)
                # the lane with the least work per tick (sum of L chi^2 of its requests)
                load = [sum(j.req.L * j.req.chi ** 2 for j in active if j.lane == k) for k in range(self.lanes)]
                lane = int(min(range(self.lanes), key=lambda k: load[k]))
                psi = MPS(d, occ, req.chi, precision=self.precision, stream=self.executors[lane].stream)
                layers = [lay for _ in range(req.steps) for lay in strang_layers(req.L)]
                active.append(Job(req, psi, gates, layers, need, now, lane))
                used += need
            self.max_active_seen = max(self.max_active_seen, len(active))
            self.max_bytes_seen = max(self.max_bytes_seen, used)
            if not active:
                if pending:                       # idle until the next arrival
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            # one tick: the next layer of every active request, merged into one call per lane
            items = [[] for _ in range(self.lanes)]
            owners = [[] for _ in range(self.lanes)]
            for job in active:
                sites, f = job.layers[job.next_layer]
                for s in sites:
                    items[job.lane].append((job.psi, s, job.gates(s, f), job.req.chi, job.req.cutoff))
                    owners[job.lane].append(job)
            if self._pool is None:
                outs = [self.executor.apply(items[0])]
            else:
                futs = [self._pool.submit(self.executors[k].apply, items[k]) for k in range(self.lanes)]
                outs = [f.result() for f in futs]
            for k in range(self.lanes):
                for job, e in zip(owners[k], outs[k][0]):
                    job.updates += 1
                    job.trunc += float(e)
            finished = []
            for job in active:
                job.next_layer += 1
                if job.next_layer == len(job.layers):
                    finished.append(job)
            for job in finished:
                d = job.psi.d
                op = np.arange(d, dtype=np.float64)
                obs = np.array([job.psi.expect(s, op) for s in range(job.req.L)])
                t = self.clock() - t0
                done.append(Result(job.req.id, job.req.arrival, job.admitted, t, job.updates, obs, job.trunc))
                job.psi.close()
                used -= job.bytes
                active.remove(job)
        return sorted(done, key=lambda r: r.id)

    def close(self):
        for ex in self.executors:
            ex.close()
        if self._pool is not None:
            self._pool.shutdown()


def summarize(results: list[Result], wall: float) -> dict:
    lat = np.array([r.latency for r in results])
    ups = sum(r.updates for r in results)
    return {"requests": len(results), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "updates": ups,
            "updates_per_s": ups / wall if wall > 0 else float("nan")}
