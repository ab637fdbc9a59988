"""Continuous-batching request loop for PT-IM steps and exchange applications on one GPU.

Requests (a PT-IM step or a V_x application of one system: its orbitals, occupations, grid and
parameters) arrive at any time.  The server keeps `slots` workers, each with its own library
context (workspace, tables) and CUDA stream, so admitted requests run concurrently on the device.
A request is admitted as soon as a worker is free and the HBM it may need fits the budget:
  reserved = sum over workers of max(workspace the worker already holds, footprint of its request)
with footprints from `pt_ptim_footprint` (an upper bound of what a step allocates).  Admission is
FIFO; a request that does not fit blocks the ones behind it until memory frees up, so large
systems are not starved.  Inputs are copied to the device when the request starts, the state stays
resident on the device while it runs, results are copied back when it ends, and every request
records its arrival, start and end times for p50/p99 latency.

All computation runs in libptim.so through `api.Context`; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import threading
import time
from collections import deque
from concurrent.futures import Future

import numpy as np
import torch

from . import api

_CDT = {"fp64": np.complex128, "fp32": np.complex64}


@dataclasses.dataclass
class Request:
    phi: np.ndarray                 # (N, nz, ny, nx) complex, host
    sigma: np.ndarray | None        # (N, N) complex128 (PT-IM step) or None
    occ: np.ndarray | None          # occupations (exchange request)
    vloc: np.ndarray | None         # (nz, ny, nx) float64 (PT-IM step)
    cell: object
    kernel: dict
    kind: str = "ptim"              # "ptim" or "exchange"
    precision: str = "fp32"
    params: dict = dataclasses.field(default_factory=dict)
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_end: float = 0.0
    footprint: int = 0
    result: dict | None = None
    error: str | None = None

    @property
    def N(self) -> int:
        return int(self.phi.shape[0])

    @property
    def latency(self) -> float:
        return self.t_end - self.t_arrival


class _Worker:
    def __init__(self, device: int):
        self.ctx = api.Context(device)
        self.stream = torch.cuda.Stream(device=device)
        self.busy = False
        self.held = 0          # workspace bytes this worker's context holds
        self.reserved = 0      # bytes reserved for the running request


class Server:
    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("the serving loop needs a CUDA GPU")
        self.device = device
        torch.cuda.set_device(device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            hbm_budget = int(0.85 * free)
        self.budget = int(hbm_budget)
        self.workers = [_Worker(device) for _ in range(slots)]
        self.queue: deque = deque()
        self.cv = threading.Condition()
        self.running = True
        self.completed: list[Request] = []
        self.rejected: list[Request] = []
        self._threads = []
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # ------------------------------------------------------------------ public
    def footprint(self, req: Request) -> int:
        depth = int(req.params.get("anderson_depth", 20))
        lib = api.ptim_footprint(req.N, req.cell, req.precision, depth if req.kind == "ptim" else 1)
        io = 2 * req.phi.size * (16 if req.precision == "fp64" else 8)  # inputs and outputs on the device
        return lib + io

    def submit(self, req: Request) -> Future:
        req.t_arrival = time.perf_counter() if req.t_arrival == 0.0 else req.t_arrival
        req.footprint = self.footprint(req)
        fut: Future = Future()
        with self.cv:
            if req.footprint > self.budget:
                req.error = "larger than the HBM budget"
                self.rejected.append(req)
                fut.set_result(req)
                return fut
            self.queue.append((req, fut))
            self.cv.notify_all()
        return fut

    def backlog(self) -> int:
        with self.cv:
            return len(self.queue)

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        self._sched.join()
        for t in self._threads:
            t.join()
        for w in self.workers:
            w.ctx.close()

    # ------------------------------------------------------------------ scheduling
    def _reserved(self) -> int:
        return sum(max(w.held, w.reserved) for w in self.workers)

    def _schedule(self):
        while True:
            trim = None
            with self.cv:
                while self.running:
                    w, trim = self._pick()
                    if w is not None or trim is not None:
                        break
                    self.cv.wait(0.05)
                if not self.running:
                    return
                if w is not None:
                    req, fut = self.queue.popleft()
                    w.busy = True
                    w.reserved = req.footprint
                else:
                    trim.busy = True  # keep it out of the pool while its workspace is released
            if trim is not None:
                trim.ctx.trim()  # synchronises the device; done outside the lock
                with self.cv:
                    trim.held = trim.ctx.workspace_bytes()
                    trim.busy = False
                    self.cv.notify_all()
                continue
            t = threading.Thread(target=self._run, args=(w, req, fut), daemon=True)
            self._threads = [x for x in self._threads if x.is_alive()] + [t]
            t.start()

    def _pick(self):
        """(worker, None) to admit the queue head, (None, idle worker to trim) when only cached
        workspace of idle workers stands in the way, else (None, None)."""
        if not self.queue:
            return None, None
        free = [w for w in self.workers if not w.busy]
        if not free:
            return None, None
        req = self.queue[0][0]
        w = max(free, key=lambda x: x.held)  # reuse the largest cached workspace
        if self._reserved() - max(w.held, w.reserved) + max(w.held, req.footprint) <= self.budget:
            return w, None
        others = [x for x in free if x is not w and x.held > 0]
        if others:
            return None, max(others, key=lambda x: x.held)
        return None, None

    def _run(self, w: _Worker, req: Request, fut: Future):
        req.t_start = time.perf_counter()
        try:
            with torch.cuda.stream(w.stream):
                req.result = self._execute(w, req)
        except Exception as e:  # noqa: BLE001
            req.error = str(e)
        req.t_end = time.perf_counter()
        with self.cv:
            w.held = w.ctx.workspace_bytes()
            w.reserved = 0
            w.busy = False
            self.completed.append(req)
            self.cv.notify_all()
        fut.set_result(req)

    def _execute(self, w: _Worker, req: Request) -> dict:
        dev = torch.device("cuda", self.device)
        cdt = _CDT["fp64" if req.precision == "fp64" else "fp32"]
        s = w.stream
        phi = torch.from_numpy(np.ascontiguousarray(req.phi.astype(cdt))).to(dev, non_blocking=True)
        if req.kind == "exchange":
            occ = torch.from_numpy(np.ascontiguousarray(req.occ, dtype=np.float64)).to(dev, non_blocking=True)
            out = w.ctx.apply_exchange(phi, occ, cell=req.cell, kernel=req.kernel, precision=req.precision,
                                       stream=s)
            res = out.to("cpu", non_blocking=True)
            s.synchronize()
            return {"vx": res.numpy()}
        sigma = torch.from_numpy(np.ascontiguousarray(req.sigma, dtype=np.complex128)).to(dev, non_blocking=True)
        vloc = torch.from_numpy(np.ascontiguousarray(req.vloc, dtype=np.float64)).to(dev, non_blocking=True)
        p = dict(dt=0.5, alpha=0.25, ecut=10.0, tol=1e-6, max_outer=20, max_inner=100, anderson_depth=20)
        p.update(req.params)
        stats = w.ctx.ptim_step(phi, sigma, vloc, cell=req.cell, kernel=req.kernel, precision=req.precision,
                                stream=s, allow_unconverged=True, **p)
        phi_h = phi.to("cpu", non_blocking=True)
        sig_h = sigma.to("cpu", non_blocking=True)
        s.synchronize()
        return {"phi": phi_h.numpy(), "sigma": sig_h.numpy(), "stats": stats}


def latency_summary(reqs) -> dict:
    lat = np.array([r.latency for r in reqs if r.error is None and r.t_end > 0])
    if lat.size == 0:
        return {"count": 0}
    return {"count": int(lat.size), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}
