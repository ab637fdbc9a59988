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

Sessions keep a system's state on the device between requests: open_session copies (Phi, sigma,
V_loc) up once, a request with `session` set runs `steps` chained PT-IM steps on that resident
state in place (no host copies of the orbitals), and close_session hands the state back.  Session
state counts against the HBM budget while it is open; requests of one session run one at a time,
in order (a queue head whose session is busy waits, keeping admission FIFO).

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
    session: int | None = None      # run on the resident state of this session (phi/sigma/vloc unused)
    steps: int = 1                  # chained PT-IM steps of a session request
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_end: float = 0.0
    footprint: int = 0
    result: dict | None = None
    error: str | None = None

    @property
    def N(self) -> int:
        return int(self.phi.shape[0]) if self.phi is not None else 0

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
        self.sessions: dict[int, dict] = {}
        self._next_session = 0
        self._threads = []
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # ------------------------------------------------------------------ public
    def footprint(self, req: Request) -> int:
        depth = int(req.params.get("anderson_depth", 20))
        if req.session is not None:
            ss = self.sessions[req.session]
            return api.ptim_footprint(ss["N"], ss["cell"], ss["precision"], depth)  # state already resident
        lib = api.ptim_footprint(req.N, req.cell, req.precision, depth if req.kind == "ptim" else 1)
        io = 2 * req.phi.size * (16 if req.precision == "fp64" else 8)  # inputs and outputs on the device
        return lib + io

    def open_session(self, phi: np.ndarray, sigma: np.ndarray, vloc: np.ndarray, cell, kernel: dict,
                     precision: str = "fp32") -> int:
        """Copy a system's state to the device once; returns the session id.  The state's bytes
        count against the HBM budget until close_session."""
        dev = torch.device("cuda", self.device)
        cdt = _CDT["fp64" if precision == "fp64" else "fp32"]
        st = {"phi": torch.from_numpy(np.ascontiguousarray(phi.astype(cdt))).to(dev),
              "sigma": torch.from_numpy(np.ascontiguousarray(sigma, dtype=np.complex128)).to(dev),
              "vloc": torch.from_numpy(np.ascontiguousarray(vloc, dtype=np.float64)).to(dev),
              "cell": cell, "kernel": kernel, "precision": precision, "N": int(phi.shape[0]), "busy": False,
              "steps_done": 0}
        st["bytes"] = sum(st[k].numel() * st[k].element_size() for k in ("phi", "sigma", "vloc"))
        torch.cuda.synchronize(dev)
        with self.cv:
            if self._reserved() + st["bytes"] > self.budget:
                raise RuntimeError("session state does not fit the HBM budget")
            sid = self._next_session
            self._next_session += 1
            self.sessions[sid] = st
        return sid

    def close_session(self, sid: int) -> dict:
        """Wait for the session's requests, copy its state back to the host and release it."""
        with self.cv:
            while self.sessions[sid]["busy"] or any(r.session == sid for r, _ in self.queue):
                self.cv.wait(0.05)
            st = self.sessions.pop(sid)
            self.cv.notify_all()
        return {"phi": st["phi"].cpu().numpy(), "sigma": st["sigma"].cpu().numpy(), "steps_done": st["steps_done"]}

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
        return sum(max(w.held, w.reserved) for w in self.workers) + sum(s["bytes"] for s in self.sessions.values())

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
                    if req.session is not None:
                        self.sessions[req.session]["busy"] = True
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
        if req.session is not None and self.sessions[req.session]["busy"]:
            return None, None  # the session's previous request is still running: keep FIFO order
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
            if req.session is not None:
                self.sessions[req.session]["busy"] = False
            self.completed.append(req)
            self.cv.notify_all()
        fut.set_result(req)

    def _execute(self, w: _Worker, req: Request) -> dict:
        dev = torch.device("cuda", self.device)
        if req.session is not None:
            ss = self.sessions[req.session]
            p = dict(dt=0.5, alpha=0.25, ecut=10.0, tol=1e-6, max_outer=20, max_inner=100, anderson_depth=20)
            p.update(req.params)
            stats = []
            for _ in range(max(1, req.steps)):
                stats.append(w.ctx.ptim_step(ss["phi"], ss["sigma"], ss["vloc"], cell=ss["cell"], kernel=ss["kernel"],
                                             precision=ss["precision"], stream=w.stream, allow_unconverged=True, **p))
            w.stream.synchronize()
            ss["steps_done"] += len(stats)
            return {"stats": stats}
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
