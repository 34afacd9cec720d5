"""Continuous-batching solve server over the C ABI.

Requests (one electrode image plus potential, velocity and step counts each)
arrive at any time.  A request is admitted as soon as a slot is free and its
device footprint fits into the remaining memory budget (first fit in arrival
order, with an ageing bound so that large requests are not passed over for
ever); admitted requests run concurrently, each on its own domain with its
own CUDA stream, so their kernels overlap on the device while earlier ones
are still running.  Larger requests get higher stream priorities (the
device's block scheduler then serves their launches first), so the long
solves that set the latency tail are slowed little by the short ones that
fill the gaps.  Fields
stay resident in device memory for the whole solve; the domain (and its
memory) is released when the request completes, which admits the next.

Each request's result depends only on its own inputs: every kernel is
deterministic and domains share no device state, so a request gives the same
result alone and in the mix.

``Server`` is host-side orchestration only; all numerical work runs in the
library's kernels.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import cdi


@dataclass
class Request:
    mask: np.ndarray
    applied_V: float
    U_mps: float
    np_steps: int
    precision: int = cdi.FP32
    flow_tol: float = 1e-8
    max_flow_steps: int = 1_000_000
    c0: float = 10.0
    Ka: float = 1e-6
    z: tuple = (1, -1)
    D: tuple = (1.33e-9, 2.03e-9)
    tag: object = None
    # filled in by the server
    priority: int = 0  # CUDA stream priority of the request (lower: served first)
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    result: dict = field(default_factory=dict)
    error: str = ""


def footprint_bytes(mask: np.ndarray, precision: int, mirror: bool = True) -> int:
    """Peak device memory a domain for this mask allocates (the allocations of
    cdi_create_domain, including its create-time work arrays), with one
    transport state."""
    dim = mask.ndim
    N = int(mask.size)
    n_pore = int((mask == 0).sum())
    n_fp = n_pore * (2 if mirror else 1)
    Nf = N * (2 if mirror else 1)
    Q = 9 if dim == 2 else 19
    T = 8 if precision == cdi.FP64 else 4
    Tpop = {cdi.FP64: 8, cdi.FP32: 4, cdi.FP32_SPLIT: 8, cdi.BF16_POP: 2,
            cdi.FP32_CPAIR: 4}[precision]
    Tc = T + (4 if precision in (cdi.FP32_SPLIT, cdi.FP32_CPAIR) else 0)  # + low words
    nx = mask.shape[-1]
    rows = N // nx
    # overflow slots: x-edge sites, plus an allowance for the sites whose
    # row-base bytes overflow (under one in a thousand sites on the grain packs)
    n_ovf = 2 * rows + n_fp // 256
    n_off = 2 if dim == 2 else 8                      # lateral row offsets
    links = (4 + (4 if dim == 2 else 8)) * n_fp + n_off * 4 * ((n_fp + 31) // 32)
    flow = (Q * Tpop * n_fp + links + (Q - 1) * 4 * n_ovf
            + Nf * (2 if dim == 2 else 4) + dim * Nf * 8)
    transport = (n_pore * (4 + 8 + 2 + 2 * (dim - 1) * 4 + dim * T + 8 + 2 * 4 * Tc)
                 + rows * ((nx + 31) // 32) * 8)
    lattice = N * (1 + 2 + 8 + 4 * 8)                 # mask, face flags, psi, CG vectors
    work = Nf * 4 + 2 * ((Nf + 2047) // 2048) * 4     # create-time rank and list work
    return flow + transport + lattice + work + (4 << 20)


def size_priority(need: int) -> int:
    """Stream priority for a request of `need` device bytes: 0 below 256 MiB,
    then one level higher per doubling (the device clamps to its range)."""
    levels = 0
    while need >= (256 << 20) << levels and levels < 5:
        levels += 1
    return -levels


class Server:
    """Admits requests while slots and memory allow; runs them concurrently.

    Admission is first-fit in arrival order: the oldest waiting request that
    fits the free slots and memory is started, so small requests need not
    queue behind a large one that does not fit yet.  To keep a large request
    from waiting for ever, a waiting request that has been passed over
    ``max_bypass`` times is served next: nothing younger is admitted until it
    fits."""

    def __init__(self, slots: int = 4, memory_budget: int = 16 << 30, device: int = 0,
                 solver=None, max_bypass: int | None = None, prioritise_large: bool = True):
        self.solver = solver or solve
        self.prioritise_large = prioritise_large
        self.slots = slots
        self.budget = memory_budget
        self.device = device
        self.max_bypass = 2 * slots if max_bypass is None else max_bypass
        self._waiting: list = []
        self._closing = False
        self.done: list = []
        self._lock = threading.Condition()
        self._in_use = 0
        self._running = 0
        self.max_running = 0
        self.max_in_use = 0
        self._admitter = threading.Thread(target=self._admit_loop, daemon=True)
        self._admitter.start()

    def submit(self, req: Request) -> None:
        req.t_arrival = time.perf_counter()
        need = footprint_bytes(req.mask, req.precision)
        with self._lock:
            self._waiting.append((req, need, [0]))
            self._lock.notify_all()

    def _pick(self):
        """Index of the request to start now, or None (lock held)."""
        if self._running >= self.slots:
            return None
        for i, (req, need, passed) in enumerate(self._waiting):
            if self._in_use + need <= self.budget:
                return i
            if passed[0] >= self.max_bypass:
                return None        # this one is due: hold the others back
        return None

    def _admit_loop(self):
        while True:
            with self._lock:
                # requests larger than the whole budget fail at once
                for item in [w for w in self._waiting if w[1] > self.budget]:
                    req, need, _ = item
                    req.error = f"request needs {need} bytes, budget {self.budget}"
                    req.t_done = time.perf_counter()
                    self.done.append(req)
                    self._waiting.remove(item)
                    self._lock.notify_all()
                i = self._pick()
                if i is None:
                    if self._closing and not self._waiting:
                        return
                    self._lock.wait(timeout=0.5)
                    continue
                req, need, _ = self._waiting.pop(i)
                req.priority = size_priority(need) if self.prioritise_large else 0
                for _, _, passed in self._waiting[:i]:
                    passed[0] += 1
                self._running += 1
                self._in_use += need
                self.max_running = max(self.max_running, self._running)
                self.max_in_use = max(self.max_in_use, self._in_use)
            threading.Thread(target=self._run, args=(req, need), daemon=True).start()

    def _run(self, req: Request, need: int):
        req.t_start = time.perf_counter()
        try:
            # a new host thread starts on device 0: bind it to the server's
            # device before the request's domain is created there
            import torch
            if torch.cuda.is_available():
                torch.cuda.set_device(self.device)
            req.result = self.solver(req)
        except Exception as e:  # a failed request fails alone
            req.error = str(e)
        req.t_done = time.perf_counter()
        with self._lock:
            self._running -= 1
            self._in_use -= need
            self.done.append(req)
            self._lock.notify_all()

    def drain(self, n_expected: int, timeout: float = 3600.0) -> list:
        """Wait until n_expected requests have completed; returns them."""
        t_end = time.perf_counter() + timeout
        with self._lock:
            while len(self.done) < n_expected:
                left = t_end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError("requests still running")
                self._lock.wait(timeout=left)
            return list(self.done)

    def close(self):
        with self._lock:
            self._closing = True
            self._lock.notify_all()
        self._admitter.join(timeout=10)


def solve(req: Request) -> dict:
    """One request end to end through the C ABI (the plain single solve), on
    a stream of the request's priority."""
    stream = None
    if req.priority:
        import torch
        stream = torch.cuda.Stream(priority=req.priority)
    with cdi.Domain(req.mask, precision=req.precision,
                    stream=stream.cuda_stream if stream is not None else None) as d:
        steps, res, st = d.solve_flow(tol=req.flow_tol, max_steps=req.max_flow_steps,
                                      U_target=req.U_mps, allow_not_converged=True)
        d.set_potential(req.applied_V, c_bulk=req.c0, tol=1e-12)
        d.init_transport(req.z, req.D, c0=req.c0, Ka=req.Ka)
        d.step(req.np_steps)
        return {"Gamma": d.adsorbed(), "C_out": d.outlet(), "flow_steps": steps,
                "flow_residual": res}


def run_sequential(requests: list, arrivals: list) -> list:
    """The plain loop: requests served one at a time in arrival order."""
    t0 = time.perf_counter()
    for req, ta in zip(requests, arrivals):
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        req.t_arrival = t0 + ta
        req.t_start = time.perf_counter()
        try:
            req.result = solve(req)
        except Exception as e:
            req.error = str(e)
        req.t_done = time.perf_counter()
    return requests


def run_served(requests: list, arrivals: list, slots: int, memory_budget: int) -> list:
    """The same stream of requests through the continuous-batching server."""
    srv = Server(slots=slots, memory_budget=memory_budget)
    t0 = time.perf_counter()
    for req, ta in zip(requests, arrivals):
        now = time.perf_counter() - t0
        if now < ta:
            time.sleep(ta - now)
        srv.submit(req)
    done = srv.drain(len(requests))
    srv.close()
    return done


def latency_stats(reqs: list) -> dict:
    lat = np.array([r.t_done - r.t_arrival for r in reqs if not r.error])
    span = max(r.t_done for r in reqs) - min(r.t_arrival for r in reqs)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(lat) / span, "failed": sum(1 for r in reqs if r.error)}
