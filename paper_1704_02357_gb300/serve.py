"""Continuous-batching server for multipole requests of mixed mesh sizes and l_max.

Requests (a data catalog, a mesh side, l_max, k edges) arrive over time. The server keeps
device-resident estimator contexts (meshes, spectra, cached randoms meshes) keyed by
(nmesh, l_max), admits a request as soon as a context of its shape is idle or a new one fits
the HBM budget (its workspace is the footprint), and enqueues the request's whole launch
sequence on that context's own CUDA stream. Requests that arrive while others are on the GPU
are admitted as slots and memory free up, and their kernels overlap on the device. Finished
requests release their context (kept warm for the next request of that shape; evicted least
recently used when a new shape needs the memory). Shapes known in advance can be built before
the stream starts (prewarm), so that no request waits behind a context's creation.

A context holds the Y_lm tables (k-space and real-space, FP64-built) when its footprint with them
is at most `table_fraction` of the budget; larger shapes are served without them (Y_lm evaluated
in FP32 per mode and per node), which keeps them admissible at the cost of the tables' accuracy.

All arithmetic runs in libpspec (pspec_run_batch on one mock, replaying the context's
captured graph); this module only schedules.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from .pspec import Estimator


@dataclass
class Request:
    rid: int
    nmesh: int
    ell_max: int
    pos: object                      # device tensor (n, 3)
    k_edges: np.ndarray
    t_arrival: float = 0.0           # seconds, server clock
    t_admit: float = math.nan
    t_done: float = math.nan
    P: Optional[np.ndarray] = None   # (n_ells, nk) when done
    sums: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival

    @property
    def queue_wait(self) -> float:
        return self.t_admit - self.t_arrival


@dataclass
class _Slot:
    est: Estimator
    key: tuple
    footprint: int
    busy: Optional[Request] = None
    out: Optional[dict] = None
    event: object = None
    last_used: float = 0.0


class Server:
    def __init__(self, box_size: float, box_corner, randoms_for: Callable[[int], object], hbm_budget: int,
                 observer=(0.0, 0.0, 0.0), window="cic", interlaced=True, compensate=True, P0=0.0, nbar=0.0,
                 max_kbins=512, max_particles=0, max_group_bytes_for: Optional[Callable[[int, int], int]] = None,
                 max_slots_per_shape: int = 2, table_fraction: float = 0.5, device=None, clock=time.perf_counter):
        self.kw = dict(box_size=box_size, box_corner=box_corner, observer=observer, window=window,
                       interlaced=interlaced, compensate=compensate, P0=P0, nbar=nbar, max_kbins=max_kbins,
                       precision="fp32")
        self.randoms_for = randoms_for
        self.budget = int(hbm_budget)
        self.max_particles = int(max_particles)
        self.max_group_bytes_for = max_group_bytes_for or (lambda n, l: 0)
        self.max_slots_per_shape = max_slots_per_shape
        self.table_fraction = float(table_fraction)
        self._tables: Dict[tuple, bool] = {}
        self.headroom = 1 << 30  # device bytes left free beside a new workspace
        self.device = device
        self.clock = clock
        self.slots: List[_Slot] = []
        self.queue: collections.deque = collections.deque()
        self.done: List[Request] = []
        self.t0 = clock()

    # ------------------------------------------------------------------ memory
    def used(self) -> int:
        return sum(s.footprint for s in self.slots)

    def tables_for(self, nmesh: int, ell_max: int) -> bool:
        """Whether contexts of this shape hold the Y_lm tables (see the module docstring)."""
        key = (nmesh, ell_max)
        if key not in self._tables:
            self._tables[key] = self._footprint(nmesh, ell_max, True) <= self.table_fraction * self.budget
        return self._tables[key]

    def _footprint(self, nmesh: int, ell_max: int, tables: Optional[bool] = None) -> int:
        from . import pspec as P
        import ctypes as C
        import torch
        if tables is None:
            tables = self.tables_for(nmesh, ell_max)
        lib = P.load()
        comp = P.compensation_code(self.kw["compensate"])
        p = P.Params(nmesh, P.WINDOWS[self.kw["window"]], int(self.kw["interlaced"]), comp,
                     P.PRECISIONS[self.kw["precision"]], ell_max, float(self.kw["box_size"]),
                     (C.c_double * 3)(*self.kw["box_corner"]), (C.c_double * 3)(*self.kw["observer"]),
                     float(self.kw["P0"]), float(self.kw["nbar"]), int(self.max_group_bytes_for(nmesh, ell_max)),
                     self.max_particles, 1, 0 if tables else -1, 0)
        n = C.c_int64(0)
        with torch.cuda.device(self.device or torch.cuda.current_device()):
            P._check(lib.pspec_workspace_size(C.byref(p), int(self.kw["max_kbins"]), C.byref(n)))
        return int(n.value) + 256

    def _free_device_bytes(self) -> int:
        import torch
        free, _ = torch.cuda.mem_get_info(self.device)
        return int(free)

    def _new_slot(self, key) -> Optional[_Slot]:
        import torch
        nmesh, ell_max = key
        need = self._footprint(nmesh, ell_max)
        if need > self.budget:
            raise ValueError(f"a ({nmesh}^3, l_max {ell_max}) context needs {need} bytes, over the HBM budget")
        # the budget bounds what this server holds; the device must also have the room now
        while self.used() + need > self.budget or need + self.headroom > self._free_device_bytes():
            idle = [s for s in self.slots if s.busy is None]
            if not idle:
                if not any(s.busy is not None for s in self.slots):
                    raise MemoryError(f"a ({nmesh}^3, l_max {ell_max}) context needs {need} bytes; "
                                      f"the device has {self._free_device_bytes()} free and nothing to evict")
                return None  # wait for a running request to finish
            victim = min(idle, key=lambda s: s.last_used)
            victim.est.close()
            self.slots.remove(victim)
            torch.cuda.empty_cache()
        stream = torch.cuda.Stream(device=self.device)
        est = Estimator(nmesh=nmesh, ell_max=ell_max, cache_randoms=True, max_particles=self.max_particles,
                        max_group_bytes=self.max_group_bytes_for(nmesh, ell_max), device=self.device, stream=stream,
                        ylm_table=self.tables_for(nmesh, ell_max), **self.kw)
        est.set_randoms(self.randoms_for(nmesh))
        slot = _Slot(est=est, key=key, footprint=need)
        self.slots.append(slot)
        return slot

    def prewarm(self, shapes: Sequence[tuple], edges_for: Callable[[int], np.ndarray], pos_for: Callable[[int], object],
                slots_per_shape: Optional[int] = None) -> None:
        """Build contexts (tables, cached randoms meshes) and capture their graphs for the given
        (nmesh, l_max) shapes before the stream starts, up to `slots_per_shape` each (default
        the per-shape cap), while the budget allows without evicting one another."""
        import torch
        n = self.max_slots_per_shape if slots_per_shape is None else slots_per_shape
        for key in shapes:
            for _ in range(n):
                if sum(1 for s in self.slots if s.key == key) >= self.max_slots_per_shape:
                    break
                if self.used() + self._footprint(*key) > self.budget:
                    break
                slot = self._new_slot(tuple(key))
                if slot is None:
                    break
                ells = list(range(0, key[1] + 1, 2))
                slot.est.run_batch([pos_for(key[0])], ells, edges_for(key[0]), use_graph=True)
                torch.cuda.synchronize()
                slot.last_used = self.now()

    # ------------------------------------------------------------------ scheduling
    def submit(self, req: Request) -> None:
        if math.isnan(req.t_arrival) or req.t_arrival == 0.0:
            req.t_arrival = self.now()
        self.queue.append(req)

    def now(self) -> float:
        return self.clock() - self.t0

    def _poll(self) -> int:
        finished = 0
        for s in self.slots:
            r = s.busy
            if r is None or not s.event.query():
                continue
            r.t_done = self.now()
            r.P = s.out["P"][0].cpu().numpy()
            r.sums = s.out["sums"][0].cpu().numpy()
            s.busy = None
            s.out = None
            s.last_used = r.t_done
            self.done.append(r)
            finished += 1
        return finished

    def _admit(self) -> int:
        import torch
        admitted = 0
        waiting = collections.deque()
        while self.queue:
            r = self.queue.popleft()
            key = (r.nmesh, r.ell_max)
            slot = next((s for s in self.slots if s.key == key and s.busy is None), None)
            if slot is None and sum(1 for s in self.slots if s.key == key) < self.max_slots_per_shape:
                slot = self._new_slot(key)
            if slot is None:
                waiting.append(r)
                continue
            r.t_admit = self.now()
            ells = list(range(0, r.ell_max + 1, 2))
            slot.busy = r
            slot.out = slot.est.run_batch([r.pos], ells, r.k_edges, use_graph=True)
            ev = torch.cuda.Event()
            ev.record(slot.est.stream)
            slot.event = ev
            admitted += 1
        self.queue = waiting
        return admitted

    def step(self) -> None:
        self._poll()
        self._admit()

    def busy(self) -> bool:
        return bool(self.queue) or any(s.busy is not None for s in self.slots)

    def run(self, requests: Sequence[Request], arrivals: Sequence[float]) -> List[Request]:
        """Replay arrivals (seconds from start) in real time; returns the finished requests."""
        order = np.argsort(arrivals)
        pending = collections.deque((arrivals[i], requests[i]) for i in order)
        self.t0 = self.clock()
        while pending or self.busy():
            t = self.now()
            while pending and pending[0][0] <= t:
                ta, r = pending.popleft()
                r.t_arrival = ta
                self.queue.append(r)
            self.step()
        return self.done

    def close(self) -> None:
        import torch
        for s in self.slots:
            s.est.close()
        self.slots.clear()
        torch.cuda.empty_cache()


def latency_summary(done: Sequence[Request], wall: float) -> Dict[str, float]:
    lat = np.array([r.latency for r in done])
    wait = np.array([r.queue_wait for r in done])
    return {"requests": len(done), "throughput_per_s": len(done) / wall if wall > 0 else float("nan"),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_queue_wait_ms": float(wait.mean() * 1e3), "p99_queue_wait_ms": float(np.percentile(wait, 99) * 1e3)}
