"""Serving loop: continuous batching of AT solves on one GPU.

Requests (problem type, size, step count, seed) arrive over time.  The
server admits a request as soon as it has arrived, a slot is free and its
state + workspace fit in the device-memory budget; admitted work stays
resident on the device until it finishes.  Every tick advances all
admitted requests by a chunk of steps, all of them slots of one batch in
the flat mode (one launch per stage over the windows of every request, so a
large request spreads over all SMs while small ones ride along), replayed
from a captured graph.  Optionally (``big_points``) requests above a size
get their own context on a second stream instead.  Finished requests are
retired at once and their memory and slot go to the next arrivals.

:func:`serve_plain` is the comparison: the same stream solved one request at
a time through a context each (plain per-request launches).
"""
from __future__ import annotations

import collections
import time

import numpy as np

from . import api
from . import workloads as W
from .batch import Batch


class Request:
    __slots__ = ("id", "arrival", "kind", "n", "steps", "seed", "pb", "init", "admit", "finish", "state", "bytes",
                 "slot", "ctx", "left")

    def __init__(self, d: dict):
        self.id, self.arrival, self.kind = d["id"], d["arrival"], d["kind"]
        self.n, self.steps, self.seed = d["n"], d["steps"], d["seed"]
        self.pb, self.init = W.serving_request(self.kind, self.n, self.seed, instance=self.id)
        self.n = self.pb["n"]
        self.admit = self.finish = None
        self.state = None
        self.slot = None
        self.ctx = None
        self.left = self.steps
        nvar = api.NVAR[self.pb["pde"]]
        self.bytes = 8 * nvar * self.n + api.workspace_bytes(self.pb)


class Server:
    def __init__(self, mem_budget=16 << 30, capacity=1024, chunk=50, big_points=None, device=0, keep_states=False,
                 max_windows=1 << 22, mode=1):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.budget = int(mem_budget)
        self.chunk = int(chunk)
        self.big = int(big_points) if big_points is not None else (1 << 62)
        self.keep = keep_states
        self.main = torch.cuda.current_stream(self.device)
        self.side = torch.cuda.Stream(self.device)
        self.batch = Batch(capacity, device=device, stream=self.main, max_windows=max_windows)
        self.batch.set_config(mode, 256, 3, True)
        self.free_slots = collections.deque(range(capacity))
        self.used = 0
        self.active = []
        self.done = []
        self.ticks = 0

    # -- admission ---------------------------------------------------------
    def _fits(self, r: Request) -> bool:
        if r.n > self.big:
            return self.used + r.bytes <= self.budget
        return bool(self.free_slots) and self.used + r.bytes <= self.budget

    def _admit(self, r: Request, now: float):
        r.admit = now
        self.used += r.bytes
        if r.n > self.big:
            with self.torch.cuda.stream(self.side):
                r.ctx = api.Solver(r.pb, r.init, device=self.device.index, stream=self.side, path="stage")
        else:
            r.slot = self.free_slots.popleft()
            r.state = self.batch.bind(r.slot, r.pb, r.init, r.steps)
        r.init = None
        self.active.append(r)

    def _retire(self, r: Request, now: float):
        r.finish = now
        if r.ctx is not None:
            if self.keep:
                r.state = r.ctx.read_state()
            r.ctx.close()
            r.ctx = None
        else:
            ent = self.batch.release(r.slot)
            if self.keep:
                r.state = ent["state"].cpu().numpy()
            self.free_slots.append(r.slot)
            r.slot = None
            if not self.keep:
                r.state = None
        self.used -= r.bytes
        self.done.append(r)

    # -- main loop ---------------------------------------------------------
    def run(self, stream: list, horizon: float = None):
        """Serve ``stream`` (dicts with arrival times in seconds); requests that
        arrive after ``horizon`` are not admitted.  Returns the finished
        requests and the elapsed wall time."""
        torch = self.torch
        pending = collections.deque(Request(d) for d in sorted(stream, key=lambda d: d["arrival"]))
        horizon = float("inf") if horizon is None else horizon
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now and pending[0].arrival <= horizon and self._fits(pending[0]):
                self._admit(pending.popleft(), now)
            if not self.active:
                if not pending or pending[0].arrival > horizon:
                    break
                wait = pending[0].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.05))
                continue
            self.batch.step(self.chunk)
            for r in self.active:
                if r.ctx is not None:
                    r.ctx.step(min(self.chunk, r.left))
            self.main.synchronize()
            self.side.synchronize()
            self.ticks += 1
            now = time.perf_counter() - t0
            still = []
            for r in self.active:
                r.left -= min(self.chunk, r.left)
                if r.left == 0:
                    self._retire(r, now)
                else:
                    still.append(r)
            self.active = still
        self.pending_left = len(pending)
        return self.done, time.perf_counter() - t0


def serve_plain(stream: list, horizon: float = None, device: int = 0, keep_states=False):
    """The same stream through one context per request, one request at a time."""
    import torch
    horizon = float("inf") if horizon is None else horizon
    reqs = [Request(d) for d in sorted(stream, key=lambda d: d["arrival"])]
    done = []
    t0 = time.perf_counter()
    for r in reqs:
        now = time.perf_counter() - t0
        if r.arrival > horizon:
            break
        if r.arrival > now:
            time.sleep(r.arrival - now)
        r.admit = time.perf_counter() - t0
        s = api.Solver(r.pb, r.init, device=device, path="stage")
        s.run(r.steps)
        r.finish = time.perf_counter() - t0
        if keep_states:
            r.state = s.read_state()
        s.close()
        r.init = None
        done.append(r)
        if horizon != float("inf") and time.perf_counter() - t0 > 4 * horizon:
            break
    return done, time.perf_counter() - t0


def summarize(done: list, elapsed: float) -> dict:
    lat = np.array([r.finish - r.arrival for r in done]) if done else np.array([np.nan])
    svc = np.array([r.finish - r.admit for r in done]) if done else np.array([np.nan])
    pts = sum(r.n * r.steps for r in done)
    return {"completed": len(done), "elapsed_s": elapsed, "solves_per_s": len(done) / elapsed if elapsed else 0.0,
            "grid_pt_updates_per_s": pts / elapsed if elapsed else 0.0,
            "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
            "service_p50_s": float(np.percentile(svc, 50)), "service_p99_s": float(np.percentile(svc, 99))}
