"""Batched and served solves through the library's batch ABI.

:class:`Batch` holds a slot table on the device and one state + workspace
(torch tensors) per bound instance.  :func:`autotune` picks the launch
configuration (threads per CTA, resident CTAs per SM) by timing real chunks
of the run; the result is cached per GPU model and batch signature.
Argument marshalling and bookkeeping only: the computation runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes
import json
import os
import time

import numpy as np

from . import api

_batch_ready = False


def _lib():
    global _batch_ready
    L = api.lib()
    if not _batch_ready:
        P, vp = ctypes.POINTER, ctypes.c_void_p
        L.at_batch_table_bytes.argtypes = [ctypes.c_int64, ctypes.c_int64]
        L.at_batch_table_bytes.restype = ctypes.c_size_t
        L.at_batch_create.argtypes = [P(vp), ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_size_t]
        L.at_batch_bind.argtypes = [vp, ctypes.c_int64, P(Instance)]
        L.at_batch_release.argtypes = [vp, ctypes.c_int64]
        L.at_batch_set_config.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.at_batch_step.argtypes = [vp, ctypes.c_int64]
        L.at_batch_run.argtypes = [vp, ctypes.c_int64]
        L.at_batch_query.argtypes = [vp, ctypes.c_int64, P(SlotInfo)]
        L.at_batch_destroy.argtypes = [vp]
        for f in ("at_batch_create", "at_batch_bind", "at_batch_release", "at_batch_set_config", "at_batch_step",
                  "at_batch_run", "at_batch_query", "at_batch_destroy"):
            getattr(L, f).restype = ctypes.c_int
        _batch_ready = True
    return L


class Instance(ctypes.Structure):
    _fields_ = [("pb", api.Problem), ("dl", api.Delays), ("state_dev", ctypes.c_void_p),
                ("workspace_dev", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t), ("nsteps", ctypes.c_int64)]


class SlotInfo(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int64), ("left", ctypes.c_int64), ("status", ctypes.c_int32),
                ("bound", ctypes.c_int32)]


INSTANCE, FLAT = 0, 1


def table_bytes(capacity: int, max_windows: int = None) -> int:
    mw = 128 * int(capacity) if max_windows is None else int(max_windows)
    return int(_lib().at_batch_table_bytes(int(capacity), mw))


class Batch:
    """A device slot table of ``capacity`` independent solves."""

    def __init__(self, capacity: int, device: int = 0, stream=None, max_windows: int = None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.capacity = int(capacity)
        self.max_windows = 128 * self.capacity if max_windows is None else int(max_windows)
        L = _lib()
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.table = torch.empty(table_bytes(capacity, self.max_windows), dtype=torch.uint8, device=self.device)
        h = ctypes.c_void_p()
        api.check(L.at_batch_create(ctypes.byref(h), device, ctypes.c_void_p(self._stream.cuda_stream),
                                    self.capacity, self.max_windows, ctypes.c_void_p(self.table.data_ptr()),
                                    self.table.numel()))
        self._h = h
        self.slots = {}  # slot -> dict(pb, state, ws, nsteps)
        self.config = (INSTANCE, 256, 3, 1)

    def bind(self, slot: int, pb: dict, init, nsteps: int, state=None, workspace=None):
        torch = self.torch
        nvar, n = api.NVAR[pb["pde"]], int(pb["n"])
        if state is None:
            state = torch.empty((nvar, n), dtype=torch.float64, device=self.device)
        if init is not None:
            src = init if isinstance(init, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(init))
            state.copy_(src.reshape(nvar, n))
        nb = api.workspace_bytes(pb)
        if workspace is None:
            workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)
        inst = Instance()
        inst.pb = api.problem_struct(pb)
        inst.dl = api.delays_struct(pb)
        inst.state_dev = state.data_ptr()
        inst.workspace_dev = workspace.data_ptr()
        inst.workspace_bytes = workspace.numel()
        inst.nsteps = int(nsteps)
        api.check(_lib().at_batch_bind(self._h, int(slot), ctypes.byref(inst)))
        self.slots[int(slot)] = dict(pb=pb, state=state, ws=workspace, nsteps=int(nsteps))
        return state

    def release(self, slot: int):
        api.check(_lib().at_batch_release(self._h, int(slot)))
        return self.slots.pop(int(slot))

    def set_config(self, mode: int = INSTANCE, block: int = 256, ctas_per_sm: int = 3, use_graph: bool = True):
        api.check(_lib().at_batch_set_config(self._h, int(mode), int(block), int(ctas_per_sm),
                                             1 if use_graph else 0))
        self.config = (int(mode), int(block), int(ctas_per_sm), 1 if use_graph else 0)

    def step(self, chunk: int):
        api.check(_lib().at_batch_step(self._h, int(chunk)))

    def run(self, chunk: int):
        api.check(_lib().at_batch_run(self._h, int(chunk)))

    def query(self, slot: int) -> SlotInfo:
        info = SlotInfo()
        api.check(_lib().at_batch_query(self._h, int(slot), ctypes.byref(info)))
        return info

    def state(self, slot: int):
        return self.slots[int(slot)]["state"]

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib().at_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# autotuner
# --------------------------------------------------------------------------
CANDIDATES = [(INSTANCE, 256, 2), (INSTANCE, 256, 3), (INSTANCE, 128, 4), (INSTANCE, 128, 6), (INSTANCE, 128, 8),
              (FLAT, 256, 1), (FLAT, 128, 1)]


def _cache_path():
    return os.environ.get("AT_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "at_gb300_tune.json"))


def signature(batch: Batch) -> str:
    kinds = {}
    pts = 0
    for s in batch.slots.values():
        pb = s["pb"]
        key = "%s%d-B%d" % (pb["pde"], pb.get("order", 0), pb["pe_size"])
        kinds[key] = kinds.get(key, 0) + 1
        pts += int(pb["n"])
    scale = int(round(np.log2(max(pts, 1))))
    return "pts2^%d:" % scale + ",".join("%s*%d" % kv for kv in sorted(kinds.items()))


def autotune(batch: Batch, chunk: int, candidates=CANDIDATES, use_cache: bool = True) -> dict:
    """Time one real chunk of the run per candidate configuration and keep the
    fastest (the arithmetic, hence every result, is the same for all).  The
    steps are not wasted: each trial advances the batch by ``chunk`` steps."""
    import torch
    gpu = torch.cuda.get_device_name(batch.device)
    sig = signature(batch)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except Exception:
            cache = {}
    key = "%s|%s|%d" % (gpu, sig, chunk)
    if use_cache and key in cache:
        c = cache[key]
        batch.set_config(c["mode"], c["block"], c["ctas_per_sm"], True)
        return dict(c, cached=True)
    timings = []
    for mode, block, per_sm in candidates:
        batch.set_config(mode, block, per_sm, False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        batch.step(chunk)
        e1.record()
        torch.cuda.synchronize()
        timings.append((e0.elapsed_time(e1), mode, block, per_sm))
    ms, mode, block, per_sm = min(timings)
    batch.set_config(mode, block, per_sm, True)
    res = {"mode": mode, "block": block, "ctas_per_sm": per_sm, "ms": ms,
           "trials": [[t, m, b, c] for t, m, b, c in timings], "cached": False}
    if use_cache:
        cache[key] = res
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(cache, open(path, "w"), indent=1)
        except Exception:
            pass
    return res
