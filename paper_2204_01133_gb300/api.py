"""Thin ctypes binding of libat_gb300.so (C ABI in include/at.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  PyTorch supplies device memory (the state and the
workspace are torch tensors owned by the :class:`Solver`) and the stream
(``torch.cuda.current_stream()`` unless one is given).

Loading fails loudly when the library has not been built; there is no CPU
path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libat_gb300.so")

AT_OK, AT_EINVAL, AT_ENOMEM, AT_ECUDA, AT_EUNSTABLE, AT_ETIMEOUT, AT_ESTATE, AT_ECORRUPT = 0, -1, -2, -3, -4, -5, -6, -7
PDE = {"advdiff": 0, "rns": 1, "euler": 2, "adv_weno": 3, "burgers": 4, "rns_chain": 5}
RK = {"rk2": 0, "rk3tvd": 1, "rk4": 2}
MODE = {"sync": 0, "as": 1, "at": 2}
DIST = {"uniform": 0, "table": 1, "geometric": 2}
READ_STATE, READ_DELAYS, READ_RING, READ_STATS = 0, 1, 2, 3
NVAR = {"advdiff": 1, "adv_weno": 1, "burgers": 1, "rns": 4, "euler": 4, "rns_chain": 4}
STAGES = {"rk2": 2, "rk3tvd": 3, "rk4": 4}

# every symbol include/at.h declares
SYMBOLS = ("at_create", "at_workspace_bytes", "at_set_problem", "at_set_delays", "at_step", "at_run",
           "at_read", "at_profile", "at_set_option", "at_set_delay_trace", "at_destroy", "at_last_error",
           "at_run_noalloc", "at_stage", "at_edges", "at_put_ext", "at_delay",
           "at_checkpoint_bytes", "at_save", "at_restore", "at_check_guards",
           "at_batch_table_bytes", "at_batch_create", "at_batch_bind", "at_batch_release", "at_batch_set_config",
           "at_batch_step", "at_batch_run", "at_batch_query", "at_batch_destroy")
PATH_AUTO, PATH_STAGE, PATH_PERSISTENT, PATH_FUSED = 0, 1, 2, 3
OPT_PATH, OPT_WAIT_LIMIT, OPT_WITHHOLD_PE, OPT_ARRIVAL, OPT_HISTORY = 0, 1, 2, 3, 4
OPT_OPEN_ENDS, OPT_PE_BASE, OPT_PE_TOTAL = 5, 6, 7  # a PE range of a domain split over ranks
WENO_RECONSTRUCT, WENO_INTERPOLATE = 0, 1  # the WENO form of a problem ("weno" key of the dict)
WENO = {"reconstruct": WENO_RECONSTRUCT, "interpolate": WENO_INTERPOLATE}
HIST_STAGE, HIST_RECOMPUTE = 0, 1  # reading B (the neighbour's stage arguments) / A (recomputed from u^m)
NOALLOC_SCRATCH_BYTES = 8 << 20


class AtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("at status %d: %s" % (code, msg))
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [
        ("pde", ctypes.c_int32), ("order", ctypes.c_int32), ("rk", ctypes.c_int32), ("pe_size", ctypes.c_int32),
        ("n", ctypes.c_int64), ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("prm", ctypes.c_double * 16),
        ("weno", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class Delays(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32), ("k_max", ctypes.c_int32), ("dist", ctypes.c_int32), ("per_stage", ctypes.c_int32),
        ("prob", ctypes.c_double * 16), ("seed", ctypes.c_uint64), ("instance", ctypes.c_uint32),
        ("pad_", ctypes.c_uint32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("level", ctypes.c_int64), ("status", ctypes.c_int32), ("stages", ctypes.c_int32), ("nvar", ctypes.c_int32),
        ("halo", ctypes.c_int32), ("q", ctypes.c_int32), ("ring_levels", ctypes.c_int32),
        ("path", ctypes.c_int32), ("pad_", ctypes.c_int32), ("kernels_launched", ctypes.c_int64), ("launches_timed", ctypes.c_int64), ("stage_ms", ctypes.c_double),
    ]


_lib = None


def lib():
    """Load libat_gb300.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libat_gb300.so is not built; run `python -m paper_2204_01133_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        L.at_create.argtypes = [P(vp), ctypes.c_int, vp]
        L.at_workspace_bytes.argtypes = [P(Problem), P(Delays)]
        L.at_workspace_bytes.restype = ctypes.c_size_t
        L.at_set_problem.argtypes = [vp, P(Problem), vp, vp, ctypes.c_int, vp, ctypes.c_size_t]
        L.at_set_delays.argtypes = [vp, P(Delays)]
        L.at_step.argtypes = [vp, ctypes.c_int64]
        L.at_run.argtypes = [vp, ctypes.c_int64]
        L.at_read.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
        L.at_destroy.argtypes = [vp]
        L.at_profile.argtypes = [vp, ctypes.c_int]
        L.at_set_option.argtypes = [vp, ctypes.c_int, ctypes.c_int64]
        L.at_set_option.restype = ctypes.c_int
        L.at_set_delay_trace.argtypes = [vp, vp, ctypes.c_int64]
        L.at_set_delay_trace.restype = ctypes.c_int
        L.at_run_noalloc.argtypes = [P(Problem), P(Delays), vp, ctypes.c_int64, ctypes.c_int, vp]
        L.at_run_noalloc.restype = ctypes.c_int
        L.at_stage.argtypes = [vp]
        L.at_stage.restype = ctypes.c_int
        L.at_edges.argtypes = [vp, ctypes.c_int64, ctypes.c_int, vp]
        L.at_edges.restype = ctypes.c_int
        L.at_put_ext.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp]
        L.at_put_ext.restype = ctypes.c_int
        L.at_delay.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.at_delay.restype = ctypes.c_int
        L.at_checkpoint_bytes.argtypes = [vp]
        L.at_checkpoint_bytes.restype = ctypes.c_size_t
        L.at_save.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.at_save.restype = ctypes.c_int
        L.at_restore.argtypes = [vp, vp, ctypes.c_size_t, ctypes.c_int]
        L.at_restore.restype = ctypes.c_int
        L.at_check_guards.argtypes = [vp]
        L.at_check_guards.restype = ctypes.c_int
        L.at_last_error.restype = ctypes.c_char_p
        for f in ("at_create", "at_set_problem", "at_set_delays", "at_step", "at_run", "at_read", "at_profile",
                  "at_destroy"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def check(code: int) -> int:
    if code != AT_OK:
        raise AtError(code, lib().at_last_error().decode())
    return code


def problem_struct(pb: dict) -> Problem:
    s = Problem()
    s.pde = PDE[pb["pde"]]
    s.order = int(pb.get("order", 4))
    s.rk = RK[pb["rk"]]
    s.pe_size = int(pb["pe_size"])
    s.n = int(pb["n"])
    s.dx = float(pb["dx"])
    s.dt = float(pb["dt"])
    for i, v in enumerate(pb.get("prm", [])):
        s.prm[i] = float(v)
    s.weno = WENO[pb.get("weno", "reconstruct")]
    return s


def delays_struct(pb: dict) -> Delays:
    d = Delays()
    d.mode = MODE[pb["mode"]]
    d.k_max = int(pb["k_max"])
    d.dist = DIST[pb.get("dist", "uniform")]
    d.per_stage = int(pb.get("per_stage", 1))
    for i, v in enumerate(pb.get("prob", [])):
        d.prob[i] = float(v)
    d.seed = int(pb.get("seed", 0))
    d.instance = int(pb.get("instance", 0))
    return d


def workspace_bytes(pb: dict) -> int:
    return int(lib().at_workspace_bytes(ctypes.byref(problem_struct(pb)), ctypes.byref(delays_struct(pb))))


def run_noalloc(pb: dict, state, nsteps: int, device: int = 0, stream=None) -> None:
    """One whole solve through the allocation-free entry point.

    ``state``: a CUDA float64 tensor [nvar][n] holding the initial state; it
    is advanced nsteps steps in place.  The library's fixed device scratch
    array replaces the workspace, so nothing is allocated; problems larger
    than ``NOALLOC_SCRATCH_BYTES`` of workspace raise AT_ENOMEM.  Calls share
    that array: do not overlap them on the GPU.
    """
    import torch
    st = stream if stream is not None else torch.cuda.current_stream(torch.device("cuda", device))
    check(lib().at_run_noalloc(ctypes.byref(problem_struct(pb)), ctypes.byref(delays_struct(pb)),
                               ctypes.c_void_p(state.data_ptr()), int(nsteps), int(device),
                               ctypes.c_void_p(st.cuda_stream)))


class Solver:
    """One AT solve on one GPU.

    ``Solver(pb, init)`` allocates the state and workspace as torch tensors on
    ``device``, binds the problem (copying ``init`` from host or device) and
    the delay model.  ``step(n)`` enqueues, ``run(n)`` also synchronises and
    checks for non-finite values, ``state()`` returns the state tensor.
    """

    def __init__(self, pb: dict, init=None, device: int = 0, stream=None, state=None, path: str = "auto"):
        import torch

        self.torch = torch
        self.pb = dict(pb)
        self.device = torch.device("cuda", device)
        self.nvar = NVAR[pb["pde"]]
        self.n = int(pb["n"])
        self.P = self.n // int(pb["pe_size"])
        self.stages = STAGES[pb["rk"]]
        weno = pb["pde"] in ("euler", "adv_weno", "burgers")
        self.halo = (4 if pb.get("weno", "reconstruct") == "interpolate" else 3) if weno else int(pb["order"]) // 2
        L = lib()
        self._stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        check(L.at_create(ctypes.byref(h), device, ctypes.c_void_p(self._stream.cuda_stream)))
        self._h = h
        self._pbs = problem_struct(pb)
        self._dls = delays_struct(pb)
        hist = pb.get("history", "stage")
        if hist not in ("stage", "recompute"):
            raise AtError(AT_EINVAL, "history is 'stage' or 'recompute'")
        if hist == "recompute":  # before at_set_delays, which seeds level 0 of the ring
            self.set_option(OPT_HISTORY, HIST_RECOMPUTE)
        # a PE range of a larger domain: global PE indices, and open outer ends
        if pb.get("pe_total", 0):
            self.set_option(OPT_PE_BASE, int(pb.get("pe_base", 0)) % int(pb["pe_total"]))
            self.set_option(OPT_PE_TOTAL, int(pb["pe_total"]))
        if pb.get("open_ends", 0):
            self.set_option(OPT_OPEN_ENDS, 1)
        nbytes = workspace_bytes(pb)
        if nbytes == 0:
            raise AtError(AT_EINVAL, lib().at_last_error().decode())
        with torch.cuda.device(self.device):
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.u = state if state is not None else torch.empty((self.nvar, self.n), dtype=torch.float64,
                                                                  device=self.device)
        self.set_problem(init)
        self.set_delays()
        if path != "auto":
            self.set_path(path)

    # -- binding calls ----------------------------------------------------
    def set_problem(self, init=None):
        torch = self.torch
        if init is None:
            ptr, on_dev, keep = None, 1, None
        elif isinstance(init, torch.Tensor) and init.is_cuda:
            keep = init.to(torch.float64).contiguous()
            ptr, on_dev = keep.data_ptr(), 1
        else:
            keep = np.ascontiguousarray(np.asarray(init, dtype=np.float64).reshape(self.nvar, self.n))
            ptr, on_dev = keep.ctypes.data, 0
        check(lib().at_set_problem(self._h, ctypes.byref(self._pbs), ctypes.c_void_p(self.u.data_ptr()),
                                   ctypes.c_void_p(ptr) if ptr else None, on_dev,
                                   ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel()))

    def set_delays(self, **over):
        if over:
            self.pb.update(over)
            self._dls = delays_struct(self.pb)
        check(lib().at_set_delays(self._h, ctypes.byref(self._dls)))

    def step(self, nsteps: int):
        check(lib().at_step(self._h, int(nsteps)))

    def run(self, nsteps: int):
        check(lib().at_run(self._h, int(nsteps)))

    def state(self):
        return self.u

    def read_state(self) -> np.ndarray:
        out = np.empty((self.nvar, self.n), dtype=np.float64)
        check(lib().at_read(self._h, READ_STATE, ctypes.c_void_p(out.ctypes.data), out.nbytes, 0))
        return out

    def read_delays(self) -> np.ndarray:
        out = np.empty((self.stages, self.P, 2), dtype=np.uint8)
        check(lib().at_read(self._h, READ_DELAYS, ctypes.c_void_p(out.ctypes.data), out.nbytes, 0))
        return out

    def set_option(self, key: int, value: int):
        check(lib().at_set_option(self._h, int(key), int(value)))

    def check_guards(self):
        """Raise AtError(AT_ECORRUPT) if a canary zone of the workspace was
        overwritten (at_check_guards)."""
        check(lib().at_check_guards(self._h))

    def checkpoint(self, device: bool = False):
        """The run between two steps as one blob (at_save): host bytes (numpy
        uint8), or a torch uint8 tensor on the context's device."""
        nb = lib().at_checkpoint_bytes(self._h)
        if nb == 0:
            raise AtError(AT_ESTATE, "no problem and delay model set")
        if device:
            out = self.torch.empty(nb, dtype=self.torch.uint8, device=self.u.device)
            check(lib().at_save(self._h, ctypes.c_void_p(out.data_ptr()), nb, 1))
        else:
            out = np.empty(nb, dtype=np.uint8)
            check(lib().at_save(self._h, ctypes.c_void_p(out.ctypes.data), nb, 0))
        return out

    def restore(self, blob):
        """Continue from a blob of checkpoint() (at_restore); the context must
        hold the same problem and delay model."""
        if isinstance(blob, np.ndarray):
            blob = np.ascontiguousarray(blob, dtype=np.uint8)
            check(lib().at_restore(self._h, ctypes.c_void_p(blob.ctypes.data), blob.nbytes, 0))
        else:
            check(lib().at_restore(self._h, ctypes.c_void_p(blob.data_ptr()), blob.numel(), 1))

    def trace_delays(self, nsteps: int):
        """Record the delay of every (step, stage, PE, side) of the next
        ``nsteps`` steps into a device buffer; ``read_trace()`` returns it
        as uint8 [nsteps][stages][P][2].  ``nsteps`` = 0 detaches it."""
        torch = self.torch
        if nsteps <= 0:
            check(lib().at_set_delay_trace(self._h, None, 0))
            self._trace = None
            return
        self._trace = torch.zeros((nsteps, self.stages, self.P, 2), dtype=torch.uint8, device=self.u.device)
        check(lib().at_set_delay_trace(self._h, ctypes.c_void_p(self._trace.data_ptr()), int(nsteps)))

    def read_trace(self) -> np.ndarray:
        self.torch.cuda.synchronize(self.u.device)
        return self._trace.cpu().numpy()

    # -- a PE range of a domain split over ranks (open ends) ---------------
    def stage(self):
        """Enqueue the next RK stage of the current step (at_stage)."""
        check(lib().at_stage(self._h))

    def edges(self, level: int, stage: int) -> np.ndarray:
        """The range's outer edge windows of U^{level,(stage)}, [2][H][nvar]."""
        out = np.empty((2, self.halo, self.nvar), dtype=np.float64)
        check(lib().at_edges(self._h, int(level), int(stage), ctypes.c_void_p(out.ctypes.data)))
        return out

    def put_ext(self, level: int, stage: int, side: int, win) -> None:
        """A neighbour's [H][nvar] edge window beyond `side` of the range."""
        w = np.ascontiguousarray(win, dtype=np.float64).reshape(self.halo, self.nvar)
        check(lib().at_put_ext(self._h, int(level), int(stage), int(side), ctypes.c_void_p(w.ctypes.data)))

    def delay(self, level: int, stage: int, pe: int, side: int) -> int:
        k = lib().at_delay(self._h, int(level), int(stage), int(pe), int(side))
        if k < 0:
            check(k)
        return k

    def set_path(self, path: str):
        self.set_option(OPT_PATH, {"auto": PATH_AUTO, "stage": PATH_STAGE, "persistent": PATH_PERSISTENT,
                                  "fused": PATH_FUSED}[path])

    def profile(self, enable: bool = True):
        check(lib().at_profile(self._h, 1 if enable else 0))

    def stats(self) -> Stats:
        s = Stats()
        check(lib().at_read(self._h, READ_STATS, ctypes.byref(s), ctypes.sizeof(s), 0))
        return s

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().at_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
