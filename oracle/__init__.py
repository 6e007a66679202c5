"""Plain FP64 CPU oracle of the asynchrony-tolerant RK-stage right-hand side.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product library
never does.  The arithmetic lives in ``at_oracle.c`` (plain C, FP64,
``-ffp-contract=off``); this module only builds it and marshals arguments.

The problem description is the plain dict produced by the seeded input
generators (``paper_2204_01133_gb300.workloads``): the oracle reads the keys
it needs and maps the names to its own enum values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "at_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_PDE = {"advdiff": 0, "rns": 1, "euler": 2, "adv_weno": 3, "burgers": 4, "rns_chain": 5}
_RK = {"rk2": 0, "rk3tvd": 1, "rk4": 2}
_MODE = {"sync": 0, "as": 1, "at": 2}
_DIST = {"uniform": 0, "table": 1, "geometric": 2}


class _Problem(ctypes.Structure):
    _fields_ = [
        ("pde", ctypes.c_int),
        ("order", ctypes.c_int),
        ("rk", ctypes.c_int),
        ("n", ctypes.c_int64),
        ("pe_size", ctypes.c_int32),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("prm", ctypes.c_double * 16),
        ("mode", ctypes.c_int),
        ("k_max", ctypes.c_int),
        ("dist", ctypes.c_int),
        ("prob", ctypes.c_double * 16),
        ("seed", ctypes.c_uint64),
        ("per_stage", ctypes.c_int),
        ("instance", ctypes.c_uint32),
        ("pe_base", ctypes.c_int64),
        ("pe_total", ctypes.c_int64),
        ("open_ends", ctypes.c_int),
        ("history", ctypes.c_int),
        ("weno_interp", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile at_oracle.c into liboracle.so (gcc, FP64, no contraction;
    OpenMP over PEs where the compiler has it, else single-threaded)."""
    hdr = os.path.join(_HERE, "at_oracle.h")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                                                           os.path.getmtime(hdr)):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    tmp = _LIB + ".%d.tmp" % os.getpid()
    r = subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [P(_Problem), P(ctypes.c_double)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        for f in ("orc_nvar", "orc_stages", "orc_q", "orc_ring_levels"):
            getattr(L, f).argtypes = [ctypes.c_void_p]
            getattr(L, f).restype = ctypes.c_int
        L.orc_level.argtypes = [ctypes.c_void_p]
        L.orc_level.restype = ctypes.c_int64
        L.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_run.restype = ctypes.c_int
        L.orc_get_state.argtypes = [ctypes.c_void_p, P(ctypes.c_double)]
        L.orc_get_delays.argtypes = [ctypes.c_void_p, P(ctypes.c_uint8)]
        L.orc_set_history.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, P(ctypes.c_double)]
        L.orc_rhs.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, P(ctypes.c_int32),
                              P(ctypes.c_double)]
        L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.orc_thresholds.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_uint64)]
        L.orc_draw.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.orc_draw.restype = ctypes.c_int
        L.orc_lagrange_weights.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]
        L.orc_weno5_js.argtypes = [P(ctypes.c_double), ctypes.c_double]
        L.orc_weno5_js.restype = ctypes.c_double
        L.orc_weno5_interp.argtypes = [P(ctypes.c_double), ctypes.c_double]
        L.orc_weno5_interp.restype = ctypes.c_double
        L.orc_edge_flux.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, P(ctypes.c_int32),
                                    ctypes.c_int64, ctypes.c_int64, P(ctypes.c_double)]
        L.orc_set_level.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_set_state.argtypes = [ctypes.c_void_p, P(ctypes.c_double)]
        L.orc_force_delays.argtypes = [ctypes.c_void_p, P(ctypes.c_int32)]
        L.orc_set_delay_trace.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
        L.orc_get_history.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
        L.orc_get_history.restype = ctypes.c_int
        L.orc_stage_begin.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_stage_rhs.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_step_end.argtypes = [ctypes.c_void_p]
        L.orc_step_end.restype = ctypes.c_int
        L.orc_get_edges.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, P(ctypes.c_double)]
        L.orc_get_edges.restype = ctypes.c_int
        L.orc_set_ext.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, P(ctypes.c_double)]
        L.orc_delay.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.orc_delay.restype = ctypes.c_int
        L.orc_halo.argtypes = [ctypes.c_void_p]
        L.orc_halo.restype = ctypes.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _problem(pb: dict) -> _Problem:
    s = _Problem()
    s.pde = _PDE[pb["pde"]]
    s.order = int(pb.get("order", 4))
    s.rk = _RK[pb["rk"]]
    s.n = int(pb["n"])
    s.pe_size = int(pb["pe_size"])
    s.dx = float(pb["dx"])
    s.dt = float(pb["dt"])
    prm = list(pb.get("prm", []))
    for i, v in enumerate(prm):
        s.prm[i] = float(v)
    s.mode = _MODE[pb["mode"]]
    s.k_max = int(pb["k_max"])
    s.dist = _DIST[pb.get("dist", "uniform")]
    for i, v in enumerate(pb.get("prob", [])):
        s.prob[i] = float(v)
    s.seed = int(pb.get("seed", 0))
    s.per_stage = int(pb.get("per_stage", 1))
    s.instance = int(pb.get("instance", 0))
    s.pe_base = int(pb.get("pe_base", 0))
    s.pe_total = int(pb.get("pe_total", 0))
    s.open_ends = int(pb.get("open_ends", 0))
    s.history = {"stage": 0, "recompute": 1}[pb.get("history", "stage")]
    s.weno_interp = {"reconstruct": 0, "interpolate": 1}[pb.get("weno", "reconstruct")]
    return s


class Oracle:
    """One oracle run: ``Oracle(problem, init)`` then ``run(nsteps)``."""

    def __init__(self, pb: dict, init: np.ndarray):
        L = lib()
        self.pb = dict(pb)
        self._s = _problem(pb)
        init = np.ascontiguousarray(init, dtype=np.float64)
        self._h = L.orc_create(ctypes.byref(self._s), _dptr(init))
        if not self._h:
            raise ValueError("oracle rejected the problem description")
        self.nvar = L.orc_nvar(self._h)
        self.stages = L.orc_stages(self._h)
        self.q = L.orc_q(self._h)
        self.ring_levels = L.orc_ring_levels(self._h)
        self.halo = L.orc_halo(self._h)
        self.n = int(pb["n"])
        self.P = self.n // int(pb["pe_size"])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def level(self) -> int:
        return int(lib().orc_level(self._h))

    def run(self, nsteps: int) -> int:
        return int(lib().orc_run(self._h, int(nsteps)))

    def state(self) -> np.ndarray:
        out = np.empty((self.nvar, self.n), dtype=np.float64)
        lib().orc_get_state(self._h, _dptr(out))
        return out

    def delays(self) -> np.ndarray:
        out = np.empty((self.stages, self.P, 2), dtype=np.uint8)
        lib().orc_get_delays(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return out

    def history(self, level: int, stage: int):
        """The stored stage argument U^{level,(stage)} [nvar][n], or None if
        it is no longer (or not yet) kept."""
        out = np.empty((self.nvar, self.n), dtype=np.float64)
        if lib().orc_get_history(self._h, int(level), int(stage), ctypes.c_void_p(out.ctypes.data)) != 0:
            return None
        return out

    def set_history(self, level: int, stage: int, field: np.ndarray) -> None:
        f = np.ascontiguousarray(field, dtype=np.float64).reshape(self.nvar, self.n)
        lib().orc_set_history(self._h, int(level), int(stage), _dptr(f))

    def rhs(self, level: int, stage: int, kforce=None) -> np.ndarray:
        K = np.empty((self.nvar, self.n), dtype=np.float64)
        kp = None
        if kforce is not None:
            kf = np.ascontiguousarray(kforce, dtype=np.int32).reshape(self.P, 2)
            kp = kf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            self._kf = kf
        lib().orc_rhs(self._h, int(level), int(stage), kp, _dptr(K))
        return K

    def edge_flux(self, level: int, stage: int, pe: int, i: int, kforce) -> np.ndarray:
        kf = np.ascontiguousarray(kforce, dtype=np.int32).reshape(self.P, 2)
        F = np.empty(self.nvar, dtype=np.float64)
        lib().orc_edge_flux(self._h, int(level), int(stage), kf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            int(pe), int(i), _dptr(F))
        return F

    def set_level(self, level: int) -> None:
        lib().orc_set_level(self._h, int(level))

    def set_state(self, u: np.ndarray) -> None:
        f = np.ascontiguousarray(u, dtype=np.float64).reshape(self.nvar, self.n)
        lib().orc_set_state(self._h, _dptr(f))

    def force_delays(self, k) -> None:
        if k is None:
            lib().orc_force_delays(self._h, None)
            return
        kf = np.ascontiguousarray(k, dtype=np.int32).reshape(self.P, 2)
        self._kfix = kf
        lib().orc_force_delays(self._h, kf.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))

    def set_delay_trace(self, trace, n0: int = 0) -> None:
        """Replay recorded delays: trace[steps][stages][P][2] (uint8) for the
        levels n0, n0 + 1, ... (None clears)."""
        if trace is None:
            lib().orc_set_delay_trace(self._h, None, 0, 0)
            return
        t = np.ascontiguousarray(trace, dtype=np.uint8)
        assert t.ndim == 4 and t.shape[2:] == (self.P, 2), t.shape
        lib().orc_set_delay_trace(self._h, ctypes.c_void_p(t.ctypes.data), int(n0), int(t.shape[0]))

    # one RK step stage by stage (a rank of a PE-range split exchanges edge
    # windows between these calls); run(1) is the same arithmetic
    def stage_begin(self, stage: int) -> None:
        lib().orc_stage_begin(self._h, int(stage))

    def stage_rhs(self, stage: int) -> None:
        lib().orc_stage_rhs(self._h, int(stage))

    def step_end(self) -> int:
        return int(lib().orc_step_end(self._h))

    def edges(self, level: int, stage: int) -> np.ndarray:
        """[2][H][nvar]: the window's left and right edge windows of U^{level,(stage)}."""
        out = np.empty((2, self.halo, self.nvar), dtype=np.float64)
        if lib().orc_get_edges(self._h, int(level), int(stage), _dptr(out)) != 0:
            raise ValueError("level %d stage %d is not stored" % (level, stage))
        return out

    def set_ext(self, level: int, stage: int, side: int, win: np.ndarray) -> None:
        """Open ends: the [H][nvar] edge window of the PE beyond `side`."""
        w = np.ascontiguousarray(win, dtype=np.float64).reshape(self.halo, self.nvar)
        lib().orc_set_ext(self._h, int(level), int(stage), int(side), _dptr(w))

    def delay(self, level: int, stage: int, pe: int, side: int) -> int:
        """The clamped delay local PE `pe` uses at (level, stage, side)."""
        return int(lib().orc_delay(self._h, int(level), int(stage), int(pe), int(side)))

    def draw(self, level: int, stage: int, pe: int, side: int) -> int:
        return int(lib().orc_draw(self._h, int(level), int(stage), int(pe), int(side)))


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's loops over PEs (0: all cores); returns the
    count in effect.  Results are the same for any count."""
    return int(lib().orc_set_threads(int(n)))


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def thresholds(k_max: int, dist: str = "uniform", prob=()):
    p = (ctypes.c_double * 16)(*[float(v) for v in prob])
    t = (ctypes.c_uint64 * 16)()
    lib().orc_thresholds(int(k_max), _DIST[dist], p, t)
    return [int(t[i]) for i in range(k_max)]


def lagrange_weights(q: int, k: int):
    w = (ctypes.c_double * 8)()
    lib().orc_lagrange_weights(int(q), int(k), w)
    return [float(w[i]) for i in range(q + 1)]


def weno5(v, eps: float = 1e-6) -> float:
    a = (ctypes.c_double * 5)(*[float(x) for x in v])
    return float(lib().orc_weno5_js(a, float(eps)))


def weno5_interp(v, eps: float = 1e-6) -> float:
    a = (ctypes.c_double * 5)(*[float(x) for x in v])
    return float(lib().orc_weno5_interp(a, float(eps)))
