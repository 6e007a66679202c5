"""One periodic domain split over ranks by PE ranges: the host side of the
edge-window exchange.

The paper's solver decomposes the domain into processing elements (PEs) that
exchange only the halo points their stencils need (Sec. 1, Sec. 2.1, Fig.
1), and a step's message carries the edge points of every RK stage (Sec.
2.3).  Here each rank owns a contiguous range of PEs and steps it with a
stage engine.  After the engine forms the stage argument U^{n,(s)}, the rank
sends the H points at each end of its range to the neighbouring rank; before
the stage's right-hand side it makes sure that the neighbour's edge windows
of every level its delays read have arrived (n-k-l for each extrapolation
weight that is not zero; Eq. at1, Appendix A), waiting at most
``wait_limit`` seconds.  Received windows are kept by (level, stage, side),
the versions of a history-ring slot, so a window that arrives early or late
is used exactly at the levels that read it, and a run is bit for bit the
one-process run whatever the arrival timing within the wait limit.  A
needed window that does not arrive in time stops the rank with AT_ETIMEOUT.
There is no collective on the data path; ``drain`` (one all-reduce of a
progress count, then matching every message still outstanding) runs after
the steps, so that ranks that stopped early and ranks that finished leave
the process group together.

The engine is anything with these calls (``oracle.Oracle`` on a window
problem with ``open_ends`` provides them, and ``ContextEngine`` wraps a
library context on the GPU whose outer buffer points read windows put into
it from outside, ``at_put_ext``):

    level, stages, halo, nvar, P     current level n and the window's sizes
    stage_begin(s)                   form U^{n,(s)}
    edges(level, s) -> [2][H][nvar]  the range's two outer edge windows
    set_ext(level, s, side, win)     a neighbour's window beyond `side`
    delay(level, s, pe, side) -> k   the delay local PE `pe` uses there
    stage_rhs(s)                     K_s of the stage
    step_end() -> status             u^{n+1}, level + 1 (0 or AT_EUNSTABLE)

The transport (``GlooTransport``) sends the windows as torch.distributed
point-to-point messages (gloo on CPU ranks) and rings a doorbell per message
in the process group's key-value store, which the receiver polls.
"""
from __future__ import annotations

import time

import numpy as np

from .api import AT_ETIMEOUT, AtError

LEFT, RIGHT = 0, 1  # side of the range a window sits beyond, as the receiver sees it


def pe_ranges(P: int, world: int):
    """Contiguous PE ranges [lo, hi) per rank; sizes differ by at most one."""
    if world < 1 or P < world:
        raise ValueError("need 1 <= world <= P (got P=%d, world=%d)" % (P, world))
    base, extra = divmod(P, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def levels_read(mode: str, q: int, n: int, k: int):
    """Levels a buffer point of level n reads at delay k: n-k-l for every
    Lagrange extrapolation weight w_l(k) = prod_{m != l} (k+m)/(m-l) that is
    not zero (all l = 0..q for k >= 1, only l = 0 at k = 0); the delayed
    level alone for AS; n for SYNC."""
    if mode == "sync":
        return [n]
    if mode == "as" or k == 0:
        return [n - k]
    return [n - k - l for l in range(q + 1)]


class ContextEngine:
    """A library context (``api.Solver`` on the range's problem with
    ``open_ends``, ``pe_base`` and ``pe_total`` in its dict) as the stage
    engine of a rank.  The stage kernels form the next stage argument as part
    of their update (Eq. rk1), so stage_begin is empty: U^{n,(s)} of the
    range's outer edges is in the ring once stage s-1 has run."""

    def __init__(self, solver):
        self.s = solver
        self.stages, self.halo, self.nvar, self.P = solver.stages, solver.halo, solver.nvar, solver.P
        self.level = 0

    def stage_begin(self, s):
        pass

    def edges(self, level, s):
        return self.s.edges(level, s)

    def set_ext(self, level, s, side, win):
        self.s.put_ext(level, s, side, win)

    def delay(self, level, s, pe, side):
        return self.s.delay(level, s, pe, side)

    def stage_rhs(self, s):
        self.s.stage()

    def step_end(self):
        self.level += 1
        return 0

    def state(self):
        return self.s.read_state()


class GlooTransport:
    """Point-to-point messages through torch.distributed (gloo on CPU
    ranks), with a doorbell per message in the process group's key-value
    store: gloo's point-to-point works cannot be polled, nor waited on with a
    time limit without closing the connection, so the receiver polls the
    doorbell and waits on the receive only once the data is on its way."""

    PREFIX = "at_range/"

    def __init__(self, rank: int, store=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist, self.rank = torch, dist, rank
        if store is None:
            store = dist.distributed_c10d._get_default_store()
        self.store = store

    def _bell(self, src: int, dst: int, tag: int) -> str:
        return "%s%d-%d/%d" % (self.PREFIX, src, dst, tag)

    def isend(self, arr: np.ndarray, dst: int, tag: int):
        t = self.torch.from_numpy(np.ascontiguousarray(arr))
        w = self.dist.isend(t, dst, tag=tag)
        bell = self._bell(self.rank, dst, tag)
        self.store.set(bell, b"1")
        return w, t, bell

    def irecv(self, shape, src: int, tag: int):
        t = self.torch.empty(shape, dtype=self.torch.float64)
        return self.dist.irecv(t, src, tag=tag), t, self._bell(src, self.rank, tag)

    def arrived(self, bell: str) -> bool:
        return self.store.check([bell])

    def max_over_ranks(self, value: int) -> int:
        t = self.torch.tensor([int(value)], dtype=self.torch.int64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return int(t.item())


class RangeRank:
    """One rank of a PE-range split (see the module docstring).

    ``hold`` injects late or lost messages on the host, for tests: a dict
    {(level, stage, direction): stages} holds the window this rank sends
    towards ``direction`` (LEFT: the left edge to the left rank; RIGHT: the
    right edge to the right rank) back until this rank has begun ``stages``
    more stages, or has to wait itself (a rank never waits while it holds
    messages back, so holding alone cannot deadlock the ranks); ``None``
    drops it until ``drain``."""

    def __init__(self, engine, rank: int, world: int, mode: str, q: int, k_max: int, wait_limit: float = 5.0,
                 transport=None, hold=None):
        self.e = engine
        self.rank, self.world = rank, world
        self.left, self.right = (rank - 1) % world, (rank + 1) % world
        self.mode, self.q, self.k_max = mode, q, k_max
        self.wait_limit = float(wait_limit)
        self.S, self.H, self.nvar = engine.stages, engine.halo, engine.nvar
        self.keep = k_max + q + 1  # levels a buffer point can still read
        self.t = transport if transport is not None else (GlooTransport(rank) if world > 1 else None)
        self.hold = dict(hold or {})
        self.held = []       # [release stage count or None, array, dst, tag]
        self.sends = []      # outstanding sends (work, buffer)
        self.bells = []      # doorbells this rank rang
        self.recvs = {}      # (level, stage, side) -> (work, buffer, doorbell)
        self.got = {}        # (level, stage, side) -> [H][nvar] window
        self.begun = 0       # stage messages sent and posted: level * S + stage + 1
        self.waited_s = 0.0  # time spent waiting for windows
        self.waits = 0       # stages that had to wait for a window

    # -- messages ---------------------------------------------------------
    def _tag(self, level: int, stage: int, side: int) -> int:
        return (level * self.S + stage) * 2 + side

    def _send(self, arr, dst, tag):
        w, buf, bell = self.t.isend(arr, dst, tag)
        self.sends.append((w, buf))
        self.bells.append(bell)

    def _release(self, everything=False, lost=False):
        """Send held windows that are due (all held ones with `everything`;
        lost ones only with `lost`, in the drain)."""
        keep = []
        for item in self.held:
            if (item[0] is None and lost) or (item[0] is not None and (everything or self.begun >= item[0])):
                self._send(item[1], item[2], item[3])
            else:
                keep.append(item)
        self.held = keep

    def _post(self, level: int, stage: int):
        """Send this range's edge windows of U^{level,(stage)} and post the
        receives of the neighbours' windows of the same stage argument."""
        ed = self.e.edges(level, stage)  # [2][H][nvar]
        for direction, dst, win in ((LEFT, self.left, ed[0]), (RIGHT, self.right, ed[1])):
            # my left edge lies beyond the left rank's right end, and vice versa
            tag = self._tag(level, stage, RIGHT if direction == LEFT else LEFT)
            key = (level, stage, direction)
            if key in self.hold:
                after = self.hold.pop(key)
                self.held.append([None if after is None else self.begun + 1 + after, win.copy(), dst, tag])
            else:
                self._send(win, dst, tag)
        for side, src in ((LEFT, self.left), (RIGHT, self.right)):
            self.recvs[(level, stage, side)] = self.t.irecv((self.H, self.nvar), src, self._tag(level, stage, side))
        self.begun = level * self.S + stage + 1
        self._release()

    def _collect(self, keys):
        """Take in the windows of `keys` whose data is on its way."""
        for key in keys:
            if key in self.got or key not in self.recvs:
                continue
            w, buf, bell = self.recvs[key]
            if self.t.arrived(bell):
                w.wait()
                del self.recvs[key]
                self.got[key] = buf.numpy().copy()

    def _need(self, level: int, stage: int):
        P = self.e.P
        need = []
        for side, pe in ((LEFT, 0), (RIGHT, P - 1)):
            k = self.e.delay(level, stage, pe, side)
            need += [(m, stage, side) for m in levels_read(self.mode, self.q, level, k) if m >= 0]
        return need

    def _wait_for(self, keys):
        self._collect(keys)
        missing = [k for k in keys if k not in self.got]
        if not missing:
            return
        self._release(everything=True)  # never wait while holding messages back
        self.waits += 1
        t0 = time.monotonic()
        while True:
            self._collect(missing)
            missing = [k for k in keys if k not in self.got]
            if not missing:
                self.waited_s += time.monotonic() - t0
                return
            if time.monotonic() - t0 > self.wait_limit:
                raise AtError(AT_ETIMEOUT, "rank %d: edge window (level, stage, side) %s did not arrive within "
                              "%.3g s" % (self.rank, missing[0], self.wait_limit))
            time.sleep(1e-4)

    # -- stepping ---------------------------------------------------------
    def step(self) -> None:
        n = self.e.level
        for s in range(self.S):
            self.e.stage_begin(s)
            if self.world > 1:
                self._post(n, s)
                need = self._need(n, s)
                self._wait_for(need)
                for key in need:
                    self.e.set_ext(key[0], key[1], key[2], self.got[key])
            self.e.stage_rhs(s)
        st = self.e.step_end()
        if st != 0:
            raise AtError(st, "rank %d: non-finite value at level %d" % (self.rank, n + 1))
        for key in [k for k in self.got if k[0] < n + 1 - self.keep]:
            del self.got[key]

    def run(self, nsteps: int) -> None:
        for _ in range(int(nsteps)):
            self.step()

    def drain(self) -> None:
        """Complete every message: release what is held, then, up to the
        furthest stage any rank began, send the windows this rank never sent
        (zeros: nobody reads them any more) and post the receives it never
        posted, and wait for all of it.  Every rank calls it once, after its
        steps or after an error."""
        if self.world == 1:
            return
        self._release(everything=True, lost=True)
        top = self.t.max_over_ranks(self.begun)
        zero = np.zeros((self.H, self.nvar))
        for i in range(self.begun, top):
            level, stage = divmod(i, self.S)
            self._send(zero, self.left, self._tag(level, stage, RIGHT))
            self._send(zero, self.right, self._tag(level, stage, LEFT))
            for side, src in ((LEFT, self.left), (RIGHT, self.right)):
                self.recvs[(level, stage, side)] = self.t.irecv((self.H, self.nvar), src,
                                                                self._tag(level, stage, side))
        self.begun = max(self.begun, top)
        # every send now has its receive posted and every receive its send
        for w, _ in self.sends:
            w.wait()
        for w, _, bell in self.recvs.values():
            w.wait()
        self.sends, self.recvs = [], {}
        self.t.dist.barrier()
        for key in self.bells:  # the doorbells this rank rang were read by now
            self.t.store.delete_key(key)
