"""Shared parity measure of the GPU tests: per-variable relative error.

err_v = max_j |gpu_v(j) - oracle_v(j)| / scale_v, with scale_v the largest
|oracle_v| over the domain, except for the momentum rho u of the reacting
Navier-Stokes and reactive Euler states, which starts at zero (fluid at
rest) and is scaled by max(max_j |rho u|, max_j rho c), c = sqrt(gamma p /
rho) the local sound speed.  Why that floor: the momentum update is
dt * (-(rho u^2 + p)_x + ...), and its rounding errors scale with the
pressure p = rho c^2 / gamma in the flux, times the acoustic CFL number
dt c / dx and the stencil's coefficient sum, i.e. eps_mach * O(1) * rho c.
A momentum error is therefore measured against the momentum of the fluid
moving at its own sound speed, never against |rho E| (the whole-state norm
over-weights energy, up to ~20 times the momentum scale in these
workloads).

Every parity assertion in the GPU tests goes through ``errors`` and
``check``; a bound is a number stated in the test, and ``check`` prints the
errors and the bound of every comparison it makes.
"""
import math

import numpy as np

TOL_STEP = 1e-12   # relative, per variable, after one RK step
TOL_RUN = 1e-10    # relative, per variable, after the whole run

_MOMENTUM_PDES = {"rns": 0, "rns_chain": 0, "euler": 1}


def _gamma(pb):
    return float(pb["prm"][0])


def _pressure(pb, o):
    """p of the conserved state (rho, rho u, rho E, rho Y)."""
    gam = _gamma(pb)
    heat = float(pb["prm"][6]) if pb["pde"] in ("rns", "rns_chain") else float(pb["prm"][3])
    rho, ru, rE, rY = o[0], o[1], o[2], o[3]
    return (gam - 1.0) * (rE - 0.5 * ru * ru / rho - heat * rY)


def scales(pb, o):
    """Per-variable scale of the oracle state o [nvar][n]."""
    o = np.asarray(o)
    sc = np.abs(o).max(axis=1)
    if pb["pde"] in _MOMENTUM_PDES:
        p = _pressure(pb, o)
        rho_c = np.sqrt(np.maximum(_gamma(pb) * p * o[0], 0.0)).max()
        sc[1] = max(sc[1], rho_c)
    return np.maximum(sc, 1e-300)


def errors(pb, g, o):
    """Per-variable relative errors of g against the oracle state o."""
    o = np.asarray(o)
    g = np.asarray(g).reshape(o.shape)
    return np.abs(g - o).max(axis=1) / scales(pb, o)


def check(pb, g, o, bound, what=""):
    """Assert every per-variable error is within ``bound`` (a scalar or one
    bound per variable); print the errors and the bound."""
    e = errors(pb, g, o)
    b = np.broadcast_to(np.asarray(bound, dtype=np.float64), e.shape)
    print("parity %s: per-variable rel err %s, bound %s"
          % (what, " ".join("%.2e" % x for x in e), " ".join("%.1e" % x for x in b)))
    assert np.all(e <= b), (what, e.tolist(), b.tolist())
    return e


# Fixed bounds of the shock cases.  One-step bound per variable (rho, rho u,
# rho E, rho Y): 20x the largest one-step self-drift over all cases
# (2.7e-12, 1.1e-11, 1.1e-10, 3.3e-12).
DET_STEP = (6e-11, 3e-10, 3e-9, 7e-11)
# Run bounds, by case: 20x the measured run self-drift (in brackets).
DET_RUN = {
    "weno-1024": 1e-8,   # 80 steps (4.7e-10)
    "weno-512": 1.3e-8,  # 80 steps (6.4e-10)
    "weno-96": 2e-7,     # 20 steps (8.9e-9): 8 PEs, four PE edges inside the slab
    "sync": 8e-9,        # 60 steps (3.6e-10)
    "as": 1.1e-8,        # 60 steps (5.4e-10)
    "full-0": 1e-8,      # 40 steps, PE 0 of 16,384 (the shock) on its 5-PE window (4.8e-10)
    "full-last": 5e-10,  # 40 steps, PE 16,383 (the rarefaction behind the slab) (2.3e-11)
    "ring": 9e-9,        # 25 steps, the history ring test's case (4.1e-10)
    "serve": 8e-9,       # 40 steps, the served detonation request (4.0e-10)
    "interp": 9e-9,      # 60 steps, the WENO interpolation form (4.4e-10)
}
# the served detonation request checked against the oracle: (requested N,
# seed, request id = instance word, steps); N rounds down to 2,560 (5 PEs of 512)
SERVE_DET = (3000, 13, 2, 40)
# the full-size detonation (N = 2^24, PEs of 1024): PEs recomputed on 5-PE
# windows; the two next to the slab take shock bounds (measured on the
# window's middle PE), the others the plain run bound
DET_FULL_STEPS = 40
DET_FULL_SHOCK = {0: "full-0", 16383: "full-last"}
DET_CASES = {  # name: (workload kwargs, steps); the same table drives the CPU drift check
    "weno-1024": (dict(n=8192, pe_size=1024, mode="at", k_max=4, seed=9), 80),
    "weno-512": (dict(n=4096, pe_size=512, mode="at", k_max=4, seed=9), 80),
    "weno-96": (dict(n=768, pe_size=96, mode="at", k_max=4, seed=9), 20),
    "sync": (dict(n=4096, pe_size=512, mode="sync", k_max=4, seed=1), 60),
    "as": (dict(n=4096, pe_size=512, mode="as", k_max=4, seed=1), 60),
    "ring": (dict(n=4096, pe_size=512, mode="at", k_max=4, seed=2), 25),
    "interp": (dict(n=4096, pe_size=512, mode="at", k_max=4, seed=4, weno="interpolate"), 60),
}


def detonation_window(pb, u0, p):
    """The 5-PE window around PE p as an oracle problem (global PE indices in
    the delay counter)."""
    P, B = pb["n"] // pb["pe_size"], pb["pe_size"]
    idx = np.arange(p - 2, p + 3) % P
    sub = np.concatenate([u0[:, i * B:(i + 1) * B] for i in idx], axis=1)
    return dict(pb, n=5 * B, pe_base=p - 2, pe_total=P), sub


def self_drift(pb, init, steps, seeds=(0, 1, 2, 3), cols=slice(None)):
    """Conditioning of a case: the largest per-variable drift of the oracle
    against itself when its initial state is perturbed by 1e-15 (relative,
    seeded), after one step and after ``steps`` steps, over the points
    ``cols`` (the middle PE of a window, or everything)."""
    import oracle
    a = oracle.Oracle(pb, init)
    assert a.run(1) == 0
    a1 = a.state()[:, cols]
    assert a.run(steps - 1) == 0
    an = a.state()[:, cols]
    e1 = np.zeros(a1.shape[0])
    en = np.zeros(a1.shape[0])
    for sd in seeds:
        rng = np.random.default_rng(sd)
        b = oracle.Oracle(pb, init * (1.0 + 1e-15 * rng.standard_normal(init.shape)))
        assert b.run(1) == 0
        e1 = np.maximum(e1, errors(pb, b.state()[:, cols], a1))
        assert b.run(steps - 1) == 0
        en = np.maximum(en, errors(pb, b.state()[:, cols], an))
    return e1, en


def shock_cases():
    """Every shock case of the GPU tests as (name, problem, initial state,
    steps, the points compared)."""
    from paper_2204_01133_gb300 import workloads as W
    out = []
    for name, (kw, steps) in DET_CASES.items():
        pb, u0 = W.detonation(**kw)
        out.append((name, pb, u0, steps, slice(None)))
    pb, u0 = W.detonation()
    B = pb["pe_size"]
    for p, name in DET_FULL_SHOCK.items():
        spb, sub = detonation_window(pb, u0, p)
        out.append((name, spb, sub, DET_FULL_STEPS, slice(2 * B, 3 * B)))
    n, seed, rid, steps = SERVE_DET
    pb, u0 = W.serving_request("detonation", n, seed, instance=rid)
    out.append(("serve", pb, u0, steps, slice(None)))
    return out
