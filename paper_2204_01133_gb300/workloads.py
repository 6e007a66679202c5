"""Seeded synthetic inputs: problem descriptions and initial states.

This module holds no part of the right-hand-side arithmetic.  It builds the
plain problem dict that both the CUDA library binding and the CPU oracle
marshal into their own structures, and the FP64 initial fields.  Names of
the dict keys follow the paper's statement of the problem (Sec. 2.1 and
Sec. 5): PDE, stencil order, RK scheme, PE size, maximum delay and delay
probabilities.

Physics constants of the workloads (``prm``):

* ``advdiff``   [c, a]                              u_t + c u_x = a u_xx
* ``adv_weno``  [c, eps]                            u_t + c u_x = 0 (WENO5)
* ``burgers``   [0, eps]                            u_t + (u^2/2)_x = 0 (WENO5)
* ``rns``       [gamma, mu, Pr, Le, A, Ea, q_c]     reacting Navier-Stokes
* ``euler``     [gamma, A, Ea, Q, eps]              reactive Euler (WENO5)

The WENO problems take ``weno`` = "reconstruct" (flux reconstruction, Eq.
atRecon) or "interpolate" (edge values by Eqs. interpS/fullSten/omg with the
fourth-order staggered difference).

All quantities are nondimensional with the unburnt state rho0 = T0 = 1 and a
gas constant of 1 (p = rho T).
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

NVAR = {"advdiff": 1, "adv_weno": 1, "burgers": 1, "rns": 4, "euler": 4}


def base_problem(**kw) -> dict:
    pb = {
        "pde": "advdiff", "order": 4, "rk": "rk4", "n": 2048, "pe_size": 64,
        "dx": 1.0, "dt": 1.0, "prm": [], "mode": "at", "k_max": 3,
        "dist": "uniform", "prob": [], "seed": 0, "per_stage": 1, "instance": 0,
    }
    pb.update(kw)
    return pb


# --------------------------------------------------------------------------
# Linear advection-diffusion, sine wave, 4th-order central + AT4, RK4
# (N = 2048, 32 PEs of 64, delays uniform on {0..3}, 10,000 steps).  The
# stated "CFL 0.5" is read as half the AT4 stability limit: with k <= 3 and
# RK4 the AT4 scheme is stable up to a diffusion number a dt / dx^2 of about
# 0.15, so the default is 0.075 (0.5 itself blows up under AT4).
# --------------------------------------------------------------------------
def advdiff(n=2048, pe_size=64, order=4, c=1.0, a=0.01, cfl=0.075, mode="at", k_max=3,
            dist="uniform", prob=(), seed=0, per_stage=1, rk="rk4", dt=None, length=2 * math.pi):
    dx = length / n
    if dt is None:
        lim = []
        if c != 0.0:
            lim.append(dx / abs(c))
        if a != 0.0:
            lim.append(dx * dx / a)
        dt = cfl * min(lim)
    pb = base_problem(pde="advdiff", order=order, rk=rk, n=n, pe_size=pe_size, dx=dx, dt=dt,
                      prm=[c, a], mode=mode, k_max=k_max, dist=dist, prob=list(prob), seed=seed,
                      per_stage=per_stage)
    x = np.arange(n, dtype=np.float64) * dx
    init = np.sin(x)[None, :].copy()
    return pb, init


def advdiff_exact(pb: dict, t: float) -> np.ndarray:
    """e^{-a t} sin(x - c t): the exact solution for the sine initial state."""
    c, a = pb["prm"][0], pb["prm"][1]
    x = np.arange(pb["n"], dtype=np.float64) * pb["dx"]
    return (math.exp(-a * t) * np.sin(x - c * t))[None, :]


# --------------------------------------------------------------------------
# Scalar linear advection with WENO5 (the order test of Sec. 3:
# x in [-1, 1], u0 = sin^4(pi x + 0.25), c = 5, RK3, dt ~ dx^2).
# --------------------------------------------------------------------------
def adv_weno(n=256, pe_size=16, c=5.0, eps=1e-6, mode="at", k_max=1, dist="uniform", prob=(),
             seed=0, per_stage=1, dt=None, dt_coef=None, rk="rk3tvd", weno="reconstruct"):
    dx = 2.0 / n
    if dt is None:
        dt = dt_coef * dx * dx if dt_coef is not None else 0.5 * dx / abs(c)
    pb = base_problem(pde="adv_weno", rk=rk, n=n, pe_size=pe_size, dx=dx, dt=dt, prm=[c, eps],
                      mode=mode, k_max=k_max, dist=dist, prob=list(prob), seed=seed,
                      per_stage=per_stage, weno=weno)
    x = -1.0 + np.arange(n, dtype=np.float64) * dx
    init = (np.sin(np.pi * x + 0.25) ** 4)[None, :].copy()
    return pb, init


def adv_weno_exact(pb: dict, t: float) -> np.ndarray:
    c = pb["prm"][0]
    x = -1.0 + np.arange(pb["n"], dtype=np.float64) * pb["dx"]
    xs = x - c * t
    return (np.sin(np.pi * xs + 0.25) ** 4)[None, :]


# --------------------------------------------------------------------------
# Inviscid Burgers with WENO5 (the nonlinear order test of Sec. 3:
# x in [-1, 1], u0 = 0.5 + sin(pi x), RK3, dt ~ dx^2).
# --------------------------------------------------------------------------
def burgers(n=256, pe_size=16, eps=1e-6, mode="at", k_max=1, dist="uniform", prob=(), seed=0, per_stage=1,
            dt=None, dt_coef=None, rk="rk3tvd", weno="reconstruct"):
    dx = 2.0 / n
    if dt is None:
        dt = dt_coef * dx * dx if dt_coef is not None else 0.4 * dx / 1.5
    pb = base_problem(pde="burgers", rk=rk, n=n, pe_size=pe_size, dx=dx, dt=dt, prm=[0.0, eps], mode=mode,
                      k_max=k_max, dist=dist, prob=list(prob), seed=seed, per_stage=per_stage, weno=weno)
    x = -1.0 + np.arange(n, dtype=np.float64) * dx
    init = (0.5 + np.sin(np.pi * x))[None, :].copy()
    return pb, init


def burgers_exact(pb: dict, t: float) -> np.ndarray:
    """Before the shock (t < 1/pi): u = u0(xi) with x = xi + u0(xi) t, xi by
    Newton's method on the characteristics."""
    x = -1.0 + np.arange(pb["n"], dtype=np.float64) * pb["dx"]
    xi = x - 0.5 * t
    for _ in range(60):
        f = xi + (0.5 + np.sin(np.pi * xi)) * t - x
        df = 1.0 + np.pi * np.cos(np.pi * xi) * t
        xi = xi - f / df
    return (0.5 + np.sin(np.pi * xi))[None, :]


# --------------------------------------------------------------------------
# Reacting Navier-Stokes, two species, one-step Arrhenius
# (gamma = 1.4, Ea/(R T0) = 20, q/(cp T0) = 5, Pr = 0.7, Le = 1,
# N = 16,384, 256 PEs of 64, 6th-order central + AT6, RK4, delays on {0..4}).
# --------------------------------------------------------------------------
RNS_GAMMA = 1.4
RNS_MU = 0.5
RNS_PR = 0.7
RNS_LE = 1.0
RNS_A = 0.5
RNS_EA = 20.0
RNS_DT = 0.003  # AT6 with k <= 4 and RK4 is stable to a diffusion number of about 0.02


def rns_prm(gamma=RNS_GAMMA, mu=RNS_MU, Pr=RNS_PR, Le=RNS_LE, A=RNS_A, Ea=RNS_EA, heat=5.0):
    cp = gamma / (gamma - 1.0)
    return [gamma, mu, Pr, Le, A, Ea, heat * cp]


def rns_conserved(rho, u, T, Y, prm) -> np.ndarray:
    """(rho, rho u, rho E, rho Y) with rho E = p/(gamma-1) + rho u^2/2 + q_c rho Y."""
    gamma, qc = prm[0], prm[6]
    p = rho * T
    rhoE = p / (gamma - 1.0) + 0.5 * rho * u * u + qc * rho * Y
    return np.stack([rho, rho * u, rhoE, rho * Y]).astype(np.float64)


def rns(case="flame", n=16384, pe_size=64, order=6, mode="at", k_max=4, dist="uniform", prob=(),
        seed=0, per_stage=1, dt=RNS_DT, T_init=3.0, Y_init=1.0, prm=None, T_unburnt=1.0, instance=0,
        form="flux"):
    """Premixed flame from a periodic double-tanh burnt region in unburnt gas
    at ``T_unburnt``, or homogeneous autoignition at ``T_init`` with a 1 %
    Gaussian temperature bump.  ``form`` = "flux" differentiates the flux
    vector (conservative); "chain" expands the product derivatives by the
    chain rule and differentiates the primitives (Sec. 4)."""
    prm = list(prm) if prm is not None else rns_prm()
    dx = 1.0
    x = np.arange(n, dtype=np.float64) * dx
    L = n * dx
    gamma, qc = prm[0], prm[6]
    cp = gamma / (gamma - 1.0)
    if case == "flame":
        w = 10.0 * dx
        s = 0.5 * (np.tanh((x - 0.375 * L) / w) - np.tanh((x - 0.625 * L) / w))
        T = T_unburnt + (qc / cp) * Y_init * s
        Y = Y_init * (1.0 - s)
    elif case == "ignition":
        sig = 0.05 * L
        T = T_init * (1.0 + 0.01 * np.exp(-((x - 0.5 * L) / sig) ** 2))
        Y = np.full(n, Y_init)
    else:
        raise ValueError(case)
    p = np.ones(n)
    rho = p / T
    u = np.zeros(n)
    init = rns_conserved(rho, u, T, Y, prm)
    if form not in ("flux", "chain"):
        raise ValueError(form)
    pb = base_problem(pde="rns" if form == "flux" else "rns_chain", order=order, rk="rk4", n=n,
                      pe_size=pe_size, dx=dx, dt=dt,
                      prm=prm, mode=mode, k_max=k_max, dist=dist, prob=list(prob), seed=seed,
                      per_stage=per_stage, instance=instance)
    return pb, init


# --------------------------------------------------------------------------
# Reactive Euler detonation (gamma = 1.2, Q = 50, Ea = 50, overdrive 1.6),
# half-reaction length resolved by 20 points, WENO5 + AT-WENO5, RK3-TVD,
# PE size 1024, delays geometric (p = 0.5) on {0..4}.
# --------------------------------------------------------------------------
DET_GAMMA = 1.2
DET_Q = 50.0
DET_EA = 50.0
DET_F = 1.6
DET_EPS = 1e-6


def _det_speed(gamma=DET_GAMMA, Q=DET_Q, f=DET_F):
    g = (gamma * gamma - 1.0) * Q / 2.0
    d_cj = math.sqrt(gamma + g) + math.sqrt(g)
    return math.sqrt(f) * d_cj


def _vn_state(D, gamma=DET_GAMMA):
    """Von Neumann (post-shock, unreacted) state of a shock at speed D into
    rho = p = 1 at rest (Rankine-Hugoniot)."""
    c0 = math.sqrt(gamma)
    M2 = (D / c0) ** 2
    rho = (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    p = 1.0 + 2.0 * gamma / (gamma + 1.0) * (M2 - 1.0)
    u = D * (1.0 - 1.0 / rho)
    return rho, u, p


def _znd_volume(D, lam, gamma=DET_GAMMA, Q=DET_Q):
    """Specific volume on the strong branch of the Rayleigh line at reaction
    progress lam (steady ZND structure, shock frame)."""
    g1 = gamma / (gamma - 1.0)
    # g1 (1 + D^2 - D^2 v) v + D^2 v^2 / 2 = g1 + D^2/2 + Q lam
    a = D * D / 2.0 - g1 * D * D
    b = g1 * (1.0 + D * D)
    c = -(g1 + D * D / 2.0 + Q * lam)
    disc = max(b * b - 4.0 * a * c, 0.0)
    r1 = (-b + math.sqrt(disc)) / (2.0 * a)
    r2 = (-b - math.sqrt(disc)) / (2.0 * a)
    return min(r for r in (r1, r2) if r > 0.0)


@lru_cache(maxsize=None)
def det_rate_constant(half_length=1.0, gamma=DET_GAMMA, Q=DET_Q, Ea=DET_EA, f=DET_F) -> float:
    """Pre-exponential A that puts the ZND half-reaction point at
    ``half_length`` behind the shock (setup only; midpoint quadrature)."""
    D = _det_speed(gamma, Q, f)
    m = 20000
    total = 0.0
    for i in range(m):
        lam = (i + 0.5) * 0.5 / m
        v = _znd_volume(D, lam, gamma, Q)
        p = 1.0 + D * D * (1.0 - v)
        T = p * v
        w = D * v
        total += w / ((1.0 - lam) * math.exp(-Ea / T)) * (0.5 / m)
    return total / half_length


def det_prm(gamma=DET_GAMMA, Q=DET_Q, Ea=DET_EA, f=DET_F, eps=DET_EPS):
    return [gamma, det_rate_constant(1.0, gamma, Q, Ea, f), Ea, Q, eps]


def euler_conserved(rho, u, p, Y, prm) -> np.ndarray:
    gamma, Q = prm[0], prm[3]
    rhoE = p / (gamma - 1.0) + 0.5 * rho * u * u + Q * rho * Y
    return np.stack([rho, rho * u, rhoE, rho * Y]).astype(np.float64)


def detonation(n=1 << 24, pe_size=1024, mode="at", k_max=4, dist="geometric", prob=(0.5,), seed=0,
               per_stage=1, cfl=0.5, slab=20.0, dt=None, edge_points=5.0, weno="reconstruct"):
    """Slab of von Neumann state over ``slab`` half-reaction lengths (from
    x = 1 to x = 1 + slab) in unburnt gas (rho = p = 1, u = 0, Y = 1);
    periodic.  The slab edges are tanh ramps ``edge_points`` cells wide: the
    shock steepens by itself within a few steps, and a ramp instead of a jump
    keeps the WENO weights of the first steps away from their most
    round-off-sensitive regime."""
    prm = det_prm()
    dx = 1.0 / 20.0
    D = _det_speed()
    rho_s, u_s, p_s = _vn_state(D)
    x = (np.arange(n, dtype=np.float64) + 0.5) * dx
    w = edge_points * dx
    s = 0.5 * (np.tanh((x - 1.0) / w) - np.tanh((x - 1.0 - slab) / w))
    rho = 1.0 + (rho_s - 1.0) * s
    u = u_s * s
    p = 1.0 + (p_s - 1.0) * s
    Y = np.ones(n)
    init = euler_conserved(rho, u, p, Y, prm)
    if dt is None:
        smax = max(abs(u_s) + math.sqrt(DET_GAMMA * p_s / rho_s), math.sqrt(DET_GAMMA))
        dt = cfl * dx / smax
    pb = base_problem(pde="euler", rk="rk3tvd", n=n, pe_size=pe_size, dx=dx, dt=dt, prm=prm,
                      mode=mode, k_max=k_max, dist=dist, prob=list(prob), seed=seed,
                      per_stage=per_stage, weno=weno)
    return pb, init


def entropy_wave(n=256, pe_size=32, mode="sync", k_max=1, dist="uniform", prob=(), seed=0,
                 u0=1.0, amp=0.2, dt=None, rk="rk3tvd", dt_coef=None, weno="reconstruct"):
    """Reactive-Euler density wave at constant u and p with no fuel: the exact
    solution is rho0(x - u0 t); x in [0, 1)."""
    prm = [DET_GAMMA, 0.0, DET_EA, DET_Q, DET_EPS]
    dx = 1.0 / n
    x = np.arange(n, dtype=np.float64) * dx
    rho = 1.0 + amp * np.sin(2 * np.pi * x)
    init = euler_conserved(rho, np.full(n, u0), np.ones(n), np.zeros(n), prm)
    if dt is None:
        dt = dt_coef * dx * dx if dt_coef is not None else 0.4 * dx / (u0 + math.sqrt(DET_GAMMA / (1 - amp)))
    pb = base_problem(pde="euler", rk=rk, n=n, pe_size=pe_size, dx=dx, dt=dt, prm=prm, mode=mode,
                      k_max=k_max, dist=dist, prob=list(prob), seed=seed, weno=weno)
    return pb, init


# --------------------------------------------------------------------------
# Batched reacting instances: N log-uniform in [256, 8192], initial (unburnt)
# temperature uniform in [900, 1400] K-equivalent (T / 300 K), equivalence
# ratio uniform in [0.5, 1.5] (initial fuel fraction 0.5 * phi), PE size in
# {32, 64}, largest delay in {2, 3, 4}, half flames and half ignitions.
# --------------------------------------------------------------------------
def batched_rns(count=4096, seed=0, nsteps=100, dt=0.002, n_min=256, n_max=8192):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        B = int(rng.choice([32, 64]))
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) / B)) * B
        n = max(n, 4 * B)
        T0 = float(rng.uniform(900.0, 1400.0)) / 300.0
        phi = float(rng.uniform(0.5, 1.5))
        k_max = int(rng.choice([2, 3, 4]))
        case = "flame" if i % 2 == 0 else "ignition"
        pb, init = rns(case=case, n=n, pe_size=B, mode="at", k_max=k_max, seed=seed * 1000003 + i, dt=dt,
                       T_init=T0, T_unburnt=T0, Y_init=0.5 * phi, instance=i)
        out.append((pb, init, nsteps))
    return out


# --------------------------------------------------------------------------
# Served requests: a Poisson stream mixing the advection-diffusion, reacting
# N-S and detonation problem types, N log-uniform in [512, 262,144], step
# counts uniform in [100, 5,000], a seed per request.
# --------------------------------------------------------------------------
def serving_request(kind: str, n: int, seed: int, instance: int):
    if kind == "advdiff":
        B = 64
        n = max(2 * B, (n // B) * B)
        pb, init = advdiff(n=n, pe_size=B, mode="at", k_max=3, seed=seed, cfl=0.075)
    elif kind == "rns":
        B = 64
        n = max(4 * B, (n // B) * B)
        pb, init = rns(case="flame" if seed % 2 == 0 else "ignition", n=n, pe_size=B, mode="at", k_max=4,
                       seed=seed, dt=0.003)
    else:
        B = 512
        n = max(2 * B, (n // B) * B)
        pb, init = detonation(n=n, pe_size=B, mode="at", k_max=4, seed=seed)
    return dict(pb, instance=instance), init


def serving_stream(rate=2000.0, duration=10.0, seed=0, n_min=512, n_max=262144, steps_min=100, steps_max=5000,
                   max_requests=None):
    """Arrival times (seconds from 0) and request descriptions; the initial
    states are made when a request is admitted (``serving_request``)."""
    rng = np.random.default_rng(seed)
    out, t, i = [], 0.0, 0
    kinds = ("advdiff", "rns", "detonation")
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t > duration or (max_requests is not None and i >= max_requests):
            break
        kind = kinds[int(rng.integers(3))]
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        steps = int(rng.integers(steps_min, steps_max + 1))
        out.append({"id": i, "arrival": t, "kind": kind, "n": n, "steps": steps, "seed": int(seed * 1000003 + i)})
        i += 1
    return out


def config_names():
    """The named benchmark configurations of configs.json (next to this file)."""
    return sorted(_configs())


def config(name: str):
    """Build a named configuration of configs.json: (the builder's output, the
    step count).  The output is (problem dict, initial state) for a single
    solve, a list of (problem, state, steps) for the batched one and a list
    of requests for the serving stream."""
    c = _configs()[name]
    return globals()[c["builder"]](**c["kwargs"]), c["steps"]


@lru_cache(maxsize=1)
def _configs():
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs.json")) as f:
        return json.load(f)
