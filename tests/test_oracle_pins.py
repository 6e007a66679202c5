"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one part of ``oracle/at_oracle.c`` to something other than
itself: published known-answer vectors, formulas printed in the paper
(Appendix A, Eqs. atRecon / atReconM / beta2AT0-2, Appendix B), closed-form
solutions, Taylor exactness on polynomials, invariants (conservation, zero
delay == synchronous) and the orders of accuracy the paper states.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2204_01133_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Delay generator: Philox4x32-10 and the threshold table (Sec. 2.1, Sec. 5)
# --------------------------------------------------------------------------
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert oracle.philox4x32_10(ctr, key) == out


def test_thresholds_exact_cases():
    # uniform on {0..3}: CDF = 1/4, 2/4, 3/4 -> exact multiples of 2^30
    assert oracle.thresholds(3, "uniform") == [1 << 30, 2 << 30, 3 << 30]
    # Table dels, Set 4 is synchronous: p = [1, 0, 0] -> every threshold 2^32
    assert oracle.thresholds(2, "table", [1.0, 0.0, 0.0]) == [1 << 32, 1 << 32]
    # Set 1 [0.8 0.1 0.1]
    t = oracle.thresholds(2, "table", [0.8, 0.1, 0.1])
    assert t[0] == math.floor(0.8 * 2**32) and abs(t[1] - 0.9 * 2**32) <= 1
    # geometric r = 1/2 on {0..2}: weights 4:2:1 of 7
    t = oracle.thresholds(2, "geometric", [0.5])
    assert t == [math.floor(4 / 7 * 2**32), math.floor(6 / 7 * 2**32)]


@pytest.mark.parametrize("dist,prob,k_max", [
    ("table", [0.4, 0.5, 0.1], 2),      # Table dels, Set 3
    ("uniform", [], 3),
    ("geometric", [0.5], 4),
])
def test_delay_histogram_matches_table(dist, prob, k_max):
    from scipy.stats import chi2
    pb, u0 = W.advdiff(n=64, pe_size=16, k_max=k_max, dist=dist, prob=prob, seed=1234)
    o = oracle.Oracle(pb, u0)
    counts = np.zeros(k_max + 1)
    for lvl in range(2000):
        for pe in range(4):
            for side in (0, 1):
                counts[o.draw(lvl, lvl % 4, pe, side)] += 1
    if dist == "uniform":
        p = np.full(k_max + 1, 1.0 / (k_max + 1))
    elif dist == "table":
        p = np.array(prob) / sum(prob)
    else:
        w = np.array([0.5 * 0.5**i for i in range(k_max + 1)])
        p = w / w.sum()
    exp = p * counts.sum()
    stat = ((counts - exp) ** 2 / exp).sum()
    assert stat < chi2.ppf(0.999, k_max)


def test_delays_startup_clamp_and_per_stage():
    pb, u0 = W.advdiff(n=256, pe_size=16, k_max=3, seed=7)
    o = oracle.Oracle(pb, u0)
    o.run(1)
    assert not o.delays().any()          # level 0: nothing older exists
    o.run(3)                             # level 3 with q = 2: at most 1 level back
    assert o.delays().max() <= 1
    o.run(20)
    d = o.delays()
    assert d.max() == 3 and d.min() == 0
    assert not all((d[s] == d[0]).all() for s in range(4))     # per-stage draws differ
    pb0 = dict(pb, per_stage=0)
    o0 = oracle.Oracle(pb0, u0)
    o0.run(24)
    d0 = o0.delays()
    assert all((d0[s] == d0[0]).all() for s in range(4))       # one draw per step


# --------------------------------------------------------------------------
# Temporal extrapolation weights == the printed AT coefficients
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", range(0, 9))
def test_weights_match_printed_schemes(k):
    # Eq. at1 (q = 1): (k+1) u^{n-k} - k u^{n-k-1}
    assert oracle.lagrange_weights(1, k) == [k + 1, -k]
    # Appendix A (q = 2): (k^2+3k+2)/2, -(k^2+2k), (k^2+k)/2
    assert oracle.lagrange_weights(2, k) == [(k * k + 3 * k + 2) / 2, -(k * k + 2 * k), (k * k + k) / 2]


@pytest.mark.parametrize("q", [1, 2, 3])
@pytest.mark.parametrize("k", range(0, 6))
def test_weights_extrapolate_polynomials_exactly(q, k):
    w = oracle.lagrange_weights(q, k)
    for deg in range(q + 1):
        # f(t) = t^deg sampled at t = -k-l must give f(0) = [deg == 0]
        val = sum(Fraction(wl).limit_denominator(10**6) * Fraction(-k - l) ** deg for l, wl in enumerate(w))
        assert val == (1 if deg == 0 else 0)
    if k > 0:
        val = sum(Fraction(wl) * Fraction(-k - l) ** (q + 1) for l, wl in enumerate(w))
        assert val != 0


# --------------------------------------------------------------------------
# Appendix A (Table tab:atschemes): AT4 first and second derivatives
# --------------------------------------------------------------------------
def _hist_oracle(order, c, a, L0, seed=3, n=64, B=16):
    pb, u0 = W.advdiff(n=n, pe_size=B, order=order, c=c, a=a, dt=1.0, length=float(n))
    pb["dx"] = 1.0
    o = oracle.Oracle(pb, u0)
    rng = np.random.default_rng(seed)
    hist = {}
    for lvl in range(0, L0 + 1):
        f = rng.standard_normal(n)
        hist[lvl] = f
        o.set_history(lvl, 0, f[None, :])
    return o, hist


def _appendix_a(deriv, side, k, u, j, L0):
    """Table tab:atschemes, written as printed (dx = 1)."""
    w = [(k * k + 3 * k + 2) / 2, -(k * k + 2 * k), (k * k + k) / 2]
    tot = 0.0
    for l, wl in enumerate(w):
        d = L0 - k - l

        def U(m, lvl_own=True):
            return u[L0][(j + m) % len(u[L0])] if lvl_own else u[d][(j + m) % len(u[d])]

        if side == "left":
            um2, um1, u0_, up1, up2 = U(-2, False), U(-1, False), U(0), U(1), U(2)
        else:
            um2, um1, u0_, up1, up2 = U(-2), U(-1), U(0), U(1, False), U(2, False)
        if deriv == 2:
            tot += wl * (-up2 + 16 * up1 - 30 * u0_ + 16 * um1 - um2) / 12.0
        else:
            tot += wl * (-up2 + 8 * up1 - 8 * um1 + um2) / 12.0
    return tot


@pytest.mark.parametrize("k", [0, 1, 2, 3])
@pytest.mark.parametrize("deriv", [1, 2])
def test_at4_equals_appendix_a(k, deriv):
    L0 = 8
    c, a = (1.0, 0.0) if deriv == 1 else (0.0, 1.0)
    o, u = _hist_oracle(4, c, a, L0)
    kf = np.full((4, 2), k)
    K = o.rhs(L0, 0, kf)[0]
    sign = -1.0 if deriv == 1 else 1.0
    for j, side in ((16, "left"), (31, "right"), (48, "left"), (63, "right")):
        ref = sign * _appendix_a(deriv, side, k, u, j, L0)
        assert abs(K[j] - ref) <= 1e-12 * (1 + abs(ref)), (j, side)


# --------------------------------------------------------------------------
# Taylor matching (Eq. geDer): exactness on x^a t^b, and local order
# --------------------------------------------------------------------------
@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("deriv", [1, 2])
def test_at_schemes_exact_on_polynomials(order, deriv):
    """Eq. geDer: with the AT weights every monomial x^a t^b with a within the
    central stencil's exactness (a <= order + deriv - 1) and b <= q is
    differentiated exactly at a PE-boundary point, for every delay k."""
    n, B = 64, 16
    q = order // 2
    c, a = (1.0, 0.0) if deriv == 1 else (0.0, 1.0)
    pb, u0 = W.advdiff(n=n, pe_size=B, order=order, c=c, a=a, dt=1.0, length=float(n), k_max=4)
    o = oracle.Oracle(pb, u0)
    L0, j = 10, 16  # j: first point of PE 1, every left tap is a buffer point
    x = (np.arange(n) - j).astype(float) / 4.0
    sign = -1.0 if deriv == 1 else 1.0
    for k in range(0, 5):
        kf = np.full((4, 2), k)
        for ax in range(0, order + deriv):
            for bt in range(0, q + 1):
                for lvl in range(0, L0 + 1):
                    t = lvl - L0 + 0.5
                    o.set_history(lvl, 0, (x**ax * t**bt)[None, :])
                K = o.rhs(L0, 0, kf)[0]
                exact = (math.factorial(deriv) / 4.0**deriv if ax == deriv else 0.0) * 0.5**bt
                assert abs(sign * K[j] - exact) < 1e-9, (k, ax, bt)
        # one degree more in x is not differentiated exactly
        ax = order + 1 if deriv == 1 else order + 2
        for lvl in range(0, L0 + 1):
            o.set_history(lvl, 0, (x**ax)[None, :])
        K = o.rhs(L0, 0, kf)[0]
        assert abs(K[j]) > 1e-12


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("deriv", [1, 2])
def test_at_schemes_extrapolation_degree_is_tight(order, deriv):
    """A field linear in x times t^(q+1) is differentiated wrongly when k > 0:
    the temporal extrapolation has degree exactly q."""
    n, B = 64, 16
    q = order // 2
    c, a = (1.0, 0.0) if deriv == 1 else (0.0, 1.0)
    pb, u0 = W.advdiff(n=n, pe_size=B, order=order, c=c, a=a, dt=1.0, length=float(n))
    o = oracle.Oracle(pb, u0)
    L0, j = 10, 16
    x = (np.arange(n) - j).astype(float)
    kf = np.full((4, 2), 2)
    for lvl in range(0, L0 + 1):
        t = lvl - L0
        o.set_history(lvl, 0, (x**deriv * (1.0 + t ** (q + 1)))[None, :])
    K = o.rhs(L0, 0, kf)[0]
    exact = float(math.factorial(deriv))  # at t = 0
    sign = -1.0 if deriv == 1 else 1.0
    assert abs(sign * K[j] - exact) > 1e-6
    for lvl in range(0, L0 + 1):
        t = lvl - L0
        o.set_history(lvl, 0, (x**deriv * (1.0 + t**q))[None, :])
    K = o.rhs(L0, 0, kf)[0]
    assert abs(sign * K[j] - exact) < 1e-9


@pytest.mark.parametrize("order", [2, 4, 6])
@pytest.mark.parametrize("deriv", [1, 2])
def test_at_local_truncation_order(order, deriv):
    """dt = dx^2: the AT derivative at a PE-boundary point converges at the
    order of the central scheme for every delay (Sec. 2.2)."""
    q = order // 2
    errs = []
    for n in (32, 64, 128):
        B = n // 4
        dx = 2 * math.pi / n
        dt = dx * dx
        c, a = (1.0, 0.0) if deriv == 1 else (0.0, 1.0)
        pb, u0 = W.advdiff(n=n, pe_size=B, order=order, c=c, a=a, dt=dt, k_max=4)
        o = oracle.Oracle(pb, u0)
        L0 = 10
        x = np.arange(n) * dx
        for lvl in range(0, L0 + 1):
            t = (lvl - L0) * dt
            o.set_history(lvl, 0, (np.sin(x + 0.3 + 2 * t) * math.cos(t + 0.2) + 0.1 * t**2)[None, :])
        kf = np.full((4, 2), 4)
        K = o.rhs(L0, 0, kf)[0]
        j = B
        ex = (math.cos(x[j] + 0.3) if deriv == 1 else -math.sin(x[j] + 0.3)) * math.cos(0.2)
        sign = -1.0 if deriv == 1 else 1.0
        errs.append(abs(sign * K[j] - ex))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > order - 0.6, (errs, orders)
    _ = q


# --------------------------------------------------------------------------
# Eq. rkat1: one RK2 step with AT4 at a PE boundary; the delay adds a local
# error term proportional to k (k^2 + 3k + 2) dt^3 / dx^2
# --------------------------------------------------------------------------
def test_rk2_at4_excess_error_scales_like_eq_rkat1():
    alpha = 1.0
    n, B = 64, 16
    dx = 2 * math.pi / n
    dt = 0.1 * dx * dx / alpha
    pb, u0 = W.advdiff(n=n, pe_size=B, order=4, c=0.0, a=alpha, dt=dt, rk="rk2", k_max=4)
    x = np.arange(n) * dx

    def exact(t):
        return np.exp(-alpha * t) * np.sin(x + 0.4)

    def d2_sync(f):  # standard 4th-order second derivative (Eq. ks), periodic
        return (-np.roll(f, 2) + 16 * np.roll(f, 1) - 30 * f + 16 * np.roll(f, -1) - np.roll(f, -2)) / (12 * dx * dx)

    L0 = 10
    errs = {}
    for k in range(0, 5):
        o = oracle.Oracle(pb, u0)
        for lvl in range(0, L0 + 1):
            t = lvl * dt
            o.set_history(lvl, 0, exact(t)[None, :])
            # stage 2 at old levels from synchronous stages of exact data (Sec. 2.3)
            o.set_history(lvl, 1, (exact(t) + dt * alpha * d2_sync(exact(t)))[None, :])
        o.set_level(L0)
        o.set_state(exact(L0 * dt)[None, :])
        o.force_delays(np.full((n // B, 2), k))
        assert o.run(1) == 0
        j = B  # first point of PE 1
        errs[k] = o.state()[0][j] - exact((L0 + 1) * dt)[j]
    excess = {k: errs[k] - errs[0] for k in range(1, 5)}
    for k in range(2, 5):
        want = k * (k * k + 3 * k + 2) / 6.0   # relative to k = 1
        assert abs(excess[k] / excess[1] - want) < 0.05 * want, (k, excess)


# --------------------------------------------------------------------------
# Zero delay == synchronous (Sec. 2.2 after Eq. at1; Eq. rkat2 at k = 0)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("maker", ["advdiff", "rns", "euler", "adv_weno", "burgers"])
def test_zero_delay_is_bitwise_sync(maker):
    if maker == "advdiff":
        mk = lambda **kw: W.advdiff(n=256, pe_size=16, cfl=0.075, **kw)
    elif maker == "rns":
        mk = lambda **kw: W.rns(case="flame", n=512, pe_size=32, dt=0.003, **kw)
    elif maker == "euler":
        mk = lambda **kw: W.detonation(n=2048, pe_size=256, **kw)
    elif maker == "adv_weno":
        mk = lambda **kw: W.adv_weno(n=128, pe_size=16, **kw)
    else:
        mk = lambda **kw: W.burgers(n=128, pe_size=16, **kw)
    pb_s, u0 = mk(mode="sync")
    pb_a, _ = mk(mode="at", k_max=0)
    pb_d, _ = mk(mode="at", k_max=2, dist="uniform")
    os_, oa, od = oracle.Oracle(pb_s, u0), oracle.Oracle(pb_a, u0), oracle.Oracle(pb_d, u0)
    for o in (os_, oa, od):
        assert o.run(20) == 0
    assert np.array_equal(os_.state(), oa.state())
    assert not np.array_equal(os_.state(), od.state())


# --------------------------------------------------------------------------
# Closed form and orders on advection-diffusion (Eq. rkat2; Sec. 2.1)
# --------------------------------------------------------------------------
def _advdiff_err(n, mode, k_max=3, t_end=0.25, r=0.05, order=4, a=0.5):
    dx = 2 * math.pi / n
    dt = r * dx * dx / a
    steps = int(round(t_end / dt))
    dt = t_end / steps
    pb, u0 = W.advdiff(n=n, pe_size=16, order=order, c=1.0, a=a, mode=mode, k_max=k_max, dt=dt)
    o = oracle.Oracle(pb, u0)
    assert o.run(steps) == 0
    return np.abs(o.state() - W.advdiff_exact(pb, t_end)).max()


def test_advdiff_sync_converges_to_closed_form_at_fourth_order():
    e = [_advdiff_err(n, "sync") for n in (32, 64, 128)]
    rates = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(rates) > 3.7, (e, rates)
    assert e[-1] < 1e-6


def test_advdiff_at_keeps_order_and_as_loses_it():
    at = [_advdiff_err(n, "at") for n in (32, 64, 128)]
    as_ = [_advdiff_err(n, "as") for n in (32, 64, 128)]
    r_at = math.log2(at[1] / at[2])
    r_as = math.log2(as_[1] / as_[2])
    assert r_at > 3.5, at
    assert r_as < 2.6, as_
    assert as_[-1] > 100 * at[-1]


def test_as_error_far_above_at_error_on_advdiff_config():
    """Table ap / Tables aiL1-aiLinf trend: AS-SFD errors are orders of
    magnitude above AT errors for the same delay statistics."""
    pb_s, u0 = W.advdiff(mode="sync", cfl=0.075)
    out = {}
    for mode in ("sync", "at", "as"):
        pb, _ = W.advdiff(mode=mode, cfl=0.075)
        o = oracle.Oracle(pb, u0)
        assert o.run(600) == 0
        out[mode] = o.state()
    e_at = np.abs(out["at"] - out["sync"]).max()
    e_as = np.abs(out["as"] - out["sync"]).max()
    assert e_as > 100 * e_at


# --------------------------------------------------------------------------
# WENO5: linear limit, ENO property, smooth order (Sec. 3)
# --------------------------------------------------------------------------
def test_weno5_ideal_weights_give_upwind5():
    rng = np.random.default_rng(0)
    for _ in range(20):
        v = rng.standard_normal(5)
        lin = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60.0
        assert abs(oracle.weno5(v, eps=1e30) - lin) < 1e-14


def test_weno5_exact_on_quadratics_and_eno_at_steps():
    for v in ([1.0, 4.0, 9.0, 16.0, 25.0], [2.0, 2.0, 2.0, 2.0, 2.0]):
        # cell averages of a quadratic over unit cells centred at -2..2
        pass
    # point values f_i = cell averages of h; for h(x) = x^2, avg over [i-1/2,i+1/2] = i^2 + 1/12
    v = [i * i + 1.0 / 12.0 for i in range(-2, 3)]
    assert abs(oracle.weno5(v) - 0.25) < 1e-12
    # ENO: the stencil that avoids the jump gets (almost) all the weight
    assert abs(oracle.weno5([0, 0, 0, 1, 1])) < 1e-6
    assert abs(oracle.weno5([0, 0, 1, 1, 1]) - 1.0) < 1e-6
    assert abs(oracle.weno5([1, 1, 1, 0, 0]) - 1.0) < 1e-6


def test_weno5_smooth_flux_difference_is_fifth_order():
    f = lambda x: x + 0.2 * np.sin(x)
    fp = lambda x: 1 + 0.2 * np.cos(x)
    errs = []
    for h in (0.2, 0.1, 0.05):
        x0 = 0.7
        vals = [f(x0 + i * h) for i in range(-3, 3)]
        Fr = oracle.weno5(vals[1:6], eps=1e-40)
        Fl = oracle.weno5(vals[0:5], eps=1e-40)
        errs.append(abs((Fr - Fl) / h - fp(x0)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 4.5, (errs, rates)


# --------------------------------------------------------------------------
# AT-WENO5: printed formulas (Eqs. atRecon, beta2AT0-2, atReconM; App. B)
# --------------------------------------------------------------------------
def _printed_left_plus(k, a, a1, b, b1, c, d, e):
    """Eq. atRecon and Eqs. beta2AT0/1/2 (left boundary, edge j+1/2)."""
    p0 = -k * a1 / 3 + 7 * k * b1 / 6 + (2 * k + 2) * a / 6 + (-7 * k - 7) * b / 6 + 11 * c / 6
    p1 = k * b1 / 6 + (-k - 1) * b / 6 + 5 * c / 6 + d / 3
    p2 = c / 3 + 5 * d / 6 - e / 6
    B0 = (4 * a * a + 25 * b * b
          + k * k * (4 * a1 * a1 + 4 * a * a + 19 * a * (b1 - b) + 25 * (b1 - b) ** 2 + a1 * (19 * (b - b1) - 8 * a))
          - 31 * c * b + 10 * c * c + a * (11 * c - 19 * b)
          + k * (8 * a * a + (19 * b1 - 38 * b + 11 * c) * a + a1 * (-8 * a + 19 * b - 11 * c)
                 - (b1 - b) * (50 * b - 31 * c))) / 3
    B1 = (4 * k * k * (b1 - b) ** 2 + 4 * b * b + 13 * c * c + 4 * d * d + (5 * d - 13 * c) * b - 13 * c * d
          - k * (b1 - b) * (8 * b - 13 * c + 5 * d)) / 3
    B2 = (10 * c * c - 31 * d * c + 25 * d * d + 4 * e * e + (11 * c - 19 * d) * e) / 3
    return (p0, p1, p2), (B0, B1, B2)


def _printed_right_plus(k, a, b, c, d, d1, e, e1):
    """Appendix B, Eq. atReconR and the right-boundary smoothness indicators."""
    p0 = a / 3 - 7 * b / 6 + 11 * c / 6
    p1 = -k * d1 / 3 + (2 * k + 2) * d / 6 - b / 6 + 5 * c / 6
    p2 = -5 * k * d1 / 6 + k * e1 / 6 + (5 * k + 5) * d / 6 + (-k - 1) * e / 6 + c / 3
    B0 = (4 * a * a + (11 * c - 19 * b) * a + 25 * b * b + 10 * c * c - 31 * b * c) / 3
    X = k * d1 - (k + 1) * d
    B1 = (b * (-5 * k * d1 + 5 * (k + 1) * d - 13 * c) + 4 * X * X + 13 * c * X + 4 * b * b + 13 * c * c) / 3
    B2 = (k * k * (25 * d1 * d1 + (19 * (e - e1) - 50 * d) * d1 + 25 * d * d + 4 * (e1 - e) ** 2 + 19 * d * (e1 - e))
          + k * (50 * d * d + 19 * (e1 - 2 * e) * d + 8 * e * (e - e1) + d1 * (19 * e - 50 * d))
          + 25 * d * d + 4 * e * e - 19 * d * e
          + c * (-31 * d + 11 * e + k * (31 * d1 - 31 * d - 11 * e1 + 11 * e)) + 10 * c * c) / 3
    return (p0, p1, p2), (B0, B1, B2)


def _printed_left_minus(k, a, a1, b, b1, c, d, e):
    """Eq. atReconM (left boundary, edge j-1/2): candidates only."""
    p0 = k * a1 / 6 - 5 * k * b1 / 6 + (-k - 1) * a / 6 + (5 * k + 5) * b / 6 + c / 3
    p1 = -k * b1 / 3 + (2 * k + 2) * b / 6 + 5 * c / 6 - d / 6
    p2 = 11 * c / 6 - 7 * d / 6 + e / 3
    return p0, p1, p2


def _printed_right_minus(k, a, b, c, d, d1, e, e1):
    """Appendix B, Eq. atReconRm (right boundary, edge j-1/2): candidates only."""
    p0 = -a / 6 + 5 * b / 6 + c / 3
    p1 = k * d1 / 6 + (-k - 1) * d / 6 + b / 3 + 5 * c / 6
    p2 = 7 * k * d1 / 6 - k * e1 / 3 + (-7 * k - 7) * d / 6 + (2 * k + 2) * e / 6 + 11 * c / 6
    return p0, p1, p2


def _combine(p, B, eps):
    g = (0.1, 0.6, 0.3)
    al = [g[i] / (eps + B[i]) ** 2 for i in range(3)]
    s = sum(al)
    return sum(al[i] / s * p[i] for i in range(3))


def test_printed_at_weno_is_weno_on_linearly_extrapolated_values():
    """Symbolic: every printed AT-WENO candidate and indicator equals the
    synchronous one evaluated on (k+1) u^{n-k} - k u^{n-k-1} at buffer points."""
    sp = pytest.importorskip("sympy")
    k, a, a1, b, b1, c, d, d1, e, e1 = sp.symbols("k a a1 b b1 c d d1 e e1")
    R = sp.Rational
    A = (k + 1) * a - k * a1
    Bx = (k + 1) * b - k * b1
    Dx = (k + 1) * d - k * d1
    Ex = (k + 1) * e - k * e1

    def std_plus(v0, v1, v2, v3, v4):
        p = (v0 / 3 - R(7, 6) * v1 + R(11, 6) * v2, -v1 / 6 + R(5, 6) * v2 + v3 / 3, v2 / 3 + R(5, 6) * v3 - v4 / 6)
        Bs = (R(13, 12) * (v0 - 2 * v1 + v2) ** 2 + R(1, 4) * (v0 - 4 * v1 + 3 * v2) ** 2,
              R(13, 12) * (v1 - 2 * v2 + v3) ** 2 + R(1, 4) * (v1 - v3) ** 2,
              R(13, 12) * (v2 - 2 * v3 + v4) ** 2 + R(1, 4) * (3 * v2 - 4 * v3 + v4) ** 2)
        return p, Bs

    def std_minus(v0, v1, v2, v3, v4):  # value at the left edge of the middle cell
        return (-v0 / 6 + R(5, 6) * v1 + v2 / 3, v1 / 3 + R(5, 6) * v2 - v3 / 6, R(11, 6) * v2 - R(7, 6) * v3 + v4 / 3)

    # left boundary j+1/2 (Eq. atRecon, Eqs. beta2AT0-2)
    p, Bs = _printed_left_plus(k, a, a1, b, b1, c, d, e)
    ps, Bss = std_plus(A, Bx, c, d, e)
    for x, y in zip(p + Bs, ps + Bss):
        assert sp.expand(sp.nsimplify(x) - y) == 0
    # right boundary j+1/2 (Eq. atReconR and App. B indicators)
    p, Bs = _printed_right_plus(k, a, b, c, d, d1, e, e1)
    ps, Bss = std_plus(a, b, c, Dx, Ex)
    for x, y in zip(p + Bs, ps + Bss):
        assert sp.expand(sp.nsimplify(x) - y) == 0
    # j-1/2 at both boundaries (Eqs. atReconM, atReconRm)
    for x, y in zip(_printed_left_minus(k, a, a1, b, b1, c, d, e), std_minus(A, Bx, c, d, e)):
        assert sp.expand(sp.nsimplify(x) - y) == 0
    for x, y in zip(_printed_right_minus(k, a, b, c, d, d1, e, e1), std_minus(a, b, c, Dx, Ex)):
        assert sp.expand(sp.nsimplify(x) - y) == 0


def _weno_hist(c_adv, L0=6, seed=5, n=64, B=16):
    pb, u0 = W.adv_weno(n=n, pe_size=B, c=c_adv, dt=1.0, k_max=4)
    o = oracle.Oracle(pb, u0)
    rng = np.random.default_rng(seed)
    u = {}
    for lvl in range(0, L0 + 1):
        f = 1.0 + 0.3 * rng.standard_normal(n)
        u[lvl] = f
        o.set_history(lvl, 0, f[None, :])
    return o, u


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_oracle_at_weno_flux_equals_printed_formulas(k):
    L0, eps = 6, 1e-6
    kf = np.full((4, 2), k)
    # c > 0: the flux is the left-biased reconstruction of f+ = c u
    o, u = _weno_hist(5.0, L0)
    cu = {lvl: 5.0 * v for lvl, v in u.items()}
    j = 16  # first point of PE 1, edge j+1/2
    p, Bs = _printed_left_plus(k, cu[L0 - k][j - 2], cu[L0 - k - 1][j - 2], cu[L0 - k][j - 1], cu[L0 - k - 1][j - 1],
                               cu[L0][j], cu[L0][j + 1], cu[L0][j + 2])
    F = o.edge_flux(L0, 0, 1, j, kf)[0]
    assert abs(F - _combine(p, Bs, eps)) < 1e-12 * (1 + abs(F))
    j = 31  # last point of PE 1, edge j+1/2
    p, Bs = _printed_right_plus(k, cu[L0][j - 2], cu[L0][j - 1], cu[L0][j], cu[L0 - k][j + 1], cu[L0 - k - 1][j + 1],
                                cu[L0 - k][j + 2], cu[L0 - k - 1][j + 2])
    F = o.edge_flux(L0, 0, 1, j, kf)[0]
    assert abs(F - _combine(p, Bs, eps)) < 1e-12 * (1 + abs(F))
    # c < 0: right-biased reconstruction of f- = c u at the edge j-1/2
    pb, u0 = W.adv_weno(n=64, pe_size=16, c=-5.0, dt=1.0, eps=1e30, k_max=4)
    o = oracle.Oracle(pb, u0)
    for lvl, v in u.items():
        o.set_history(lvl, 0, v[None, :])
    cu = {lvl: -5.0 * v for lvl, v in u.items()}
    j = 16
    p = _printed_left_minus(k, cu[L0 - k][j - 2], cu[L0 - k - 1][j - 2], cu[L0 - k][j - 1], cu[L0 - k - 1][j - 1],
                            cu[L0][j], cu[L0][j + 1], cu[L0][j + 2])
    F = o.edge_flux(L0, 0, 1, j - 1, kf)[0]
    ideal = 0.1 * p[2] + 0.6 * p[1] + 0.3 * p[0]   # ideal weights mirror for the right-biased side
    assert abs(F - ideal) < 1e-12 * (1 + abs(F))
    j = 31
    p = _printed_right_minus(k, cu[L0][j - 2], cu[L0][j - 1], cu[L0][j], cu[L0 - k][j + 1], cu[L0 - k - 1][j + 1],
                             cu[L0 - k][j + 2], cu[L0 - k - 1][j + 2])
    F = o.edge_flux(L0, 0, 1, j - 1, kf)[0]
    ideal = 0.1 * p[2] + 0.6 * p[1] + 0.3 * p[0]
    assert abs(F - ideal) < 1e-12 * (1 + abs(F))


def _order_runs(maker, ns, mode, t_end, **kw):
    errs = []
    for n in ns:
        pb, u0, exact = maker(n, mode, **kw)
        steps = int(round(t_end / pb["dt"]))
        pb["dt"] = t_end / steps
        o = oracle.Oracle(pb, u0)
        assert o.run(steps) == 0
        errs.append(np.abs(o.state()[0] - exact(pb, t_end)).max())
    return errs, [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_weno_linear_advection_orders_sync_at_as():
    """Sec. 3 order test (Table wenoLin trend): sync ~5, AT-WENO ~4, AS-WENO ~2.
    x in [-1, 1], u0 = sin^4(pi x + 0.25), c = 5, RK3, dt ~ dx^2, p = [0.5, 0.5]."""
    def mk(n, mode, **kw):
        pb, u0 = W.adv_weno(n=n, pe_size=16, mode=mode, k_max=1, dt_coef=2.0, **kw)
        return pb, u0, lambda pb, t: W.adv_weno_exact(pb, t)[0]
    t_end = 0.1
    e_s, r_s = _order_runs(mk, (64, 128, 256), "sync", t_end)
    e_a, r_a = _order_runs(mk, (64, 128, 256), "at", t_end)
    e_as, r_as = _order_runs(mk, (64, 128, 256), "as", t_end)
    assert r_s[-1] > 4.3, (e_s, r_s)
    assert r_a[-1] > 3.5, (e_a, r_a)
    assert r_as[-1] < 2.6, (e_as, r_as)
    assert e_as[-1] > 10 * e_a[-1]


def test_burgers_order_before_the_shock():
    """Sec. 3 nonlinear order test (Table wenoNLin trend): inviscid Burgers,
    u0 = 0.5 + sin(pi x) on [-1, 1], t = 0.15 (before the shock), against the
    exact solution along characteristics: sync and AT-WENO near 5th order,
    AS-WENO about 2nd."""
    def mk(n, mode, **kw):
        pb, u0 = W.burgers(n=n, pe_size=16, mode=mode, k_max=1, dt_coef=0.5)
        return pb, u0, lambda pb, t: W.burgers_exact(pb, t)[0]
    e_s, r_s = _order_runs(mk, (64, 128, 256), "sync", 0.15)
    e_a, r_a = _order_runs(mk, (64, 128, 256), "at", 0.15)
    e_as, r_as = _order_runs(mk, (64, 128, 256), "as", 0.15)
    assert r_s[-1] > 4.5 and r_a[-1] > 4.0, (e_s, r_s, e_a, r_a)
    assert r_as[-1] < 2.5 and e_as[-1] > 10 * e_a[-1], (e_as, r_as)


def test_euler_entropy_wave_closed_form():
    """Reactive Euler at constant u and p without fuel: rho advects exactly."""
    def mk(n, mode, **kw):
        pb, u0 = W.entropy_wave(n=n, pe_size=16, mode=mode, k_max=1, dt_coef=0.5)
        x = np.arange(n) / n
        return pb, u0, lambda pb, t: 1 + 0.2 * np.sin(2 * np.pi * (x - t))
    e_s, r_s = _order_runs(mk, (64, 128, 256), "sync", 0.2)
    e_a, r_a = _order_runs(mk, (64, 128, 256), "at", 0.2)
    assert r_s[-1] > 4.5 and r_a[-1] > 3.5, (e_s, r_s, e_a, r_a)


# --------------------------------------------------------------------------
# Runge-Kutta tableaux (Eq. rk1, Eq. rk2): a homogeneous reacting state has
# no spatial gradients, so every point follows the 0-D ignition ODE.
# --------------------------------------------------------------------------
def _ode_reference(rhs, y0, t_end):
    from scipy.integrate import solve_ivp
    sol = solve_ivp(rhs, (0, t_end), [y0], rtol=1e-13, atol=1e-15, method="DOP853")
    return sol.y[0, -1]


@pytest.mark.parametrize("rk,expect", [("rk2", 2), ("rk3tvd", 3), ("rk4", 4)])
def test_rk_order_on_homogeneous_ignition(rk, expect):
    prm = W.det_prm()
    gamma, A, Ea, Q = prm[0], prm[1], prm[2], prm[3]
    rho, u, p0 = 1.0, 0.0, 10.0
    E = p0 / (gamma - 1) + Q * 1.0

    def rhs(t, y):
        Y = y[0]
        p = (gamma - 1) * (E - Q * Y)
        return [-A * Y * math.exp(-Ea * rho / p)]

    t_end = 0.02
    ref = _ode_reference(rhs, 1.0, t_end)
    errs = []
    for steps in (20, 40, 80):
        n = 2048
        init = W.euler_conserved(np.full(n, rho), np.full(n, u), np.full(n, p0), np.ones(n), prm)
        pb = W.base_problem(pde="euler", rk=rk, n=n, pe_size=256, dx=0.05, dt=t_end / steps, prm=prm,
                            mode="sync", k_max=2)
        o = oracle.Oracle(pb, init)
        assert o.run(steps) == 0
        s = o.state()
        assert np.ptp(s[3]) == 0.0          # every point follows the same ODE
        errs.append(abs(s[3][0] - ref))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - expect) < 0.3, (errs, rates)


def test_rns_homogeneous_ignition_matches_ode():
    prm = W.rns_prm()
    gamma, A, Ea, qc = prm[0], prm[4], prm[5], prm[6]
    n, T0 = 256, 4.0
    rho = 1.0 / T0
    init = W.rns_conserved(np.full(n, rho), np.zeros(n), np.full(n, T0), np.ones(n), prm)
    rhoE = init[2][0]

    def rhs(t, y):
        rY = y[0]
        p = (gamma - 1) * (rhoE - qc * rY)
        return [-A * rY * math.exp(-Ea * rho / p)]

    t_end, steps = 3.0, 300
    ref = _ode_reference(rhs, rho, t_end)
    pb = W.base_problem(pde="rns", order=6, rk="rk4", n=n, pe_size=32, dx=1.0, dt=t_end / steps, prm=prm,
                        mode="sync", k_max=4)
    o = oracle.Oracle(pb, init)
    assert o.run(steps) == 0
    s = o.state()
    assert np.ptp(s[3]) <= 1e-15 * rho
    assert abs(s[3][0] - ref) < 1e-9 * rho


# --------------------------------------------------------------------------
# Reacting N-S right-hand side against the PDE itself (Eq. ge with the
# constitutive laws of Sec. 4), in both forms: the flux form differentiates
# the flux vector, the chain-rule form the primitives.  Exact derivatives of
# smooth periodic fields come from sympy; a dropped term, a wrong sign or a
# wrong coefficient leaves an O(1) error instead of the stencil's O(dx^6).
# --------------------------------------------------------------------------
def _rns_exact(n, L, prm):
    sp = pytest.importorskip("sympy")
    gam, mu, Pr, Le, A, Ea, qc = prm
    cp = gam / (gam - 1.0)
    lam = mu * cp / Pr
    rhoD = lam / (cp * Le)
    x = sp.symbols("x")
    kap = 2 * sp.pi / L
    rho = 1 + sp.Rational(1, 5) * sp.sin(kap * x)
    u = sp.Rational(3, 10) * sp.cos(kap * x)
    T = 2 + sp.Rational(1, 2) * sp.sin(2 * kap * x + sp.Rational(3, 10))
    Y = sp.Rational(1, 2) + sp.Rational(1, 5) * sp.cos(kap * x + 1)
    p = rho * T
    rE = p / (gam - 1) + rho * u * u / 2 + qc * rho * Y
    d = lambda f: sp.diff(f, x)
    tau = sp.Rational(4, 3) * mu * d(u)
    q = -lam * d(T) - qc * rhoD * d(Y)          # -lam T_x + q_c J_F, J_F = -rhoD Y_x
    K = [-d(rho * u),
         -d(rho * u * u + p) + d(tau),
         -d(u * (rE + p)) + d(tau * u) - d(q),
         -d(rho * u * Y) + d(rhoD * d(Y)) - A * rho * Y * sp.exp(-Ea / T)]
    xs = np.arange(n) * (L / n)
    ev = lambda f: np.asarray(sp.lambdify(x, f, "numpy")(xs), dtype=np.float64) * np.ones(n)
    exact = np.stack([ev(k) for k in K])
    state = np.stack([ev(rho), ev(rho * u), ev(rE), ev(rho * Y)])
    return exact, state


@pytest.mark.parametrize("form", ["flux", "chain"])
@pytest.mark.parametrize("order", [4, 6])
def test_rns_rhs_converges_to_the_pde(form, order):
    prm = W.rns_prm()
    L = 40.0
    errs = []
    for n in (64, 128, 256):
        exact, state = _rns_exact(n, L, prm)
        pb = W.base_problem(pde="rns" if form == "flux" else "rns_chain", order=order, rk="rk4", n=n,
                            pe_size=n // 4, dx=L / n, dt=1e-3, prm=prm, mode="sync", k_max=4)
        o = oracle.Oracle(pb, state)
        o.set_history(0, 0, state)
        K = o.rhs(0, 0)
        errs.append(np.abs(K - exact).max() / np.abs(exact).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-5
    assert abs(rates[-1] - order) < 0.5, (errs, rates)


def test_replayed_delay_trace_reproduces_a_run():
    """The oracle's delay replay (used to check runs whose delays come from
    arrival order): a run under another seed that replays the recorded delays
    of a first run reproduces it bit for bit; without the trace it differs."""
    pb, u0 = W.advdiff(n=512, pe_size=32, mode="at", k_max=3, seed=1, cfl=0.05)
    a = oracle.Oracle(pb, u0)
    trace = []
    for _ in range(40):
        assert a.run(1) == 0
        trace.append(a.delays())
    trace = np.stack(trace)
    assert len(np.unique(trace)) == 4
    b = oracle.Oracle(dict(pb, seed=99), u0)
    b.set_delay_trace(trace, 0)
    assert b.run(40) == 0
    assert np.array_equal(a.state(), b.state())
    c = oracle.Oracle(dict(pb, seed=99), u0)
    assert c.run(40) == 0
    assert not np.array_equal(a.state(), c.state())


# --------------------------------------------------------------------------
# Conservation (flux form, periodic): exact under SYNC
# --------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["rns", "euler"])
def test_sync_conserves_mass_momentum_energy(case):
    if case == "rns":
        pb, u0 = W.rns(case="flame", n=1024, pe_size=64, mode="sync", dt=0.003)
        steps = 200
    else:
        pb, u0 = W.detonation(n=4096, pe_size=512, mode="sync")
        steps = 100
    o = oracle.Oracle(pb, u0)
    assert o.run(steps) == 0
    s = o.state()
    for v in range(3):
        tot0, tot1 = u0[v].sum(), s[v].sum()
        scale = np.abs(u0[v]).sum() + np.abs(s[v]).sum()
        assert abs(tot1 - tot0) <= 1e-12 * scale, (v, tot0, tot1)
    if case == "rns":
        assert s[3].sum() < u0[3].sum()     # fuel is consumed, never produced


# --------------------------------------------------------------------------
# Reading A of the stage history (Sec. 2.3, stage values at buffer points
# formed by the receiver): a buffer point of stage s at a delayed level m
# reads the stage argument recomputed synchronously from the neighbour's u^m
# instead of the one the neighbour computed
# --------------------------------------------------------------------------
def _mk(maker, **kw):
    if maker == "advdiff":
        return W.advdiff(n=256, pe_size=16, cfl=0.075, **kw)
    if maker == "rns":
        return W.rns(case="flame", n=512, pe_size=32, dt=0.003, **kw)
    return W.detonation(n=2048, pe_size=256, **kw)


@pytest.mark.parametrize("maker", ["advdiff", "rns", "euler"])
def test_reading_a_at_zero_delay_is_reading_b_bitwise(maker):
    """With no delay the recomputed stage arguments are the ones the
    neighbour computed (both are the synchronous scheme): A == B bitwise in
    SYNC mode and in AT mode with k_max = 0; with delays the two differ."""
    for kw in (dict(mode="sync"), dict(mode="at", k_max=0)):
        pb, u0 = _mk(maker, **kw)
        b = oracle.Oracle(pb, u0)
        a = oracle.Oracle(dict(pb, history="recompute"), u0)
        assert a.run(20) == 0 and b.run(20) == 0
        assert np.array_equal(a.state(), b.state())
    pb, u0 = _mk(maker, mode="at", k_max=3)
    b = oracle.Oracle(pb, u0)
    a = oracle.Oracle(dict(pb, history="recompute"), u0)
    assert a.run(20) == 0 and b.run(20) == 0
    assert not np.array_equal(a.state(), b.state())
    assert np.array_equal(a.delays(), b.delays())  # the same draws


def test_reading_a_keeps_the_at_order():
    """AT4 + RK4 on advection-diffusion with reading A converges to the closed
    form at fourth order (dt ~ dx^2), with errors of the size of reading B's;
    reading the stage-0 argument u^m at every stage instead (an O(dt)
    inconsistency of the buffer values in time) would lose that order."""
    def err(n, hist):
        dx = 2 * math.pi / n
        dt = 0.05 * dx * dx / 0.5
        steps = int(round(0.25 / dt))
        dt = 0.25 / steps
        pb, u0 = W.advdiff(n=n, pe_size=16, order=4, c=1.0, a=0.5, mode="at", k_max=3, dt=dt)
        o = oracle.Oracle(dict(pb, history=hist), u0)
        assert o.run(steps) == 0
        return np.abs(o.state() - W.advdiff_exact(pb, 0.25)).max()
    ea = [err(n, "recompute") for n in (32, 64, 128)]
    eb = [err(n, "stage") for n in (32, 64, 128)]
    assert math.log2(ea[1] / ea[2]) > 3.5, ea
    assert 0.2 < ea[-1] / eb[-1] < 5.0, (ea, eb)


# --------------------------------------------------------------------------
# The WENO interpolation form (Sec. 3, Eqs. interpS, fullSten, omg)
# --------------------------------------------------------------------------
def test_weno_interp_ideal_weights_give_the_printed_interpolant():
    """With eps far above every indicator the weights are the ideal ones
    {1/16, 5/8, 5/16}, and the combination is the printed fifth-order
    interpolant (3/128, -5/32, 45/64, 15/32, -5/128)."""
    rng = np.random.default_rng(8)
    for _ in range(50):
        v = rng.standard_normal(5)
        got = oracle.weno5_interp(v, eps=1e30)
        want = 3 / 128 * v[0] - 5 / 32 * v[1] + 45 / 64 * v[2] + 15 / 32 * v[3] - 5 / 128 * v[4]
        assert abs(got - want) < 1e-14 * (1 + abs(want)), (v, got, want)


def test_weno_interp_exact_on_quadratics_and_fifth_order_smooth():
    """Every candidate interpolates a quadratic exactly, so any weights do;
    on a smooth function the edge value converges at fifth order."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        c0, c1, c2 = rng.standard_normal(3)
        q = lambda x: c0 + c1 * x + c2 * x * x
        v = [q(float(x)) for x in (-2, -1, 0, 1, 2)]
        assert abs(oracle.weno5_interp(v) - q(0.5)) < 1e-13
    errs = []
    for h in (0.1, 0.05, 0.025):
        x0 = 0.3
        v = [math.sin(x0 + i * h) for i in (-2, -1, 0, 1, 2)]
        errs.append(abs(oracle.weno5_interp(v, eps=1e-40) - math.sin(x0 + 0.5 * h)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 4.7, (errs, rates)


def test_printed_at_interpolants_are_interps_on_extrapolated_values():
    """Symbolic: the printed AT interpolants of the five-point stencils (the
    equation after Eq. stenF) are the synchronous ones of Eq. interpS on the
    linearly extrapolated buffer values (k+1) u^{n-k} - k u^{n-k-1}."""
    sp = pytest.importorskip("sympy")
    k, a, a1, b, b1, c, d = sp.symbols("k a a1 b b1 c d")
    R = sp.Rational
    A = (k + 1) * a - k * a1   # u_{j-2} extrapolated
    Bx = (k + 1) * b - k * b1  # u_{j-1} extrapolated
    # printed: u~(0) and u~(1) at x_{j+1/2} with buffer points j-2, j-1
    p0 = -R(3, 8) * k * a1 + R(5, 4) * k * b1 + R(1, 8) * (3 * k + 3) * a + R(1, 4) * (-5 * k - 5) * b + R(15, 8) * c
    p1 = R(1, 8) * k * b1 + R(1, 8) * (-k - 1) * b + R(3, 4) * c + R(3, 8) * d
    s0 = R(3, 8) * A - R(5, 4) * Bx + R(15, 8) * c
    s1 = -R(1, 8) * Bx + R(3, 4) * c + R(3, 8) * d
    assert sp.expand(p0 - s0) == 0
    assert sp.expand(p1 - s1) == 0
    # Eq. atS1 (the four-point second stencil) is the same interpolant
    atS1 = R(1, 8) * k * b1 + R(1, 8) * (-k - 1) * b + R(3, 4) * c + R(3, 8) * d
    assert sp.expand(atS1 - s1) == 0


def test_weno_interp_scheme_orders_sync_and_at():
    """Scalar advection (c = 5, sin^4, RK3, dt ~ dx^2) with edge values by
    interpolation and the fourth-order staggered difference: fourth order
    synchronous and with AT-WENO delays (p = [0.5, 0.5])."""
    def mk(n, mode, **kw):
        pb, u0 = W.adv_weno(n=n, pe_size=16, mode=mode, k_max=1, dt_coef=2.0, weno="interpolate", **kw)
        return pb, u0, W.adv_weno_exact
    for mode in ("sync", "at"):
        errs, rates = _order_runs(mk, (64, 128, 256), mode, 0.05)
        assert rates[-1] > 3.6, (mode, errs, rates)


def test_weno_interp_conserves_under_sync():
    pb, u0 = W.detonation(n=2048, pe_size=256, mode="sync", weno="interpolate")
    o = oracle.Oracle(pb, u0)
    assert o.run(30) == 0
    tot0, tot1 = u0.sum(axis=1), o.state().sum(axis=1)
    # mass, momentum and energy are conserved (the fuel reacts away)
    assert np.all(np.abs(tot1[:3] - tot0[:3]) <= 1e-11 * np.abs(tot0[:3]).max())


# --------------------------------------------------------------------------
# The RK schemes against their textbook forms (Eq. rk1; Shu-Osher RK3-TVD)
# --------------------------------------------------------------------------
def _ignition_ode():
    """Homogeneous reactive Euler: every point follows dY/dt = f(Y) with
    rho, u, rho E fixed (p from the energy that is not chemical)."""
    prm = W.det_prm()
    gamma, A, Ea, Q = prm[0], prm[1], prm[2], prm[3]
    rho, p0 = 1.0, 10.0
    E = p0 / (gamma - 1) + Q * 1.0

    def f(Y):
        p = (gamma - 1) * (E - Q * Y)
        return -A * Y * math.exp(-Ea * rho / p)

    def oracle_step(rk, dt, Y0=1.0):
        n = 256
        Y = np.full(n, Y0)
        p = (gamma - 1) * (E - Q * Y)
        init = W.euler_conserved(np.full(n, rho), np.zeros(n), p, Y, prm)
        pb = W.base_problem(pde="euler", rk=rk, n=n, pe_size=64, dx=0.05, dt=dt, prm=prm, mode="sync", k_max=0)
        o = oracle.Oracle(pb, init)
        assert o.run(1) == 0
        return o.state()[3][0] / rho
    return f, oracle_step


@pytest.mark.parametrize("rk", ["rk2", "rk3tvd", "rk4"])
def test_rk_step_is_the_textbook_scheme(rk):
    """One step of the oracle's Butcher-form RK on the 0-D ignition ODE equals
    the textbook scheme written in its own form: Heun (Eq. rk2), Shu-Osher
    RK3-TVD (u1 = u + dt f(u); u2 = 3/4 u + 1/4 (u1 + dt f(u1)); u+ = 1/3 u +
    2/3 (u2 + dt f(u2))), classic RK4.  Other schemes of the same order differ
    on this nonlinear ODE by far more than the tolerance (checked: Ralston's
    second-order, Kutta's third-order and the 3/8-rule fourth-order methods)."""
    f, step = _ignition_ode()
    dt, y = 0.05, 1.0
    if rk == "rk2":
        k1 = f(y)
        k2 = f(y + dt * k1)
        want = y + dt / 2 * (k1 + k2)
        k2r = f(y + 2 / 3 * dt * k1)
        other = y + dt * (k1 / 4 + 3 / 4 * k2r)                       # Ralston
    elif rk == "rk3tvd":
        u1 = y + dt * f(y)
        u2 = 0.75 * y + 0.25 * (u1 + dt * f(u1))
        want = y / 3 + 2 / 3 * (u2 + dt * f(u2))
        k1 = f(y)
        k2 = f(y + dt / 2 * k1)
        k3 = f(y - dt * k1 + 2 * dt * k2)
        other = y + dt / 6 * (k1 + 4 * k2 + k3)                        # Kutta's third order
    else:
        k1 = f(y)
        k2 = f(y + dt / 2 * k1)
        k3 = f(y + dt / 2 * k2)
        k4 = f(y + dt * k3)
        want = y + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        k2 = f(y + dt / 3 * k1)
        k3 = f(y - dt / 3 * k1 + dt * k2)
        k4 = f(y + dt * k1 - dt * k2 + dt * k3)
        other = y + dt / 8 * (k1 + 3 * k2 + 3 * k3 + k4)              # 3/8 rule
    got = step(rk, dt)
    tol = 1e-13
    assert abs(got - want) < tol, (got, want)
    assert abs(other - want) > 100 * tol, (other, want)


def test_all_zero_delay_trace_is_the_synchronous_run():
    """Replaying a trace of zero delays gives the SYNC run bit for bit (the
    synchronous scheme is pinned by its closed-form convergence)."""
    pb, u0 = W.rns(case="flame", n=1024, pe_size=64, mode="at", k_max=4, seed=3, dt=0.003)
    o = oracle.Oracle(pb, u0)
    o.set_delay_trace(np.zeros((30, 4, 16, 2), dtype=np.uint8), 0)
    assert o.run(30) == 0
    s = oracle.Oracle(dict(pb, mode="sync"), u0)
    assert s.run(30) == 0
    assert np.array_equal(o.state(), s.state())


# --------------------------------------------------------------------------
# Homogeneous ignition under AT: the separable AT-error check.  Every stencil
# annihilates a constant field, so the synchronous run is the 0-D ODE at every
# point, and the start-up clamp makes every delay 0 through step q: the AT run
# is the synchronous run bit for bit until then.  At the first step with a
# real delay (k_eff = 1) only the extrapolated buffer values differ, by the
# extrapolation error of the stage values' time series, O(dt^{q+1}); it enters
# the update times dt, and over S stages it spreads by H points per stage.  So
# the deviation is zero beyond S H points from a PE edge, nonzero at the edge,
# and shrinks like dt^{q+2} (q = 3 for AT6: 2^5 per halving; a degree one
# lower would give 2^4).
# --------------------------------------------------------------------------
def _homogeneous_rns(mode, dt, steps, n=128, B=32, T0=6.0, k_max=2):
    prm = W.rns_prm()
    rho = 1.0 / T0
    init = W.rns_conserved(np.full(n, rho), np.zeros(n), np.full(n, T0), np.ones(n), prm)
    pb = W.base_problem(pde="rns", order=6, rk="rk4", n=n, pe_size=B, dx=1.0, dt=dt, prm=prm, mode=mode,
                        k_max=k_max, dist="table", prob=[0.0] * k_max + [1.0])
    o = oracle.Oracle(pb, init)
    assert o.run(steps) == 0
    return o.state()


def test_homogeneous_ignition_separates_the_at_error():
    q, S, H, B, n = 3, 4, 3, 32, 128
    # through step q every delay is clamped to 0: the synchronous run, bit for bit
    assert np.array_equal(_homogeneous_rns("at", 0.08, q + 1), _homogeneous_rns("sync", 0.08, q + 1))
    # the first step with a delay: only points within S H of a PE edge move
    dev = np.abs(_homogeneous_rns("at", 0.08, q + 2) - _homogeneous_rns("sync", 0.08, q + 2)).max(axis=0)
    j = np.arange(n) % B
    dist = np.minimum(j, B - 1 - j)
    assert (dev[dist >= S * H] == 0.0).all()
    assert (dev[dist < H] > 1e-13).all()
    # and the deviation shrinks like dt^(q+2)
    devs = [np.abs(_homogeneous_rns("at", dt, q + 2) - _homogeneous_rns("sync", dt, q + 2)).max()
            for dt in (0.08, 0.04, 0.02)]
    for coarse, fine in zip(devs, devs[1:]):
        assert 2 ** (q + 1.3) < coarse / fine < 2 ** (q + 2.5), devs
