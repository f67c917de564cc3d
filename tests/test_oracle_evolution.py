"""Pins of the oracle's timestep (reading R14): accelerations taken at the
half-step drifted positions x + v dt/2, then v' = v + a dt and
x' = x + (v + v') dt/2.  That is the drift-kick-drift leapfrog; it must
reproduce a constant-acceleration parabola exactly and the leapfrog's known
discrete harmonic motion."""
import math

import numpy as np
import pytest


def _state(x, v):
    x = np.asarray(x, dtype=float)
    v = np.asarray(v, dtype=float)
    return dict(x=x[0].copy(), y=x[1].copy(), z=x[2].copy(), vx=v[0].copy(), vy=v[1].copy(), vz=v[2].copy())


def _pos(p):
    return np.stack([p["x"], p["y"], p["z"]])


def _vel(p):
    return np.stack([p["vx"], p["vy"], p["vz"]])


def test_constant_acceleration_is_a_parabola(oracle_mod):
    rng = np.random.default_rng(0)
    n = 5
    x0 = rng.random((3, n))
    v0 = rng.normal(size=(3, n))
    a = rng.normal(size=(3, n))
    dt, steps = 0.01, 200
    p = _state(x0, v0)
    for _ in range(steps):
        oracle_mod.kick_drift(p, a, dt)
    t = dt * steps
    assert np.allclose(_vel(p), v0 + a * t, rtol=0, atol=1e-12)
    assert np.allclose(_pos(p), x0 + v0 * t + 0.5 * a * t * t, rtol=0, atol=1e-12)


def test_harmonic_motion_matches_the_discrete_leapfrog(oracle_mod):
    """a = -w^2 x at the drifted position: one step is a linear map of trace
    2 cos th, cos th = 1 - (w dt)^2 / 2, and determinant 1, so the positions obey
    x_{k+1} + x_{k-1} = 2 cos(th) x_k and the map's quadratic invariant holds."""
    w, dt = 2.0, 0.05
    x0, v0 = 0.3, -0.7
    p = _state([[x0], [0.0], [0.0]], [[v0], [0.0], [0.0]])
    th = math.acos(1 - (w * dt) ** 2 / 2)
    # the map is [[a, b], [c, a]] with a = 1 - (w dt)^2/2, b = dt (1 - (w dt)^2/4),
    # c = -w^2 dt (det 1), which conserves -c x^2 + b v^2, i.e.
    # w^2 x^2 + (1 - (w dt / 2)^2) v^2
    inv = lambda x, v: w * w * x * x + (1 - (w * dt / 2) ** 2) * v * v
    I0 = inv(x0, v0)
    xs = []
    for k in range(1, 2001):
        xh = p["x"] + p["vx"] * dt / 2
        a = np.array([[-w * w * xh[0]], [0.0], [0.0]])
        oracle_mod.kick_drift(p, a, dt)
        assert inv(p["x"][0], p["vx"][0]) == pytest.approx(I0, rel=1e-12)
        xs.append(p["x"][0])
    # the discrete frequency: successive positions obey x_{k+1} + x_{k-1} = 2 cos(th) x_k
    xs = np.array(xs)
    assert np.allclose(xs[2:] + xs[:-2], 2 * math.cos(th) * xs[1:-1], rtol=0, atol=1e-12)


def test_two_body_kepler_conserves_angular_momentum(oracle_mod):
    """Point masses with Newtonian forces evaluated at the drifted positions: the
    force is central, so the map conserves the total angular momentum to
    rounding and keeps the energy bounded."""
    m = np.array([1.0, 0.1])
    a_sep = 0.3
    vrel = math.sqrt((m[0] + m[1]) / a_sep)
    x = np.array([[0.0, a_sep], [0.0, 0.0], [0.0, 0.0]])
    v = np.array([[0.0, 0.0], [-m[1] / m.sum() * vrel, m[0] / m.sum() * vrel], [0.0, 0.0]])
    x -= (x * m).sum(1, keepdims=True) / m.sum()
    p = _state(x, v)
    dt = 1e-3

    def ang(p):
        return float(np.sum(m * (p["x"] * p["vy"] - p["y"] * p["vx"])))

    def energy(p):
        d = math.dist((p["x"][0], p["y"][0], p["z"][0]), (p["x"][1], p["y"][1], p["z"][1]))
        return 0.5 * float(np.sum(m * (p["vx"] ** 2 + p["vy"] ** 2 + p["vz"] ** 2))) - m[0] * m[1] / d

    L0, E0 = ang(p), energy(p)
    for _ in range(3000):
        xh = _pos(p) + _vel(p) * dt / 2
        d = xh[:, 1] - xh[:, 0]
        r3 = np.linalg.norm(d) ** 3
        acc = np.stack([m[1] * d / r3, -m[0] * d / r3], axis=1)
        oracle_mod.kick_drift(p, acc, dt)
    assert ang(p) == pytest.approx(L0, rel=1e-12)
    assert energy(p) == pytest.approx(E0, rel=1e-5)
    sep = math.dist((p["x"][0], p["y"][0]), (p["x"][1], p["y"][1]))
    assert sep == pytest.approx(a_sep, rel=1e-4)


def test_self_force_without_subcycling_is_at_rounding_level(oracle_mod):
    """Sec. 3.1, first case: one particle (m = 1) from (0.15, 0.15, 0.15) with
    v = (1, 1, 1) crosses the Fig. 1 hierarchy (16^3 isolated root, three static
    levels) to t = 0.4 at dt = 3e-3 for every level.  The paper finds the
    velocity error |v - v0| / |v0| at about 1e-14: the solver adds no self-force.
    A sign or index slip in the level carry, the Green's function split or the
    TSC weights would leave an O(1) self-force on the refined levels."""
    import apm_inputs as W
    grids = [oracle_mod.Grid(*g) for g in W.grids_from_bounds(16, W.FIG1_BOUNDS)]
    cfg = oracle_mod.Config(periodic=False)
    p = dict(x=np.array([0.15]), y=np.array([0.15]), z=np.array([0.15]), vx=np.array([1.0]),
             vy=np.array([1.0]), vz=np.array([1.0]), m=np.array([1.0]))
    dt = 3e-3
    steps = int(round(0.4 / dt))
    worst, deepest = 0.0, False
    for _ in range(steps):
        r = oracle_mod.apm_step(cfg, grids, p, 0.5 * dt)
        oracle_mod.kick_drift(p, r.pacc, dt)
        worst = max(worst, float(np.linalg.norm(_vel(p)[:, 0] - 1.0) / math.sqrt(3)))
        deepest |= 0.40625 < p["x"][0] < 0.59375
    assert deepest                                    # it reached level 3
    assert p["x"][0] == pytest.approx(0.15 + steps * dt, abs=1e-12)
    assert worst < 1e-12, worst
