"""Pins of the oracle's TSC deposit, baryon copy and drift (Sec. 2)."""
import math

import numpy as np
import pytest

from apm_inputs import GridDesc


def _tsc_shape(s):
    """Triangular-shaped-cloud assignment function of the particle-cell distance s
    (cell units): 3/4 - s^2 for |s| <= 1/2, (3/2 - |s|)^2 / 2 for 1/2 < |s| <= 3/2."""
    s = abs(s)
    if s <= 0.5:
        return 0.75 - s * s
    if s <= 1.5:
        return 0.5 * (1.5 - s) ** 2
    return 0.0


def test_tsc_weights_match_shape_function(oracle_mod):
    """The fixed-point weights (reading R11) are the TSC shape function of the
    particle-centre distance up to the position rounding (2^-32 cell, slopes <= 1)."""
    rng = np.random.default_rng(0)
    delta = 1.0 / 64
    tol = 2.0 ** -32 + 2.0 ** -52
    for x in rng.random(400):
        i, w = oracle_mod.tsc_weights(x, delta)
        assert i in (math.floor(x / delta), math.floor(x / delta + 2.0 ** -32))
        for o in range(3):
            centre = (i + o - 1 + 0.5) * delta
            assert abs(w[o] - _tsc_shape((x - centre) / delta)) < tol
        assert abs(w.sum() - 1.0) <= 4 * 2.0 ** -53


def test_tsc_weights_exact_at_dyadic_offsets(oracle_mod):
    # offsets that are multiples of 2^-31 cell are represented exactly: the
    # weights equal the shape function
    delta = 1.0 / 32
    for t in (0.0, 0.25, 0.5, 0.75, 0.125, 1.0 / 3.0):
        x = (7 + t) * delta
        i, w = oracle_mod.tsc_weights(x, delta)
        tq = round(t * 2 ** 31) / 2 ** 31
        exact = [0.5 * (1 - tq) ** 2, 0.75 - (tq - 0.5) ** 2, 0.5 * tq ** 2]
        assert i == 7
        for k in range(3):
            assert abs(w[k] - exact[k]) <= 2.0 ** -53


def test_cic_and_tsc_agree_at_cell_corner(oracle_mod):
    # Sec. 2: "both CIC and TSC ... are equivalent for a particle located at a corner"
    delta = 1.0 / 32
    for j in (3, 17, 30):
        x = j * delta
        it, wt = oracle_mod.tsc_weights(x, delta)
        ic, wc = oracle_mod.cic_weights(x, delta)
        tsc = {it - 1: wt[0], it: wt[1], it + 1: wt[2]}
        cic = {ic: wc[0], ic + 1: wc[1]}
        for c in set(tsc) | set(cic):
            assert tsc.get(c, 0.0) == cic.get(c, 0.0)


def _parts(pos, m, vel=None):
    n = pos.shape[1]
    vel = np.zeros((3, n)) if vel is None else vel
    return dict(x=pos[0].copy(), y=pos[1].copy(), z=pos[2].copy(), vx=vel[0].copy(),
                vy=vel[1].copy(), vz=vel[2].copy(), m=np.asarray(m, dtype=float))


def _child_setup(oracle_mod, periodic=False):
    cfg = oracle_mod.Config(periodic=periodic)
    grids = [GridDesc(0, -1, (0, 0, 0), (16, 16, 16)), GridDesc(1, 0, (10, 12, 8), (8, 6, 10))]
    return cfg, [oracle_mod.Grid(*g) for g in grids]


def _total_fixed(m, F):
    return sum(int(np.rint(v * 2.0 ** F)) for v in m)


def test_deposit_conserves_integer_mass(oracle_mod):
    cfg, grids = _child_setup(oracle_mod)
    plan = oracle_mod.plan_grid(cfg, grids, 1)
    rng = np.random.default_rng(1)
    n = 300
    lo = (np.array(plan.lo) + 1.5) * plan.delta
    hi = (np.array(plan.lo) + np.array(plan.G) - 1.5) * plan.delta
    pos = lo[:, None] + rng.random((3, n)) * (hi - lo)[:, None]
    m = rng.random(n) * 1e-3
    gmf, st = oracle_mod.deposit(cfg, grids, 1, _parts(pos, m), 0.0)
    assert st == 0
    assert int(gmf.sum()) == _total_fixed(m, cfg.mass_frac_bits)


@pytest.mark.parametrize("periodic", [False, True])
def test_root_deposit_conserves_mass_at_edges(oracle_mod, periodic):
    # reading R7 (isolated: fold into the edge cells) / periodic wrap: no mass lost
    cfg = oracle_mod.Config(periodic=periodic)
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (8, 8, 8))]
    rng = np.random.default_rng(2)
    n = 200
    pos = rng.random((3, n))
    pos[:, :50] = rng.choice([0.001, 0.999, 0.0625, 0.5], size=(3, 50))
    m = rng.random(n)
    gmf, st = oracle_mod.deposit(cfg, grids, 0, _parts(pos, m), 0.0)
    assert st == 0
    assert int(gmf.sum()) == _total_fixed(m, cfg.mass_frac_bits)


def test_deposit_order_independent(oracle_mod):
    cfg, grids = _child_setup(oracle_mod)
    rng = np.random.default_rng(3)
    n = 500
    pos = 0.35 + 0.3 * rng.random((3, n))
    m = rng.random(n)
    g1, _ = oracle_mod.deposit(cfg, grids, 1, _parts(pos, m), 0.0)
    perm = rng.permutation(n)
    g2, _ = oracle_mod.deposit(cfg, grids, 1, _parts(pos[:, perm], m[perm]), 0.0)
    assert np.array_equal(g1, g2)


def test_deposit_matches_brute_force_shape_function(oracle_mod):
    """Independent statement of the deposit: each of the 27 cells around each
    particle gets rint(m W(sx) W(sy) W(sz) 2^F) with the TSC shape function of the
    particle-centre distance; the centre cell takes the remainder; cells outside
    the GMF box are dropped.  The charges agree to the fixed-point weight
    resolution; integer totals must agree exactly."""
    cfg, grids = _child_setup(oracle_mod)
    plan = oracle_mod.plan_grid(cfg, grids, 1)
    rng = np.random.default_rng(4)
    n = 12
    pos = (np.array(plan.lo)[:, None] + rng.random((3, n)) * np.array(plan.G)[:, None]) * plan.delta
    m = rng.random(n)
    gmf, _ = oracle_mod.deposit(cfg, grids, 1, _parts(pos, m), 0.0)
    F = cfg.mass_frac_bits
    ref = np.zeros_like(gmf)
    kept = 0
    for p in range(n):
        u = pos[:, p] / plan.delta
        ic = np.floor(u).astype(int)
        q = {}
        for c in range(-1, 2):
            for b in range(-1, 2):
                for a in range(-1, 2):
                    off = np.array([a, b, c])
                    s = u - (ic + off + 0.5)
                    w = _tsc_shape(s[0]) * _tsc_shape(s[1]) * _tsc_shape(s[2])
                    q[(a, b, c)] = int(np.rint(m[p] * w * 2.0 ** F))
        q[(0, 0, 0)] = int(np.rint(m[p] * 2.0 ** F)) - sum(v for k, v in q.items() if k != (0, 0, 0))
        for (a, b, c), v in q.items():
            g = ic + np.array([a, b, c]) - np.array(plan.lo)
            if np.all(g >= 0) and np.all(g < np.array(plan.G)):
                ref[g[2], g[1], g[0]] += v
                kept += v
    # the shape function and the fixed-point weights (reading R11) differ by at
    # most 2^-32 per axis (position rounding), so a charge by at most 3 2^-32 m 2^F
    tol = sum(3 * 2.0 ** -32 * mp * 2.0 ** F for mp in m) + 2 * n
    assert np.max(np.abs(gmf - ref)) <= tol
    fully_inside = all(np.all(np.floor(pos[:, p] / plan.delta) - 1 >= plan.lo) and
                       np.all(np.floor(pos[:, p] / plan.delta) + 1 < np.array(plan.lo) + plan.G)
                       for p in range(n))
    if fully_inside:
        assert int(gmf.sum()) == kept
    assert np.count_nonzero(gmf) > 0


def test_baryons_interior_and_parent_border(oracle_mod):
    # Sec. 2: interior from the grid's own gas, border from the parent's baryons
    cfg, grids = _child_setup(oracle_mod)
    g = grids[1]
    pg = grids[0]
    plan = oracle_mod.plan_grid(cfg, grids, 1)
    rng = np.random.default_rng(5)
    gas = rng.random(g.dims[::-1]) + 0.5
    pgas = rng.random(pg.dims[::-1]) + 0.5
    empty = _parts(np.zeros((3, 0)), [])
    gmf, _ = oracle_mod.deposit(cfg, grids, 1, empty, 0.0, gas=gas, parent_gas=pgas)
    F = cfg.mass_frac_bits
    vol = plan.delta ** 3
    B = plan.B
    for (x, y, z) in [(0, 0, 0), (B, B, B), (B + 3, B + 2, B + 5), (plan.G[0] - 1, 2, B + 1),
                      (B - 1, B + 1, B + 1), (B + g.dims[0], B, B)]:
        c = np.array([x, y, z]) - B
        if np.all(c >= 0) and np.all(c < np.array(g.dims)):
            rho = gas[c[2], c[1], c[0]]
        else:
            pc = (np.array(g.start) + c) // 2 - np.array(pg.start)
            rho = pgas[pc[2], pc[1], pc[0]]
        assert gmf[z, y, x] == int(np.rint(rho * vol * 2.0 ** F))


def test_drift_and_periodic_wrap(oracle_mod):
    # Sec. 2: half-step drift before the deposit
    assert oracle_mod.drift(0.25, 2.0, 0.125, 1.0, 0) == 0.5
    assert oracle_mod.drift(0.999, 1.0, 0.0105, 1.0, 1) == pytest.approx(0.0095, abs=1e-15)
    assert oracle_mod.drift(0.01, -1.0, 0.03, 1.0, 1) == pytest.approx(0.98, abs=1e-15)


def test_status_flags(oracle_mod):
    cfg = oracle_mod.Config()
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (8, 8, 8))]
    pos = np.array([[1.2, 0.5], [0.5, 0.5], [0.5, 0.5]])
    _, st = oracle_mod.deposit(cfg, grids, 0, _parts(pos, [1.0, 1.0]), 0.0)
    assert st & 2   # out of box (still folded)
    _, st = oracle_mod.deposit(cfg, grids, 0, _parts(pos[:, 1:], [4096.0]), 0.0)
    assert st & 1   # 4096 * 2^52 >= 2^62: overflow, skipped


def test_border_past_an_isolated_root_has_no_baryons(oracle_mod):
    """A level-1 grid whose GMF border reaches past an isolated root (start 2 on
    a 16^3 root: border cells from -3, root cells from -2): nothing lies outside
    an isolated domain, so those border cells hold zero baryon mass, the others
    the parent's density, and every particle's mass is still conserved."""
    cfg = oracle_mod.Config(periodic=False)
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (16, 16, 16)), oracle_mod.Grid(1, 0, (2, 10, 10), (8, 8, 8))]
    plan = oracle_mod.plan_grid(cfg, grids, 1)
    B = plan.B
    rng = np.random.default_rng(8)
    pgas = rng.random((16, 16, 16)) + 0.5
    empty = _parts(np.zeros((3, 0)), [])
    gmf, _ = oracle_mod.deposit(cfg, grids, 1, empty, 0.0, gas=None, parent_gas=pgas)
    vol = plan.delta ** 3
    F = cfg.mass_frac_bits
    for x in range(plan.G[0]):
        gx = 2 + x - B                               # global level-1 cell
        for (y, z) in [(0, 0), (B, B + 3), (plan.G[1] - 1, B)]:
            c = np.array([x, y, z]) - B
            if np.all(c >= 0) and np.all(c < 8):
                want = 0                             # interior, no own gas
            elif gx < 0:
                want = 0                             # past the root's face
            else:
                pc = (np.array([2, 10, 10]) + c) // 2
                want = int(np.rint(pgas[pc[2], pc[1], pc[0]] * vol * 2.0 ** F))
            assert gmf[z, y, x] == want, (x, y, z)
    # particles in the root cells next to the face deposit their whole mass
    pos = np.array([[0.01, 0.02], [0.33, 0.34], [0.35, 0.36]])
    m = [1.0, 0.5]
    parts = _parts(pos, m)
    gmf, st = oracle_mod.deposit(cfg, grids, 1, parts, 0.0)
    assert st == 0
    assert int(gmf.sum()) == sum(int(np.rint(v * 2.0 ** F)) for v in m)
