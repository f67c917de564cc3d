"""Pins of the oracle's gradient operators (Sec. 2.2 allows a finite difference
or the Fourier-space gradient D = -ik; reading R15): each operator's symbol
against the action of its real-space stencil on a sampled sine, the single-mode
potential and acceleration of the Sec. 3.4 sine wave, the continuum limit of
the influence function, zero self-force and opposite pair forces, the point-mass
far field, and the isolated root's doubled grid for the four-point stencil."""
import math

import numpy as np
import pytest

import apm_inputs as W

GRADS = ["fd2", "fd4", "spectral"]


def _parts(x, y, z, m):
    x = np.atleast_1d(np.asarray(x, float))
    return dict(x=x, y=np.atleast_1d(np.asarray(y, float)), z=np.atleast_1d(np.asarray(z, float)),
                vx=0 * x, vy=0 * x, vz=0 * x, m=np.atleast_1d(np.asarray(m, float)))


EMPTY = _parts([], [], [], [])


def _stencil_symbol(grad, k, d):
    """D(k) from the stencil applied to samples of sin(k x): the centred
    differences of HE (two and four points) return D(k) cos(k x); a spectral
    derivative returns k cos(k x)."""
    x = np.linspace(0.1, 2.3, 7)
    f = lambda s: np.sin(k * (x + s * d))
    if grad == "fd2":
        y = (f(1) - f(-1)) / (2 * d)
    elif grad == "fd4":
        y = (8 * (f(1) - f(-1)) - (f(2) - f(-2))) / (12 * d)
    else:
        return k
    return float(np.mean(y / np.cos(k * x)))


@pytest.mark.parametrize("grad", GRADS)
def test_operator_symbol_matches_its_stencil(oracle_mod, grad):
    M, d = 48, 1.0 / 48
    for kc in (1, 3, 7, 13, 20, -5, -17):
        k = 2 * math.pi * kc / (M * d)
        assert oracle_mod.grad_d(grad, kc, M, d) == pytest.approx(_stencil_symbol(grad, k, d), rel=1e-12)
    # the Nyquist mode: both differences vanish there, the spectral one is set to 0
    assert abs(oracle_mod.grad_d(grad, M // 2, M, d)) < 1e-12 / d
    # accuracy orders at small k delta: 1 - (k d)^2/6, 1 - (k d)^4/30, exact
    k = 2 * math.pi / (M * d)
    err = abs(oracle_mod.grad_d(grad, 1, M, d) / k - 1)
    th = k * d
    want = {"fd2": th ** 2 / 6, "fd4": th ** 4 / 30, "spectral": 0.0}[grad]
    assert err == pytest.approx(want, rel=2e-2, abs=1e-15)


@pytest.mark.parametrize("grad", ["fd4", "spectral"])
@pytest.mark.parametrize("period,axis", [(1.0, 0), (0.2, 1), (0.25, 2)])
def test_sine_wave_single_mode_per_gradient(oracle_mod, grad, period, axis):
    """Sec. 3.4 on the periodic root: phi = G(k) sin(k x) and
    A = -G(k) D(k) cos(k x) exactly, with D(k) the operator's symbol from its
    stencil (k itself for the spectral gradient); no other component."""
    cfg = oracle_mod.Config(periodic=True, mass_frac_bits=60, gradient=grad)
    grids = [oracle_mod.Grid(*W.GridDesc(0, -1, (0, 0, 0), (32, 32, 32)))]
    gas = W.sine_wave_gas(grids, period, axis=axis)
    res = oracle_mod.apm_step(cfg, grids, EMPTY, 0.0, gas=gas)
    plan = oracle_mod.plan_grid(cfg, grids, 0)
    kap = [0, 0, 0]
    kap[axis] = int(round(1.0 / period))
    Gk = oracle_mod.green_opt(kap, plan.M, plan.delta, plan.a_lev, 0.0, 0, gradient=grad)
    d = plan.delta
    k = 2 * math.pi / period
    xc = (np.arange(32) + 0.5) * d
    phi = np.moveaxis(res.phi[0][1:-1, 1:-1, 1:-1], 2 - axis, 0)
    exp_phi = Gk * np.sin(k * xc)
    assert np.max(np.abs(phi - exp_phi[:, None, None])) < 1e-12 * np.max(np.abs(exp_phi))
    A = np.moveaxis(res.acc[0][axis][1:-1, 1:-1, 1:-1], 2 - axis, 0)
    exp_A = -Gk * _stencil_symbol(grad, k, d) * np.cos(k * xc)
    assert np.max(np.abs(A - exp_A[:, None, None])) < 1e-11 * np.max(np.abs(exp_A))
    for j in range(3):
        if j != axis:
            assert np.max(np.abs(res.acc[0][j])) < 1e-12 * np.max(np.abs(exp_A))


@pytest.mark.parametrize("grad", GRADS)
def test_influence_function_continuum_limit(oracle_mod, grad):
    """G-hat(k) -> -4 pi S-hat(k a / 2)^2 / k^2 as delta -> 0 at fixed k and a
    (root reference force), for every operator, as delta^2 (the TSC assignment's
    order: 16 times smaller per factor 4 in resolution)."""
    a = 0.05
    errs = []
    for n in (64, 256, 1024):
        d = 1.0 / n
        k = 2 * math.pi * 3
        g = oracle_mod.green_opt((3, 1, 0), (n, n, n), d, a, 0.0, 0, gradient=grad)
        kk = math.hypot(k, 2 * math.pi)
        cont = -4 * math.pi * oracle_mod.shat(kk * a / 2) ** 2 / kk ** 2
        errs.append(abs(g / cont - 1))
    assert 14 < errs[0] / errs[1] < 18 and 14 < errs[1] / errs[2] < 18 and errs[2] < 2e-4, errs


@pytest.mark.parametrize("grad", GRADS)
def test_no_self_force_and_opposite_pair_forces(oracle_mod, grad):
    """An even Green's function, an odd gradient and the same TSC weights both
    ways give no self-force and exactly opposite pair forces (single isolated
    grid), for every operator; through the Fig. 1 hierarchy the self-force
    stays at rounding level."""
    cfg = oracle_mod.Config(gradient=grad)
    root = [oracle_mod.Grid(*W.GridDesc(0, -1, (0, 0, 0), (24, 24, 24)))]
    rng = np.random.default_rng(4)
    for _ in range(3):
        x = 0.2 + 0.6 * rng.random(3)
        res = oracle_mod.apm_step(cfg, root, _parts(*x, 1.0), 0.0)
        assert np.max(np.abs(res.pacc)) < 1e-11
    x = 0.25 + 0.5 * rng.random((3, 2))
    m = np.array([1.0, 0.3])
    res = oracle_mod.apm_step(cfg, root, _parts(x[0], x[1], x[2], m), 0.0)
    mom = res.pacc @ m
    assert np.max(np.abs(mom)) < 1e-12 * np.max(np.abs(res.pacc[:, 0]))
    fig1 = [oracle_mod.Grid(*g) for g in W.grids_from_bounds(16, W.FIG1_BOUNDS)]
    for x in (0.15, 0.3, 0.45, 0.5):
        res = oracle_mod.apm_step(cfg, fig1, _parts(x, x + 0.01, x - 0.02, 1.0), 0.0)
        assert np.max(np.abs(res.pacc)) < 1e-10


def test_point_mass_force_isotropy_improves_with_the_operator(oracle_mod):
    """Radial force of a unit mass on massless particles at r = 0.3 (4.8 cells of
    a 16^3 isolated root, beyond the softening 3.4 cells), over 300 random
    directions and 10 sub-cell offsets: the mean is Newtonian within a percent
    for every operator, and the scatter, which comes from the operator's
    anisotropy, falls from the two-point to the four-point difference to the
    spectral gradient (measured 3.9%, 0.7%, 0.18%)."""
    rng = np.random.default_rng(1)
    n, r = 300, 0.3
    dirs = rng.normal(size=(3, n))
    dirs /= np.linalg.norm(dirs, axis=0)
    centres = 0.5 + rng.random((10, 3)) / 16
    spread = {}
    for grad in GRADS:
        cfg = oracle_mod.Config(gradient=grad)
        root = [oracle_mod.Grid(0, -1, (0, 0, 0), (16, 16, 16))]
        vals = []
        for c in centres:
            pos = c[:, None] + r * dirs
            p = _parts(np.r_[c[0], pos[0]], np.r_[c[1], pos[1]], np.r_[c[2], pos[2]], np.r_[1.0, np.zeros(n)])
            res = oracle_mod.apm_step(cfg, root, p, 0.0)
            vals.append(-(res.pacc[:, 1:] * dirs).sum(0) * r * r)
        v = np.concatenate(vals)
        assert abs(v.mean() - 1) < 0.01, (grad, v.mean())
        spread[grad] = v.std()
    assert spread["spectral"] < 0.005 < spread["fd4"] < 0.015 < spread["fd2"] < 0.06, spread


def test_fd4_isolated_root_window_sees_unwrapped_offsets(oracle_mod):
    """Reading R15: with the four-point stencil the root's edge cells read phi at
    cells -2 and N + 1.  Without the k-space correction the isolated-root
    potential is the direct sum of the S-S pair potential over the cell masses,
    so on M >= 2N + 2 it equals that sum on the whole window [-2, N + 2), which
    the doubled grid M = 2N would not give at offsets N + 1."""
    N = 8
    cfg = oracle_mod.Config(gradient="fd4", root_correction=False, mass_frac_bits=60)
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (N, N, N))]
    plan = oracle_mod.plan_grid(cfg, grids, 0)
    assert plan.M == (18, 18, 18) and plan.W == (14, 14, 14)
    p = _parts([0.02, 0.97, 0.51], [0.03, 0.5, 0.98], [0.96, 0.04, 0.5], [1.0, 0.7, 0.4])
    gmf, _ = oracle_mod.deposit(cfg, grids, 0, p, 0.0)
    phis = oracle_mod.solve(cfg, grids, 0, gmf)
    mass = np.ldexp(gmf.astype(float), -cfg.mass_frac_bits)
    d, a = plan.delta, plan.a_lev
    src = np.argwhere(mass != 0)          # [z, y, x]
    h = 3
    for c in [(-2, 0, 3), (N + 1, 4, N - 1), (-2, -2, -2), (N + 1, N + 1, N + 1), (3, -1, N)]:
        want = 0.0
        for s in src:
            off = np.array(c) - s[::-1]
            want += mass[tuple(s)] * oracle_mod.psi(np.linalg.norm(off) * d / a) / a
        got = phis[c[2] + h, c[1] + h, c[0] + h]
        assert got == pytest.approx(want, rel=1e-12), c


@pytest.mark.parametrize("M", [(12, 10, 9), (16, 15, 14)])
def test_spectral_solve_equals_numpy_fft_route(oracle_mod, M):
    """orc_solve_spectral against numpy's FFT on a random mass field: the mass
    on the M grid, its transform times the table, times -i k_j (0 on an even
    M's Nyquist mode) for A_j, transformed back and windowed.  Pins the
    spectral solve's transforms, product, sign and window on every mode."""
    import ctypes
    rng = np.random.default_rng(7)
    G = (M[0] - 3, M[1] - 2, M[2] - 4)
    W = (M[0] + 2, M[1] - 1, M[2] + 1)          # longer than M on x and z: wraps
    s0 = (M[0] - 2, 3, M[2] - 1)
    F = 40
    delta = 1.0 / 16
    gmf = rng.integers(-2 ** 40, 2 ** 40, size=G[::-1], dtype=np.int64)
    H = tuple(m // 2 + 1 for m in M)
    T = rng.normal(size=H[::-1])                 # any table even in every kappa_j
    out = np.zeros((4,) + W[::-1])
    lib = oracle_mod.lib()
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lib.orc_solve_spectral(P(gmf), P(np.array(G, dtype=np.int64)), F, P(np.array(M, dtype=np.int64)),
                           P(np.array(s0, dtype=np.int64)), P(np.array(W, dtype=np.int64)), P(T), delta,
                           P(out), 1)
    mass = np.zeros(M[::-1])
    mass[:G[2], :G[1], :G[0]] = np.ldexp(gmf.astype(float), -F)
    rho = np.fft.fftn(mass)
    idx = [np.minimum(np.arange(m), m - np.arange(m)) for m in M]
    Tf = T[np.ix_(idx[2], idx[1], idx[0])]
    phi_hat = Tf * rho
    comps = [phi_hat]
    for j in range(3):
        m = M[j]
        kc = np.where(np.arange(m) <= m // 2, np.arange(m), np.arange(m) - m)
        k = 2 * np.pi * kc / (m * delta)
        if m % 2 == 0:
            k[m // 2] = 0.0
        shape = [1, 1, 1]
        shape[2 - j] = m
        comps.append(-1j * k.reshape(shape) * phi_hat)
    for c, spec in enumerate(comps):
        field = np.fft.ifftn(spec).real
        sel = np.ix_(*[(s0[a] + np.arange(W[a])) % M[a] for a in (2, 1, 0)])
        want = field[sel]
        assert np.allclose(out[c], want, rtol=0, atol=1e-12 * np.abs(want).max()), c
