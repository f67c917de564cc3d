"""Pins of the oracle's DFT and per-grid solve against numpy's FFT and brute force."""
import numpy as np
import pytest


def test_dft_matches_numpy(oracle_mod):
    rng = np.random.default_rng(0)
    a = rng.normal(size=(5, 6, 4)) + 1j * rng.normal(size=(5, 6, 4))
    re, im = oracle_mod.dft3(a.real, a.imag, -1)
    ref = np.fft.fftn(a)
    assert np.max(np.abs(re + 1j * im - ref)) < 1e-12 * np.max(np.abs(ref))
    re, im = oracle_mod.dft3(a.real, a.imag, +1)
    ref = np.fft.ifftn(a) * a.size
    assert np.max(np.abs(re + 1j * im - ref)) < 1e-12 * np.max(np.abs(ref))


def _small_child(oracle_mod, N=(4, 7, 16), start=(40, 41, 38)):
    cfg = oracle_mod.Config()
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (32,) * 3), oracle_mod.Grid(1, 0, start, N)]
    return cfg, grids, oracle_mod.plan_grid(cfg, grids, 1)


def _numpy_solve(oracle_mod, cfg, plan, gmf):
    """Circular convolution on the M grid by numpy's FFT (independent of orc_dft3)."""
    T = oracle_mod.full_table(cfg, plan)
    M = plan.M
    rho = np.zeros(M[::-1])
    G = plan.G
    rho[:G[2], :G[1], :G[0]] = np.ldexp(gmf.astype(np.float64), -cfg.mass_frac_bits)
    phi = np.fft.ifftn(np.fft.fftn(rho) * T).real
    idx = [(plan.s0[j] + np.arange(plan.W[j])) % M[j] for j in range(3)]
    return phi[np.ix_(idx[2], idx[1], idx[0])], T


def test_solve_is_circular_convolution_on_M(oracle_mod):
    # reading R6: the potential is the circular convolution on the M grid
    cfg, grids, plan = _small_child(oracle_mod)
    assert plan.M == (24, 27, 36)
    rng = np.random.default_rng(1)
    gmf = rng.integers(0, 1 << 40, size=plan.G[::-1], dtype=np.int64)
    phis = oracle_mod.solve(cfg, grids, 1, gmf)
    ref, T = _numpy_solve(oracle_mod, cfg, plan, gmf)
    assert np.max(np.abs(phis - ref)) < 1e-12 * np.max(np.abs(ref))
    # brute-force direct sum at a few output cells, with the real-space kernel
    g = np.fft.ifftn(T).real
    mass = np.ldexp(gmf.astype(np.float64), -cfg.mass_frac_bits)
    M = plan.M
    jz, jy, jx = np.meshgrid(*[np.arange(plan.G[j]) for j in (2, 1, 0)], indexing="ij")
    for o in [(0, 0, 0), (3, 5, 7), (plan.W[0] - 1, plan.W[1] - 1, plan.W[2] - 1), (2, 9, 0)]:
        om = [(plan.s0[j] + o[j]) % M[j] for j in range(3)]
        direct = np.sum(g[(om[2] - jz) % M[2], (om[1] - jy) % M[1], (om[0] - jx) % M[0]] * mass)
        assert abs(phis[o[2], o[1], o[0]] - direct) < 1e-12 * np.max(np.abs(ref))


def test_unit_mass_reproduces_kernel(oracle_mod):
    cfg, grids, plan = _small_child(oracle_mod, N=(6, 6, 6))
    gmf = np.zeros(plan.G[::-1], dtype=np.int64)
    j0 = (7, 4, 9)  # (x, y, z) GMF-local
    gmf[j0[2], j0[1], j0[0]] = 1 << cfg.mass_frac_bits
    phis = oracle_mod.solve(cfg, grids, 1, gmf)
    g = np.fft.ifftn(oracle_mod.full_table(cfg, plan)).real
    M = plan.M
    for o in [(0, 0, 0), (5, 6, 7), (9, 1, 3)]:
        d = [(plan.s0[j] + o[j] - j0[j]) % M[j] for j in range(3)]
        assert phis[o[2], o[1], o[0]] == pytest.approx(g[d[2], d[1], d[0]], rel=1e-11, abs=1e-9)


def test_solve_linear(oracle_mod):
    cfg, grids, plan = _small_child(oracle_mod, N=(5, 3, 4))
    rng = np.random.default_rng(2)
    a = rng.integers(0, 1 << 40, size=plan.G[::-1], dtype=np.int64)
    b = rng.integers(0, 1 << 40, size=plan.G[::-1], dtype=np.int64)
    pa = oracle_mod.solve(cfg, grids, 1, a)
    pb = oracle_mod.solve(cfg, grids, 1, b)
    pab = oracle_mod.solve(cfg, grids, 1, a + b)
    assert np.max(np.abs(pab - pa - pb)) < 1e-12 * np.max(np.abs(pab))


@pytest.mark.parametrize("periodic", [False, True])
def test_root_solve_matches_numpy(oracle_mod, periodic):
    # isolated root: doubled grid, window [-2, N+2) wraps; periodic: M = N
    cfg = oracle_mod.Config(periodic=periodic)
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (8, 8, 8))]
    plan = oracle_mod.plan_grid(cfg, grids, 0)
    assert plan.M == ((8,) * 3 if periodic else (16,) * 3)
    rng = np.random.default_rng(3)
    gmf = rng.integers(0, 1 << 44, size=(8, 8, 8), dtype=np.int64)
    phis = oracle_mod.solve(cfg, grids, 0, gmf)
    ref, _ = _numpy_solve(oracle_mod, cfg, plan, gmf)
    assert np.max(np.abs(phis - ref)) < 1e-12 * np.max(np.abs(ref))


def test_isolated_root_table_is_transform_of_real_space_kernel(oracle_mod):
    # reading R4 with the correction off: T = DFT of psi at minimum-image offsets
    cfg = oracle_mod.Config(periodic=False, root_correction=False)
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (6, 6, 6))]
    plan = oracle_mod.plan_grid(cfg, grids, 0)
    M = plan.M
    d = [np.where(np.arange(m) <= m // 2, np.arange(m), np.arange(m) - m) * plan.delta for m in M]
    zz, yy, xx = np.meshgrid(d[2], d[1], d[0], indexing="ij")
    r = np.sqrt(xx * xx + yy * yy + zz * zz) / plan.a_lev
    g = np.vectorize(oracle_mod.psi)(r) / plan.a_lev
    ref = np.fft.fftn(g).real
    T = oracle_mod.full_table(cfg, plan)
    assert np.max(np.abs(T - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(6, 10, 15), (8, 9, 7), (150, 2, 3), (64, 4, 5), (1, 49, 12), (11, 13, 2)])
def test_textbook_fft_mode_equals_naive_dft(shape, oracle_mod):
    oracle = oracle_mod
    """The oracle's textbook FFT mode (recursive Cooley-Tukey by smallest prime
    factor) computes the same unnormalised DFT as its naive sum, forward and
    inverse, on smooth and prime lengths (shape given as (x, y, z))."""
    rng = np.random.default_rng(sum(shape))
    re = rng.normal(size=shape[::-1])
    im = rng.normal(size=shape[::-1])
    prev = oracle.set_transform("dft")
    try:
        for sign in (-1, 1):
            ar, ai = oracle.dft3(re, im, sign)
            oracle.set_transform("fft")
            br, bi = oracle.dft3(re, im, sign)
            oracle.set_transform("dft")
            a = ar + 1j * ai
            b = br + 1j * bi
            assert np.linalg.norm(b - a) <= 1e-13 * np.linalg.norm(a)
            ref = np.fft.fftn(re + 1j * im) if sign < 0 else np.fft.ifftn(re + 1j * im) * re.size
            assert np.linalg.norm(b - ref) <= 1e-13 * np.linalg.norm(ref)
    finally:
        oracle.set_transform(prev)


def test_textbook_fft_mode_solve_matches_naive_solve(oracle_mod):
    oracle = oracle_mod
    """A periodic-root solve through the FFT mode equals the naive-DFT solve."""
    n = 24
    cfg = oracle.Config(periodic=True)
    grids = [oracle.Grid(0, -1, (0, 0, 0), (n, n, n))]
    gmf = np.random.default_rng(5).integers(0, 1 << 40, size=(n, n, n))
    prev = oracle.set_transform("dft")
    try:
        a = oracle.solve(cfg, grids, 0, gmf)
        oracle.set_transform("fft")
        b = oracle.solve(cfg, grids, 0, gmf)
    finally:
        oracle.set_transform(prev)
    assert np.linalg.norm(b - a) <= 1e-13 * np.linalg.norm(a)
