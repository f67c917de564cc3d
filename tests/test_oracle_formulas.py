"""Pins of the oracle's scalar formulas against quadrature, series and limits.

Each check ties an oracle routine to something other than itself: a numerical
integral of the paper's real-space definition, a library routine, a limit or
a symmetry the mathematics fixes.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

ETAS = [0.05, 0.3, 0.9, 1.0, 1.7, 4.0, 9.5]


def _shat_from_S(eta, a=1.0):
    """3-D Fourier transform of Eq. S2 (uniformly decreasing sphere), by quadrature."""
    k = 2.0 * eta / a

    def S(r):
        return 48.0 / (math.pi * a ** 4) * (a / 2.0 - r)

    f = lambda r: S(r) * math.sin(k * r) / (k * r) * 4.0 * math.pi * r * r
    return quad(f, 0.0, a / 2.0, epsabs=1e-15, limit=200)[0]


@pytest.mark.parametrize("eta", ETAS)
def test_shat_is_transform_of_smoothing_sphere(oracle_mod, eta):
    # Sec. 2.2 Eq. S2 -> Eq. S2k
    assert abs(oracle_mod.shat(eta) - _shat_from_S(eta)) < 1e-13


def test_smoothing_sphere_normalised():
    a = 0.37
    m = quad(lambda r: 48.0 / (math.pi * a ** 4) * (a / 2 - r) * 4 * math.pi * r * r, 0, a / 2)[0]
    assert abs(m - 1.0) < 1e-14


def test_shat_series_matches_closed_form(oracle_mod):
    # reading R3: the series branch below eta = 1 agrees with the closed form
    # where the closed form is still accurate
    for eta in np.linspace(0.6, 0.999, 25):
        assert abs(oracle_mod.shat(eta) - oracle_mod.shat_closed(eta)) < 2e-14
    # continuity across the switch: just below 1 the series equals the closed form
    assert abs(oracle_mod.shat(1.0 - 1e-12) - oracle_mod.shat_closed(1.0 - 1e-12)) < 1e-14


def test_shat_small_argument(oracle_mod):
    for eta in [1e-6, 1e-3, 0.02]:
        ref = 1.0 - eta ** 2 / 15.0 + eta ** 4 / 560.0 - eta ** 6 / 37800.0
        assert abs(oracle_mod.shat(eta) - ref) < 1e-15
    # the closed form alone is useless there (cancellation), the reason for R3
    assert abs(oracle_mod.shat_closed(1e-4) - 1.0) > 1e-6


@pytest.mark.parametrize("x", [0.01, 0.4, 1.0, 1.3, 1.5707963])
def test_alias_sum_identity(oracle_mod, x):
    # Eq. assignment2 with U^2 = prod sinc^6 (reading R2): sum over all
    # Brillouin zones of sinc^6(x + pi n) = 1 - sin^2 x + 2/15 sin^4 x
    n = np.arange(-20000, 20001)
    xs = x + math.pi * n
    s = np.sum((np.sin(xs) / xs) ** 6)
    closed = 1.0 - math.sin(x) ** 2 + 2.0 / 15.0 * math.sin(x) ** 4
    assert abs(s - closed) < 1e-13
    # and sinc^3 (U itself) does not satisfy it: the printed Eq. assignment is U^2
    s3 = np.sum(np.abs(np.sin(xs) / xs) ** 3)
    if x > 0.3:
        assert abs(s3 - closed) > 1e-3
    assert abs(oracle_mod.lib().orc_sinc(x) - math.sin(x) / x) < 1e-16


def test_oracle_alias_sum_matches_brute_force(oracle_mod):
    # the oracle's denominator of Eq. influence against an explicit sum of
    # U^2(k_n) = prod sinc^6(k_j delta/2 + pi n_j) over many Brillouin zones
    n = np.arange(-4000, 4001)
    for kap, M in [((3, 7, 11), (36, 40, 45)), ((18, 0, 20), (36, 40, 45)), ((1, 2, 0), (8, 8, 8))]:
        ref = 1.0
        for j in range(3):
            kc = kap[j] - M[j] if kap[j] > M[j] // 2 else kap[j]
            xs = math.pi * kc / M[j] + math.pi * n
            with np.errstate(invalid="ignore", divide="ignore"):
                sc = np.where(xs == 0, 1.0, np.sin(xs) / xs)
            ref *= np.sum(sc ** 6)
        assert abs(oracle_mod.alias_sum(kap, M) - ref) < 1e-12


@pytest.mark.parametrize("xi", [0.05, 0.2, 0.45, 0.5, 0.6, 0.8, 1.0, 1.4])
def test_psi_is_pair_potential_of_smoothing_spheres(oracle_mod, xi):
    # reading R4: psi is the inverse transform of -4 pi S^2/k^2 (a = 1):
    # psi(r) = -(2/pi) int_0^inf S(k/2)^2 sin(kr)/(kr) dk
    r = xi
    f = lambda k: oracle_mod.shat(k / 2.0) ** 2 * math.sin(k * r) / (k * r)
    tot = 0.0
    for lo in np.arange(0.0, 3000.0, 4.0):
        tot += quad(f, lo, lo + 4.0, limit=100, epsabs=1e-14)[0]
    assert abs(oracle_mod.psi(xi) - (-2.0 / math.pi) * tot) < 2e-9


def test_psi_continuity_and_far_field(oracle_mod):
    for x0 in (0.5, 1.0):
        assert abs(oracle_mod.psi(x0 - 1e-12) - oracle_mod.psi(x0 + 1e-12)) < 1e-10
    assert oracle_mod.psi(2.5) == -1.0 / 2.5
    assert abs(oracle_mod.psi(0.5) + 19.0 / 10.0) < 1e-14


def test_green_continuum_limit_root(oracle_mod):
    # Eq. influence -> -4 pi S^2 / k^2 when the mesh is much finer than 1/k
    # (TSC, FD and aliasing corrections vanish); fixes sign and 4 pi (reading R1)
    a = 0.05
    for kap in [(3, 2, 1), (5, 0, 0), (2, 7, 4)]:
        M = (1 << 16,) * 3
        delta = 1.0 / M[0]
        k = 2 * math.pi * np.array(kap)
        kk = float(k @ k)
        g = oracle_mod.green_opt(kap, M, delta, a, 0.0, 0)
        ref = -4 * math.pi * oracle_mod.shat(math.sqrt(kk) * a / 2) ** 2 / kk
        assert abs(g / ref - 1.0) < 1e-6


def test_green_continuum_limit_refined(oracle_mod):
    # short-range kernel: (S_l^2 - S_{l-1}^2)/k^2 (Eq. reference); the mesh
    # corrections vanish as delta^2 (16x smaller per 4x finer mesh)
    al, ap = 0.02, 0.04
    for kap in [(9, 4, 1), (20, 0, 3)]:
        k = 2 * math.pi * np.array(kap)
        kk = float(k @ k)
        q = math.sqrt(kk)
        ref = -4 * math.pi * (oracle_mod.shat(q * al / 2) ** 2 - oracle_mod.shat(q * ap / 2) ** 2) / kk
        errs = []
        for mv in (1 << 12, 1 << 14, 1 << 16):
            g = oracle_mod.green_opt(kap, (mv,) * 3, 1.0 / mv, al, ap, 1)
            errs.append(abs(g / ref - 1.0))
        assert errs[-1] < 5e-6
        assert 12.0 < errs[0] / errs[1] < 20.0 and 12.0 < errs[1] / errs[2] < 20.0


def test_green_refined_k0_limit(oracle_mod):
    # reading R5: the kappa = 0 value of a refined level is the k -> 0 limit
    al = 3.4 / 64.0
    ap = 2 * al
    lim = -4 * math.pi * (ap * ap - al * al) / 30.0
    # (at much smaller k the difference of two S^2 near 1 loses digits)
    g = oracle_mod.green_opt((1, 0, 0), (1 << 16, 4, 4), 1.0 / 64.0, al, ap, 1)
    assert abs(g / lim - 1.0) < 1e-6
    cfg = oracle_mod.Config()
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (32,) * 3), oracle_mod.Grid(1, 0, (20,) * 3, (8,) * 3)]
    plan = oracle_mod.plan_grid(cfg, grids, 1)
    T = oracle_mod.green_table(cfg, plan)
    assert abs(T[0, 0, 0] * plan.delta ** 3 / (-4 * math.pi * (plan.a_par ** 2 - plan.a_lev ** 2) / 30) - 1) < 1e-15


def test_green_even_in_each_component(oracle_mod):
    M = (36, 40, 45)
    d = 1.0 / 128
    for kap in [(3, 7, 11), (18, 1, 22), (5, 20, 0), (17, 13, 8)]:
        g0 = oracle_mod.green_opt(kap, M, d, 3.4 * d, 6.8 * d, 1)
        for j in range(3):
            km = list(kap)
            km[j] = (M[j] - kap[j]) % M[j]
            assert abs(oracle_mod.green_opt(km, M, d, 3.4 * d, 6.8 * d, 1) - g0) <= 1e-13 * abs(g0)


def test_green_table_degenerate_modes_zero(oracle_mod):
    # reading R5: where the FD gradient vanishes identically the table is 0
    cfg = oracle_mod.Config(periodic=True)
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (16, 16, 16))]
    T = oracle_mod.green_table(cfg, oracle_mod.plan_grid(cfg, grids, 0))
    for z in (0, 8):
        for y in (0, 8):
            for x in (0, 8):
                assert T[z, y, x] == 0.0
    # attractive away from the Nyquist corner (next to the degenerate modes the
    # optimal kernel may change sign)
    assert np.all(T[1:7, 1:7, 1:7] < 0)


def test_green_table_matches_pointwise(oracle_mod):
    cfg = oracle_mod.Config()
    grids = [oracle_mod.Grid(0, -1, (0, 0, 0), (32,) * 3), oracle_mod.Grid(1, 0, (20, 22, 24), (6, 9, 12))]
    plan = oracle_mod.plan_grid(cfg, grids, 1)
    assert plan.M == (27, 30, 32) and plan.B == 5
    T = oracle_mod.green_table(cfg, plan)
    for kap in [(1, 2, 3), (13, 15, 16), (0, 0, 5)]:
        ref = oracle_mod.green_opt(kap, plan.M, plan.delta, plan.a_lev, plan.a_par, 1) / plan.delta ** 3
        assert T[kap[2], kap[1], kap[0]] == pytest.approx(ref, rel=1e-15)


def test_plan_rules(oracle_mod):
    # reading R6: B = ceil(0.65 * 2 * 3.4) = 5, M = smallest 7-smooth >= N + 20
    cfg = oracle_mod.Config()
    assert oracle_mod.border_cells(cfg) == 5
    assert [oracle_mod.smooth7_at_least(n + 20) for n in (16, 32, 64, 128, 25, 29)] == \
        [36, 54, 84, 150, 45, 49]
