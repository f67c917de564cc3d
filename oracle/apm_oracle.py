"""Python composition of the oracle's C core (test infrastructure only).

Everything numeric happens in apm_oracle.c (FP64, -ffp-contract=off); this
module only holds the oracle's own plan of each grid (border, FFT length,
output window) and calls the C routines in the order of Sec. 2 / Sec. 2.2 of
the paper:

    drift -> TSC deposit + baryons (GMF) -> per-grid FFT convolution with the
    Green's table -> FD acceleration + parent carry -> TSC interpolation.

Array conventions: 3-D fields are numpy arrays indexed [z, y, x] (x fastest);
particles are a dict of float64 arrays x, y, z, vx, vy, vz, m.
"""
import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

from . import build_oracle

_lib = None


def lib():
    """Load (building if needed) the oracle's C core."""
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        d, i64, i32, ci = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        P = ctypes.c_void_p
        L.orc_shat.restype = d
        L.orc_shat.argtypes = [d]
        L.orc_shat_closed.restype = d
        L.orc_shat_closed.argtypes = [d]
        L.orc_sinc.restype = d
        L.orc_sinc.argtypes = [d]
        L.orc_psi.restype = d
        L.orc_psi.argtypes = [d]
        L.orc_alias_sum.restype = d
        L.orc_alias_sum.argtypes = [P, P]
        L.orc_green_opt.restype = d
        L.orc_green_opt.argtypes = [P, P, d, d, d, ci, ci]
        L.orc_grad_d.restype = d
        L.orc_grad_d.argtypes = [ci, i64, i64, d]
        L.orc_dft3.restype = None
        L.orc_dft3.argtypes = [P, P, P, ci, ci]
        L.orc_set_transform.restype = None
        L.orc_set_transform.argtypes = [ci]
        L.orc_get_transform.restype = ci
        L.orc_get_transform.argtypes = []
        L.orc_green_table.restype = None
        L.orc_green_table.argtypes = [ci, P, d, d, d, ci, ci, P, ci]
        L.orc_drift.restype = d
        L.orc_drift.argtypes = [d, d, d, d, ci]
        L.orc_kick_drift.restype = None
        L.orc_kick_drift.argtypes = [i64, P, P, P, P, P, P, P, d]
        L.orc_tsc_weights.restype = i64
        L.orc_tsc_weights.argtypes = [d, d, P]
        L.orc_cic_weights.restype = i64
        L.orc_cic_weights.argtypes = [d, d, P]
        L.orc_deposit.restype = ci
        L.orc_deposit.argtypes = [i64, P, P, P, P, P, P, P, d, d, ci, d, ci, P, P, ci, ci, P]
        L.orc_gas.restype = None
        L.orc_gas.argtypes = [P, P, i64, P, P, P, P, ci, d, ci, P]
        L.orc_solve.restype = None
        L.orc_solve.argtypes = [P, P, ci, P, P, P, P, P, ci]
        L.orc_accel.restype = None
        L.orc_solve_spectral.restype = None
        L.orc_solve_spectral.argtypes = [P, P, ci, P, P, P, P, d, P, ci]
        L.orc_accel.argtypes = [P, P, ci, d, P, P, P, P, P, ci, P, P]
        L.orc_interp.restype = None
        L.orc_interp.argtypes = [i64, P, P, P, P, P, P, d, d, ci, d, ci, P, P, ci, P, P, i32, P]
        L.orc_cells.restype = None
        L.orc_cells.argtypes = [i64, P, P, P, P, P, P, d, d, ci, d, ci, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i64(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int64))


def nthreads():
    return int(os.environ.get("APM_ORACLE_THREADS", "0"))


# --------------------------------------------------------------------------
# Scalar formulas (Sec. 2.2)
# --------------------------------------------------------------------------
def shat(eta):
    """S-hat(eta), Eq. S2k (series below eta = 1)."""
    return lib().orc_shat(float(eta))


def shat_closed(eta):
    return lib().orc_shat_closed(float(eta))


def psi(xi):
    """Pair potential of two unit S spheres of diameter a at r = xi a, times a."""
    return lib().orc_psi(float(xi))


def alias_sum(kappa, M):
    """Closed-form Brillouin-zone sum of U^2 (Eq. assignment2)."""
    return lib().orc_alias_sum(_p(_i64(kappa)), _p(_i64(M)))


GRADIENTS = {"fd2": 0, "fd4": 1, "spectral": 2}


def grad_d(gradient, kc, M, delta):
    """Gradient operator D_j at the centred mode kc of an M grid (orc_grad_d)."""
    return lib().orc_grad_d(GRADIENTS[gradient], int(kc), int(M), float(delta))


def green_opt(kappa, M, delta, a_lev, a_par, use_parent, gradient="fd2"):
    """Optimal influence function at one mode (Eq. influence), continuum units."""
    k = _i64(kappa)
    m = _i64(M)
    return lib().orc_green_opt(_p(k), _p(m), float(delta), float(a_lev), float(a_par),
                               int(use_parent), GRADIENTS[gradient])


def set_transform(mode):
    """The transform of every separable 3-D DFT in the oracle: "dft" (the naive
    sum, default) or "fft" (the textbook mixed-radix FFT, the same unnormalised
    DFT in O(M log M), for the benchmark-size grids).  Returns the previous
    mode."""
    prev = "fft" if lib().orc_get_transform() == 1 else "dft"
    lib().orc_set_transform(1 if mode == "fft" else 0)
    return prev


def dft3(re, im, sign):
    """Naive separable DFT of a complex array indexed [z, y, x] (in place copy)."""
    re = np.ascontiguousarray(re, dtype=np.float64).copy()
    im = np.ascontiguousarray(im, dtype=np.float64).copy()
    M = _i64(re.shape[::-1])
    lib().orc_dft3(_p(re), _p(im), _p(M), int(sign), nthreads())
    return re, im


def tsc_weights(x, delta):
    w = np.zeros(3)
    i = lib().orc_tsc_weights(float(x), float(delta), _p(w))
    return i, w


def cic_weights(x, delta):
    w = np.zeros(2)
    i = lib().orc_cic_weights(float(x), float(delta), _p(w))
    return i, w


def drift(x, v, half_dt, box, periodic):
    return lib().orc_drift(float(x), float(v), float(half_dt), float(box), int(periodic))


def kick_drift(particles, acc, dt):
    """One timestep in place (orc_kick_drift): particles is a dict of float64
    arrays x, y, z, vx, vy, vz; acc is (3, n), evaluated at x + v dt/2."""
    n = len(particles["x"])
    arr = {k: np.ascontiguousarray(particles[k], dtype=np.float64) for k in ("x", "y", "z", "vx", "vy", "vz")}
    a = np.ascontiguousarray(acc, dtype=np.float64).reshape(3, n)
    lib().orc_kick_drift(n, *[_p(arr[k]) for k in ("x", "y", "z", "vx", "vy", "vz")], _p(a), float(dt))
    for k in arr:
        particles[k] = arr[k]
    return particles


# --------------------------------------------------------------------------
# Hierarchy and per-grid plan
# --------------------------------------------------------------------------
@dataclass
class Config:
    box: float = 1.0
    a_over_dx: float = 3.4       # Sec. 2.2: a = 3.4 delta_l
    refine: int = 2              # Sec. 2.2: R = 2
    pad_factor: float = 0.65     # Sec. 2.2: 0.65 R a / delta extra cells
    periodic: bool = False       # root boundary (Sec. 3: isolated except Sec. 3.4)
    mass_frac_bits: int = 52     # fixed-point fraction bits of the GMF
    root_correction: bool = True # reading R4
    gradient: str = "fd2"        # Sec. 2.2 gradient operator: "fd2", "fd4", "spectral" (R15)


@dataclass
class Grid:
    level: int
    parent: int
    start: tuple   # global level-cell index of interior cell 0 (x, y, z)
    dims: tuple    # interior cells (x, y, z)


def smooth7_at_least(n):
    """Smallest integer >= n whose prime factors are all in {2, 3, 5, 7}."""
    m = max(int(n), 1)
    while True:
        r = m
        for p in (2, 3, 5, 7):
            while r % p == 0:
                r //= p
        if r == 1:
            return m
        m += 1


def even_smooth7_at_least(n):
    """Smallest even integer >= n whose prime factors are all in {2, 3, 5, 7}."""
    m = smooth7_at_least(n)
    while m % 2:
        m = smooth7_at_least(m + 1)
    return m


def border_cells(cfg):
    """Reading R6: B = ceil(0.65 R a/delta) cells per side (= 5 for R = 2, 3.4)."""
    return int(math.ceil(cfg.pad_factor * cfg.refine * cfg.a_over_dx - 1e-12))


@dataclass
class Plan:
    level: int
    delta: float
    a_lev: float
    a_par: float
    B: int
    G: tuple       # GMF box (x, y, z)
    lo: tuple      # global level index of GMF cell 0
    M: tuple       # FFT lengths
    s0: tuple      # M-grid index of output cell -h
    W: tuple       # output window (N + 2h), h = 3 for the four-point gradient, else 2
    mode: int      # 0 refined (drop), 1 isolated root (fold), 2 periodic root (wrap)
    kind: int      # green table kind: 0 refined, 1 periodic root, 2 isolated root


def root_delta(cfg, grids):
    """Root cell size; fixed-point positions are counted in 2^-31 root cells."""
    return cfg.box / grids[0].dims[0]


def plan_grid(cfg, grids, gi):
    g = grids[gi]
    N0 = grids[0].dims[0]
    delta = cfg.box / (N0 * cfg.refine ** g.level)
    a_lev = cfg.a_over_dx * delta
    N = tuple(int(v) for v in g.dims)
    h = 3 if cfg.gradient == "fd4" else 2
    W = tuple(v + 2 * h for v in N)
    if g.level == 0:
        if cfg.periodic:
            M = N
            kind, mode = 1, 2
        elif cfg.gradient == "fd4":
            # reading R15: the four-point difference at the root's edge cells
            # reads phi two cells outside, at offsets up to N + 1 from the
            # masses, which the doubled grid must hold without wrapping
            M = tuple(even_smooth7_at_least(2 * v + 2) for v in N)
            kind, mode = 2, 1
        else:
            M = tuple(2 * v for v in N)
            kind, mode = 2, 1
        return Plan(0, delta, a_lev, 0.0, 0, N, (0, 0, 0), M, (-h, -h, -h), W, mode, kind)
    B = border_cells(cfg)
    G = tuple(v + 2 * B for v in N)
    M = tuple(smooth7_at_least(v + 4 * B) for v in N)
    lo = tuple(int(s) - B for s in g.start)
    return Plan(g.level, delta, a_lev, cfg.refine * a_lev, B, G, lo, M,
                (B - h, B - h, B - h), W, 0, 0)


_table_cache = {}


def green_table(cfg, plan):
    """Octant table T[kz, ky, kx] (kappa_j in [0, M_j/2]) in DFT units."""
    key = (plan.kind, plan.M, plan.delta, plan.a_lev, plan.a_par, cfg.root_correction, cfg.gradient)
    if key not in _table_cache:
        H = tuple(m // 2 + 1 for m in plan.M)
        T = np.zeros(H[::-1], dtype=np.float64)
        lib().orc_green_table(plan.kind, _p(_i64(plan.M)), plan.delta, plan.a_lev, plan.a_par,
                              int(cfg.root_correction), GRADIENTS[cfg.gradient], _p(T), nthreads())
        _table_cache[key] = T
    return _table_cache[key]


def full_table(cfg, plan):
    """The table expanded to the whole M grid (indexed [kz, ky, kx])."""
    T = green_table(cfg, plan)
    idx = [np.minimum(np.arange(m), m - np.arange(m)) for m in plan.M]
    return T[np.ix_(idx[2], idx[1], idx[0])]


# --------------------------------------------------------------------------
# Steps of one APM solve
# --------------------------------------------------------------------------
def _parts(particles):
    keys = ("x", "y", "z", "vx", "vy", "vz", "m")
    arrs = [np.ascontiguousarray(particles[k], dtype=np.float64) for k in keys]
    return arrs, len(arrs[0])


def deposit(cfg, grids, gi, particles, half_dt, gas=None, parent_gas=None):
    """GMF (int64, [z, y, x]) of grid gi: TSC particles + baryons (Sec. 2).

    Returns (gmf, status bits)."""
    plan = plan_grid(cfg, grids, gi)
    g = grids[gi]
    G = plan.G
    gmf = np.zeros(G[::-1], dtype=np.int64)
    if gas is not None or (parent_gas is not None and plan.B > 0):
        N = _i64(g.dims)
        if g.parent >= 0:
            pg = grids[g.parent]
            Np, pstart = _i64(pg.dims), _i64(pg.start)
        else:
            Np, pstart = _i64([1, 1, 1]), _i64([0, 0, 0])
        gas_a = None if gas is None else np.ascontiguousarray(gas, dtype=np.float64)
        pg_a = None if parent_gas is None else np.ascontiguousarray(parent_gas, dtype=np.float64)
        lib().orc_gas(_p(gas_a), _p(N), plan.B, _p(pg_a), _p(Np), _p(pstart), _p(_i64(g.start)),
                      cfg.refine, plan.delta, cfg.mass_frac_bits, _p(gmf))
    (x, y, z, vx, vy, vz, m), n = _parts(particles)
    st = lib().orc_deposit(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), _p(m), float(half_dt),
                           cfg.box, int(cfg.periodic), root_delta(cfg, grids), plan.level,
                           _p(_i64(plan.lo)), _p(_i64(plan.G)), plan.mode, cfg.mass_frac_bits,
                           _p(gmf))
    return gmf, st


def solve(cfg, grids, gi, gmf):
    """Phi_short on [-h, N+h)^3 ([z, y, x]) of grid gi (Sec. 2.2, readings R4-R6);
    with the spectral gradient (R15) a (4, ...) array: phi_short, A_x, A_y, A_z."""
    plan = plan_grid(cfg, grids, gi)
    T = green_table(cfg, plan)
    W = plan.W
    g = np.ascontiguousarray(gmf, dtype=np.int64)
    if cfg.gradient == "spectral":
        phis = np.zeros((4,) + W[::-1], dtype=np.float64)
        lib().orc_solve_spectral(_p(g), _p(_i64(plan.G)), cfg.mass_frac_bits, _p(_i64(plan.M)),
                                 _p(_i64(plan.s0)), _p(_i64(W)), _p(T), plan.delta, _p(phis),
                                 nthreads())
        return phis
    phis = np.zeros(W[::-1], dtype=np.float64)
    lib().orc_solve(_p(g), _p(_i64(plan.G)), cfg.mass_frac_bits, _p(_i64(plan.M)),
                    _p(_i64(plan.s0)), _p(_i64(W)), _p(T), _p(phis), nthreads())
    return phis


def accel(cfg, grids, gi, phis, parent_phi=None, parent_acc=None):
    """(phi, acc) on [-1, N+1)^3: gradient of Phi_short (R8, R15) plus trilinear
    parent carry."""
    plan = plan_grid(cfg, grids, gi)
    g = grids[gi]
    E = tuple(v + 2 for v in g.dims)
    phi = np.zeros(E[::-1], dtype=np.float64)
    acc = np.zeros((3,) + E[::-1], dtype=np.float64)
    if parent_phi is not None:
        pg = grids[g.parent]
        Np, pstart = _i64(pg.dims), _i64(pg.start)
        pphi = np.ascontiguousarray(parent_phi, dtype=np.float64)
        pacc = np.ascontiguousarray(parent_acc, dtype=np.float64)
    else:
        Np, pstart, pphi, pacc = _i64([1, 1, 1]), _i64([0, 0, 0]), None, None
    ps = np.ascontiguousarray(phis, dtype=np.float64)
    lib().orc_accel(_p(ps), _p(_i64(g.dims)), GRADIENTS[cfg.gradient], plan.delta,
                    _p(_i64(g.start)), _p(pphi), _p(pacc), _p(Np), _p(pstart), cfg.refine, _p(phi),
                    _p(acc))
    return phi, acc


def owners(cfg, grids, particles, half_dt):
    """Index of the finest grid whose interior holds each drifted particle, -1 if none
    (design reading C11)."""
    (x, y, z, vx, vy, vz, m), n = _parts(particles)
    own = np.full(n, -1, dtype=np.int32)
    own_level = np.full(n, -1, dtype=np.int32)
    N0 = grids[0].dims[0]
    levels = sorted(set(g.level for g in grids))
    cells = {}
    for lev in levels:
        c = np.zeros((3, n), dtype=np.int64)
        lib().orc_cells(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), float(half_dt), cfg.box,
                        int(cfg.periodic), root_delta(cfg, grids), lev, _p(c))
        cells[lev] = c
    for gi, g in enumerate(grids):
        c = cells[g.level]
        inside = np.ones(n, dtype=bool)
        for j in range(3):
            inside &= (c[j] >= g.start[j]) & (c[j] < g.start[j] + g.dims[j])
        better = inside & (own_level < g.level)
        own[better] = gi
        own_level[better] = g.level
    return own


def interp(cfg, grids, gi, acc, particles, half_dt, owner, out):
    """Writes out[:, p] (3 x n) for the particles owned by grid gi."""
    plan = plan_grid(cfg, grids, gi)
    g = grids[gi]
    (x, y, z, vx, vy, vz, m), n = _parts(particles)
    a = np.ascontiguousarray(acc, dtype=np.float64)
    own = np.ascontiguousarray(owner, dtype=np.int32)
    mode = 1 if plan.mode == 1 else 0
    lib().orc_interp(n, _p(x), _p(y), _p(z), _p(vx), _p(vy), _p(vz), float(half_dt), cfg.box,
                     int(cfg.periodic), root_delta(cfg, grids), plan.level, _p(_i64(g.start)),
                     _p(_i64(g.dims)), mode, _p(a), _p(own), int(gi), _p(out))


@dataclass
class StepResult:
    gmf: list = field(default_factory=list)
    phis: list = field(default_factory=list)
    phi: list = field(default_factory=list)
    acc: list = field(default_factory=list)
    owner: np.ndarray = None
    pacc: np.ndarray = None
    status: int = 0


def apm_step(cfg, grids, particles, half_dt, gas=None):
    """One full APM solve over the hierarchy, levels top-down (Sec. 2, 2.2).

    gas: None or a list (one entry per grid, None allowed) of interior densities."""
    ng = len(grids)
    res = StepResult(gmf=[None] * ng, phis=[None] * ng, phi=[None] * ng, acc=[None] * ng)
    levels = sorted(set(g.level for g in grids))
    for lev in levels:
        for gi, g in enumerate(grids):
            if g.level != lev:
                continue
            gg = None if gas is None else gas[gi]
            pg = None if (gas is None or g.parent < 0) else gas[g.parent]
            gmf, st = deposit(cfg, grids, gi, particles, half_dt, gg, pg)
            res.status |= st
            res.gmf[gi] = gmf
            res.phis[gi] = solve(cfg, grids, gi, gmf)
            if g.parent >= 0:
                res.phi[gi], res.acc[gi] = accel(cfg, grids, gi, res.phis[gi],
                                                 res.phi[g.parent], res.acc[g.parent])
            else:
                res.phi[gi], res.acc[gi] = accel(cfg, grids, gi, res.phis[gi])
    n = len(particles["x"])
    res.owner = owners(cfg, grids, particles, half_dt)
    res.pacc = np.zeros((3, n), dtype=np.float64)
    for gi in range(ng):
        interp(cfg, grids, gi, res.acc[gi], particles, half_dt, res.owner, res.pacc)
    return res
