"""Seeded synthetic workloads (see the package docstring).

A grid is described by the plain tuple GridDesc(level, parent, start, dims):
level 0 is the root (one grid, covering the whole box); `start` is the global
level-l cell index of the grid's first interior cell and `dims` its interior
cell counts, both (x, y, z).  Densities are numpy arrays indexed [z, y, x].
Particles are a dict of float64 arrays x, y, z, vx, vy, vz, m.
"""
import math
from collections import namedtuple
from dataclasses import dataclass, field

import numpy as np

GridDesc = namedtuple("GridDesc", "level parent start dims")

# nesting margin, in parent cells, between a child's interior and the edge of
# its parent's interior (a child's mass border of 5 cells is 2.5 parent cells)
NEST_MARGIN = 3


@dataclass
class Workload:
    name: str
    periodic: bool
    grids: list
    particles: dict
    gas: list = None               # per grid interior density, or None
    half_dt: float = 0.0
    mass_frac_bits: int = 52
    solve_levels: list = None      # levels that are solved (None: all)
    spatial_order: bool = False    # the particles are stored in spatial order (a lattice)
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_particles(self):
        return int(len(self.particles["x"]))

    def interior_cells(self, levels=None):
        lv = self.solve_levels if levels is None else levels
        return int(sum(int(np.prod(g.dims)) for g in self.grids if lv is None or g.level in lv))



# workload key -> name (the names the benchmark reports and keys its DRAM
# traffic file by)
NAMES = {
    "c1": "isolated_root32_p4096",
    "c2": "two_level_iso64",
    "c3": "periodic128_3lev_plummer1M",
    "c4": "batched512_level",
    "c5": "cosmo512_2lev_zeldovich16M",
    "c5s": "cosmo256_2lev_zeldovich2M",
}

def _particles(x, y, z, vx=None, vy=None, vz=None, m=None):
    n = len(x)
    z0 = np.zeros(n)
    return dict(x=np.ascontiguousarray(x, dtype=np.float64),
                y=np.ascontiguousarray(y, dtype=np.float64),
                z=np.ascontiguousarray(z, dtype=np.float64),
                vx=np.ascontiguousarray(z0 if vx is None else vx, dtype=np.float64),
                vy=np.ascontiguousarray(z0 if vy is None else vy, dtype=np.float64),
                vz=np.ascontiguousarray(z0 if vz is None else vz, dtype=np.float64),
                m=np.ascontiguousarray(m, dtype=np.float64))


def concat_particles(*ps):
    return {k: np.concatenate([p[k] for p in ps]) for k in ps[0]}


def grids_from_bounds(root_n, bounds, refine=2):
    """Nested chain of grids from physical bounds [lo, hi]^3 per level (Sec. 3 setups)."""
    grids = [GridDesc(0, -1, (0, 0, 0), (root_n,) * 3)]
    for lev, (lo, hi) in enumerate(bounds, start=1):
        n_l = root_n * refine ** lev
        s = int(round(lo * n_l))
        e = int(round(hi * n_l))
        grids.append(GridDesc(lev, lev - 1, (s,) * 3, (e - s,) * 3))
    return grids


# ----------------------------------------------------------------------------
# Hierarchies of the paper's tests (Sec. 2.2 Fig. 1, Sec. 3.1-3.5)
# ----------------------------------------------------------------------------
FIG1_BOUNDS = [(0.1875, 0.8125), (0.3125, 0.6875), (0.40625, 0.59375)]   # Sec. 2.2, 3.1
POINT_SOURCE_CENTRE = [(0.4375, 0.5625)]                                  # Sec. 3.2
POINT_SOURCE_CORNER = [(0.5, 0.5625)]                                     # Sec. 3.2
SINE_WAVE_BOUNDS = [(0.34375, 0.65625), (0.421875, 0.578125)]            # Sec. 3.4


def uniform_sphere_gas(grids, radius=0.3, rho0=1.0, rho_out=1e-10, box=1.0, centre=0.5):
    """Sec. 3.3 case i = 1: rho0 inside r <= R, rho_out outside, at cell centres."""
    out = []
    N0 = grids[0].dims[0]
    for g in grids:
        d = box / (N0 * 2 ** g.level)
        ax = [(np.arange(g.dims[j]) + g.start[j] + 0.5) * d - centre for j in range(3)]
        zz, yy, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        r = np.sqrt(xx * xx + yy * yy + zz * zz)
        out.append(np.where(r <= radius, rho0, rho_out))
    return out


def sine_wave_gas(grids, period, axis=0, box=1.0):
    """Sec. 3.4: rho = 2 + sin(2 pi x / P) at cell centres (along `axis`)."""
    out = []
    N0 = grids[0].dims[0]
    for g in grids:
        d = box / (N0 * 2 ** g.level)
        c = (np.arange(g.dims[axis]) + g.start[axis] + 0.5) * d
        prof = 2.0 + np.sin(2.0 * np.pi * c / period)
        shape = [1, 1, 1]
        shape[2 - axis] = g.dims[axis]
        full = np.broadcast_to(prof.reshape(shape), tuple(g.dims[::-1]))
        out.append(np.ascontiguousarray(full, dtype=np.float64))
    return out


# ----------------------------------------------------------------------------
# Benchmark-shaped configurations
# ----------------------------------------------------------------------------
def config_isolated_root32(seed=1):
    """Isolated 32^3 root (zero-padded to 64^3), 4096 equal-mass uniform particles, no gas."""
    rng = np.random.default_rng(seed)
    n = 4096
    pos = rng.random((3, n))
    grids = [GridDesc(0, -1, (0, 0, 0), (32, 32, 32))]
    return Workload(NAMES["c1"], False, grids,
                    _particles(pos[0], pos[1], pos[2], m=np.full(n, 1.0 / n)),
                    notes="uniform positions, m = 1/4096, no drift")


def _gaussian(x, y, z, sigma):
    return np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) / (2.0 * sigma * sigma))


def config_two_level(seed=2):
    """Isolated 64^3 root + centred 64^3 child (R = 2); two point masses 1 : 0.1
    eight child cells apart plus a Gaussian gas sphere (sigma = 6 root cells,
    peak 1); random velocities drifted half a timestep (dt = 3e-3, Sec. 3.5)."""
    rng = np.random.default_rng(seed)
    grids = [GridDesc(0, -1, (0, 0, 0), (64, 64, 64)),
             GridDesc(1, 0, (32, 32, 32), (64, 64, 64))]
    x = np.array([0.5, 0.5 + 8.0 / 128.0])
    y = np.array([0.5, 0.5])
    z = np.array([0.5, 0.5])
    v = rng.uniform(-1.0, 1.0, size=(3, 2))
    parts = _particles(x, y, z, v[0], v[1], v[2], m=np.array([1.0, 0.1]))
    sigma = 6.0 / 64.0
    # child: sampled at child cell centres
    dc = 1.0 / 128.0
    ax = (np.arange(64) + 32 + 0.5) * dc
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    gas_c = _gaussian(xx, yy, zz, sigma)
    # root: sampled at root cell centres, replaced by the mean of the 8 child
    # cells where the child covers it (so both levels hold the same mass)
    d0 = 1.0 / 64.0
    ax0 = (np.arange(64) + 0.5) * d0
    zz, yy, xx = np.meshgrid(ax0, ax0, ax0, indexing="ij")
    gas_r = _gaussian(xx, yy, zz, sigma)
    restr = gas_c.reshape(32, 2, 32, 2, 32, 2).mean(axis=(1, 3, 5))
    gas_r[16:48, 16:48, 16:48] = restr
    return Workload(NAMES["c2"], False, grids, parts, gas=[gas_r, gas_c],
                    half_dt=1.5e-3, notes="Gaussian gas, two particles, half-step drift")


def _densest_cell(cells, lo, hi):
    """Densest cell (nearest-grid-point counts) among integer cells in [lo, hi)."""
    m = np.all((cells >= lo[:, None]) & (cells < hi[:, None]), axis=0)
    c = cells[:, m] - lo[:, None]
    ext = hi - lo
    lin = c[0] + ext[0] * (c[1] + ext[1] * c[2])
    cnt = np.bincount(lin, minlength=int(np.prod(ext)))
    best = int(np.argmax(cnt))   # ties: lowest linear index
    return lo + np.array([best % ext[0], (best // ext[0]) % ext[1], best // (ext[0] * ext[1])])


def _centred_child(pc, child_n, pstart, pdims, refine=2):
    """Start (child cells) of a child of child_n cells centred on parent cell pc,
    aligned to parent cells and clamped to the nesting margin."""
    half = child_n // (2 * refine)
    span = child_n // refine
    lo = pstart + NEST_MARGIN
    hi = pstart + pdims - NEST_MARGIN - span
    ps = np.clip(pc - half, lo, hi)
    return tuple(int(v) for v in refine * ps)


def config_plummer(seed=3, n=1 << 20, levels=3, child_n=64, root_n=128):
    """Periodic 128^3 root + 3 nested 64^3 levels, each centred on the densest cell
    of its parent; Plummer sphere of scale 4 root cells, m = 1/n."""
    rng = np.random.default_rng(seed)
    a = 4.0 / root_n
    X = rng.random(n)
    X = np.where(X <= 0.0, 1e-300, X)
    r = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
    u = rng.normal(size=(3, n))
    u /= np.linalg.norm(u, axis=0)
    pos = np.mod(0.5 + r * u, 1.0)
    v = rng.normal(scale=0.1, size=(3, n))
    parts = _particles(pos[0], pos[1], pos[2], v[0], v[1], v[2], m=np.full(n, 1.0 / n))
    grids = [GridDesc(0, -1, (0, 0, 0), (root_n,) * 3)]
    for lev in range(1, levels + 1):
        par = grids[-1]
        pn = root_n * 2 ** (lev - 1)
        cells = np.floor(pos * pn).astype(np.int64)
        pc = _densest_cell(cells, np.array(par.start), np.array(par.start) + np.array(par.dims))
        st = _centred_child(pc, child_n, np.array(par.start), np.array(par.dims))
        grids.append(GridDesc(lev, lev - 1, st, (child_n,) * 3))
    return Workload(NAMES["c3"], True, grids, parts, half_dt=1e-3,
                    notes="Plummer sphere, scale radius 4 root cells")


def config_batched_level(seed=4, n_grids=512, root_n=512):
    """One refined level of 512 subgrids (per-axis sizes log-uniform in [16, 64]),
    each with lognormal gas (sigma_ln = 1) over its interior and 2000-20000
    uniform particles whose total mass equals the interior gas mass.  The
    subgrids sit in an 8^3 lattice of 128-cell slots of level 1 (delta = 1/1024)
    inside an isolated 512^3 root that only serves as their parent."""
    rng = np.random.default_rng(seed)
    grids = [GridDesc(0, -1, (0, 0, 0), (root_n,) * 3)]
    d1 = 1.0 / (root_n * 2)
    side = int(round(n_grids ** (1.0 / 3.0)))
    assert side ** 3 == n_grids
    slot = (root_n * 2) // side
    gas, xs, ys, zs, ms = [None], [], [], [], []
    for gk in range(n_grids):
        ix, iy, iz = gk % side, (gk // side) % side, gk // (side * side)
        dims = tuple(int(round(math.exp(rng.uniform(math.log(16), math.log(64))))) for _ in range(3))
        start = []
        for j, sl in enumerate((ix, iy, iz)):
            free = slot - dims[j] - 16
            off = 8 + 2 * int(rng.integers(0, free // 2 + 1))
            start.append(sl * slot + off)
        grids.append(GridDesc(1, 0, tuple(start), dims))
        g = np.exp(rng.normal(size=dims[::-1]) - 0.5)
        gas.append(g)
        npart = int(rng.integers(2000, 20001))
        mass = float(g.sum()) * d1 ** 3
        lo = np.array(start) * d1
        ext = np.array(dims) * d1
        p = lo[:, None] + rng.random((3, npart)) * ext[:, None]
        xs.append(p[0]); ys.append(p[1]); zs.append(p[2])
        ms.append(np.full(npart, mass / npart))
    parts = _particles(np.concatenate(xs), np.concatenate(ys), np.concatenate(zs),
                       m=np.concatenate(ms))
    return Workload(NAMES["c4"], False, grids, parts, gas=gas, solve_levels=[1],
                    mass_frac_bits=60,
                    notes="short-range level solve only; the root is the container")


def zeldovich_lattice(n_side, seed, rms_spacing=0.5, box=1.0):
    """Lattice of n_side^3 particles displaced by a Gaussian random field with
    P(k) ~ k^-2 (Zel'dovich: psi = grad laplacian^-1 delta), rms displacement
    rms_spacing lattice spacings.  Returns positions and displacements (3, n)."""
    rng = np.random.default_rng(seed)
    n = n_side
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(k1, k1, kr, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    amp = np.sqrt(1.0 / k2)                      # sqrt(P(k)), P ~ k^-2
    dk = (rng.normal(size=k2.shape) + 1j * rng.normal(size=k2.shape)) * amp
    dk[0, 0, 0] = 0.0
    disp = []
    for kc in (kx, ky, kz):
        disp.append(np.fft.irfftn(1j * kc / k2 * dk, s=(n, n, n), axes=(0, 1, 2)).astype(np.float64))
    del dk
    disp = np.stack([d.reshape(-1) for d in disp])
    rms = np.sqrt(np.mean(np.sum(disp * disp, axis=0)))
    disp *= (rms_spacing * box / n) / rms
    q = (np.arange(n) + 0.5) * (box / n)
    qz, qy, qx = np.meshgrid(q, q, q, indexing="ij")
    pos = np.stack([qx.reshape(-1), qy.reshape(-1), qz.reshape(-1)]) + disp
    return np.mod(pos, box), disp


def _place_greedy(centres, counts, n_grids, span, pstart, pdims):
    """Greedy placement of n_grids boxes of `span` parent cells centred on the
    densest candidate cells (ties: lowest index), interiors not overlapping,
    each clamped to the nesting margin.  Returns the boxes' start cells."""
    order = np.lexsort((np.arange(len(counts)), -counts))
    lo_lim = pstart + NEST_MARGIN
    hi_lim = pstart + pdims - NEST_MARGIN - span
    bs = np.zeros((0, 3), np.int64)
    for idx in order:
        s = np.clip(centres[:, idx] - span // 2, lo_lim, hi_lim)
        if len(bs) and np.any(np.all((s[None, :] < bs + span) & (bs < (s + span)[None, :]), axis=1)):
            continue
        bs = np.vstack([bs, s[None, :]])
        if len(bs) == n_grids:
            break
    return [tuple(int(v) for v in b) for b in bs]


def _block_counts(pos_cells, lo, n_blocks, block):
    """Nearest-grid-point particle counts on n_blocks^3 blocks of `block` cells
    starting at cell lo; returns (block centre cells (3, nb), counts)."""
    b = (pos_cells - lo[:, None]) // block
    ok = np.all((b >= 0) & (b < n_blocks), axis=0)
    b = b[:, ok]
    cnt = np.bincount(b[0] + n_blocks * (b[1] + n_blocks * b[2]), minlength=n_blocks ** 3)
    i = np.arange(n_blocks ** 3)
    ctr = np.stack([i % n_blocks, (i // n_blocks) % n_blocks, i // (n_blocks * n_blocks)])
    return lo[:, None] + ctr * block + block // 2, cnt


def config_cosmo512(seed=5, root_n=512, lattice=256, n_sub=64, sub_n=128):
    """Periodic 512^3 root, 256^3 = 16,777,216 particles on a lattice displaced
    by a P(k) ~ k^-2 Gaussian field (Zel'dovich), m = 2^-24, plus two refined
    levels of 64 subgrids of 128^3 each placed greedily on the densest regions
    (particle counts on blocks of 8 parent cells)."""
    pos, disp = zeldovich_lattice(lattice, seed)
    n = pos.shape[1]
    vel = 10.0 * disp
    parts = _particles(pos[0], pos[1], pos[2], vel[0], vel[1], vel[2], m=np.full(n, 1.0 / n))
    del vel, disp
    grids = [GridDesc(0, -1, (0, 0, 0), (root_n,) * 3)]
    span = sub_n // 2
    blk = 8
    c0 = np.floor(pos * root_n).astype(np.int64)
    ctr, cnt = _block_counts(c0, np.zeros(3, np.int64), root_n // blk, blk)
    for s in _place_greedy(ctr, cnt, n_sub, span, np.zeros(3, np.int64),
                           np.full(3, root_n, np.int64)):
        grids.append(GridDesc(1, 0, tuple(2 * v for v in s), (sub_n,) * 3))
    del c0
    c1 = np.floor(pos * (root_n * 2)).astype(np.int64)
    for gi in range(1, len(grids)):
        par = grids[gi]
        pst = np.array(par.start, np.int64)
        pdm = np.array(par.dims, np.int64)
        m = np.all((c1 >= pst[:, None]) & (c1 < (pst + pdm)[:, None]), axis=0)
        ctr, cnt = _block_counts(c1[:, m], pst, int(pdm[0]) // (2 * blk), 2 * blk)
        best = int(np.argmax(cnt))
        st = _centred_child(ctr[:, best], sub_n, pst, pdm)
        grids.append(GridDesc(2, gi, st, (sub_n,) * 3))
    return Workload(NAMES["c5"], True, grids, parts, half_dt=5e-4, spatial_order=True,
                    notes="Zel'dovich lattice, P(k) ~ k^-2, v = 10 psi")


def config_cosmo_small(seed=6):
    """Reduced cosmological workload for profiling captures: periodic 256^3 root,
    128^3 = 2,097,152 Zel'dovich particles, two levels of 8 subgrids of 128^3
    (inputs still larger than the 129 MB L2: 134 MB root mass field + particles)."""
    w = config_cosmo512(seed=seed, root_n=256, lattice=128, n_sub=8, sub_n=128)
    w.name = NAMES["c5s"]
    return w


CONFIGS = {
    "c1": config_isolated_root32,
    "c2": config_two_level,
    "c3": config_plummer,
    "c4": config_batched_level,
    "c5": config_cosmo512,
    "c5s": config_cosmo_small,
}
