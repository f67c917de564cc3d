"""GPU parity of the CUDA path (through the C ABI) against the oracle on seeded
inputs: deposit bit-exact, FP64 within 1e-12 and FP32 within 2e-5 / 1e-4
(relative L2), over grids spanning several FFT tiles with ragged tails, every
radix, odd FFT lengths, overlapping GMF borders, border baryons from the parent,
periodic and isolated roots, and the edge cases of the method."""
import numpy as np
import pytest

import apm_inputs as W
from apm_inputs import GridDesc
from gpu_helpers import compare, rel_l2, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

PRECISIONS = ["fp64", "fp32"]


def _random_particles(rng, n, lo=0.0, hi=1.0, vscale=1.0, mass=1.0):
    pos = lo + (hi - lo) * rng.random((3, n))
    v = rng.normal(scale=vscale, size=(3, n))
    return dict(x=pos[0], y=pos[1], z=pos[2], vx=v[0], vy=v[1], vz=v[2],
                m=mass * (0.5 + rng.random(n)))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_isolated_root32_4096_particles(precision):
    w = W.config_isolated_root32()
    ref = run_oracle(w.grids, w.particles, w.half_dt)
    gpu = run_gpu(w.grids, w.particles, w.half_dt, precision=precision)
    compare(gpu, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_two_level_isolated_gas_and_drift(precision):
    w = W.config_two_level()
    ref = run_oracle(w.grids, w.particles, w.half_dt, gas=w.gas)
    gpu = run_gpu(w.grids, w.particles, w.half_dt, gas=w.gas, precision=precision)
    compare(gpu, ref, precision)


def _periodic_hierarchy():
    # two level-1 siblings whose GMF borders overlap, and a level-2 grid
    return [GridDesc(0, -1, (0, 0, 0), (24, 24, 24)),
            GridDesc(1, 0, (8, 8, 10), (14, 12, 16)),
            GridDesc(1, 0, (22, 8, 12), (18, 14, 10)),
            GridDesc(2, 1, (24, 24, 28), (12, 10, 14))]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_periodic_root_siblings_and_grandchild(precision):
    grids = _periodic_hierarchy()
    rng = np.random.default_rng(11)
    parts = W.concat_particles(_random_particles(rng, 300, vscale=0.5),
                               _random_particles(rng, 300, 0.2, 0.55, vscale=0.5),
                               _random_particles(rng, 100, 0.97, 1.0, vscale=2.0))
    gas = [rng.random(g.dims[::-1]) + 0.1 for g in grids]
    ref = run_oracle(grids, parts, 2e-3, gas=gas, periodic=True)
    gpu = run_gpu(grids, parts, 2e-3, gas=gas, periodic=True, precision=precision)
    compare(gpu, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_odd_and_mixed_fft_lengths(precision):
    # dims + 20 = 45, 49, 63 / 75, 81, 36: radices 3, 5, 7 and odd lengths
    grids = [GridDesc(0, -1, (0, 0, 0), (48, 48, 48)),
             GridDesc(1, 0, (10, 12, 14), (25, 29, 43)),
             GridDesc(1, 0, (10, 44, 62), (55, 26, 16))]
    rng = np.random.default_rng(12)
    parts = W.concat_particles(_random_particles(rng, 400, 0.1, 0.9, vscale=0.1),
                               _random_particles(rng, 400, 0.15, 0.5, vscale=0.1))
    gas = [None, rng.random((43, 29, 25)), None]
    ref = run_oracle(grids, parts, 1e-3, gas=gas)
    gpu = run_gpu(grids, parts, 1e-3, gas=gas, precision=precision)
    for gi in (1, 2):
        assert tuple(gpu["info"][gi]["fft"]) in ((45, 49, 63), (75, 48, 36))
    compare(gpu, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_odd_starts_odd_root_and_grandchild(precision):
    """Odd interior starts and sizes on every axis: the parent carry pairs level
    cells (2k+1, 2k+2) between the same parent centres, so odd starts put the
    first and last cell of a row in half-filled pairs; the isolated root has an
    odd N (21, M = 42)."""
    grids = [GridDesc(0, -1, (0, 0, 0), (21, 21, 21)),
             GridDesc(1, 0, (9, 11, 13), (15, 12, 9)),
             GridDesc(1, 0, (27, 7, 25), (9, 17, 11)),
             GridDesc(2, 1, (25, 27, 31), (11, 9, 7))]
    rng = np.random.default_rng(13)
    parts = W.concat_particles(_random_particles(rng, 500, 0.05, 0.95, vscale=0.2),
                               _random_particles(rng, 300, 0.3, 0.42, vscale=0.2))
    gas = [None, rng.random((9, 12, 15)) + 0.2, None, rng.random((7, 9, 11)) + 0.2]
    ref = run_oracle(grids, parts, 1e-3, gas=gas)
    gpu = run_gpu(grids, parts, 1e-3, gas=gas, precision=precision)
    compare(gpu, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_borders_past_an_isolated_root(precision):
    """Level-1 grids at the faces of an isolated 24^3 root: their GMF borders
    reach past the box (no baryons there), the carry stays inside; a level-2
    grid below one of them; gas everywhere and particles crowding the faces."""
    grids = [GridDesc(0, -1, (0, 0, 0), (24, 24, 24)),
             GridDesc(1, 0, (2, 3, 36), (12, 10, 10)),
             GridDesc(1, 0, (30, 30, 2), (16, 14, 12)),
             GridDesc(2, 1, (9, 11, 78), (14, 10, 8))]
    rng = np.random.default_rng(29)
    near = _random_particles(rng, 400, 0.002, 0.3, vscale=0.1)
    near["z"] = 0.75 + 0.248 * rng.random(400)
    far = _random_particles(rng, 400, 0.6, 0.998, vscale=0.1)
    far["z"] = 0.002 + 0.248 * rng.random(400)
    parts = W.concat_particles(near, far, _random_particles(rng, 300, 0.02, 0.98, vscale=0.1))
    gas = [rng.random(g.dims[::-1]) + 0.1 for g in grids]
    ref = run_oracle(grids, parts, 1e-3, gas=gas)
    gpu = run_gpu(grids, parts, 1e-3, gas=gas, precision=precision)
    compare(gpu, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("pad_factor,a_over_dx", [(0.3, 3.4), (0.15, 2.5), (1.0, 5.0)])
def test_padding_and_softening_parameters(precision, pad_factor, a_over_dx):
    """The accuracy studies' parameters: border B = ceil(pad 2 a/delta) from 2 to
    10 cells (down to fewer than the window's 2 extra cells) and a/delta from
    2.5 to 5, on an isolated root with a child and a grandchild."""
    grids = [GridDesc(0, -1, (0, 0, 0), (32, 32, 32)),
             GridDesc(1, 0, (22, 20, 24), (20, 22, 18)),
             GridDesc(2, 1, (58, 54, 60), (12, 14, 10))]
    rng = np.random.default_rng(17)
    parts = W.concat_particles(_random_particles(rng, 600, 0.1, 0.9, vscale=0.2),
                               _random_particles(rng, 300, 0.4, 0.6, vscale=0.2))
    gas = [None, rng.random((18, 22, 20)) + 0.2, None]
    ref = run_oracle(grids, parts, 1e-3, gas=gas, pad_factor=pad_factor, a_over_dx=a_over_dx)
    gpu = run_gpu(grids, parts, 1e-3, gas=gas, precision=precision, pad_factor=pad_factor,
                  a_over_dx=a_over_dx)
    compare(gpu, ref, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_all_level_calls_equal_per_level_calls_bitwise(precision):
    """apm_deposit_all / apm_interp_all against apm_deposit / apm_interp level by
    level on a three-level periodic hierarchy with gas and particles everywhere
    (including outside every refined grid and in the grandchild)."""
    grids = _periodic_hierarchy()
    rng = np.random.default_rng(14)
    parts = W.concat_particles(_random_particles(rng, 800, vscale=0.5),
                               _random_particles(rng, 400, 0.3, 0.6, vscale=0.5))
    gas = [rng.random(g.dims[::-1]) + 0.1 for g in grids]
    a = run_gpu(grids, parts, 2e-3, gas=gas, periodic=True, precision=precision, batched=True)
    b = run_gpu(grids, parts, 2e-3, gas=gas, periodic=True, precision=precision, batched=False)
    for gi in a["gmf"]:
        assert np.array_equal(a["gmf"][gi], b["gmf"][gi]), gi
        assert np.array_equal(a["acc"][gi], b["acc"][gi]), gi
    assert np.array_equal(a["pacc"], b["pacc"])


def test_edge_particles_faces_corners_border_and_outside():
    grids = [GridDesc(0, -1, (0, 0, 0), (16, 16, 16)), GridDesc(1, 0, (10, 10, 10), (8, 8, 8))]
    d0, d1 = 1 / 16, 1 / 32
    xs = [5 * d1, 10 * d1, 13 * d1, 14.5 * d1, 18 * d1, 8 * d1, 0.0, 15 * d0, 1.0 - 1e-16]
    parts = dict(x=np.array(xs), y=np.array(xs[::-1]), z=np.array(xs[2:] + xs[:2]),
                 vx=np.zeros(len(xs)), vy=np.zeros(len(xs)), vz=np.zeros(len(xs)),
                 m=np.linspace(0.5, 1.5, len(xs)))
    ref = run_oracle(grids, parts, 0.0)
    gpu = run_gpu(grids, parts, 0.0, precision="fp64")
    compare(gpu, ref, "fp64")


def test_particle_outside_isolated_box_is_flagged_and_folded():
    from paper_1410_0010_gb300 import ApmError
    grids = [GridDesc(0, -1, (0, 0, 0), (8, 8, 8))]
    parts = dict(x=np.array([1.3, 0.5]), y=np.array([0.5, 0.5]), z=np.array([0.5, 0.2]),
                 vx=np.zeros(2), vy=np.zeros(2), vz=np.zeros(2), m=np.array([1.0, 2.0]))
    with pytest.raises(ApmError, match="OUT_OF_BOX"):
        run_gpu(grids, parts, 0.0, precision="fp64")


def test_fixed_point_overflow_is_flagged():
    from paper_1410_0010_gb300 import ApmError
    grids = [GridDesc(0, -1, (0, 0, 0), (8, 8, 8))]
    parts = dict(x=np.array([0.5]), y=np.array([0.5]), z=np.array([0.5]), vx=np.zeros(1),
                 vy=np.zeros(1), vz=np.zeros(1), m=np.array([4096.0]))
    with pytest.raises(ApmError, match="OVERFLOW"):
        run_gpu(grids, parts, 0.0, precision="fp64")


def test_no_particles_and_empty_grid():
    grids = [GridDesc(0, -1, (0, 0, 0), (16, 16, 16)), GridDesc(1, 0, (10, 10, 10), (8, 8, 8))]
    z = np.zeros(0)
    parts = dict(x=z, y=z, z=z, vx=z, vy=z, vz=z, m=z)
    rng = np.random.default_rng(3)
    gas = [rng.random((16, 16, 16)), None]
    ref = run_oracle(grids, parts, 0.0, gas=gas)
    gpu = run_gpu(grids, parts, 0.0, gas=gas, precision="fp64")
    compare(gpu, ref, "fp64", check_pacc=False)


def test_deposit_is_order_independent_bitwise():
    grids = _periodic_hierarchy()
    rng = np.random.default_rng(13)
    parts = W.concat_particles(_random_particles(rng, 2000), _random_particles(rng, 2000, 0.2, 0.55))
    a = run_gpu(grids, parts, 1e-3, periodic=True, precision="fp32")
    perm = rng.permutation(len(parts["x"]))
    b = run_gpu(grids, {k: v[perm] for k, v in parts.items()}, 1e-3, periodic=True, precision="fp32")
    for gi in a["gmf"]:
        assert np.array_equal(a["gmf"][gi], b["gmf"][gi])
    assert rel_l2(a["pacc"][:, perm], b["pacc"]) < 1e-6


def _x_rows(rng, n_rows, per_row, n_cells, spacing=2.0, jitter=0.3, lo=0.0, hi=1.0, wrap=True):
    """Rows of particles stored x-fastest, `spacing` cells apart along x with a
    small jitter (some neighbours 1 or 3 cells apart), each row at a random
    (y, z) inside [lo, hi) and a random x start (wrapping past 1 when `wrap`)."""
    d = 1.0 / n_cells
    xs, ys, zs = [], [], []
    for _ in range(n_rows):
        x0 = rng.random() if wrap else lo + 0.1 * (hi - lo) * rng.random()
        y0, z0 = lo + (hi - lo) * rng.random(), lo + (hi - lo) * rng.random()
        x = x0 + d * (spacing * np.arange(per_row) + jitter * rng.standard_normal(per_row))
        xs.append(np.mod(x, 1.0) if wrap else np.clip(x, lo, hi - 1e-9))
        ys.append(np.full(per_row, y0))
        zs.append(np.full(per_row, z0))
    x, y, z = (np.concatenate(a) for a in (xs, ys, zs))
    n = len(x)
    return dict(x=x, y=y, z=z, vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n))


@pytest.mark.parametrize("periodic", [True, False])
def test_root_deposit_of_x_ordered_particles_bit_exact(periodic):
    """The root deposit merges the charges that x-neighbouring lanes give the
    same cells (one reduction instead of two).  Rows of particles two cells
    apart (some one or three) exercise it: rows that wrap the periodic root,
    rows whose clouds fold at an isolated root's faces, warps mixing the
    32-bit and 64-bit product widths, a ragged last warp, and a refined level
    below the root.  The mass field stays bit-exact against the oracle."""
    rng = np.random.default_rng(21 if periodic else 22)
    n_cells = 24
    grids = [GridDesc(0, -1, (0, 0, 0), (n_cells,) * 3), GridDesc(1, 0, (12, 10, 14), (16, 16, 12))]
    if periodic:
        parts = _x_rows(rng, 37, 29, n_cells)
    else:
        # rows hugging the low and high faces: their clouds fold onto the edge cells
        edge = 0.5 / n_cells
        parts = W.concat_particles(_x_rows(rng, 20, 11, n_cells, lo=edge, hi=1.0 - edge, wrap=False),
                                   _x_rows(rng, 17, 9, n_cells, spacing=1.0, lo=0.0, hi=1.0, wrap=False))
        for k in ("y", "z"):
            sel = rng.random(len(parts[k])) < 0.3
            parts[k][sel] = np.where(rng.random(sel.sum()) < 0.5, 0.2 / n_cells, 1.0 - 0.2 / n_cells)
    n = len(parts["x"])
    # most masses below 2^-20 (32-bit products at 52 fraction bits), some not
    m = np.full(n, 2.0 ** -24) * (1.0 + rng.random(n))
    m[rng.random(n) < 0.05] = 0.25
    parts["m"] = m
    ref = run_oracle(grids, parts, 0.0, periodic=periodic)
    gpu = run_gpu(grids, parts, 0.0, periodic=periodic, precision="fp64")
    compare(gpu, ref, "fp64")
    per_level = run_gpu(grids, parts, 0.0, periodic=periodic, precision="fp64", batched=False)
    for gi in gpu["gmf"]:
        assert np.array_equal(gpu["gmf"][gi], per_level["gmf"][gi]), gi


def test_sine_wave_periodic_mode_matches_closed_form_on_gpu():
    """Sec. 3.4 on the GPU: the FP64 path reproduces the single-mode solution."""
    import oracle
    grids = [GridDesc(0, -1, (0, 0, 0), (32, 32, 32))]
    gas = W.sine_wave_gas(grids, 0.25, axis=1)
    z = np.zeros(0)
    parts = dict(x=z, y=z, z=z, vx=z, vy=z, vz=z, m=z)
    gpu = run_gpu(grids, parts, 0.0, gas=gas, periodic=True, precision="fp64", mass_frac_bits=60)
    d = 1 / 32
    Gk = oracle.green_opt((0, 4, 0), (32, 32, 32), d, 3.4 * d, 0.0, 0)
    yc = (np.arange(32) + 0.5) * d
    phi = gpu["phi"][0][1:-1, 1:-1, 1:-1]
    exp = Gk * np.sin(2 * np.pi * yc / 0.25)
    assert np.max(np.abs(phi - exp[None, :, None])) < 1e-11 * np.max(np.abs(exp))
