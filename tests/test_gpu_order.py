"""The particle processing order (apm_reserve_order / apm_order_particles):
the interpolation (and, with apm_set_deposit_tiles, the deposit through its
shared-memory tiles) visit the particles bin by bin, and every output must be
bit-identical to the unordered calls, per level and for all
levels at once, in FP32 and FP64, also when the order was computed from other
positions (before a kick-drift)."""
import numpy as np
import pytest

from apm_inputs import GridDesc

pytestmark = pytest.mark.gpu

GRIDS = [GridDesc(0, -1, (0, 0, 0), (64, 64, 64)),
         GridDesc(1, 0, (20, 24, 28), (40, 44, 36)),
         GridDesc(1, 0, (70, 30, 70), (30, 30, 30)),
         GridDesc(2, 1, (50, 58, 66), (40, 40, 40))]


def _particles(n, seed):
    import torch
    rng = np.random.default_rng(seed)
    # clumps: most particles inside the refined grids, in random memory order
    pos = np.concatenate([0.05 + 0.9 * rng.random((3, n // 2)),
                          0.33 + 0.2 * rng.random((3, n - n // 2))], axis=1)
    v = rng.normal(scale=0.3, size=(3, n))
    m = (0.5 + rng.random(n)) / n
    d = {"x": pos[0], "y": pos[1], "z": pos[2], "vx": v[0], "vy": v[1], "vz": v[2], "m": m}
    return {k: torch.as_tensor(np.ascontiguousarray(a), device="cuda") for k, a in d.items()}


def _fields(bufs):
    return [t.clone() for b in bufs for key in ("gmf", "phis", "acc") for t in b[key]]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("batched", [True, False])
@pytest.mark.parametrize("tiles", [False, True])
def test_ordered_particle_calls_are_bit_identical(precision, batched, tiles):
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    n = 300000
    P = Particles(_particles(n, 17))
    s = Solver(GRIDS, periodic=True, precision=precision, device=0)
    bufs = s.alloc_all()
    pacc = torch.zeros((3, n), dtype=s.dtype, device="cuda")
    s.step(P, 2e-3, bufs, pacc, batched=batched)
    ref, ref_pacc = _fields(bufs), pacc.clone()
    s.set_deposit_tiles(tiles)
    s.reserve_order(n)
    s.profile(True)
    for b in bufs:
        for key in ("gmf", "phis", "acc"):
            for t in b[key]:
                t.fill_(-7)
    pacc.fill_(float("nan"))
    s.step(P, 2e-3, bufs, pacc, batched=batched)
    prof = s.profile_read()
    s.profile(False)
    s.sync_status()
    assert prof["particle_order"][0] == 1
    assert all(torch.equal(a, b) for a, b in zip(_fields(bufs), ref))
    assert torch.equal(pacc, ref_pacc)
    # an order computed before the particles moved still gives the exact result
    s.kick_drift(P, pacc, 4e-3)
    s.order_capacity = 0          # keep the old order: step() does not re-order
    s.step(P, 2e-3, bufs, pacc, batched=batched)
    moved, moved_pacc = _fields(bufs), pacc.clone()
    s.reserve_order(0)
    s.step(P, 2e-3, bufs, pacc, batched=batched)
    assert all(torch.equal(a, b) for a, b in zip(_fields(bufs), moved))
    assert torch.equal(pacc, moved_pacc)
    s.close()


def test_order_needs_a_large_enough_workspace():
    from paper_1410_0010_gb300._lib import ApmError
    from paper_1410_0010_gb300.solver import Particles, Solver
    n = 100000
    P = Particles(_particles(n, 3))
    s = Solver(GRIDS, periodic=True, precision="fp32", device=0)
    with pytest.raises(ApmError):
        s.order_particles(P, 0.0)        # no workspace reserved
    s.reserve_order(n - 1)
    with pytest.raises(ApmError):
        s.order_particles(P, 0.0)        # more particles than reserved
    s.reserve_order(n)
    s.order_particles(P, 0.0)
    s.sync_status()
    s.close()


@pytest.mark.parametrize("layout", ["clump", "stale"])
def test_ordered_deposit_tile_edge_cases(layout):
    """The ordered deposit's shared-memory tiles: every particle inside a few
    cells (all charges of a CTA land in the same tile cells, inside the
    level-2 grid), and an order left from positions that were then redrawn at
    random (a CTA's particles spread over the box, so most charges fall
    outside its tile and go straight to L2).  The mass fields must equal the
    unordered deposit's bit for bit, for the all-level and per-level calls."""
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    n = 200000
    rng = np.random.default_rng(29)
    d = _particles(n, 5)
    if layout == "clump":   # a cube of 2 root cells inside the level-2 grid
        for k in ("x", "y", "z"):
            d[k].copy_(torch.as_tensor(0.26 + (2.0 / 64) * rng.random(n), device="cuda"))
    P = Particles(d)
    s = Solver(GRIDS, periodic=True, precision="fp32", device=0)
    s.set_deposit_tiles(True)
    bufs = s.alloc_all()
    s.reserve_order(n)
    s.order_particles(P, 2e-3)
    if layout == "stale":
        for k in ("x", "y", "z"):
            d[k].copy_(torch.as_tensor(rng.random(n), device="cuda"))
    gmf = s._per_grid(bufs, "gmf")
    s.deposit_all(P, 2e-3, gmf, None)
    ordered = [t.clone() for t in gmf]
    for lev in range(s.n_levels):
        s.deposit(lev, P, 2e-3, bufs[lev]["gmf"])
    per_level = [t.clone() for t in gmf]
    s.reserve_order(0)
    s.deposit_all(P, 2e-3, gmf, None)
    s.sync_status()
    assert all(torch.equal(a, b) for a, b in zip(ordered, gmf))
    assert all(torch.equal(a, b) for a, b in zip(per_level, gmf))
    assert sum(int(t.abs().sum()) > 0 for t in ordered) >= 3   # root, level-1 and level-2 grids
    s.close()


def test_deposit_tiles_flag_is_validated():
    from paper_1410_0010_gb300._lib import ApmError, lib
    from paper_1410_0010_gb300.solver import Solver
    s = Solver(GRIDS, periodic=True, precision="fp32", device=0)
    assert lib().apm_set_deposit_tiles(s._ctx, 2) != 0
    s.set_deposit_tiles(True)
    s.set_deposit_tiles(False)
    with pytest.raises(ApmError):
        from paper_1410_0010_gb300._lib import check
        check(lib().apm_set_deposit_tiles(s._ctx, -1), "apm_set_deposit_tiles")
    s.close()
