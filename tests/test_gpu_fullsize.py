"""Parity at the benchmark sizes, in the launch configuration bench.py times
(every grid of a level batched in one launch sequence, FP32 path).

* periodic 128^3 root + three 64^3 levels, 2^20 Plummer particles: the whole
  solve against the oracle, element by element, for every gradient operator;
* 512 batched subgrids of one level with gas: every grid on the GPU, a sample
  of grids (GMF bit-exact, potential, accelerations) against the oracle, for
  every gradient operator;
  The sampled grids' particle accelerations against the oracle's
  interpolation of its own accelerations;
* periodic 512^3 root + 2 x 64 subgrids of 128^3, 16.8M particles: root GMF
  bit-exact against the oracle's full deposit; the whole 512^3 root potential,
  element by element, against the oracle's solve in its textbook-FFT mode; the
  root potential mode by mode; two 128^3 subgrids solved fully by the oracle;
  the chain root -> level 1 -> level 2 through the oracle's own carry on the
  level-2 grid holding the most particles, its level-1 parent and that
  parent's 64^3 footprint on the root, with the particle accelerations they
  own; FD, parent carry and particle interpolation on samples;
* the periodic 128^3 + three levels hierarchy in FP64 against the oracle at
  the FP64 tolerance, and its deposit through shared-memory tiles (particles
  in bin order) bit-exact against the direct deposit.
"""
import numpy as np
import pytest

import apm_inputs as W
from gpu_helpers import TOL, compare, rel_l2, run_gpu, run_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def plummer():
    w = W.config_plummer()
    return w, {}


def _plummer_ref(plummer, gradient):
    w, cache = plummer
    if gradient not in cache:
        cache[gradient] = run_oracle(w.grids, w.particles, w.half_dt, periodic=True, gradient=gradient)
    return cache[gradient]


@pytest.mark.parametrize("gradient", ["fd2", "fd4", "spectral"])
def test_plummer_periodic_three_levels_full(plummer, gradient):
    w, _ = plummer
    ref = _plummer_ref(plummer, gradient)
    gpu = run_gpu(w.grids, w.particles, w.half_dt, periodic=True, precision="fp32", gradient=gradient)
    compare(gpu, ref, "fp32")


def test_plummer_deposit_tiles_bit_exact(plummer):
    """The deposit through shared-memory tiles (particles in bin order,
    apm_set_deposit_tiles: the mode bench.py picks for this workload) at full
    size: every grid's mass field equals the direct deposit's bit for bit,
    all levels at once and level by level."""
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    w, _ = plummer
    P = Particles({k: torch.as_tensor(np.ascontiguousarray(v), device="cuda") for k, v in w.particles.items()})
    s = Solver(w.grids, periodic=True, precision="fp32", mass_frac_bits=w.mass_frac_bits, device=0)
    bufs = s.alloc_all()
    gmf = s._per_grid(bufs, "gmf")
    s.deposit_all(P, w.half_dt, gmf, None)
    direct = [t.clone() for t in gmf]
    s.reserve_order(w.n_particles)
    s.set_deposit_tiles(True)
    s.order_particles(P, w.half_dt)
    for t in gmf:
        t.fill_(-1)
    s.deposit_all(P, w.half_dt, gmf, None)
    s.sync_status()
    assert all(torch.equal(a, b) for a, b in zip(gmf, direct))
    for lev in range(s.n_levels):
        for t in bufs[lev]["gmf"]:
            t.fill_(-1)
        s.deposit(lev, P, w.half_dt, bufs[lev]["gmf"])
    s.sync_status()
    assert all(torch.equal(a, b) for a, b in zip(gmf, direct))
    s.close()


def test_plummer_periodic_three_levels_full_fp64(plummer):
    """The FP64 GPU path at a benchmark size: every grid's GMF bit-exact and
    every field and particle acceleration within 1e-12 of the oracle."""
    w, _ = plummer
    ref = _plummer_ref(plummer, "fd2")
    gpu = run_gpu(w.grids, w.particles, w.half_dt, periodic=True, precision="fp64")
    compare(gpu, ref, "fp64")


@pytest.mark.parametrize("gradient", ["fd2", "spectral"])
def test_batched_level_sampled_grids(gradient):
    """The two- and spectral gradient operators at the batched size (512 grids
    of one level); the spectral solve's acceleration components at the
    acceleration tolerance.  The four-point operator needs an even transform
    length >= 2 N0 + 2 on an isolated root: 1050 for this 512^3 container,
    past the 1024 limit, so the hierarchy is refused (checked below)."""
    import oracle
    w = W.config_batched_level()
    gpu = run_gpu(w.grids, w.particles, w.half_dt, gas=w.gas, precision="fp32",
                  mass_frac_bits=w.mass_frac_bits, levels=w.solve_levels, gradient=gradient)
    cfg = oracle.Config(periodic=False, mass_frac_bits=w.mass_frac_bits, gradient=gradient)
    grids = [oracle.Grid(*g) for g in w.grids]
    rng = np.random.default_rng(40)
    sample = sorted(rng.choice(np.arange(1, len(grids)), size=6, replace=False).tolist())
    own = oracle.owners(cfg, grids, w.particles, w.half_dt) if gradient == "fd2" else None
    for gi in sample:
        gmf, st = oracle.deposit(cfg, grids, gi, w.particles, w.half_dt, gas=w.gas[gi])
        assert np.array_equal(gpu["gmf"][gi], gmf), gi
        phis = oracle.solve(cfg, grids, gi, gmf)
        if gradient == "spectral":
            assert rel_l2(gpu["phis"][gi][1:], phis[1:]) <= TOL["fp32"]["acc"], gi
            assert rel_l2(gpu["phis"][gi][0], phis[0]) <= TOL["fp32"]["phis"], gi
        else:
            assert rel_l2(gpu["phis"][gi], phis) <= TOL["fp32"]["phis"], gi
        phi, acc = oracle.accel(cfg, grids, gi, phis)
        assert rel_l2(gpu["phi"][gi], phi) <= TOL["fp32"]["phi"], gi
        assert rel_l2(gpu["acc"][gi], acc) <= TOL["fp32"]["acc"], gi
        if gradient != "fd2":
            continue
        # the particles this grid owns: the oracle's interpolation of its own
        # accelerations against the GPU's particle accelerations
        sel = own == gi
        assert sel.sum() >= 2000, gi
        parts = {k: v[sel] for k, v in w.particles.items()}
        out = np.zeros((3, int(sel.sum())))
        oracle.interp(cfg, grids, gi, acc, parts, w.half_dt, own[sel], out)
        assert rel_l2(gpu["pacc"][:, sel], out) <= TOL["fp32"]["pacc"], gi


def test_four_point_isolated_root_over_511_cells_is_refused():
    from paper_1410_0010_gb300._lib import ApmError
    from paper_1410_0010_gb300.solver import Solver
    w = W.config_batched_level()
    with pytest.raises(ApmError) as e:
        Solver(w.grids[:1], periodic=False, precision="fp32", device=0, gradient="fd4")
    assert e.value.code == 8          # APM_E_UNSUPPORTED
    s = Solver([(0, -1, (0, 0, 0), (510, 510, 510))], periodic=False, precision="fp32", device=0,
               gradient="fd4")
    assert s.info[0]["fft"] == (1024, 1024, 1024)   # 2 * 510 + 2 = 1022 -> 1024
    s.close()


@pytest.fixture(scope="module")
def cosmo():
    """The 512^3 workload solved once on the GPU (FP32), with the arrays the
    checks below read."""
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    w = W.config_cosmo512()
    dev = torch.device("cuda", 0)
    s = Solver(w.grids, periodic=True, precision="fp32", mass_frac_bits=w.mass_frac_bits, device=0)
    P = Particles({k: torch.as_tensor(v, device=dev) for k, v in w.particles.items()})
    bufs = s.alloc_all()
    pacc = torch.zeros((3, w.n_particles), dtype=torch.float32, device=dev)
    s.step(P, w.half_dt, bufs, pacc)
    s.sync_status()
    l1 = s.level_grids[1][:2]
    # the chain: the level-2 grid whose interior holds the most particles (the
    # workload's own positions), and its level-1 parent
    pos = np.stack([w.particles[k] for k in ("x", "y", "z")])
    l2_ids = s.level_grids[2]
    counts = []
    for gi in l2_ids:
        _, _, start, dims = w.grids[gi]
        d2 = 1.0 / (w.grids[0].dims[0] * 4)
        lo = np.array(start)[:, None] * d2
        hi = lo + np.array(dims)[:, None] * d2
        counts.append(int(np.all((pos >= lo) & (pos < hi), axis=0).sum()))
    g2 = l2_ids[int(np.argmax(counts))]
    g1 = w.grids[g2][1]

    def grab(lev, gi):
        k = s.info[gi]["level_index"]
        return {key: bufs[lev][key][k].cpu().numpy() for key in ("gmf", "phis", "phi", "acc")}

    out = dict(w=w, solver=s, root_gmf=bufs[0]["gmf"][0].cpu().numpy(),
               chain=(g1, g2), chain_l1=grab(1, g1), chain_l2=grab(2, g2),
               root_phis=bufs[0]["phis"][0].cpu().numpy(),
               root_phi=bufs[0]["phi"][0].cpu().numpy(), root_acc=bufs[0]["acc"][0].cpu().numpy(),
               l1_ids=l1, l1={k: {key: bufs[1][key][s.info[gi]["level_index"]].cpu().numpy()
                                  for key in ("gmf", "phis", "phi", "acc")} for k, gi in enumerate(l1)},
               pacc=pacc.cpu().numpy())
    del bufs, P
    torch.cuda.empty_cache()
    return out


def test_cosmo_root_mass_field_bit_exact(cosmo):
    import oracle
    w = cosmo["w"]
    cfg = oracle.Config(periodic=True, mass_frac_bits=w.mass_frac_bits)
    gmf, st = oracle.deposit(cfg, [oracle.Grid(*g) for g in w.grids], 0, w.particles, w.half_dt)
    assert st == 0
    assert np.array_equal(cosmo["root_gmf"], gmf)


def _root_oracle(cosmo):
    """The oracle's root potential (textbook-FFT mode) and its own FD fields."""
    import oracle
    if "root_ref" not in cosmo:
        w = cosmo["w"]
        cfg = oracle.Config(periodic=True, mass_frac_bits=w.mass_frac_bits)
        grids = [oracle.Grid(*g) for g in w.grids]
        gmf, st = oracle.deposit(cfg, grids, 0, w.particles, w.half_dt)
        assert st == 0
        prev = oracle.set_transform("fft")
        try:
            phis = oracle.solve(cfg, grids, 0, gmf)
        finally:
            oracle.set_transform(prev)
        phi, acc = oracle.accel(cfg, grids, 0, phis)
        cosmo["root_ref"] = (phis, phi, acc)
    return cosmo["root_ref"]


def test_cosmo_root_potential_element_by_element(cosmo):
    """The whole 512^3 root: phi_short, phi and the accelerations against the
    oracle's chain (its own deposit, FFT-mode solve and FD), every cell."""
    phis, phi, acc = _root_oracle(cosmo)
    assert rel_l2(cosmo["root_phis"], phis) <= TOL["fp32"]["phis"]
    assert rel_l2(cosmo["root_phi"], phi) <= TOL["fp32"]["phi"]
    assert rel_l2(cosmo["root_acc"], acc) <= TOL["fp32"]["acc"]


def test_cosmo_chain_root_level1_level2(cosmo):
    """The oracle's whole chain on the level-2 grid holding the most particles,
    its level-1 parent and that parent's 64^3 footprint on the root: deposit,
    solve, FD and the carry of the oracle's own parent fields, element by
    element, then the particle accelerations these grids own."""
    import oracle
    w = cosmo["w"]
    cfg = oracle.Config(periodic=True, mass_frac_bits=w.mass_frac_bits)
    grids = [oracle.Grid(*g) for g in w.grids]
    _, phi0, acc0 = _root_oracle(cosmo)
    g1, g2 = cosmo["chain"]
    # the parent's footprint on the root: cells [s/2 - 1, (s + N)/2 + 1) of the
    # root window [-1, N0 + 1)
    _, _, start1, dims1 = w.grids[g1]
    sl = tuple(slice(start1[j] // 2, (start1[j] + dims1[j]) // 2 + 2) for j in (2, 1, 0))
    assert rel_l2(cosmo["root_phi"][sl], phi0[sl]) <= TOL["fp32"]["phi"]
    assert rel_l2(cosmo["root_acc"][(slice(None),) + sl], acc0[(slice(None),) + sl]) <= TOL["fp32"]["acc"]
    fields = {}
    parent = (phi0, acc0)
    prev = oracle.set_transform("fft")
    try:
        for gi, got in ((g1, cosmo["chain_l1"]), (g2, cosmo["chain_l2"])):
            gmf, st = oracle.deposit(cfg, grids, gi, w.particles, w.half_dt)
            assert np.array_equal(got["gmf"], gmf), gi
            phis = oracle.solve(cfg, grids, gi, gmf)
            phi, acc = oracle.accel(cfg, grids, gi, phis, parent[0], parent[1])
            assert rel_l2(got["phis"], phis) <= TOL["fp32"]["phis"], gi
            assert rel_l2(got["phi"], phi) <= TOL["fp32"]["phi"], gi
            assert rel_l2(got["acc"], acc) <= TOL["fp32"]["acc"], gi
            fields[gi] = acc
            parent = (phi, acc)
    finally:
        oracle.set_transform(prev)
    own = oracle.owners(cfg, grids, w.particles, w.half_dt)
    for gi in (g1, g2):
        sel = own == gi
        assert sel.sum() > 1000, gi
        parts = {k: v[sel] for k, v in w.particles.items()}
        out = np.zeros((3, int(sel.sum())))
        oracle.interp(cfg, grids, gi, fields[gi], parts, w.half_dt, own[sel], out)
        assert rel_l2(cosmo["pacc"][:, sel], out) <= TOL["fp32"]["pacc"], gi


def test_cosmo_root_potential_mode_by_mode(cosmo):
    """Phi = IDFT(T DFT(m)) on the periodic 512^3 root: at sampled modes the DFT of
    the GPU potential equals T(kappa) times the DFT of the cell masses."""
    import oracle
    w = cosmo["w"]
    n = w.grids[0].dims[0]
    d = 1.0 / n
    m = np.ldexp(cosmo["root_gmf"].astype(np.float64), -w.mass_frac_bits)
    phi = cosmo["root_phis"][2:-2, 2:-2, 2:-2].astype(np.float64)   # cells [0, n)
    ar = np.arange(n)
    rng = np.random.default_rng(41)
    modes = [(1, 0, 0), (0, 3, 1), (5, 7, 2), (40, 11, 90), (n // 2 - 1, 3, 200)] + \
        [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(4)]
    # FP32 round-off of the output field, seen in one Fourier mode
    floor = 2e-6 * float(np.sqrt(np.mean(phi * phi))) * n ** 1.5

    def dft(f, kap):
        ex, ey, ez = [np.exp(-2j * np.pi * kap[j] * ar / n) for j in range(3)]
        zy = f @ ex.real + 1j * (f @ ex.imag)            # sum over x -> [z, y]
        z = zy @ ey                                      # sum over y -> [z]
        return z @ ez

    for kap in modes:
        dm = dft(m, kap)
        dp = dft(phi, kap)
        fk = [min(k, n - k) for k in kap]
        T = oracle.green_opt(fk, (n, n, n), d, 3.4 * d, 0.0, 0) / d ** 3
        expect = T * dm
        assert abs(dp - expect) <= 2e-5 * abs(expect) + floor, kap


def test_cosmo_subgrids_full_oracle_solve(cosmo):
    import oracle
    w = cosmo["w"]
    cfg = oracle.Config(periodic=True, mass_frac_bits=w.mass_frac_bits)
    grids = [oracle.Grid(*g) for g in w.grids]
    for k, gi in enumerate(cosmo["l1_ids"]):
        gmf, st = oracle.deposit(cfg, grids, gi, w.particles, w.half_dt)
        assert np.array_equal(cosmo["l1"][k]["gmf"], gmf)
        phis = oracle.solve(cfg, grids, gi, gmf)
        assert rel_l2(cosmo["l1"][k]["phis"], phis) <= TOL["fp32"]["phis"]


def test_cosmo_fd_carry_and_interpolation(cosmo):
    """The root accelerations are the FD of its potential; a level-1 grid's fields
    are its FD plus the trilinear carry of the root fields; particle accelerations
    are the TSC interpolation of the owning grid's field (oracle routines applied
    to the GPU's own inputs)."""
    import oracle
    w = cosmo["w"]
    cfg = oracle.Config(periodic=True, mass_frac_bits=w.mass_frac_bits)
    grids = [oracle.Grid(*g) for g in w.grids]
    phi0, acc0 = oracle.accel(cfg, grids, 0, cosmo["root_phis"])
    assert rel_l2(cosmo["root_phi"], phi0) <= TOL["fp32"]["phi"]
    assert rel_l2(cosmo["root_acc"], acc0) <= TOL["fp32"]["acc"]
    gi = cosmo["l1_ids"][0]
    phi1, acc1 = oracle.accel(cfg, grids, gi, cosmo["l1"][0]["phis"], cosmo["root_phi"],
                              cosmo["root_acc"])
    assert rel_l2(cosmo["l1"][0]["phi"], phi1) <= TOL["fp32"]["phi"]
    assert rel_l2(cosmo["l1"][0]["acc"], acc1) <= TOL["fp32"]["acc"]
    # particles: a sample owned by the root and by the first level-1 grid
    rng = np.random.default_rng(42)
    sub = np.sort(rng.choice(w.n_particles, size=200000, replace=False))
    parts = {k: v[sub] for k, v in w.particles.items()}
    own = oracle.owners(cfg, grids, parts, w.half_dt)
    out = np.zeros((3, len(sub)))
    oracle.interp(cfg, grids, 0, cosmo["root_acc"].astype(np.float64), parts, w.half_dt, own, out)
    oracle.interp(cfg, grids, gi, cosmo["l1"][0]["acc"].astype(np.float64), parts, w.half_dt, own, out)
    sel = (own == 0) | (own == gi)
    assert sel.sum() > 1000
    got = cosmo["pacc"][:, sub][:, sel]
    assert rel_l2(got, out[:, sel]) <= TOL["fp32"]["pacc"]
