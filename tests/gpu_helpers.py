"""Helpers of the GPU parity tests: run one APM solve through the C ABI and
through the oracle on the same seeded inputs and compare element by element.

Tolerances (relative L2 over each grid's output, acceleration as a 3-vector):
  deposit: bit-exact (int64 fixed point);
  FP64 path: 1e-12 for phi_short, phi, acc and particle accelerations;
  FP32 path: 2e-5 for phi_short and phi, 1e-4 for acc and particle accelerations.
"""
import numpy as np

TOL = {
    "fp64": dict(phis=1e-12, phi=1e-12, acc=1e-12, pacc=1e-12),
    "fp32": dict(phis=2e-5, phi=2e-5, acc=1e-4, pacc=1e-4),
}


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def run_gpu(grids, particles, half_dt, gas=None, periodic=False, precision="fp64",
            mass_frac_bits=52, root_correction=True, levels=None, batched=True, gradient="fd2",
            pad_factor=0.65, a_over_dx=3.4):
    import torch

    from paper_1410_0010_gb300.solver import Solver
    dev = torch.device("cuda", 0)
    s = Solver(grids, periodic=periodic, precision=precision, mass_frac_bits=mass_frac_bits,
               root_correction=root_correction, device=0, gradient=gradient, pad_factor=pad_factor,
               a_over_dx=a_over_dx)
    tp = {k: torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device=dev)
          for k, v in particles.items()}
    tg = None
    if gas is not None:
        tg = [None if g is None else torch.as_tensor(np.ascontiguousarray(g, dtype=np.float64), device=dev)
              for g in gas]
    bufs = s.alloc_all()
    n = len(particles["x"])
    pacc = torch.zeros((3, n), dtype=s.dtype, device=dev)
    s.step(tp, half_dt, bufs, pacc, gas=tg, levels=levels, batched=batched)
    s.sync_status()
    out = dict(gmf={}, phis={}, phi={}, acc={}, info=s.info, solver=s)
    for lev, ids in enumerate(s.level_grids):
        if levels is not None and lev not in levels:
            continue
        for k, gi in enumerate(ids):
            for key in ("gmf", "phis", "phi", "acc"):
                out[key][gi] = bufs[lev][key][k].cpu().numpy()
    out["pacc"] = pacc.cpu().numpy()
    return out


def run_oracle(grids, particles, half_dt, gas=None, periodic=False, mass_frac_bits=52,
               root_correction=True, gradient="fd2", pad_factor=0.65, a_over_dx=3.4):
    import oracle
    cfg = oracle.Config(periodic=periodic, mass_frac_bits=mass_frac_bits,
                        root_correction=root_correction, gradient=gradient, pad_factor=pad_factor,
                        a_over_dx=a_over_dx)
    return oracle.apm_step(cfg, [oracle.Grid(*g) for g in grids], particles, half_dt, gas=gas)


def compare(gpu, ref, precision, grids=None, check_pacc=True):
    tol = TOL[precision]
    report = {}
    for gi in gpu["gmf"]:
        assert np.array_equal(gpu["gmf"][gi], ref.gmf[gi]), f"GMF of grid {gi} not bit-exact"
        for key in ("phis", "phi", "acc"):
            g, r = gpu[key][gi], getattr(ref, key)[gi]
            if key == "phis" and r.ndim == 4:
                # spectral gradient: phi_short, then A_x, A_y, A_z (acceleration tolerance)
                e = rel_l2(g[1:], r[1:])
                report[("phis_acc", gi)] = e
                assert e <= tol["acc"], f"spectral A of grid {gi}: rel L2 {e:.3e} > {tol['acc']:.0e}"
                g, r = g[0], r[0]
            e = rel_l2(g, r)
            report[(key, gi)] = e
            assert e <= tol[key], f"{key} of grid {gi}: rel L2 {e:.3e} > {tol[key]:.0e}"
    if check_pacc:
        e = rel_l2(gpu["pacc"], ref.pacc)
        report[("pacc", -1)] = e
        assert e <= tol["pacc"], f"particle accelerations: rel L2 {e:.3e} > {tol['pacc']:.0e}"
    return report
