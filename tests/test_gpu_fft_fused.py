"""The fused plane kernels (k_xy_fast: x then y forward over a z plane; k_yx_fast:
y then x inverse over a window plane) for grids with equal x and y transform
lengths: against the same solve with the passes unfused (plan 0) and against
the FP64 path.  The grids cover odd GMF heights
(G1 odd: a zero row inside the last line), odd window heights (W1 odd: one
output row in the last line), a wrapped window start and the isolated root."""
import numpy as np
import pytest

from apm_inputs import GridDesc
from gpu_helpers import TOL

pytestmark = pytest.mark.gpu

GRIDS = [GridDesc(0, -1, (0, 0, 0), (32, 32, 32)),            # M = 64 (isolated: doubled)
         GridDesc(1, 0, (10, 12, 14), (25, 25, 30)),           # G1 = 35, W1 = 29, M = 45
         GridDesc(1, 0, (38, 36, 12), (16, 16, 40)),           # M = 36
         GridDesc(2, 1, (26, 30, 34), (30, 30, 24))]           # G1 = 40, W1 = 34, M = 50


def _solve(precision, fuse=True):
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    rng = np.random.default_rng(12)
    n = 60000
    pos = 0.05 + 0.9 * rng.random((3, n))
    v = rng.normal(scale=0.2, size=(3, n))
    d = {"x": pos[0], "y": pos[1], "z": pos[2], "vx": v[0], "vy": v[1], "vz": v[2], "m": (0.5 + rng.random(n)) / n}
    P = Particles({k: torch.as_tensor(np.ascontiguousarray(a), device="cuda") for k, a in d.items()})
    s = Solver(GRIDS, periodic=False, precision=precision, device=0)
    if fuse and precision == "fp32":   # plan 2 on both x passes: the fused plane kernels
        for lev in range(s.n_levels):
            sh = s.fft_shapes(lev)
            sh["plan"] = [2, 0, 0, 0, 2]
            s.set_fft_shapes(lev, sh)
    kinds = [s.pass_kernels(lev) for lev in range(s.n_levels)]
    bufs = s.alloc_all()
    pacc = torch.zeros((3, n), dtype=s.dtype, device="cuda")
    s.profile(True)
    s.step(P, 1e-3, bufs, pacc)
    prof = s.profile_read()
    s.profile(False)
    s.sync_status()
    out = [("phis", t.double().cpu().numpy()) for b in bufs for t in b["phis"]] + \
          [("acc", t.double().cpu().numpy()) for b in bufs for t in b["acc"]]
    s.close()
    return out, pacc.double().cpu().numpy(), prof, kinds


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_fused_planes_match_unfused_and_fp64():
    fused, pf, prof_f, kinds_f = _solve("fp32")
    plain, pp, prof_p, kinds_p = _solve("fp32", fuse=False)
    ref, pr, _, kinds_r = _solve("fp64")
    # per level and pass, the kernel of each grid: fused (2) on both x passes,
    # nothing (3) on both y passes; unfused: compile-time plans (1); FP64: the
    # runtime-planned kernel (0)
    for lev in range(3):
        assert kinds_f[lev] == [[2] * len(kinds_f[lev][0]) if q in (0, 4) else
                                ([3] * len(kinds_f[lev][0]) if q in (1, 3) else [1] * len(kinds_f[lev][0]))
                                for q in range(5)]
        assert all(k == 1 for row in kinds_p[lev] for k in row)
        assert all(k == 0 for row in kinds_r[lev] for k in row)
    # fused: the y passes launch nothing on these levels (every grid fused);
    # unfused: one launch per length on each level (64; 45 and 36; 50)
    assert prof_f["fft_y_fwd"][0] == 0 and prof_f["fft_y_inv"][0] == 0
    assert prof_p["fft_y_fwd"][0] == 4 and prof_p["fft_y_inv"][0] == 4
    assert prof_f["fft_x_fwd"][0] == 4 and prof_f["fft_x_inv"][0] == 4
    for (kind, a), (_, b), (_, r) in zip(fused, plain, ref):
        assert _rel(a, b) <= 2e-6
        assert _rel(a, r) <= TOL["fp32"][kind]
    assert _rel(pf, pp) <= 2e-6
    assert _rel(pf, pr) <= TOL["fp32"]["pacc"]
