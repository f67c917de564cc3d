"""The FP32 passes with compile-time plans (fft_fast.cuh: y forward, z, y
inverse, x forward) against the runtime-planned kernels (APM_FFT_FAST=0) and
the FP64 path, on hierarchies whose FFT lengths cover every length with a
compile-time plan: every {2,3,5,7}-smooth length from 36 to 84, 128, 150, 256
and 512.  The two FP32 paths round differently, so they are compared at a
tolerance (2e-6, ten times the FP32 rounding seen against FP64); both stay
within the FP32 parity tolerances of the FP64 path (2e-5 potential, 1e-4
accelerations)."""
import os

import numpy as np
import pytest

from apm_inputs import GridDesc
from gpu_helpers import TOL

pytestmark = pytest.mark.gpu

CASES = {
    # isolated 32^3 root (M = 64), a 44^3 level-1 grid (M = 64) and a 64^3
    # level-2 grid (M = 84)
    "iso32_m64_m84": (False, [GridDesc(0, -1, (0, 0, 0), (32, 32, 32)),
                              GridDesc(1, 0, (10, 10, 10), (44, 44, 44)),
                              GridDesc(2, 1, (30, 30, 30), (64, 64, 64))]),
    # periodic 128^3 root (M = 128) with a 130^3 child (M = 150)
    "per128_m150": (True, [GridDesc(0, -1, (0, 0, 0), (128, 128, 128)),
                           GridDesc(1, 0, (40, 50, 60), (130, 130, 130))]),
    "per256": (True, [GridDesc(0, -1, (0, 0, 0), (256, 256, 256))]),
    # isolated 128^3 root (M = 256) and one level of 18 uneven grids whose
    # lengths N + 20 -> M cover every {2,3,5,7}-smooth M from 36 to 84 (the
    # batched level's lengths)
    "iso128_m36_to_m84": (False, [GridDesc(0, -1, (0, 0, 0), (128, 128, 128))] + [
        GridDesc(1, 0, (12 + 80 * (i % 3), 12 + 80 * ((i // 3) % 3), 12 + 80 * (i // 9)), (n, n + i % 3, n))
        for i, n in enumerate([16, 20, 22, 25, 28, 29, 30, 34, 36, 40, 43, 44, 50, 52, 55, 60, 61, 64])]),
    "per512": (True, [GridDesc(0, -1, (0, 0, 0), (512, 512, 512))]),
}


def _solve(grids, periodic, precision, fast, parts):
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    old = os.environ.get("APM_FFT_FAST")
    os.environ["APM_FFT_FAST"] = "1" if fast else "0"
    try:
        s = Solver(grids, periodic=periodic, precision=precision, device=0)
    finally:
        if old is None:
            del os.environ["APM_FFT_FAST"]
        else:
            os.environ["APM_FFT_FAST"] = old
    dev = torch.device("cuda", 0)
    P = Particles({k: torch.as_tensor(np.ascontiguousarray(v), device=dev) for k, v in parts.items()})
    bufs = s.alloc_all()
    pacc = torch.zeros((3, P.n), dtype=s.dtype, device=dev)
    s.step(P, 1e-3, bufs, pacc)
    s.sync_status()
    out = [[("phis", t.double().cpu().numpy()) for t in b["phis"]] +
           [("acc", t.double().cpu().numpy()) for t in b["acc"]] for b in bufs]
    ms = [s.info[i]["fft"] for i in range(len(grids))]
    s.close()
    return out, pacc.double().cpu().numpy(), ms


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


@pytest.mark.parametrize("case", list(CASES))
def test_fast_column_passes_match_runtime_plans(case):
    periodic, grids = CASES[case]
    rng = np.random.default_rng(7)
    n = 200000
    pos = 0.02 + 0.96 * rng.random((3, n)) if not periodic else rng.random((3, n))
    parts = dict(x=pos[0], y=pos[1], z=pos[2], vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n),
                 m=(0.5 + rng.random(n)) / n)
    fast, pf, ms = _solve(grids, periodic, "fp32", True, parts)
    slow, ps, _ = _solve(grids, periodic, "fp32", False, parts)
    ref, pr, _ = _solve(grids, periodic, "fp64", False, parts)
    lengths = {m for M in ms for m in M}
    assert lengths & {36, 64, 84, 128, 150, 256, 512}
    for lev in range(len(fast)):
        for (kind, a), (_, b), (_, r) in zip(fast[lev], slow[lev], ref[lev]):
            assert _rel(a, b) <= 2e-6
            assert _rel(a, r) <= TOL["fp32"][kind]
    assert _rel(pf, ps) <= 2e-6
    assert _rel(pf, pr) <= 1e-4
