"""The bounds-checked debug build (-DAPM_BOUNDS_CHECK): every data- or
hierarchy-dependent global index of the baryon, deposit, acceleration and
interpolation kernels is tested before use, and a violation would set the
status word's bounds bit (APM_E_BOUNDS).  On the hierarchies of the parity
tests (isolated and periodic roots, siblings, grandchildren, borders past an
isolated root's faces, odd starts), with every gradient operator and both
precisions, no access is out of range."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from apm_inputs import GridDesc
from paper_1410_0010_gb300.solver import Particles, Solver

maps = open("/proc/self/maps").read()
dev = torch.device("cuda", 0)
rng = np.random.default_rng(5)
HIER = {
    "isolated": ([GridDesc(0, -1, (0, 0, 0), (24, 24, 24)), GridDesc(1, 0, (2, 3, 36), (12, 10, 10)),
                  GridDesc(1, 0, (30, 30, 2), (16, 14, 12)), GridDesc(2, 1, (9, 11, 78), (14, 10, 8))], False),
    "periodic": ([GridDesc(0, -1, (0, 0, 0), (24, 24, 24)), GridDesc(1, 0, (8, 8, 10), (14, 12, 16)),
                  GridDesc(1, 0, (22, 8, 12), (18, 14, 10)), GridDesc(2, 1, (24, 24, 28), (12, 10, 14))], True),
    "odd": ([GridDesc(0, -1, (0, 0, 0), (21, 21, 21)), GridDesc(1, 0, (9, 11, 13), (15, 12, 9)),
             GridDesc(1, 0, (27, 7, 25), (9, 17, 11)), GridDesc(2, 1, (25, 27, 31), (11, 9, 7))], False),
}
n = 3000
runs = 0
for name, (grids, periodic) in HIER.items():
    pos = 0.002 + 0.996 * rng.random((3, n))
    pos[:, :800] = 0.3 + 0.3 * rng.random((3, 800))
    v = rng.normal(scale=0.2, size=(3, n))
    parts = dict(x=pos[0], y=pos[1], z=pos[2], vx=v[0], vy=v[1], vz=v[2], m=0.5 + rng.random(n))
    P = Particles({k: torch.as_tensor(np.ascontiguousarray(a), device=dev) for k, a in parts.items()})
    gas = [torch.as_tensor(rng.random(tuple(g.dims)[::-1]) + 0.1, device=dev) for g in grids]
    for grad in ("fd2", "fd4", "spectral"):
        for prec in ("fp32", "fp64"):
            s = Solver(grids, periodic=periodic, precision=prec, device=0, gradient=grad)
            bufs = s.alloc_all()
            pacc = torch.zeros((3, n), dtype=s.dtype, device=dev)
            s.step(P, 1e-4, bufs, pacc, gas=gas)
            s.step(P, 1e-4, bufs, pacc, gas=gas, batched=False)
            s.sync_status()            # raises on APM_E_BOUNDS (or any other latched error)
            assert bool(torch.isfinite(pacc).all())
            s.close()
            runs += 1
print("CHECKED" if "_build_bounds/libapm.so" in open("/proc/self/maps").read() else "NOT-CHECKED", runs)
"""


def test_bounds_checked_build_finds_no_violation():
    sys.path.insert(0, ROOT)
    from paper_1410_0010_gb300 import buildlib
    lib = buildlib.build_bounds_checked()
    env = dict(os.environ, APM_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True, timeout=900,
                       cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "CHECKED 18" in r.stdout, r.stdout
