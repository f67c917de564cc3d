"""The allocation-free entry point apm_solve_periodic_noalloc.

Some callers cannot call cudaMalloc: applications that give the whole device
to their own memory pool at start-up, and loops that must not stall on the
device-wide synchronisation cudaFree implies.  This entry point gives them the
periodic-root potential while keeping every intermediate in a fixed device
array of the library.  Its output must equal what the existing entry point
apm_solve_level gives for the same grid, call after call, and the FP64 oracle
within the FP32 tolerance.  The sizes cover a power of two, a mixed radix
(48 = 3 * 16) and the largest grid the array holds (128, 21.3 of its 24 MiB).

This file is collected last on purpose: a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5     # the FP32 potential tolerance of the parity tests


def _rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n", [32, 48, 128])
def test_noalloc_solve_matches_solve_level_and_oracle_on_consecutive_calls(n):
    import torch

    import oracle
    from paper_1410_0010_gb300 import _lib
    from paper_1410_0010_gb300.solver import Solver

    torch.cuda.set_device(0)
    grids = [(0, -1, (0, 0, 0), (n, n, n))]
    solver = Solver(grids, periodic=True, precision="fp32", device=0)
    cfg = oracle.Config(periodic=True)
    ogrids = [oracle.Grid(*g) for g in grids]
    lib = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(21 + n)
    for call in range(2):
        masses = rng.integers(0, 1 << 44, size=(n, n, n))
        if call == 1:
            masses[n // 3, n // 2, n // 5] += 1 << 50     # a point mass on a random field
        gmf = torch.tensor(masses, dtype=torch.int64, device="cuda")
        ref = torch.empty((n + 4,) * 3, dtype=torch.float32, device="cuda")
        solver.solve_level(0, [gmf], [ref])
        out = torch.full((n + 4,) * 3, float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.apm_solve_periodic_noalloc(n, 1.0, 3.4, 52, gmf.data_ptr(), out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel_l2(got, ref.cpu().numpy()) <= FP32_TOL
        want = oracle.solve(cfg, ogrids, 0, masses)
        assert _rel_l2(got, want) <= FP32_TOL, f"n={n} call {call}: against the oracle"
    solver.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch

    from paper_1410_0010_gb300 import _lib
    lib = _lib.lib()
    g = torch.zeros(8, dtype=torch.int64, device="cuda")
    o = torch.zeros(8, dtype=torch.float32, device="cuda")
    assert lib.apm_solve_periodic_noalloc(256, 1.0, 3.4, 52, g.data_ptr(), o.data_ptr(), None) == 1
    assert lib.apm_solve_periodic_noalloc(22, 1.0, 3.4, 52, g.data_ptr(), o.data_ptr(), None) == 1
    assert lib.apm_solve_periodic_noalloc(32, 1.0, 3.4, 52, None, o.data_ptr(), None) == 1
