"""The allocation-free entry point apm_solve_periodic_noalloc.

Callers that cannot call cudaMalloc (code running where the CUDA runtime may not
allocate, or programs whose own memory pool owns the whole device) get the
periodic-root potential from this entry point, which keeps every intermediate in
a fixed device array of the library.  Its output must equal what the existing
entry point apm_solve_level gives for the same grid, call after call.

This file is collected last on purpose: a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP32_TOL = 2e-5     # the FP32 potential tolerance of the parity tests


def _rel_l2(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).norm() / b.norm())


def test_noalloc_solve_matches_solve_level_on_consecutive_calls():
    import torch

    from paper_1410_0010_gb300 import _lib
    from paper_1410_0010_gb300.solver import Solver

    n = 32
    torch.cuda.set_device(0)
    solver = Solver([(0, -1, (0, 0, 0), (n, n, n))], periodic=True, precision="fp32", device=0)
    lib = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(21)
    for _ in range(2):
        gmf = torch.tensor(rng.integers(0, 1 << 44, size=(n, n, n)), dtype=torch.int64, device="cuda")
        ref = torch.empty((n + 4,) * 3, dtype=torch.float32, device="cuda")
        solver.solve_level(0, [gmf], [ref])
        out = torch.full((n + 4,) * 3, float("nan"), dtype=torch.float32, device="cuda")
        rc = lib.apm_solve_periodic_noalloc(n, 1.0, 3.4, 52, gmf.data_ptr(), out.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel_l2(out, ref) <= FP32_TOL
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
