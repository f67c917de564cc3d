"""Library-owned CUDA graphs (apm_graph_begin / end / launch / destroy): a
replayed step equals the eager one bit for bit; the legacy default stream
cannot be captured; a synchronising call inside a capture makes the capture
fail with APM_E_STATE and leaves the stream usable; destroyed ids are
rejected; a new hierarchy frees every graph."""
import ctypes

import numpy as np
import pytest

from apm_inputs import GridDesc

pytestmark = pytest.mark.gpu

GRIDS = [GridDesc(0, -1, (0, 0, 0), (32, 32, 32)), GridDesc(1, 0, (12, 14, 16), (24, 20, 28))]


def _setup(precision="fp32"):
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    rng = np.random.default_rng(9)
    n = 5000
    pos = 0.2 + 0.6 * rng.random((3, n))
    v = rng.normal(scale=0.2, size=(3, n))
    d = {"x": pos[0], "y": pos[1], "z": pos[2], "vx": v[0], "vy": v[1], "vz": v[2], "m": (0.5 + rng.random(n)) / n}
    P = Particles({k: torch.as_tensor(np.ascontiguousarray(a), device="cuda") for k, a in d.items()})
    s = Solver(GRIDS, periodic=False, precision=precision, device=0)
    return s, P


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_replayed_step_equals_eager_step(precision):
    import torch
    s, P = _setup(precision)
    bufs = s.alloc_all()
    pacc = torch.zeros((3, P.n), dtype=s.dtype, device="cuda")
    s.step(P, 1e-3, bufs, pacc)
    ref = [t.clone() for b in bufs for key in ("gmf", "phis", "acc") for t in b[key]] + [pacc.clone()]
    g = s.capture(lambda: s.step(P, 1e-3, bufs, pacc))
    for b in bufs:
        for t in b["phis"] + b["acc"]:
            t.fill_(float("nan"))
    pacc.fill_(float("nan"))
    for _ in range(3):
        g.replay()
    s.sync_status()
    got = [t for b in bufs for key in ("gmf", "phis", "acc") for t in b[key]] + [pacc]
    assert all(torch.equal(a, b) for a, b in zip(got, ref))
    g.destroy()
    s.close()


def test_graph_errors():
    import torch

    from paper_1410_0010_gb300 import _lib
    L = _lib.lib()
    s, P = _setup()
    bufs = s.alloc_all()
    s.step(P, 1e-3, bufs, None)
    # the legacy default stream cannot be captured
    assert L.apm_graph_begin(s._ctx, None) == 1            # APM_E_INVALID
    # a synchronising call inside the capture: the capture fails, the stream stays usable
    side = torch.cuda.Stream()
    h = ctypes.c_void_p(side.cuda_stream)
    assert L.apm_graph_begin(s._ctx, h) == 0
    assert L.apm_graph_begin(s._ctx, h) == 9                # APM_E_STATE: already capturing
    L.apm_sync_status(s._ctx, h)                            # synchronises: invalidates the capture
    gid = ctypes.c_int32(-1)
    assert L.apm_graph_end(s._ctx, h, ctypes.byref(gid)) == 9
    torch.cuda.synchronize()
    s.step(P, 1e-3, bufs, None, stream=side)                # the stream still works
    side.synchronize()
    s.sync_status()
    # ids: a destroyed graph and an unknown id are rejected
    g = s.capture(lambda: s.step(P, 1e-3, bufs, None))
    g.replay()
    assert L.apm_graph_destroy(s._ctx, g.gid) == 0
    assert L.apm_graph_launch(s._ctx, g.gid, None) == 1
    assert L.apm_graph_destroy(s._ctx, 12345) == 1
    s.close()
