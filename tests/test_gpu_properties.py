"""Property tests of the CUDA path that need no oracle: translation by a whole
root cell on a periodic root.  With dyadic positions (multiples of 2^-30)
and no drift, moving every particle by one cell along an axis is exact in
FP64, so the mass field is the original rolled by one cell, bit for bit;
the potential and accelerations are rolled too, to rounding, and every
particle's acceleration is unchanged to rounding."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = 32
TOL = {"fp64": 1e-12, "fp32": 2e-5}


def _solve(parts, precision, gradient):
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    dev = torch.device("cuda", 0)
    s = Solver([(0, -1, (0, 0, 0), (N, N, N))], periodic=True, precision=precision, device=0,
               gradient=gradient)
    P = Particles({k: torch.as_tensor(np.ascontiguousarray(v), device=dev) for k, v in parts.items()})
    bufs = s.alloc_all()
    pacc = torch.zeros((3, len(parts["x"])), dtype=s.dtype, device=dev)
    s.step(P, 0.0, bufs, pacc)
    s.sync_status()
    out = {k: bufs[0][k][0].cpu().numpy() for k in ("gmf", "phi", "acc")}
    out["pacc"] = pacc.cpu().numpy()
    s.close()
    return out


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - np.asarray(b, float)) / np.linalg.norm(np.asarray(b, float)))


@pytest.mark.parametrize("gradient", ["fd2", "spectral"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("axis", [0, 2])
def test_translation_by_one_cell_on_a_periodic_root(gradient, precision, axis):
    rng = np.random.default_rng(61)
    n = 5000
    pos = np.floor(rng.random((3, n)) * 2.0 ** 30) / 2.0 ** 30          # dyadic
    parts = dict(x=pos[0], y=pos[1], z=pos[2], vx=np.zeros(n), vy=np.zeros(n), vz=np.zeros(n),
                 m=0.5 + rng.random(n))
    moved = dict(parts)
    key = "xyz"[axis]
    moved[key] = (pos[axis] + 1.0 / N) % 1.0                          # exact: 2^-5 on a 2^-30 grid
    a = _solve(parts, precision, gradient)
    b = _solve(moved, precision, gradient)
    ax = 2 - axis                                                      # arrays are [z, y, x]
    assert np.array_equal(b["gmf"], np.roll(a["gmf"], 1, axis=ax))
    inner = (slice(1, -1),) * 3                                        # interior cells of the [-1, N] window
    pa, pb = a["phi"][inner], b["phi"][inner]
    assert _rel(pb, np.roll(pa, 1, axis=ax)) < TOL[precision]
    for j in range(3):
        assert _rel(b["acc"][j][inner], np.roll(a["acc"][j][inner], 1, axis=ax)) < 5 * TOL[precision]
    assert _rel(b["pacc"], a["pacc"]) < 5 * TOL[precision]
