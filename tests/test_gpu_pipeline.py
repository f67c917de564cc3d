"""StepPipeline: the end-to-end driver's overlapped copies must not change a
result.  Five steps cycle through three different particle sets (so every
buffer set is reused while the other solves); each step's downloaded
accelerations equal, bit for bit, a plain solve of the same inputs."""
import numpy as np
import pytest

from apm_inputs import GridDesc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_pipelined_steps_equal_plain_steps(precision):
    import torch

    from paper_1410_0010_gb300.solver import PARTICLE_KEYS, Particles, Solver, StepPipeline
    grids = [GridDesc(0, -1, (0, 0, 0), (32, 32, 32)), GridDesc(1, 0, (16, 18, 20), (24, 20, 22))]
    n = 20000
    rng = np.random.default_rng(23)
    sets = []
    for _ in range(3):
        pos = 0.05 + 0.9 * rng.random((3, n))
        v = rng.normal(scale=0.3, size=(3, n))
        a = dict(x=pos[0], y=pos[1], z=pos[2], vx=v[0], vy=v[1], vz=v[2], m=0.5 + rng.random(n))
        sets.append({k: torch.from_numpy(np.ascontiguousarray(a[k])).pin_memory() for k in PARTICLE_KEYS})
    s = Solver(grids, precision=precision, device=0)
    bufs = s.alloc_all()
    dev = torch.device("cuda", 0)
    want = []
    for h in sets:
        P = Particles({k: h[k].to(dev) for k in PARTICLE_KEYS})
        pacc = torch.zeros((3, n), dtype=s.dtype, device=dev)
        s.step(P, 1e-3, bufs, pacc)
        want.append(pacc.cpu())
    s.sync_status()
    pipe = StepPipeline(s, bufs, sets[0], 1e-3)
    steps = 5
    outs = [torch.empty((3, n), dtype=s.dtype).pin_memory() for _ in range(steps)]
    pipe.run(steps, inputs=lambda k: sets[k % 3], outputs=lambda k: outs[k])
    torch.cuda.synchronize()
    s.sync_status()
    for k in range(steps):
        assert torch.equal(outs[k], want[k % 3]), k
    h2d, d2h = pipe.bytes_per_step()
    assert h2d == 7 * 8 * n and d2h == 3 * n * (4 if precision == "fp32" else 8)
    s.close()
