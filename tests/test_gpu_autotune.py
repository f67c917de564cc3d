"""The FFT pass autotuner (apm_autotune_level) and the launch shapes it picks
(apm_get_fft_shapes / apm_set_fft_shapes).  A shape regroups whole lines per
CTA and sets the CTA size; it must never change a result, bit for bit, and the
tuned solve must leave the same potential as the plain one."""
import json

import numpy as np
import pytest

import apm_inputs as W
from apm_inputs import GridDesc

pytestmark = pytest.mark.gpu

# uneven grids in one level: several FFT lengths per pass
GRIDS = [GridDesc(0, -1, (0, 0, 0), (48, 48, 48)),
         GridDesc(1, 0, (10, 12, 14), (25, 29, 43)),
         GridDesc(1, 0, (10, 44, 62), (55, 26, 16)),
         GridDesc(1, 0, (66, 10, 10), (24, 24, 24))]


def _setup(precision):
    import torch

    from paper_1410_0010_gb300.solver import Particles, Solver
    rng = np.random.default_rng(31)
    n = 3000
    pos = 0.1 + 0.8 * rng.random((3, n))
    v = rng.normal(scale=0.1, size=(3, n))
    dev = torch.device("cuda", 0)
    parts = dict(x=pos[0], y=pos[1], z=pos[2], vx=v[0], vy=v[1], vz=v[2], m=0.5 + rng.random(n))
    P = Particles({k: torch.as_tensor(np.ascontiguousarray(a), device=dev) for k, a in parts.items()})
    s = Solver(GRIDS, periodic=False, precision=precision, device=0)
    return s, P


def _fields(bufs):
    return [[t.clone() for t in b["phis"]] + [t.clone() for t in b["acc"]] for b in bufs]


def _same(a, b):
    import torch
    return all(torch.equal(x, y) for la, lb in zip(a, b) for x, y in zip(la, lb))


def _rel(a, b):
    import torch
    num = sum(float(torch.linalg.vector_norm((x.double() - y.double()).flatten()) ** 2)
              for la, lb in zip(a, b) for x, y in zip(la, lb))
    den = sum(float(torch.linalg.vector_norm(y.double().flatten()) ** 2) for lb in b for y in lb)
    return (num / den) ** 0.5


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tuned_and_forced_shapes_give_identical_bits(precision):
    """Budgets, thread counts and packing regroup or reorder whole lines: with
    the plans held fixed they never change a bit.  The tuner may also pick
    another plan (compile-time or runtime kernel, largest radix), which rounds
    differently: the tuned solve stays within 2e-5 (the FP32 potential
    tolerance; measured 2e-6) of the default one over all its fields and is
    reproduced bit for bit by setting the shapes it reports."""
    import torch
    s, P = _setup(precision)
    bufs = s.alloc_all()
    pacc = torch.zeros((3, P.n), dtype=s.dtype, device="cuda")
    s.step(P, 1e-3, bufs, pacc)
    ref = _fields(bufs)
    ref_pacc = pacc.clone()
    default = s.fft_shapes(1)
    assert default["threads"] == [256] * 5
    assert default["plan"] == [0] * 5 and default["packing"] == 0
    assert default["max_radix"] == (8 if precision == "fp64" else 16)
    # forced extreme shapes and the other packing, default plans: the same bits
    for budget, threads, packing in ((1, 128, 0), (8192, 128, 1), (100000, 256, 1)):
        for lev in range(s.n_levels):
            s.set_fft_shapes(lev, {"budget": [budget] * 5, "threads": [threads] * 5, "packing": packing})
        s.step(P, 1e-3, bufs, pacc)
        assert _same(_fields(bufs), ref), (budget, threads, packing)
        assert torch.equal(pacc, ref_pacc)
    for lev in range(s.n_levels):
        s.set_fft_shapes(lev, default)
    # the tuned solve
    for b in bufs:
        for t in b["phis"]:
            t.fill_(float("nan"))
    s.step(P, 1e-3, bufs, None, tune=True)
    assert _rel(_fields(bufs), ref) <= 2e-5
    tuned = [s.fft_shapes(lev) for lev in range(s.n_levels)]
    for sh in tuned:
        assert all(t in (128, 256) for t in sh["threads"])
        assert sh["max_radix"] in ((8,) if precision == "fp64" else (8, 16))
    s.step(P, 1e-3, bufs, pacc)
    tuned_fields, tuned_pacc = _fields(bufs), pacc.clone()
    # the reported shapes reproduce the tuned solve, bit for bit
    s.close()
    s2, _ = _setup(precision)
    bufs2 = s2.alloc_all()
    for lev, sh in enumerate(tuned):
        s2.set_fft_shapes(lev, sh)
    s2.step(P, 1e-3, bufs2, pacc)
    assert _same(_fields(bufs2), tuned_fields)
    assert torch.equal(pacc, tuned_pacc)
    s2.close()


def test_runtime_plans_and_radix_stay_within_tolerance():
    """Every plan choice on FP32: the runtime-planned kernels with radices up
    to 16 or 8 against the compile-time plans, within 2e-5 over all fields."""
    import torch
    s, P = _setup("fp32")
    bufs = s.alloc_all()
    pacc = torch.zeros((3, P.n), dtype=s.dtype, device="cuda")
    s.step(P, 1e-3, bufs, pacc)
    ref = _fields(bufs)
    for plan, radix in (([1] * 5, 16), ([1] * 5, 8), ([0, 1, 0, 1, 0], 8), ([2, 0, 0, 0, 2], 16)):
        for lev in range(s.n_levels):
            sh = s.fft_shapes(lev)
            sh.update(plan=plan, max_radix=radix)
            s.set_fft_shapes(lev, sh)
            assert s.fft_shapes(lev)["plan"] == plan and s.fft_shapes(lev)["max_radix"] == radix
        s.step(P, 1e-3, bufs, pacc)
        assert _rel(_fields(bufs), ref) <= 2e-5, (plan, radix)
    s.close()


def test_shape_validation_and_roundtrip():
    from paper_1410_0010_gb300._lib import ApmError
    s, _ = _setup("fp32")
    sh = {"budget": [512, 1024, 2048, 4096, 8192], "threads": [128, 256, 128, 256, 128],
          "plan": [2, 1, 0, 1, 2], "max_radix": 8, "packing": 1}
    s.set_fft_shapes(1, sh)
    assert s.fft_shapes(1) == sh
    base = {"budget": [2048] * 5, "threads": [256] * 5, "plan": [0] * 5, "max_radix": 16, "packing": 0}
    for bad in ({"budget": [0] * 5}, {"threads": [48] * 5}, {"threads": [512] * 5}, {"threads": [64] * 5},
                {"plan": [3] * 5}, {"plan": [0, 2, 0, 0, 0]}, {"max_radix": 12}, {"packing": 2}):
        with pytest.raises(ApmError):
            s.set_fft_shapes(1, dict(base, **bad))
    assert s.fft_shapes(1) == sh
    s.close()


def test_cache_file_roundtrip(tmp_path):
    s, P = _setup("fp32")
    bufs = s.alloc_all()
    cache = str(tmp_path / "shapes.json")
    first = s.autotune(P, 1e-3, bufs, cache=cache)
    table = json.load(open(cache))
    assert len(table) == s.n_levels
    s.close()
    # a second context on the same shapes reads them back without tuning
    s2, P2 = _setup("fp32")
    bufs2 = s2.alloc_all()
    for lev in range(s2.n_levels):
        s2.set_fft_shapes(lev, {"budget": [2048] * 5, "threads": [256] * 5})
    again = s2.autotune(P2, 1e-3, bufs2, cache=cache)
    assert again == first
    s2.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("gradient", ["fd2", "spectral"])
def test_per_grid_launches_give_identical_bits(precision, gradient):
    """apm_set_grid_batching(0): the level solve and the accelerations run one
    launch sequence per grid (the plain per-grid path) and must reproduce the
    batched launches bit for bit."""
    import torch

    from paper_1410_0010_gb300.solver import Solver
    s, P = _setup(precision)
    s.close()
    s = Solver(GRIDS, periodic=False, precision=precision, device=0, gradient=gradient)
    bufs = s.alloc_all()
    pacc = torch.zeros((3, P.n), dtype=s.dtype, device="cuda")
    s.step(P, 1e-3, bufs, pacc)
    ref, ref_pacc = _fields(bufs), pacc.clone()
    s.set_grid_batching(False)
    for b in bufs:
        for t in b["phis"] + b["acc"]:
            t.fill_(float("nan"))
    pacc.fill_(float("nan"))
    s.profile(True)
    s.step(P, 1e-3, bufs, pacc)
    prof = s.profile_read()
    s.profile(False)
    s.sync_status()
    assert _same(_fields(bufs), ref)
    assert torch.equal(pacc, ref_pacc)
    # three refined grids: three x-forward launches on level 1, one on the root
    assert prof["fft_x_fwd"][0] == 4
    assert prof["accel_carry"][0] == 4
    s.set_grid_batching(True)
    s.close()
