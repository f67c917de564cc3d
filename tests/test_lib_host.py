"""Host-side checks of libapm that need no GPU: the library builds and loads,
exports every function include/apm.h declares, and its host-only entry points
(defaults, status strings, hierarchy validation, argument checks) behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1410_0010_gb300 import _lib, buildlib
    buildlib.build()
    return _lib.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "apm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(apm_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_function(L):
    from paper_1410_0010_gb300 import _lib
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
        assert n in _lib.SIGNATURES, f"binding lacks {n}"


def test_defaults_are_the_papers(L):
    from paper_1410_0010_gb300._lib import ApmConfig
    c = ApmConfig()
    L.apm_config_default(ctypes.byref(c))
    assert c.a_over_dx == 3.4 and c.refine == 2 and c.pad_factor == 0.65   # Sec. 2.2
    assert c.box == 1.0 and c.root_bc == 0 and c.mass_frac_bits == 52 and c.device == -1
    assert c.gradient == 0                                                  # two-point difference
    assert L.apm_version().startswith(b"apm-gb300")
    for code in range(11):
        assert len(L.apm_status_string(code)) >= 2
    assert L.apm_status_string(99) == b"unknown status"


def test_create_rejects_bad_config_before_touching_cuda(L):
    from paper_1410_0010_gb300._lib import ApmConfig
    c = ApmConfig()
    L.apm_config_default(ctypes.byref(c))
    ctx = ctypes.c_void_p()
    bad = [("box", -1.0), ("mass_frac_bits", 63), ("mass_frac_bits", 0), ("root_bc", 5),
           ("precision", 7), ("refine", 1), ("gradient", 3), ("gradient", -1)]
    for field, value in bad:
        cc = ApmConfig()
        ctypes.pointer(cc)[0] = c
        setattr(cc, field, value)
        assert L.apm_create(ctypes.byref(cc), ctypes.byref(ctx)) == 1, field
    cc = ApmConfig()
    ctypes.pointer(cc)[0] = c
    cc.refine = 4
    assert L.apm_create(ctypes.byref(cc), ctypes.byref(ctx)) == 8   # unsupported


def test_calls_without_context_fail_cleanly(L):
    assert L.apm_deposit(None, 0, None, 0.0, None, None, None, None) == 1
    assert L.apm_solve_level(None, 0, None, None, None) == 1
    assert L.apm_accel(None, 0, None, None, None, None, None, None) == 1
    assert L.apm_interp(None, 0, None, None, 0.0, None, None) == 1
    assert L.apm_sync_status(None, None) == 1
    assert L.apm_num_levels(None) == 0
    L.apm_destroy(None)


def _grids(descs):
    from paper_1410_0010_gb300._lib import ApmGrid
    arr = (ApmGrid * len(descs))()
    for i, (lev, par, st, dm) in enumerate(descs):
        arr[i].level, arr[i].parent = lev, par
        for j in range(3):
            arr[i].start[j], arr[i].dims[j] = st[j], dm[j]
    return arr


def _validate(L, descs, periodic=False):
    from paper_1410_0010_gb300._lib import APM_BC_PERIODIC, ApmConfig
    c = ApmConfig()
    L.apm_config_default(ctypes.byref(c))
    if periodic:
        c.root_bc = APM_BC_PERIODIC
    return L.apm_validate_hierarchy(ctypes.byref(c), _grids(descs), len(descs))


ROOT32 = (0, -1, (0, 0, 0), (32, 32, 32))


def test_validation_accepts_the_papers_hierarchies(L):
    import apm_inputs as W
    for bounds in (W.FIG1_BOUNDS, W.POINT_SOURCE_CENTRE, W.POINT_SOURCE_CORNER, W.SINE_WAVE_BOUNDS):
        root = 64 if bounds is W.SINE_WAVE_BOUNDS else 32
        descs = [tuple(g) for g in W.grids_from_bounds(root, bounds)]
        assert _validate(L, descs) == 0, bounds


def test_validation_nesting_rules(L):
    ok = [ROOT32, (1, 0, (12, 12, 12), (20, 20, 20))]
    assert _validate(L, ok) == 0
    # parent cells of the border: child start 10 -> border cells from 5 -> parent 2: ok;
    # start 4 -> border from -1 -> parent -1: outside a periodic root
    assert _validate(L, [ROOT32, (1, 0, (4, 12, 12), (8, 8, 8))], periodic=True) == 2
    assert _validate(L, [ROOT32, (1, 0, (6, 12, 12), (8, 8, 8))], periodic=True) == 0
    # upper edge: parent cell floor((start + N + B - 1)/2) must be < 32
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 52), (8, 8, 8))], periodic=True) == 2
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 52), (8, 8, 6))], periodic=True) == 0
    # an isolated root has nothing outside it: the border may leave the box, the
    # carry of cells [-1, N] may not (start 1: cell -1 reads parent cell -1)
    assert _validate(L, [ROOT32, (1, 0, (4, 12, 12), (8, 8, 8))]) == 0
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 52), (8, 8, 8))]) == 0
    assert _validate(L, [ROOT32, (1, 0, (2, 12, 12), (8, 8, 8))]) == 0
    assert _validate(L, [ROOT32, (1, 0, (1, 12, 12), (8, 8, 8))]) == 2
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 54), (8, 8, 8))]) == 0
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 55), (8, 8, 8))]) == 2
    # deeper levels keep the full rule: level 2 at start 8 has border cells from 3,
    # in level-1 cell 1, outside its parent (cells [2, 22))
    lev1 = (1, 0, (2, 2, 2), (20, 20, 20))
    assert _validate(L, [ROOT32, lev1, (2, 1, (10, 10, 10), (8, 8, 8))]) == 0
    assert _validate(L, [ROOT32, lev1, (2, 1, (8, 10, 10), (8, 8, 8))]) == 2
    # overlapping siblings
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 12), (10, 10, 10)),
                         (1, 0, (20, 20, 20), (10, 10, 10))]) == 2
    # touching siblings are fine
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 12), (10, 10, 10)),
                         (1, 0, (22, 12, 12), (10, 10, 10))]) == 0
    # wrong parent level, missing level, second root, bad root
    assert _validate(L, [ROOT32, (2, 0, (40, 40, 40), (8, 8, 8))]) == 2
    assert _validate(L, [ROOT32, ROOT32]) == 2
    assert _validate(L, [(0, -1, (0, 0, 0), (32, 32, 16))]) == 1
    assert _validate(L, [(0, -1, (1, 0, 0), (32, 32, 32))]) == 2
    assert _validate(L, [ROOT32, (1, 0, (12, 12, 12), (0, 4, 4))]) == 1


def test_package_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1410_0010_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        _lib.lib()


def test_binding_checks_tensors_before_the_c_abi():
    import torch

    from paper_1410_0010_gb300.solver import check_field
    ok = torch.zeros((3, 5), dtype=torch.float32)
    check_field(ok, (3, 5), torch.float32, None, "acc")
    with pytest.raises(ValueError, match="shape"):
        check_field(ok, (3, 6), torch.float32, None, "acc")
    with pytest.raises(ValueError, match="dtype"):
        check_field(ok, (3, 5), torch.float64, None, "acc")
    with pytest.raises(ValueError, match="contiguous"):
        check_field(torch.zeros((5, 3)).t(), (3, 5), torch.float32, None, "acc")
    with pytest.raises(ValueError, match="context"):
        check_field(ok, (3, 5), torch.float32, torch.device("cuda", 0), "acc")
    with pytest.raises(TypeError):
        check_field([0.0], (1,), torch.float32, None, "acc")


def _rules_hold(descs, periodic, B=5):
    """The nesting rules of apm_set_hierarchy written out (reading R9): a root
    first; every other grid's parent one level up; levels contiguous; the
    parent cells that a child's GMF border (floor((start - B) / 2) ..
    floor((start + N + B - 1) / 2)) and the carry of its cells [-1, N] read lie
    in the parent's interior, except that a level-1 border may leave an
    isolated root; sibling interiors disjoint."""
    import math
    root = descs[0]
    if root[0] != 0 or root[1] != -1 or any(root[2]) or len(set(root[3])) != 1:
        return False
    levels = set()
    for i, (lev, par, st, dm) in enumerate(descs):
        if i == 0:
            continue
        if lev < 1 or not (0 <= par < len(descs)) or par == i or descs[par][0] != lev - 1:
            return False
        levels.add(lev)
        p = descs[par]
        past_root = par == 0 and not periodic
        for j in range(3):
            lo_b, hi_b = (st[j] - B) // 2, (st[j] + dm[j] + B - 1) // 2
            lo_c = math.floor((st[j] - 1 + 0.5) / 2 - 0.5)
            hi_c = math.floor((st[j] + dm[j] + 0.5) / 2 - 0.5) + 1
            lo, hi = (lo_c, hi_c) if past_root else (min(lo_b, lo_c), max(hi_b, hi_c))
            if lo < p[2][j] or hi >= p[2][j] + p[3][j]:
                return False
    if levels and levels != set(range(1, max(levels) + 1)):
        return False
    for i in range(1, len(descs)):
        for k in range(i + 1, len(descs)):
            a, b = descs[i], descs[k]
            if a[0] == b[0] and all(a[2][j] < b[2][j] + b[3][j] and b[2][j] < a[2][j] + a[3][j]
                                    for j in range(3)):
                return False
    return True


def test_validation_agrees_with_the_rules_on_random_hierarchies(L):
    import random
    rnd = random.Random(12)
    agree = {True: 0, False: 0}
    nested = 0
    for t in range(600):
        n0 = rnd.choice([16, 20, 24])
        descs = [(0, -1, (0, 0, 0), (n0, n0, n0))]
        for lev in range(1, rnd.randint(2, 4)):
            parents = [i for i, d in enumerate(descs) if d[0] == lev - 1]
            for _ in range(1 if rnd.random() < 0.75 else 2):
                par = rnd.choice(parents)
                p = descs[par]
                st, dm = [], []
                near = rnd.random() < 0.8
                for j in range(3):
                    lo, hi = 2 * p[2][j], 2 * (p[2][j] + p[3][j])
                    if near:                    # near the legal range: margins of 5 to 8 cells,
                        m = lambda: rnd.randint(5, 8) if rnd.random() < 0.9 else rnd.randint(2, 4)
                        s0 = lo + m()             # now and then 2 to 4 (the border leaves the parent)
                        e0 = max(s0 + 2, hi - m())
                    else:                       # anywhere around the parent
                        s0 = lo + rnd.randint(-2, hi - lo)
                        e0 = s0 + rnd.randint(2, hi - lo)
                    st.append(s0)
                    dm.append(e0 - s0)
                descs.append((lev, par, tuple(st), tuple(dm)))
        periodic = rnd.random() < 0.5
        want = _rules_hold(descs, periodic)
        got = _validate(L, descs, periodic=periodic)
        assert (got == 0) == want, (descs, periodic, got)
        agree[want] += 1
        nested += want and len(descs) > 1
    assert agree[False] > 100 and nested > 100, (agree, nested)
