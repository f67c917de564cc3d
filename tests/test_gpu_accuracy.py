"""The accuracy studies (paper_1410_0010_gb300.accuracy) on the GPU, FP64, with
the trends the paper states or the method implies:
* padding (Sec. 2.2): the refined level's accelerations converge as the border
  grows, and the paper's 0.65 R a / delta (B = 5) is within 1e-4 of a border
  of 9 cells, where B = 2 is off by more than 1e-3;
* softening (Sec. 2.2, after HE): the error against the S2 reference force
  falls as a / delta grows;
* the mesh force is Newtonian beyond the softening within a few percent on
  average, and its scatter falls from the two-point to the four-point to the
  spectral gradient;
* Fig. 2 (Sec. 2.2): each refined level adds force only inside about twice its
  own softening, and the total follows 1/r^2 outside the finest softening."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_padding_converges_at_the_papers_border():
    from paper_1410_0010_gb300 import accuracy as A
    rows = A.padding_sweep(pads=(0.15, 0.3, 0.45, 0.65, 0.8))
    errs = [r["rel_l2"] for r in rows]
    print("padding", [(r["pad_factor"], r["border"], f"{r['rel_l2']:.2e}") for r in rows])
    assert [r["border"] for r in rows] == [2, 3, 4, 5, 6]
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[0] > 1e-3 and errs[3] < 1e-4


def test_force_errors_softening_and_gradients():
    from paper_1410_0010_gb300 import accuracy as A
    base = A.force_errors(centres=4, per_centre=300)
    print("fd2", base)
    assert abs(base["far"]["mean"]) < 0.01 and base["far"]["rms"] < 0.03
    assert abs(base["near"]["mean"]) < 0.03 and base["near"]["rms"] < 0.06
    soft = [A.force_errors(centres=4, per_centre=300, a_over_dx=v)["near"]["rms"] for v in (2.0, 3.4, 5.0)]
    print("softening near rms", soft)
    assert soft[0] > soft[1] > soft[2]
    far = {g: A.force_errors(centres=4, per_centre=300, gradient=g)["far"]["rms"] for g in ("fd2", "fd4", "spectral")}
    print("far rms by gradient", far)
    assert far["spectral"] < far["fd4"] < far["fd2"]


def test_force_decomposition_fig2():
    from paper_1410_0010_gb300 import accuracy as A
    t = A.force_decomposition()
    r = np.array(t["r"])
    newton = np.array(t["newton"])
    for lev in range(1, len(t["levels"])):
        own = np.array([np.nan if v is None else v for v in t["levels"][lev]])
        a = t["a"][lev]
        far = (r > 2.5 * a) & np.isfinite(own)
        near = (r > 0.5 * a) & (r < a) & np.isfinite(own)
        assert far.any() and near.any()
        # confined: beyond 2.5 a_l the level adds under 1% of 1/r^2
        assert np.all(np.abs(own[far]) < 0.01 * newton[far]), (lev, own[far] / newton[far])
        # and between a_l / 2 and a_l it carries a good part of the force
        assert np.all(own[near] > 0.1 * newton[near]), (lev, own[near] / newton[near])
    ratio = np.array([np.nan if v is None else v for v in t["total_ratio"]])
    outside = (r > 2 * t["a"][-1]) & (r < 0.3) & np.isfinite(ratio)
    print("total / Newton", dict(zip(np.round(r[outside], 4), np.round(ratio[outside], 3))))
    assert np.all(np.abs(ratio[outside] - 1) < 0.03)
