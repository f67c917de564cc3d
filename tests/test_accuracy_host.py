"""The accuracy studies' reference force (paper_1410_0010_gb300.accuracy): its
quadrature of the S2 pair force from Eq. S2k against the derivative of the
oracle's closed-form pair potential, and its Newtonian limit."""
import math

import pytest


def test_s2_pair_force_matches_the_pair_potential(oracle_mod):
    pytest.importorskip("scipy")
    from paper_1410_0010_gb300 import accuracy as A
    a = 0.1
    for r in (0.002, 0.01, 0.03, 0.05, 0.07, 0.09, 0.0995):
        h = 1e-6
        ref = (oracle_mod.psi(r / a + h) - oracle_mod.psi(r / a - h)) / (2 * h) / a ** 2
        assert A.s2_pair_force(r, a) == pytest.approx(ref, rel=1e-7), r
    assert A.s2_pair_force(0.25, a) == 1 / 0.25 ** 2
    # the series and the closed form of S-hat meet at eta = 0.1
    e = 0.0999999
    assert A.s_hat(e) == pytest.approx(12 / e ** 4 * (2 - 2 * math.cos(e) - e * math.sin(e)), rel=1e-9)
