"""Pin of the oracle's influence function by the property that defines it.

Sec. 2.2 introduces Eq. influence as the Green's function that minimises the
error of the mesh force against the reference force (after Hockney &
Eastwood).  This test computes that minimiser directly in real space, with no
use of Eq. influence, Eq. brillouin or Eq. assignment2, and checks that the
oracle's refined-level table equals it on every non-degenerate mode.

Set-up (cell units, delta = 1): a periodic M^3 grid, a unit source at x1 and a
unit test particle at x2.  With a table G the mesh force is TSC deposit at x1,
convolution with G on the grid, the gradient operator, TSC interpolation at
x2.  The error measure is the mean over x1 in one cell and the integral over
x2 in the box of |F_mesh - R(x2 - x1)|^2, where R is the short-range
reference force of Eq. reference, i.e. minus the gradient of
psi_{a_l}(r) - psi_{a_{l-1}}(r) with psi the S2-S2 pair potential (compact:
zero beyond a_{l-1} = 6.8 cells, so one periodic image suffices for M >= 14).

The measure is quadratic in G and separates by mode: with only the mode kappa
switched on, the mesh force is -i D(kappa) P(x2) conj(P(x1)) / M^3 with
P(x) = sum_c W(x - c) exp(i k c) (W the TSC weight), so the least-squares
value is
    G_ls(kappa) = Re[i sum_j D_j int R_j(r) B(r) dr] / (|D|^2 <|P|^2>^2)
with B(r) = <P(x) conj(P(x + r))> over x in a cell.  P and B factor by axis;
each 1-D factor is piecewise polynomial with breakpoints at cell faces, so
Gauss-Legendre rules on the pieces integrate them exactly, and the remaining
r integral (smooth R against a piecewise polynomial) converges fast in the
number of nodes per cell: the residual falls from 3e-5 (4 nodes) to 3e-7 (6)
and 1e-7 (8) of max|T|.

The oracle truncates the Brillouin sum to n in [-1,1]^3; the minimiser has no
truncation, and the difference is far below the tolerance.  Mistakes planted
in the oracle's alias numerator move its table by 3e-4 to 3e-3 of max|T| and
fail this pin: using k for k_n in D.k_n, dropping the n_x aliases, and scaling
the n != 0 terms by 1.01.
"""
import numpy as np
import pytest

import oracle

A_LEV, A_PAR = 3.4, 6.8        # a_l = 3.4 delta_l, a_{l-1} = R a_l with R = 2 (Sec. 2.2)
NODES = 8                      # Gauss-Legendre nodes per cell for the r integral
TOL = 2e-6                     # of max|T|; measured residual <= 1.1e-7 at 8 nodes

# S2-S2 pair potential psi(xi), xi = r/a, as polynomial pieces (highest power
# first); the middle piece adds -3/(35 xi).  Checked against oracle.psi, which
# its own pins tie to the transform of S-hat^2 / k^2.
_P_IN = np.array([-192 / 35, 256 / 35, 32 / 5, -64 / 5, 0, 32 / 5, 0, -104 / 35])
_P_MID = np.array([64 / 35, -256 / 35, 32 / 5, 64 / 5, -32, 128 / 5, -32 / 5, -64 / 35])


def _psi(xi):
    xs = np.maximum(xi, 1e-300)
    return np.where(xi <= 0.5, np.polyval(_P_IN, xi),
                    np.where(xi <= 1.0, np.polyval(_P_MID, xi) - 3 / (35 * xs), -1 / xs))


def _dpsi(xi):
    xs = np.maximum(xi, 1e-300)
    return np.where(xi <= 0.5, np.polyval(np.polyder(_P_IN), xi),
                    np.where(xi <= 1.0, np.polyval(np.polyder(_P_MID), xi) + 3 / (35 * xs * xs),
                             1 / (xs * xs)))


def _tsc(u):
    """TSC weight of a cell whose centre is u cells away (Sec. 2)."""
    au = np.abs(u)
    return np.where(au < 0.5, 0.75 - au * au, np.where(au < 1.5, 0.5 * (1.5 - au) ** 2, 0.0))


def _p(x, kap, M):
    """1-D factor of P: sum over cells c of W(x - c - 1/2) exp(2 pi i kap c / M)."""
    c0 = np.floor(x).astype(np.int64)
    out = np.zeros(np.shape(x), complex)
    for d in (-1, 0, 1):
        c = c0 + d
        out += _tsc(x - c - 0.5) * np.exp(2j * np.pi * kap * np.mod(c, M) / M)
    return out


_G3, _W3 = np.polynomial.legendre.leggauss(3)   # exact for the degree-4 products


def _b(r, kap, M):
    """int_0^1 p(x) conj(p(x + r)) dx, split at the face x + r crosses."""
    fr = r - np.floor(r)
    out = np.zeros(r.shape, complex)
    for lo, hi in ((np.zeros_like(fr), 1 - fr), (1 - fr, np.ones_like(fr))):
        h = hi - lo
        for g, w in zip(_G3, _W3):
            x = lo + (g + 1) / 2 * h
            out += w * h / 2 * _p(x, kap, M) * np.conj(_p(x + r, kap, M))
    return out


def _pp(kap, M):
    """<|p|^2> over one cell (exact)."""
    x = (_G3 + 1) / 2
    return float(np.sum(_W3 / 2 * np.abs(_p(x, kap, M)) ** 2))


def _d(gradient, kap, M):
    """The gradient operator's symbol times delta (readings R8, R15)."""
    th = 2 * np.pi * kap / M
    if gradient == "fd2":
        return np.sin(th)
    if gradient == "fd4":
        return (8 * np.sin(th) - np.sin(2 * th)) / 6
    return np.where(2 * kap == M, 0.0, th)


def least_squares_table(M, gradient):
    """Octant [kz, ky, kx] of the table minimising the mean-square mesh-force
    error, and the mask of the modes where it is defined (D != 0)."""
    H = M // 2 + 1
    gq, wq = np.polynomial.legendre.leggauss(NODES)
    cells = np.arange(-(M // 2), M - M // 2)
    r1 = (cells[:, None] + (gq[None, :] + 1) / 2).ravel()
    w1 = np.tile(wq / 2, M)
    RZ, RY, RX = np.meshgrid(r1, r1, r1, indexing="ij")
    rn = np.sqrt(RX ** 2 + RY ** 2 + RZ ** 2)
    dpot = _dpsi(rn / A_LEV) / A_LEV ** 2 - _dpsi(rn / A_PAR) / A_PAR ** 2
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(rn > 0, -dpot / rn, 0.0)        # R = f r: force on the test particle
    W = w1[:, None, None] * w1[None, :, None] * w1[None, None, :]
    kaps = np.arange(H)
    B = np.stack([_b(r1, k, M) for k in kaps])
    I = [np.einsum("zyx,cz,by,ax->cba", f * comp * W, B, B, B, optimize=True) for comp in (RX, RY, RZ)]
    D = _d(gradient, kaps, M)
    PP = np.array([_pp(k, M) for k in kaps])
    KZ, KY, KX = np.meshgrid(kaps, kaps, kaps, indexing="ij")
    num = np.real(1j * (D[KX] * I[0] + D[KY] * I[1] + D[KZ] * I[2]))
    den = (D[KX] ** 2 + D[KY] ** 2 + D[KZ] ** 2) * (PP[KX] * PP[KY] * PP[KZ]) ** 2
    ok = den > 1e-12 * den.max()
    return np.where(ok, num / np.where(ok, den, 1.0), 0.0), ok


def _oracle_table(M, gradient):
    cfg = oracle.Config(periodic=False, gradient=gradient)
    plan = oracle.Plan(1, 1.0, A_LEV, A_PAR, 5, (M, M, M), (0, 0, 0), (M, M, M), (0, 0, 0),
                       (M, M, M), 0, 0)
    return oracle.green_table(cfg, plan)


def test_pair_potential_pieces_match_oracle():
    xi = np.linspace(0.01, 1.6, 160)
    np.testing.assert_allclose(_psi(xi), [oracle.psi(v) for v in xi], rtol=1e-13, atol=1e-13)
    h = 1e-6       # the derivative pieces against a difference of the oracle's psi
    fd = np.array([(oracle.psi(v + h) - oracle.psi(v - h)) / (2 * h) for v in xi])
    np.testing.assert_allclose(_dpsi(xi), fd, rtol=1e-7, atol=1e-7)


@pytest.mark.parametrize("M,gradient", [(16, "fd2"), (15, "fd2"), (18, "fd2"), (16, "fd4"),
                                        (16, "spectral"), (18, "spectral")])
def test_refined_table_is_the_force_error_minimiser(M, gradient):
    T = _oracle_table(M, gradient)
    G, ok = least_squares_table(M, gradient)
    scale = np.abs(T).max()
    err = np.abs(G - T)[ok].max() / scale
    assert err < TOL, f"M={M} {gradient}: max |G_ls - T| = {err:.2e} of max|T|"
    # modes with D = 0 are the degenerate set of reading R5 plus kappa = 0
    assert np.all(T[~ok][1:] == 0.0)
