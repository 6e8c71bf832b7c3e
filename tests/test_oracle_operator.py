"""Pins of the oracle's implicit operator M_alpha = D + alpha K (Eq. 1 viscous / semi-implicit
terms; Sec. 4.1 stencil operators) against closed forms and invariants."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I
from tests.helpers import centres, exact_volumes


def _manufactured_error(nr, s, alpha=1.0, r0=1.0, r1=4.0):
    d = I.GridDesc(nr, nr, 2 * nr, r0, r1, s)
    g = O.Grid.from_desc(d)
    R, TH, PH = centres(d)
    kap = math.pi / (2 * (r1 - r0))
    Rr = np.sin(kap * (R - r0))
    Y = 0.5 * np.sin(TH) * np.cos(PH) + 0.3 * np.cos(TH)     # l = 1 harmonics
    T = 1 + Y
    u = Rr * T                                               # u(r0) = 0, du/dr(r1) = 0
    rho = (r0 / R) ** 2
    # div(rho grad u) with rho r^2 = r0^2:  (r0/r)^2 u_rr + (r0^2/r^4) Lap_S u,  Lap_S Y = -2 Y
    L = (r0 ** 2 / R ** 2) * (-kap ** 2 * Rr * T) + (r0 ** 2 / R ** 4) * Rr * (-2 * Y)
    V = exact_volumes(d)[:, :, None]
    f = (rho * u - alpha * L) * V
    x, it, rr, st = g.pcg(alpha, f, tol=1e-13)
    assert st == O.OK
    e = x - u
    return math.sqrt(np.sum(V * e * e) / np.sum(V * u * u))


def test_manufactured_second_order():
    # nested refinement: stretch s -> sqrt(s) keeps the radial mapping smooth
    errs = [_manufactured_error(nr, 1.2 ** (0.5 ** lev)) for lev, nr in enumerate([8, 16, 32])]
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert errs[-1] < 5e-4
    assert ratios[-1] > 3.7, (errs, ratios)


def _rand_grid(seed=0, nr=6, nt=5, np_=8, s=1.1):
    d = I.GridDesc(nr, nt, np_, 1.0, 5.0, s)
    return d, O.Grid.from_desc(d), np.random.default_rng(seed)


def test_symmetry_and_positivity():
    d, g, rng = _rand_grid()
    for alpha in (0.0, 0.37, 25.0):
        x = rng.normal(size=(3, d.nr, d.nt, d.np))
        y = rng.normal(size=(3, d.nr, d.nt, d.np))
        Mx, My = g.apply_M(alpha, x), g.apply_M(alpha, y)
        a, b = np.sum(x * My), np.sum(Mx * y)
        assert abs(a - b) <= 1e-14 * (np.abs(x * My).sum())
        rhoV = ((1.0 / centres(d)[0]) ** 2 * exact_volumes(d)[:, :, None])
        assert np.sum(x * Mx) >= rhoV.min() * np.sum(x * x) * (1 - 1e-12)


def test_neumann_row_sums_zero():
    d, g, rng = _rand_grid(1)
    q = g.apply_K_neumann(np.ones((2, d.nr, d.nt, d.np)))
    assert np.all(q == 0.0)


def test_dirichlet_only_on_inner_shell():
    d, g, _ = _rand_grid(2)
    one = np.ones((1, d.nr, d.nt, d.np))
    k1 = g.apply_M(1.0, one) - g.apply_M(0.0, one)
    assert np.all(k1[0, 1:] == 0.0)
    assert np.all(k1[0, 0] > 0.0)


def test_mass_matrix_is_rho_volume():
    # M_0 = D = rho_c V_c: volumes tile the shell exactly, sum V = 4/3 pi (r1^3 - r0^3)
    d, g, _ = _rand_grid(3, nr=7, nt=6, np_=10, s=1.3)
    V = g.volumes()
    assert abs(V.sum() * d.np - 4.0 / 3.0 * math.pi * (d.r1 ** 3 - d.r0 ** 3)) < 1e-12 * d.r1 ** 3
    np.testing.assert_allclose(V, exact_volumes(d), rtol=1e-13)
    q = g.apply_M(0.0, np.ones((1, d.nr, d.nt, d.np)))
    R = centres(d)[0]
    np.testing.assert_allclose(q[0], (d.r0 / R) ** 2 * exact_volumes(d)[:, :, None], rtol=1e-13)


def test_diag_matches_operator_diagonal():
    d, g, _ = _rand_grid(4)
    alpha = 0.8
    D = g.diag(alpha)
    for (i, j, k) in [(0, 0, 0), (d.nr - 1, d.nt - 1, 3), (2, 2, 5)]:
        e = np.zeros((1, d.nr, d.nt, d.np))
        e[0, i, j, k] = 1.0
        assert abs(g.apply_M(alpha, e)[0, i, j, k] - D[i, j]) <= 1e-14 * D[i, j]
