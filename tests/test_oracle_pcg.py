"""Pins of the oracle's PCG with the point-Jacobi preconditioner PC1 (Sec. 2.2), in the
Hestenes-Stiefel form and in the single-reduction (Chronopoulos-Gear) form: every pin runs on
both, and the two forms give the same iterates up to rounding."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_1811_02605_gb300 import inputs as I


def _dense(g, alpha, n):
    M = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        M[:, c] = g.apply_M(alpha, e.reshape(1, g.nr, g.nt, g.np)).ravel()
    return M


@pytest.mark.parametrize("cg", [False, True], ids=["hs", "cg"])
def test_dense_direct_solve_6x6x8(cg):
    d = I.GridDesc(6, 6, 8, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    n = d.nr * d.nt * d.np
    rng = np.random.default_rng(7)
    for alpha in (0.05, 3.0):
        M = _dense(g, alpha, n)
        assert np.allclose(M, M.T, rtol=0, atol=1e-14 * np.abs(M).max())
        cf = sla.cho_factor(M)
        b = rng.normal(size=(3, n))
        xd = np.stack([sla.cho_solve(cf, b[c]) for c in range(3)])
        x, it, rr, st = g.pcg(alpha, b.reshape(3, d.nr, d.nt, d.np), tol=1e-14, cg=cg)
        assert st == O.OK and rr <= 1e-14
        err = np.linalg.norm(x.ravel() - xd.ravel()) / np.linalg.norm(xd.ravel())
        assert err <= 1e-12, err


@pytest.mark.parametrize("cg", [False, True], ids=["hs", "cg"])
def test_alpha_zero_one_iteration(cg):
    d = I.GridDesc(5, 4, 6, 1.0, 3.0, 1.1)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(1).normal(size=(3, 5, 4, 6))
    x, it, rr, st = g.pcg(0.0, b, tol=1e-12, cg=cg)
    assert it == 1 and st == O.OK


@pytest.mark.parametrize("cg", [False, True], ids=["hs", "cg"])
def test_zero_rhs_gives_zero(cg):
    d = I.GridDesc(5, 4, 6, 1.0, 3.0, 1.1)
    g = O.Grid.from_desc(d)
    x0 = np.ones((3, 5, 4, 6))
    x, it, rr, st = g.pcg(1.0, np.zeros((3, 5, 4, 6)), x0=x0, cg=cg)
    assert it == 0 and np.all(x == 0.0)


@pytest.mark.parametrize("cg", [False, True], ids=["hs", "cg"])
def test_energy_norm_error_decreases(cg):
    # CG minimises the M-norm of the error over the Krylov space: monotone decrease
    d = I.GridDesc(6, 6, 8, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(3).normal(size=(1, 6, 6, 8))
    alpha = 2.0
    xs, _, _, _ = g.pcg(alpha, b, tol=1e-15, cg=cg)
    prev = np.inf
    for k in range(1, 40):
        x, it, _, _ = g.pcg(alpha, b, fixed_iters=k, cg=cg)
        assert it == k
        e = x - xs
        en = float(np.sum(e * g.apply_M(alpha, e)))
        assert en <= prev * (1 + 1e-10)
        prev = en
    assert prev < 1e-6 * float(np.sum(xs * g.apply_M(alpha, xs)))


@pytest.mark.parametrize("cg", [False, True], ids=["hs", "cg"])
def test_warm_start_exact_solution_zero_iterations(cg):
    d = I.GridDesc(5, 4, 6, 1.0, 3.0, 1.1)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(2).normal(size=(3, 5, 4, 6))
    xs, _, _, _ = g.pcg(0.5, b, tol=1e-14, cg=cg)
    x, it, rr, st = g.pcg(0.5, b, x0=xs, tol=1e-9, cg=cg)
    assert it == 0 and st == O.OK


@pytest.mark.parametrize("cg", [False, True], ids=["hs", "cg"])
def test_noconv_reported(cg):
    d = I.GridDesc(6, 6, 8, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(4).normal(size=(3, 6, 6, 8))
    x, it, rr, st = g.pcg(50.0, b, tol=1e-14, max_iter=3, cg=cg)
    assert st == O.ERR_NOCONV and it == 3 and rr > 1e-14


def test_single_reduction_form_matches_hestenes_stiefel_iterates():
    # same Krylov iterates in exact arithmetic: after k iterations the two forms agree to
    # rounding, and both reach tol 1e-9 in the same number of iterations (+-1)
    d = I.GridDesc(7, 6, 10, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(11).normal(size=(3, 7, 6, 10))
    for alpha in (0.3, 5.0):
        for k in (1, 2, 5, 12):
            xa, _, _, _ = g.pcg(alpha, b, fixed_iters=k)
            xb, _, _, _ = g.pcg(alpha, b, fixed_iters=k, cg=True)
            assert np.linalg.norm(xa - xb) <= 1e-12 * np.linalg.norm(xa), (alpha, k)
        _, ia, _, _ = g.pcg(alpha, b, tol=1e-9)
        _, ib, _, _ = g.pcg(alpha, b, tol=1e-9, cg=True)
        assert abs(ia - ib) <= 1, (ia, ib)


def test_dot_is_compensated():
    # reading P12: the oracle's inner product does not depend on the order of the terms beyond
    # rounding. Terms with heavy cancellation: the exact value (rational arithmetic on the float
    # inputs) rounded to double must be reproduced to within 2 ulps, for the terms in any order
    from fractions import Fraction
    rng = np.random.default_rng(31)
    n = 4000
    a = rng.normal(size=n) * np.exp(rng.uniform(-20, 20, size=n))
    b = rng.normal(size=n)
    b[n // 2:] = -a[: n // 2] * b[: n // 2] / a[n // 2:]     # products cancel pairwise up to rounding
    b[-1] = 1.0
    exact = float(sum(Fraction(x) * Fraction(y) for x, y in zip(a, b)))
    for perm in (np.arange(n), rng.permutation(n), np.arange(n)[::-1]):
        got = O.dot(a[perm], b[perm])
        assert abs(got - exact) <= 2 * np.spacing(abs(exact)), (got, exact)
    # a plain sequential sum of the same terms is far off (the check has teeth)
    naive = 0.0
    for x, y in zip(a, b):
        naive += x * y
    assert abs(naive - exact) > 1e3 * np.spacing(abs(exact))
