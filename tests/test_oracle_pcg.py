"""Pins of the oracle's PCG with the point-Jacobi preconditioner PC1 (Sec. 2.2)."""
import numpy as np
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


def test_dense_direct_solve_6x6x8():
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
        x, it, rr, st = g.pcg(alpha, b.reshape(3, d.nr, d.nt, d.np), tol=1e-14)
        assert st == O.OK and rr <= 1e-14
        err = np.linalg.norm(x.ravel() - xd.ravel()) / np.linalg.norm(xd.ravel())
        assert err <= 1e-12, err


def test_alpha_zero_one_iteration():
    d = I.GridDesc(5, 4, 6, 1.0, 3.0, 1.1)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(1).normal(size=(3, 5, 4, 6))
    x, it, rr, st = g.pcg(0.0, b, tol=1e-12)
    assert it == 1 and st == O.OK


def test_zero_rhs_gives_zero():
    d = I.GridDesc(5, 4, 6, 1.0, 3.0, 1.1)
    g = O.Grid.from_desc(d)
    x0 = np.ones((3, 5, 4, 6))
    x, it, rr, st = g.pcg(1.0, np.zeros((3, 5, 4, 6)), x0=x0)
    assert it == 0 and np.all(x == 0.0)


def test_energy_norm_error_decreases():
    # CG minimises the M-norm of the error over the Krylov space: monotone decrease
    d = I.GridDesc(6, 6, 8, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(3).normal(size=(1, 6, 6, 8))
    alpha = 2.0
    xs, _, _, _ = g.pcg(alpha, b, tol=1e-15)
    prev = np.inf
    for k in range(1, 40):
        x, it, _, _ = g.pcg(alpha, b, fixed_iters=k)
        assert it == k
        e = x - xs
        en = float(np.sum(e * g.apply_M(alpha, e)))
        assert en <= prev * (1 + 1e-10)
        prev = en
    assert prev < 1e-6 * float(np.sum(xs * g.apply_M(alpha, xs)))


def test_warm_start_exact_solution_zero_iterations():
    d = I.GridDesc(5, 4, 6, 1.0, 3.0, 1.1)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(2).normal(size=(3, 5, 4, 6))
    xs, _, _, _ = g.pcg(0.5, b, tol=1e-14)
    x, it, rr, st = g.pcg(0.5, b, x0=xs, tol=1e-9)
    assert it == 0 and st == O.OK


def test_noconv_reported():
    d = I.GridDesc(6, 6, 8, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    b = np.random.default_rng(4).normal(size=(3, 6, 6, 8))
    x, it, rr, st = g.pcg(50.0, b, tol=1e-14, max_iter=3)
    assert st == O.ERR_NOCONV and it == 3 and rr > 1e-14
