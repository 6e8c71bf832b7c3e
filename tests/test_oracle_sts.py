"""Pins of the oracle's RKL2 super time-stepping for viscosity (Sec. 2.2 STS option, algorithm 3;
Meyer, Balsara & Aslam 2014) against the exact propagator exp(dt A), A = -nu D^-1 K, of a small grid
(dense matrix from the oracle's operator, matrix exponential from numpy's eigendecomposition)."""
import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I

D = I.GridDesc(4, 4, 6, 1.0, 3.0, 1.1)


def _dense_A(g, nu):
    n = g.N
    K = np.empty((n, n))
    for c in range(n):
        e = np.zeros((1, g.nr, g.nt, g.np))
        e.ravel()[c] = 1.0
        K[:, c] = (g.apply_M(1.0, e) - g.apply_M(0.0, e)).ravel()
    rhoV = g.apply_M(0.0, np.ones((1, g.nr, g.nt, g.np))).ravel()
    # A = -nu D^-1 K is similar to the symmetric S = -nu D^-1/2 K D^-1/2
    Dh = 1.0 / np.sqrt(rhoV)
    S = -nu * (Dh[:, None] * K * Dh[None, :])
    w, Q = np.linalg.eigh(S)
    return w, Q, Dh


def _expm_apply(w, Q, Dh, t, v):
    # exp(t A) v = D^-1/2 Q exp(t w) Q^T D^1/2 v
    y = Q.T @ (v / Dh)
    return Dh * (Q @ (np.exp(t * w) * y))


def test_rkl2_local_error_third_order_fixed_stages():
    g = O.Grid.from_desc(D)
    nu = 0.05
    w, Q, Dh = _dense_A(g, nu)
    rng = np.random.default_rng(3)
    v = rng.normal(size=(3, D.nr, D.nt, D.np))
    errs = []
    for dt in (2e-3, 1e-3, 5e-4):
        x, s = g.rkl2(v, nu, dt, stages=7)
        ex = np.stack([_expm_apply(w, Q, Dh, dt, v[c].ravel()).reshape(v[c].shape) for c in range(3)])
        errs.append(np.linalg.norm(x - ex) / np.linalg.norm(ex))
    r = [errs[i] / errs[i + 1] for i in range(2)]
    assert 7.0 < r[-1] < 9.0, (errs, r)


def test_rkl2_automatic_stages_are_stable_and_second_order_in_time():
    g = O.Grid.from_desc(D)
    nu = 0.05
    w, Q, Dh = _dense_A(g, nu)
    lam = -w.min()
    rng = np.random.default_rng(4)
    v = rng.normal(size=(3, D.nr, D.nt, D.np))
    T = 0.4
    errs = []
    for n in (4, 8, 16):
        dt = T / n
        s = g.rkl2_stages(nu, dt)
        assert (s * s + s - 2) / 2.0 >= dt * lam  # Gershgorin bound covers the true spectrum
        x = v.copy()
        for _ in range(n):
            x, _ = g.rkl2(x, nu, dt)
        ex = np.stack([_expm_apply(w, Q, Dh, T, v[c].ravel()).reshape(v[c].shape) for c in range(3)])
        errs.append(np.linalg.norm(x - ex) / np.linalg.norm(ex))
    r = [errs[i] / errs[i + 1] for i in range(2)]
    assert r[-1] > 3.2, (errs, r)
    # amplification of the stiffest eigenmode stays <= 1 at the chosen stage count
    dt = 0.2
    s = g.rkl2_stages(nu, dt)
    top = (Q[:, np.argmin(w)] * Dh).reshape(1, D.nr, D.nt, D.np)
    vt = np.concatenate([top, top, top])
    x, _ = g.rkl2(vt, nu, dt, stages=s)
    assert np.linalg.norm(x) <= np.linalg.norm(vt) * (1 + 1e-12)


def test_rkl2_uniform_field_decays_from_the_dirichlet_wall_only():
    # K 1 is zero except in the inner shell (Dirichlet face at r0): a uniform field loses momentum
    # there first; the outer shell, several cells away, is still almost untouched after one step
    g = O.Grid.from_desc(D)
    one = np.ones((3, D.nr, D.nt, D.np))
    x, s = g.rkl2(one, 0.05, 0.02)
    assert np.all(x[:, 0] < 1.0)
    assert np.abs(x[:, -1] - 1.0).max() < 0.05 * np.abs(x[:, 0] - 1.0).max()


def test_step_sts_matches_step_without_viscosity_and_damps_with_it():
    d = I.GridDesc(8, 8, 16, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    st = I.initial_state(d, 0, False)
    a, ia = g.step(st, nu=0.0, dt_fixed=0.05, tol=1e-12)
    b, ib = g.step_sts(st, nu=0.0, dt_fixed=0.05, tol=1e-12)
    for k in a:
        assert np.allclose(a[k], b[k], rtol=1e-12, atol=1e-15)
    c, ic = g.step_sts(st, nu=5e-2, dt_fixed=0.05, tol=1e-12)
    e, ie = g.step(st, nu=5e-2, dt_fixed=0.05, tol=1e-12)
    assert ic["iters"][2] >= 2
    ke = lambda s_: float(np.sum(s_["vr"] ** 2 + s_["vt"] ** 2 + s_["vp"] ** 2))
    assert ke(c) < ke(a) and ke(e) < ke(a)
    # explicit STS and implicit backward Euler approximate the same viscous decay (first order apart)
    assert abs(ke(c) - ke(e)) < 0.1 * (ke(a) - ke(e))
