"""Pins of the oracle's adjoint step (reading P15: dt, alpha_SI, alpha_nu and upwind directions
frozen) against central finite differences of the oracle's own forward step with the same frozen
coefficients: <lam_n, d> = d/de <lam_{n+1}, step(x + e d)>."""
import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I

KEYS = ("vr", "vt", "vp", "br", "bt", "bp")


def _dot(a, b):
    return sum(float(np.sum(a[k] * b[k])) for k in KEYS)


def _axpy(x, h, d):
    return {k: x[k] + h * d[k] for k in KEYS}


def _setup(seed=0, eta=0.0, scale_v=20.0, d=I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1)):
    g = O.Grid.from_desc(d)
    st = I.initial_state(d, seed, False)
    for k in ("vr", "vt", "vp"):
        st[k] = st[k] * scale_v
    v = np.stack([st["vr"], st["vt"], st["vp"]])
    c = g.coeffs(v, st["br"], st["bt"], st["bp"], nu=1e-3, cfl=0.3)
    rng = np.random.default_rng(100 + seed)
    lam = {k: rng.normal(size=st[k].shape) for k in KEYS}
    lam["bt"][:, 0] = 0.0
    lam["bt"][:, -1] = 0.0
    return g, st, c, lam, rng


def _fd_check(g, st, c, lam, rng, eta, ndir=4, sts=False, nu=1e-3, res_implicit=False):
    dt, asi = c["dt"], c["alpha_si"]
    adj, status = g.adjoint_step(st, lam, dt, asi, nu=nu, eta=eta, cfl=0.3, sts=sts, res_implicit=res_implicit)
    assert status == O.OK

    def L(x):
        out, info = g.step(x, nu=nu, eta=eta, cfl=0.3, dt_fixed=dt, asi_fixed=asi, tol=1e-14, max_iter=200000,
                           sts=sts, res_implicit=res_implicit)
        assert info["status"] == O.OK
        return _dot(lam, out)

    errs = []
    for _ in range(ndir):
        dvec = {k: rng.normal(size=st[k].shape) for k in KEYS}
        dvec["bt"][:, 0] = 0.0
        dvec["bt"][:, -1] = 0.0
        nx = np.sqrt(_dot(st, st))
        nd = np.sqrt(_dot(dvec, dvec))
        h = 1e-6 * nx / nd
        fd = (L(_axpy(st, h, dvec)) - L(_axpy(st, -h, dvec))) / (2 * h)
        ad = _dot(adj, dvec)
        errs.append(abs(fd - ad) / max(abs(fd), abs(ad)))
    return errs


def test_adjoint_matches_central_differences():
    g, st, c, lam, rng = _setup(0)
    assert c["alpha_si"] > 0
    errs = _fd_check(g, st, c, lam, rng, 0.0)
    assert max(errs) < 1e-6, errs


def test_adjoint_with_resistivity_matches_central_differences():
    g, st, c, lam, rng = _setup(1)
    errs = _fd_check(g, st, c, lam, rng, 3e-3, ndir=3)
    assert max(errs) < 1e-6, errs


def test_adjoint_is_linear_in_cotangent():
    g, st, c, lam, rng = _setup(2)
    a1, _ = g.adjoint_step(st, lam, c["dt"], c["alpha_si"])
    lam2 = {k: 2.0 * lam[k] for k in KEYS}
    a2, _ = g.adjoint_step(st, lam2, c["dt"], c["alpha_si"])
    for k in KEYS:
        np.testing.assert_allclose(a2[k], 2.0 * a1[k], rtol=1e-9, atol=1e-12 * np.abs(a1[k]).max())


def test_inner_boundary_flux_gradient_nonzero():
    # B_r(r0) is constant in time but drives the force and E: its cotangent is nonzero
    g, st, c, lam, rng = _setup(3)
    a, _ = g.adjoint_step(st, lam, c["dt"], c["alpha_si"])
    assert np.abs(a["br"][0]).max() > 0.0


def test_adjoint_of_sts_step_matches_central_differences():
    # viscosity by RKL2 with enough stages that the polynomial is far from the identity
    g, st, c, lam, rng = _setup(3)
    nu = 1.0
    assert g.rkl2_stages(nu, c["dt"]) >= 5
    errs = _fd_check(g, st, c, lam, rng, 0.0, ndir=3, sts=True, nu=nu)
    assert max(errs) < 1e-6, errs


def test_rkl2_polynomial_is_self_adjoint_in_the_mass_inner_product():
    # P(dt L) with L = -nu D^-1 K and K symmetric satisfies <u, D P v> = <P u, D v>; the adjoint of
    # the STS step relies on it (P^T = D P D^-1)
    d = I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1)
    g = O.Grid.from_desc(d)
    rng = np.random.default_rng(7)
    u, v = rng.normal(size=(2, 3, d.nr, d.nt, d.np))
    D = g.apply_M(0.0, np.ones((1, d.nr, d.nt, d.np)))   # M_0 = D = rho V
    pu, s = g.rkl2(u, 1.0, 0.1)
    pv, _ = g.rkl2(v, 1.0, 0.1)
    assert s >= 5
    a, b = float(np.sum(u * D * pv)), float(np.sum(pu * D * v))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


def test_adjoint_with_implicit_resistivity_matches_central_differences():
    # the resistive face solve's transpose is W M_res^-1 (M_res symmetric); a large eta makes the
    # solve far from the identity
    g, st, c, lam, rng = _setup(4)
    errs = _fd_check(g, st, c, lam, rng, 0.05, ndir=3, res_implicit=True)
    assert max(errs) < 1e-6, errs
