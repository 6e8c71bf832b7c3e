"""Pins of the oracle's implicit resistivity (Eq. 1 curl-curl term, Sec. 2.2 resistive PCG+PC1;
reading R8): the edge current of an analytic field against its exact curl at second order, the
system's symmetry, positivity and diagonal by dense probing, the PCG solve against a dense solve,
and the invariants of the face update (div B, wall fluxes, magnetic energy)."""
import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I


def _field(g):
    """Face averages of B = cos(th) r^ + r th^ + r sin(th) ph^ (exact integrals over each face)."""
    r = g.radial_nodes()
    nt, np_ = g.nt, g.np
    th = np.linspace(0.0, np.pi, nt + 1)
    s = g.shapes
    # B_r faces (r_i, th_j..th_j+1): average of cos over the area element sin dth
    avg_cos = 0.5 * (np.sin(th[1:]) ** 2 - np.sin(th[:-1]) ** 2) / (np.cos(th[:-1]) - np.cos(th[1:]))
    br = np.broadcast_to(avg_cos[None, :, None], s["br"]).copy()
    # B_th faces (r_i..r_i+1, th_j): average of r over r dr
    avg_r = (2.0 / 3.0) * (r[1:] ** 3 - r[:-1] ** 3) / (r[1:] ** 2 - r[:-1] ** 2)
    bt = np.broadcast_to(avg_r[:, None, None], s["bt"]).copy()
    bt[:, 0] = 0.0
    bt[:, -1] = 0.0
    # B_ph faces (r_i..r_i+1, th_j..th_j+1): average of r sin over r dr dth
    num = ((r[1:] ** 3 - r[:-1] ** 3) / 3.0)[:, None] * (np.cos(th[:-1]) - np.cos(th[1:]))[None, :]
    den = ((r[1:] ** 2 - r[:-1] ** 2) / 2.0)[:, None] * (np.pi / nt)
    bp = np.broadcast_to((num / den)[:, :, None], s["bp"]).copy()
    return br, bt, bp, r, th


def _edge_errors(d):
    g = O.Grid.from_desc(d)
    br, bt, bp, r, th = _field(g)
    jr, jt, jp = g.res_current(br, bt, bp)
    nr, nt = d.nr, d.nt
    rc = 0.5 * (r[1:] + r[:-1])
    thc = 0.5 * (th[1:] + th[:-1])
    e_r = np.abs(jr[:, 1:nt] - 2.0 * np.cos(th[1:nt])[None, :, None]).max()
    e_pole = max(np.abs(jr[:, 0] - 2.0).max(), np.abs(jr[:, nt] + 2.0).max())
    e_t = np.abs(jt[1:nr] + 2.0 * np.sin(thc)[None, :, None]).max()
    jp_ex = 2.0 + np.sin(th[1:nt])[None, :] / r[1:nr, None]
    e_p = np.abs(jp[1:nr, 1:nt] - jp_ex[:, :, None]).max()
    # walls carry no resistive current
    assert np.all(jt[0] == 0.0) and np.all(jt[nr] == 0.0) and np.all(jp[0] == 0.0) and np.all(jp[nr] == 0.0)
    return np.array([e_r, e_pole, e_t, e_p])


def test_edge_current_of_analytic_field_second_order():
    # J = curl B = (2 cos th, -2 sin th, 2 + sin th / r) exactly
    coarse = _edge_errors(I.GridDesc(8, 8, 16, 1.0, 2.0, 1.0))
    fine = _edge_errors(I.GridDesc(16, 16, 32, 1.0, 2.0, 1.0))
    assert np.all(fine < 0.02), fine
    assert np.all(coarse / fine > 3.0), coarse / fine


def _dense(g, dte):
    n = g.res_size
    M = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        M[:, c] = g.res_apply(dte, e)
    return M


@pytest.mark.parametrize("dte", [1e-3, 0.3])
def test_system_symmetric_positive_definite_with_its_diagonal(dte):
    g = O.Grid.from_desc(I.GridDesc(4, 4, 6, 1.0, 3.0, 1.2))
    M = _dense(g, dte)
    scale = np.abs(M).max()
    assert np.abs(M - M.T).max() <= 1e-13 * scale
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0.0
    np.testing.assert_allclose(np.diag(M), g.res_diag(dte), rtol=1e-13, atol=1e-15 * scale)
    # the operator is not W: the curl-curl part couples faces
    assert np.count_nonzero(np.abs(M - np.diag(np.diag(M))) > 1e-14 * scale) > g.res_size


def test_pcg_matches_dense_solve():
    g = O.Grid.from_desc(I.GridDesc(4, 4, 6, 1.0, 3.0, 1.2))
    dte = 0.2
    M = _dense(g, dte)
    b = np.random.default_rng(5).normal(size=g.res_size)
    xd = np.linalg.solve(M, b)
    x, it, rr, st = g.res_pcg(dte, b, tol=1e-14)
    assert st == O.OK and rr <= 1e-14
    assert np.linalg.norm(x - xd) <= 1e-11 * np.linalg.norm(xd)
    # zero right-hand side, zero resistivity
    x0, it0, _, _ = g.res_pcg(dte, np.zeros(g.res_size))
    assert it0 == 0 and np.all(x0 == 0.0)
    x1, it1, _, st1 = g.res_pcg(0.0, b, tol=1e-13)
    assert st1 == O.OK and it1 == 1


def test_solve_keeps_div_b_wall_fluxes_and_lowers_energy():
    d = I.GridDesc(8, 6, 12, 1.0, 4.0, 1.1)
    g = O.Grid.from_desc(d)
    st = I.initial_state(d, 3, False)
    rng = np.random.default_rng(8)
    br, bt, bp = st["br"], st["bt"], st["bp"]
    # add a divergence-free perturbation with current: the CT update of random edge E
    er, et, ep = (rng.normal(size=g.shapes[k]) for k in ("er", "et", "ep"))
    et[0] = 0.0
    ep[0] = 0.0
    br, bt, bp = g.ct(er, et, ep, 0.05, br, bt, bp)
    (nbr, nbt, nbp), it, rr, s = g.res_solve(0.05, br, bt, bp, tol=1e-12)
    assert s == O.OK and it > 3
    db0, db1 = g.divb(br, bt, bp), g.divb(nbr, nbt, nbp)
    flux = np.abs(br).max() * (d.r1 ** 2)
    assert np.abs(db1 - db0).max() <= 1e-12 * flux
    assert np.array_equal(nbr[0], br[0]) and np.array_equal(nbr[-1], br[-1])
    assert np.all(nbt[:, 0] == 0.0) and np.all(nbt[:, -1] == 0.0)
    w = g.res_apply(0.0, np.ones(g.res_size))     # dte = 0: the face weights W
    e0 = float(np.sum(w * g.res_stack(br, bt, bp) ** 2))
    e1 = float(np.sum(w * g.res_stack(nbr, nbt, nbp) ** 2))
    assert e1 < e0


def test_step_with_implicit_resistivity():
    d = I.GridDesc(8, 8, 16, 1.0, 10.0, 1.05)
    st0 = I.initial_state(d, 0, False)
    g = O.Grid.from_desc(d)
    # eta = 0: the resistive solve is W B = W B*, one iteration, same step as the explicit form
    a, ia = g.step(st0, eta=0.0, tol=1e-12)
    b, ib = g.step(st0, eta=0.0, tol=1e-12, res_implicit=True)
    assert ib["status"] == O.OK and ib["res_iters"] <= 1
    for k in ("vr", "vt", "vp", "br", "bt", "bp"):
        assert np.linalg.norm(a[k] - b[k]) <= 1e-13 * np.linalg.norm(a[k]), k
    # eta > 0: div B unchanged over steps, inner flux fixed
    s = st0
    div0 = g.divb(s["br"], s["bt"], s["bp"])
    for _ in range(3):
        s, inf = g.step(s, eta=5e-3, tol=1e-10, res_implicit=True)
        assert inf["status"] == O.OK and inf["res_iters"] >= 2
    assert np.abs(g.divb(s["br"], s["bt"], s["bp"]) - div0).max() <= 1e-12 * np.abs(st0["br"]).max()
    assert np.array_equal(s["br"][0], st0["br"][0])
