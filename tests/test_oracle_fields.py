"""Pins of the oracle's explicit pieces: current density, momentum force, electric field and
constrained-transport induction, step coefficients (Eq. 1; Sec. 2.1 for S; Sec. 2.2 for the
explicit upwind predictor-corrector)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I
from tests.helpers import cart, centres, dipole_B, exact_volumes, to_sph, wl2, zero_faces


def _grid(nr, s=1.0, r1=4.0):
    d = I.GridDesc(nr, nr, 2 * nr, 1.0, r1, s)
    return d, O.Grid.from_desc(d)


def _rates(errs):
    return [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]


# ----------------------------------------------------------------------------- current density
def _j_error(nr, kind):
    d, g = _grid(nr)
    R, TH, PH = centres(d)
    if kind == "rotation":   # B = z x x, J = 2 z
        br, bt, bp = I.magnetic_field(d, dipole=False,
                                      potential=lambda x: np.stack([0 * x[0], 0 * x[0], -(x[0] ** 2 + x[1] ** 2) / 2]))
        ex, sc = np.stack([2 * np.cos(TH), -2 * np.sin(TH), 0 * TH]), 2.0
    elif kind == "dipole":   # potential field: J = 0
        br, bt, bp = I.magnetic_field(d, dipole=True)
        ex, sc = np.zeros((3,) + R.shape), 1.0 / R ** 3
    else:                    # B = sin(theta) phi_hat: J = (2 cos/r, -sin/r, 0)
        br, bt, bp = I.magnetic_field(d, dipole=False,
                                      potential=lambda x: x * (x[2] / np.sqrt(np.sum(x * x, axis=0)))[None])
        ex, sc = np.stack([2 * np.cos(TH) / R, -np.sin(TH) / R, 0 * TH]), 1.0 / R
    J = g.current_centre(br, bt, bp)
    V = exact_volumes(d)[:, :, None]
    return wl2(V, np.sum((J - ex) ** 2, axis=0), sc ** 2 * np.ones_like(R), slice(1, -1))


@pytest.mark.parametrize("kind,rate", [("rotation", 3.8), ("dipole", 3.3), ("azimuthal", 3.8)])
def test_current_second_order_interior(kind, rate):
    errs = [_j_error(nr, kind) for nr in (8, 16, 32)]
    assert _rates(errs)[-1] > rate, errs


def test_current_outer_ghost_rule_exact_for_r_independent_field():
    # B = sin(theta) phi_hat: the zero-gradient ghost is exact, J_theta(r1) = -B_phi / r1
    d, g = _grid(16)
    br, bt, bp = I.magnetic_field(d, dipole=False,
                                  potential=lambda x: x * (x[2] / np.sqrt(np.sum(x * x, axis=0)))[None])
    jr, jt, jp = g.current_edges(br, bt, bp)
    thc = (np.arange(d.nt) + 0.5) * math.pi / d.nt
    # face-averaged sin(theta) over the band vs sin(theta_c): O(dth^2)
    assert np.abs(jt[-1, :, 0] + np.sin(thc) / d.r1).max() < 2e-3
    assert np.all(jp[:, 0] == 0.0) and np.all(jp[:, -1] == 0.0)


def test_polar_current_is_cap_circulation():
    # J_r on the polar axis is single-valued and -> 2 for B = z x x
    d, g = _grid(32)
    br, bt, bp = I.magnetic_field(d, dipole=False,
                                  potential=lambda x: np.stack([0 * x[0], 0 * x[0], -(x[0] ** 2 + x[1] ** 2) / 2]))
    jr, _, _ = g.current_edges(br, bt, bp)
    assert np.all(jr[:, 0, :] == jr[:, 0, :1])
    assert np.abs(jr[:, 0, 0] - 2.0).max() < 1e-2
    assert np.abs(jr[:, -1, 0] + 2.0).max() < 1e-2   # z-hat is -r-hat at the south pole


# ----------------------------------------------------------------------------- momentum force
def _force_error(nr, kind, seed=5):
    d, g = _grid(nr)
    R, TH, PH = centres(d)
    X = cart(R, TH, PH)
    br, bt, bp = zero_faces(d)
    if kind == "uniform":            # (v.grad)v = 0
        vc, ex, sc = np.stack([np.ones_like(R), 0 * R, 0 * R]), 0 * X, 1.0
    elif kind == "rotation":         # (v.grad)v = -(x, y, 0)
        vc, ex, sc = np.stack([-X[1], X[0], 0 * R]), np.stack([X[0], X[1], 0 * R]), R
    elif kind == "modes":
        m = I.draw_modes(np.random.default_rng(seed), 1.0, 1.0 / 4.0)
        f = lambda x: I.modes_eval(m, x)
        h = 1e-5
        vc = f(X)
        adv = np.zeros_like(X)
        for a in range(3):
            e = np.zeros((3, 1, 1, 1))
            e[a] = 1.0
            adv += vc[a][None] * (f(X + h * e) - f(X - h * e)) / (2 * h)
        ex, sc = -adv, 1.0
    else:                            # J x B / rho with B = z x x, v = 0: 2 z x B
        vc = 0 * X
        br, bt, bp = I.magnetic_field(d, dipole=False,
                                      potential=lambda x: np.stack([0 * x[0], 0 * x[0], -(x[0] ** 2 + x[1] ** 2) / 2]))
        B = np.stack([-X[1], X[0], 0 * R])
        ex = np.stack([-2 * B[1], 2 * B[0], 0 * R]) * (R / d.r0) ** 2
        sc = R ** 3
    v = np.ascontiguousarray(to_sph(vc, TH, PH))
    exs = to_sph(ex, TH, PH)
    dt = 0.1
    b = g.force(v, br, bt, bp, dt)
    V = exact_volumes(d)[:, :, None]
    F = b / ((d.r0 / R) ** 2 * V * dt)
    return wl2(V, np.sum((F - exs) ** 2, axis=0), sc ** 2 * np.ones_like(R), slice(1, -1))


def test_force_rigid_rotation_exact():
    # only the curvature terms act: exact to round-off
    for nr in (8, 16):
        assert _force_error(nr, "rotation") < 1e-13


@pytest.mark.parametrize("kind", ["uniform", "modes"])
def test_force_upwind_first_order(kind):
    errs = [_force_error(nr, kind) for nr in (8, 16, 32)]
    r = _rates(errs)
    assert 1.8 < r[-1] < 2.3, (errs, r)


def test_force_lorentz_second_order():
    errs = [_force_error(nr, "lorentz") for nr in (8, 16, 32)]
    assert _rates(errs)[-1] > 3.5, errs


def test_force_zero_state():
    d, g = _grid(6)
    br, bt, bp = zero_faces(d)
    assert np.all(g.force(np.zeros((3, 6, 6, 12)), br, bt, bp, 0.3) == 0.0)


# ----------------------------------------------------------------------------- induction / CT
def test_ct_preserves_divergence_for_arbitrary_E():
    d = I.GridDesc(6, 5, 8, 1.0, 3.0, 1.2)
    g = O.Grid.from_desc(d)
    st = I.initial_state(d, 0, False)
    br, bt, bp = st["br"], st["bt"], st["bp"]
    rng = np.random.default_rng(11)
    s = g.shapes
    er, et, ep = (rng.normal(size=s["er"]), rng.normal(size=s["et"]), rng.normal(size=s["ep"]))
    er[:, 0, :] = er[:, 0, :1]       # the polar axis edge is single-valued
    er[:, -1, :] = er[:, -1, :1]
    d0 = g.divb(br, bt, bp)
    br2, bt2, bp2 = g.ct(er, et, ep, 0.7, br, bt, bp)
    d1 = g.divb(br2, bt2, bp2)
    V = exact_volumes(d)
    r = I.radial_nodes(d)
    scale = np.abs(br2).max() * (r[-1] ** 2) * 4 * math.pi + np.abs(bt2).max() * r[-1] ** 2 + np.abs(bp2).max() * r[-1] ** 2
    assert np.abs(d1 - d0).max() <= 1e-13 * scale
    assert np.all(bt2[:, 0] == 0.0) and np.all(bt2[:, -1] == 0.0)


def test_ct_line_tied_inner_boundary_and_static():
    d = I.GridDesc(6, 6, 8, 1.0, 3.0, 1.1)
    g = O.Grid.from_desc(d)
    st = I.initial_state(d, 0, False)
    v = np.stack([st["vr"], st["vt"], st["vp"]])
    er, et, ep = g.efield_edges(v, st["br"], st["bt"], st["bp"])
    br2, bt2, bp2 = g.ct(er, et, ep, 0.5, st["br"], st["bt"], st["bp"])
    assert np.all(br2[0] == st["br"][0])
    assert not np.all(br2[-1] == st["br"][-1])     # outer shell evolves
    z = np.zeros_like(v)
    er, et, ep = g.efield_edges(z, st["br"], st["bt"], st["bp"])
    br3, bt3, bp3 = g.ct(er, et, ep, 0.5, st["br"], st["bt"], st["bp"])
    assert np.array_equal(br3, st["br"]) and np.array_equal(bt3, st["bt"]) and np.array_equal(bp3, st["bp"])


def _dipole_rate(V0, X):
    # dB/dt = curl(v x B) = -(v.grad)B for uniform v and the dipole, by central differences
    h = 1e-6
    dB = np.zeros_like(X)
    for a in range(3):
        e = np.zeros((3, 1, 1, 1))
        e[a] = 1.0
        dB -= V0[a] * (dipole_B(X + h * e) - dipole_B(X - h * e)) / (2 * h)
    return dB


def _ct_translation_errors(nr):
    """Error of dB/dt from one CT update of a dipole carried by a uniform flow, on the three face
    families, split into the rows next to the poles and the rest (r boundaries left out)."""
    d, g = _grid(nr)
    br, bt, bp = I.magnetic_field(d, dipole=True)
    R, TH, PH = centres(d)
    V0 = np.array([1.0, 0.5, 0.2])
    v = np.ascontiguousarray(to_sph(np.broadcast_to(V0.reshape(3, 1, 1, 1), (3,) + R.shape), TH, PH))
    er, et, ep = g.efield_edges(v, br, bt, bp)
    dt = 1e-3
    br2, bt2, bp2 = g.ct(er, et, ep, dt, br, bt, bp)
    r = I.radial_nodes(d)
    rc = 0.5 * (r[1:] + r[:-1])
    thc = (np.arange(nr) + 0.5) * math.pi / nr
    thn = np.arange(nr + 1) * math.pi / nr
    phn = np.arange(2 * nr) * 2 * math.pi / (2 * nr)
    phc = (np.arange(2 * nr) + 0.5) * 2 * math.pi / (2 * nr)
    rms = lambda a: float(np.sqrt(np.mean(a ** 2)))
    out = {}
    RR, TT, PP = np.meshgrid(rc, thc, phn, indexing="ij")          # phi faces
    dB = _dipole_rate(V0, cart(RR, TT, PP))
    e = ((bp2 - bp) / dt - (-dB[0] * np.sin(PP) + dB[1] * np.cos(PP))) * RR ** 3
    out["bp_all"], out["bp_pole"] = rms(e[2:-2]), rms(e[2:-2][:, [0, -1]])
    RR, TT, PP = np.meshgrid(rc, thn, phc, indexing="ij")          # theta faces
    dB = _dipole_rate(V0, cart(RR, TT, PP))
    e = ((bt2 - bt) / dt - to_sph(dB, TT, PP)[1]) * RR ** 3
    out["bt_all"], out["bt_pole"] = rms(e[2:-2, 1:-1]), rms(e[2:-2][:, [1, -2]])
    RR, TT, PP = np.meshgrid(r, thc, phc, indexing="ij")           # r faces
    dB = _dipole_rate(V0, cart(RR, TT, PP))
    e = ((br2 - br) / dt - to_sph(dB, TT, PP)[0]) * RR ** 3
    out["br_pole"] = rms(e[2:-2][:, [0, -1]])
    return out


@pytest.fixture(scope="module")
def ct_translation():
    return [_ct_translation_errors(nr) for nr in (16, 32, 64)]


def test_ct_translation_second_order_over_all_theta(ct_translation):
    # every theta row, the two polar rings included
    for key in ("bp_all", "bt_all"):
        errs = [e[key] for e in ct_translation]
        r = _rates(errs)
        assert r[-1] > 3.0 and r[-1] > r[0], (key, errs)


def test_ct_translation_converges_in_polar_rings(ct_translation):
    # the faces next to the poles: phi and theta faces at second order; the polar-cap r faces at
    # first order (their flux average of B_r's first phi harmonic, which grows like sin(theta),
    # is centred at theta ~ 2 dth / 3 rather than at the cell's dth / 2)
    for key, lo in (("bp_pole", 3.0), ("bt_pole", 3.0), ("br_pole", 1.8)):
        errs = [e[key] for e in ct_translation]
        r = _rates(errs)
        assert r[-1] > lo and errs[-1] < errs[0], (key, errs, r)


_U = np.array([0.3, -0.2, 0.5])


def _uniform_potential(x):
    # A = U x x / 2, so B = curl A = U
    return 0.5 * np.stack([_U[1] * x[2] - _U[2] * x[1], _U[2] * x[0] - _U[0] * x[2], _U[0] * x[1] - _U[1] * x[0]])


def test_bcentre_polar_pole_value_is_first_harmonic_over_cos_dtheta():
    # B_theta,c in a polar ring is the mean of the face value and the pole value. Face rings next
    # to the poles made of phi harmonics 0, 1 and 2 (random amplitudes per shell): the pole value
    # along meridian phi_k must be the harmonic-1 part divided by cos(dth), to round-off
    rng = np.random.default_rng(7)
    for nr, np_ in ((6, 8), (8, 16), (5, 12)):
        d = I.GridDesc(nr, nr, np_, 1.0, 4.0, 1.1)
        g = O.Grid.from_desc(d)
        br, bt, bp = zero_faces(d)
        phc = (np.arange(np_) + 0.5) * 2 * math.pi / np_
        c = math.cos(math.pi / nr)
        for j, jf in ((0, 1), (nr - 1, nr - 1)):
            a1, b1, a0, a2, b2 = rng.normal(size=(5, nr, 1))
            h1 = a1 * np.cos(phc) + b1 * np.sin(phc)
            bt[:, jf] = c * h1 + a0 + a2 * np.cos(2 * phc) + b2 * np.sin(2 * phc)
            bc = g.bcentre(br, bt, bp)
            pole = 2 * bc[1][:, j] - bt[:, jf]
            assert np.abs(pole - h1).max() < 1e-13, (nr, np_, j)


def _bcentre_polar_errors(nr):
    d, g = _grid(nr)
    br, bt, bp = I.magnetic_field(d, dipole=True, potential=_uniform_potential)
    R, TH, PH = centres(d)
    ex = to_sph(dipole_B(cart(R, TH, PH)) + _U.reshape(3, 1, 1, 1), TH, PH)
    e = (g.bcentre(br, bt, bp) - ex)[:, 1:-1][:, :, [0, -1]]
    return [float(np.sqrt(np.mean(e[c] ** 2))) for c in range(3)]


def test_bcentre_polar_rings_convergence():
    # dipole plus a uniform field (horizontal on the axis): B_theta and B_phi at the polar-ring
    # centres at second order; B_r at first order (the polar-cap face centroid, as above)
    errs = np.array([_bcentre_polar_errors(nr) for nr in (8, 16, 32)])
    for c, lo in ((0, 1.8), (1, 3.5), (2, 3.5)):
        r = _rates(list(errs[:, c]))
        assert r[-1] > lo, (c, errs[:, c], r)


def _polar_axis_er_error(nr):
    d, g = _grid(nr)
    br, bt, bp = I.magnetic_field(d, dipole=True, potential=_uniform_potential)
    R, TH, PH = centres(d)
    V0 = np.array([1.0, 0.5, 0.2])
    v = np.ascontiguousarray(to_sph(np.broadcast_to(V0.reshape(3, 1, 1, 1), (3,) + R.shape), TH, PH))
    er, _, _ = g.efield_edges(v, br, bt, bp)
    r = I.radial_nodes(d)
    rc = 0.5 * (r[1:] + r[:-1])
    errs = []
    for s, col in ((1.0, 0), (-1.0, -1)):       # r-hat is +z on the north axis, -z on the south
        X = np.stack([0 * rc, 0 * rc, s * rc])
        B = dipole_B(X[:, :, None, None])[:, :, 0, 0] + _U[:, None]
        Ez = -(V0[0] * B[1] - V0[1] * B[0])
        assert np.all(er[:, col, :] == er[:, col, :1])
        errs.append(er[:, col, 0] - s * Ez)
    return float(np.sqrt(np.mean(np.concatenate(errs) ** 2)))


def test_efield_polar_axis_value_second_order():
    # the polar radial edge takes the mean of E_r over the polar ring: for a uniform flow across a
    # dipole plus a uniform field it tends to E_r = -(v x B).r_hat on the axis at second order
    errs = [_polar_axis_er_error(nr) for nr in (8, 16, 32)]
    r = _rates(errs)
    assert r[-1] > 3.7 and errs[-1] < 1e-3, (errs, r)


def test_efield_outer_edges_two_cell_mean_and_polar_ring_single_valued():
    d = I.GridDesc(4, 4, 6, 1.0, 3.0, 1.0)
    g = O.Grid.from_desc(d)
    rng = np.random.default_rng(2)
    br = rng.normal(size=(5, 4, 6)); bt = rng.normal(size=(4, 5, 6)); bp = rng.normal(size=(4, 4, 6))
    bt[:, 0] = 0; bt[:, -1] = 0
    v = rng.normal(size=(3, 4, 4, 6))
    er, et, ep = g.efield_edges(v, br, bt, bp)
    assert np.all(et[0] == 0.0) and np.all(ep[0] == 0.0)
    assert np.all(er[:, 0, :] == er[:, 0, :1]) and np.all(er[:, -1, :] == er[:, -1, :1])
    # linearity in v and antisymmetry: E(-v) = -E(v)
    er2, et2, ep2 = g.efield_edges(-v, br, bt, bp)
    assert np.array_equal(er2, -er) and np.array_equal(et2, -et) and np.array_equal(ep2, -ep)


# ----------------------------------------------------------------------------- coefficients
def test_coeffs_cfl_and_scaling():
    d = I.GridDesc(8, 8, 16, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    st = I.initial_state(d, 0, False)
    v = np.stack([st["vr"], st["vt"], st["vp"]])
    c1 = g.coeffs(v, st["br"], st["bt"], st["bp"], nu=2e-3, cfl=0.3)
    assert abs(c1["cf"] - 0.3) < 1e-15
    assert c1["alpha_nu"] == 2e-3 * c1["dt"]
    c2 = g.coeffs(2 * v, st["br"], st["bt"], st["bp"], nu=2e-3, cfl=0.3)
    assert abs(c2["dt"] - 0.5 * c1["dt"]) < 1e-15 * c1["dt"]
    assert abs(c2["cw"] - 0.5 * c1["cw"]) < 1e-14 * c1["cw"]
    # S > 0 iff C_w > 1 - C_f; the SI coefficient vanishes without field
    br, bt, bp = zero_faces(d)
    c3 = g.coeffs(v, br, bt, bp, cfl=0.3)
    assert c3["cw"] == 0.0 and c3["alpha_si"] == 0.0
    assert c1["alpha_si"] > 0.0
    # frozen dt / alpha overrides
    c4 = g.coeffs(v, st["br"], st["bt"], st["bp"], dt_fixed=1e-3, asi_fixed=0.25)
    assert c4["dt"] == 1e-3 and c4["alpha_si"] == 0.25
    # dt_max clips the CFL step
    c5 = g.coeffs(v, st["br"], st["bt"], st["bp"], cfl=0.3, dt_max=0.1 * c1["dt"])
    assert c5["dt"] == 0.1 * c1["dt"] and abs(c5["cf"] - 0.03) < 1e-15


def test_coeffs_single_cell_ktilde_between_spacing_bounds():
    # with v nonzero in one cell, dt = cfl / (k~ |v|) there; k~^2 lies between 1/h_min^2 and
    # 3/h_min^2 of that cell's three spacings (radial width, r dtheta, r sin(theta) dphi)
    d = I.GridDesc(8, 8, 16, 1.0, 20.0, 1.05)
    g = O.Grid.from_desc(d)
    br, bt, bp = zero_faces(d)
    r = I.radial_nodes(d)
    for (i, j) in [(0, 0), (3, 4), (7, 7)]:
        v = np.zeros((3, 8, 8, 16))
        v[1, i, j, 5] = 0.5
        c = g.coeffs(v, br, bt, bp, cfl=0.4)
        kt = 0.4 / (c["dt"] * 0.5)
        rc = 0.5 * (r[i] + r[i + 1])
        hs = [r[i + 1] - r[i], rc * math.pi / 8, rc * math.sin((j + 0.5) * math.pi / 8) * 2 * math.pi / 16]
        hmin = min(hs)
        assert 1 / hmin ** 2 <= kt ** 2 * (1 + 1e-12) and kt ** 2 <= 3 / hmin ** 2
        assert abs(kt ** 2 - sum(1 / h ** 2 for h in hs)) < 1e-10 * kt ** 2
