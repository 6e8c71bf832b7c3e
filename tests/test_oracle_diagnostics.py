"""Pins of the oracle's field diagnostics (Sec. 3.1 validates runs by the integrated energies and by
|J x B| and |J . B|) against integrals of analytic fields over the shell, at second order."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I
from tests.helpers import cart, centres, to_sph

R0, R1 = 1.0, 3.0
C_Z = 0.7


def _grid(nr):
    d = I.GridDesc(nr, nr, 2 * nr, R0, R1, 1.0)
    return d, O.Grid.from_desc(d)


def _rot_plus_z(x):
    # A = (0, 0, -(x^2 + y^2)/2) + c (-y/2, x/2, 0): B = (-y, x, c), J = (0, 0, 2)
    return np.stack([-C_Z * x[1] / 2, C_Z * x[0] / 2, -(x[0] ** 2 + x[1] ** 2) / 2])


def _zero_v(d):
    return {k: np.zeros((d.nr, d.nt, d.np)) for k in ("vr", "vt", "vp")}


def _rates(e):
    return [e[i] / e[i + 1] for i in range(len(e) - 1)]


def test_magnetic_energy_second_order_current_integrals_first_order():
    # B = (-y, x, c): |B|^2 = x^2 + y^2 + c^2, J x B = (-2x, -2y, 0), J . B = 2c. The energy converges
    # at second order. The current integrals converge at first order: in the first and last shells
    # the zero-gradient ghost of tangential B beyond r0 and r1 (reading R4) leaves J off by O(1) for
    # a field that varies in r, on a volume fraction O(h) (interior J converges at second order,
    # pinned in test_oracle_fields)
    vol = 4 * math.pi / 3 * (R1 ** 3 - R0 ** 3)
    int_rho2 = (R1 ** 5 - R0 ** 5) / 5 * (4 / 3) * 2 * math.pi          # int (x^2 + y^2) dV
    int_rho = (R1 ** 4 - R0 ** 4) / 4 * (math.pi / 2) * 2 * math.pi     # int sqrt(x^2 + y^2) dV
    ex = dict(magnetic_energy=0.5 * (int_rho2 + C_Z ** 2 * vol), int_jxb=2 * int_rho, int_jdotb=2 * C_Z * vol)
    errs = {k: [] for k in ex}
    for nr in (8, 16, 32):
        d, g = _grid(nr)
        br, bt, bp = I.magnetic_field(d, dipole=False, potential=_rot_plus_z)
        st = dict(br=br, bt=bt, bp=bp, **_zero_v(d))
        dg = g.diagnostics(st)
        for k in ex:
            errs[k].append(abs(dg[k] - ex[k]) / ex[k])
        assert dg["kinetic_energy"] == 0.0
    for k, lo in (("magnetic_energy", 3.5), ("int_jxb", 1.8), ("int_jdotb", 1.8)):
        r = _rates(errs[k])
        assert r[-1] > lo and r[-1] < 2 * lo + 0.5 and errs[k][-1] < 2e-2, (k, errs[k], r)


def test_kinetic_energy_of_rigid_rotation_second_order():
    # v = z x x = (-y, x, 0), rho = (r0/r)^2: 1/2 int rho |v|^2 dV = 1/2 r0^2 int sin^2 dV
    ex = 0.5 * R0 ** 2 * (R1 ** 3 - R0 ** 3) / 3 * (4 / 3) * 2 * math.pi
    errs = []
    for nr in (8, 16, 32):
        d, g = _grid(nr)
        R, TH, PH = centres(d)
        X = cart(R, TH, PH)
        v = to_sph(np.stack([-X[1], X[0], 0 * R]), TH, PH)
        br, bt, bp = I.magnetic_field(d, dipole=False, potential=lambda x: 0 * x)
        dg = g.diagnostics(dict(br=br, bt=bt, bp=bp, vr=v[0], vt=v[1], vp=v[2]))
        errs.append(abs(dg["kinetic_energy"] - ex) / ex)
        assert dg["magnetic_energy"] == 0.0 and dg["int_jxb"] == 0.0
    r = _rates(errs)
    assert r[-1] > 3.5, (errs, r)


def test_divergence_free_fields_and_potential_field_current():
    # every piece of the inputs is a vector potential: div_h B = 0 to round-off; the dipole is a
    # potential field, so int |J x B| vanishes under refinement (at first order: the boundary shells'
    # ghost rule, as above)
    errs = []
    for nr in (8, 16, 32):
        d, g = _grid(nr)
        br, bt, bp = I.magnetic_field(d, dipole=True)
        dg = g.diagnostics(dict(br=br, bt=bt, bp=bp, **_zero_v(d)))
        bmax = max(np.abs(br).max(), np.abs(bp).max())
        assert dg["max_divb"] <= 1e-12 * bmax * nr, (nr, dg["max_divb"])
        errs.append(dg["int_jxb"] / math.sqrt(dg["magnetic_energy"]))
    r = _rates(errs)
    assert r[-1] > 1.8 and errs[-1] < errs[0] / 3, (errs, r)
    # a planted monopole flux shows up in max |div B|
    d, g = _grid(8)
    br, bt, bp = I.magnetic_field(d, dipole=True)
    br[3, 2, 5] += 1e-3
    assert g.diagnostics(dict(br=br, bt=bt, bp=bp, **_zero_v(d)))["max_divb"] > 1e-4
