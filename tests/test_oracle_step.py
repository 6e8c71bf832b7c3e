"""Pins of the oracle's full predictor-corrector step (Sec. 2.2). Agreement with the paper's own
code (MAS) cannot be checked: its code and inputs are not public (parity unpinned there). These
tests pin invariants and the composition: zero state, divergence and line-tying invariants,
second-order time self-convergence without viscosity, and the viscous solve acting alone."""
import numpy as np

import oracle as O
from paper_1811_02605_gb300 import inputs as I
from tests.helpers import exact_volumes, zero_faces


def _small(nr=6, nt=6, np_=12, s=1.1, r1=4.0, index=0):
    d = I.GridDesc(nr, nt, np_, 1.0, r1, s)
    return d, O.Grid.from_desc(d), I.initial_state(d, index, False)


def test_zero_state_stays_zero():
    d, g, _ = _small()
    br, bt, bp = zero_faces(d)
    z = np.zeros((d.nr, d.nt, d.np))
    st = dict(br=br, bt=bt, bp=bp, vr=z, vt=z, vp=z)
    out, info = g.step(st, dt_fixed=0.1)
    assert info["status"] == O.OK
    for k in out:
        assert np.all(out[k] == 0.0)
    assert info["iters"] == [0, 0, 0]


def test_divergence_and_inner_flux_invariant_over_steps():
    d, g, st = _small(8, 8, 16, 1.05, 20.0)
    div0 = g.divb(st["br"], st["bt"], st["bp"])
    s = st
    for _ in range(3):
        s, info = g.step(s, tol=1e-10)
        assert info["status"] == O.OK
    div1 = g.divb(s["br"], s["bt"], s["bp"])
    r = I.radial_nodes(d)
    scale = np.abs(s["br"]).max() * r[-1] ** 2
    assert np.abs(div1 - div0).max() <= 1e-13 * scale
    assert np.array_equal(s["br"][0], st["br"][0])
    assert np.all(s["bt"][:, 0] == 0.0) and np.all(s["bt"][:, -1] == 0.0)


def _run(g, st, dt, n, asi=None):
    s = st
    for _ in range(n):
        s, info = g.step(s, nu=0.0, dt_fixed=dt, tol=1e-14, max_iter=20000)
        assert info["status"] == O.OK
    return s


def test_time_self_convergence_second_order_without_viscosity():
    d, g, st = _small(6, 6, 12, 1.1, 4.0, index=3)
    # stronger flow so the nonlinear terms matter over the interval
    for k in ("vr", "vt", "vp"):
        st[k] = st[k] * 10.0
    T = 0.2
    sols = [_run(g, st, T / n, n) for n in (4, 8, 16)]
    def diff(a, b):
        return np.sqrt(sum(np.sum((a[k] - b[k]) ** 2) for k in ("vr", "vt", "vp", "br", "bt", "bp")))
    e1, e2 = diff(sols[0], sols[1]), diff(sols[1], sols[2])
    assert e1 > 0 and 3.0 < e1 / e2 < 5.0, (e1, e2)


def test_viscous_solve_alone():
    # B = 0 and v = 0 except a smooth field: F = -(v.grad)v only. With the same state, the
    # step's viscous stage is M_nu v^{n+1} = rho V v**: checking it through alpha_nu scaling,
    # a larger nu must damp the kinetic energy more.
    d, g, st = _small(8, 8, 16, 1.05, 20.0, index=2)
    br, bt, bp = zero_faces(d)
    st = dict(st, br=br, bt=bt, bp=bp)
    V = exact_volumes(d)[:, :, None]
    def ke(s):
        return float(np.sum(V * (s["vr"] ** 2 + s["vt"] ** 2 + s["vp"] ** 2)))
    out0, i0 = g.step(st, nu=0.0, dt_fixed=0.05, tol=1e-12)
    out1, i1 = g.step(st, nu=1e-2, dt_fixed=0.05, tol=1e-12)
    out2, i2 = g.step(st, nu=1e-1, dt_fixed=0.05, tol=1e-12)
    # M_0 = D and the warm start x0 = v** is already its solution: zero iterations
    assert i0["alpha_si"] == 0.0 and i0["iters"][2] == 0
    assert ke(out2) < ke(out1) < ke(out0)
    # without viscosity and field the step is the explicit predictor-corrector alone
    for k in ("br", "bt", "bp"):
        assert np.all(out0[k] == 0.0)


def test_step_with_single_reduction_pcg_agrees_within_solver_tolerance():
    # the two PCG forms share their iterates up to rounding, so a step differs by O(tol) at most
    d = I.GridDesc(8, 8, 16, 1.0, 10.0, 1.05)
    st = I.initial_state(d, 0, False)
    g = O.Grid.from_desc(d)
    a, ia = g.step(st, tol=1e-10)
    b, ib = g.step(st, tol=1e-10, cg=True)
    assert ia["status"] == O.OK and ib["status"] == O.OK
    for q in range(3):
        assert abs(ia["iters"][q] - ib["iters"][q]) <= 1
    for k in ("vr", "vt", "vp", "br", "bt", "bp"):
        assert np.linalg.norm(a[k] - b[k]) <= 1e-8 * np.linalg.norm(a[k]), k


def test_openmp_timing_build_matches_plain_build():
    # the benchmark times the oracle built with -fopenmp on all host cores; it must compute the
    # same step as the plain build (dot products in fixed chunks: agreement to rounding)
    w, st = I.workload("parity_32x32x64")
    d = w["desc"]
    n = O.set_threads(4)
    assert n == 4
    a, ia = O.Grid.from_desc(d).step(st, nu=w["nu"], cfl=w["cfl"], tol=w["tol"])
    b, ib = O.Grid.from_desc(d, omp=True).step(st, nu=w["nu"], cfl=w["cfl"], tol=w["tol"])
    assert ia["iters"] == ib["iters"] and ia["dt"] == ib["dt"]
    for k in a:
        assert np.linalg.norm(a[k] - b[k]) <= 1e-12 * np.linalg.norm(a[k]), k
    assert O.set_threads(0, omp=False) == 1
