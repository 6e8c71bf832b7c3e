"""GPU (sm_103a) library against the FP64 CPU oracle, element by element, through the C ABI.

Tolerances: the explicit kernels and the operator evaluate the same formulas in a different
rounding order (and with fused multiply-adds), so they agree to a few ulps relative to the
largest term (1e-13 relative L2 for the operator, 1e-11 for the force, whose components are
small differences of larger terms). PCG at tol 1e-9: same iteration count within +-1 and solution
within 1e-11 relative L2 of the oracle's iterate after the same number of iterations (both follow
the same Krylov recurrence; the scaled form differs only in rounding; when the counts differ by one
the oracle is rerun for exactly the GPU's count)."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import dev_state, fields, grid, oracle_iterate_at, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

GRIDS = [
    I.GridDesc(5, 6, 8, 1.0, 3.0, 1.1),          # tiny, odd nr, several tiles of nothing: edges only
    I.GridDesc(32, 32, 64, 1.0, 20.0, 1.05),     # parity workload
    I.GridDesc(23, 17, 46, 1.0, 10.0, 1.07),     # ragged: np not a multiple of 4, odd nt
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1811_02605_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


def _state(d, index=0, rope=False):
    return I.initial_state(d, index, rope)


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_operator_matches_oracle(d):
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(1)
    for nc in (1, 3):
        p = rng.normal(size=(nc, d.nr, d.nt, d.np))
        for alpha in (0.0, 0.3, 17.0):
            q = torch.empty(p.shape, dtype=torch.float64, device="cuda")
            P.mhd_apply_operator(g, alpha, to_dev(p), q)
            torch.cuda.synchronize()
            ref = og.apply_M(alpha, p)
            assert rel_l2(to_np(q), ref) < 1e-13


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_coeffs_match_oracle(d):
    st = _state(d)
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st)
    prm = P.make_params(nu=1e-3, cfl=0.4)
    got = P.mhd_step_coeffs(g, prm, fields(ds))
    ref = og.coeffs(np.stack([st["vr"], st["vt"], st["vp"]]), st["br"], st["bt"], st["bp"], nu=1e-3, cfl=0.4)
    for k in ("dt", "cf", "cw", "alpha_si", "alpha_nu"):
        assert abs(got[k] - ref[k]) <= 1e-13 * abs(ref[k]), (k, got[k], ref[k])


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_force_matches_oracle(d):
    st = _state(d, rope=False)
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st)
    b = torch.empty((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    P.mhd_force(g, fields(ds), 0.037, b)
    torch.cuda.synchronize()
    ref = og.force(np.stack([st["vr"], st["vt"], st["vp"]]), st["br"], st["bt"], st["bp"], 0.037)
    # the phi component is a small difference of large advective and Lorentz terms; FMA
    # contraction and the order of the sums move it by a few ulps of those terms
    for c in range(3):
        assert rel_l2(to_np(b)[c], ref[c]) < 1e-11, c


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
@pytest.mark.parametrize("eta", [0.0, 2e-3])
def test_induction_matches_oracle(d, eta):
    st = _state(d)
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st)
    vbar = np.stack([st["vr"], st["vt"], st["vp"]]) * 3.0
    P.mhd_induction(g, to_dev(vbar), eta, 0.05, fields(ds))
    torch.cuda.synchronize()
    er, et, ep = og.efield_edges(vbar, st["br"], st["bt"], st["bp"], eta)
    br, bt, bp = og.ct(er, et, ep, 0.05, st["br"], st["bt"], st["bp"])
    for name, ref in (("br", br), ("bt", bt), ("bp", bp)):
        dlt_ref = ref - st[name]
        dlt = to_np(ds[name]) - st[name]
        assert rel_l2(dlt, dlt_ref) < 1e-11, name
        assert rel_l2(to_np(ds[name]), ref) < 1e-14, name
    assert np.array_equal(to_np(ds["br"])[0], st["br"][0])


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_pcg_fp64_matches_oracle(d):
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(3)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    x0 = rng.normal(size=b.shape) * 0.1
    for alpha in (0.05, 4.0):
        prm = P.make_params(tol=1e-9, max_iter=5000)
        x = to_dev(x0)
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, prm)
        xr, itr, rrr, str_ = og.pcg(alpha, b, x0=x0, tol=1e-9, max_iter=5000)
        assert st == P.MHD_OK and str_ == O.OK
        assert abs(it - itr) <= 1, (it, itr)
        assert rr <= 1e-9
        xo = oracle_iterate_at(og, alpha, b, it, itr, xr, x0=x0)
        assert rel_l2(to_np(x), xo) < 1e-11, (it, itr)


def test_pcg_fixed_iteration_trajectory():
    # max_iter caps the GPU solve; the oracle's fixed-count mode gives the same iterate
    d = GRIDS[1]
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(9)
    b = rng.normal(size=(3, d.nr, d.nt, d.np))
    for k in (1, 2, 7, 40):
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        st, it, ou, rr = P.pcg_solve(g, 2.5, to_dev(b), x, P.make_params(tol=1e-30, max_iter=k))
        assert st == P.MHD_ERR_NOCONV and it == k
        xr, itr, _, _ = og.pcg(2.5, b, fixed_iters=k)
        assert rel_l2(to_np(x), xr) < 1e-12, k


def test_pcg_edge_cases():
    d = GRIDS[0]
    g = grid(d)
    z = torch.zeros((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    x = torch.ones_like(z)
    st, it, ou, rr = P.pcg_solve(g, 1.0, z, x, P.make_params())
    assert st == P.MHD_OK and it == 0 and torch.all(x == 0)
    # alpha = 0: M = D, the Jacobi preconditioner solves it in one iteration
    b = torch.randn((2, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st, it, ou, rr = P.pcg_solve(g, 0.0, b, x, P.make_params(tol=1e-12))
    assert st == P.MHD_OK and it == 1
    # non-finite right-hand side is reported, not hung on
    b[0, 0, 0, 0] = float("nan")
    x = torch.zeros_like(b)
    st, it, ou, rr = P.pcg_solve(g, 1.0, b, x, P.make_params())
    assert st == P.MHD_ERR_NONFINITE
    with pytest.raises(P.MhdError):
        P.pcg_solve(g, -1.0, z, x, P.make_params())


@pytest.mark.parametrize("d", GRIDS[:2], ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_pcg_mixed_reaches_fp64_tolerance(d):
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(4)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    alpha = 4.0
    xr, itr, _, _ = og.pcg(alpha, b, tol=1e-13)
    x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
    prm = P.make_params(tol=1e-9, inner_tol=1e-5, precision=P.PREC_MIXED, max_outer=20)
    st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, prm)
    assert st == P.MHD_OK and rr <= 1e-9 and ou >= 1
    # true residual in FP64
    res = b - og.apply_M(alpha, to_np(x))
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(b) * 1.0000001
    assert rel_l2(to_np(x), xr) < 1e-6


def _run_steps(d, st0, nsteps, prm_kw, index=0):
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st0)
    f = fields(ds)
    s = st0
    out = []
    for n in range(nsteps):
        stat, info = P.mhd_step(g, P.make_params(**prm_kw), f)
        torch.cuda.synchronize()
        s, oinfo = og.step(s, **{k: v for k, v in prm_kw.items() if k in ("nu", "eta", "cfl", "dt_fixed", "tol")})
        out.append((stat, info, oinfo, {k: to_np(v) for k, v in ds.items()}, s))
    return out


def test_step_fp64_parity_workload_10_steps():
    w, st0 = I.workload("parity_32x32x64")
    res = _run_steps(w["desc"], st0, 10, dict(nu=w["nu"], cfl=w["cfl"], tol=w["tol"]))
    for n, (stat, info, oinfo, gpu, ref) in enumerate(res):
        assert stat == P.MHD_OK and oinfo["status"] == O.OK
        assert abs(info["dt"] - oinfo["dt"]) <= 1e-12 * oinfo["dt"]
        for q in range(3):
            assert abs(info["iters"][q] - oinfo["iters"][q]) <= 1, (n, info["iters"], oinfo["iters"])
        for k in ("vr", "vt", "vp", "br", "bt", "bp"):
            e = rel_l2(gpu[k], ref[k])
            assert e <= 1e-11, (n, k, e)


def test_step_fp64_ragged_grid_with_resistivity():
    d = I.GridDesc(9, 7, 10, 1.0, 6.0, 1.08)
    st0 = I.initial_state(d, 2, False)
    res = _run_steps(d, st0, 3, dict(nu=5e-3, eta=1e-3, cfl=0.3, tol=1e-10))
    for n, (stat, info, oinfo, gpu, ref) in enumerate(res):
        assert stat == P.MHD_OK
        for k in ("vr", "vt", "vp", "br", "bt", "bp"):
            assert rel_l2(gpu[k], ref[k]) <= 1e-11, (n, k)


def test_step_mixed_against_fp64_oracle():
    w, st0 = I.workload("parity_32x32x64")
    res = _run_steps(w["desc"], st0, 3, dict(nu=w["nu"], cfl=w["cfl"], tol=w["tol"], precision=P.PREC_MIXED,
                                              inner_tol=1e-5, max_outer=30))
    for n, (stat, info, oinfo, gpu, ref) in enumerate(res):
        assert stat == P.MHD_OK
        assert max(info["relres"]) <= 1e-9
        for k in ("vr", "vt", "vp", "br", "bt", "bp"):
            assert rel_l2(gpu[k], ref[k]) <= 1e-7, (n, k, rel_l2(gpu[k], ref[k]))


@pytest.mark.parametrize("restart,inner", [(0, 0.1), (1, 1e-5), (0, 1e-5)], ids=["reliable", "restart", "reliable-small"])
def test_pcg_mixed_tiled_path(restart, inner):
    # np = 256 takes the plane-marching FP32 kernels; nt = 18 leaves a ragged last row tile
    d = I.GridDesc(20, 18, 256, 1.0, 10.0, 1.05)
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(12)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    alpha = 2.0
    xr, _, _, _ = og.pcg(alpha, b, tol=1e-13)
    x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
    prm = P.make_params(tol=1e-9, inner_tol=inner, precision=P.PREC_MIXED, max_outer=60, max_iter=5000,
                        mixed_restart=restart)
    st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, prm)
    assert st == P.MHD_OK and rr <= 1e-9
    res = b - og.apply_M(alpha, to_np(x))
    assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(b) * 1.0000001
    assert rel_l2(to_np(x), xr) < 1e-6
    # one and two components too
    for nc in (1, 2):
        x = torch.zeros((nc,) + b.shape[1:], dtype=torch.float64, device="cuda")
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b[:nc]), x, prm)
        assert st == P.MHD_OK and rr <= 1e-9
        xr1, _, _, _ = og.pcg(alpha, b[:nc], tol=1e-13)
        assert rel_l2(to_np(x), xr1) < 1e-6


def test_step_mixed_tiled_against_fp64_oracle():
    d = I.GridDesc(16, 16, 128, 1.0, 10.0, 1.05)
    st0 = I.initial_state(d, 4, False)
    res = _run_steps(d, st0, 2, dict(nu=1e-3, cfl=0.4, tol=1e-9, precision=P.PREC_MIXED, inner_tol=0.1,
                                     max_outer=60, max_iter=5000))
    for n, (stat, info, oinfo, gpu, ref) in enumerate(res):
        assert stat == P.MHD_OK and max(info["relres"]) <= 1e-9
        for k in ("vr", "vt", "vp", "br", "bt", "bp"):
            assert rel_l2(gpu[k], ref[k]) <= 1e-7, (n, k, rel_l2(gpu[k], ref[k]))


def test_pcg_fp64_tiled_path_matches_oracle():
    # np = 256: the FP64 solve may use the fused p-update + stencil kernel (autotuned per grid)
    d = I.GridDesc(20, 18, 256, 1.0, 10.0, 1.05)
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(21)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    x0 = rng.normal(size=b.shape) * 0.01
    for alpha in (0.3, 6.0):
        x = to_dev(x0)
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, P.make_params(tol=1e-9, max_iter=5000))
        xr, itr, _, s2 = og.pcg(alpha, b, x0=x0, tol=1e-9, max_iter=5000)
        assert st == P.MHD_OK and abs(it - itr) <= 1, (it, itr)
        xo = oracle_iterate_at(og, alpha, b, it, itr, xr, x0=x0)
        assert rel_l2(to_np(x), xo) < 1e-11, (it, itr)
    for k in (1, 3, 11):
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        st, it, ou, rr = P.pcg_solve(g, 2.0, to_dev(b), x, P.make_params(tol=1e-30, max_iter=k))
        xr, _, _, _ = og.pcg(2.0, b, fixed_iters=k)
        assert it == k and rel_l2(to_np(x), xr) < 1e-12, k


def test_step_fp64_tiled_grid_parity():
    d = I.GridDesc(16, 16, 128, 1.0, 10.0, 1.05)
    st0 = I.initial_state(d, 6, False)
    res = _run_steps(d, st0, 3, dict(nu=1e-3, cfl=0.4, tol=1e-9))
    for n, (stat, info, oinfo, gpu, ref) in enumerate(res):
        assert stat == P.MHD_OK
        for q in range(3):
            assert abs(info["iters"][q] - oinfo["iters"][q]) <= 1
        for k in ("vr", "vt", "vp", "br", "bt", "bp"):
            assert rel_l2(gpu[k], ref[k]) <= 1e-11, (n, k, rel_l2(gpu[k], ref[k]))


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_diagnostics_match_oracle(d):
    st = _state(d, rope=False)
    for k in ("vr", "vt", "vp"):
        st[k] = st[k] * 5.0
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st)
    got = P.mhd_diagnostics(g, fields(ds))
    ref = og.diagnostics(st)
    for k in ("magnetic_energy", "kinetic_energy", "int_jxb", "int_jdotb"):
        assert abs(got[k] - ref[k]) <= 1e-12 * abs(ref[k]), (k, got[k], ref[k])
    scale = float(np.abs(st["br"]).max()) * d.nr
    assert got["max_divb"] <= 1e-12 * scale and ref["max_divb"] <= 1e-12 * scale
    # after steps of the GPU path the constrained transport keeps div_h B at round-off
    for _ in range(3):
        P.mhd_step(g, P.make_params(nu=1e-3, cfl=0.4, eta=2e-3), fields(ds))
    after = P.mhd_diagnostics(g, fields(ds))
    assert after["max_divb"] <= 1e-11 * scale, after["max_divb"]
    assert abs(after["magnetic_energy"] - got["magnetic_energy"]) < 0.1 * got["magnetic_energy"]
