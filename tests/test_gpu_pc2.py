"""GPU PC2 (Sec. 2.2 block-Jacobi ILU(0), phi-line blocks; one warp per line, affine scans)
against the oracle's og_pcg_pc2 with the same blocks and og_step_opts(OG_OPT_PC2), through the C
ABI: iteration counts within one, solutions and fields within 1e-11 where the counts agree. Grids
cover phi lengths with one, several and sixteen elements per lane and ragged last lanes."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import dev_state, fields, grid, oracle_iterate_at, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu
KEYS = ("vr", "vt", "vp", "br", "bt", "bp")
GRIDS = [I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1), I.GridDesc(9, 7, 10, 1.0, 6.0, 1.08),
         I.GridDesc(5, 6, 66, 1.0, 8.0, 1.1), I.GridDesc(6, 8, 512, 1.0, 10.0, 1.2),
         I.GridDesc(32, 32, 64, 1.0, 20.0, 1.05)]


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
@pytest.mark.parametrize("nc", [1, 3])
def test_pcg_pc2_matches_oracle(d, nc):
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(17)
    b = rng.normal(size=(nc, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    x0 = rng.normal(size=b.shape) * 0.1
    for alpha in (0.05, 4.0):
        x = to_dev(x0)
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, P.make_params(tol=1e-9, max_iter=5000, preconditioner=1))
        xr, itr, _, str_ = og.pcg(alpha, b, x0=x0, tol=1e-9, max_iter=5000, pc2="lines")
        assert st == P.MHD_OK and str_ == O.OK
        assert abs(it - itr) <= 1, (it, itr)
        assert rr <= 1e-9
        xo = oracle_iterate_at(og, alpha, b, it, itr, xr, x0=x0, pc2="lines")
        assert rel_l2(to_np(x), xo) < 1e-11, (it, itr)


def test_pcg_pc2_fixed_iteration_trajectory():
    d = GRIDS[3]
    g, og = grid(d), O.Grid.from_desc(d)
    b = np.random.default_rng(9).normal(size=(3, d.nr, d.nt, d.np))
    for k in (1, 2, 5, 12):
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        st, it, ou, rr = P.pcg_solve(g, 2.5, to_dev(b), x, P.make_params(tol=1e-30, max_iter=k, preconditioner=1))
        assert st == P.MHD_ERR_NOCONV and it == k
        xr, _, _, _ = og.pcg(2.5, b, fixed_iters=k, pc2="lines")
        assert rel_l2(to_np(x), xr) < 1e-12, k


def test_pcg_pc2_edge_cases():
    d = GRIDS[0]
    g = grid(d)
    z = torch.zeros((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    x = torch.ones_like(z)
    st, it, ou, rr = P.pcg_solve(g, 1.0, z, x, P.make_params(preconditioner=1))   # b = 0
    assert st == P.MHD_OK and it == 0 and float(x.abs().max()) == 0.0
    b = torch.ones_like(z)
    st, it, ou, rr = P.pcg_solve(g, 0.0, b, x, P.make_params(tol=1e-12, preconditioner=1))   # M = D: exact
    assert st == P.MHD_OK and it == 1
    for bad in (dict(preconditioner=1, pcg_variant=1), dict(preconditioner=2)):
        with pytest.raises(P.MhdError):
            P.pcg_solve(g, 1.0, b, x, P.make_params(**bad))


def test_step_pc2_parity_workload_10_steps():
    w, st0 = I.workload("parity_32x32x64")
    d = w["desc"]
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st0)
    f = fields(ds)
    s = st0
    prm = P.make_params(nu=w["nu"], cfl=w["cfl"], tol=w["tol"], preconditioner=1)
    for n in range(10):
        stat, info = P.mhd_step(g, prm, f)
        torch.cuda.synchronize()
        s, oinfo = og.step(s, nu=w["nu"], cfl=w["cfl"], tol=w["tol"], pc2=True)
        assert stat == P.MHD_OK and oinfo["status"] == O.OK
        for q in range(3):
            assert abs(info["iters"][q] - oinfo["iters"][q]) <= 1, (n, info["iters"], oinfo["iters"])
        for k in KEYS:
            e = rel_l2(to_np(ds[k]), s[k])
            assert e <= 1e-11, (n, k, e)


def test_adjoint_with_pc2_solves_matches_oracle():
    # the adjoint's three solves under PC2 reach the same tolerance, so the cotangent agrees with
    # the oracle's (PC1) adjoint to the solver tolerance
    d = I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1)
    st = I.initial_state(d, 0, False)
    for k in ("vr", "vt", "vp"):
        st[k] = st[k] * 20.0
    og = O.Grid.from_desc(d)
    c = og.coeffs(np.stack([st["vr"], st["vt"], st["vp"]]), st["br"], st["bt"], st["bp"], nu=1e-3, cfl=0.3)
    rng = np.random.default_rng(200)
    lam = {k: rng.normal(size=st[k].shape) for k in KEYS}
    lam["bt"][:, 0] = 0.0
    lam["bt"][:, -1] = 0.0
    ref, s1 = og.adjoint_step(st, lam, c["dt"], c["alpha_si"], cfl=0.3, tol=1e-13)
    ds, dl = dev_state(st), dev_state(lam)
    out = {k: torch.empty_like(v) for k, v in ds.items()}
    prm = P.make_params(nu=1e-3, cfl=0.3, tol=1e-13, alpha_si_fixed=c["alpha_si"], max_iter=200000, preconditioner=1)
    s2 = P.mhd_adjoint_step(grid(d), prm, fields(ds), c["dt"], fields(dl), fields(out))
    torch.cuda.synchronize()
    assert s1 == O.OK and s2 == P.MHD_OK
    for k in KEYS:
        assert rel_l2(to_np(out[k]), ref[k]) < 1e-9, k


@pytest.mark.parametrize("d", [GRIDS[1], GRIDS[3], GRIDS[4]], ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
@pytest.mark.parametrize("restart,inner", [(0, 0.1), (1, 1e-5)], ids=["reliable", "restart"])
def test_pcg_mixed_pc2_reaches_fp64_tolerance(d, restart, inner):
    # FP32 inner PCG with the FP32 phi-line preconditioner, FP64 residual replacement: the TRUE FP64
    # residual reaches tol and the solution matches the oracle's converged one
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(31)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    alpha = 4.0
    xr, _, _, _ = og.pcg(alpha, b, tol=1e-13, pc2="lines")
    for nc in (3, 1):
        x = torch.zeros((nc,) + b.shape[1:], dtype=torch.float64, device="cuda")
        prm = P.make_params(tol=1e-9, inner_tol=inner, precision=P.PREC_MIXED, max_outer=60, max_iter=5000,
                            mixed_restart=restart, preconditioner=1)
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b[:nc]), x, prm)
        assert st == P.MHD_OK and rr <= 1e-9 and ou >= 1
        res = b[:nc] - og.apply_M(alpha, to_np(x))
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(b[:nc]) * 1.0000001
        assert rel_l2(to_np(x), xr[:nc]) < 1e-6


def test_step_mixed_pc2_against_fp64_oracle():
    w, st0 = I.workload("parity_32x32x64")
    d = w["desc"]
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st0)
    f = fields(ds)
    s = st0
    prm = P.make_params(nu=w["nu"], cfl=w["cfl"], tol=w["tol"], precision=P.PREC_MIXED, inner_tol=0.1,
                        max_outer=60, max_iter=5000, preconditioner=1)
    for n in range(3):
        stat, info = P.mhd_step(g, prm, f)
        torch.cuda.synchronize()
        s, oinfo = og.step(s, nu=w["nu"], cfl=w["cfl"], tol=w["tol"], pc2=True)
        assert stat == P.MHD_OK and max(info["relres"]) <= 1e-9
        for k in KEYS:
            e = rel_l2(to_np(ds[k]), s[k])
            assert e <= 1e-7, (n, k, e)
