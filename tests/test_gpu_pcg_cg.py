"""GPU single-reduction (Chronopoulos-Gear) Jacobi PCG against the oracle's og_pcg_cg and
og_step_cg, through the C ABI: iteration counts within one, solutions and fields within 1e-11
rel-L2 of the oracle's iterate after the GPU's own iteration count (the same gates as the Hestenes-Stiefel form)."""
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
         I.GridDesc(32, 32, 64, 1.0, 20.0, 1.05)]


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
@pytest.mark.parametrize("nc", [1, 3])
def test_pcg_cg_matches_oracle(d, nc):
    g, og = grid(d), O.Grid.from_desc(d)
    rng = np.random.default_rng(13)
    b = rng.normal(size=(nc, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    x0 = rng.normal(size=b.shape) * 0.1
    for alpha in (0.05, 4.0):
        x = to_dev(x0)
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, P.make_params(tol=1e-9, max_iter=5000, pcg_variant=1))
        xr, itr, _, str_ = og.pcg(alpha, b, x0=x0, tol=1e-9, max_iter=5000, cg=True)
        assert st == P.MHD_OK and str_ == O.OK
        assert abs(it - itr) <= 1, (it, itr)
        assert rr <= 1e-9
        xo = oracle_iterate_at(og, alpha, b, it, itr, xr, x0=x0, cg=True)
        assert rel_l2(to_np(x), xo) < 1e-11, (it, itr)


def test_pcg_cg_fixed_iteration_trajectory():
    d = GRIDS[1]
    g, og = grid(d), O.Grid.from_desc(d)
    b = np.random.default_rng(9).normal(size=(3, d.nr, d.nt, d.np))
    for k in (1, 2, 7, 40):
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        st, it, ou, rr = P.pcg_solve(g, 2.5, to_dev(b), x, P.make_params(tol=1e-30, max_iter=k, pcg_variant=1))
        assert st == P.MHD_ERR_NOCONV and it == k
        xr, _, _, _ = og.pcg(2.5, b, fixed_iters=k, cg=True)
        assert rel_l2(to_np(x), xr) < 1e-12, k


def test_pcg_cg_edge_cases():
    d = GRIDS[0]
    g = grid(d)
    prm = P.make_params(pcg_variant=1)
    z = torch.zeros((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
    x = torch.ones_like(z)
    st, it, ou, rr = P.pcg_solve(g, 1.0, z, x, prm)          # b = 0: x = 0, no iteration
    assert st == P.MHD_OK and it == 0 and float(x.abs().max()) == 0.0
    b = torch.ones_like(z)
    st, it, ou, rr = P.pcg_solve(g, 0.0, b, x, P.make_params(tol=1e-12, pcg_variant=1))   # M = D
    assert st == P.MHD_OK and it == 1
    with pytest.raises(P.MhdError):
        P.pcg_solve(g, 1.0, b, x, P.make_params(pcg_variant=1, precision=P.PREC_MIXED))
    with pytest.raises(P.MhdError):
        P.pcg_solve(g, 1.0, b, x, P.make_params(pcg_variant=2))


def test_step_cg_parity_workload_10_steps():
    w, st0 = I.workload("parity_32x32x64")
    d = w["desc"]
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st0)
    f = fields(ds)
    s = st0
    prm = P.make_params(nu=w["nu"], cfl=w["cfl"], tol=w["tol"], pcg_variant=1)
    for n in range(10):
        stat, info = P.mhd_step(g, prm, f)
        torch.cuda.synchronize()
        s, oinfo = og.step(s, nu=w["nu"], cfl=w["cfl"], tol=w["tol"], cg=True)
        assert stat == P.MHD_OK and oinfo["status"] == O.OK
        for q in range(3):
            assert abs(info["iters"][q] - oinfo["iters"][q]) <= 1, (n, info["iters"], oinfo["iters"])
        for k in KEYS:
            e = rel_l2(to_np(ds[k]), s[k])
            assert e <= 1e-11, (n, k, e)
