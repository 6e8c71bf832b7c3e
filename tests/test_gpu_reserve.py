"""mhd_grid_reserve and pcg_batch_reserve: after them, the calls of the reserved features make no
device allocation. Checked through the device's free memory (cudaMemGetInfo) before and after
steps of every form, an adjoint step and a batched solve, with every torch tensor of the test
allocated beforehand. A control shows that an unreserved grid's first adjoint step does allocate
(its workspace is about 26 N doubles), so the check can see an allocation."""
import numpy as np
import pytest
import torch

import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import dev_state, fields, grid, to_dev

pytestmark = pytest.mark.gpu
KEYS = ("vr", "vt", "vp", "br", "bt", "bp")


def _free():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_reserved_grid_allocates_nothing_later():
    d = I.GridDesc(24, 20, 128, 1.0, 10.0, 1.05)
    st = I.initial_state(d, 1, False)
    g = grid(d)
    P.mhd_grid_reserve(g, P.RESERVE_ALL)
    forms = [dict(), dict(precision=P.PREC_MIXED, inner_tol=0.1, max_outer=60), dict(pcg_variant=1),
             dict(preconditioner=1), dict(preconditioner=1, precision=P.PREC_MIXED, inner_tol=1e-3, max_outer=60),
             dict(resistivity_implicit=1, eta=2e-3), dict(viscosity_sts=1)]
    states = [dev_state(st) for _ in forms]
    lam = {k: to_dev(np.random.default_rng(3).normal(size=v.shape)) for k, v in st.items()}
    lam["bt"][:, 0] = 0.0
    lam["bt"][:, -1] = 0.0
    adj_in, adj_out = dev_state(st), {k: torch.empty_like(v) for k, v in lam.items()}
    torch.cuda.synchronize()
    f0 = _free()
    infos = []
    for kw, ds in zip(forms, states):
        for _ in range(2):
            s, info = P.mhd_step(g, P.make_params(nu=1e-3, cfl=0.4, tol=1e-9, max_iter=20000, **kw), fields(ds))
            assert s == P.MHD_OK, (kw, P.mhd_last_error(g))
            infos.append(info)
    prm = P.make_params(nu=1e-3, cfl=0.4, tol=1e-12, max_iter=200000, alpha_si_fixed=infos[0]["alpha_si"])
    assert P.mhd_adjoint_step(g, prm, fields(adj_in), infos[0]["dt"], fields(lam), fields(adj_out)) == P.MHD_OK
    f1 = _free()
    assert f1 == f0, (f0 - f1)


def test_unreserved_adjoint_step_allocates():
    d = I.GridDesc(24, 20, 128, 1.0, 10.0, 1.05)
    st = I.initial_state(d, 1, False)
    g = grid(d)
    ds = dev_state(st)
    lam = {k: torch.zeros_like(v) for k, v in ds.items()}
    out = {k: torch.empty_like(v) for k, v in ds.items()}
    s, info = P.mhd_step(g, P.make_params(nu=1e-3, cfl=0.4), fields(dev_state(st)))
    f0 = _free()
    prm = P.make_params(nu=1e-3, cfl=0.4, tol=1e-12, alpha_si_fixed=info["alpha_si"])
    assert P.mhd_adjoint_step(g, prm, fields(ds), info["dt"], fields(lam), fields(out)) == P.MHD_OK
    f1 = _free()
    assert f0 - f1 >= 8 * 20 * d.nr * d.nt * d.np, (f0 - f1)


def test_reserved_batch_allocates_nothing_later():
    items = I.batched_items(64)[:5]
    grids, bs, xs, alphas = [], [], [], []
    for it in items:
        d = it["desc"]
        g = grid(d)
        grids.append(g)
        b = I.smooth_field(d, it["modes"])
        bs.append(to_dev(b))
        xs.append(torch.zeros_like(bs[-1]))
        alphas.append(1.0)
    prm = P.make_params(tol=1e-9, max_iter=20000)
    P.pcg_batch_reserve(grids, alphas, bs, xs, prm)
    assert all(float(x.abs().max()) == 0.0 for x in xs)   # nothing solved
    f0 = _free()
    for _ in range(2):
        st, it, rr = P.pcg_solve_batched(grids, alphas, bs, xs, prm)
        assert st == P.MHD_OK and max(rr) <= 1e-9
    f1 = _free()
    assert f1 == f0, (f0 - f1)
