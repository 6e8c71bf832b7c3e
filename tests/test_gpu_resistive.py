"""GPU implicit resistivity (Eq. 1 curl-curl term by PCG with PC1, Sec. 2.2) against the oracle's
og_step_opts(OG_OPT_RES_IMPLICIT), through the C ABI: fields within 1e-11 rel-L2 per step and
iteration counts within one, div B and the wall fluxes kept."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import dev_state, fields, grid, rel_l2, to_np

pytestmark = pytest.mark.gpu
KEYS = ("vr", "vt", "vp", "br", "bt", "bp")
GRIDS = [I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1), I.GridDesc(9, 7, 10, 1.0, 6.0, 1.08),
         I.GridDesc(32, 32, 64, 1.0, 20.0, 1.05)]


# (eta, tol, iteration slack). At eta = 5e-3 the workload tolerance 1e-9 already resolves the
# 1e-11 gate. At eta = 0.05 the face system is ill conditioned (about 250 iterations on 32x32x64):
# two solutions that each meet tol 1e-9 or even 1e-12 differ by up to 2e-10 in the small B_phi
# (measured on the oracle alone, tol 1e-12 against 1e-14), so the gate is applied with every solve
# at tol 3e-14, where the counts near the rounding floor may differ by a few.
CASES = [(5e-3, 1e-9, 1), (0.05, 3e-14, 8)]


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
@pytest.mark.parametrize("eta,tol,slack", CASES, ids=["eta5e-3", "eta5e-2"])
def test_implicit_resistivity_step_parity(d, eta, tol, slack):
    st0 = I.initial_state(d, 2, False)
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st0)
    f = fields(ds)
    s = st0
    prm = P.make_params(nu=1e-3, eta=eta, cfl=0.4, tol=tol, max_iter=100000, resistivity_implicit=1)
    div0 = og.divb(st0["br"], st0["bt"], st0["bp"])
    for n in range(3):
        stat, info = P.mhd_step(g, prm, f)
        torch.cuda.synchronize()
        s, oinfo = og.step(s, nu=1e-3, eta=eta, cfl=0.4, tol=tol, max_iter=100000, res_implicit=True)
        assert stat == P.MHD_OK and oinfo["status"] == O.OK
        assert abs(info["iters_res"] - oinfo["res_iters"]) <= slack, (info["iters_res"], oinfo["res_iters"])
        assert info["iters_res"] >= 1 and info["relres_res"] <= tol
        for q in range(3):
            assert abs(info["iters"][q] - oinfo["iters"][q]) <= slack
        for k in KEYS:
            e = rel_l2(to_np(ds[k]), s[k])
            assert e <= 1e-11, (n, k, e)
    got = {k: to_np(v) for k, v in ds.items()}
    assert np.abs(og.divb(got["br"], got["bt"], got["bp"]) - div0).max() <= 1e-12 * np.abs(st0["br"]).max()
    assert np.array_equal(got["br"][0], st0["br"][0])


def test_implicit_resistivity_zero_eta_is_the_ideal_step():
    d = GRIDS[2]
    st0 = I.initial_state(d, 1, False)
    g = grid(d)
    a, b = dev_state(st0), dev_state(st0)
    s1, i1 = P.mhd_step(g, P.make_params(eta=0.0, tol=1e-12, resistivity_implicit=1), fields(a))
    s2, i2 = P.mhd_step(g, P.make_params(eta=0.0, tol=1e-12), fields(b))
    assert s1 == P.MHD_OK and s2 == P.MHD_OK and i1["iters_res"] == 0
    for k in KEYS:
        assert rel_l2(to_np(a[k]), to_np(b[k])) <= 1e-13, k


def test_implicit_resistivity_bad_flag_rejected():
    d = GRIDS[0]
    g = grid(d)
    st = dev_state(I.initial_state(d, 0, False))
    with pytest.raises(P.MhdError):
        P.mhd_step(g, P.make_params(resistivity_implicit=2), fields(st))


@pytest.mark.parametrize("d", [GRIDS[0], GRIDS[1]], ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_adjoint_with_implicit_resistivity_matches_oracle(d):
    st = I.initial_state(d, 1, False)
    for k in ("vr", "vt", "vp"):
        st[k] = st[k] * 20.0
    og = O.Grid.from_desc(d)
    eta = 0.05
    c = og.coeffs(np.stack([st["vr"], st["vt"], st["vp"]]), st["br"], st["bt"], st["bp"], nu=1e-3, cfl=0.3)
    rng = np.random.default_rng(301)
    lam = {k: rng.normal(size=st[k].shape) for k in KEYS}
    lam["bt"][:, 0] = 0.0
    lam["bt"][:, -1] = 0.0
    ref, s1 = og.adjoint_step(st, lam, c["dt"], c["alpha_si"], eta=eta, cfl=0.3, tol=1e-13, res_implicit=True)
    ds, dl = dev_state(st), dev_state(lam)
    out = {k: torch.empty_like(v) for k, v in ds.items()}
    prm = P.make_params(nu=1e-3, eta=eta, cfl=0.3, tol=1e-13, alpha_si_fixed=c["alpha_si"], max_iter=200000,
                        resistivity_implicit=1)
    s2 = P.mhd_adjoint_step(grid(d), prm, fields(ds), c["dt"], fields(dl), fields(out))
    torch.cuda.synchronize()
    assert s1 == O.OK and s2 == P.MHD_OK
    for k in KEYS:
        e = rel_l2(to_np(out[k]), ref[k])
        assert e < 1e-9, (k, e)
