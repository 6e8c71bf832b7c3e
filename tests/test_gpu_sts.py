"""GPU viscosity by RKL2 super time-stepping (Sec. 2.2 STS option, algorithm 3) against the
oracle's og_step_sts / adjoint, through the C ABI: same stage count, fields within 1e-11 rel-L2
per step; the adjoint within 1e-9 (as for the PCG adjoint)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import dev_state, fields, grid, rel_l2, to_np

pytestmark = pytest.mark.gpu
KEYS = ("vr", "vt", "vp", "br", "bt", "bp")


def _run(d, st0, nsteps, nu, eta=0.0, cfl=0.4, tol=1e-9):
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st0)
    f = fields(ds)
    s = st0
    prm = P.make_params(nu=nu, eta=eta, cfl=cfl, tol=tol, viscosity_sts=1)
    out = []
    for n in range(nsteps):
        stat, info = P.mhd_step(g, prm, f)
        torch.cuda.synchronize()
        s, oinfo = og.step_sts(s, nu=nu, eta=eta, cfl=cfl, tol=tol)
        out.append((stat, info, oinfo, {k: to_np(v) for k, v in ds.items()}, s))
    return out


def _check(res, min_stages):
    for n, (stat, info, oinfo, gpu, ref) in enumerate(res):
        assert stat == P.MHD_OK and oinfo["status"] == O.OK
        assert abs(info["dt"] - oinfo["dt"]) <= 1e-12 * oinfo["dt"]
        assert info["iters"][2] == oinfo["iters"][2] >= min_stages, (info["iters"], oinfo["iters"])
        for q in range(2):
            assert abs(info["iters"][q] - oinfo["iters"][q]) <= 1, (n, info["iters"], oinfo["iters"])
        for k in KEYS:
            e = rel_l2(gpu[k], ref[k])
            assert e <= 1e-11, (n, k, e)


def test_sts_step_parity_workload_grid():
    # the 32x32x64 parity grid at its own viscosity (a few stages) and at 100x (tens of stages)
    w, st0 = I.workload("parity_32x32x64")
    _check(_run(w["desc"], st0, 3, w["nu"]), 2)
    _check(_run(w["desc"], st0, 3, 100 * w["nu"]), 20)


@pytest.mark.parametrize("d,eta", [(I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1), 0.0),
                                   (I.GridDesc(9, 7, 10, 1.0, 6.0, 1.08), 2e-3)],
                         ids=["6x6x12", "9x7x10-eta"])
def test_sts_step_parity_small_and_ragged(d, eta):
    st0 = I.initial_state(d, 4, False)
    _check(_run(d, st0, 3, 0.5, eta=eta), 2)


def test_sts_at_zero_viscosity_equals_pcg_step():
    # nu = 0: L = 0, every stage returns v** exactly; the PCG viscous solve of D v = D v** gives
    # v** to its tolerance
    w, st0 = I.workload("parity_32x32x64")
    d = w["desc"]
    g = grid(d)
    a, b = dev_state(st0), dev_state(st0)
    s1, i1 = P.mhd_step(g, P.make_params(nu=0.0, cfl=0.4, tol=1e-12, viscosity_sts=1), fields(a))
    s2, i2 = P.mhd_step(g, P.make_params(nu=0.0, cfl=0.4, tol=1e-12), fields(b))
    assert s1 == P.MHD_OK and s2 == P.MHD_OK and i1["iters"][2] == 2
    for k in KEYS:
        assert rel_l2(to_np(a[k]), to_np(b[k])) <= 1e-12, k


def test_sts_rejects_bad_flag():
    d = I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1)
    g = grid(d)
    ds = dev_state(I.initial_state(d, 0, False))
    with pytest.raises(P.MhdError):
        P.mhd_step(g, P.make_params(viscosity_sts=2), fields(ds))


@pytest.mark.parametrize("d", [I.GridDesc(6, 6, 12, 1.0, 4.0, 1.1), I.GridDesc(16, 12, 24, 1.0, 10.0, 1.05)],
                         ids=["6x6x12", "16x12x24"])
def test_sts_adjoint_matches_oracle(d):
    st = I.initial_state(d, 1, False)
    for k in ("vr", "vt", "vp"):
        st[k] = st[k] * 20.0
    og = O.Grid.from_desc(d)
    nu = 1.0
    c = og.coeffs(np.stack([st["vr"], st["vt"], st["vp"]]), st["br"], st["bt"], st["bp"], nu=nu, cfl=0.3)
    assert og.rkl2_stages(nu, c["dt"]) >= 4
    rng = np.random.default_rng(300)
    lam = {k: rng.normal(size=st[k].shape) for k in KEYS}
    lam["bt"][:, 0] = 0.0
    lam["bt"][:, -1] = 0.0
    ref, s1 = og.adjoint_step(st, lam, c["dt"], c["alpha_si"], nu=nu, cfl=0.3, tol=1e-13, sts=True)
    ds, dl = dev_state(st), dev_state(lam)
    out = {k: torch.empty_like(v) for k, v in ds.items()}
    prm = P.make_params(nu=nu, cfl=0.3, tol=1e-13, alpha_si_fixed=c["alpha_si"], max_iter=200000,
                        viscosity_sts=1)
    s2 = P.mhd_adjoint_step(grid(d), prm, fields(ds), c["dt"], fields(dl), fields(out))
    torch.cuda.synchronize()
    assert s1 == O.OK and s2 == P.MHD_OK
    for k in KEYS:
        e = rel_l2(to_np(out[k]), ref[k])
        assert e < 1e-9, (k, e)
