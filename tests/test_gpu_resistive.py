"""GPU implicit resistivity (Eq. 1 curl-curl term by PCG with PC1, Sec. 2.2) against the oracle's
og_step_opts(OG_OPT_RES_IMPLICIT), through the C ABI: fields within 1e-11 rel-L2 per step and
iteration counts within one, div B and the wall fluxes kept. At eta = 0.05 the step's own rounding
sensitivity (measured on the oracle) sets a 1e-10 gate."""
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


def _steps(d, eta, tol, max_iter, nsteps=3):
    st0 = I.initial_state(d, 2, False)
    g, og = grid(d), O.Grid.from_desc(d)
    ds = dev_state(st0)
    f = fields(ds)
    s = st0
    prm = P.make_params(nu=1e-3, eta=eta, cfl=0.4, tol=tol, max_iter=max_iter, resistivity_implicit=1)
    out = []
    for n in range(nsteps):
        stat, info = P.mhd_step(g, prm, f)
        torch.cuda.synchronize()
        s, oinfo = og.step(s, nu=1e-3, eta=eta, cfl=0.4, tol=tol, max_iter=max_iter, res_implicit=True)
        out.append((stat, info, oinfo, {k: to_np(v) for k, v in ds.items()}, s))
    return st0, og, out


def _invariants(og, st0, got):
    div0 = og.divb(st0["br"], st0["bt"], st0["bp"])
    assert np.abs(og.divb(got["br"], got["bt"], got["bp"]) - div0).max() <= 1e-12 * np.abs(st0["br"]).max()
    assert np.array_equal(got["br"][0], st0["br"][0])


def _check_counts(res, tol):
    for n, (stat, info, oinfo, got, ref) in enumerate(res):
        assert stat == P.MHD_OK and oinfo["status"] == O.OK
        assert abs(info["iters_res"] - oinfo["res_iters"]) <= 1, (n, info["iters_res"], oinfo["res_iters"])
        assert info["iters_res"] >= 1 and info["relres_res"] <= tol
        for q in range(3):
            assert abs(info["iters"][q] - oinfo["iters"][q]) <= 1, (n, info["iters"], oinfo["iters"])


def _check_fields(res, gate):
    for n, (stat, info, oinfo, got, ref) in enumerate(res):
        for k in KEYS:
            e = rel_l2(got[k], ref[k])
            assert e <= gate, (n, k, e)


# Every solve of a step (SI, viscous, resistive) runs at the tolerance given. At the workload
# tolerance 1e-9 the iteration counts agree within one. Converged iterates of two correct CG
# implementations agree to about 1% of their distance from the exact solution, which at tol 1e-9
# and this conditioning is above 1e-11 in the small B_phi (1.5e-11 at eta = 5e-3), so the 1e-11
# field gate is applied to steps at tol 1e-11.
@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_implicit_resistivity_step_parity(d):
    st0, og, res = _steps(d, 5e-3, 1e-9, 100000)
    _check_counts(res, 1e-9)
    _invariants(og, st0, res[-1][3])
    st0, og, res = _steps(d, 5e-3, 1e-11, 100000)
    _check_counts(res, 1e-11)
    _check_fields(res, 1e-11)
    _invariants(og, st0, res[-1][3])


@pytest.mark.parametrize("d", GRIDS, ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_implicit_resistivity_strong_eta_parity(d):
    # eta = 0.05: the face system is ill conditioned (about 250 iterations on 32x32x64) and the step
    # is sensitive to rounding: two oracle builds that differ only in the summation order of their
    # dot products disagree after 3 steps on 32x32x64 by 8.5e-8 in B_phi at tol 1e-9 (resistive
    # counts 112 against 113), 4.2e-10 at tol 1e-11, 1.7e-11 at tol 1e-12 (counts equal). Counts
    # within one at tol 1e-9; fields at tol 1e-12 within 1e-10, six times the oracle's own spread
    st0, og, res = _steps(d, 0.05, 1e-9, 100000)
    _check_counts(res, 1e-9)
    _invariants(og, st0, res[-1][3])
    st0, og, res = _steps(d, 0.05, 1e-12, 100000)
    _check_counts(res, 1e-12)
    _check_fields(res, 1e-10)
    _invariants(og, st0, res[-1][3])


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
