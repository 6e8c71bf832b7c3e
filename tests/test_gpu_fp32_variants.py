"""The FP32 inner-iteration variants of mixed-precision PCG, each forced in turn (MHD_FORCE_SLAB is
read when a grid tunes its FP32 kernels): -1 the split kernels (p update, stencil, update), -2 the p
update folded into the stencil with p double-buffered, -3 and -4 the recompute pair (no q stored,
x updated every second iteration; -4 with the r update walking the grid backwards; -5 at 6 CTAs per
SM), -6 to -8 the single-reduction pair (one reduction per iteration, p formed and A p applied in the
update kernel, r double-buffered; -7 and -8 with the residual kernel unrolled over the components),
-132 and -116
the same pair as plane-marching kernels whose rows are staged by bulk asynchronous copies (work
units of 32 or 16 planes), 16 the plane-marching pair. Each must reach
the FP64 tolerance on the true residual and agree with the oracle's FP64 solution (Sec. 2.2 PCG;
mixed precision is the FP32-inner / FP64-refinement reading of the solver)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import grid, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _system(d, seed):
    og = O.Grid.from_desc(d)
    rng = np.random.default_rng(seed)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    return og, b


@pytest.mark.parametrize("variant", ["-1", "-2", "-3", "-4", "-5", "-6", "-7", "-8", "-132", "-116", "16"])
@pytest.mark.parametrize("restart,inner", [(0, 0.1), (1, 1e-5)])
def test_mixed_variant_matches_fp64_oracle(monkeypatch, variant, restart, inner):
    # np = 256 (float4 groups, plane-marching tiles possible); nt = 18 leaves a ragged row tile
    d = I.GridDesc(20, 18, 256, 1.0, 10.0, 1.05)
    monkeypatch.setenv("MHD_FORCE_SLAB", variant)
    g = grid(d)
    og, b = _system(d, 31)
    alpha = 2.0
    xr, itr, _, _ = og.pcg(alpha, b, tol=1e-13)
    prm = P.make_params(tol=1e-9, inner_tol=inner, precision=P.PREC_MIXED, max_outer=60, max_iter=5000,
                        mixed_restart=restart)
    for nc in (3, 1, 2):
        x = torch.zeros((nc,) + b.shape[1:], dtype=torch.float64, device="cuda")
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b[:nc]), x, prm)
        assert st == P.MHD_OK and rr <= 1e-9, (variant, nc, st, rr)
        # the forced form is the one that ran (no FP64 solve on this grid: that form is untuned)
        assert P.mhd_grid_kernel_forms(g) == (0, int(variant)), (variant, P.mhd_grid_kernel_forms(g))
        res = b[:nc] - og.apply_M(alpha, to_np(x))
        assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(b[:nc]) * 1.0000001
        ref = xr if nc == 3 else og.pcg(alpha, b[:nc], tol=1e-13)[0]
        assert rel_l2(to_np(x), ref) < 1e-6, (variant, nc)


@pytest.mark.parametrize("variant", ["-2", "-3", "-4", "-6", "-7"])
def test_fused_variant_float2_groups_and_nonzero_start(monkeypatch, variant):
    # np = 250: not a multiple of 4, so the FP32 kernels work on float2 groups; x0 != 0
    d = I.GridDesc(12, 14, 250, 1.0, 6.0, 1.04)
    monkeypatch.setenv("MHD_FORCE_SLAB", variant)
    g = grid(d)
    og, b = _system(d, 32)
    rng = np.random.default_rng(33)
    x0 = rng.normal(size=b.shape) * 0.05
    for alpha in (0.4, 7.0):
        xr, _, _, _ = og.pcg(alpha, b, x0=x0, tol=1e-13)
        x = to_dev(x0)
        prm = P.make_params(tol=1e-9, inner_tol=0.1, precision=P.PREC_MIXED, max_outer=60, max_iter=5000)
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, prm)
        assert st == P.MHD_OK and rr <= 1e-9
        assert rel_l2(to_np(x), xr) < 1e-6, alpha


def test_fused_and_split_take_the_same_iterations(monkeypatch):
    # the fused kernel forms every p value with the same fma as the p update kernel, so the two
    # variants differ only in the reduction order of <p, q> (launch shape): iteration and
    # correction counts agree to within one
    d = I.GridDesc(24, 20, 128, 1.0, 10.0, 1.05)
    og, b = _system(d, 34)
    out = {}
    for variant in ("-1", "-2"):
        monkeypatch.setenv("MHD_FORCE_SLAB", variant)
        g = grid(d)
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        prm = P.make_params(tol=1e-9, inner_tol=0.1, precision=P.PREC_MIXED, max_outer=60, max_iter=5000)
        st, it, ou, rr = P.pcg_solve(g, 3.0, to_dev(b), x, prm)
        assert st == P.MHD_OK
        out[variant] = (it, ou, to_np(x))
    assert abs(out["-1"][0] - out["-2"][0]) <= 1 and abs(out["-1"][1] - out["-2"][1]) <= 1
    assert rel_l2(out["-2"][2], out["-1"][2]) < 1e-6


@pytest.mark.parametrize("variant", ["-1", "-2"])
@pytest.mark.parametrize("d", [I.GridDesc(10, 12, 64, 1.0, 5.0, 1.06), I.GridDesc(8, 10, 90, 1.0, 4.0, 1.05)],
                         ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_mixed_pc2_variant_matches_fp64_oracle(monkeypatch, variant, d):
    # the FP32 PC2 iteration with the p update split (-1) or folded into the stencil (-2; z~ in the
    # PC2 workspace, p~ alternating between the halves of the p double buffer); np = 90 takes the
    # float2 groups and the generic line kernel
    monkeypatch.setenv("MHD_FORCE_SLAB", variant)
    g = grid(d)
    og, b = _system(d, 35)
    alpha = 4.0
    xr, _, _, _ = og.pcg(alpha, b, tol=1e-13, pc2="lines")
    for restart, inner in ((0, 1e-3), (1, 1e-5)):
        for nc in (3, 2):
            x = torch.zeros((nc,) + b.shape[1:], dtype=torch.float64, device="cuda")
            prm = P.make_params(tol=1e-9, inner_tol=inner, precision=P.PREC_MIXED, max_outer=60, max_iter=5000,
                                mixed_restart=restart, preconditioner=1)
            st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b[:nc]), x, prm)
            assert st == P.MHD_OK and rr <= 1e-9, (variant, restart, nc, st, rr)
            res = b[:nc] - og.apply_M(alpha, to_np(x))
            assert np.linalg.norm(res) <= 1e-9 * np.linalg.norm(b[:nc]) * 1.0000001
            assert rel_l2(to_np(x), xr[:nc]) < 1e-6, (variant, restart, nc)


@pytest.mark.parametrize("k", [1, 2, 3, 8])
def test_recompute_pair_pending_x_update(monkeypatch, k):
    # the recompute pair adds alpha p to x two iterations at a time; an inner solve cut after an
    # odd or an even number of iterations must hand the pending update to the FP64 correction.
    # One outer pass with k inner iterations, against the fused variant (same arithmetic up to the
    # reduction order of the dot products): a lost alpha_k p_k would move x by O(1)
    d = I.GridDesc(12, 10, 128, 1.0, 5.0, 1.06)
    og, b = _system(d, 36)
    out = {}
    for variant in ("-2", "-3", "-4", "-6", "-7", "-132"):
        monkeypatch.setenv("MHD_FORCE_SLAB", variant)
        g = grid(d)
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        prm = P.make_params(tol=1e-14, inner_tol=1e-12, precision=P.PREC_MIXED, max_outer=1, max_iter=k)
        st, it, ou, rr = P.pcg_solve(g, 3.0, to_dev(b), x, prm)
        assert st == P.MHD_ERR_NOCONV and it == k and ou == 1, (variant, st, it, ou)
        out[variant] = to_np(x)
    # the single-reduction pair forms alpha from another (in exact arithmetic equal) expression,
    # so its FP32 iterates differ from the Hestenes-Stiefel ones by a few FP32 roundings per step
    for variant in ("-3", "-4", "-6", "-7", "-132"):
        gate = 1e-5 if variant in ("-6", "-7") else 1e-6
        assert rel_l2(out[variant], out["-2"]) < gate, (variant, k, rel_l2(out[variant], out["-2"]))


def test_recompute_pair_and_fused_take_the_same_iterations(monkeypatch):
    d = I.GridDesc(24, 20, 128, 1.0, 10.0, 1.05)
    og, b = _system(d, 34)
    out = {}
    for variant in ("-2", "-3", "-4", "-6", "-132"):
        monkeypatch.setenv("MHD_FORCE_SLAB", variant)
        g = grid(d)
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        prm = P.make_params(tol=1e-9, inner_tol=0.1, precision=P.PREC_MIXED, max_outer=60, max_iter=5000)
        st, it, ou, rr = P.pcg_solve(g, 3.0, to_dev(b), x, prm)
        assert st == P.MHD_OK and rr <= 1e-9
        out[variant] = (it, ou, to_np(x))
    for variant in ("-3", "-4", "-132"):
        assert abs(out[variant][0] - out["-2"][0]) <= 1 and abs(out[variant][1] - out["-2"][1]) <= 1
        assert rel_l2(out[variant][2], out["-2"][2]) < 1e-6
    # single-reduction pair: the same stop test on the true FP64 residual; its inner recurrence
    # rounds differently, so the counts agree within 5% and the solutions to the solver tolerance
    assert abs(out["-6"][0] - out["-2"][0]) <= max(2, 0.05 * out["-2"][0]), (out["-6"][0], out["-2"][0])
    assert rel_l2(out["-6"][2], out["-2"][2]) < 1e-6


def test_bulk_pair_ragged_rows_and_small_slabs(monkeypatch):
    # nt = 7 leaves a partial row tile (TJ = 4), nr = 9 with 16-plane units a single slab, np = 384;
    # two components too (the units of the third are skipped)
    d = I.GridDesc(9, 7, 384, 1.0, 4.0, 1.05)
    og, b = _system(d, 37)
    monkeypatch.setenv("MHD_FORCE_SLAB", "-116")
    g = grid(d)
    for nc in (3, 2, 1):
        xr, _, _, _ = og.pcg(2.0, b[:nc], tol=1e-13)
        x = torch.zeros((nc,) + b.shape[1:], dtype=torch.float64, device="cuda")
        prm = P.make_params(tol=1e-9, inner_tol=0.1, precision=P.PREC_MIXED, max_outer=60, max_iter=5000)
        st, it, ou, rr = P.pcg_solve(g, 2.0, to_dev(b[:nc]), x, prm)
        assert st == P.MHD_OK and rr <= 1e-9, (nc, st, rr)
        assert rel_l2(to_np(x), xr) < 1e-6, nc
