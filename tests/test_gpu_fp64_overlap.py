"""The FP64 PCG iteration with its components overlapped (MHD_FORCE_SLAB=-64: the p update of one
component on a second stream while the stencil of the previous one runs; <p, q> summed from the
components' shares), against the FP64 oracle and against the split iteration. The stencil of
Eq. 10's operator couples no components, so the overlap changes only the order in which <p, q> is
summed: the iterate after the same number of iterations agrees with the oracle's to 1e-11 relative
L2 (Sec. 2.2 PCG, point-Jacobi preconditioning)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import grid, oracle_iterate_at, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu


def _system(d, seed):
    og = O.Grid.from_desc(d)
    rng = np.random.default_rng(seed)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    return og, b, rng


@pytest.mark.parametrize("d", [I.GridDesc(20, 18, 256, 1.0, 10.0, 1.05), I.GridDesc(23, 17, 46, 1.0, 10.0, 1.07)],
                         ids=lambda d: f"{d.nr}x{d.nt}x{d.np}")
def test_overlapped_fp64_matches_oracle(monkeypatch, d):
    monkeypatch.setenv("MHD_FORCE_SLAB", "-64")
    g = grid(d)
    og, b, rng = _system(d, 41)
    x0 = rng.normal(size=b.shape) * 0.1
    for alpha in (0.05, 4.0):
        for nc in (3, 1, 2):
            prm = P.make_params(tol=1e-11, max_iter=5000)
            x = to_dev(x0[:nc])
            st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b[:nc]), x, prm)
            xr, itr, _, str_ = og.pcg(alpha, b[:nc], x0=x0[:nc], tol=1e-11, max_iter=5000)
            assert st == P.MHD_OK and str_ == O.OK and rr <= 1e-11, (nc, st, rr)
            assert abs(it - itr) <= 1, (nc, it, itr)
            xo = oracle_iterate_at(og, alpha, b[:nc], it, itr, xr, x0=x0[:nc])
            assert rel_l2(to_np(x), xo) < 1e-11, (alpha, nc, it, itr, rel_l2(to_np(x), xo))


@pytest.mark.parametrize("k", [1, 2, 7])
def test_overlapped_fp64_fixed_trajectory(monkeypatch, k):
    # a solve cut after k iterations: the deferred x update of the last p must reach x, and every
    # component's p update must see the same beta
    d = I.GridDesc(16, 12, 128, 1.0, 6.0, 1.05)
    og, b, rng = _system(d, 42)
    out = {}
    for variant in ("-1", "-64"):
        monkeypatch.setenv("MHD_FORCE_SLAB", variant)
        g = grid(d)
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        prm = P.make_params(tol=1e-30, max_iter=k)
        st, it, ou, rr = P.pcg_solve(g, 2.0, to_dev(b), x, prm)
        assert st == P.MHD_ERR_NOCONV and it == k, (variant, st, it)
        out[variant] = to_np(x)
    xo, _, _, _ = og.pcg(2.0, b, fixed_iters=k)
    for variant in ("-1", "-64"):
        assert rel_l2(out[variant], xo) < 1e-11, (variant, k, rel_l2(out[variant], xo))


def test_overlapped_fp64_graph_batches_and_reuse(monkeypatch):
    # long solves run the iteration from captured graphs (the side stream joins the capture);
    # a second solve on the same grid and a zero right-hand side component
    monkeypatch.setenv("MHD_FORCE_SLAB", "-64")
    d = I.GridDesc(24, 20, 64, 1.0, 20.0, 1.05)
    g = grid(d)
    og, b, _ = _system(d, 43)
    b[1] = 0.0
    for alpha in (0.5, 0.5):
        x = torch.zeros(b.shape, dtype=torch.float64, device="cuda")
        st, it, ou, rr = P.pcg_solve(g, alpha, to_dev(b), x, P.make_params(tol=1e-11, max_iter=5000))
        xr, itr, _, _ = og.pcg(alpha, b, tol=1e-11, max_iter=5000)
        assert st == P.MHD_OK and it > 32 and abs(it - itr) <= 1
        assert rel_l2(to_np(x), oracle_iterate_at(og, alpha, b, it, itr, xr)) < 1e-11
