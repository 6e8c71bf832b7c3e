"""Slab grids of the CUDA library (domain decomposition in r, Sec. 4.2) on one GPU: a slab's rows
of M p against the whole grid's operator, and the decomposed point-Jacobi PCG with the library's
slab calls as the local arithmetic (three emulated ranks, one thread each, exchanging boundary
planes and summing inner-product shares in the process) against the single-domain oracle."""
import threading

import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import dist
from paper_1811_02605_gb300 import inputs as I
from tests.gpu_util import grid, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu
D = I.GridDesc(23, 17, 46, 1.0, 10.0, 1.07)   # ragged: odd nr and nt, np not a multiple of 4


@pytest.mark.parametrize("world", [2, 3])
def test_slab_rows_equal_whole_grid_operator(world):
    g = grid(D)
    rng = np.random.default_rng(41)
    for nc in (1, 3):
        p = to_dev(rng.normal(size=(nc, D.nr, D.nt, D.np)))
        for alpha in (0.0, 0.3, 17.0):
            q = torch.empty_like(p)
            P.mhd_apply_operator(g, alpha, p, q)
            for r in range(world):
                i0, i1 = dist.slab_bounds(D.nr, world, r)
                s = P.mhd_grid_create_slab(D.nr, D.nt, D.np, D.r0, D.r1, D.stretch, i0, i1)
                ps = p[:, i0:i1].contiguous()
                lo = p[:, i0 - 1].contiguous() if i0 > 0 else None
                hi = p[:, i1].contiguous() if i1 < D.nr else None
                qs = torch.empty_like(ps)
                pq = P.mhd_slab_apply(s, alpha, ps, lo, hi, qs)
                torch.cuda.synchronize()
                ref = q[:, i0:i1]
                assert float((qs - ref).abs().max()) <= 1e-14 * float(ref.abs().max()), (r, alpha, nc)
                assert abs(pq - float(torch.sum(ps * qs))) <= 1e-12 * abs(pq)


def test_slab_grid_refuses_whole_grid_calls_and_wrong_ghosts():
    s = P.mhd_grid_create_slab(D.nr, D.nt, D.np, D.r0, D.r1, D.stretch, 5, 12)
    p = torch.zeros((1, 7, D.nt, D.np), dtype=torch.float64, device="cuda")
    q = torch.empty_like(p)
    with pytest.raises(P.MhdError):
        P.mhd_apply_operator(s, 1.0, p, q)
    with pytest.raises(P.MhdError):   # an interior slab needs both ghost planes
        P.mhd_slab_apply(s, 1.0, p, None, None, q)
    with pytest.raises(P.MhdError):
        P.mhd_grid_create_slab(D.nr, D.nt, D.np, D.r0, D.r1, D.stretch, 20, 21)


@pytest.mark.parametrize("world", [1, 3])
def test_decomposed_pcg_on_gpu_matches_oracle(world):
    og = O.Grid.from_desc(D)
    rng = np.random.default_rng(3)
    b = rng.normal(size=(3, D.nr, D.nt, D.np)) * og.volumes()[None, :, :, None]
    x0 = rng.normal(size=b.shape) * 0.1
    for alpha in (0.05, 4.0):
        hub = dist.ThreadComm.Hub(world)
        parts = [None] * world
        errors = []

        def run(r):
            try:
                i0, i1 = dist.slab_bounds(D.nr, world, r)
                ops = dist.GpuSlabOps(D, i0, i1)
                xl = to_dev(x0[:, i0:i1])
                st, it, rr = dist.pcg(ops, dist.ThreadComm(hub, r), alpha, to_dev(b[:, i0:i1]), xl, tol=1e-9)
                parts[r] = ((i0, i1), st, it, rr, to_np(xl))
            except Exception as e:   # surfaced below; the other ranks would wait at the barrier
                errors.append(e)
                hub.barrier.abort()

        ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        assert not errors, errors
        xr, itr, _, _ = og.pcg(alpha, b, x0=x0, tol=1e-9)
        it = parts[0][2]
        assert all(p[1] == "ok" and p[2] == it for p in parts)
        assert abs(it - itr) <= 1, (it, itr)
        if it != itr:
            xr = og.pcg(alpha, b, x0=x0, fixed_iters=it)[0]
        x = np.zeros_like(b)
        for (i0, i1), _, _, _, xl in parts:
            x[:, i0:i1] = xl
        assert rel_l2(x, xr) < 1e-11, (world, alpha, it, itr)
