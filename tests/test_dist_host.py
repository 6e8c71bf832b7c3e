"""The decomposed point-Jacobi PCG (r slabs, one per rank; Sec. 4.2: each rank exchanges its
boundary planes for every operator application and sums the shares of every inner product):
world size 2 as gloo processes on the host and world sizes 1 to 4 as threads, with the oracle's
operator restricted to each slab as the local arithmetic, against the single-domain oracle PCG:
iteration counts within one and iterates within 1e-11 of the oracle's after the same count."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp

import oracle as O
from paper_1811_02605_gb300 import dist
from paper_1811_02605_gb300 import inputs as I
from tests.dist_helpers import OracleSlabOps

D = I.GridDesc(12, 10, 16, 1.0, 6.0, 1.06)


def _system(seed=3):
    og = O.Grid.from_desc(D)
    rng = np.random.default_rng(seed)
    b = rng.normal(size=(3, D.nr, D.nt, D.np)) * og.volumes()[None, :, :, None]
    x0 = rng.normal(size=b.shape) * 0.1
    return og, b, x0


def _rank_solve(og, comm, b, x0, alpha, **kw):
    i0, i1 = dist.slab_bounds(D.nr, comm.world, comm.rank)
    ops = OracleSlabOps(og, i0, i1)
    bl = torch.from_numpy(np.array(b[:, i0:i1], copy=True))
    xl = torch.from_numpy(np.array(x0[:, i0:i1], copy=True))
    st, it, rr = dist.pcg(ops, comm, alpha, bl, xl, **kw)
    return (i0, i1), st, it, rr, xl.numpy()


def _check(og, b, x0, alpha, parts):
    xr, itr, rrr, str_ = og.pcg(alpha, b, x0=x0, tol=1e-9)
    it = parts[0][2]
    assert all(p[1] == "ok" and p[2] == it for p in parts)
    assert abs(it - itr) <= 1, (it, itr)
    if it != itr:
        xr = og.pcg(alpha, b, x0=x0, fixed_iters=it)[0]
    x = np.zeros_like(b)
    for (i0, i1), _, _, _, xl in parts:
        x[:, i0:i1] = xl
    assert np.linalg.norm(x - xr) <= 1e-11 * np.linalg.norm(xr), (it, itr)


def test_slab_bounds_cover_the_rows():
    for nr in (4, 7, 12, 256):
        for world in (1, 2, 3):
            if nr < 2 * world:
                continue
            b = [dist.slab_bounds(nr, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == nr
            assert all(b[q][1] == b[q + 1][0] for q in range(world - 1))
            sizes = [i1 - i0 for i0, i1 in b]
            assert min(sizes) >= 2 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        dist.slab_bounds(3, 2, 0)


@pytest.mark.parametrize("world", [1, 2, 3, 4])
def test_decomposed_pcg_threads_match_oracle(world):
    import threading
    og, b, x0 = _system()
    for alpha in (0.05, 4.0):
        hub = dist.ThreadComm.Hub(world)
        parts = [None] * world

        def run(r):
            parts[r] = _rank_solve(og, dist.ThreadComm(hub, r), b, x0, alpha, tol=1e-9)

        ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        _check(og, b, x0, alpha, parts)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gloo_rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    og, b, x0 = _system()
    res = {}
    for alpha in (0.05, 4.0):
        res[alpha] = _rank_solve(og, dist.TorchComm(), b, x0, alpha, tol=1e-9)
    out[rank] = res
    tdist.barrier()
    tdist.destroy_process_group()


def test_decomposed_pcg_gloo_two_ranks_match_oracle():
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_gloo_rank, args=(2, port, out), nprocs=2, start_method="spawn")
    og, b, x0 = _system()
    for alpha in (0.05, 4.0):
        _check(og, b, x0, alpha, [out[0][alpha], out[1][alpha]])
