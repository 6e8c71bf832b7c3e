"""Domain decomposition of the implicit solve in r (Sec. 4.2: the code runs one MPI rank per GPU,
each rank owning part of the mesh; every operator application exchanges the boundary values it
needs with the neighbouring ranks, and every inner product sums its ranks' shares with an
allreduce of a few doubles).

The grid's radial rows are cut into contiguous slabs, one per rank, phi whole (so the periodic
wrap stays local) and theta whole (so the polar rings need no exchange). A rank holds its slab's
rows of every PCG vector ([ncomp][rows][nt][np]) and, for the operator, the one plane of p on
each side that belongs to its neighbours.

`pcg` is the point-Jacobi PCG of the single-grid solver's reading (Hestenes-Stiefel, one stacked
system, stop test ||r|| <= tol ||b|| on the recursive residual before each iteration, count =
number of x updates) in its unscaled form z = r / diag(M), written once for every rank (SPMD).
Per iteration it exchanges the boundary planes of p (one plane of ncomp x nt x np doubles with each
neighbour) and makes two allreduces, of 8 bytes (<p, q>) and 16 bytes (<r, z>, <r, r>).

The local arithmetic is in a `SlabOps` object: `GpuSlabOps` runs it in the CUDA library (a slab
grid, mhd_grid_create_slab, and its mhd_slab_* calls). The communication is a `Comm`: `TorchComm`
uses torch.distributed (NCCL between GPUs, gloo between host processes) with point-to-point
sends of the boundary planes; `ThreadComm` joins the slabs of several threads of one process
(one emulated rank per thread), which lets one GPU run a decomposed solve end to end.
"""
from __future__ import annotations

import math
import threading


def slab_bounds(nr: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [i0, i1) of rank `rank`: contiguous, sizes differing by at most one, at least 2 each."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank or world size")
    if nr < 2 * world:
        raise ValueError(f"{nr} radial rows cannot give {world} slabs of at least 2 rows")
    base, extra = divmod(nr, world)
    i0 = rank * base + min(rank, extra)
    return i0, i0 + base + (1 if rank < extra else 0)


class Comm:
    """What a rank needs from its neighbours: sums over all ranks and the boundary planes."""
    rank: int
    world: int

    def allreduce_sum(self, vals: list[float]) -> list[float]:
        raise NotImplementedError

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi) -> None:
        """Send send_lo to rank - 1 and send_hi to rank + 1, receive into recv_lo (from rank - 1)
        and recv_hi (from rank + 1); None where there is no neighbour."""
        raise NotImplementedError


class TorchComm(Comm):
    """torch.distributed: the process group's ranks are the slabs' ranks, in order."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allreduce_sum(self, vals):
        import torch
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor(vals, dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, group=self.group)
        return [float(v) for v in t.tolist()]

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        ops = []
        P2POp, d = self.dist.P2POp, self.dist
        if send_lo is not None:
            ops.append(P2POp(d.isend, send_lo, self.rank - 1, self.group))
            ops.append(P2POp(d.irecv, recv_lo, self.rank - 1, self.group))
        if send_hi is not None:
            ops.append(P2POp(d.isend, send_hi, self.rank + 1, self.group))
            ops.append(P2POp(d.irecv, recv_hi, self.rank + 1, self.group))
        if ops:
            for req in d.batch_isend_irecv(ops):
                req.wait()


class ThreadComm(Comm):
    """The ranks are threads of one process, one per slab; `hub` is shared by all of them."""

    class Hub:
        def __init__(self, world: int):
            self.world = world
            self.barrier = threading.Barrier(world)
            self.vals = [None] * world
            self.planes = [None] * world

    def __init__(self, hub: "ThreadComm.Hub", rank: int):
        self.hub = hub
        self.rank = rank
        self.world = hub.world

    def allreduce_sum(self, vals):
        h = self.hub
        h.vals[self.rank] = list(vals)
        h.barrier.wait()
        out = [sum(h.vals[r][q] for r in range(self.world)) for q in range(len(vals))]
        h.barrier.wait()
        return out

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        import torch
        on_gpu = any(t is not None and t.is_cuda for t in (send_lo, send_hi, recv_lo, recv_hi))
        h = self.hub
        h.planes[self.rank] = (send_lo, send_hi)
        if on_gpu:
            torch.cuda.synchronize()   # the planes are complete before a neighbour copies them
        h.barrier.wait()
        if recv_lo is not None:
            recv_lo.copy_(h.planes[self.rank - 1][1])
        if recv_hi is not None:
            recv_hi.copy_(h.planes[self.rank + 1][0])
        if on_gpu:
            torch.cuda.synchronize()
        h.barrier.wait()   # nobody reuses its send buffers before both neighbours have copied them


class SlabOps:
    """The local arithmetic of one slab: vectors are [ncomp][rows][nt][np]."""

    def apply(self, alpha, p, p_lo, p_hi, q) -> float:
        """q = M_alpha p on the slab's rows, ghost planes p_lo / p_hi (None at r0 / r1); the
        slab's share of <p, q>."""
        raise NotImplementedError

    def update(self, alpha, a, x, p, r, q, z) -> tuple[float, float]:
        """x += a p (x None: skipped), r -= a q, z = r / diag(M_alpha); shares of <r, z>, <r, r>."""
        raise NotImplementedError

    def pupdate(self, beta, z, p) -> None:
        """p = z + beta p (p = z when beta == 0)."""
        raise NotImplementedError


class GpuSlabOps(SlabOps):
    """A slab grid of the CUDA library (mhd_grid_create_slab) on torch's current stream, where the
    boundary planes are also packed and exchanged; vectors are CUDA float64 tensors."""

    def __init__(self, desc, i0: int, i1: int):
        import paper_1811_02605_gb300 as P
        self.P = P
        self.grid = P.mhd_grid_create_slab(desc.nr, desc.nt, desc.np, desc.r0, desc.r1, desc.stretch, i0, i1)

    def apply(self, alpha, p, p_lo, p_hi, q):
        return self.P.mhd_slab_apply(self.grid, alpha, p, p_lo, p_hi, q)

    def update(self, alpha, a, x, p, r, q, z):
        return self.P.mhd_slab_update(self.grid, alpha, a, x, p, r, q, z)

    def pupdate(self, beta, z, p):
        self.P.mhd_slab_pupdate(self.grid, beta, z, p)


def _planes(v, comm):
    """The boundary planes of v to send (contiguous copies) and the ghost buffers to fill."""
    import torch
    nc, rows, nt, np_ = v.shape
    send_lo = v[:, 0].contiguous() if comm.rank > 0 else None
    send_hi = v[:, rows - 1].contiguous() if comm.rank < comm.world - 1 else None
    recv_lo = torch.empty((nc, nt, np_), dtype=v.dtype, device=v.device) if comm.rank > 0 else None
    recv_hi = torch.empty((nc, nt, np_), dtype=v.dtype, device=v.device) if comm.rank < comm.world - 1 else None
    return send_lo, send_hi, recv_lo, recv_hi


def apply_with_halo(ops: SlabOps, comm: Comm, alpha, v, out) -> float:
    """out = M_alpha v on this rank's slab, after the exchange of v's boundary planes; returns the
    slab's share of <v, out>."""
    s_lo, s_hi, r_lo, r_hi = _planes(v, comm)
    comm.exchange(s_lo, s_hi, r_lo, r_hi)
    return ops.apply(alpha, v, r_lo, r_hi, out)


def pcg(ops: SlabOps, comm: Comm, alpha: float, b, x, tol: float = 1e-9, max_iter: int = 100000,
        fixed_iters: int = 0):
    """Solve M_alpha x = b over all ranks (x holds this rank's rows of x0). Returns
    (status, iterations, ||r|| / ||b||) with status "ok", "noconv" or "breakdown"; with
    fixed_iters > 0 exactly that many iterations run."""
    import torch
    r = torch.empty_like(b)
    z = torch.empty_like(b)
    p = torch.empty_like(b)
    q = torch.empty_like(b)
    # r = b - M x0, z = r / d; <b, b> from the same update with a = 0 on a copy of b
    r.copy_(b)
    _, bb = ops.update(alpha, 0.0, None, None, r, q.zero_(), z)
    apply_with_halo(ops, comm, alpha, x, q)
    r.copy_(b)
    rz, rr = ops.update(alpha, 1.0, None, None, r, q, z)
    bb, rz, rr = comm.allreduce_sum([bb, rz, rr])
    bnorm = math.sqrt(bb)
    if bnorm == 0.0:
        x.zero_()
        return "ok", 0, 0.0
    ops.pupdate(0.0, z, p)
    k = 0
    status = "ok"
    rn = math.sqrt(rr)
    while True:
        if fixed_iters > 0:
            if k >= fixed_iters:
                break
        else:
            if rn <= tol * bnorm:
                break
            if k >= max_iter:
                status = "noconv"
                break
        pq = comm.allreduce_sum([apply_with_halo(ops, comm, alpha, p, q)])[0]
        if not pq > 0.0:
            status = "breakdown"
            break
        a = rz / pq
        rz_new, rr = comm.allreduce_sum(list(ops.update(alpha, a, x, p, r, q, z)))
        k += 1
        rn = math.sqrt(rr)
        ops.pupdate(rz_new / rz, z, p)
        rz = rz_new
    return status, k, rn / bnorm
