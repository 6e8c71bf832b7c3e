"""Test-side local arithmetic for the decomposed PCG driver: the oracle's operator restricted to a
slab (the operator is a 7-point stencil, so the slab's rows of M p depend only on p at the slab's
rows and the ghost planes on either side; they are taken from the oracle applied to a vector that
holds just those planes)."""
import numpy as np

import oracle as O
from paper_1811_02605_gb300 import dist


class OracleSlabOps(dist.SlabOps):
    def __init__(self, og, i0, i1):
        self.og, self.i0, self.i1 = og, i0, i1

    def apply(self, alpha, p, p_lo, p_hi, q):
        og = self.og
        pn = p.numpy()
        full = np.zeros((pn.shape[0], og.nr, og.nt, og.np))
        full[:, self.i0:self.i1] = pn
        if p_lo is not None:
            full[:, self.i0 - 1] = p_lo.numpy()
        if p_hi is not None:
            full[:, self.i1] = p_hi.numpy()
        q.numpy()[...] = og.apply_M(alpha, full)[:, self.i0:self.i1]
        return O.dot(pn, q.numpy())

    def update(self, alpha, a, x, p, r, q, z):
        d = self.og.diag(alpha)[self.i0:self.i1][None, :, :, None]
        rn, qn, zn = r.numpy(), q.numpy(), z.numpy()
        if x is not None:
            xn = x.numpy()
            xn += a * p.numpy()
        rn -= a * qn
        zn[...] = rn / d
        return O.dot(rn, zn), O.dot(rn, rn)

    def pupdate(self, beta, z, p):
        if beta == 0.0:
            p.numpy()[...] = z.numpy()
        else:
            pn = p.numpy()
            pn[...] = z.numpy() + beta * pn
