"""Helpers for GPU parity tests: move generator inputs to the device, run the library."""
import numpy as np
import torch

import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I

DEV = "cuda"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def to_np(t):
    return t.detach().cpu().numpy()


def grid(d, stream=None):
    return P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch, stream)


def dev_state(st):
    return {k: to_dev(v) for k, v in st.items()}


def fields(ds):
    return P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_iterate_at(og, alpha, b, it, itr, xr, x0=None, **kw):
    """The oracle's PCG iterate after the GPU's own iteration count `it`: xr (the oracle's
    converged iterate after itr iterations) when the counts agree, else a fixed-count oracle run
    from the same start, so that the 1e-11 gate always compares the same number of Krylov steps."""
    if it == itr:
        return xr
    x, _, _, _ = og.pcg(alpha, b, x0=x0, fixed_iters=it, **kw)
    return x
