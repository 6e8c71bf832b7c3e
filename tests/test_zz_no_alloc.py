"""mhd_force_noalloc against mhd_force, through the C ABI.

mhd_force_noalloc serves callers that cannot allocate device memory (a host code with a fixed
device-memory budget that owns every buffer, a latency-bound loop where cudaMalloc may
synchronise the device, or an allocator policy that forbids new allocations). It takes the grid
description instead of a grid object and keeps its scratch in a static device array. The test
runs it twice in a row on different inputs (the array keeps the previous call's contents) and
compares each result with the grid-based mhd_force and with the CPU oracle's force, within the
force tolerance of the parity tests. This file is collected last so a first-failure run has
already run every other test."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1811_02605_gb300 as P
from paper_1811_02605_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_force_noalloc_matches_mhd_force_two_calls():
    from paper_1811_02605_gb300 import build as B
    B.build()
    for idx, d in enumerate([I.GridDesc(24, 20, 40, 1.0, 8.0, 1.06), I.GridDesc(32, 32, 64, 1.0, 20.0, 1.05)]):
        g = P.mhd_grid_create(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch)
        desc = P.GridDesc(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch)
        for call in range(2):
            st = I.initial_state(d, 10 * idx + call, False)
            ds = {k: _dev(v) for k, v in st.items()}
            f = P.make_fields(ds["br"], ds["bt"], ds["bp"], ds["vr"], ds["vt"], ds["vp"])
            ref = torch.empty((3, d.nr, d.nt, d.np), dtype=torch.float64, device="cuda")
            out = torch.full_like(ref, float("nan"))
            dt = 0.01 * (call + 1)
            P.mhd_force(g, f, dt, ref)
            assert P.mhd_force_noalloc(desc, f, dt, out) == P.MHD_OK
            torch.cuda.synchronize()
            for c in range(3):
                assert _rel(out[c], ref[c]) < 1e-11, (idx, call, c)
            oref = O.Grid.from_desc(d).force(np.stack([st["vr"], st["vt"], st["vp"]]), st["br"], st["bt"], st["bp"], dt)
            got = out.cpu().numpy()
            for c in range(3):
                e = np.linalg.norm(got[c] - oref[c]) / np.linalg.norm(oref[c])
                assert e < 1e-11, (idx, call, c, e)


def test_force_noalloc_rejects_too_large_grid():
    desc = P.GridDesc(128, 64, 64, 1.0, 2.0, 1.0)   # 524,288 cells > 262,144
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    f = P.make_fields(z, z, z, z, z, z)
    assert P.mhd_force_noalloc(desc, f, 0.1, z) == P.MHD_ERR_ARG
