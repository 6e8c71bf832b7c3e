"""The seeded synthetic inputs (paper_1811_02605_gb300/inputs.py, shared by the oracle and the GPU
path as data only) against the recipe they state: grid sizes, radial range and stretch of each
workload, determinism of the seeded draws, div_h B = 0 to round-off (every magnetic piece is built
from a vector potential by Stokes), and the batched-system recipe."""
import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I


def test_workload_table():
    w = I.WORKLOADS
    assert w["parity_32x32x64"]["desc"] == I.GridDesc(32, 32, 64, 1.0, 20.0, 1.05)
    assert w["fluxrope_256x256x512"]["desc"] == I.GridDesc(256, 256, 512, 1.0, 30.0, 1.02)
    assert w["fluxrope_256x256x512"]["rope"] and not w["parity_32x32x64"]["rope"]
    for k in w:
        assert w[k]["tol"] == 1e-9 and w[k]["cfl"] == 0.4 and w[k]["nu"] == 1e-3


@pytest.mark.parametrize("rope", [False, True])
def test_initial_state_is_seeded_and_divergence_free(rope):
    d = I.GridDesc(12, 10, 16, 1.0, 2.0, 1.05)
    a = I.initial_state(d, 3, rope)
    b = I.initial_state(d, 3, rope)
    c = I.initial_state(d, 4, rope)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert any(not np.array_equal(a[k], c[k]) for k in a)
    g = O.Grid.from_desc(d)
    div = g.divb(a["br"], a["bt"], a["bp"])
    scale = max(np.abs(a["br"]).max(), np.abs(a["bt"]).max(), np.abs(a["bp"]).max())
    # div_h B is a sum of face fluxes divided by the volume: round-off relative to |B| / h
    assert np.abs(div).max() * d.r0 * (np.pi / d.nt) <= 1e-13 * scale


def test_batched_recipe():
    items = I.batched_items(16)
    for it in items:
        d = it["desc"]
        assert d.nr == d.nt and d.np == 2 * d.nt and d.nt in range(32, 129, 16)
        assert 1.02 <= d.stretch <= 1.08 and d.r0 == 1.0 and d.r1 == 20.0
    assert len({it["seed"] for it in items}) == len(items)
    again = I.batched_items(16)
    assert [it["desc"] for it in again] == [it["desc"] for it in items]
