"""Pins of the oracle's PC2 (Sec. 2.2: block-Jacobi with zero-fill incomplete LU; reading R9):
for one whole-grid block and for one block per periodic phi line, the defining ILU(0) property
(the factor product equals the block-diagonal part of M_alpha on its pattern), the block
structure itself (no coupling between blocks), symmetry and positivity of the preconditioner, the
PCG+PC2 solution against a dense solve, and fewer iterations than PC1 on the stretched operator."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_1811_02605_gb300 import inputs as I

D = I.GridDesc(4, 5, 6, 1.0, 6.0, 1.2)


def _dense(fn, n, shape):
    M = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        M[:, c] = fn(e.reshape(shape)).ravel()
    return M


def _same_line(d):
    ij = np.arange(d.nr * d.nt * d.np) // d.np
    return ij[:, None] == ij[None, :]


@pytest.mark.parametrize("blocks", ["whole", "lines"])
@pytest.mark.parametrize("alpha", [0.05, 3.0])
def test_ilu0_product_matches_operator_on_its_block_pattern(alpha, blocks):
    g = O.Grid.from_desc(D)
    n = D.nr * D.nt * D.np
    shape = (1, D.nr, D.nt, D.np)
    dt, st = g.ilu0(alpha, blocks)
    assert st == 0 and np.all(dt > 0)
    M = _dense(lambda x: g.apply_M(alpha, x), n, shape)
    Pinv = _dense(lambda x: g.ilu0_apply(alpha, dt, x, blocks), n, shape)
    P = np.linalg.inv(Pinv)
    Mb = M * _same_line(D) if blocks == "lines" else M
    pattern = Mb != 0.0
    scale = np.abs(M).max()
    # zero fill: (dt + L) dt^-1 (dt + U) reproduces every entry of the block part of M on its pattern
    assert np.abs((P - Mb)[pattern]).max() <= 1e-12 * scale
    # and differs outside it (the dropped fill), so the test is not vacuous
    assert np.abs((P - Mb)[~pattern]).max() > 1e-6 * scale
    if blocks == "lines":
        # block-Jacobi: nothing couples two phi lines
        assert np.all(P[~_same_line(D)] == 0.0) or np.abs(P[~_same_line(D)]).max() <= 1e-12 * scale
        assert np.all(Pinv[~_same_line(D)] == 0.0)
    # symmetric positive definite preconditioner
    assert np.abs(P - P.T).max() <= 1e-12 * scale
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0.0
    # the factors rebuilt from dt and the strict triangles give the same P
    Dt = np.diag(dt.ravel())
    P2 = (Dt + np.tril(Mb, -1)) @ np.diag(1.0 / dt.ravel()) @ (Dt + np.triu(Mb, 1))
    assert np.abs(P2 - P).max() <= 1e-11 * scale


@pytest.mark.parametrize("blocks", ["whole", "lines"])
def test_pcg_pc2_matches_dense_solve_and_beats_pc1(blocks):
    d = I.GridDesc(8, 8, 12, 1.0, 20.0, 1.3)
    g = O.Grid.from_desc(d)
    n = d.nr * d.nt * d.np
    rng = np.random.default_rng(21)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * g.volumes()[None, :, :, None]
    alpha = 5.0
    M = _dense(lambda x: g.apply_M(alpha, x), n, (1, d.nr, d.nt, d.np))
    cf = sla.cho_factor(M)
    xd = np.stack([sla.cho_solve(cf, b[c].ravel()) for c in range(3)]).reshape(b.shape)
    x2, it2, rr2, st2 = g.pcg(alpha, b, tol=1e-13, pc2=blocks)
    assert st2 == O.OK and rr2 <= 1e-13
    assert np.linalg.norm(x2 - xd) <= 1e-10 * np.linalg.norm(xd)
    _, it1, _, _ = g.pcg(alpha, b, tol=1e-9)
    _, it2b, _, _ = g.pcg(alpha, b, tol=1e-9, pc2=blocks)
    assert it2b < it1, (it2b, it1)
    # b = 0 and alpha = 0 (M diagonal: ILU(0) is exact, one iteration)
    x0, i0, _, _ = g.pcg(alpha, np.zeros_like(b), pc2=blocks)
    assert i0 == 0 and np.all(x0 == 0.0)
    _, ia, _, sa = g.pcg(0.0, b, tol=1e-12, pc2=blocks)
    assert sa == O.OK and ia == 1


def test_line_blocks_capture_the_polar_phi_coupling():
    # on the parity workload's SI operator the phi-line blocks do most of what one whole block does
    w, st = I.workload("parity_32x32x64")
    g = O.Grid.from_desc(w["desc"])
    v = np.stack([st["vr"], st["vt"], st["vp"]])
    c = g.coeffs(v, st["br"], st["bt"], st["bp"])
    b = g.force(v, st["br"], st["bt"], st["bp"], c["dt"])
    _, i1, _, _ = g.pcg(c["alpha_si"], b, tol=1e-9)
    _, il, _, _ = g.pcg(c["alpha_si"], b, tol=1e-9, pc2="lines")
    _, iw, _, _ = g.pcg(c["alpha_si"], b, tol=1e-9, pc2="whole")
    assert iw <= il < i1 / 3, (i1, il, iw)


def test_step_with_pc2_agrees_within_solver_tolerance():
    d = I.GridDesc(8, 8, 16, 1.0, 10.0, 1.05)
    st = I.initial_state(d, 0, False)
    g = O.Grid.from_desc(d)
    a, ia = g.step(st, tol=1e-11)
    b, ib = g.step(st, tol=1e-11, pc2=True)
    assert ia["status"] == O.OK and ib["status"] == O.OK
    assert ib["iters"][0] < ia["iters"][0]
    for k in ("vr", "vt", "vp", "br", "bt", "bp"):
        assert np.linalg.norm(a[k] - b[k]) <= 1e-8 * np.linalg.norm(a[k]), k
