"""The scalar recurrence of the single-reduction pair that the FP32 inner iteration runs (Sec. 2.2
PCG with point-Jacobi preconditioning, in the Jacobi-scaled variables): one reduction per
iteration gives gamma = <r, r> and delta = <r, A r>, and
    <p, A p> = delta + beta (2 <r, A p_old> + beta <p_old, A p_old>),
where <r, A p_old> was summed when r was formed and <p_old, A p_old> is the previous denominator.
Written out here in FP64 numpy on the oracle's operator, it must reproduce the oracle's
Hestenes-Stiefel PCG iterates after the same number of iterations; the Chronopoulos-Gear shortcut
for the cross term (-gamma / alpha_old) must too, in exact arithmetic, and does to rounding here.
The CPU pins the algebra; the GPU kernels' own parity is in tests/test_gpu_fp32_variants.py."""
import numpy as np
import pytest

import oracle as O
from paper_1811_02605_gb300 import inputs as I


def _pair(og, alpha, b, iters, cross="exact"):
    dg = og.diag(alpha)[None, :, :, None]
    s = 1.0 / np.sqrt(dg)

    def A(y):
        return s * og.apply_M(alpha, s * y)

    y = np.zeros_like(b)
    r = s * b
    p = np.zeros_like(b)
    gamma_prev = alpha_prev = pq = wp = None
    for k in range(iters):
        w = A(r)
        gamma, delta = float(np.vdot(r, r)), float(np.vdot(r, w))
        if k == 0:
            beta, den = 0.0, delta
        else:
            beta = gamma / gamma_prev
            x_term = wp if cross == "exact" else -gamma / alpha_prev
            den = delta + beta * (2.0 * x_term + beta * pq)
        a = gamma / den
        p = r + beta * p
        q = A(p)
        y = y + a * p
        r = r - a * q
        wp = float(np.vdot(r, q))   # <r_new, A p>, summed by the update kernel
        gamma_prev, alpha_prev, pq = gamma, a, den
    return s * y


@pytest.mark.parametrize("iters", [1, 2, 5, 12])
def test_pair_recurrence_reproduces_hestenes_stiefel_iterates(iters):
    d = I.GridDesc(10, 8, 16, 1.0, 5.0, 1.06)
    og = O.Grid.from_desc(d)
    rng = np.random.default_rng(51)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    for alpha in (0.3, 6.0):
        ref, _, _, _ = og.pcg(alpha, b, fixed_iters=iters)
        for cross in ("exact", "chronopoulos_gear"):
            x = _pair(og, alpha, b, iters, cross)
            err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
            assert err < 1e-10, (alpha, iters, cross, err)


def test_pair_recurrence_wrong_cross_term_sign_is_caught():
    # a dropped factor or sign in the denominator moves the iterates at once
    d = I.GridDesc(10, 8, 16, 1.0, 5.0, 1.06)
    og = O.Grid.from_desc(d)
    rng = np.random.default_rng(52)
    b = rng.normal(size=(3, d.nr, d.nt, d.np)) * og.volumes()[None, :, :, None]
    ref, _, _, _ = og.pcg(2.0, b, fixed_iters=4)
    dg = og.diag(2.0)[None, :, :, None]
    s = 1.0 / np.sqrt(dg)

    def A(y):
        return s * og.apply_M(2.0, s * y)

    y, r, p = np.zeros_like(b), s * b, np.zeros_like(b)
    gp = pq = wp = None
    for k in range(4):
        w = A(r)
        g, dl = float(np.vdot(r, r)), float(np.vdot(r, w))
        beta = 0.0 if k == 0 else g / gp
        den = dl if k == 0 else dl + beta * (-2.0 * wp + beta * pq)   # planted sign error
        a = g / den
        p = r + beta * p
        q = A(p)
        y, r = y + a * p, r - a * q
        wp = float(np.vdot(r, q))
        gp, pq = g, den
    assert np.linalg.norm(s * y - ref) / np.linalg.norm(ref) > 1e-3
