"""Test helpers: independent geometry and analytic fields (no oracle or library code)."""
import math

import numpy as np

from paper_1811_02605_gb300 import inputs as I


def centres(d):
    r = I.radial_nodes(d)
    rc = 0.5 * (r[1:] + r[:-1])
    thc = (np.arange(d.nt) + 0.5) * math.pi / d.nt
    phc = (np.arange(d.np) + 0.5) * 2 * math.pi / d.np
    return np.meshgrid(rc, thc, phc, indexing="ij")


def exact_volumes(d):
    """Exact volume of each spherical cell, [nr, nt]."""
    r = I.radial_nodes(d)
    th = np.arange(d.nt + 1) * math.pi / d.nt
    c = np.cos(th)
    c[0], c[-1] = 1.0, -1.0
    return ((r[1:] ** 3 - r[:-1] ** 3) / 3)[:, None] * (c[:-1] - c[1:])[None, :] * (2 * math.pi / d.np)


def cart(R, TH, PH):
    return np.stack([R * np.sin(TH) * np.cos(PH), R * np.sin(TH) * np.sin(PH), R * np.cos(TH)])


def to_sph(vec, TH, PH):
    """Cartesian vector field -> (r, theta, phi) components at (TH, PH)."""
    st, ct, sp, cp = np.sin(TH), np.cos(TH), np.sin(PH), np.cos(PH)
    return np.stack([vec[0] * st * cp + vec[1] * st * sp + vec[2] * ct,
                     vec[0] * ct * cp + vec[1] * ct * sp - vec[2] * st,
                     -vec[0] * sp + vec[1] * cp])


def wl2(V, err2, ref2, sl=slice(None)):
    """Volume-weighted relative L2 over the radial slice `sl`."""
    return math.sqrt(np.sum((V * err2)[sl]) / np.sum((V * ref2)[sl]))


def dipole_B(x):
    r = np.sqrt(np.sum(x * x, axis=0))
    m = np.zeros_like(x)
    m[2] = 1.0
    return (3 * x[2][None] * x / r ** 2 - m) / r ** 3


def zero_faces(d):
    return (np.zeros((d.nr + 1, d.nt, d.np)), np.zeros((d.nr, d.nt + 1, d.np)),
            np.zeros((d.nr, d.nt, d.np)))
