"""Seeded synthetic inputs for the zero-beta MHD step (shared by the library's tests, the
benchmark and the CPU oracle's tests).

This module draws random numbers and evaluates smooth analytic fields. It holds none of the
step's arithmetic: no operator, no solver, no force, no induction update. The only grid
quantities it needs are node/centre coordinates, edge lengths and face areas, which it computes
itself from the grid definition (geometric radial stretch, uniform theta in [0, pi], periodic phi).

Magnetic field: every piece of the initial field is given as a vector potential A. The
generator integrates A along each cell edge (midpoint rule on the edge) and forms the magnetic
flux through each face as the signed sum of the four edge integrals around it (Stokes' theorem),
then divides by the face area. Because each edge integral enters two faces of a cell with
opposite signs, the discrete divergence of the generated B is zero to round-off.

Layouts (all float64, C order, phi fastest):
  br [nr+1][nt][np]   radial faces at r_i
  bt [nr][nt+1][np]   theta faces at theta_j (j = 0 and nt are the poles, stored as 0)
  bp [nr][nt][np]     phi faces at phi_k
  vr, vt, vp [nr][nt][np] cell centres

Workloads (Sec. 3 of the paper describes the production flux-rope run these stand in for; its
grid and boundary data are not public, so the shapes below are synthetic):
  parity_32x32x64     32x32x64, r in [1,20], stretch 1.05, dipole + 1e-3 5-mode perturbation
  fluxrope_256x256x512 256x256x512, r in [1,30], stretch 1.02, dipole + perturbation + flux rope
  adjoint_128x128x256  128x128x256, r in [1,20], stretch 1.05**0.25
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SEED_BASE = 1811


@dataclass(frozen=True)
class GridDesc:
    nr: int
    nt: int
    np: int
    r0: float
    r1: float
    stretch: float


WORKLOADS = {
    "parity_32x32x64": dict(desc=GridDesc(32, 32, 64, 1.0, 20.0, 1.05), index=0, rope=False,
                            nu=1e-3, eta=0.0, cfl=0.4, steps=10, tol=1e-9),
    "fluxrope_256x256x512": dict(desc=GridDesc(256, 256, 512, 1.0, 30.0, 1.02), index=1, rope=True,
                                 nu=1e-3, eta=0.0, cfl=0.4, steps=20, tol=1e-9),
    "adjoint_128x128x256": dict(desc=GridDesc(128, 128, 256, 1.0, 20.0, 1.05 ** 0.25), index=4,
                                rope=False, nu=1e-3, eta=0.0, cfl=0.4, steps=20, tol=1e-9),
}


# ----------------------------------------------------------------------------------------------
# grid coordinates (definition of the grid, not of the method)
# ----------------------------------------------------------------------------------------------
def radial_nodes(d: GridDesc) -> np.ndarray:
    """r_0 = r0, r_{i+1} = r_i + h0 s^i with h0 = (r1-r0)(s-1)/(s^nr-1); powers by repeated
    multiplication so every platform produces the same bits."""
    s = float(d.stretch)
    if s == 1.0:
        h0 = (d.r1 - d.r0) / d.nr
    else:
        snr = 1.0
        for _ in range(d.nr):
            snr *= s
        h0 = (d.r1 - d.r0) * (s - 1.0) / (snr - 1.0)
    r = np.empty(d.nr + 1)
    r[0] = d.r0
    dr = h0
    for i in range(d.nr):
        r[i + 1] = r[i] + dr
        dr *= s
    return r


def theta_nodes(nt: int):
    """theta_j = j*pi/nt with exact polar sin/cos values."""
    th = np.arange(nt + 1) * (math.pi / nt)
    s = np.sin(th)
    c = np.cos(th)
    s[0] = 0.0
    s[nt] = 0.0
    c[0] = 1.0
    c[nt] = -1.0
    return th, s, c


def _sph_basis(th, ph):
    st, ct = np.sin(th), np.cos(th)
    sp, cp = np.sin(ph), np.cos(ph)
    rhat = np.stack([st * cp, st * sp, ct + 0 * sp])
    that = np.stack([ct * cp, ct * sp, -st + 0 * sp])
    phat = np.stack([-sp + 0 * st, cp + 0 * st, 0 * sp + 0 * st])
    return rhat, that, phat


# ----------------------------------------------------------------------------------------------
# analytic vector potentials (Cartesian components at Cartesian points x[3,...])
# ----------------------------------------------------------------------------------------------
@dataclass
class Modes:
    k: np.ndarray      # [5,3]
    u: np.ndarray      # [5,3] unit, orthogonal to k
    phase: np.ndarray  # [5]
    amp: float


def draw_modes(rng: np.random.Generator, amp: float, scale: float, n: int = 5) -> Modes:
    """n smooth Fourier modes: integer wave-vector components in [-3,3] (not all zero) times
    `scale`, a random unit polarisation orthogonal to k, and a random phase."""
    ks, us, ps = [], [], []
    for _ in range(n):
        while True:
            kk = rng.integers(-3, 4, size=3)
            if np.any(kk != 0):
                break
        k = kk.astype(float) * scale
        w = rng.normal(size=3)
        w -= k * (w @ k) / (k @ k)
        w /= np.linalg.norm(w)
        ks.append(k)
        us.append(w)
        ps.append(rng.uniform(0.0, 2.0 * math.pi))
    return Modes(np.array(ks), np.array(us), np.array(ps), amp)


def modes_eval(m: Modes, x: np.ndarray) -> np.ndarray:
    """sum_m amp * u_m * sin(k_m . x + phase_m) at points x[3, ...]."""
    out = np.zeros_like(x)
    ushape = (3,) + (1,) * (x.ndim - 1)
    for k, u, p in zip(m.k, m.u, m.phase):
        s = np.sin(k[0] * x[0] + k[1] * x[1] + k[2] * x[2] + p)
        out += m.amp * u.reshape(ushape) * s[None]
    return out


@dataclass
class Rope:
    centre: np.ndarray   # centre of the axis circle
    normal: np.ndarray   # normal of the plane containing the axis circle
    R: float             # major radius
    a: float             # minor radius
    B0: float
    tau: float


def default_rope() -> Rope:
    # axis circle of radius 0.3 in the plane tangent to r=1.2 at (theta=pi/2, phi=pi)
    c = np.array([-1.2, 0.0, 0.0])
    n = np.array([1.0, 0.0, 0.0])
    b_dip = 1.0 / 1.2 ** 3  # |B| of the unit dipole at r=1.2 on the equator
    return Rope(c, n, 0.3, 0.05, 0.1 * b_dip, 1.0)


def rope_potential(rp: Rope, x: np.ndarray) -> np.ndarray:
    """Localised twisted-rope potential: an azimuthal-around-axis part (B0 d/2) e^{-d^2/a^2}
    whose curl is the axial (toroidal) field B0 (1-d^2/a^2) e^{-d^2/a^2}, plus an axial part
    tau B0 (a^2/2) e^{-d^2/a^2} whose curl is the twist. Zero beyond d = 6a."""
    shp = x.shape[1:]
    X = x.reshape(3, -1)
    y = X - rp.centre[:, None]
    yn = rp.normal @ y
    yp = y - rp.normal[:, None] * yn[None]
    ypl = np.sqrt(np.sum(yp * yp, axis=0))
    out = np.zeros_like(X)
    ok = ypl > 1e-12
    e = np.zeros_like(X)
    e[:, ok] = yp[:, ok] / ypl[ok]
    P = rp.centre[:, None] + rp.R * e
    dv = X - P
    d = np.sqrt(np.sum(dv * dv, axis=0))
    near = ok & (d < 6.0 * rp.a)
    if np.any(near):
        t = np.cross(rp.normal[None, :], e[:, near].T).T        # axis tangent
        dn = d[near]
        rho = np.zeros_like(dv[:, near])
        nz = dn > 1e-14
        rho[:, nz] = dv[:, near][:, nz] / dn[nz]
        psi = np.cross(t.T, rho.T).T                             # azimuth around the axis
        g = np.exp(-dn * dn / (rp.a * rp.a))
        a_psi = rp.B0 * 0.5 * dn * g
        a_ax = rp.tau * rp.B0 * 0.5 * rp.a * rp.a * g
        out[:, near] = psi * a_psi + t * a_ax
    return out.reshape(3, *shp)


def _cart(r, th, ph):
    st = np.sin(th)
    return np.stack([r * st * np.cos(ph), r * st * np.sin(ph), r * np.cos(th) + 0 * ph])


# ----------------------------------------------------------------------------------------------
# magnetic field on faces
# ----------------------------------------------------------------------------------------------
def _edge_integrals_shell(d: GridDesc, r, th, sth, i, kind, pert: Modes | None, rope: Rope | None,
                          dipole: bool, potential=None):
    """Line integrals of A along the edges of one radial index i.
    kind 'r': r-edges (r_i..r_{i+1}) at (theta_j, phi_k), shape [nt+1, np]
    kind 't': theta-edges at (r_i, phi_k), shape [nt, np]
    kind 'p': phi-edges at (r_i, theta_j), shape [nt+1, np]"""
    nt, npp = d.nt, d.np
    dth = math.pi / nt
    dph = 2.0 * math.pi / npp
    phn = np.arange(npp) * dph
    phc = phn + 0.5 * dph
    thc = (np.arange(nt) + 0.5) * dth
    if kind == "r":
        rm = 0.5 * (r[i] + r[i + 1])
        TH, PH = np.meshgrid(th, phn, indexing="ij")
        L = r[i + 1] - r[i]
        st = np.broadcast_to(sth[:, None], TH.shape)
        ct = np.cos(TH)
        ct[0, :] = 1.0
        ct[nt, :] = -1.0
        cp, sp = np.cos(PH), np.sin(PH)
        tang = np.stack([st * cp, st * sp, ct])
        pos = np.stack([rm * st * cp, rm * st * sp, rm * ct])
        a_tan_dip = 0.0
    elif kind == "t":
        TH, PH = np.meshgrid(thc, phn, indexing="ij")
        L = r[i] * dth
        st, ct = np.sin(TH), np.cos(TH)
        cp, sp = np.cos(PH), np.sin(PH)
        tang = np.stack([ct * cp, ct * sp, -st])
        pos = np.stack([r[i] * st * cp, r[i] * st * sp, r[i] * ct])
        a_tan_dip = 0.0
    else:
        TH, PH = np.meshgrid(th, phc, indexing="ij")
        st = np.broadcast_to(sth[:, None], TH.shape)
        ct = np.cos(TH)
        ct[0, :] = 1.0
        ct[nt, :] = -1.0
        L = r[i] * st * dph
        cp, sp = np.cos(PH), np.sin(PH)
        tang = np.stack([-sp, cp, 0.0 * sp])
        pos = np.stack([r[i] * st * cp, r[i] * st * sp, r[i] * ct])
        # unit dipole A_phi = sin(theta)/r^2
        a_tan_dip = st / (r[i] * r[i]) if dipole else 0.0
    a = np.zeros_like(pos)
    if pert is not None:
        a = a + modes_eval(pert, pos)
    if rope is not None:
        a = a + rope_potential(rope, pos)
    if potential is not None:
        a = a + potential(pos)
    at = np.sum(a * tang, axis=0) + a_tan_dip
    return at * L


def magnetic_field(d: GridDesc, pert: Modes | None = None, rope: Rope | None = None,
                   dipole: bool = True, potential=None):
    """Face-averaged B = (flux of A's circulation) / area on the staggered grid. `potential`
    is an optional extra vector potential: a callable taking Cartesian points x[3, ...] and
    returning Cartesian A[3, ...]."""
    nr, nt, npp = d.nr, d.nt, d.np
    r = radial_nodes(d)
    th, sth, cth = theta_nodes(nt)
    dth = math.pi / nt
    dph = 2.0 * math.pi / npp
    br = np.zeros((nr + 1, nt, npp))
    bt = np.zeros((nr, nt + 1, npp))
    bp = np.zeros((nr, nt, npp))
    args = (pert, rope, dipole, potential)
    Lt_next = _edge_integrals_shell(d, r, th, sth, 0, "t", *args)
    Lp_next = _edge_integrals_shell(d, r, th, sth, 0, "p", *args)
    for i in range(nr + 1):
        Lt, Lp = Lt_next, Lp_next
        # radial faces at r_i
        area_r = r[i] ** 2 * (cth[:-1] - cth[1:]) * dph
        flux = Lt + Lp[1:] - np.roll(Lt, -1, axis=1) - Lp[:-1]
        br[i] = flux / area_r[:, None]
        if i == nr:
            break
        Lt_next = _edge_integrals_shell(d, r, th, sth, i + 1, "t", *args)
        Lp_next = _edge_integrals_shell(d, r, th, sth, i + 1, "p", *args)
        Lr = _edge_integrals_shell(d, r, th, sth, i, "r", *args)
        ring = (r[i + 1] ** 2 - r[i] ** 2) * 0.5
        # theta faces (interior j only; polar faces have zero area and stay 0)
        flux_t = Lp + np.roll(Lr, -1, axis=1) - Lp_next - Lr
        area_t = sth[1:nt] * ring * dph
        bt[i, 1:nt] = flux_t[1:nt] / area_t[:, None]
        # phi faces
        flux_p = Lr[:-1] + Lt_next - Lr[1:] - Lt
        area_p = ring * dth
        bp[i] = flux_p / area_p
    return br, bt, bp


def velocity_field(d: GridDesc, modes, ramp: float = 0.1):
    """v = sum of smooth modes (Cartesian), times (1 - exp(-(r-r0)/ramp)), projected on the
    local spherical basis at cell centres. `modes` may also be a callable returning a Cartesian
    vector field at points x[3, ...]."""
    r = radial_nodes(d)
    rc = 0.5 * (r[:-1] + r[1:])
    thc = (np.arange(d.nt) + 0.5) * (math.pi / d.nt)
    phc = (np.arange(d.np) + 0.5) * (2.0 * math.pi / d.np)
    TH, PH = np.meshgrid(thc, phc, indexing="ij")
    rhat, that, phat = _sph_basis(TH, PH)
    vr = np.empty((d.nr, d.nt, d.np))
    vt = np.empty_like(vr)
    vp = np.empty_like(vr)
    for i in range(d.nr):
        pos = rc[i] * rhat
        w = modes(pos) if callable(modes) else modes_eval(modes, pos)
        w = w * (1.0 - math.exp(-(rc[i] - d.r0) / ramp))
        vr[i] = np.sum(w * rhat, axis=0)
        vt[i] = np.sum(w * that, axis=0)
        vp[i] = np.sum(w * phat, axis=0)
    return vr, vt, vp


def initial_state(d: GridDesc, index: int, rope: bool):
    """Dipole + 5-mode perturbation (amp 1e-3) [+ flux rope], and the 1e-2 5-mode velocity.
    Seed: numpy default_rng(1811 + index); B modes drawn first, then v modes."""
    rng = np.random.default_rng(SEED_BASE + index)
    bmodes = draw_modes(rng, 1e-3, 1.0 / d.r1)
    vmodes = draw_modes(rng, 1e-2, 1.0 / d.r1)
    br, bt, bp = magnetic_field(d, bmodes, default_rope() if rope else None)
    vr, vt, vp = velocity_field(d, vmodes)
    return dict(br=br, bt=bt, bp=bp, vr=vr, vt=vt, vp=vp)


def workload(name: str):
    w = WORKLOADS[name]
    return w, initial_state(w["desc"], w["index"], w["rope"])


# ----------------------------------------------------------------------------------------------
# batched solves and adjoint inputs
# ----------------------------------------------------------------------------------------------
def batched_items(n: int = 64, nt_min: int = 32, nt_max: int = 128):
    """Item i (seed 1811*100 + i): nt from {32, 48, ..., 128}, nr = nt, np = 2 nt, r in [1, 20],
    stretch uniform in [1.02, 1.08], and a smooth 5-mode right-hand-side field."""
    items = []
    choices = list(range(nt_min, nt_max + 1, 16))
    for i in range(n):
        rng = np.random.default_rng(SEED_BASE * 100 + i)
        nt = int(rng.choice(choices))
        s = float(rng.uniform(1.02, 1.08))
        desc = GridDesc(nt, nt, 2 * nt, 1.0, 20.0, s)
        modes = draw_modes(rng, 1.0, 1.0 / desc.r1)
        items.append(dict(desc=desc, modes=modes, seed=SEED_BASE * 100 + i))
    return items


def smooth_field(d: GridDesc, modes: Modes):
    """Three-component smooth field at cell centres, shape [3, nr, nt, np] (no ramp)."""
    vr, vt, vp = velocity_field(d, modes, ramp=1e-300)
    return np.stack([vr, vt, vp])


def outer_target(d: GridDesc, seed: int):
    """Smooth seeded target for B_r on the outer shell, shape [nt, np]."""
    rng = np.random.default_rng(seed)
    thc = (np.arange(d.nt) + 0.5) * (math.pi / d.nt)
    phc = (np.arange(d.np) + 0.5) * (2.0 * math.pi / d.np)
    TH, PH = np.meshgrid(thc, phc, indexing="ij")
    out = np.zeros((d.nt, d.np))
    for _ in range(5):
        l = int(rng.integers(1, 4))
        m = int(rng.integers(0, l + 1))
        out += rng.normal() * 1e-4 * np.cos(l * TH) * np.cos(m * PH + rng.uniform(0, 2 * math.pi))
    return out


def unit_direction(shape, seed: int):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=shape)
    return x / np.linalg.norm(x)
