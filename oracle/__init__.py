"""ctypes binding of the plain FP64 CPU oracle (mhd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the package's smoke check and the
benchmark's CPU-baseline leg. The CUDA library never imports or links it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.c")
_SO = os.path.join(_HERE, "_build", "libmhd_oracle.so")
_SO_OMP = os.path.join(_HERE, "_build", "libmhd_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

OK, ERR_ARG, ERR_NOCONV = 0, 1, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no fused multiply-add)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mhd_oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def build_omp(force: bool = False) -> str:
    """The timing build: the same source with -fopenmp (the benchmark's CPU baseline on all host
    cores). The default build above stays plain sequential C."""
    os.makedirs(os.path.dirname(_SO_OMP), exist_ok=True)
    if force or not os.path.exists(_SO_OMP) or os.path.getmtime(_SO_OMP) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mhd_oracle.h"))):
        tmp = _SO_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO_OMP)
    return _SO_OMP


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def lib_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            _lib_omp = C.CDLL(build_omp())
            _declare(_lib_omp)
    return _lib_omp


def set_threads(n: int = 0, omp: bool = True) -> int:
    """Threads of the timing build (n > 0 sets them); returns the count in use (1: plain build)."""
    L = lib_omp() if omp else lib()
    return int(L.og_set_threads(int(n)))


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _declare(L):
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    L.og_set_threads.restype = i
    L.og_set_threads.argtypes = [i]
    L.og_create.restype = vp
    L.og_create.argtypes = [i, i, i, d, d, d]
    L.og_destroy.argtypes = [vp]
    for name in ("og_radial_nodes", "og_volumes", "og_ktilde2"):
        getattr(L, name).argtypes = [vp, _dp]
    L.og_dot.restype = d
    L.og_dot.argtypes = [C.c_longlong, _dp, _dp]
    L.og_apply_M.argtypes = [vp, d, i, _dp, _dp]
    L.og_apply_K_neumann.argtypes = [vp, i, _dp, _dp]
    L.og_diag.argtypes = [vp, d, _dp]
    L.og_pcg.restype = i
    L.og_pcg.argtypes = [vp, d, i, _dp, _dp, d, i, i, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.og_pcg_cg.restype = i
    L.og_pcg_cg.argtypes = L.og_pcg.argtypes
    L.og_coeffs.restype = i
    L.og_coeffs.argtypes = [vp, d, d, d, d, d, _dp, _dp, _dp, _dp, _dp]
    L.og_bcentre.argtypes = [vp, _dp, _dp, _dp, _dp]
    L.og_current_edges.argtypes = [vp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.og_current_centre.argtypes = [vp, _dp, _dp, _dp, _dp]
    L.og_force.argtypes = [vp, _dp, _dp, _dp, _dp, d, _dp]
    L.og_efield_edges.argtypes = [vp, _dp, _dp, _dp, _dp, d, _dp, _dp, _dp]
    L.og_ct.argtypes = [vp, _dp, _dp, _dp, d, _dp, _dp, _dp]
    L.og_divb.argtypes = [vp, _dp, _dp, _dp, _dp]
    L.og_diagnostics.argtypes = [vp, _dp, _dp, _dp, _dp, _dp]
    L.og_step.restype = i
    L.og_step.argtypes = [vp, d, d, d, d, d, d, d, i, _dp, _dp, _dp, _dp, _dp]
    L.og_step_cg.restype = i
    L.og_step_cg.argtypes = L.og_step.argtypes
    L.og_step_opts.restype = i
    L.og_step_opts.argtypes = [vp, i, d, d, d, d, d, d, d, i, _dp, _dp, _dp, _dp, _dp]
    L.og_ilu0.restype = i
    L.og_ilu0.argtypes = [vp, d, i, _dp]
    L.og_ilu0_apply.argtypes = [vp, d, i, _dp, i, _dp, _dp]
    L.og_pcg_pc2.restype = i
    L.og_pcg_pc2.argtypes = [vp, d, i, i, _dp, _dp, d, i, i, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.og_res_size.restype = C.c_longlong
    L.og_res_size.argtypes = [vp]
    L.og_res_current.argtypes = [vp] + [_dp] * 6
    L.og_res_apply.argtypes = [vp, d, _dp, _dp]
    L.og_res_diag.argtypes = [vp, d, _dp]
    L.og_res_pcg.restype = i
    L.og_res_pcg.argtypes = [vp, d, _dp, _dp, d, i, i, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.og_res_solve.restype = i
    L.og_res_solve.argtypes = [vp, d, _dp, _dp, _dp, d, i, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    if hasattr(L, "og_adjoint_step"):
        L.og_adjoint_step.restype = i
        L.og_adjoint_step.argtypes = [vp, d, d, d, d, d, d, i] + [_dp] * 12
        L.og_adjoint_step_sts.restype = i
        L.og_adjoint_step_sts.argtypes = [vp, d, d, d, d, d, d, i] + [_dp] * 12
        L.og_adjoint_step_opts.restype = i
        L.og_adjoint_step_opts.argtypes = [vp, i, d, d, d, d, d, d, i] + [_dp] * 12
        L.og_rkl2_stages.restype = i
        L.og_rkl2_stages.argtypes = [vp, d, d]
        L.og_rkl2.restype = i
        L.og_rkl2.argtypes = [vp, d, d, i, _dp]
        L.og_step_sts.restype = i
        L.og_step_sts.argtypes = [vp] + [d] * 7 + [i] + [_dp] * 5


OPT_PCG_CG, OPT_STS, OPT_RES_IMPLICIT, OPT_PC2 = 1, 2, 4, 8


def _blocks(name):
    return {"whole": 0, "lines": 1}[name]


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def dot(a, b):
    """The oracle's inner product (compensated, as in every PCG of the oracle)."""
    a, b = _c(a).ravel(), _c(b).ravel()
    assert a.size == b.size
    return lib().og_dot(a.size, a, b)


class Grid:
    """Oracle grid: nr x nt x np cells, r in [r0, r1] with geometric stretch."""

    def __init__(self, nr, nt, np_, r0, r1, stretch, omp=False):
        self.L = lib_omp() if omp else lib()
        self.h = self.L.og_create(nr, nt, np_, r0, r1, stretch)
        if not self.h:
            raise ValueError("bad grid")
        self.nr, self.nt, self.np = nr, nt, np_
        self.N = nr * nt * np_
        self.r0, self.r1, self.stretch = r0, r1, stretch

    @classmethod
    def from_desc(cls, d, omp=False):
        return cls(d.nr, d.nt, d.np, d.r0, d.r1, d.stretch, omp=omp)

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.og_destroy(h)
            self.h = None

    # shapes
    @property
    def shapes(self):
        nr, nt, n = self.nr, self.nt, self.np
        return dict(br=(nr + 1, nt, n), bt=(nr, nt + 1, n), bp=(nr, nt, n),
                    er=(nr, nt + 1, n), et=(nr + 1, nt, n), ep=(nr + 1, nt + 1, n))

    def radial_nodes(self):
        o = np.empty(self.nr + 1)
        self.L.og_radial_nodes(self.h, o)
        return o

    def volumes(self):
        o = np.empty((self.nr, self.nt))
        self.L.og_volumes(self.h, o)
        return o

    def ktilde2(self):
        o = np.empty((self.nr, self.nt))
        self.L.og_ktilde2(self.h, o)
        return o

    def apply_M(self, alpha, p):
        p = _c(p)
        nc = p.size // self.N
        q = np.empty_like(p)
        self.L.og_apply_M(self.h, alpha, nc, p, q)
        return q

    def apply_K_neumann(self, p):
        p = _c(p)
        q = np.empty_like(p)
        self.L.og_apply_K_neumann(self.h, p.size // self.N, p, q)
        return q

    def diag(self, alpha):
        o = np.empty((self.nr, self.nt))
        self.L.og_diag(self.h, alpha, o)
        return o

    def pcg(self, alpha, b, x0=None, tol=1e-9, max_iter=100000, fixed_iters=0, cg=False, pc2=None):
        """Jacobi PCG; cg=True: the single-reduction (Chronopoulos-Gear) form; pc2="lines" or
        "whole": PCG with the block-Jacobi ILU(0) preconditioner PC2 (phi-line blocks or one
        block)."""
        b = _c(b)
        x = np.zeros_like(b) if x0 is None else _c(x0).copy()
        it = C.c_int(0)
        rr = C.c_double(0)
        if pc2 is not None:
            st = self.L.og_pcg_pc2(self.h, alpha, _blocks(pc2), b.size // self.N, b, x, tol, max_iter, fixed_iters,
                                   C.byref(it), C.byref(rr))
            return x, it.value, rr.value, st
        fn = self.L.og_pcg_cg if cg else self.L.og_pcg
        st = fn(self.h, alpha, b.size // self.N, b, x, tol, max_iter, fixed_iters, C.byref(it), C.byref(rr))
        return x, it.value, rr.value, st

    def coeffs(self, v, br, bt, bp, nu=1e-3, cfl=0.4, dt_fixed=0.0, dt_max=0.0, asi_fixed=-1.0):
        o = np.empty(5)
        st = self.L.og_coeffs(self.h, nu, cfl, dt_fixed, dt_max, asi_fixed, _c(v), _c(br), _c(bt),
                              _c(bp), o)
        if st != OK:
            raise ValueError(f"og_coeffs status {st}")
        return dict(dt=o[0], cf=o[1], cw=o[2], alpha_si=o[3], alpha_nu=o[4])

    def bcentre(self, br, bt, bp):
        o = np.empty((3, self.nr, self.nt, self.np))
        self.L.og_bcentre(self.h, _c(br), _c(bt), _c(bp), o)
        return o

    def current_edges(self, br, bt, bp):
        s = self.shapes
        jr, jt, jp = np.empty(s["er"]), np.empty(s["et"]), np.empty(s["ep"])
        self.L.og_current_edges(self.h, _c(br), _c(bt), _c(bp), jr, jt, jp)
        return jr, jt, jp

    def current_centre(self, br, bt, bp):
        o = np.empty((3, self.nr, self.nt, self.np))
        self.L.og_current_centre(self.h, _c(br), _c(bt), _c(bp), o)
        return o

    def force(self, v, br, bt, bp, dt):
        o = np.empty((3, self.nr, self.nt, self.np))
        self.L.og_force(self.h, _c(v), _c(br), _c(bt), _c(bp), dt, o)
        return o

    def efield_edges(self, vbar, br, bt, bp, eta=0.0):
        s = self.shapes
        er, et, ep = np.empty(s["er"]), np.empty(s["et"]), np.empty(s["ep"])
        self.L.og_efield_edges(self.h, _c(vbar), _c(br), _c(bt), _c(bp), eta, er, et, ep)
        return er, et, ep

    def ct(self, er, et, ep, dt, br, bt, bp):
        br, bt, bp = _c(br).copy(), _c(bt).copy(), _c(bp).copy()
        self.L.og_ct(self.h, _c(er), _c(et), _c(ep), dt, br, bt, bp)
        return br, bt, bp

    def divb(self, br, bt, bp):
        o = np.empty((self.nr, self.nt, self.np))
        self.L.og_divb(self.h, _c(br), _c(bt), _c(bp), o)
        return o

    def step(self, state, nu=1e-3, eta=0.0, cfl=0.4, dt_fixed=0.0, dt_max=0.0, asi_fixed=-1.0,
             tol=1e-9, max_iter=100000, cg=False, sts=False, res_implicit=False, pc2=False):
        """One step on a copy of `state` (dict br, bt, bp, vr, vt, vp). Returns (new, info).
        cg: every solve in the single-reduction PCG form; sts: viscosity by RKL2 (iters[2] =
        stages); res_implicit: resistivity by the implicit face solve (info res_iters, res_relres);
        pc2: every cell solve with the phi-line block-Jacobi ILU(0) preconditioner."""
        v = np.ascontiguousarray(np.stack([state["vr"], state["vt"], state["vp"]]), dtype=np.float64)
        br, bt, bp = _c(state["br"]).copy(), _c(state["bt"]).copy(), _c(state["bp"]).copy()
        info = np.zeros(13)
        opts = ((OPT_PCG_CG if cg else 0) | (OPT_STS if sts else 0) | (OPT_RES_IMPLICIT if res_implicit else 0) |
                (OPT_PC2 if pc2 else 0))
        st = self.L.og_step_opts(self.h, opts, nu, eta, cfl, dt_fixed, dt_max, asi_fixed, tol, max_iter, v, br,
                                 bt, bp, info)
        out = dict(br=br, bt=bt, bp=bp, vr=v[0].copy(), vt=v[1].copy(), vp=v[2].copy())
        inf = dict(status=st, dt=info[0], cf=info[1], cw=info[2], alpha_si=info[3],
                   alpha_nu=info[4], iters=[int(info[5]), int(info[6]), int(info[7])],
                   relres=list(info[8:11]))
        if res_implicit:
            inf["res_iters"], inf["res_relres"] = int(info[11]), float(info[12])
        return out, inf

    def ilu0(self, alpha, blocks="lines"):
        """modified diagonal of the ILU(0) factorisation of M_alpha, shape (nr, nt, np)"""
        o = np.empty((self.nr, self.nt, self.np))
        st = self.L.og_ilu0(self.h, alpha, _blocks(blocks), o)
        return o, st

    def ilu0_apply(self, alpha, dt, r, blocks="lines"):
        r = _c(r)
        z = np.empty_like(r)
        self.L.og_ilu0_apply(self.h, alpha, _blocks(blocks), _c(dt), r.size // self.N, r, z)
        return z

    # implicit resistivity: stacked face vectors [br | bt | bp]
    @property
    def res_size(self):
        return int(self.L.og_res_size(self.h))

    def res_split(self, x):
        s = self.shapes
        nbr, nbt = int(np.prod(s["br"])), int(np.prod(s["bt"]))
        return (x[:nbr].reshape(s["br"]), x[nbr:nbr + nbt].reshape(s["bt"]), x[nbr + nbt:].reshape(s["bp"]))

    def res_stack(self, br, bt, bp):
        return np.concatenate([_c(br).ravel(), _c(bt).ravel(), _c(bp).ravel()])

    def res_current(self, br, bt, bp):
        s = self.shapes
        jr, jt, jp = np.empty(s["er"]), np.empty(s["et"]), np.empty(s["ep"])
        self.L.og_res_current(self.h, _c(br), _c(bt), _c(bp), jr, jt, jp)
        return jr, jt, jp

    def res_apply(self, dte, x):
        y = np.empty(self.res_size)
        self.L.og_res_apply(self.h, dte, _c(x), y)
        return y

    def res_diag(self, dte):
        y = np.empty(self.res_size)
        self.L.og_res_diag(self.h, dte, y)
        return y

    def res_pcg(self, dte, b, x0=None, tol=1e-9, max_iter=100000, fixed_iters=0):
        b = _c(b)
        x = np.zeros_like(b) if x0 is None else _c(x0).copy()
        it, rr = C.c_int(0), C.c_double(0)
        st = self.L.og_res_pcg(self.h, dte, b, x, tol, max_iter, fixed_iters, C.byref(it), C.byref(rr))
        return x, it.value, rr.value, st

    def res_solve(self, dte, br, bt, bp, tol=1e-9, max_iter=100000):
        br, bt, bp = _c(br).copy(), _c(bt).copy(), _c(bp).copy()
        it, rr = C.c_int(0), C.c_double(0)
        st = self.L.og_res_solve(self.h, dte, br, bt, bp, tol, max_iter, C.byref(it), C.byref(rr))
        return (br, bt, bp), it.value, rr.value, st


def _adjoint(self, state, lam, dt, asi, nu=1e-3, eta=0.0, cfl=0.4, tol=1e-13, max_iter=200000, sts=False,
             res_implicit=False):
    """Cotangent of state n from the cotangent `lam` of state n+1 (dicts with br, bt, bp, vr, vt, vp).
    sts / res_implicit: adjoint of the step with viscosity by RKL2 / resistivity by the implicit
    face solve."""
    v = np.ascontiguousarray(np.stack([state["vr"], state["vt"], state["vp"]]), dtype=np.float64)
    lv1 = np.ascontiguousarray(np.stack([lam["vr"], lam["vt"], lam["vp"]]), dtype=np.float64)
    s = self.shapes
    lv = np.empty_like(v)
    lbr, lbt, lbp = np.empty(s["br"]), np.empty(s["bt"]), np.empty(s["bp"])
    opts = (OPT_STS if sts else 0) | (OPT_RES_IMPLICIT if res_implicit else 0)
    st = self.L.og_adjoint_step_opts(self.h, opts, nu, eta, cfl, dt, asi, tol, max_iter, v, _c(state["br"]),
                                     _c(state["bt"]), _c(state["bp"]), lv1, _c(lam["br"]), _c(lam["bt"]),
                                     _c(lam["bp"]), lv, lbr, lbt, lbp)
    out = dict(br=lbr, bt=lbt, bp=lbp, vr=lv[0].copy(), vt=lv[1].copy(), vp=lv[2].copy())
    return out, st


Grid.adjoint_step = _adjoint


def _diagnostics(self, state):
    """dict: magnetic and kinetic energy, int |J x B| dV, int |J . B| dV, max |div_h B|."""
    v = np.ascontiguousarray(np.stack([state["vr"], state["vt"], state["vp"]]), dtype=np.float64)
    o = np.empty(5)
    self.L.og_diagnostics(self.h, v, _c(state["br"]), _c(state["bt"]), _c(state["bp"]), o)
    return dict(magnetic_energy=o[0], kinetic_energy=o[1], int_jxb=o[2], int_jdotb=o[3], max_divb=o[4])


Grid.diagnostics = _diagnostics


def _rkl2_stages(self, nu, dt):
    return self.L.og_rkl2_stages(self.h, nu, dt)


def _rkl2(self, v, nu, dt, stages=0):
    """v [3, nr, nt, np] advanced over dt by RKL2 super time-stepping; returns (v_new, stages)."""
    x = _c(v).copy()
    s = self.L.og_rkl2(self.h, nu, dt, stages, x)
    return x, s


def _step_sts(self, state, **kw):
    """step with the viscous PCG solve replaced by RKL2 (info iters[2] = stage count)."""
    return self.step(state, sts=True, **kw)


Grid.step_sts = _step_sts
Grid.rkl2_stages = _rkl2_stages
Grid.rkl2 = _rkl2
