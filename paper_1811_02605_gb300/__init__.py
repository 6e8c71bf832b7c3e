"""Python binding of the sm_103a zero-beta MHD library (include/mhd.h).

Argument marshalling only: every step of the computation runs in the CUDA library libmhd.so,
which must have been built (``paper_1811_02605_gb300.build.build()``); importing the functions
without it raises. Device buffers are torch CUDA float64 tensors (contiguous); the library never
takes ownership of them.

The functions keep the C names:
    mhd_grid_create, mhd_grid_destroy, mhd_grid_sizes, mhd_step_coeffs, mhd_step,
    mhd_apply_operator, mhd_force, mhd_induction, pcg_solve, pcg_solve_batched,
    mhd_adjoint_step, mhd_grid_reserve, pcg_batch_reserve, mhd_last_error
"""
from __future__ import annotations

import ctypes as C
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmhd.so")

MHD_OK, MHD_ERR_ARG, MHD_ERR_CUDA, MHD_ERR_NOCONV, MHD_ERR_NONFINITE, MHD_ERR_TIMEOUT, MHD_ERR_OOM = range(7)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NOCONV", 4: "ERR_NONFINITE",
                5: "ERR_TIMEOUT", 6: "ERR_OOM"}
PREC_FP64, PREC_MIXED = 0, 1
(RESERVE_PC1, RESERVE_MIXED, RESERVE_CG, RESERVE_PC2, RESERVE_RESISTIVITY, RESERVE_ADJOINT,
 RESERVE_ALL) = 1, 2, 4, 8, 16, 32, 63

# C ABI symbols declared in include/mhd.h
SYMBOLS = ["mhd_grid_create", "mhd_grid_destroy", "mhd_grid_sizes", "mhd_step_coeffs", "mhd_step",
           "mhd_apply_operator", "mhd_force", "mhd_induction", "pcg_solve", "pcg_solve_batched",
           "mhd_adjoint_step", "mhd_force_noalloc", "mhd_grid_reserve", "pcg_batch_reserve",
           "mhd_grid_create_slab", "mhd_slab_apply", "mhd_slab_update", "mhd_slab_pupdate", "mhd_diagnostics",
           "mhd_profile_enable", "mhd_profile_read", "mhd_grid_kernel_forms", "mhd_last_error"]

KERNELS = ["pupdate64", "spmv64", "update64", "pupdate32", "spmv32", "update32", "outer_res", "force",
           "induction", "coeffs", "sts", "res", "pc2", "pspmv32", "pfold32", "rupd32", "cgr32", "cgu32"]


class GridDesc(C.Structure):
    _fields_ = [("nr", C.c_int), ("nt", C.c_int), ("np", C.c_int),
                ("r0", C.c_double), ("r1", C.c_double), ("stretch", C.c_double)]


class Params(C.Structure):
    _fields_ = [("nu", C.c_double), ("eta", C.c_double), ("cfl", C.c_double),
                ("dt_fixed", C.c_double), ("dt_max", C.c_double), ("alpha_si_fixed", C.c_double),
                ("tol", C.c_double), ("inner_tol", C.c_double),
                ("max_iter", C.c_int), ("max_outer", C.c_int), ("precision", C.c_int),
                ("mixed_restart", C.c_int), ("viscosity_sts", C.c_int), ("pcg_variant", C.c_int),
                ("resistivity_implicit", C.c_int), ("preconditioner", C.c_int)]


class Fields(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("br", "bt", "bp", "vr", "vt", "vp")]


class StepInfo(C.Structure):
    _fields_ = [("dt", C.c_double), ("cf", C.c_double), ("cw", C.c_double),
                ("alpha_si", C.c_double), ("alpha_nu", C.c_double),
                ("iters", C.c_int * 3), ("outer", C.c_int * 3), ("relres", C.c_double * 3),
                ("iters_res", C.c_int), ("relres_res", C.c_double)]

    def as_dict(self):
        return dict(dt=self.dt, cf=self.cf, cw=self.cw, alpha_si=self.alpha_si, alpha_nu=self.alpha_nu,
                    iters=list(self.iters), outer=list(self.outer), relres=list(self.relres),
                    iters_res=self.iters_res, relres_res=self.relres_res)


class MhdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def lib():
    """Load libmhd.so; raises if the CUDA library has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run "
                                   "paper_1811_02605_gb300.build.build() first")
            L = C.CDLL(LIB_PATH)
            vp, i, d = C.c_void_p, C.c_int, C.c_double
            L.mhd_grid_create.argtypes = [C.POINTER(GridDesc), vp, C.POINTER(vp)]
            L.mhd_grid_destroy.argtypes = [vp]
            L.mhd_grid_sizes.argtypes = [vp, C.POINTER(C.c_longlong)]
            L.mhd_step_coeffs.argtypes = [vp, C.POINTER(Params), C.POINTER(Fields), C.POINTER(StepInfo)]
            L.mhd_step.argtypes = [vp, C.POINTER(Params), C.POINTER(Fields), C.POINTER(StepInfo)]
            L.mhd_apply_operator.argtypes = [vp, d, i, vp, vp]
            L.mhd_force.argtypes = [vp, C.POINTER(Fields), d, vp]
            L.mhd_induction.argtypes = [vp, vp, d, d, C.POINTER(Fields)]
            L.pcg_solve.argtypes = [vp, d, i, vp, vp, C.POINTER(Params), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int), C.POINTER(C.c_double)]
            L.pcg_solve_batched.argtypes = [i, C.POINTER(vp), C.POINTER(C.c_double), C.POINTER(vp),
                                            C.POINTER(vp), C.POINTER(Params), C.POINTER(C.c_int),
                                            C.POINTER(C.c_double)]
            L.mhd_adjoint_step.argtypes = [vp, C.POINTER(Params), C.POINTER(Fields), d,
                                           C.POINTER(Fields), C.POINTER(Fields)]
            L.mhd_force_noalloc.argtypes = [C.POINTER(GridDesc), C.POINTER(Fields), d, vp, vp]
            L.mhd_grid_reserve.argtypes = [vp, i]
            L.mhd_diagnostics.argtypes = [vp, C.POINTER(Fields), C.POINTER(C.c_double)]
            L.mhd_grid_create_slab.argtypes = [C.POINTER(GridDesc), i, i, vp, C.POINTER(vp)]
            L.mhd_slab_apply.argtypes = [vp, d, i, vp, vp, vp, vp, C.POINTER(C.c_double)]
            L.mhd_slab_update.argtypes = [vp, d, i, d, vp, vp, vp, vp, vp, C.POINTER(C.c_double)]
            L.mhd_slab_pupdate.argtypes = [vp, i, d, vp, vp]
            L.pcg_batch_reserve.argtypes = [i, C.POINTER(vp), C.POINTER(C.c_double), C.POINTER(vp), C.POINTER(vp),
                                            C.POINTER(Params)]
            L.mhd_profile_enable.argtypes = [vp, i]
            L.mhd_profile_read.argtypes = [vp, i, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
            L.mhd_grid_kernel_forms.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.mhd_last_error.argtypes = [vp]
            L.mhd_last_error.restype = C.c_char_p
            for name in SYMBOLS:
                if name != "mhd_last_error":
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _ptr(t, what="tensor"):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch tensor")
    if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous float64 CUDA tensor (got {t.dtype} on {t.device})")
    return C.c_void_p(t.data_ptr())


def mhd_last_error(grid=None) -> str:
    h = grid.handle if isinstance(grid, Grid) else grid
    s = lib().mhd_last_error(h)
    return s.decode() if s else ""


def _check(st, grid=None, soft=(MHD_OK,)):
    if st not in soft:
        raise MhdError(st, mhd_last_error(grid))
    return st


def make_params(nu=1e-3, eta=0.0, cfl=0.4, dt_fixed=0.0, dt_max=0.0, alpha_si_fixed=-1.0, tol=1e-9,
                inner_tol=1e-5, max_iter=100000, max_outer=30, precision=PREC_FP64,
                mixed_restart=0, viscosity_sts=0, pcg_variant=0, resistivity_implicit=0,
                preconditioner=0) -> Params:
    return Params(nu, eta, cfl, dt_fixed, dt_max, alpha_si_fixed, tol, inner_tol, max_iter, max_outer,
                  precision, mixed_restart, viscosity_sts, pcg_variant, resistivity_implicit, preconditioner)


def make_fields(br, bt, bp, vr=None, vt=None, vp=None) -> Fields:
    f = Fields()
    f.br, f.bt, f.bp = (_ptr(br, "br").value, _ptr(bt, "bt").value, _ptr(bp, "bp").value)
    if vr is not None:
        f.vr, f.vt, f.vp = (_ptr(vr, "vr").value, _ptr(vt, "vt").value, _ptr(vp, "vp").value)
    return f


class Grid:
    """Owner of an mhd_grid_t handle (destroyed with the object)."""

    def __init__(self, handle, desc):
        self.handle = handle
        self.desc = desc

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            try:
                lib().mhd_grid_destroy(h)
            except Exception:
                pass
            self.handle = None

    @property
    def shapes(self):
        nr, nt, n = self.desc.nr, self.desc.nt, self.desc.np
        return dict(br=(nr + 1, nt, n), bt=(nr, nt + 1, n), bp=(nr, nt, n), v=(3, nr, nt, n))


def mhd_grid_create(nr, nt, np_, r0, r1, stretch, stream=None) -> Grid:
    """stream: a torch.cuda.Stream, an integer cudaStream_t, or None for torch's current stream."""
    import torch
    if stream is None:
        s = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        s = stream.cuda_stream
    else:
        s = int(stream)
    d = GridDesc(nr, nt, np_, r0, r1, stretch)
    h = C.c_void_p()
    _check(lib().mhd_grid_create(C.byref(d), C.c_void_p(s), C.byref(h)))
    return Grid(h, d)


def mhd_grid_create_slab(nr, nt, np_, r0, r1, stretch, i0, i1, stream=None) -> Grid:
    """Radial rows [i0, i1) of the grid (nr, nt, np_, r0, r1, stretch); see include/mhd.h. The
    returned Grid's desc is the slab's own (nr = i1 - i0)."""
    import torch
    if stream is None:
        s = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        s = stream.cuda_stream
    else:
        s = int(stream)
    d = GridDesc(nr, nt, np_, r0, r1, stretch)
    h = C.c_void_p()
    _check(lib().mhd_grid_create_slab(C.byref(d), int(i0), int(i1), C.c_void_p(s), C.byref(h)))
    return Grid(h, GridDesc(i1 - i0, nt, np_, r0, r1, stretch))


def mhd_slab_apply(grid: Grid, alpha: float, p, p_lo, p_hi, q) -> float:
    """q = M_alpha p on the slab (ghost planes p_lo, p_hi or None); returns the slab's <p, q>."""
    nc = p.numel() // (grid.desc.nr * grid.desc.nt * grid.desc.np)
    pq = C.c_double(0)
    _check(lib().mhd_slab_apply(grid.handle, float(alpha), nc, _ptr(p, "p"),
                                None if p_lo is None else _ptr(p_lo, "p_lo"),
                                None if p_hi is None else _ptr(p_hi, "p_hi"), _ptr(q, "q"), C.byref(pq)), grid)
    return pq.value


def mhd_slab_update(grid: Grid, alpha: float, a: float, x, p, r, q, z):
    """x += a p (x may be None), r -= a q, z = r / diag; returns the slab's (<r, z>, <r, r>)."""
    nc = r.numel() // (grid.desc.nr * grid.desc.nt * grid.desc.np)
    dots = (C.c_double * 2)()
    _check(lib().mhd_slab_update(grid.handle, float(alpha), nc, float(a), None if x is None else _ptr(x, "x"),
                                 None if p is None else _ptr(p, "p"), _ptr(r, "r"), _ptr(q, "q"), _ptr(z, "z"),
                                 dots), grid)
    return dots[0], dots[1]


def mhd_slab_pupdate(grid: Grid, beta: float, z, p):
    nc = z.numel() // (grid.desc.nr * grid.desc.nt * grid.desc.np)
    _check(lib().mhd_slab_pupdate(grid.handle, nc, float(beta), _ptr(z, "z"), _ptr(p, "p")), grid)


def mhd_grid_destroy(grid: Grid):
    if grid.handle:
        _check(lib().mhd_grid_destroy(grid.handle))
        grid.handle = None


def mhd_grid_sizes(grid: Grid):
    a = (C.c_longlong * 6)()
    _check(lib().mhd_grid_sizes(grid.handle, a), grid)
    return list(a)


def mhd_step_coeffs(grid: Grid, params: Params, fields: Fields) -> dict:
    info = StepInfo()
    _check(lib().mhd_step_coeffs(grid.handle, C.byref(params), C.byref(fields), C.byref(info)), grid)
    return info.as_dict()


def mhd_step(grid: Grid, params: Params, fields: Fields):
    """One step in place; returns (status, info dict). Raises on argument/CUDA errors."""
    info = StepInfo()
    st = lib().mhd_step(grid.handle, C.byref(params), C.byref(fields), C.byref(info))
    _check(st, grid, soft=(MHD_OK, MHD_ERR_NOCONV, MHD_ERR_NONFINITE))
    return st, info.as_dict()


def mhd_apply_operator(grid: Grid, alpha: float, p, q):
    nc = p.numel() // (grid.desc.nr * grid.desc.nt * grid.desc.np)
    _check(lib().mhd_apply_operator(grid.handle, float(alpha), nc, _ptr(p, "p"), _ptr(q, "q")), grid)


def mhd_force(grid: Grid, fields: Fields, dt: float, b):
    _check(lib().mhd_force(grid.handle, C.byref(fields), float(dt), _ptr(b, "b")), grid)


def mhd_induction(grid: Grid, vbar, eta: float, dt: float, fields: Fields):
    _check(lib().mhd_induction(grid.handle, _ptr(vbar, "vbar"), float(eta), float(dt), C.byref(fields)), grid)


def pcg_solve(grid: Grid, alpha: float, b, x, params: Params):
    """Solve M_alpha x = b in place on x (x holds x0). Returns (status, iters, outer, relres)."""
    nc = b.numel() // (grid.desc.nr * grid.desc.nt * grid.desc.np)
    it, ou, rr = C.c_int(0), C.c_int(0), C.c_double(0)
    st = lib().pcg_solve(grid.handle, float(alpha), nc, _ptr(b, "b"), _ptr(x, "x"), C.byref(params),
                         C.byref(it), C.byref(ou), C.byref(rr))
    _check(st, grid, soft=(MHD_OK, MHD_ERR_NOCONV, MHD_ERR_NONFINITE))
    return st, it.value, ou.value, rr.value


def pcg_solve_batched(grids, alphas, bs, xs, params: Params):
    """Batched solves; returns (status, iters list, relres list)."""
    n = len(grids)
    hs = (C.c_void_p * n)(*[g.handle.value if hasattr(g.handle, "value") else g.handle for g in grids])
    al = (C.c_double * n)(*[float(a) for a in alphas])
    bp = (C.c_void_p * n)(*[_ptr(b, "b").value for b in bs])
    xp = (C.c_void_p * n)(*[_ptr(x, "x").value for x in xs])
    it = (C.c_int * n)()
    rr = (C.c_double * n)()
    st = lib().pcg_solve_batched(n, hs, al, bp, xp, C.byref(params), it, rr)
    _check(st, None, soft=(MHD_OK, MHD_ERR_NOCONV, MHD_ERR_NONFINITE))
    return st, list(it), list(rr)


def mhd_adjoint_step(grid: Grid, params: Params, state_n: Fields, dt: float, adj_np1: Fields, adj_n: Fields):
    st = lib().mhd_adjoint_step(grid.handle, C.byref(params), C.byref(state_n), float(dt), C.byref(adj_np1),
                                C.byref(adj_n))
    _check(st, grid, soft=(MHD_OK, MHD_ERR_NOCONV, MHD_ERR_NONFINITE))
    return st


def mhd_diagnostics(grid: Grid, fields: Fields) -> dict:
    """Magnetic and kinetic energy, int |J x B| dV, int |J . B| dV, max |div_h B| (include/mhd.h)."""
    o = (C.c_double * 5)()
    _check(lib().mhd_diagnostics(grid.handle, C.byref(fields), o), grid)
    return dict(magnetic_energy=o[0], kinetic_energy=o[1], int_jxb=o[2], int_jdotb=o[3], max_divb=o[4])


def mhd_grid_reserve(grid: Grid, features: int = RESERVE_ALL):
    """Allocate now what the named features would allocate on first use (see include/mhd.h)."""
    _check(lib().mhd_grid_reserve(grid.handle, int(features)), grid)


def pcg_batch_reserve(grids, alphas, bs, xs, params: Params):
    """Build the plan and graph of this batch for pcg_solve_batched (solves nothing)."""
    n = len(grids)
    hs = (C.c_void_p * n)(*[g.handle.value if hasattr(g.handle, "value") else g.handle for g in grids])
    al = (C.c_double * n)(*[float(a) for a in alphas])
    bp = (C.c_void_p * n)(*[_ptr(b, "b").value for b in bs])
    xp = (C.c_void_p * n)(*[_ptr(x, "x").value for x in xs])
    _check(lib().pcg_batch_reserve(n, hs, al, bp, xp, C.byref(params)), None)


def mhd_profile_enable(grid: Grid, enable: bool = True):
    _check(lib().mhd_profile_enable(grid.handle, 1 if enable else 0), grid)


def mhd_profile_read(grid: Grid) -> dict:
    """{kernel name: (total_ms, launches)} since profiling was enabled."""
    out = {}
    for k, name in enumerate(KERNELS):
        ms, n = C.c_double(0), C.c_longlong(0)
        _check(lib().mhd_profile_read(grid.handle, k, C.byref(ms), C.byref(n)), grid)
        out[name] = (ms.value, n.value)
    return out


def mhd_grid_kernel_forms(grid: Grid) -> tuple[int, int]:
    """(fp64_form, fp32_form): the autotuner's choices in the codes of MHD_FORCE_SLAB (0: not tuned)."""
    a, b = C.c_int(0), C.c_int(0)
    _check(lib().mhd_grid_kernel_forms(grid.handle, C.byref(a), C.byref(b)), grid)
    return a.value, b.value


def mhd_force_noalloc(desc: GridDesc, fields: Fields, dt: float, b, stream=None):
    """Momentum force without a grid object and without any device allocation (scratch lives in
    a static device array of the library; see include/mhd.h). Returns the status code."""
    import torch
    if stream is None:
        s = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        s = stream.cuda_stream
    else:
        s = int(stream)
    st = lib().mhd_force_noalloc(C.byref(desc), C.byref(fields), float(dt), _ptr(b, "b"), C.c_void_p(s))
    return st
