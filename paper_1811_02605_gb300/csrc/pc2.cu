// PC2 (Sec. 2.2): PCG with a block-Jacobi preconditioner that uses a zero-fill incomplete LU
// factorisation (ILU(0)) in each block. The blocks are the periodic phi lines (i, j) of each
// component: the r and theta couplings are left out of the preconditioner, so every line is an
// independent block (nr nt of them per component) instead of one block per MPI rank as in the
// paper. For a periodic tridiagonal block zero fill changes only the diagonal:
//     dt_0 = m,  dt_k = m - w^2 / dt_{k-1},  dt_{np-1} -= w^2 / dt_0,
// m the diagonal on the line and -w its phi coupling, and P = (dt + L) dt^-1 (dt + U).
//
// The solve runs on the Jacobi-scaled system A~ = S M S (S = diag(M)^-1/2, unit diagonal, the
// PC1 path's tables and stencil kernels), whose ILU(0) is S ILU(0)(M) S: the same iterates as PCG
// with PC2 on M, in exact arithmetic. On a line of A~: m = 1 and w = the scaled phi coefficient.
//
// z = P^-1 r is a forward and a backward substitution along each line, both first-order linear
// recurrences u_k = a_k u_{k-1} + b_k, which one warp per line evaluates as an affine scan: each
// lane composes the maps of its segment of ceil(np/32) elements, a five-step shuffle scan composes
// the segments, and each lane replays its segment from the value entering it. The multipliers
// (a_k = w / dt_k) do not depend on the component, so their segment products and the scan's
// per-step multipliers are formed once per line and reused by the three components; per
// component only the additive parts are scanned. The periodic wrap enters as u_0 in the last
// forward step and as z_{np-1} in the first backward one, both known before the replays.
//
// FP64 solves use the line kernel in double; the mixed-precision inner solves use it in float
// (vectors, factor and scans in FP32; each lane's dot partials over one line, at most 3 np / 32
// products, are formed in FP32 and summed over lines in FP64),
// with the FP64 outer residual of the reliable-update scheme followed by one preconditioner pass
// that recomputes z and <r, z> for the replaced residual.
#include <cmath>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

enum { kIter = 0, kInit = 1, kReliable = 2 };

struct Pc2Work {
    double* idt;      // [N] 1 / dt of the scaled lines (FP64)
    float* idt32;     // [N] the same in FP32
    float* z32;       // [3N] z~ of the FP32 iteration (the p double buffer keeps both halves for p~)
    int warps[2];     // warps per CTA of the line kernel, [0] FP64, [1] FP32
    size_t smem[2];   // its dynamic shared memory
    int line_blocks[2];
};

// 1 / dt along every phi line of A~ (one thread per line); a non-positive pivot flags a breakdown
__global__ void k_pc2_factor(Dims d, OpTab<double> t, double* __restrict__ idt, float* __restrict__ idt32,
                             PcgScalars* sc) {
    const int nl = d.nr * d.nt;
    for (int ij = blockIdx.x * blockDim.x + threadIdx.x; ij < nl; ij += gridDim.x * blockDim.x) {
        const double w = t.ap[ij];
        const double w2 = w * w;
        const long long base = (long long)ij * d.np;
        double dt = 1.0;
        bool bad = false;
        idt[base] = 1.0;
        idt32[base] = 1.0f;
        for (int k = 1; k < d.np; k++) {
            dt = 1.0 - w2 / dt;
            if (k == d.np - 1) dt -= w2;
            bad = bad || !(dt > 0.0);
            const double id = 1.0 / dt;
            idt[base + k] = id;
            idt32[base + k] = (float)id;
        }
        if (bad) sc->done = 4;
    }
}

// Shared memory per warp: 1/dt, w/dt and a work line, each np + ceil(np / S) elements (one pad
// after each lane segment of S = ceil(np / 32) elements; element k sits at k + k / S).
__host__ __device__ inline int padded_len(int np) {
    const int S = (np + 31) / 32;
    return np + (np + S - 1) / S;
}

// One warp per phi line of the scaled system.
//   kIter:     x~ += alpha p~ (FP64), r~ -= alpha q~; z~ = P~^-1 r~; <r~, z~> and
//              ||r||^2 = sum dg r~^2; last CTA: beta = rho_new / rho, stop test, iteration count.
//              FP32 defers the x update: alpha is handed on in sc->ax, and the p update of the
//              next iteration (or the correction kernel when the inner solve stops here) adds
//              alpha p~ to x~.
//   kInit:     z~ = P~^-1 r~, p~ = z~; last CTA: rho, beta = 0, stop test (after the FP64 set-up).
//   kReliable: z~ = P~^-1 r~ for the replaced residual; last CTA: rho = <r~, z~>, and the
//              recurrence continues (beta = rho / rho_prev) while rho stays within 4x of the
//              recursive one, else restarts (beta = 0); the stop flags are the outer kernel's.
// SEG > 0: np = 32 SEG exactly, so the segment length is a compile-time constant: the segment
// loops unroll (their shared-memory loads issue together) and the bounds tests vanish (the first
// and last elements of the line are lane 0's first and lane 31's last). SEG = 0: any np.
template <typename T, int NC, int MODE, int SEG>
__global__ void __launch_bounds__(kThreads) k_pc2_line(Dims d, OpTab<T> t, const double* __restrict__ dgv,
                                                       const T* __restrict__ idt, T* __restrict__ x,
                                                       T* __restrict__ p, T* __restrict__ r,
                                                       const T* __restrict__ q, T* __restrict__ z,
                                                       PcgScalars* sc, double* __restrict__ partials, int restart) {
    if (sc->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* smem = reinterpret_cast<T*>(smem_raw);
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = d.np;
    const int S = SEG > 0 ? SEG : (np + 31) >> 5;
    const int P = padded_len(np);
    T* ib = smem + (size_t)warp * 3 * P;   // 1 / dt_k
    T* gb = ib + P;                        // w / dt_k
    T* ub = gb + P;                        // work line
    const T al = (MODE == kIter) ? (T)sc->alpha : T(0);
    const T zero = T(0);
    const int k0 = lane * S;
    const int s0 = lane * (S + 1);         // element k0 + t of this lane's segment sits at s0 + t
    constexpr bool exact = SEG > 0;
    // FP32: x~ += alpha p~ moves to the next p update, which leaves this HBM-bound kernel 52 instead
    // of 88 B per cell; FP64: the kernel is bound by its FP64 instructions and the x update stays here
    constexpr bool kDeferX = sizeof(T) == 4;
    // element k0 + t is in the line / is its first / is its last element
#define IN_LINE(tt) (exact || k0 + (tt) < np)
#define FIRST(tt) ((tt) == 0 && lane == 0)
#define LAST(tt) (exact ? ((tt) == S - 1 && lane == 31) : (k0 + (tt) == np - 1))
    double a_rz = 0.0, a_rr = 0.0;   // per-line partials (in T) are added here in FP64
    const int nl = d.nr * d.nt;
    for (int line = blockIdx.x * warps + warp; line < nl; line += gridDim.x * warps) {
        const T w = t.ap[line];
        const long long base = (long long)line * np;
        for (int k = lane; k < np; k += 32) {
            const T id = idt[base + k];
            ib[k + k / S] = id;
            gb[k + k / S] = w * id;
        }
        __syncwarp();
        // component-independent multipliers: forward a_k (a_0 = 0), backward c_k (c_{np-1} = 0)
        T A = T(1), Cm = T(1);
#pragma unroll
        for (int tt = 0; tt < S; tt++) {
            if (IN_LINE(tt)) {
                const T g = gb[s0 + tt];
                A *= FIRST(tt) ? zero : g;
                Cm *= LAST(tt) ? zero : g;
            }
        }
        T As[5], Cs[5];
#pragma unroll
        for (int st = 0; st < 5; st++) {
            const int o = 1 << st;
            const T Ao = __shfl_up_sync(kFull, A, o), Co = __shfl_down_sync(kFull, Cm, o);
            As[st] = A;
            Cs[st] = Cm;
            if (lane >= o) A *= Ao;
            if (lane + o < 32) Cm *= Co;
        }
        T line_rz = zero, line_rr = zero;
#pragma unroll 1
        for (int c = 0; c < NC; c++) {
            const long long off = c * d.N + base;
            for (int k = lane; k < np; k += 32) {
                T rv = r[off + k];
                if (MODE == kIter) {
                    if constexpr (!kDeferX) x[off + k] = fma(al, p[off + k], x[off + k]);
                    rv = fma(-al, q[off + k], rv);
                    r[off + k] = rv;
                }
                ub[k + k / S] = rv;
            }
            __syncwarp();
            // forward: u_0 = r_0 / dt_0; u_k = (r_k + w u_{k-1}) / dt_k; the last also + w u_0 / dt
            const T u0 = ub[0] * ib[0];
            __syncwarp();
            T B = zero;
#pragma unroll
            for (int tt = 0; tt < S; tt++) {
                if (IN_LINE(tt)) {
                    const int sx = s0 + tt;
                    T bk = ub[sx] * ib[sx];
                    if (LAST(tt)) bk = fma(gb[sx], u0, bk);
                    ub[sx] = bk;
                    B = fma(FIRST(tt) ? zero : gb[sx], B, bk);
                }
            }
#pragma unroll
            for (int st = 0; st < 5; st++) {
                const int o = 1 << st;
                const T Bo = __shfl_up_sync(kFull, B, o);
                if (lane >= o) B = fma(As[st], Bo, B);
            }
            T u = __shfl_up_sync(kFull, B, 1);
            if (lane == 0) u = zero;
#pragma unroll
            for (int tt = 0; tt < S; tt++) {
                if (IN_LINE(tt)) {
                    const int sx = s0 + tt;
                    u = fma(FIRST(tt) ? zero : gb[sx], u, ub[sx]);
                    ub[sx] = u;
                }
            }
            __syncwarp();
            // backward: z_{np-1} = u_{np-1}; z_k = u_k + w z_{k+1} / dt_k; the first also + w z_{np-1} / dt_0
            const T zl = ub[(np - 1) + (np - 1) / S];
            __syncwarp();
            T E = zero;
#pragma unroll
            for (int tt = S - 1; tt >= 0; tt--) {
                if (IN_LINE(tt)) {
                    const int sx = s0 + tt;
                    T e = ub[sx];
                    if (FIRST(tt)) e = fma(gb[sx], zl, e);
                    ub[sx] = e;
                    E = fma(LAST(tt) ? zero : gb[sx], E, e);
                }
            }
#pragma unroll
            for (int st = 0; st < 5; st++) {
                const int o = 1 << st;
                const T Eo = __shfl_down_sync(kFull, E, o);
                if (lane + o < 32) E = fma(Cs[st], Eo, E);
            }
            T zz = __shfl_down_sync(kFull, E, 1);
            if (lane == 31) zz = zero;
#pragma unroll
            for (int tt = S - 1; tt >= 0; tt--) {
                if (IN_LINE(tt)) {
                    const int sx = s0 + tt;
                    zz = fma(LAST(tt) ? zero : gb[sx], zz, ub[sx]);
                    ub[sx] = zz;
                }
            }
            __syncwarp();
            for (int k = lane; k < np; k += 32) {
                const T zv = ub[k + k / S];
                const T rv = r[off + k];
                z[off + k] = zv;
                if (MODE == kInit) p[off + k] = zv;
                line_rz = fma(rv, zv, line_rz);
                line_rr = fma(rv, rv, line_rr);
            }
            __syncwarp();
        }
        a_rz += (double)line_rz;
        a_rr = fma(dgv[line], (double)line_rr, a_rr);
    }
#undef IN_LINE
#undef FIRST
#undef LAST
    double val[2] = {a_rz, a_rr}, out[2];
    if (reduce_last<2>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double rz = out[0], rr = out[1];
        if (MODE == kReliable) {
            const bool keep = !restart && sc->rho_prev > 0.0 && rz <= 4.0 * sc->rho;
            sc->beta = keep ? rz / sc->rho_prev : 0.0;
            sc->rho = rz;
            sc->rr = rr;
            if (!isfinite(rz) || !isfinite(rr)) {
                sc->done = 3;
                sc->outer_done = 3;
            } else if (!(rz > 0.0)) {
                sc->done = 4;
            }
            return;
        }
        if (MODE == kInit) {
            sc->beta = 0.0;
        } else {
            sc->iter += 1;
            sc->total_iter += 1;
            sc->beta = rz / sc->rho;
            sc->rho_prev = sc->rho;
            if (kDeferX) sc->ax = sc->alpha;   // x~ += alpha p~ is left to the next p update
        }
        sc->rho = rz;
        sc->rr = rr;
        if (!isfinite(rz) || !isfinite(rr)) sc->done = 3;
        else if (sc->bb == 0.0 || sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
        else if (sc->iter >= sc->max_iter) sc->done = 2;
        else if (!(rz > 0.0)) sc->done = 4;
    }
}

template <typename T>
size_t line_smem(const Dims& d, int warps) {
    return (size_t)warps * 3 * padded_len(d.np) * sizeof(T);
}

// compile-time segment length for np = 512 (16 elements per lane), else the generic kernel
int seg_of(const Dims& d) { return (d.np == 512) ? 16 : 0; }

template <typename T, int MODE, int SEG>
cudaError_t set_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_pc2_line<T, 1, MODE, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pc2_line<T, 2, MODE, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pc2_line<T, 3, MODE, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes);
    return e;
}

template <typename T, int SEG>
cudaError_t set_smem_all(size_t bytes) {
    cudaError_t e = set_smem<T, kIter, SEG>(bytes);
    if (e == cudaSuccess) e = set_smem<T, kInit, SEG>(bytes);
    if (e == cudaSuccess) e = set_smem<T, kReliable, SEG>(bytes);
    return e;
}

// launch shape of the line kernel for element type T: up to 8 warps per CTA within 200 KB
template <typename T>
mhd_status_t line_shape(mhd_grid_s* g, Pc2Work* w, int slot) {
    int warps = 8;
    while (warps > 1 && line_smem<T>(g->d, warps) > 200 * 1024) warps >>= 1;
    if (line_smem<T>(g->d, warps) > 200 * 1024) return set_error(g, MHD_ERR_ARG, "PC2: np too large for the line kernel");
    const size_t bytes = line_smem<T>(g->d, warps);
    const bool s16 = seg_of(g->d) == 16;
    if ((s16 ? set_smem_all<T, 16>(bytes) : set_smem_all<T, 0>(bytes)) != cudaSuccess)
        return check_cuda(g, "PC2: shared memory attribute");
    int per_sm = 0;
    if (s16)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pc2_line<T, 3, kIter, 16>, 32 * warps, bytes);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pc2_line<T, 3, kIter, 0>, 32 * warps, bytes);
    if (per_sm < 1) per_sm = 1;
    const int nl = g->d.nr * g->d.nt;
    w->warps[slot] = warps;
    w->smem[slot] = bytes;
    w->line_blocks[slot] = std::min(std::min(g->num_sms * per_sm, (nl + warps - 1) / warps), kMaxBlocks);
    return MHD_OK;
}

mhd_status_t pc2_workspace(mhd_grid_s* g, Pc2Work** out) {
    if (g->pc2_mem) {
        *out = reinterpret_cast<Pc2Work*>(g->pc2_mem);
        return MHD_OK;
    }
    auto* w = new Pc2Work{};
    const size_t N = (size_t)g->d.N;
    if (cudaMalloc(&w->idt, sizeof(double) * N) != cudaSuccess ||
        cudaMalloc(&w->idt32, sizeof(float) * N) != cudaSuccess ||
        cudaMalloc(&w->z32, sizeof(float) * 3 * N) != cudaSuccess) {
        if (w->idt) cudaFree(w->idt);
        if (w->idt32) cudaFree(w->idt32);
        delete w;
        cudaGetLastError();
        return set_error(g, MHD_ERR_OOM, "PC2: workspace allocation failed");
    }
    mhd_status_t st = line_shape<double>(g, w, 0);
    if (st == MHD_OK) st = line_shape<float>(g, w, 1);
    if (st == MHD_OK && cudaMemsetAsync(w->z32, 0, sizeof(float) * 3 * N, g->stream) != cudaSuccess)
        st = check_cuda(g, "PC2: workspace clear");
    if (st != MHD_OK) {
        cudaFree(w->idt);
        cudaFree(w->idt32);
        cudaFree(w->z32);
        delete w;
        return st;
    }
    g->pc2_mem = w;
    *out = w;
    return MHD_OK;
}

template <typename T, int MODE, int SEG>
void launch_seg(mhd_grid_s* g, cudaStream_t st, const Pc2Work* w, int nc, int restart) {
    const Dims d = g->d;
    const int slot = sizeof(T) == 8 ? 0 : 1;
    const dim3 grid(w->line_blocks[slot]), block(32 * w->warps[slot]);
    const size_t sm = w->smem[slot];
    T *x, *p, *r, *q;
    const T* idt;
    OpTab<T> t;
    if constexpr (sizeof(T) == 8) {
        x = g->x64; p = g->p64; r = g->r64; q = g->q64; idt = w->idt; t = g->t64;
    } else {
        x = g->x32; p = g->p32; r = g->r32; q = g->q32; idt = w->idt32; t = g->t32;
    }
    // z~: FP64 in the second half of the p double buffer, FP32 in the workspace
    T* z;
    if constexpr (sizeof(T) == 8) z = p + 3 * (size_t)d.N;
    else z = w->z32;
    if (nc == 3)
        k_pc2_line<T, 3, MODE, SEG><<<grid, block, sm, st>>>(d, t, g->tu.dg, idt, x, p, r, q, z, g->sc, g->partials,
                                                              restart);
    else if (nc == 2)
        k_pc2_line<T, 2, MODE, SEG><<<grid, block, sm, st>>>(d, t, g->tu.dg, idt, x, p, r, q, z, g->sc, g->partials,
                                                              restart);
    else
        k_pc2_line<T, 1, MODE, SEG><<<grid, block, sm, st>>>(d, t, g->tu.dg, idt, x, p, r, q, z, g->sc, g->partials,
                                                              restart);
}

template <typename T, int MODE>
void launch_line(mhd_grid_s* g, cudaStream_t st, int nc, int restart = 0) {
    const auto* w = reinterpret_cast<const Pc2Work*>(g->pc2_mem);
    if (seg_of(g->d) == 16) launch_seg<T, MODE, 16>(g, st, w, nc, restart);
    else launch_seg<T, MODE, 0>(g, st, w, nc, restart);
}

}  // namespace

void pc2_free(mhd_grid_s* g) {
    if (!g->pc2_mem) return;
    auto* w = reinterpret_cast<Pc2Work*>(g->pc2_mem);
    cudaFree(w->idt);
    cudaFree(w->idt32);
    cudaFree(w->z32);
    delete w;
    g->pc2_mem = nullptr;
}

float* pc2_z32(mhd_grid_s* g) { return reinterpret_cast<Pc2Work*>(g->pc2_mem)->z32; }

// factorise the lines of A~ for the current tables (FP64 and FP32 copies)
mhd_status_t pc2_factor(mhd_grid_s* g) {
    Pc2Work* w = nullptr;
    mhd_status_t st = pc2_workspace(g, &w);
    if (st != MHD_OK) return st;
    const int nl = g->d.nr * g->d.nt;
    k_pc2_factor<<<(nl + kThreads - 1) / kThreads, kThreads, 0, g->stream>>>(g->d, g->t64, w->idt, w->idt32, g->sc);
    return check_cuda(g, "PC2 factorisation");
}

// FP64: after the scaled set-up (x~, r~, rr, bb, done) form z~ = P~^-1 r~, p~ = z~, rho
void pc2_init64(mhd_grid_s* g, int nc) { launch_line<double, kInit>(g, g->stream, nc); }

// FP32 inner solves: after the outer residual replaced r~32, recompute z~32 and rho and decide
// between continuing the recurrence and restarting it
void pc2_reliable32(mhd_grid_s* g, int nc, int restart) { launch_line<float, kReliable>(g, g->stream, nc, restart); }

// the line kernel of one iteration (x / r update, z = P^-1 r, dots)
void pc2_enqueue_line(mhd_grid_s* g, cudaStream_t st, int nc, bool fp32) {
    if (fp32) launch_line<float, kIter>(g, st, nc);
    else launch_line<double, kIter>(g, st, nc);
}

// PC2 workspace, allocated ahead of the first PC2 solve
mhd_status_t pc2_reserve(mhd_grid_s* g) {
    Pc2Work* w = nullptr;
    return pc2_workspace(g, &w);
}

}  // namespace mhd
