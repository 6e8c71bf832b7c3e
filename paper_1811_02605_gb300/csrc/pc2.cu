// PC2 (Sec. 2.2): PCG with a block-Jacobi preconditioner that uses a zero-fill incomplete LU
// factorisation (ILU(0)) in each block. The blocks are the periodic phi lines (i, j) of each
// component: the r and theta couplings are left out of the preconditioner, so every line is an
// independent block (nr nt of them per component) instead of one block per MPI rank as in the
// paper. For a periodic tridiagonal block zero fill changes only the diagonal:
//     dt_0 = m,  dt_k = m - w^2 / dt_{k-1},  dt_{np-1} -= w^2 / dt_0,
// m the diagonal on the line and -w its phi coupling, and P = (dt + L) dt^-1 (dt + U).
//
// The solve runs on the Jacobi-scaled system A~ = S M S (S = diag(M)^-1/2, unit diagonal, the
// PC1 path's tables and stencil kernel), whose ILU(0) is S ILU(0)(M) S: the same iterates as PCG
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
#include <cmath>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Pc2Work {
    double* idt;      // [N] 1 / dt of the scaled lines
    int warps;        // warps per CTA of the line kernel
    size_t smem;      // its dynamic shared memory
    int line_blocks;
};

// 1 / dt along every phi line of A~ (one thread per line); a non-positive pivot flags a breakdown
__global__ void k_pc2_factor(Dims d, OpTab<double> t, double* __restrict__ idt, PcgScalars* sc) {
    const int nl = d.nr * d.nt;
    for (int ij = blockIdx.x * blockDim.x + threadIdx.x; ij < nl; ij += gridDim.x * blockDim.x) {
        const double w = t.ap[ij];
        const double w2 = w * w;
        double* o = idt + (long long)ij * d.np;
        double dt = 1.0;
        bool bad = false;
        o[0] = 1.0;
        for (int k = 1; k < d.np; k++) {
            dt = 1.0 - w2 / dt;
            if (k == d.np - 1) dt -= w2;
            bad = bad || !(dt > 0.0);
            o[k] = 1.0 / dt;
        }
        if (bad) sc->done = 4;
    }
}

// Shared memory per warp: 1/dt, w/dt and a work line, each np + ceil(np / S) doubles (one pad
// after each lane segment of S = ceil(np / 32) elements; element k sits at k + k / S).
__host__ __device__ inline int padded_len(int np) {
    const int S = (np + 31) / 32;
    return np + (np + S - 1) / S;
}

// One warp per phi line of the scaled system: (unless INIT) x~ += alpha p~, r~ -= alpha q~; then
// z~ = P~^-1 r~; <r~, z~> and ||r||^2 = sum dg r~^2. INIT sets p~ = z~. Last CTA: beta (0 for
// INIT), stop test.
// SEG > 0: the segment length S is a compile-time constant (np in (32 (SEG - 1), 32 SEG]), so the
// segment loops unroll and their shared-memory loads issue together; SEG = 0: any np.
template <int NC, bool INIT, int SEG>
__global__ void __launch_bounds__(kThreads) k_pc2_line(Dims d, OpTab<double> t, const double* __restrict__ dgv,
                                                       const double* __restrict__ idt, double* __restrict__ x,
                                                       double* __restrict__ p, double* __restrict__ r,
                                                       const double* __restrict__ q, double* __restrict__ z,
                                                       PcgScalars* sc, double* __restrict__ partials) {
    if (sc->done) return;
    extern __shared__ double smem[];
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = d.np;
    const int S = SEG > 0 ? SEG : (np + 31) >> 5;
    const int P = padded_len(np);
    double* ib = smem + (size_t)warp * 3 * P;   // 1 / dt_k
    double* gb = ib + P;                        // w / dt_k
    double* ub = gb + P;                        // work line
    const double al = INIT ? 0.0 : sc->alpha;
    const int k0 = lane * S;
    double a_rz = 0.0, a_rr = 0.0;
    const int nl = d.nr * d.nt;
    for (int line = blockIdx.x * warps + warp; line < nl; line += gridDim.x * warps) {
        const double w = t.ap[line];
        const long long base = (long long)line * np;
        for (int k = lane; k < np; k += 32) {
            const double id = idt[base + k];
            ib[k + k / S] = id;
            gb[k + k / S] = w * id;
        }
        __syncwarp();
        // component-independent multipliers: forward a_k (a_0 = 0), backward c_k (c_{np-1} = 0);
        // element k0 + t of this lane's segment sits at s0 + t
        const int s0 = lane * (S + 1);
        double A = 1.0, Cm = 1.0;
#pragma unroll
        for (int tt = 0; tt < S; tt++) {
            const int k = k0 + tt;
            if (k < np) {
                const double g = gb[s0 + tt];
                A *= (k == 0) ? 0.0 : g;
                Cm *= (k == np - 1) ? 0.0 : g;
            }
        }
        double As[5], Cs[5];
#pragma unroll
        for (int st = 0; st < 5; st++) {
            const int o = 1 << st;
            const double Ao = __shfl_up_sync(kFull, A, o), Co = __shfl_down_sync(kFull, Cm, o);
            As[st] = A;
            Cs[st] = Cm;
            if (lane >= o) A *= Ao;
            if (lane + o < 32) Cm *= Co;
        }
        double line_rr = 0.0;
#pragma unroll 1
        for (int c = 0; c < NC; c++) {
            const long long off = c * d.N + base;
            for (int k = lane; k < np; k += 32) {
                double rv = r[off + k];
                if (!INIT) {
                    x[off + k] = fma(al, p[off + k], x[off + k]);
                    rv = fma(-al, q[off + k], rv);
                    r[off + k] = rv;
                }
                ub[k + k / S] = rv;
            }
            __syncwarp();
            // forward: u_0 = r_0 / dt_0; u_k = (r_k + w u_{k-1}) / dt_k; the last also + w u_0 / dt
            const double u0 = ub[0] * ib[0];
            __syncwarp();
            double B = 0.0;
#pragma unroll
            for (int tt = 0; tt < S; tt++) {
                const int k = k0 + tt;
                if (k < np) {
                    const int sx = s0 + tt;
                    double bk = ub[sx] * ib[sx];
                    if (k == np - 1) bk = fma(gb[sx], u0, bk);
                    ub[sx] = bk;
                    B = fma((k == 0) ? 0.0 : gb[sx], B, bk);
                }
            }
#pragma unroll
            for (int st = 0; st < 5; st++) {
                const int o = 1 << st;
                const double Bo = __shfl_up_sync(kFull, B, o);
                if (lane >= o) B = fma(As[st], Bo, B);
            }
            double u = __shfl_up_sync(kFull, B, 1);
            if (lane == 0) u = 0.0;
#pragma unroll
            for (int tt = 0; tt < S; tt++) {
                const int k = k0 + tt;
                if (k < np) {
                    const int sx = s0 + tt;
                    u = fma((k == 0) ? 0.0 : gb[sx], u, ub[sx]);
                    ub[sx] = u;
                }
            }
            __syncwarp();
            // backward: z_{np-1} = u_{np-1}; z_k = u_k + w z_{k+1} / dt_k; the first also + w z_{np-1} / dt_0
            const double zl = ub[(np - 1) + (np - 1) / S];
            __syncwarp();
            double E = 0.0;
#pragma unroll
            for (int tt = S - 1; tt >= 0; tt--) {
                const int k = k0 + tt;
                if (k < np) {
                    const int sx = s0 + tt;
                    double e = ub[sx];
                    if (k == 0) e = fma(gb[sx], zl, e);
                    ub[sx] = e;
                    E = fma((k == np - 1) ? 0.0 : gb[sx], E, e);
                }
            }
#pragma unroll
            for (int st = 0; st < 5; st++) {
                const int o = 1 << st;
                const double Eo = __shfl_down_sync(kFull, E, o);
                if (lane + o < 32) E = fma(Cs[st], Eo, E);
            }
            double zz = __shfl_down_sync(kFull, E, 1);
            if (lane == 31) zz = 0.0;
#pragma unroll
            for (int tt = S - 1; tt >= 0; tt--) {
                const int k = k0 + tt;
                if (k < np) {
                    const int sx = s0 + tt;
                    zz = fma((k == np - 1) ? 0.0 : gb[sx], zz, ub[sx]);
                    ub[sx] = zz;
                }
            }
            __syncwarp();
            for (int k = lane; k < np; k += 32) {
                const double zv = ub[k + k / S];
                const double rv = r[off + k];
                z[off + k] = zv;
                if (INIT) p[off + k] = zv;
                a_rz = fma(rv, zv, a_rz);
                line_rr = fma(rv, rv, line_rr);
            }
            __syncwarp();
        }
        a_rr = fma(dgv[line], line_rr, a_rr);
    }
    double val[2] = {a_rz, a_rr}, out[2];
    if (reduce_last<2>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double rz = out[0], rr = out[1];
        if (INIT) {
            sc->beta = 0.0;
        } else {
            sc->iter += 1;
            sc->total_iter += 1;
            sc->beta = rz / sc->rho;
        }
        sc->rho = rz;
        sc->rr = rr;
        if (!isfinite(rz) || !isfinite(rr)) sc->done = 3;
        else if (sc->bb == 0.0 || sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
        else if (sc->iter >= sc->max_iter) sc->done = 2;
        else if (!(rz > 0.0)) sc->done = 4;
    }
}

size_t line_smem(const Dims& d, int warps) { return (size_t)warps * 3 * padded_len(d.np) * sizeof(double); }

template <bool INIT, int SEG>
cudaError_t set_smem(size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_pc2_line<1, INIT, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pc2_line<2, INIT, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pc2_line<3, INIT, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e;
}

// compile-time segment length for np in [481, 512] (16 elements per lane), else the generic kernel
int seg_of(const Dims& d) { return ((d.np + 31) / 32 == 16) ? 16 : 0; }

mhd_status_t pc2_workspace(mhd_grid_s* g, Pc2Work** out) {
    if (g->pc2_mem) {
        *out = reinterpret_cast<Pc2Work*>(g->pc2_mem);
        return MHD_OK;
    }
    // line kernel shape: up to 8 warps per CTA within 200 KB of shared memory
    int warps = 8;
    while (warps > 1 && line_smem(g->d, warps) > 200 * 1024) warps >>= 1;
    if (line_smem(g->d, warps) > 200 * 1024) return set_error(g, MHD_ERR_ARG, "PC2: np too large for the phi-line kernel");
    auto* w = new Pc2Work{};
    if (cudaMalloc(&w->idt, sizeof(double) * (size_t)g->d.N) != cudaSuccess) {
        delete w;
        cudaGetLastError();
        return set_error(g, MHD_ERR_OOM, "PC2: workspace allocation failed");
    }
    w->warps = warps;
    w->smem = line_smem(g->d, warps);
    const bool s16 = seg_of(g->d) == 16;
    if ((s16 ? set_smem<false, 16>(w->smem) : set_smem<false, 0>(w->smem)) != cudaSuccess ||
        (s16 ? set_smem<true, 16>(w->smem) : set_smem<true, 0>(w->smem)) != cudaSuccess) {
        cudaFree(w->idt);
        delete w;
        return check_cuda(g, "PC2: shared memory attribute");
    }
    int per_sm = 0;
    if (s16) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pc2_line<3, false, 16>, 32 * warps, w->smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pc2_line<3, false, 0>, 32 * warps, w->smem);
    if (per_sm < 1) per_sm = 1;
    const int nl = g->d.nr * g->d.nt;
    w->line_blocks = std::min(std::min(g->num_sms * per_sm, (nl + warps - 1) / warps), kMaxBlocks);
    g->pc2_mem = w;
    *out = w;
    return MHD_OK;
}

template <bool INIT, int SEG>
void launch_line_seg(mhd_grid_s* g, cudaStream_t st, const Pc2Work* w, int nc) {
    const Dims d = g->d;
    double* z = g->p64 + 3 * (size_t)d.N;
    const dim3 grid(w->line_blocks), block(32 * w->warps);
    if (nc == 3)
        k_pc2_line<3, INIT, SEG><<<grid, block, w->smem, st>>>(d, g->t64, g->tu.dg, w->idt, g->x64, g->p64, g->r64,
                                                                g->q64, z, g->sc, g->partials);
    else if (nc == 2)
        k_pc2_line<2, INIT, SEG><<<grid, block, w->smem, st>>>(d, g->t64, g->tu.dg, w->idt, g->x64, g->p64, g->r64,
                                                                g->q64, z, g->sc, g->partials);
    else
        k_pc2_line<1, INIT, SEG><<<grid, block, w->smem, st>>>(d, g->t64, g->tu.dg, w->idt, g->x64, g->p64, g->r64,
                                                                g->q64, z, g->sc, g->partials);
}

template <bool INIT>
void launch_line(mhd_grid_s* g, cudaStream_t st, const Pc2Work* w, int nc) {
    if (seg_of(g->d) == 16) launch_line_seg<INIT, 16>(g, st, w, nc);
    else launch_line_seg<INIT, 0>(g, st, w, nc);
}

}  // namespace

void pc2_free(mhd_grid_s* g) {
    if (!g->pc2_mem) return;
    auto* w = reinterpret_cast<Pc2Work*>(g->pc2_mem);
    cudaFree(w->idt);
    delete w;
    g->pc2_mem = nullptr;
}

// after the scaled set-up (x~, r~, rr, bb, done): factorise the lines and form z~ = P~^-1 r~,
// p~ = z~, rho = <r~, z~>
mhd_status_t pc2_prepare(mhd_grid_s* g, int nc) {
    Pc2Work* w = nullptr;
    mhd_status_t st = pc2_workspace(g, &w);
    if (st != MHD_OK) return st;
    const int nl = g->d.nr * g->d.nt;
    k_pc2_factor<<<(nl + kThreads - 1) / kThreads, kThreads, 0, g->stream>>>(g->d, g->t64, w->idt, g->sc);
    launch_line<true>(g, g->stream, w, nc);
    return check_cuda(g, "PC2 set-up");
}

// the line kernel of one iteration (x / r update, z = P^-1 r, dots); the workspace exists
void pc2_enqueue_line(mhd_grid_s* g, cudaStream_t st, int nc) {
    launch_line<false>(g, st, reinterpret_cast<const Pc2Work*>(g->pc2_mem), nc);
}

}  // namespace mhd
