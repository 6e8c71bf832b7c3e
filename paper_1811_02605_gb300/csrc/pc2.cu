// PC2 (Sec. 2.2): PCG with a block-Jacobi preconditioner that uses a zero-fill incomplete LU
// factorisation (ILU(0)) in each block. The blocks are the periodic phi lines (i, j) of each
// component: the r and theta couplings are left out of the preconditioner, so every line is an
// independent block (nr nt of them per component) instead of one block per MPI rank as in the
// paper. For a periodic tridiagonal block zero fill changes only the diagonal:
//     dt_0 = m,  dt_k = m - w^2 / dt_{k-1},  dt_{np-1} -= w^2 / dt_0,
// m the diagonal of M_alpha on the line and -w its phi coupling, and P = (dt + L) dt^-1 (dt + U).
// z = P^-1 r is a forward and a backward substitution along each line; both are first-order
// linear recurrences, which one warp per line evaluates as an affine scan: each lane composes the
// maps of its segment, a shuffle scan composes the segments, and each lane replays its segment
// from the value entering it. The periodic wrap enters as u_0 in the last forward step and as
// z_{np-1} in the last backward step, both known before the replay.
//
// One iteration: p = z + beta p; q = M p with <p, q> (alpha); x += alpha p, r -= alpha q, z =
// P^-1 r with <r, z> and ||r||^2 (beta, stop test). The vectors are unscaled (x, r, p, z, q);
// the factorisation (1 / dt, N values shared by the components) is built once per solve.
#include <cmath>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Pc2Work {
    double* idt;                  // [N] 1 / dt
    cudaGraphExec_t graph[4];     // batches of iterations, by ncomp
    int warps;                    // warps per CTA of the line kernel
    size_t smem;                  // its dynamic shared memory
    int line_blocks;
};

// 1 / dt along every phi line (one thread per line); a non-positive pivot flags a breakdown
__global__ void k_pc2_factor(Dims d, OpTab64u tu, double* __restrict__ idt, PcgScalars* sc) {
    const int nl = d.nr * d.nt;
    for (int ij = blockIdx.x * blockDim.x + threadIdx.x; ij < nl; ij += gridDim.x * blockDim.x) {
        const double m = tu.dg[ij], w = tu.awp[ij];
        const double w2 = w * w;
        double* o = idt + (long long)ij * d.np;
        double dt = m;
        bool bad = !(dt > 0.0);
        o[0] = 1.0 / dt;
        for (int k = 1; k < d.np; k++) {
            dt = m - w2 / dt;
            if (k == d.np - 1) dt -= w2 / m;
            bad = bad || !(dt > 0.0);
            o[k] = 1.0 / dt;
        }
        if (bad) sc->done = 4;
    }
}

// x = x0, r = b - M x0, ||b||^2
template <int NC>
__global__ void __launch_bounds__(kThreads) k_pc2_init(Dims d, OpTab64u tu, const double* __restrict__ b,
                                                       const double* __restrict__ x0, double* __restrict__ x,
                                                       double* __restrict__ r, PcgScalars* sc,
                                                       double* __restrict__ partials) {
    const int nt = d.nt;
    const long long plane = (long long)nt * d.np;
    double a_bb = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < d.N; c += (long long)gridDim.x * blockDim.x) {
        const long long ij = c / d.np;
        const int k = (int)(c - ij * d.np);
        const int i = (int)(ij / nt), j = (int)(ij - (long long)i * nt);
        const double m = tu.dg[ij], wp = tu.awp[ij];
        const double wl = tu.awr[i * nt + j], wh = tu.awr[(i + 1) * nt + j];
        const double tl = tu.awt[i * (nt + 1) + j], th = tu.awt[i * (nt + 1) + j + 1];
        const long long row = ij * d.np;
        const int km = (k == 0) ? d.np - 1 : k - 1, kp = (k + 1 == d.np) ? 0 : k + 1;
#pragma unroll
        for (int q = 0; q < NC; q++) {
            const double* u = x0 + q * d.N;
            double mx = m * u[c] - wp * (u[row + km] + u[row + kp]);
            if (i > 0) mx -= wl * u[c - plane];
            if (i < d.nr - 1) mx -= wh * u[c + plane];
            if (j > 0) mx -= tl * u[c - d.np];
            if (j < nt - 1) mx -= th * u[c + d.np];
            const double bv = b[q * d.N + c];
            x[q * d.N + c] = u[c];
            r[q * d.N + c] = bv - mx;
            a_bb = fma(bv, bv, a_bb);
        }
    }
    double val[1] = {a_bb}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        sc->bb = out[0];
        if (!isfinite(out[0])) sc->done = 3;
    }
}

// p = z + beta p
template <int NC>
__global__ void __launch_bounds__(kThreads) k_pc2_pupdate(Dims d, const double* __restrict__ z, double* __restrict__ p,
                                                          const PcgScalars* sc) {
    if (sc->done) return;
    const double be = sc->beta;
    const long long n = (long long)NC * d.N / 2;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        const double2 zv = reinterpret_cast<const double2*>(z)[g];
        double2 pv = reinterpret_cast<double2*>(p)[g];
        pv.x = fma(be, pv.x, zv.x);
        pv.y = fma(be, pv.y, zv.y);
        reinterpret_cast<double2*>(p)[g] = pv;
    }
}

// q = M p (unscaled tables) and <p, q>; last CTA: alpha
template <int NC>
__global__ void __launch_bounds__(kThreads, 4) k_pc2_spmv(Dims d, OpTab64u tu, const double* __restrict__ p,
                                                          double* __restrict__ q, PcgScalars* sc,
                                                          double* __restrict__ partials) {
    if (sc->done) return;
    const int nt = d.nt;
    const long long plane = (long long)nt * d.np;
    const unsigned int G = (unsigned int)(d.N / 2);
    const unsigned int npv = d.np / 2;
    double acc = 0.0;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const unsigned int ij = g / npv;
        const int k0 = (int)(g - ij * npv) * 2;
        const int i = (int)(ij / nt), j = (int)(ij - (unsigned)i * nt);
        const long long base = (long long)ij * d.np + k0;
        const double m = tu.dg[ij], wp = tu.awp[ij];
        const double wl = tu.awr[i * nt + j], wh = tu.awr[(i + 1) * nt + j];
        const double tl = tu.awt[i * (nt + 1) + j], th = tu.awt[i * (nt + 1) + j + 1];
        const long long row = base - k0;
        const int km = (k0 == 0) ? d.np - 1 : k0 - 1;
        const int kp = (k0 + 2 == d.np) ? 0 : k0 + 2;
#pragma unroll 1
        for (int c = 0; c < NC; c++) {
            const double* u = p + c * d.N;
            const double2 v = *reinterpret_cast<const double2*>(u + base);
            double o0 = fma(m, v.x, -wp * (u[row + km] + v.y));
            double o1 = fma(m, v.y, -wp * (v.x + u[row + kp]));
            if (i > 0) {
                const double2 n = *reinterpret_cast<const double2*>(u + base - plane);
                o0 = fma(-wl, n.x, o0);
                o1 = fma(-wl, n.y, o1);
            }
            if (i < d.nr - 1) {
                const double2 n = *reinterpret_cast<const double2*>(u + base + plane);
                o0 = fma(-wh, n.x, o0);
                o1 = fma(-wh, n.y, o1);
            }
            if (j > 0) {
                const double2 n = *reinterpret_cast<const double2*>(u + base - d.np);
                o0 = fma(-tl, n.x, o0);
                o1 = fma(-tl, n.y, o1);
            }
            if (j < nt - 1) {
                const double2 n = *reinterpret_cast<const double2*>(u + base + d.np);
                o0 = fma(-th, n.x, o0);
                o1 = fma(-th, n.y, o1);
            }
            *reinterpret_cast<double2*>(q + c * d.N + base) = make_double2(o0, o1);
            acc = fma(v.x, o0, fma(v.y, o1, acc));
        }
    }
    double val[1] = {acc}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double pq = out[0];
        sc->pq = pq;
        if (!isfinite(pq)) sc->done = 3;
        else if (!(pq > 0.0)) sc->done = 4;
        else sc->alpha = sc->rho / pq;
    }
}

// One warp per phi line: (unless INIT) x += alpha p, r -= alpha q; then z = P^-1 r by the two
// affine scans; <r, z>, ||r||^2. INIT also sets p = z. Last CTA: beta (0 for INIT), stop test.
// Shared memory per warp: 1/dt and a work line, each np + ceil(np / S) doubles (one pad after each
// lane segment, S = ceil(np / 32) elements per lane; element k sits at k + k / S).
template <int NC, bool INIT>
__global__ void __launch_bounds__(kThreads) k_pc2_line(Dims d, OpTab64u tu, const double* __restrict__ idt,
                                                       double* __restrict__ x, double* __restrict__ p,
                                                       double* __restrict__ r, const double* __restrict__ q,
                                                       double* __restrict__ z, PcgScalars* sc,
                                                       double* __restrict__ partials) {
    if (sc->done) return;
    extern __shared__ double smem[];
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = d.np;
    const int S = (np + 31) >> 5;
    const int P = np + (np + S - 1) / S;   // one pad after every lane segment that holds data
    double* ib = smem + (size_t)warp * 2 * P;
    double* ub = ib + P;
    const double al = INIT ? 0.0 : sc->alpha;
    const int k0 = lane * S, k1 = min(k0 + S, np);
    double a_rz = 0.0, a_rr = 0.0;
    const int nl = d.nr * d.nt;
    for (int line = blockIdx.x * warps + warp; line < nl; line += gridDim.x * warps) {
        const double w = tu.awp[line];
        const long long base = (long long)line * np;
        for (int k = lane; k < np; k += 32) ib[k + k / S] = idt[base + k];
        __syncwarp();
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
            // forward: u_0 = r_0 / dt_0; u_k = (r_k + w u_{k-1}) / dt_k; the last also + w u_0
            const double u0 = ub[0] * ib[0];
            __syncwarp();
            double A = 1.0, B = 0.0;
            for (int k = k0; k < k1; k++) {
                const int s = k + k / S;
                const double id = ib[s];
                const double a = (k == 0) ? 0.0 : w * id;
                double bk = ub[s] * id;
                if (k == np - 1) bk = fma(w * u0, id, bk);
                ub[s] = bk;
                B = fma(a, B, bk);
                A *= a;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double Ao = __shfl_up_sync(kFull, A, o), Bo = __shfl_up_sync(kFull, B, o);
                if (lane >= o) {
                    B = fma(A, Bo, B);
                    A *= Ao;
                }
            }
            double u = __shfl_up_sync(kFull, B, 1);
            if (lane == 0) u = 0.0;
            for (int k = k0; k < k1; k++) {
                const int s = k + k / S;
                const double a = (k == 0) ? 0.0 : w * ib[s];
                u = fma(a, u, ub[s]);
                ub[s] = u;
            }
            __syncwarp();
            // backward: z_{np-1} = u_{np-1}; z_k = u_k + w z_{k+1} / dt_k; the first also + w z_{np-1} / dt_0
            const double zl = ub[(np - 1) + (np - 1) / S];
            __syncwarp();
            double Cc = 1.0, E = 0.0;
            for (int k = k1 - 1; k >= k0; k--) {
                const int s = k + k / S;
                const double id = ib[s];
                const double cc = (k == np - 1) ? 0.0 : w * id;
                double e = ub[s];
                if (k == 0) e = fma(w * id, zl, e);
                ub[s] = e;
                E = fma(cc, E, e);
                Cc *= cc;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const double Co = __shfl_down_sync(kFull, Cc, o), Eo = __shfl_down_sync(kFull, E, o);
                if (lane + o < 32) {
                    E = fma(Cc, Eo, E);
                    Cc *= Co;
                }
            }
            double zz = __shfl_down_sync(kFull, E, 1);
            if (lane == 31) zz = 0.0;
            for (int k = k1 - 1; k >= k0; k--) {
                const int s = k + k / S;
                const double cc = (k == np - 1) ? 0.0 : w * ib[s];
                zz = fma(cc, zz, ub[s]);
                ub[s] = zz;
            }
            __syncwarp();
            for (int k = lane; k < np; k += 32) {
                const double zv = ub[k + k / S];
                const double rv = r[off + k];
                z[off + k] = zv;
                if (INIT) p[off + k] = zv;
                a_rz = fma(rv, zv, a_rz);
                a_rr = fma(rv, rv, a_rr);
            }
            __syncwarp();
        }
    }
    double val[2] = {a_rz, a_rr}, out[2];
    if (reduce_last<2>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double rz = out[0], rr = out[1];
        if (INIT) {
            sc->beta = 0.0;
            sc->iter = 0;
            sc->total_iter = 0;
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

__global__ void k_pc2_setup(PcgScalars* sc, double tol, int max_iter) {
    sc->tol = tol;
    sc->max_iter = max_iter;
    sc->done = 0;
    sc->iter = 0;
    sc->total_iter = 0;
    sc->outer = 0;
    sc->count = 0u;
}

size_t line_smem(const Dims& d, int warps) {
    const int S = (d.np + 31) / 32;
    return (size_t)warps * 2 * (d.np + (d.np + S - 1) / S) * sizeof(double);
}

mhd_status_t pc2_workspace(mhd_grid_s* g, Pc2Work** out) {
    if (g->pc2_mem) {
        *out = reinterpret_cast<Pc2Work*>(g->pc2_mem);
        return MHD_OK;
    }
    auto* w = new Pc2Work{};
    if (cudaMalloc(&w->idt, sizeof(double) * (size_t)g->d.N) != cudaSuccess) {
        delete w;
        cudaGetLastError();
        return set_error(g, MHD_ERR_OOM, "PC2: workspace allocation failed");
    }
    // line kernel shape: up to 8 warps per CTA within 200 KB of shared memory
    int warps = 8;
    while (warps > 1 && line_smem(g->d, warps) > 200 * 1024) warps >>= 1;
    if (line_smem(g->d, warps) > 200 * 1024) {
        cudaFree(w->idt);
        delete w;
        return set_error(g, MHD_ERR_ARG, "PC2: np too large for the phi-line kernel");
    }
    w->warps = warps;
    w->smem = line_smem(g->d, warps);
    const int a1 = cudaFuncSetAttribute(k_pc2_line<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->smem);
    const int a2 = cudaFuncSetAttribute(k_pc2_line<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->smem);
    const int a3 = cudaFuncSetAttribute(k_pc2_line<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->smem);
    const int a4 = cudaFuncSetAttribute(k_pc2_line<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->smem);
    const int a5 = cudaFuncSetAttribute(k_pc2_line<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->smem);
    const int a6 = cudaFuncSetAttribute(k_pc2_line<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)w->smem);
    if (a1 || a2 || a3 || a4 || a5 || a6) {
        cudaFree(w->idt);
        delete w;
        return check_cuda(g, "PC2: shared memory attribute");
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pc2_line<3, false>, 32 * warps, w->smem);
    if (per_sm < 1) per_sm = 1;
    const int nl = g->d.nr * g->d.nt;
    w->line_blocks = std::min(std::min(g->num_sms * per_sm, (nl + warps - 1) / warps), kMaxBlocks);
    g->pc2_mem = w;
    *out = w;
    return MHD_OK;
}

template <int NC>
void pc2_iteration(mhd_grid_s* g, cudaStream_t st, Pc2Work* w) {
    const Dims d = g->d;
    double* z = g->p64 + 3 * (size_t)d.N;
    int ps = prof_begin(g, st, MHD_KERNEL_PUPDATE64);
    k_pc2_pupdate<NC><<<grid_blocks(g, (long long)NC * d.N / 2, 4), kThreads, 0, st>>>(d, z, g->p64, g->sc);
    prof_end(g, st, ps);
    ps = prof_begin(g, st, MHD_KERNEL_SPMV64);
    k_pc2_spmv<NC><<<grid_blocks(g, d.N / 2, 4), kThreads, 0, st>>>(d, g->tu, g->p64, g->q64, g->sc, g->partials);
    prof_end(g, st, ps);
    ps = prof_begin(g, st, MHD_KERNEL_PC2);
    k_pc2_line<NC, false><<<w->line_blocks, 32 * w->warps, w->smem, st>>>(d, g->tu, w->idt, g->x64, g->p64, g->r64,
                                                                            g->q64, z, g->sc, g->partials);
    prof_end(g, st, ps);
}

void pc2_enqueue(mhd_grid_s* g, cudaStream_t st, Pc2Work* w, int nc) {
    if (nc == 3) pc2_iteration<3>(g, st, w);
    else if (nc == 2) pc2_iteration<2>(g, st, w);
    else pc2_iteration<1>(g, st, w);
}

mhd_status_t pc2_graph(mhd_grid_s* g, Pc2Work* w, int nc) {
    if (w->graph[nc]) return MHD_OK;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return check_cuda(g, "PC2 graph stream");
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return check_cuda(g, "PC2 graph capture");
    }
    for (int it = 0; it < g->graph_batch; it++) pc2_enqueue(g, cs, w, nc);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return set_error(g, MHD_ERR_CUDA, std::string("PC2 end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&w->graph[nc], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_error(g, MHD_ERR_CUDA, std::string("PC2 instantiate: ") + cudaGetErrorString(e));
    return MHD_OK;
}

mhd_status_t pc2_read(mhd_grid_s* g) {
    if (cudaMemcpyAsync(g->h_sc, g->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        return check_cuda(g, "PC2 read scalars");
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "PC2 sync");
    prof_flush(g);
    return MHD_OK;
}

}  // namespace

void pc2_free(mhd_grid_s* g) {
    if (!g->pc2_mem) return;
    auto* w = reinterpret_cast<Pc2Work*>(g->pc2_mem);
    for (auto& ge : w->graph)
        if (ge) cudaGraphExecDestroy(ge);
    cudaFree(w->idt);
    delete w;
    g->pc2_mem = nullptr;
}

// FP64 PCG with PC2 for M_alpha (the tables of alpha are already built); x holds x0 on entry
mhd_status_t pc2_solve(mhd_grid_s* g, int nc, const double* b, double* x, const double* x0, const mhd_params_t* prm,
                       int* iters, int* outer, double* relres) {
    Pc2Work* w = nullptr;
    mhd_status_t st = pc2_workspace(g, &w);
    if (st != MHD_OK) return st;
    if (!g->prof && (st = pc2_graph(g, w, nc)) != MHD_OK) return st;
    const Dims d = g->d;
    double* z = g->p64 + 3 * (size_t)d.N;
    k_pc2_setup<<<1, 1, 0, g->stream>>>(g->sc, prm->tol, prm->max_iter);
    const int nl = d.nr * d.nt;
    k_pc2_factor<<<(nl + kThreads - 1) / kThreads, kThreads, 0, g->stream>>>(d, g->tu, w->idt, g->sc);
    const int bi = grid_blocks(g, d.N, 4);
    if (nc == 3) k_pc2_init<3><<<bi, kThreads, 0, g->stream>>>(d, g->tu, b, x0, g->x64, g->r64, g->sc, g->partials);
    else if (nc == 2) k_pc2_init<2><<<bi, kThreads, 0, g->stream>>>(d, g->tu, b, x0, g->x64, g->r64, g->sc, g->partials);
    else k_pc2_init<1><<<bi, kThreads, 0, g->stream>>>(d, g->tu, b, x0, g->x64, g->r64, g->sc, g->partials);
    if (nc == 3)
        k_pc2_line<3, true><<<w->line_blocks, 32 * w->warps, w->smem, g->stream>>>(d, g->tu, w->idt, g->x64, g->p64,
                                                                                     g->r64, g->q64, z, g->sc, g->partials);
    else if (nc == 2)
        k_pc2_line<2, true><<<w->line_blocks, 32 * w->warps, w->smem, g->stream>>>(d, g->tu, w->idt, g->x64, g->p64,
                                                                                     g->r64, g->q64, z, g->sc, g->partials);
    else
        k_pc2_line<1, true><<<w->line_blocks, 32 * w->warps, w->smem, g->stream>>>(d, g->tu, w->idt, g->x64, g->p64,
                                                                                     g->r64, g->q64, z, g->sc, g->partials);
    if ((st = check_cuda(g, "PC2 set-up")) != MHD_OK) return st;
    for (;;) {
        if ((st = pc2_read(g)) != MHD_OK) return st;
        if (g->h_sc->done) break;
        if (g->prof) {
            for (int it = 0; it < 2 * g->graph_batch; it++) pc2_enqueue(g, g->stream, w, nc);
            if ((st = check_cuda(g, "PC2 iteration launch")) != MHD_OK) return st;
            continue;
        }
        if (cudaGraphLaunch(w->graph[nc], g->stream) != cudaSuccess) return check_cuda(g, "PC2 graph launch");
        if (cudaGraphLaunch(w->graph[nc], g->stream) != cudaSuccess) return check_cuda(g, "PC2 graph launch");
    }
    const PcgScalars h = *g->h_sc;
    if (h.bb == 0.0) cudaMemsetAsync(x, 0, sizeof(double) * nc * d.N, g->stream);
    else cudaMemcpyAsync(x, g->x64, sizeof(double) * nc * d.N, cudaMemcpyDeviceToDevice, g->stream);
    if ((st = check_cuda(g, "PC2 finish")) != MHD_OK) return st;
    if (iters) *iters = h.iter;
    if (outer) *outer = 0;
    if (relres) *relres = (h.bb > 0) ? std::sqrt(h.rr) / std::sqrt(h.bb) : 0.0;
    if (h.done == 1) return MHD_OK;
    if (h.done == 3) return set_error(g, MHD_ERR_NONFINITE, "PC2 pcg: non-finite value in a reduction");
    if (h.done == 4) return set_error(g, MHD_ERR_NOCONV, "PC2 pcg: breakdown (non-positive pivot or curvature)");
    return set_error(g, MHD_ERR_NOCONV, "PC2 pcg: no convergence within max_iter");
}

}  // namespace mhd
