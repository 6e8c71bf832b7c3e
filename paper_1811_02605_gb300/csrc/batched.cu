// Batched FP64 PCG: many independent systems M_alpha_s x_s = b_s on grids of different sizes,
// solved together by ONE persistent cooperative kernel launch (replayed from a CUDA graph).
//
// Each system uses its own grid's tables and workspace (the scaled CG of pcg.cu: p = r + beta p,
// q = A~ p, x += alpha p, r -= alpha q). The cells of all systems are cut into equal chunks; CTA b
// takes chunks b, b + nblocks, ... Each chunk writes one partial per dot product. After a grid
// barrier every CTA sums the partials of every system in chunk order, so all CTAs derive the same
// alpha, beta and stop decisions without a further barrier (three grid barriers per iteration).
// A converged system drops out of the work list; the launch ends when every system is done.
//
// The grid barrier is a generation counter in global memory. Every wait is bounded: after an
// iteration limit or a %globaltimer budget the CTA records MHD_ERR_TIMEOUT and returns, and the
// others then time out at the same barrier instead of hanging.
//
// The chunk size and the number of CTAs per SM are chosen by a small autotuner: on the first
// call for a batch shape it times a few iterations of each candidate and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "mhd_internal.cuh"

namespace mhd {
// kernels of pcg.cu launched from here (host stubs resolve across translation units)
__global__ void k_tables(Dims d, Geo G, const double* __restrict__ alpha_p, OpTab<double> t, OpTab<float> t32,
                         OpTab64u tu, int want32);
__global__ void k_init64(Dims d, int nc, const double* __restrict__ b, const double* __restrict__ x0,
                         double* __restrict__ xs, double* __restrict__ r, double* __restrict__ p, OpTab<double> t,
                         OpTab64u tu, PcgScalars* sc, double* __restrict__ partials);
__global__ void k_finish64(Dims d, int nc, const double* __restrict__ xs, const double* __restrict__ p,
                           double* __restrict__ x, const double* __restrict__ s, const PcgScalars* sc);
}  // namespace mhd

using namespace mhd;

namespace {

constexpr int kMaxSys = 256;
constexpr int kBT = 256;  // threads per CTA

struct SysDesc {
    Dims d;
    double *x, *r, *p, *q;
    const double *ar, *at, *ap, *dg;
    PcgScalars* sc;
    int c0, c1;  // chunk range
};

struct Chunk {
    int sys;
    unsigned int g0, g1;  // phi-pair groups [g0, g1)
};

struct BarrierState {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded grid barrier; returns false if any CTA gave up
__device__ bool grid_barrier(BarrierState* bs, unsigned int nblocks, unsigned long long budget_ns) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned int* vgen = &bs->gen;
        volatile int* verr = &bs->err;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bs->count, 1u);
        if (arrived == nblocks - 1) {
            bs->count = 0u;
            __threadfence();
            atomicAdd(&bs->gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer();
            unsigned long long polls = 0;
            while (*vgen == g) {
                if (*verr) break;
                if (++polls > (1ull << 28) || ((polls & 255) == 0 && globaltimer() - t0 > budget_ns)) {
                    atomicExch(&bs->err, 1);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok = (*verr == 0);
    }
    __syncthreads();
    return ok;
}

__device__ __forceinline__ double block_sum(double v, double* sm) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kBT / 32; w++) s += sm[w];
    return s;  // valid in thread 0
}

__global__ void __launch_bounds__(kBT) k_batched_pcg(const SysDesc* __restrict__ sys, int nsys,
                                                     const Chunk* __restrict__ chunks, int nchunks,
                                                     double* __restrict__ part, BarrierState* bs,
                                                     unsigned long long budget_ns, unsigned int extra) {
    __shared__ double s_rho[kMaxSys], s_alpha[kMaxSys], s_beta[kMaxSys], s_bb[kMaxSys], s_tol[kMaxSys];
    __shared__ int s_state[kMaxSys], s_iter[kMaxSys], s_max[kMaxSys];
    __shared__ double red[kBT / 32];
    __shared__ int any_active;
    double* part_pq = part;
    double* part_rho = part + nchunks;
    double* part_rr = part + 2 * nchunks;
    const unsigned int nb = gridDim.x;
    const unsigned int expect = nb + extra;  // extra > 0 only under fault injection

    for (int s = threadIdx.x; s < nsys; s += kBT) {
        const PcgScalars* sc = sys[s].sc;
        s_rho[s] = sc->rho;
        s_bb[s] = sc->bb;
        s_tol[s] = sc->tol;
        s_max[s] = sc->max_iter;
        s_state[s] = sc->done;
        s_iter[s] = 0;
        s_beta[s] = 0.0;
        s_alpha[s] = 0.0;
    }
    __syncthreads();

    for (;;) {
        if (threadIdx.x == 0) {
            int a = 0;
            for (int s = 0; s < nsys; s++) a |= (s_state[s] == 0);
            any_active = a;
        }
        __syncthreads();
        if (!any_active) break;

        // P1: p = r + beta p
        for (int c = blockIdx.x; c < nchunks; c += nb) {
            const Chunk ch = chunks[c];
            if (s_state[ch.sys]) continue;
            const SysDesc& S = sys[ch.sys];
            const double beta = s_beta[ch.sys];
            for (int k = 0; k < 3; k++) {
                const double* r = S.r + k * S.d.N;
                double* p = S.p + k * S.d.N;
                for (unsigned int g = ch.g0 + threadIdx.x; g < ch.g1; g += kBT) {
                    const double2 rv = *reinterpret_cast<const double2*>(r + 2ull * g);
                    double2 pv = *reinterpret_cast<double2*>(p + 2ull * g);
                    pv.x = fma(beta, pv.x, rv.x);
                    pv.y = fma(beta, pv.y, rv.y);
                    *reinterpret_cast<double2*>(p + 2ull * g) = pv;
                }
            }
        }
        if (!grid_barrier(bs, expect, budget_ns)) return;

        // P2: q = A~ p, partial <p, q> per chunk
        for (int c = blockIdx.x; c < nchunks; c += nb) {
            const Chunk ch = chunks[c];
            if (s_state[ch.sys]) continue;
            const SysDesc& S = sys[ch.sys];
            const Dims d = S.d;
            const long long plane = (long long)d.nt * d.np;
            const unsigned int npv = d.np / 2;
            double acc = 0.0;
            for (unsigned int g = ch.g0 + threadIdx.x; g < ch.g1; g += kBT) {
                const unsigned int ij = g / npv;
                const int k0 = (int)(g - ij * npv) * 2;
                const int i = (int)(ij / d.nt), j = (int)(ij - (unsigned)i * d.nt);
                const long long base = (long long)ij * d.np + k0;
                const double cr_lo = S.ar[i * d.nt + j], cr_hi = S.ar[(i + 1) * d.nt + j];
                const double ct_lo = S.at[i * (d.nt + 1) + j], ct_hi = S.at[i * (d.nt + 1) + j + 1];
                const double cp = S.ap[ij];
                const int km = (k0 == 0) ? d.np - 1 : k0 - 1;
                const int kp = (k0 + 2 == d.np) ? 0 : k0 + 2;
                for (int k = 0; k < 3; k++) {
                    const double* u = S.p + k * d.N;
                    const double2 v = *reinterpret_cast<const double2*>(u + base);
                    const long long row = base - k0;
                    double o0 = fma(-cp, u[row + km] + v.y, v.x);
                    double o1 = fma(-cp, v.x + u[row + kp], v.y);
                    if (i > 0) {
                        const double2 n = *reinterpret_cast<const double2*>(u + base - plane);
                        o0 = fma(-cr_lo, n.x, o0);
                        o1 = fma(-cr_lo, n.y, o1);
                    }
                    if (i < d.nr - 1) {
                        const double2 n = *reinterpret_cast<const double2*>(u + base + plane);
                        o0 = fma(-cr_hi, n.x, o0);
                        o1 = fma(-cr_hi, n.y, o1);
                    }
                    if (j > 0) {
                        const double2 n = *reinterpret_cast<const double2*>(u + base - d.np);
                        o0 = fma(-ct_lo, n.x, o0);
                        o1 = fma(-ct_lo, n.y, o1);
                    }
                    if (j < d.nt - 1) {
                        const double2 n = *reinterpret_cast<const double2*>(u + base + d.np);
                        o0 = fma(-ct_hi, n.x, o0);
                        o1 = fma(-ct_hi, n.y, o1);
                    }
                    *reinterpret_cast<double2*>(S.q + k * d.N + base) = make_double2(o0, o1);
                    acc = fma(v.x, o0, acc);
                    acc = fma(v.y, o1, acc);
                }
            }
            const double t = block_sum(acc, red);
            if (threadIdx.x == 0) part_pq[c] = t;
        }
        if (!grid_barrier(bs, expect, budget_ns)) return;

        // alpha per active system: one warp per system, lanes strided over its chunks and a fixed
        // shuffle tree, so every CTA forms identical values
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            for (int s = w; s < nsys; s += kBT / 32) {
                if (s_state[s]) continue;
                double pq = 0.0;
                for (int c = sys[s].c0 + lane; c < sys[s].c1; c += 32) pq += __ldcg(&part_pq[c]);
                for (int o = 16; o > 0; o >>= 1) pq += __shfl_xor_sync(0xffffffffu, pq, o);
                if (lane == 0) {
                    if (!isfinite(pq)) s_state[s] = 3;
                    else if (!(pq > 0.0)) s_state[s] = 4;
                    else s_alpha[s] = s_rho[s] / pq;
                }
            }
        }
        __syncthreads();

        // P3: x += alpha p, r -= alpha q, partial rho and rr per chunk
        for (int c = blockIdx.x; c < nchunks; c += nb) {
            const Chunk ch = chunks[c];
            if (s_state[ch.sys]) continue;
            const SysDesc& S = sys[ch.sys];
            const double al = s_alpha[ch.sys];
            const unsigned int npv = S.d.np / 2;
            double a_rho = 0.0, a_rr = 0.0;
            for (unsigned int g = ch.g0 + threadIdx.x; g < ch.g1; g += kBT) {
                double cell = 0.0;
                for (int k = 0; k < 3; k++) {
                    double* x = S.x + k * S.d.N + 2ull * g;
                    double* r = S.r + k * S.d.N + 2ull * g;
                    const double2 pv = *reinterpret_cast<const double2*>(S.p + k * S.d.N + 2ull * g);
                    const double2 qv = *reinterpret_cast<const double2*>(S.q + k * S.d.N + 2ull * g);
                    double2 xv = *reinterpret_cast<double2*>(x);
                    double2 rv = *reinterpret_cast<double2*>(r);
                    xv.x = fma(al, pv.x, xv.x);
                    xv.y = fma(al, pv.y, xv.y);
                    rv.x = fma(-al, qv.x, rv.x);
                    rv.y = fma(-al, qv.y, rv.y);
                    *reinterpret_cast<double2*>(x) = xv;
                    *reinterpret_cast<double2*>(r) = rv;
                    cell = fma(rv.x, rv.x, cell);
                    cell = fma(rv.y, rv.y, cell);
                }
                a_rho += cell;
                a_rr = fma(S.dg[g / npv], cell, a_rr);
            }
            const double t1 = block_sum(a_rho, red);
            const double t2 = block_sum(a_rr, red);
            if (threadIdx.x == 0) {
                part_rho[c] = t1;
                part_rr[c] = t2;
            }
        }
        if (!grid_barrier(bs, expect, budget_ns)) return;

        // beta and the stop test per active system (one warp per system)
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            for (int s = w; s < nsys; s += kBT / 32) {
                if (s_state[s]) continue;
                double rho = 0.0, rr = 0.0;
                for (int c = sys[s].c0 + lane; c < sys[s].c1; c += 32) {
                    rho += __ldcg(&part_rho[c]);
                    rr += __ldcg(&part_rr[c]);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    rho += __shfl_xor_sync(0xffffffffu, rho, o);
                    rr += __shfl_xor_sync(0xffffffffu, rr, o);
                }
                if (lane == 0) {
                    s_iter[s] += 1;
                    s_beta[s] = rho / s_rho[s];
                    s_rho[s] = rho;
                    int stt = 0;
                    if (!isfinite(rr) || !isfinite(rho)) stt = 3;
                    else if (sqrt(rr) <= s_tol[s] * sqrt(s_bb[s])) stt = 1;
                    else if (s_iter[s] >= s_max[s]) stt = 2;
                    if (stt && blockIdx.x == 0) sys[s].sc->rr = rr;
                    s_state[s] = stt;
                }
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        for (int s = threadIdx.x; s < nsys; s += kBT) {
            PcgScalars* sc = sys[s].sc;
            sc->iter = s_iter[s];
            sc->rho = s_rho[s];
            sc->done = s_state[s];
        }
    }
}

// ----------------------------------------------------------------------------------------------
// host: batch plans (device descriptors, graph) cached per batch signature
// ----------------------------------------------------------------------------------------------
struct Plan {
    int n = 0;
    std::vector<mhd_grid_s*> grids;
    std::vector<const double*> b;
    std::vector<double*> x;
    SysDesc* d_sys = nullptr;
    Chunk* d_chunks = nullptr;
    double* d_part = nullptr;
    BarrierState* d_bar = nullptr;
    double* d_alpha = nullptr;   // device alphas [n]
    double* h_alpha = nullptr;   // pinned host staging [n]
    int nchunks = 0;
    int blocks = 0;
    unsigned int chunk_groups = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t trial = nullptr;
    double tol = 0;
    int max_iter = 0;
    unsigned long long budget_ns = 20ull * 1000 * 1000 * 1000;  // 20 s per barrier wait
    unsigned int extra = 0;  // fault injection: barrier arrivals that never come
};

std::mutex g_mu;
std::map<std::vector<const void*>, Plan*> g_plans;

void free_plan(Plan* P) {
    if (P->graph) cudaGraphExecDestroy(P->graph);
    if (P->trial) cudaGraphExecDestroy(P->trial);
    if (P->d_sys) cudaFree(P->d_sys);
    if (P->d_chunks) cudaFree(P->d_chunks);
    if (P->d_part) cudaFree(P->d_part);
    if (P->d_bar) cudaFree(P->d_bar);
    if (P->d_alpha) cudaFree(P->d_alpha);
    if (P->h_alpha) cudaFreeHost(P->h_alpha);
    delete P;
}

mhd_status_t fail(mhd_status_t st, const char* msg) { return set_error(nullptr, st, msg); }

int max_coop_blocks_per_sm() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batched_pcg, kBT, 0);
    return nb;
}

// (re)build the chunk list and device descriptors for a chunk size and CTA count
mhd_status_t build_layout(Plan& P, unsigned int chunk_groups, int blocks) {
    std::vector<SysDesc> sd(P.n);
    std::vector<Chunk> ch;
    for (int s = 0; s < P.n; s++) {
        mhd_grid_s* g = P.grids[s];
        SysDesc& S = sd[s];
        S.d = g->d;
        S.x = g->x64;
        S.r = g->r64;
        S.p = g->p64;
        S.q = g->q64;
        S.ar = g->t64.ar;
        S.at = g->t64.at;
        S.ap = g->t64.ap;
        S.dg = g->tu.dg;
        S.sc = g->sc;
        S.c0 = (int)ch.size();
        const unsigned int G = (unsigned int)(g->d.N / 2);
        for (unsigned int g0 = 0; g0 < G; g0 += chunk_groups) ch.push_back(Chunk{s, g0, std::min(G, g0 + chunk_groups)});
        S.c1 = (int)ch.size();
    }
    cudaStream_t st = P.grids[0]->stream;
    if (P.d_chunks) cudaFree(P.d_chunks);
    if (P.d_part) cudaFree(P.d_part);
    P.d_chunks = nullptr;
    P.d_part = nullptr;
    if (cudaMalloc(&P.d_chunks, sizeof(Chunk) * ch.size()) != cudaSuccess ||
        cudaMalloc(&P.d_part, sizeof(double) * 3 * ch.size()) != cudaSuccess)
        return fail(MHD_ERR_OOM, "pcg_solve_batched: allocation failed");
    cudaMemcpyAsync(P.d_sys, sd.data(), sizeof(SysDesc) * P.n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(P.d_chunks, ch.data(), sizeof(Chunk) * ch.size(), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(P.d_bar, 0, sizeof(BarrierState), st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(MHD_ERR_CUDA, "pcg_solve_batched: upload failed");
    P.nchunks = (int)ch.size();
    P.chunk_groups = chunk_groups;
    P.blocks = blocks;
    return MHD_OK;
}

__global__ void k_batch_setup(PcgScalars* const* scs, int n, double tol, int max_iter) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    PcgScalars* sc = scs[s];
    sc->tol = tol;
    sc->inner_tol = 0.0;
    sc->max_iter = max_iter;
    sc->done = 0;
    sc->iter = 0;
    sc->total_iter = 0;
    sc->outer = 0;
    sc->outer_done = 0;
    sc->ax = 0.0;
    sc->count = 0u;
}

// enqueue one batched solve on stream st (captured into a graph by the caller)
void enqueue_batch(Plan& P, cudaStream_t st, bool finish, int max_iter_override) {
    cudaMemcpyAsync(P.d_alpha, P.h_alpha, sizeof(double) * P.n, cudaMemcpyHostToDevice, st);
    for (int s = 0; s < P.n; s++) {
        mhd_grid_s* g = P.grids[s];
        const int nij = g->d.nr * g->d.nt;
        k_tables<<<(nij + 255) / 256, 256, 0, st>>>(g->d, g->geo, P.d_alpha + s, g->t64, g->t32, g->tu, 0);
    }
    // per-system scalar set-up (scalar pointers kept in the spare tail of d_part's neighbour)
    PcgScalars** scs = reinterpret_cast<PcgScalars**>(P.d_sys + P.n);
    k_batch_setup<<<(P.n + 127) / 128, 128, 0, st>>>(scs, P.n, P.tol, max_iter_override);
    for (int s = 0; s < P.n; s++) {
        mhd_grid_s* g = P.grids[s];
        const int blocks = grid_blocks(g, g->d.N / 2, 4);
        k_init64<<<blocks, kThreads, 0, st>>>(g->d, 3, P.b[s], P.x[s], g->x64, g->r64, g->p64, g->t64, g->tu, g->sc,
                                              g->partials);
    }
    cudaMemsetAsync(P.d_bar, 0, sizeof(BarrierState), st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.blocks);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_batched_pcg, (const SysDesc*)P.d_sys, P.n, (const Chunk*)P.d_chunks, P.nchunks, P.d_part,
                       P.d_bar, P.budget_ns, P.extra);
    if (finish) {
        for (int s = 0; s < P.n; s++) {
            mhd_grid_s* g = P.grids[s];
            const int blocks = grid_blocks(g, g->d.N / 2, 4);
            k_finish64<<<blocks, kThreads, 0, st>>>(g->d, 3, g->x64, g->p64, P.x[s], g->t64.s, g->sc);
        }
    }
}

mhd_status_t capture(Plan& P, bool finish, int max_iter, cudaGraphExec_t* out) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return fail(MHD_ERR_CUDA, "pcg_solve_batched: stream");
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return fail(MHD_ERR_CUDA, "pcg_solve_batched: capture");
    }
    enqueue_batch(P, cs, finish, max_iter);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return fail(MHD_ERR_CUDA, cudaGetErrorString(e));
    if (*out) cudaGraphExecDestroy(*out);
    *out = nullptr;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MHD_ERR_CUDA, cudaGetErrorString(e));
    return MHD_OK;
}

// autotuner: time a few iterations of each (chunk size, CTAs per SM) candidate
mhd_status_t autotune(Plan& P) {
    const int nsm = P.grids[0]->num_sms;
    const int maxb = std::max(1, max_coop_blocks_per_sm());
    const unsigned int chunk_cands[] = {4096, 16384, 65536};
    std::vector<int> bps;
    for (int b : {1, 2, 4, 8})
        if (b <= maxb) bps.push_back(b);
    cudaStream_t st = P.grids[0]->stream;
    double best = 1e30;
    unsigned int best_c = chunk_cands[1];
    int best_b = std::min(maxb, 2) * nsm;
    const int trial_iters = 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (unsigned int cg : chunk_cands) {
        for (int b : bps) {
            if (build_layout(P, cg, b * nsm) != MHD_OK) return MHD_ERR_OOM;
            if (capture(P, false, trial_iters, &P.trial) != MHD_OK) return MHD_ERR_CUDA;
            cudaGraphLaunch(P.trial, st);  // warm
            cudaEventRecord(e0, st);
            cudaGraphLaunch(P.trial, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(MHD_ERR_CUDA, "autotune sync");
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_c = cg;
                best_b = b * nsm;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (P.trial) cudaGraphExecDestroy(P.trial);
    P.trial = nullptr;
    return build_layout(P, best_c, best_b);
}

}  // namespace

namespace mhd {
// drop cached batch plans that use a grid about to be destroyed
void batched_forget(mhd_grid_s* g) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        bool uses = false;
        for (mhd_grid_s* q : it->second ? it->second->grids : std::vector<mhd_grid_s*>{})
            if (q == g) uses = true;
        if (uses || !it->second) {
            if (it->second) free_plan(it->second);
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}
}  // namespace mhd

namespace {
// the plan of a batch (built and timed on first use) and its graph for these params
mhd_status_t prepare(int n, const mhd_grid_t* grids, const double* alpha, const double* const* b, double* const* x,
                     const mhd_params_t* params, Plan** out) {
    if (n < 1 || n > kMaxSys || !grids || !alpha || !b || !x || !params)
        return fail(MHD_ERR_ARG, "pcg_solve_batched: need 1 <= n <= 256 and non-null arrays");
    if (params->precision != MHD_PREC_FP64 || !(params->tol > 0.0) || params->max_iter < 0)
        return fail(MHD_ERR_ARG, "pcg_solve_batched: FP64 only; need tol > 0, max_iter >= 0");
    for (int s = 0; s < n; s++) {
        if (!grids[s] || !b[s] || !x[s] || !(alpha[s] >= 0.0))
            return fail(MHD_ERR_ARG, "pcg_solve_batched: null grid/vector or negative alpha");
        if ((const double*)x[s] == b[s]) return fail(MHD_ERR_ARG, "pcg_solve_batched: x aliases b");
        if (grids[s]->slab_nr_global > 0) return fail(MHD_ERR_ARG, "pcg_solve_batched: a slab grid");
        for (int t = 0; t < s; t++)
            if (grids[t] == grids[s]) return fail(MHD_ERR_ARG, "pcg_solve_batched: a grid appears twice");
    }
    std::vector<const void*> key;
    for (int s = 0; s < n; s++) {
        key.push_back(grids[s]);
        key.push_back(b[s]);
        key.push_back(x[s]);
    }
    Plan*& pp = g_plans[key];
    cudaStream_t st = grids[0]->stream;
    if (!pp) {
        Plan* P = new Plan();
        P->n = n;
        for (int s = 0; s < n; s++) {
            P->grids.push_back(grids[s]);
            P->b.push_back(b[s]);
            P->x.push_back(x[s]);
        }
        // d_sys holds n SysDesc followed by n PcgScalars pointers
        if (cudaMalloc(&P->d_sys, sizeof(SysDesc) * n + sizeof(PcgScalars*) * n) != cudaSuccess ||
            cudaMalloc(&P->d_bar, sizeof(BarrierState)) != cudaSuccess ||
            cudaMalloc(&P->d_alpha, sizeof(double) * n) != cudaSuccess ||
            cudaMallocHost(&P->h_alpha, sizeof(double) * n) != cudaSuccess) {
            free_plan(P);
            g_plans.erase(key);
            return fail(MHD_ERR_OOM, "pcg_solve_batched: allocation failed");
        }
        std::vector<PcgScalars*> scs(n);
        for (int s = 0; s < n; s++) scs[s] = grids[s]->sc;
        cudaMemcpy(P->d_sys + n, scs.data(), sizeof(PcgScalars*) * n, cudaMemcpyHostToDevice);
        std::memcpy(P->h_alpha, alpha, sizeof(double) * n);
        P->tol = params->tol;
        P->max_iter = params->max_iter;
        mhd_status_t stt = autotune(*P);
        if (stt != MHD_OK) {
            free_plan(P);
            g_plans.erase(key);
            return stt;
        }
        pp = P;
    }
    Plan& P = *pp;
    std::memcpy(P.h_alpha, alpha, sizeof(double) * n);
    // Fault injection for tests (no GPU fault): MHD_FAULT_BARRIER_MS=<ms> makes every grid barrier
    // wait for one arrival that never comes, with a budget of <ms>; the launch must then return
    // MHD_ERR_TIMEOUT with the context intact.
    unsigned int extra = 0;
    unsigned long long budget = 20ull * 1000 * 1000 * 1000;
    if (const char* f = std::getenv("MHD_FAULT_BARRIER_MS")) {
        const long ms = std::strtol(f, nullptr, 10);
        if (ms > 0) {
            extra = 1;
            budget = (unsigned long long)ms * 1000 * 1000;
        }
    }
    if (!P.graph || P.tol != params->tol || P.max_iter != params->max_iter || P.extra != extra ||
        P.budget_ns != budget) {
        P.tol = params->tol;
        P.max_iter = params->max_iter;
        P.extra = extra;
        P.budget_ns = budget;
        mhd_status_t stt = capture(P, true, P.max_iter, &P.graph);
        if (stt != MHD_OK) return stt;
    }
    *out = &P;
    return MHD_OK;
}
}  // namespace

extern "C" mhd_status_t pcg_solve_batched(int n, const mhd_grid_t* grids, const double* alpha,
                                          const double* const* b, double* const* x,
                                          const mhd_params_t* params, int* iters, double* relres) {
    std::lock_guard<std::mutex> lk(g_mu);
    NvtxRange range("pcg_solve_batched");
    Plan* pp = nullptr;
    mhd_status_t sp = prepare(n, grids, alpha, b, x, params, &pp);
    if (sp != MHD_OK) return sp;
    Plan& P = *pp;
    cudaStream_t st = grids[0]->stream;
    if (cudaGraphLaunch(P.graph, st) != cudaSuccess) return fail(MHD_ERR_CUDA, "pcg_solve_batched: graph launch");
    BarrierState hb;
    if (cudaMemcpyAsync(&hb, P.d_bar, sizeof(hb), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(MHD_ERR_CUDA, "pcg_solve_batched: sync failed");
    mhd_status_t worst = MHD_OK;
    for (int s = 0; s < n; s++) {
        PcgScalars h;
        cudaMemcpy(&h, grids[s]->sc, sizeof(h), cudaMemcpyDeviceToHost);
        if (iters) iters[s] = h.iter;
        if (relres) relres[s] = (h.bb > 0) ? std::sqrt(h.rr) / std::sqrt(h.bb) : 0.0;
        if (h.done == 3 && worst == MHD_OK) worst = MHD_ERR_NONFINITE;
        if ((h.done == 2 || h.done == 4) && worst == MHD_OK) worst = MHD_ERR_NOCONV;
    }
    if (hb.err) return fail(MHD_ERR_TIMEOUT, "pcg_solve_batched: a grid barrier timed out");
    if (worst == MHD_ERR_NOCONV) return fail(worst, "pcg_solve_batched: a system missed the tolerance");
    if (worst == MHD_ERR_NONFINITE) return fail(worst, "pcg_solve_batched: non-finite value");
    return MHD_OK;
}

extern "C" mhd_status_t pcg_batch_reserve(int n, const mhd_grid_t* grids, const double* alpha,
                                          const double* const* b, double* const* x, const mhd_params_t* params) {
    std::lock_guard<std::mutex> lk(g_mu);
    Plan* pp = nullptr;
    return prepare(n, grids, alpha, b, x, params, &pp);
}
