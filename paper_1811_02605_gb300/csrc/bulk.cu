// FP32 CG iteration of the mixed-precision inner solve as a pair of plane-marching kernels whose
// input rows are staged in shared memory by bulk asynchronous copies (cp.async.bulk, completion
// on an mbarrier), a ring of planes in flight per CTA (3 in kernel A, 4 in kernel B).
//
// The arithmetic is that of the recompute pair in pcg.cu (k_pfold32 / k_rupd32):
//   A: p~ = r~ + beta p~_old on the tile and its neighbours, <p~, A~ p~>, p~ stored (3 passes);
//   B: q~ = A~ p~ from the stored p~, r~ -= alpha q~, <r~, r~>, sum dg r~^2, and on every second
//      iteration x~ = fma(alpha_k, p~_k, fma(alpha_{k-1}, p~_{k-1}, x~)) (4.5 passes on average).
// What changes is how the neighbours reach the threads. The grid-stride kernels fetch every value
// seven times through L2 (once as a centre and once for each neighbour), which binds them on L2
// traffic rather than on HBM. Here a CTA owns one component and TJ theta rows of full phi rows and
// walks along r; a thread owns one float4 of one row, so its r neighbours are the previous and next
// plane in its registers and its theta and phi neighbours are in a shared-memory tile of the plane.
// Each input row is fetched once per CTA (the halo rows j0-1 and j0+TJ once more by the
// neighbouring tile, which works on the same planes at the same time, so mostly from L2).
//
// Work units: (slab of planes, component, row tile), slab-major, handed round-robin to a grid of
// resident CTAs. Each unit primes its ring with its first planes and drains it at its end, so no
// copy is ever in flight when a CTA leaves a unit.
//
// Every mbarrier wait is bounded (a %globaltimer budget). A CTA whose wait runs out sets
// PcgScalars::done = 6, waits (bounded again) for the copies it has issued, and returns; every
// later kernel of the solve then returns at once and the solver reports MHD_ERR_TIMEOUT.
//
// Requirements (checked on the host, bulk32_ok): np a multiple of 128 and at most 512 (a CTA is
// (TJ+2) np/4 threads); rows of np floats are then 16-byte aligned and a multiple of 16 bytes, as
// the bulk copy needs.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;  // mbarrier wait budget (2 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of the given parity to complete; false when the budget runs out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    const unsigned long long t0 = now_ns();
    for (;;) {
        uint32_t ok;
        // the suspend-time hint lets the hardware park the thread until the phase completes (or
        // 0.1 ms pass) instead of spinning on the barrier
        asm volatile(
            "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, %3;\n selp.b32 %0, 1, 0, P1;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity), "r"(100000u)
            : "memory");
        if (ok) return true;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}

struct Unit {
    int c, i0, i1, j0;
};

__device__ __forceinline__ Unit unit_of(const Dims& d, int u, int slab, int tj) {
    const int ntj = (d.nt + tj - 1) / tj;
    const int per_slab = 3 * ntj;
    Unit q;
    const int s = u / per_slab;
    const int rest = u - s * per_slab;
    q.c = rest / ntj;
    q.j0 = (rest - q.c * ntj) * tj;
    q.i0 = s * slab;
    q.i1 = min(d.nr, q.i0 + slab);
    return q;
}

// per-thread compensated FP32 sum (Neumaier), handed to FP64 once per thread
struct Acc32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

__device__ __forceinline__ void ld4s(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}

}  // namespace

// thread 0 issues the copies of one plane of a unit into ring slot `slot`: for each theta row
// j0-1 .. j0+TJ inside the grid, one row of np floats from each source array (narr of them, the
// rows of array a at stage offset a (TJ+2) np). Planes outside the grid are not copied; the
// barrier's phase then completes on the arrival alone.
template <int TJ>
__device__ __forceinline__ void issue_plane(const Dims& d, int c, int j0, int plane, float* st, uint64_t* bar,
                                         const float* src0, const float* src1, int narr) {
    const int np = d.np, nt = d.nt;
    uint32_t nrow = 0;
    if (plane >= 0 && plane < d.nr)
        for (int jj = 0; jj < TJ + 2; jj++) {
            const int j = j0 - 1 + jj;
            nrow += (j >= 0 && j < nt) ? 1u : 0u;
        }
    mbar_expect(bar, (uint32_t)narr * nrow * (uint32_t)np * 4u);
    if (plane < 0 || plane >= d.nr) return;
    for (int jj = 0; jj < TJ + 2; jj++) {
        const int j = j0 - 1 + jj;
        if (j < 0 || j >= nt) continue;
        const long long g0 = c * d.N + ((long long)plane * nt + j) * np;
        bulk_g2s(st + (long long)jj * np, src0 + g0, (uint32_t)np * 4u, bar);
        if (narr > 1) bulk_g2s(st + (long long)(TJ + 2 + jj) * np, src1 + g0, (uint32_t)np * 4u, bar);
    }
}

// ------------------------------------------------------------------------------------------
// Thread layout of both kernels: (TJ + 2) rows x ncol = np/4 columns; thread (row, col) owns the
// float4 at phi 4 col of theta row j0 - 1 + row. Rows 0 and TJ + 1 are the halo rows: their threads
// form p~ there for the theta neighbours and do no stencil. Per plane step every thread forms its
// p~ value, stores it in the plane tile P (triple-buffered over the steps, so one barrier per
// step suffices), and the interior threads evaluate the stencil of the previous plane from its
// tile (theta and phi neighbours) and their registers (the planes before and after).
// ------------------------------------------------------------------------------------------
constexpr int kTJ = 4;
constexpr int kThreadsMax = (kTJ + 2) * 128;   // np <= 512

// A: p~ = r~ + beta p~_old, <p~, A~ p~>, p~ stored. Shared memory: SA stages x {r~, p~_old} x
// (TJ+2) rows of np floats, then the plane tile [3][TJ+2][np].
constexpr int kStagesA = 3;
__global__ void __launch_bounds__(kThreadsMax, 2) k_bulk_a32(Dims d, const float* __restrict__ r,
                                                             float* __restrict__ pbuf, OpTab<float> t,
                                                             PcgScalars* sc, double* __restrict__ partials, int nc,
                                                             int slab, int units) {
    constexpr int TJ = kTJ, S = kStagesA;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[S];
    if (sc->done) return;
    const int np = d.np, nt = d.nt, nr = d.nr;
    const int ncol = np / 4;
    const int row = threadIdx.x / ncol, col = threadIdx.x - row * ncol;
    const int k0 = 4 * col;
    const bool inner = (row >= 1 && row <= TJ);
    float* stage = reinterpret_cast<float*>(smem_raw);
    const long long stage_floats = 2LL * (TJ + 2) * np;
    float* tile = stage + S * stage_floats;   // [3][TJ+2][np]
    const long long tile_floats = (long long)(TJ + 2) * np;
    const long long N = d.N;
    const long long plane_sz = (long long)nt * np;
    const int par = sc->par;
    const float* __restrict__ pold = pbuf + (long long)par * 3 * N;
    float* __restrict__ pnew = pbuf + (long long)(1 - par) * 3 * N;
    const float beta = (float)sc->beta;
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; q++) mbar_init(&full[q], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](const Unit& U, long long q, int plane) {
        const int slot = (int)(q % S);
        issue_plane<TJ>(d, U.c, U.j0, plane, stage + slot * stage_floats, &full[slot], r, pold, 2);
    };

    Acc32 acc;
    long long gstep = 0, issued = 0, fail_step = 0;
    bool failed = false;
    for (int u = blockIdx.x; u < units && !failed; u += gridDim.x) {
        const Unit U = unit_of(d, u, slab, TJ);
        if (U.c >= nc) continue;
        const int nsteps = (U.i1 - U.i0) + 2;   // planes i0-1 .. i1
        if (threadIdx.x == 0)
            for (int q = 0; q < S && q < nsteps; q++) {
                issue(U, gstep + q, U.i0 - 1 + q);
                issued++;
            }
        const int j = U.j0 - 1 + row;
        const bool jvalid = (j >= 0 && j < nt);
        float pm[4] = {0.f, 0.f, 0.f, 0.f}, pc[4] = {0.f, 0.f, 0.f, 0.f}, pn[4];
        for (int s = 0; s < nsteps; s++) {
            const int plane = U.i0 - 1 + s;
            const long long gs = gstep + s;
            const int slot = (int)(gs % S);
            const bool ok = mbar_wait(&full[slot], (uint32_t)((gs / S) & 1));
            if (ok && jvalid && plane >= 0 && plane < nr) {
                const float* st = stage + slot * stage_floats;
                float rv[4], pv[4];
                ld4s(st + (long long)row * np + k0, rv);
                ld4s(st + (long long)(TJ + 2 + row) * np + k0, pv);
#pragma unroll
                for (int e = 0; e < 4; e++) pn[e] = fmaf(beta, pv[e], rv[e]);
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++) pn[e] = 0.f;
            }
            float* tw = tile + (gs % 3) * tile_floats;
            *reinterpret_cast<float4*>(tw + (long long)row * np + k0) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            if (__syncthreads_or(!ok)) {
                failed = true;
                fail_step = gs;
                break;
            }
            if (threadIdx.x == 0 && s + S < nsteps) {
                issue(U, gs + S, plane + S);
                issued++;
            }
            const int ic = plane - 1;   // the plane whose neighbours are all in place now
            if (s >= 2 && inner && j < nt) {
                const float* tr = tile + ((gs + 2) % 3) * tile_floats + (long long)row * np;   // plane ic
                const float cr_lo = t.ar[ic * nt + j], cr_hi = t.ar[(ic + 1) * nt + j];
                const float ct_lo = t.at[ic * (nt + 1) + j], ct_hi = t.at[ic * (nt + 1) + j + 1];
                const float cp = t.ap[ic * nt + j];
                const float ukm = tr[(k0 == 0) ? np - 1 : k0 - 1];
                const float ukp = tr[(k0 + 4 == np) ? 0 : k0 + 4];
                float up[4], dn[4];
                ld4s(tr - np + k0, up);
                ld4s(tr + np + k0, dn);
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float left = (e == 0) ? ukm : pc[e - 1];
                    const float right = (e == 3) ? ukp : pc[e + 1];
                    o[e] = fmaf(-cp, left + right, pc[e]);
                    o[e] = fmaf(-cr_lo, pm[e], o[e]);
                    o[e] = fmaf(-cr_hi, pn[e], o[e]);
                    o[e] = fmaf(-ct_lo, up[e], o[e]);
                    o[e] = fmaf(-ct_hi, dn[e], o[e]);
                }
                float part = pc[0] * o[0];
#pragma unroll
                for (int e = 1; e < 4; e++) part = fmaf(pc[e], o[e], part);
                acc.add(part);
                const long long g0 = U.c * N + (long long)ic * plane_sz + (long long)j * np + k0;
                *reinterpret_cast<float4*>(pnew + g0) = make_float4(pc[0], pc[1], pc[2], pc[3]);
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                pm[e] = pc[e];
                pc[e] = pn[e];
            }
        }
        if (!failed) gstep += nsteps;
    }
    if (failed) {
        // record the timeout, then wait (bounded) for the copies this CTA has issued
        if (threadIdx.x == 0) {
            atomicExch(&sc->done, 6);
            for (long long q = fail_step; q < issued; q++)
                if (!mbar_wait(&full[q % S], (uint32_t)((q / S) & 1))) break;
        }
        __syncthreads();
        return;
    }
    double val[1] = {acc.get()}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double pq = out[0];
        sc->pq = pq;
        sc->par = 1 - par;
        if (sc->done == 0) {
            if (!isfinite(pq)) sc->done = 3;
            else if (!(pq > 0.0)) sc->done = 4;
            else sc->alpha = sc->rho / pq;
        }
    }
}

// B: q~ = A~ p~ from the stored p~, r~ -= alpha q~, dots, x~ every second iteration. Shared memory:
// SB stages x (TJ+2) rows of p~, then the plane tile; r~ is read at the cell with a plain float4
// load issued one plane step ahead, x~ and p~_{k-1} (every second iteration) when they are used.
constexpr int kStagesB = 4;
__global__ void __launch_bounds__(kThreadsMax, 1) k_bulk_b32(Dims d, float* __restrict__ x, float* __restrict__ r,
                                                             const float* __restrict__ pbuf, OpTab<float> t,
                                                             const double* __restrict__ dg, PcgScalars* sc,
                                                             double* __restrict__ partials, int nc, int slab,
                                                             int units) {
    constexpr int TJ = kTJ, S = kStagesB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[S];
    if (sc->done) return;
    const int np = d.np, nt = d.nt, nr = d.nr;
    const int ncol = np / 4;
    const int row = threadIdx.x / ncol, col = threadIdx.x - row * ncol;
    const int k0 = 4 * col;
    const bool inner = (row >= 1 && row <= TJ);
    float* stage = reinterpret_cast<float*>(smem_raw);
    const long long stage_floats = (long long)(TJ + 2) * np;
    float* tile = stage + S * stage_floats;
    const long long tile_floats = (long long)(TJ + 2) * np;
    const long long N = d.N;
    const long long plane_sz = (long long)nt * np;
    const int par = sc->par;
    const float* __restrict__ p = pbuf + (long long)par * 3 * N;
    const float* __restrict__ pprev = pbuf + (long long)(1 - par) * 3 * N;
    const float al = (float)sc->alpha;
    const float axp = (float)sc->ax;
    const bool pair = (sc->ax != 0.0);
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; q++) mbar_init(&full[q], 1);
        mbar_fence_init();
    }
    __syncthreads();

    auto issue = [&](const Unit& U, long long q, int plane) {
        const int slot = (int)(q % S);
        issue_plane<TJ>(d, U.c, U.j0, plane, stage + slot * stage_floats, &full[slot], p, nullptr, 1);
    };

    Acc32 a_rho;
    double a_rr = 0.0;
    long long gstep = 0, issued = 0, fail_step = 0;
    bool failed = false;
    for (int u = blockIdx.x; u < units && !failed; u += gridDim.x) {
        const Unit U = unit_of(d, u, slab, TJ);
        if (U.c >= nc) continue;
        const int nsteps = (U.i1 - U.i0) + 2;
        if (threadIdx.x == 0)
            for (int q = 0; q < S && q < nsteps; q++) {
                issue(U, gstep + q, U.i0 - 1 + q);
                issued++;
            }
        const int j = U.j0 - 1 + row;
        const bool jvalid = (j >= 0 && j < nt);
        const bool mine = inner && jvalid;   // this thread updates r~ (and x~) of its cell column
        float pm[4] = {0.f, 0.f, 0.f, 0.f}, pc[4] = {0.f, 0.f, 0.f, 0.f}, pn[4];
        float rnx[4] = {0.f, 0.f, 0.f, 0.f};
        for (int s = 0; s < nsteps; s++) {
            const int plane = U.i0 - 1 + s;
            const long long gs = gstep + s;
            const int slot = (int)(gs % S);
            const bool ok = mbar_wait(&full[slot], (uint32_t)((gs / S) & 1));
            if (ok && jvalid && plane >= 0 && plane < nr) {
                ld4s(stage + slot * stage_floats + (long long)row * np + k0, pn);
            } else {
#pragma unroll
                for (int e = 0; e < 4; e++) pn[e] = 0.f;
            }
            float* tw = tile + (gs % 3) * tile_floats;
            *reinterpret_cast<float4*>(tw + (long long)row * np + k0) = make_float4(pn[0], pn[1], pn[2], pn[3]);
            if (__syncthreads_or(!ok)) {
                failed = true;
                fail_step = gs;
                break;
            }
            if (threadIdx.x == 0 && s + S < nsteps) {
                issue(U, gs + S, plane + S);
                issued++;
            }
            // r~ of this step's plane, evaluated at the next step
            float rcur[4];
#pragma unroll
            for (int e = 0; e < 4; e++) rcur[e] = rnx[e];
            if (mine && plane >= U.i0 && plane < U.i1)
                ld4s(r + U.c * N + (long long)plane * plane_sz + (long long)j * np + k0, rnx);
            const int ic = plane - 1;
            if (s >= 2 && mine) {
                const long long g0 = U.c * N + (long long)ic * plane_sz + (long long)j * np + k0;
                float xcur[4], ppcur[4];
                if (pair) {
                    ld4s(x + g0, xcur);
                    ld4s(pprev + g0, ppcur);
                }
                const float* tr = tile + ((gs + 2) % 3) * tile_floats + (long long)row * np;
                const float cr_lo = t.ar[ic * nt + j], cr_hi = t.ar[(ic + 1) * nt + j];
                const float ct_lo = t.at[ic * (nt + 1) + j], ct_hi = t.at[ic * (nt + 1) + j + 1];
                const float cp = t.ap[ic * nt + j];
                const float ukm = tr[(k0 == 0) ? np - 1 : k0 - 1];
                const float ukp = tr[(k0 + 4 == np) ? 0 : k0 + 4];
                float up[4], dn[4];
                ld4s(tr - np + k0, up);
                ld4s(tr + np + k0, dn);
                float rv[4], rs = 0.f;
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const float left = (e == 0) ? ukm : pc[e - 1];
                    const float right = (e == 3) ? ukp : pc[e + 1];
                    float o = fmaf(-cp, left + right, pc[e]);
                    o = fmaf(-cr_lo, pm[e], o);
                    o = fmaf(-cr_hi, pn[e], o);
                    o = fmaf(-ct_lo, up[e], o);
                    o = fmaf(-ct_hi, dn[e], o);
                    rv[e] = fmaf(-al, o, rcur[e]);
                    rs = fmaf(rv[e], rv[e], rs);
                }
                *reinterpret_cast<float4*>(r + g0) = make_float4(rv[0], rv[1], rv[2], rv[3]);
                if (pair) {
                    float xv[4];
#pragma unroll
                    for (int e = 0; e < 4; e++) xv[e] = fmaf(al, pc[e], fmaf(axp, ppcur[e], xcur[e]));
                    *reinterpret_cast<float4*>(x + g0) = make_float4(xv[0], xv[1], xv[2], xv[3]);
                }
                a_rho.add(rs);
                a_rr = fma(dg[ic * nt + j], (double)rs, a_rr);
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                pm[e] = pc[e];
                pc[e] = pn[e];
            }
        }
        if (!failed) gstep += nsteps;
    }
    if (failed) {
        if (threadIdx.x == 0) {
            atomicExch(&sc->done, 6);
            for (long long q = fail_step; q < issued; q++)
                if (!mbar_wait(&full[q % S], (uint32_t)((q / S) & 1))) break;
        }
        __syncthreads();
        return;
    }
    double val[2] = {a_rho.get(), a_rr}, out[2];
    if (reduce_last<2>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double rho = out[0], rr = out[1];
        sc->iter += 1;
        sc->total_iter += 1;
        sc->rho_prev = sc->rho;
        sc->beta = rho / sc->rho;
        sc->rho = rho;
        sc->rr = rr;
        sc->ax = pair ? 0.0 : sc->alpha;
        if (sc->done == 0) {
            if (!isfinite(rr) || !isfinite(rho)) sc->done = 3;
            else if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
            else if (sc->iter >= sc->max_iter) sc->done = 2;
        }
    }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
namespace {
size_t smem_a(int np) {
    return sizeof(float) * ((size_t)kStagesA * 2 * (kTJ + 2) * np + (size_t)3 * (kTJ + 2) * np);
}
size_t smem_b(int np) { return sizeof(float) * ((size_t)kStagesB * (kTJ + 2) * np + (size_t)3 * (kTJ + 2) * np); }

int units_of(const mhd_grid_s* g, int slab) {
    const int ntj = (g->d.nt + kTJ - 1) / kTJ;
    return ((g->d.nr + slab - 1) / slab) * 3 * ntj;
}

// resident CTAs per SM of a kernel at its shared-memory size (per kernel, per size)
template <auto K>
int resident(size_t smem, int threads) {
    static size_t last_smem = 0;
    static int last_threads = 0, last = 0;
    if (smem == last_smem && threads == last_threads && last > 0) return last;
    if (cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    last_smem = smem;
    last_threads = threads;
    last = b;
    return b;
}
}  // namespace

bool bulk32_ok(const mhd_grid_s* g) {
    const int np = g->d.np;
    if ((np % 128) != 0 || (kTJ + 2) * (np / 4) > kThreadsMax) return false;
    return smem_a(np) <= 200 * 1024 && smem_b(np) <= 200 * 1024;
}

// slab: planes per work unit
void enqueue_bulk32(mhd_grid_s* g, cudaStream_t st, int nc, int slab) {
    const Dims d = g->d;
    const int threads = (kTJ + 2) * (d.np / 4);
    const int units = units_of(g, slab);
    const size_t sa = smem_a(d.np), sb = smem_b(d.np);
    const int ra = resident<k_bulk_a32>(sa, threads);
    const int rb = resident<k_bulk_b32>(sb, threads);
    const int ga = std::max(1, std::min(units, std::min(kMaxBlocks, std::max(ra, 1) * g->num_sms)));
    const int gb = std::max(1, std::min(units, std::min(kMaxBlocks, std::max(rb, 1) * g->num_sms)));
    int s = prof_begin(g, st, MHD_KERNEL_PFOLD32);
    k_bulk_a32<<<ga, threads, sa, st>>>(d, g->r32, g->p32, g->t32, g->sc, g->partials, nc, slab, units);
    prof_end(g, st, s);
    s = prof_begin(g, st, MHD_KERNEL_RUPD32);
    k_bulk_b32<<<gb, threads, sb, st>>>(d, g->x32, g->r32, g->p32, g->t32, g->tu.dg, g->sc, g->partials, nc, slab,
                                        units);
    prof_end(g, st, s);
}

}  // namespace mhd
