// FP32 CG iteration in two plane-marching kernels (the inner solve of the mixed-precision path).
//
// The split form (p update, stencil, update) moves 10 passes of a 3-component vector per
// iteration. Here:
//   A: p_new = r + beta p_old at every point the stencil needs, q = A~ p_new, <p_new, q>;
//      writes p_new only (3 passes: r, p_old in, p_new out)
//   B: q = A~ p_new again (identical arithmetic, so bit-identical q), x += alpha p, r -= alpha q,
//      <r~, r~> and sum dg r~^2 (5 passes: x, r, p_new in, x, r out)
// 8 passes in all. p is double-buffered (A reads one buffer and writes the other); the buffer in
// use is a device-side parity flipped by B's last CTA, so an inner solve that stops after any
// number of iterations leaves the next one reading the right buffer.
//
// Tiling: a CTA owns TJ theta rows x 128 phi points of the (theta, phi) plane and walks along r
// over a slab of planes. Each interior warp keeps its row's values at planes i-1, i, i+1 in
// registers; the plane i tile plus one halo row above and below (two extra warps) and one halo
// column on each side sits in shared memory for the theta and phi neighbours. Every p value of
// plane i is computed once per CTA (halo rows and columns are recomputed by the neighbouring CTA),
// so HBM sees each vector about once per kernel.
#include <cmath>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

namespace {

constexpr int TJ = 8;             // interior rows per CTA
constexpr int WARPS = TJ + 2;     // plus one halo row above and below
constexpr int TK = 128;           // phi points per CTA (32 lanes x float4)
constexpr int SW = TK + 8;        // shared row stride: halo-left at 3, interior at 4..131, halo-right at 132

struct AccF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

struct Tile {
    int i0, i1, j0, k0;
};

__device__ __forceinline__ Tile tile_of(const Dims& d, int slab) {
    const int tiles_k = d.np / TK;
    const int tiles_j = (d.nt + TJ - 1) / TJ;
    int b = blockIdx.x;
    const int tk = b % tiles_k;
    b /= tiles_k;
    const int tj = b % tiles_j;
    const int sl = b / tiles_j;
    Tile t;
    t.k0 = tk * TK;
    t.j0 = tj * TJ;
    t.i0 = sl * slab;
    t.i1 = min(d.nr, t.i0 + slab);
    return t;
}

// q at the 4 points of this lane (row w of the tile): o = p - ap (left + right) - at_lo up -
// at_hi down - ar_lo pm - ar_hi pn
__device__ __forceinline__ void stencil4(const float* __restrict__ smc, int w, int lane, const float (&pm)[4],
                                         const float (&pc)[4], const float (&pn)[4], float ar_lo, float ar_hi,
                                         float at_lo, float at_hi, float ap, float (&q)[4]) {
    const float* row = smc + w * SW + 4 + lane * 4;
    const float4 up = *reinterpret_cast<const float4*>(row - SW);
    const float4 dn = *reinterpret_cast<const float4*>(row + SW);
    const float lft = row[-1], rgt = row[4];
    const float u[4] = {up.x, up.y, up.z, up.w};
    const float dd[4] = {dn.x, dn.y, dn.z, dn.w};
#pragma unroll
    for (int e = 0; e < 4; e++) {
        const float l = (e == 0) ? lft : pc[e - 1];
        const float r = (e == 3) ? rgt : pc[e + 1];
        float o = fmaf(-ap, l + r, pc[e]);
        o = fmaf(-at_lo, u[e], o);
        o = fmaf(-at_hi, dd[e], o);
        o = fmaf(-ar_lo, pm[e], o);
        o = fmaf(-ar_hi, pn[e], o);
        q[e] = o;
    }
}

}  // namespace

// A: fused p update + stencil + <p, q>   (NC components, unrolled so the plane values stay in
// registers)
template <int NC>
__global__ void __launch_bounds__(WARPS * 32, 2) k_tiled_a32(Dims d, const float* __restrict__ r,
                                                              float* __restrict__ pbuf, OpTab<float> t,
                                                              PcgScalars* sc, double* __restrict__ partials,
                                                              int slab) {
    __shared__ __align__(16) float sm[3][WARPS * SW];
    if (sc->done) return;
    const long long N = d.N;
    const float beta = (float)sc->beta;
    const int par = sc->par;
    const float* __restrict__ pold = pbuf + (long long)par * 3 * N;
    float* __restrict__ pnew = pbuf + (long long)(1 - par) * 3 * N;
    const Tile T = tile_of(d, slab);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = T.j0 - 1 + w;
    const bool row_ok = (j >= 0 && j < d.nt);
    const bool interior = row_ok && w >= 1 && w <= TJ;
    const int kq = T.k0 + lane * 4;
    const int kl = (T.k0 == 0) ? d.np - 1 : T.k0 - 1;
    const int kr = (T.k0 + TK == d.np) ? 0 : T.k0 + TK;
    const long long plane = (long long)d.nt * d.np;

    auto pnew4 = [&](int i, int c, float (&o)[4]) {
        const long long base = c * N + (long long)i * plane + (long long)j * d.np + kq;
        const float4 rv = *reinterpret_cast<const float4*>(r + base);
        const float4 pv = *reinterpret_cast<const float4*>(pold + base);
        o[0] = fmaf(beta, pv.x, rv.x);
        o[1] = fmaf(beta, pv.y, rv.y);
        o[2] = fmaf(beta, pv.z, rv.z);
        o[3] = fmaf(beta, pv.w, rv.w);
    };
    auto pnew1 = [&](int i, int c, int k) {
        const long long idx = c * N + (long long)i * plane + (long long)j * d.np + k;
        return fmaf(beta, pold[idx], r[idx]);
    };

    float pm[3][4], pc[3][4], pn[3][4];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int e = 0; e < 4; e++) pm[c][e] = pc[c][e] = pn[c][e] = 0.f;
    if (row_ok && T.i0 < T.i1) {
#pragma unroll
        for (int c = 0; c < NC; c++) {
            pnew4(T.i0, c, pc[c]);
            if (interior && T.i0 > 0) pnew4(T.i0 - 1, c, pm[c]);
        }
    }
    AccF acc;
    for (int i = T.i0; i < T.i1; i++) {
        if (interior && i + 1 < d.nr) {
#pragma unroll
        for (int c = 0; c < NC; c++) pnew4(i + 1, c, pn[c]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int e = 0; e < 4; e++) pn[c][e] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < NC; c++) {
            float* rowp = &sm[c][w * SW + 4 + lane * 4];
            *reinterpret_cast<float4*>(rowp) = make_float4(pc[c][0], pc[c][1], pc[c][2], pc[c][3]);
            if (lane == 0) sm[c][w * SW + 3] = row_ok ? pnew1(i, c, kl) : 0.f;
            if (lane == 31) sm[c][w * SW + 4 + TK] = row_ok ? pnew1(i, c, kr) : 0.f;
        }
        __syncthreads();
        if (interior) {
            const float ar_lo = t.ar[i * d.nt + j], ar_hi = t.ar[(i + 1) * d.nt + j];
            const float at_lo = t.at[i * (d.nt + 1) + j], at_hi = t.at[i * (d.nt + 1) + j + 1];
            const float ap = t.ap[i * d.nt + j];
#pragma unroll
        for (int c = 0; c < NC; c++) {
                float q[4];
                stencil4(sm[c], w, lane, pm[c], pc[c], pn[c], ar_lo, ar_hi, at_lo, at_hi, ap, q);
                float part = pc[c][0] * q[0];
                part = fmaf(pc[c][1], q[1], part);
                part = fmaf(pc[c][2], q[2], part);
                part = fmaf(pc[c][3], q[3], part);
                acc.add(part);
                const long long base = c * N + (long long)i * plane + (long long)j * d.np + kq;
                *reinterpret_cast<float4*>(pnew + base) = make_float4(pc[c][0], pc[c][1], pc[c][2], pc[c][3]);
            }
        }
        __syncthreads();
        if (interior) {
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    pm[c][e] = pc[c][e];
                    pc[c][e] = pn[c][e];
                }
        } else if (row_ok && i + 1 < T.i1) {
#pragma unroll
        for (int c = 0; c < NC; c++) pnew4(i + 1, c, pc[c]);
        }
    }
    double val[1] = {acc.get()}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double pq = out[0];
        sc->pq = pq;
        if (!isfinite(pq)) sc->done = 3;
        else if (!(pq > 0.0)) sc->done = 4;
        else sc->alpha = sc->rho / pq;
    }
}

// B: q = A~ p_new (recomputed), x += alpha p, r -= alpha q, dots, stop test
template <int NC>
__global__ void __launch_bounds__(WARPS * 32, 2) k_tiled_b32(Dims d, float* __restrict__ x,
                                                              float* __restrict__ r, const float* __restrict__ pbuf,
                                                              OpTab<float> t, const double* __restrict__ dg,
                                                              PcgScalars* sc, double* __restrict__ partials,
                                                              int slab) {
    __shared__ __align__(16) float sm[3][WARPS * SW];
    if (sc->done) return;
    const long long N = d.N;
    const float al = (float)sc->alpha;
    const int par = sc->par;
    const float* __restrict__ p = pbuf + (long long)(1 - par) * 3 * N;
    const Tile T = tile_of(d, slab);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = T.j0 - 1 + w;
    const bool row_ok = (j >= 0 && j < d.nt);
    const bool interior = row_ok && w >= 1 && w <= TJ;
    const int kq = T.k0 + lane * 4;
    const int kl = (T.k0 == 0) ? d.np - 1 : T.k0 - 1;
    const int kr = (T.k0 + TK == d.np) ? 0 : T.k0 + TK;
    const long long plane = (long long)d.nt * d.np;
    auto ld4 = [&](int i, int c, float (&o)[4]) {
        const float4 v = *reinterpret_cast<const float4*>(p + c * N + (long long)i * plane + (long long)j * d.np + kq);
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
        o[3] = v.w;
    };
    float pm[3][4], pc[3][4], pn[3][4];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int e = 0; e < 4; e++) pm[c][e] = pc[c][e] = pn[c][e] = 0.f;
    if (row_ok && T.i0 < T.i1) {
#pragma unroll
        for (int c = 0; c < NC; c++) {
            ld4(T.i0, c, pc[c]);
            if (interior && T.i0 > 0) ld4(T.i0 - 1, c, pm[c]);
        }
    }
    AccF a_rho;
    double a_rr = 0.0;
    for (int i = T.i0; i < T.i1; i++) {
        if (interior && i + 1 < d.nr) {
#pragma unroll
        for (int c = 0; c < NC; c++) ld4(i + 1, c, pn[c]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int e = 0; e < 4; e++) pn[c][e] = 0.f;
        }
#pragma unroll
        for (int c = 0; c < NC; c++) {
            *reinterpret_cast<float4*>(&sm[c][w * SW + 4 + lane * 4]) = make_float4(pc[c][0], pc[c][1], pc[c][2], pc[c][3]);
            const long long rowbase = c * N + (long long)i * plane + (long long)j * d.np;
            if (lane == 0) sm[c][w * SW + 3] = row_ok ? p[rowbase + kl] : 0.f;
            if (lane == 31) sm[c][w * SW + 4 + TK] = row_ok ? p[rowbase + kr] : 0.f;
        }
        __syncthreads();
        if (interior) {
            const float ar_lo = t.ar[i * d.nt + j], ar_hi = t.ar[(i + 1) * d.nt + j];
            const float at_lo = t.at[i * (d.nt + 1) + j], at_hi = t.at[i * (d.nt + 1) + j + 1];
            const float ap = t.ap[i * d.nt + j];
            float rs = 0.f;
#pragma unroll
        for (int c = 0; c < NC; c++) {
                float q[4];
                stencil4(sm[c], w, lane, pm[c], pc[c], pn[c], ar_lo, ar_hi, at_lo, at_hi, ap, q);
                const long long base = c * N + (long long)i * plane + (long long)j * d.np + kq;
                float4 xv = *reinterpret_cast<const float4*>(x + base);
                float4 rv = *reinterpret_cast<const float4*>(r + base);
                xv.x = fmaf(al, pc[c][0], xv.x);
                xv.y = fmaf(al, pc[c][1], xv.y);
                xv.z = fmaf(al, pc[c][2], xv.z);
                xv.w = fmaf(al, pc[c][3], xv.w);
                rv.x = fmaf(-al, q[0], rv.x);
                rv.y = fmaf(-al, q[1], rv.y);
                rv.z = fmaf(-al, q[2], rv.z);
                rv.w = fmaf(-al, q[3], rv.w);
                *reinterpret_cast<float4*>(x + base) = xv;
                *reinterpret_cast<float4*>(r + base) = rv;
                rs = fmaf(rv.x, rv.x, rs);
                rs = fmaf(rv.y, rv.y, rs);
                rs = fmaf(rv.z, rv.z, rs);
                rs = fmaf(rv.w, rv.w, rs);
            }
            a_rho.add(rs);
            a_rr = fma(dg[i * d.nt + j], (double)rs, a_rr);
        }
        __syncthreads();
        if (interior) {
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    pm[c][e] = pc[c][e];
                    pc[c][e] = pn[c][e];
                }
        } else if (row_ok && i + 1 < T.i1) {
#pragma unroll
        for (int c = 0; c < NC; c++) ld4(i + 1, c, pc[c]);
        }
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
        sc->par = 1 - sc->par;
        if (!isfinite(rr) || !isfinite(rho)) sc->done = 3;
        else if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
        else if (sc->iter >= sc->max_iter) sc->done = 2;
    }
}

bool tiled32_ok(const mhd_grid_s* g) { return (g->d.np % TK) == 0; }

int tiled32_blocks(const mhd_grid_s* g, int slab) {
    const int tiles_k = g->d.np / TK;
    const int tiles_j = (g->d.nt + TJ - 1) / TJ;
    const int slabs = (g->d.nr + slab - 1) / slab;
    return tiles_k * tiles_j * slabs;
}

void enqueue_tiled32(mhd_grid_s* g, cudaStream_t st, int nc, int slab, int prof_a, int prof_b) {
    const int blocks = tiled32_blocks(g, slab);
    int s = prof_begin(g, st, prof_a);
    if (nc == 3) k_tiled_a32<3><<<blocks, WARPS * 32, 0, st>>>(g->d, g->r32, g->p32, g->t32, g->sc, g->partials, slab);
    else if (nc == 2) k_tiled_a32<2><<<blocks, WARPS * 32, 0, st>>>(g->d, g->r32, g->p32, g->t32, g->sc, g->partials, slab);
    else k_tiled_a32<1><<<blocks, WARPS * 32, 0, st>>>(g->d, g->r32, g->p32, g->t32, g->sc, g->partials, slab);
    prof_end(g, st, s);
    s = prof_begin(g, st, prof_b);
    if (nc == 3)
        k_tiled_b32<3><<<blocks, WARPS * 32, 0, st>>>(g->d, g->x32, g->r32, g->p32, g->t32, g->tu.dg, g->sc, g->partials, slab);
    else if (nc == 2)
        k_tiled_b32<2><<<blocks, WARPS * 32, 0, st>>>(g->d, g->x32, g->r32, g->p32, g->t32, g->tu.dg, g->sc, g->partials, slab);
    else
        k_tiled_b32<1><<<blocks, WARPS * 32, 0, st>>>(g->d, g->x32, g->r32, g->p32, g->t32, g->tu.dg, g->sc, g->partials, slab);
    prof_end(g, st, s);
}

// ---------------------------------------------------------------------------------------------
// FP64: fused p update + stencil + <p, q> with q stored (the FP64 iteration is bound by its FP64
// instruction count, so q is kept rather than recomputed). Replaces the split p-update and
// stencil kernels: the p update then costs ~1.25 FMA per point inside an ALU-bound kernel
// instead of a separate memory-bound pass.
// ---------------------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ void ld4d(const double* __restrict__ a, double (&o)[4]) {
    const double2 u = *reinterpret_cast<const double2*>(a);
    const double2 v = *reinterpret_cast<const double2*>(a + 2);
    o[0] = u.x;
    o[1] = u.y;
    o[2] = v.x;
    o[3] = v.y;
}
__device__ __forceinline__ void st4d(double* __restrict__ a, const double (&o)[4]) {
    *reinterpret_cast<double2*>(a) = make_double2(o[0], o[1]);
    *reinterpret_cast<double2*>(a + 2) = make_double2(o[2], o[3]);
}

}  // namespace

__global__ void __launch_bounds__(WARPS * 32, 1) k_tiled_a64(Dims d, const double* __restrict__ r,
                                                              double* __restrict__ pbuf, double* __restrict__ q,
                                                              OpTab<double> t, PcgScalars* sc,
                                                              double* __restrict__ partials, int slab) {
    __shared__ __align__(16) double sm[3][WARPS * SW];
    if (sc->done) return;
    const long long N = d.N;
    const double beta = sc->beta;
    const int par = sc->par;
    const double* __restrict__ pold = pbuf + (long long)par * 3 * N;
    double* __restrict__ pnew = pbuf + (long long)(1 - par) * 3 * N;
    const Tile T = tile_of(d, slab);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = T.j0 - 1 + w;
    const bool row_ok = (j >= 0 && j < d.nt);
    const bool interior = row_ok && w >= 1 && w <= TJ;
    const int kq = T.k0 + lane * 4;
    const int kl = (T.k0 == 0) ? d.np - 1 : T.k0 - 1;
    const int kr = (T.k0 + TK == d.np) ? 0 : T.k0 + TK;
    const long long plane = (long long)d.nt * d.np;
    auto pnew4 = [&](int i, int c, double (&o)[4]) {
        const long long base = c * N + (long long)i * plane + (long long)j * d.np + kq;
        double rv[4], pv[4];
        ld4d(r + base, rv);
        ld4d(pold + base, pv);
#pragma unroll
        for (int e = 0; e < 4; e++) o[e] = fma(beta, pv[e], rv[e]);
    };
    auto pnew1 = [&](int i, int c, int k) {
        const long long idx = c * N + (long long)i * plane + (long long)j * d.np + k;
        return fma(beta, pold[idx], r[idx]);
    };
    double pm[3][4], pc[3][4], pn[3][4];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int e = 0; e < 4; e++) pm[c][e] = pc[c][e] = pn[c][e] = 0.0;
    if (row_ok && T.i0 < T.i1) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            pnew4(T.i0, c, pc[c]);
            if (interior && T.i0 > 0) pnew4(T.i0 - 1, c, pm[c]);
        }
    }
    double acc = 0.0;
    for (int i = T.i0; i < T.i1; i++) {
        if (interior && i + 1 < d.nr) {
#pragma unroll
            for (int c = 0; c < 3; c++) pnew4(i + 1, c, pn[c]);
        } else {
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int e = 0; e < 4; e++) pn[c][e] = 0.0;
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            st4d(&sm[c][w * SW + 4 + lane * 4], pc[c]);
            if (lane == 0) sm[c][w * SW + 3] = row_ok ? pnew1(i, c, kl) : 0.0;
            if (lane == 31) sm[c][w * SW + 4 + TK] = row_ok ? pnew1(i, c, kr) : 0.0;
        }
        __syncthreads();
        if (interior) {
            const double ar_lo = t.ar[i * d.nt + j], ar_hi = t.ar[(i + 1) * d.nt + j];
            const double at_lo = t.at[i * (d.nt + 1) + j], at_hi = t.at[i * (d.nt + 1) + j + 1];
            const double ap = t.ap[i * d.nt + j];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const double* row = &sm[c][w * SW + 4 + lane * 4];
                double up[4], dn[4], qv[4];
                ld4d(row - SW, up);
                ld4d(row + SW, dn);
                const double lft = row[-1], rgt = row[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const double l = (e == 0) ? lft : pc[c][e - 1];
                    const double rr = (e == 3) ? rgt : pc[c][e + 1];
                    double o = fma(-ap, l + rr, pc[c][e]);
                    if (j > 0) o = fma(-at_lo, up[e], o);
                    if (j < d.nt - 1) o = fma(-at_hi, dn[e], o);
                    if (i > 0) o = fma(-ar_lo, pm[c][e], o);
                    if (i < d.nr - 1) o = fma(-ar_hi, pn[c][e], o);
                    qv[e] = o;
                    acc = fma(pc[c][e], o, acc);
                }
                const long long base = c * N + (long long)i * plane + (long long)j * d.np + kq;
                st4d(pnew + base, pc[c]);
                st4d(q + base, qv);
            }
        }
        __syncthreads();
        if (interior) {
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    pm[c][e] = pc[c][e];
                    pc[c][e] = pn[c][e];
                }
        } else if (row_ok && i + 1 < T.i1) {
#pragma unroll
            for (int c = 0; c < 3; c++) pnew4(i + 1, c, pc[c]);
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

void enqueue_tiled64_a(mhd_grid_s* g, cudaStream_t st, int slab, int prof_id) {
    const int blocks = tiled32_blocks(g, slab);
    const int s = prof_begin(g, st, prof_id);
    k_tiled_a64<<<blocks, WARPS * 32, 0, st>>>(g->d, g->r64, g->p64, g->q64, g->t64, g->sc, g->partials, slab);
    prof_end(g, st, s);
}

}  // namespace mhd
