// PCG with the point-Jacobi preconditioner PC1 (Sec. 2.2) for M_alpha = D + alpha K, on
// stacked 3-component vectors, in FP64 or FP32-inner / FP64-refinement form.
//
// Point-Jacobi PCG on M x = b produces, in exact arithmetic, the same iterates as plain CG on
// the symmetrically scaled system A~ y = S b with A~ = S M S, S = diag(M)^(-1/2), x = S y:
// its residual r~ = S r, and <r~, r~> = <r, D^-1 r> is PCG's <r, z>. The scaled form has a unit
// diagonal, so the stencil needs one multiply-add per neighbour and no preconditioner pass.
// That matters on this part: FP64 runs at 2 FMA/clk/SM, so the FP64 iteration is bound by its
// FP64 instruction count, not by HBM.
//
// One iteration is three kernels: the p update (which also adds the previous iteration's alpha p
// to x: the x update is deferred by one kernel, so the update kernel need not read p or x), the
// stencil with <p, q>, and the r update with the dot products and the stop test. In the FP32
// inner solves the first two can run as one kernel with p double-buffered (chosen per grid by
// timing).
//
// Reductions: every thread accumulates its share in FP64 (FP32 path: compensated FP32 per
// thread, then FP64), CTAs reduce with warp shuffles, write one partial each, and the last CTA
// to arrive sums the partials in CTA order and finishes the scalar recurrence (alpha, beta,
// stop test). Results are deterministic for a fixed launch shape.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "mhd_internal.cuh"
#include "reduce.cuh"

namespace mhd {

// ------------------------------------------------------------------------------------------
// vector access along phi
// ------------------------------------------------------------------------------------------
template <typename T, int V>
__device__ __forceinline__ void ldv(const T* __restrict__ p, T (&o)[V]) {
    if constexpr (sizeof(T) == 8 && V == 2) {
        double2 t = *reinterpret_cast<const double2*>(p);
        o[0] = t.x; o[1] = t.y;
    } else if constexpr (sizeof(T) == 4 && V == 4) {
        float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else if constexpr (sizeof(T) == 4 && V == 2) {
        float2 t = *reinterpret_cast<const float2*>(p);
        o[0] = t.x; o[1] = t.y;
    }
}

template <typename T, int V>
__device__ __forceinline__ void stv(T* __restrict__ p, const T (&o)[V]) {
    if constexpr (sizeof(T) == 8 && V == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    } else if constexpr (sizeof(T) == 4 && V == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (sizeof(T) == 4 && V == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    }
}

template <typename T, int V>
__device__ __forceinline__ void zerov(T (&o)[V]) {
#pragma unroll
    for (int e = 0; e < V; e++) o[e] = T(0);
}

// Per-thread accumulator: plain FP64 for FP64 data; for FP32 data a compensated FP32 sum
// (Neumaier) that is handed to FP64 once per thread.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void fma_add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
        s = t;
    }
    __device__ __forceinline__ void fma_add(float a, float b) { add(a * b); }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// ------------------------------------------------------------------------------------------
// operator tables for one alpha
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double diag_at(const Geo& G, int nt, double a, int i, int j) {
    const double s = G.wr[i * nt + j] + G.wr[(i + 1) * nt + j] + G.wt[i * (nt + 1) + j] +
                     G.wt[i * (nt + 1) + j + 1] + 2.0 * G.wp[i * nt + j];
    return G.rhoV[i * nt + j] + a * s;
}

__global__ void k_tables(Dims d, Geo G, const double* __restrict__ alpha_p, OpTab<double> t,
                         OpTab<float> t32, OpTab64u tu, int want32) {
    const int nr = d.nr, nt = d.nt;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nr * nt) return;
    const int i = idx / nt, j = idx - i * nt;
    const double a = *alpha_p;
    const double dc = diag_at(G, nt, a, i, j);
    const double s = 1.0 / sqrt(dc);
    const double ar = (i > 0) ? a * G.wr[i * nt + j] * s * (1.0 / sqrt(diag_at(G, nt, a, i - 1, j))) : 0.0;
    const double at = (j > 0) ? a * G.wt[i * (nt + 1) + j] * s * (1.0 / sqrt(diag_at(G, nt, a, i, j - 1))) : 0.0;
    const double ap = a * G.wp[idx] * s * s;
    t.s[idx] = s;
    t.ar[i * nt + j] = ar;
    t.at[i * (nt + 1) + j] = at;
    t.ap[idx] = ap;
    tu.dg[idx] = dc;
    tu.awr[i * nt + j] = (i > 0) ? a * G.wr[i * nt + j] : 0.0;
    tu.awt[i * (nt + 1) + j] = (j > 0) ? a * G.wt[i * (nt + 1) + j] : 0.0;
    tu.awp[idx] = a * G.wp[idx];
    if (i == nr - 1) { t.ar[nr * nt + j] = 0.0; tu.awr[nr * nt + j] = 0.0; }
    if (j == nt - 1) { t.at[i * (nt + 1) + nt] = 0.0; tu.awt[i * (nt + 1) + nt] = 0.0; }
    if (want32) {
        t32.s[idx] = (float)s;
        t32.ar[i * nt + j] = (float)ar;
        t32.at[i * (nt + 1) + j] = (float)at;
        t32.ap[idx] = (float)ap;
        if (i == nr - 1) t32.ar[nr * nt + j] = 0.f;
        if (j == nt - 1) t32.at[i * (nt + 1) + nt] = 0.f;
    }
}

// ------------------------------------------------------------------------------------------
// index decomposition of a phi-vector group g -> (i, j, k0)
// ------------------------------------------------------------------------------------------
struct Cell {
    int i, j, k0;
    long long ij, base;
};
template <int V>
__device__ __forceinline__ Cell decompose(const Dims& d, unsigned int g) {
    Cell c;
    const unsigned int npv = d.np / V;
    const unsigned int ij = g / npv;
    c.k0 = (int)(g - ij * npv) * V;
    c.i = (int)(ij / d.nt);
    c.j = (int)(ij - (unsigned)c.i * d.nt);
    c.ij = ij;
    c.base = (long long)ij * d.np + c.k0;
    return c;
}

// stencil of the scaled operator at one phi-vector: o = u - sum a_nb u_nb
template <typename T, int V>
__device__ __forceinline__ void scaled_stencil(const Dims& d, const Cell& c, const T* __restrict__ u,
                                               T cr_lo, T cr_hi, T ct_lo, T ct_hi, T cp, T (&v)[V],
                                               T (&o)[V]) {
    const long long plane = (long long)d.nt * d.np;
    ldv<T, V>(u + c.base, v);
    const long long row = c.base - c.k0;
    const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
    const int kp = (c.k0 + V == d.np) ? 0 : c.k0 + V;
    const T ukm = u[row + km], ukp = u[row + kp];
#pragma unroll
    for (int e = 0; e < V; e++) {
        const T left = (e == 0) ? ukm : v[e - 1];
        const T right = (e == V - 1) ? ukp : v[e + 1];
        o[e] = fma(-cp, left + right, v[e]);
    }
    T n[V];
    if (c.i > 0) {
        ldv<T, V>(u + c.base - plane, n);
#pragma unroll
        for (int e = 0; e < V; e++) o[e] = fma(-cr_lo, n[e], o[e]);
    }
    if (c.i < d.nr - 1) {
        ldv<T, V>(u + c.base + plane, n);
#pragma unroll
        for (int e = 0; e < V; e++) o[e] = fma(-cr_hi, n[e], o[e]);
    }
    if (c.j > 0) {
        ldv<T, V>(u + c.base - d.np, n);
#pragma unroll
        for (int e = 0; e < V; e++) o[e] = fma(-ct_lo, n[e], o[e]);
    }
    if (c.j < d.nt - 1) {
        ldv<T, V>(u + c.base + d.np, n);
#pragma unroll
        for (int e = 0; e < V; e++) o[e] = fma(-ct_hi, n[e], o[e]);
    }
}

// ------------------------------------------------------------------------------------------
// FP64 / FP32 CG iteration kernels on the scaled system
// ------------------------------------------------------------------------------------------
// A1: p = r + beta p. XD (deferred x update): first x += alpha_prev p with the alpha of the
// previous iteration (sc->ax), so the update kernel B need not read p or touch x; the product
// and its rounding are those of an immediate x update, one kernel later.
template <typename T, int V, int NC, bool XD = false>
__global__ void __launch_bounds__(kThreads) k_pupdate(Dims d, const T* __restrict__ r,
                                                      T* __restrict__ p, T* __restrict__ x,
                                                      const PcgScalars* sc) {
    if (sc->done) return;
    const T beta = (T)sc->beta;
    const T ax = XD ? (T)sc->ax : T(0);
    const unsigned int G = (unsigned int)(d.N / V);
#pragma unroll
    for (int c = 0; c < NC; c++) {
        const T* rc = r + c * d.N;
        T* pc = p + c * d.N;
        for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
            T a[V], b[V];
            ldv<T, V>(rc + (long long)g * V, a);
            ldv<T, V>(pc + (long long)g * V, b);
            if constexpr (XD) {
                T xv[V];
                ldv<T, V>(x + c * d.N + (long long)g * V, xv);
#pragma unroll
                for (int e = 0; e < V; e++) xv[e] = fma(ax, b[e], xv[e]);
                stv<T, V>(x + c * d.N + (long long)g * V, xv);
            }
#pragma unroll
            for (int e = 0; e < V; e++) b[e] = fma(beta, b[e], a[e]);
            stv<T, V>(pc + (long long)g * V, b);
        }
    }
}

// A2: q = A~ p and <p, q>; last CTA forms alpha = rho / <p, q>
template <typename T, int V, int NC>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 6 : 4) k_spmv_dot(Dims d, const T* __restrict__ p,
                                                       T* __restrict__ q, OpTab<T> t, PcgScalars* sc,
                                                       double* __restrict__ partials) {
    if (sc->done) return;
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / V);
    Acc<T> acc;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<V>(d, g);
        const T cr_lo = t.ar[c.i * nt + c.j], cr_hi = t.ar[(c.i + 1) * nt + c.j];
        const T ct_lo = t.at[c.i * (nt + 1) + c.j], ct_hi = t.at[c.i * (nt + 1) + c.j + 1];
        const T cp = t.ap[c.ij];
        // one component at a time: holding all three components' neighbours at once raises the
        // register count past two CTAs per SM and was measured slower
#pragma unroll 1
        for (int k = 0; k < NC; k++) {
            T v[V], o[V];
            scaled_stencil<T, V>(d, c, p + k * d.N, cr_lo, cr_hi, ct_lo, ct_hi, cp, v, o);
            stv<T, V>(q + k * d.N + c.base, o);
#pragma unroll
            for (int e = 0; e < V; e++) acc.fma_add(v[e], o[e]);
        }
    }
    double val[1] = {acc.get()}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double pq = out[0];
        sc->pq = pq;
        sc->ax = 0.0;   // the p update of this iteration has applied any deferred x update
        if (!finite(pq)) sc->done = 3;
        else if (!(pq > 0.0)) sc->done = 4;
        else sc->alpha = sc->rho / pq;
    }
}

// A2 for one component c of the FP64 iteration whose components overlap: q_c = A~ p_c and the
// component's share of <p, q> into sc->pqc[c] (the last component's last CTA also clears the
// deferred x update: every component's p update has applied it by then)
template <int V>
__global__ void __launch_bounds__(kThreads, 3) k_spmv_dotc(Dims d, int c, int last, const double* __restrict__ p,
                                                           double* __restrict__ q, OpTab<double> t, PcgScalars* sc,
                                                           double* __restrict__ partials) {
    if (sc->done) return;
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / V);
    double acc = 0.0;
    const double* pc = p + c * d.N;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell cl = decompose<V>(d, g);
        const double cr_lo = t.ar[cl.i * nt + cl.j], cr_hi = t.ar[(cl.i + 1) * nt + cl.j];
        const double ct_lo = t.at[cl.i * (nt + 1) + cl.j], ct_hi = t.at[cl.i * (nt + 1) + cl.j + 1];
        const double cp = t.ap[cl.ij];
        double v[V], o[V];
        scaled_stencil<double, V>(d, cl, pc, cr_lo, cr_hi, ct_lo, ct_hi, cp, v, o);
        stv<double, V>(q + c * d.N + cl.base, o);
#pragma unroll
        for (int e = 0; e < V; e++) acc = fma(v[e], o[e], acc);
    }
    double val[1] = {acc}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        sc->pqc[c] = out[0];
        if (last) sc->ax = 0.0;
    }
}

// <p, q> from the component shares, alpha = rho / <p, q> (one thread)
__global__ void k_alpha_from_parts(PcgScalars* sc, int nc) {
    if (sc->done) return;
    double pq = 0.0;
    for (int c = 0; c < nc; c++) pq += sc->pqc[c];
    sc->pq = pq;
    if (!finite(pq)) sc->done = 3;
    else if (!(pq > 0.0)) sc->done = 4;
    else sc->alpha = sc->rho / pq;
}

// A1+A2 for the FP32 inner iteration in one pass: p~ = r~ + beta p~_old is formed at the cell and,
// from r~ and p~_old, at each of its six neighbours (the same fma as the p update kernel, so every
// value equals the one its own thread stores); the cell's p~ goes to the other half of the p double
// buffer (sc->par names the half holding the current p~), x~ gets the deferred ax p~_old, and
// q~ = A~ p~ with <p~, q~>. Per cell: r~ (with PC2: z~), p~_old and x~ in; p~, x~ and q~ out (6
// passes against the 8 of the separate p update and stencil); the neighbour reads are L1 and L2
// hits. Last CTA: alpha = rho / <p~, q~>, and par flips (every CTA read it at its start).
template <int V, int NC>
__global__ void __launch_bounds__(kThreads, 4) k_pspmv32(Dims d, const float* __restrict__ r,
                                                         float* __restrict__ pbuf, float* __restrict__ x,
                                                         float* __restrict__ q, OpTab<float> t, PcgScalars* sc,
                                                         double* __restrict__ partials) {
    if (sc->done) return;
    const int par = sc->par;
    const float* __restrict__ pold = pbuf + (long long)par * 3 * d.N;
    float* __restrict__ pnew = pbuf + (long long)(1 - par) * 3 * d.N;
    const float beta = (float)sc->beta, ax = (float)sc->ax;
    const int nt = d.nt;
    const long long plane = (long long)nt * d.np;
    const unsigned int G = (unsigned int)(d.N / V);
    Acc<float> acc;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<V>(d, g);
        const float cr_lo = t.ar[c.i * nt + c.j], cr_hi = t.ar[(c.i + 1) * nt + c.j];
        const float ct_lo = t.at[c.i * (nt + 1) + c.j], ct_hi = t.at[c.i * (nt + 1) + c.j + 1];
        const float cp = t.ap[c.ij];
        const long long row = c.base - c.k0;
        const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
        const int kp = (c.k0 + V == d.np) ? 0 : c.k0 + V;
#pragma unroll 1
        for (int k = 0; k < NC; k++) {
            const float* rk = r + k * d.N;
            const float* pk = pold + k * d.N;
            float rv[V], pv[V], xv[V], v[V], o[V], nr_[V], np_[V];
            ldv<float, V>(rk + c.base, rv);
            ldv<float, V>(pk + c.base, pv);
            ldv<float, V>(x + k * d.N + c.base, xv);
#pragma unroll
            for (int e = 0; e < V; e++) {
                v[e] = fmaf(beta, pv[e], rv[e]);
                xv[e] = fmaf(ax, pv[e], xv[e]);
            }
            stv<float, V>(x + k * d.N + c.base, xv);
            stv<float, V>(pnew + k * d.N + c.base, v);
            const float ukm = fmaf(beta, pk[row + km], rk[row + km]);
            const float ukp = fmaf(beta, pk[row + kp], rk[row + kp]);
#pragma unroll
            for (int e = 0; e < V; e++) {
                const float left = (e == 0) ? ukm : v[e - 1];
                const float right = (e == V - 1) ? ukp : v[e + 1];
                o[e] = fmaf(-cp, left + right, v[e]);
            }
            if (c.i > 0) {
                ldv<float, V>(rk + c.base - plane, nr_);
                ldv<float, V>(pk + c.base - plane, np_);
#pragma unroll
                for (int e = 0; e < V; e++) o[e] = fmaf(-cr_lo, fmaf(beta, np_[e], nr_[e]), o[e]);
            }
            if (c.i < d.nr - 1) {
                ldv<float, V>(rk + c.base + plane, nr_);
                ldv<float, V>(pk + c.base + plane, np_);
#pragma unroll
                for (int e = 0; e < V; e++) o[e] = fmaf(-cr_hi, fmaf(beta, np_[e], nr_[e]), o[e]);
            }
            if (c.j > 0) {
                ldv<float, V>(rk + c.base - d.np, nr_);
                ldv<float, V>(pk + c.base - d.np, np_);
#pragma unroll
                for (int e = 0; e < V; e++) o[e] = fmaf(-ct_lo, fmaf(beta, np_[e], nr_[e]), o[e]);
            }
            if (c.j < d.nt - 1) {
                ldv<float, V>(rk + c.base + d.np, nr_);
                ldv<float, V>(pk + c.base + d.np, np_);
#pragma unroll
                for (int e = 0; e < V; e++) o[e] = fmaf(-ct_hi, fmaf(beta, np_[e], nr_[e]), o[e]);
            }
            stv<float, V>(q + k * d.N + c.base, o);
#pragma unroll
            for (int e = 0; e < V; e++) acc.fma_add(v[e], o[e]);
        }
    }
    double val[1] = {acc.get()}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double pq = out[0];
        sc->pq = pq;
        sc->ax = 0.0;   // applied above
        sc->par = 1 - par;
        if (!finite(pq)) sc->done = 3;
        else if (!(pq > 0.0)) sc->done = 4;
        else sc->alpha = sc->rho / pq;
    }
}

// ------------------------------------------------------------------------------------------
// FP32 inner iteration without a stored q~ (the recompute pair), two kernels per iteration:
//   P (k_pfold32): p~ = r~ + beta p~_old at the cell and, from r~ and p~_old, at its six
//      neighbours (the fma of the p update kernel), so <p~, A~ p~> needs no q~ in memory; p~ goes
//      to the other half of the p double buffer. r~ and p~_old in, p~ out: 3 passes.
//   R (k_rupd32): q~ = A~ p~ once more from the stored p~ (the same expression in the same order,
//      so the same bits as P's on-the-fly values), r~ -= alpha q~ with <r~, r~> and sum dg r~^2.
//      x~ is updated two iterations at a time: on every second iteration
//      x~ = fma(alpha_k, p~_k, fma(alpha_{k-1}, p~_{k-1}, x~)), the two roundings of two single
//      updates, with p~_{k-1} still in the other half of the double buffer (sc->ax holds
//      alpha_{k-1} while an update is pending). p~ and r~ in, r~ out, and on every second
//      iteration x~ and p~_{k-1} in, x~ out: 4.5 passes on average.
// The iterates equal those of the split kernels up to the order of the <p~, q~> reduction.
// REV: R walks the groups from the last to the first, so it starts on the p~ that P wrote last
// (still in L2) and ends on the r~ that the next P reads first.
// Neighbour loads are unconditional: at a wall the address is clamped to the cell itself and the
// coefficient of that face is exactly 0 in the tables, so fma(-0, u, o) = o and the result has the
// same bits as the branching form, while every load of the stencil can be in flight at once.
template <int V>
struct Nbr {
    long long im, ip, jm, jp;   // offsets of the four neighbour groups (0 at a wall)
    __device__ __forceinline__ Nbr(const Dims& d, const Cell& c) {
        const long long plane = (long long)d.nt * d.np;
        im = (c.i > 0) ? -plane : 0;
        ip = (c.i < d.nr - 1) ? plane : 0;
        jm = (c.j > 0) ? -(long long)d.np : 0;
        jp = (c.j < d.nt - 1) ? (long long)d.np : 0;
    }
};

template <int V, int NC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_pfold32(Dims d, const float* __restrict__ r,
                                                            float* __restrict__ pbuf, OpTab<float> t,
                                                            PcgScalars* sc, double* __restrict__ partials) {
    if (sc->done) return;
    const int par = sc->par;
    const float* __restrict__ pold = pbuf + (long long)par * 3 * d.N;
    float* __restrict__ pnew = pbuf + (long long)(1 - par) * 3 * d.N;
    const float beta = (float)sc->beta;
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / V);
    Acc<float> acc;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<V>(d, g);
        const Nbr<V> nb(d, c);
        const float cr_lo = t.ar[c.i * nt + c.j], cr_hi = t.ar[(c.i + 1) * nt + c.j];
        const float ct_lo = t.at[c.i * (nt + 1) + c.j], ct_hi = t.at[c.i * (nt + 1) + c.j + 1];
        const float cp = t.ap[c.ij];
        const long long row = c.base - c.k0;
        const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
        const int kp = (c.k0 + V == d.np) ? 0 : c.k0 + V;
#pragma unroll 1
        for (int k = 0; k < NC; k++) {
            const float* rk = r + k * d.N;
            const float* pk = pold + k * d.N;
            float rv[V], pv[V], v[V], o[V], a0[V], a1[V], b0[V], b1[V], c0[V], c1[V], e0[V], e1[V];
            ldv<float, V>(rk + c.base, rv);
            ldv<float, V>(pk + c.base, pv);
            const float rkm = rk[row + km], pkm = pk[row + km], rkp = rk[row + kp], pkp = pk[row + kp];
            ldv<float, V>(rk + c.base + nb.im, a0);
            ldv<float, V>(pk + c.base + nb.im, a1);
            ldv<float, V>(rk + c.base + nb.ip, b0);
            ldv<float, V>(pk + c.base + nb.ip, b1);
            ldv<float, V>(rk + c.base + nb.jm, c0);
            ldv<float, V>(pk + c.base + nb.jm, c1);
            ldv<float, V>(rk + c.base + nb.jp, e0);
            ldv<float, V>(pk + c.base + nb.jp, e1);
#pragma unroll
            for (int e = 0; e < V; e++) v[e] = fmaf(beta, pv[e], rv[e]);
            stv<float, V>(pnew + k * d.N + c.base, v);
            const float ukm = fmaf(beta, pkm, rkm);
            const float ukp = fmaf(beta, pkp, rkp);
#pragma unroll
            for (int e = 0; e < V; e++) {
                const float left = (e == 0) ? ukm : v[e - 1];
                const float right = (e == V - 1) ? ukp : v[e + 1];
                o[e] = fmaf(-cp, left + right, v[e]);
                o[e] = fmaf(-cr_lo, fmaf(beta, a1[e], a0[e]), o[e]);
                o[e] = fmaf(-cr_hi, fmaf(beta, b1[e], b0[e]), o[e]);
                o[e] = fmaf(-ct_lo, fmaf(beta, c1[e], c0[e]), o[e]);
                o[e] = fmaf(-ct_hi, fmaf(beta, e1[e], e0[e]), o[e]);
            }
#pragma unroll
            for (int e = 0; e < V; e++) acc.fma_add(v[e], o[e]);
        }
    }
    double val[1] = {acc.get()}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double pq = out[0];
        sc->pq = pq;
        sc->par = 1 - par;
        if (!finite(pq)) sc->done = 3;
        else if (!(pq > 0.0)) sc->done = 4;
        else sc->alpha = sc->rho / pq;
    }
}

template <int V, int NC, bool REV, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_rupd32(Dims d, float* __restrict__ x, float* __restrict__ r,
                                                           const float* __restrict__ pbuf, OpTab<float> t,
                                                           const double* __restrict__ dg, PcgScalars* sc,
                                                           double* __restrict__ partials) {
    if (sc->done) return;
    const int par = sc->par;   // P has flipped it: the half holding p~_k
    const float* __restrict__ p = pbuf + (long long)par * 3 * d.N;
    const float* __restrict__ pprev = pbuf + (long long)(1 - par) * 3 * d.N;
    const float al = (float)sc->alpha;
    const float axp = (float)sc->ax;
    const bool pair = (sc->ax != 0.0);
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / V);
    Acc<float> a_rho;
    double a_rr = 0.0;
    for (unsigned int g0 = blockIdx.x * blockDim.x + threadIdx.x; g0 < G; g0 += gridDim.x * blockDim.x) {
        const unsigned int g = REV ? G - 1u - g0 : g0;
        const Cell c = decompose<V>(d, g);
        const Nbr<V> nb(d, c);
        const float cr_lo = t.ar[c.i * nt + c.j], cr_hi = t.ar[(c.i + 1) * nt + c.j];
        const float ct_lo = t.at[c.i * (nt + 1) + c.j], ct_hi = t.at[c.i * (nt + 1) + c.j + 1];
        const float cp = t.ap[c.ij];
        const long long row = c.base - c.k0;
        const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
        const int kp = (c.k0 + V == d.np) ? 0 : c.k0 + V;
        float rs[V];
        zerov<float, V>(rs);
#pragma unroll 1
        for (int k = 0; k < NC; k++) {
            const float* pk = p + k * d.N;
            float v[V], o[V], rv[V], a[V], b[V], cc[V], e4[V];
            ldv<float, V>(pk + c.base, v);
            const float ukm = pk[row + km], ukp = pk[row + kp];
            ldv<float, V>(pk + c.base + nb.im, a);
            ldv<float, V>(pk + c.base + nb.ip, b);
            ldv<float, V>(pk + c.base + nb.jm, cc);
            ldv<float, V>(pk + c.base + nb.jp, e4);
            ldv<float, V>(r + k * d.N + c.base, rv);
#pragma unroll
            for (int e = 0; e < V; e++) {
                const float left = (e == 0) ? ukm : v[e - 1];
                const float right = (e == V - 1) ? ukp : v[e + 1];
                o[e] = fmaf(-cp, left + right, v[e]);
                o[e] = fmaf(-cr_lo, a[e], o[e]);
                o[e] = fmaf(-cr_hi, b[e], o[e]);
                o[e] = fmaf(-ct_lo, cc[e], o[e]);
                o[e] = fmaf(-ct_hi, e4[e], o[e]);
                rv[e] = fmaf(-al, o[e], rv[e]);
                rs[e] = fmaf(rv[e], rv[e], rs[e]);
            }
            stv<float, V>(r + k * d.N + c.base, rv);
            if (pair) {
                float xv[V], pp[V];
                ldv<float, V>(x + k * d.N + c.base, xv);
                ldv<float, V>(pprev + k * d.N + c.base, pp);
#pragma unroll
                for (int e = 0; e < V; e++) xv[e] = fmaf(al, v[e], fmaf(axp, pp[e], xv[e]));
                stv<float, V>(x + k * d.N + c.base, xv);
            }
        }
        float cell = rs[0];
#pragma unroll
        for (int e = 1; e < V; e++) cell += rs[e];
        a_rho.add(cell);
        a_rr = fma(dg[c.ij], (double)cell, a_rr);
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
        sc->ax = pair ? 0.0 : sc->alpha;   // pending: alpha_k p~_k, p~_k in the current half
        if (!finite(rr) || !finite(rho)) sc->done = 3;
        else if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
        else if (sc->iter >= sc->max_iter) sc->done = 2;
    }
}

// B: x += alpha p, r -= alpha q, rho = <r~, r~>, rr = sum dg r~^2; last CTA: beta, stop test.
// PAR: p lives in the buffer that a fused p-update kernel just wrote (the other half of a double
// buffer of stride 3N, chosen by the device-side parity), and the parity flips at the end.
// XD: x is left alone and alpha is handed on in sc->ax to the next p update (or to the finish or
// correction kernel when the solve stops here).
template <typename T, int V, int NC, bool PAR = false, bool XD = false>
__global__ void __launch_bounds__(kThreads) k_update(Dims d, T* __restrict__ x,
                                                     const T* __restrict__ p_in, T* __restrict__ r,
                                                     const T* __restrict__ q,
                                                     const double* __restrict__ dg, PcgScalars* sc,
                                                     double* __restrict__ partials) {
    if (sc->done) return;
    const T* __restrict__ p = PAR ? p_in + (long long)(1 - sc->par) * 3 * d.N : p_in;
    const T al = (T)sc->alpha;
    const unsigned int G = (unsigned int)(d.N / V);
    const unsigned int npv = d.np / V;
    Acc<T> a_rho;
    double a_rr = 0.0;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const long long off = (long long)g * V;
        T rs[V];
        zerov<T, V>(rs);
#pragma unroll
        for (int k = 0; k < NC; k++) {
            T rv[V], qv[V];
            ldv<T, V>(r + k * d.N + off, rv);
            ldv<T, V>(q + k * d.N + off, qv);
            if constexpr (!XD) {
                T xv[V], pv[V];
                ldv<T, V>(x + k * d.N + off, xv);
                ldv<T, V>(p + k * d.N + off, pv);
#pragma unroll
                for (int e = 0; e < V; e++) xv[e] = fma(al, pv[e], xv[e]);
                stv<T, V>(x + k * d.N + off, xv);
            }
#pragma unroll
            for (int e = 0; e < V; e++) {
                rv[e] = fma(-al, qv[e], rv[e]);
                rs[e] = fma(rv[e], rv[e], rs[e]);
            }
            stv<T, V>(r + k * d.N + off, rv);
        }
        T cell = rs[0];
#pragma unroll
        for (int e = 1; e < V; e++) cell += rs[e];
        a_rho.add(cell);
        a_rr = fma(dg[g / npv], (double)cell, a_rr);
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
        if (XD) sc->ax = sc->alpha;
        if (PAR) sc->par = 1 - sc->par;
        if (!finite(rr) || !finite(rho)) sc->done = 3;
        else if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
        else if (sc->iter >= sc->max_iter) sc->done = 2;
    }
}

// ------------------------------------------------------------------------------------------
// FP32 single-reduction pair (one reduction per iteration; nothing but p, r and x stored)
// ------------------------------------------------------------------------------------------
// With p~ = r~ + beta p~_old, <p~, A~ p~> = delta + 2 beta <r~, A~ p~_old> + beta^2 <p~_old, A~ p~_old>,
// delta = <r~, A~ r~>. The update kernel that formed r~ = r~_old - alpha A~ p~_old also sums
// <r~, A~ p~_old> (A~ p~_old is at hand there), and <p~_old, A~ p~_old> is the previous iteration's
// denominator, so one reduction per iteration (gamma = <r~, r~>, delta, sum dg r~^2 in the
// residual kernel) gives alpha = gamma / <p~, A~ p~> and beta = gamma / gamma_prev: the
// Hestenes-Stiefel scalars, without relying on the orthogonality that the Chronopoulos-Gear form
// takes for <r~, A~ p~_old> (the FP64 residual replacement of the mixed solve breaks it; that
// form, tried first, stagnated after the first replacement at inner tolerance 1e-5). After a
// replacement the FP64 residual kernel sums <r~, A~ p~_old> for the replaced residual itself.
// The update kernel forms p~ at the cell and its six neighbours and applies A~ there, so an
// iteration moves r~ in (residual kernel), r~ and p~_old in, p~ and r~ out (update kernel) and x~
// in and out every second iteration: 6 vector passes, the algorithmic minimum. r~ is
// double-buffered with the q~ workspace (the update reads r~ at its neighbours while it writes the
// new r~), on the parity of p~.
//
// R (k_cgr32): A~ r~ at the cell; gamma, delta, sum dg r~^2. Its last CTA takes the stop test
// and forms beta and alpha for the update.

// one component of R at one cell group: r~ at the cell and its neighbours, A~ r~, the partial sums
template <int V>
__device__ __forceinline__ void cgr_component(const Dims& d, const Cell& c, const Nbr<V>& nb, const float* rk,
                                              long long row, int km, int kp, float cr_lo, float cr_hi,
                                              float ct_lo, float ct_hi, float cp, float (&rs)[V],
                                              float& dsum) {
    float v[V], o[V], a[V], b[V], cc[V], e4[V];
    ldv<float, V>(rk + c.base, v);
    const float ukm = rk[row + km], ukp = rk[row + kp];
    ldv<float, V>(rk + c.base + nb.im, a);
    ldv<float, V>(rk + c.base + nb.ip, b);
    ldv<float, V>(rk + c.base + nb.jm, cc);
    ldv<float, V>(rk + c.base + nb.jp, e4);
#pragma unroll
    for (int e = 0; e < V; e++) {
        const float left = (e == 0) ? ukm : v[e - 1];
        const float right = (e == V - 1) ? ukp : v[e + 1];
        o[e] = fmaf(-cp, left + right, v[e]);
        o[e] = fmaf(-cr_lo, a[e], o[e]);
        o[e] = fmaf(-cr_hi, b[e], o[e]);
        o[e] = fmaf(-ct_lo, cc[e], o[e]);
        o[e] = fmaf(-ct_hi, e4[e], o[e]);
        rs[e] = fmaf(v[e], v[e], rs[e]);
        dsum = fmaf(v[e], o[e], dsum);
    }
}

// UNR: the component loop unrolled (every component's loads can be in flight at once, at fewer
// CTAs per SM: MINB)
// last CTA of the residual kernel: the stop test, then beta and alpha for the next update
__device__ __forceinline__ void cgr_finish(PcgScalars* sc, const double* out) {
    const double gam = out[0], del = out[1], rr = out[2];
    const double beta = (sc->iter == 0) ? sc->beta : gam / sc->rho;
    const double wp = sc->wp;   // <r~, A~ p~_old>, from the update kernel or the replacement
    sc->rho_prev = sc->rho;
    sc->rho = gam;
    sc->rr = rr;
    if (!finite(gam) || !finite(del) || !finite(rr)) sc->done = 3;
    else if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) sc->done = 1;
    else if (sc->iter >= sc->max_iter) sc->done = 2;
    else {
        const double den = (beta == 0.0) ? del : del + beta * (2.0 * wp + beta * sc->pq);
        if (!finite(den)) sc->done = 3;
        else if (!(den > 0.0)) sc->done = 4;
        else {
            sc->beta = beta;
            sc->pq = den;
            sc->alpha = gam / den;
        }
    }
}

template <int V, int NC, int MINB, bool UNR>
__global__ void __launch_bounds__(kThreads, MINB) k_cgr32(Dims d, const float* __restrict__ ra,
                                                          const float* __restrict__ rb, OpTab<float> t,
                                                          const double* __restrict__ dg, PcgScalars* sc,
                                                          double* __restrict__ partials) {
    if (sc->done) return;
    const float* __restrict__ r = sc->par ? rb : ra;
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / V);
    Acc<float> a_g, a_d;
    double a_rr = 0.0;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<V>(d, g);
        const Nbr<V> nb(d, c);
        const float cr_lo = t.ar[c.i * nt + c.j], cr_hi = t.ar[(c.i + 1) * nt + c.j];
        const float ct_lo = t.at[c.i * (nt + 1) + c.j], ct_hi = t.at[c.i * (nt + 1) + c.j + 1];
        const float cp = t.ap[c.ij];
        const long long row = c.base - c.k0;
        const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
        const int kp = (c.k0 + V == d.np) ? 0 : c.k0 + V;
        float rs[V];
        zerov<float, V>(rs);
        // <r~, A~ r~> of the cell group in plain FP32 (at most 12 terms), then into the compensated
        // per-thread sum once per group: a compensated add per term doubled the kernel's instructions
        float dsum = 0.f;
        if constexpr (UNR) {
#pragma unroll
            for (int k = 0; k < NC; k++)
                cgr_component<V>(d, c, nb, r + k * d.N, row, km, kp, cr_lo, cr_hi, ct_lo, ct_hi, cp, rs, dsum);
        } else {
#pragma unroll 1
            for (int k = 0; k < NC; k++)
                cgr_component<V>(d, c, nb, r + k * d.N, row, km, kp, cr_lo, cr_hi, ct_lo, ct_hi, cp, rs, dsum);
        }
        a_d.add(dsum);
        float cell = rs[0];
#pragma unroll
        for (int e = 1; e < V; e++) cell += rs[e];
        a_g.add(cell);
        a_rr = fma(dg[c.ij], (double)cell, a_rr);
    }
    double val[3] = {a_g.get(), a_d.get(), a_rr}, out[3];
    if (reduce_last<3>(val, partials, &sc->count, out) && threadIdx.x == 0) cgr_finish(sc, out);
}

// U (k_cgu32): p~ = r~ + beta p~_old at the cell and its neighbours, q~ = A~ p~ at the cell,
// r~ -= alpha q~ into the other r~ half, p~ into the other p~ half, <r~_new, q~> for the next
// denominator; x~ += alpha p~ + ax p~_old every second iteration (p~_old is at hand: the pending
// update is always the previous p~). Last CTA: parity flip, deferred alpha, iteration count.
template <int V, int NC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_cgu32(Dims d, float* __restrict__ x, float* __restrict__ ra,
                                                       float* __restrict__ rb, float* __restrict__ pbuf,
                                                       OpTab<float> t, PcgScalars* sc,
                                                       double* __restrict__ partials) {
    if (sc->done) return;
    const int par = sc->par;
    const float* __restrict__ r = par ? rb : ra;
    float* __restrict__ rn = par ? ra : rb;
    const float* __restrict__ pold = pbuf + (long long)par * 3 * d.N;
    float* __restrict__ pnew = pbuf + (long long)(1 - par) * 3 * d.N;
    const float beta = (float)sc->beta, al = (float)sc->alpha, axp = (float)sc->ax;
    const bool pair = (sc->ax != 0.0);
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / V);
    // the cross term: plain FP32 per thread (one register; a compensated sum spilled here), FP64
    // across threads
    float a_rq = 0.f;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<V>(d, g);
        const Nbr<V> nb(d, c);
        const float cr_lo = t.ar[c.i * nt + c.j], cr_hi = t.ar[(c.i + 1) * nt + c.j];
        const float ct_lo = t.at[c.i * (nt + 1) + c.j], ct_hi = t.at[c.i * (nt + 1) + c.j + 1];
        const float cp = t.ap[c.ij];
        const long long row = c.base - c.k0;
        const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
        const int kp = (c.k0 + V == d.np) ? 0 : c.k0 + V;
#pragma unroll 1
        for (int k = 0; k < NC; k++) {
            const float* rk = r + k * d.N;
            const float* pk = pold + k * d.N;
            float rv[V], pv[V], v[V], o[V], a0[V], a1[V], b0[V], b1[V], c0[V], c1[V], e0[V], e1[V];
            ldv<float, V>(rk + c.base, rv);
            ldv<float, V>(pk + c.base, pv);
            const float rkm = rk[row + km], pkm = pk[row + km], rkp = rk[row + kp], pkp = pk[row + kp];
            ldv<float, V>(rk + c.base + nb.im, a0);
            ldv<float, V>(pk + c.base + nb.im, a1);
            ldv<float, V>(rk + c.base + nb.ip, b0);
            ldv<float, V>(pk + c.base + nb.ip, b1);
            ldv<float, V>(rk + c.base + nb.jm, c0);
            ldv<float, V>(pk + c.base + nb.jm, c1);
            ldv<float, V>(rk + c.base + nb.jp, e0);
            ldv<float, V>(pk + c.base + nb.jp, e1);
#pragma unroll
            for (int e = 0; e < V; e++) v[e] = fmaf(beta, pv[e], rv[e]);
            stv<float, V>(pnew + k * d.N + c.base, v);
            const float ukm = fmaf(beta, pkm, rkm);
            const float ukp = fmaf(beta, pkp, rkp);
#pragma unroll
            for (int e = 0; e < V; e++) {
                const float left = (e == 0) ? ukm : v[e - 1];
                const float right = (e == V - 1) ? ukp : v[e + 1];
                o[e] = fmaf(-cp, left + right, v[e]);
                o[e] = fmaf(-cr_lo, fmaf(beta, a1[e], a0[e]), o[e]);
                o[e] = fmaf(-cr_hi, fmaf(beta, b1[e], b0[e]), o[e]);
                o[e] = fmaf(-ct_lo, fmaf(beta, c1[e], c0[e]), o[e]);
                o[e] = fmaf(-ct_hi, fmaf(beta, e1[e], e0[e]), o[e]);
                rv[e] = fmaf(-al, o[e], rv[e]);
                a_rq = fmaf(rv[e], o[e], a_rq);
            }
            stv<float, V>(rn + k * d.N + c.base, rv);
            if (pair) {
                float xv[V];
                ldv<float, V>(x + k * d.N + c.base, xv);
#pragma unroll
                for (int e = 0; e < V; e++) xv[e] = fmaf(al, v[e], fmaf(axp, pv[e], xv[e]));
                stv<float, V>(x + k * d.N + c.base, xv);
            }
        }
    }
    double val[1] = {(double)a_rq}, out[1];
    if (reduce_last<1>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        sc->wp = out[0];
        sc->par = 1 - par;
        sc->ax = pair ? 0.0 : sc->alpha;   // pending: alpha p~, p~ in the new current half
        sc->iter += 1;
        sc->total_iter += 1;
    }
}

// ------------------------------------------------------------------------------------------
// single-reduction (Chronopoulos-Gear) form, FP64: s = A~ p is carried by its own recurrence,
// so one stencil pass w = A~ r yields every inner product of an iteration
// ------------------------------------------------------------------------------------------
// C1: w = A~ r, gamma = <r~, r~>, delta = <w, r~>, rr = sum dg r~^2; last CTA: stop test on the
// current residual, then beta, alpha (first iteration: beta = 0, alpha = gamma / delta) and the
// iteration count of the update that follows
template <int NC>
__global__ void __launch_bounds__(kThreads, 4) k_cg_spmv(Dims d, const double* __restrict__ r,
                                                         double* __restrict__ w, OpTab<double> t,
                                                         const double* __restrict__ dg, PcgScalars* sc,
                                                         double* __restrict__ partials) {
    if (sc->done) return;
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / 2);
    double a_g = 0.0, a_d = 0.0, a_rr = 0.0;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<2>(d, g);
        const double cr_lo = t.ar[c.i * nt + c.j], cr_hi = t.ar[(c.i + 1) * nt + c.j];
        const double ct_lo = t.at[c.i * (nt + 1) + c.j], ct_hi = t.at[c.i * (nt + 1) + c.j + 1];
        const double cp = t.ap[c.ij];
        double cell = 0.0;
#pragma unroll 1
        for (int k = 0; k < NC; k++) {
            double v[2], o[2];
            scaled_stencil<double, 2>(d, c, r + k * d.N, cr_lo, cr_hi, ct_lo, ct_hi, cp, v, o);
            stv<double, 2>(w + k * d.N + c.base, o);
            cell = fma(v[0], v[0], fma(v[1], v[1], cell));
            a_d = fma(v[0], o[0], fma(v[1], o[1], a_d));
        }
        a_g += cell;
        a_rr = fma(dg[c.ij], cell, a_rr);
    }
    double val[3] = {a_g, a_d, a_rr}, out[3];
    if (reduce_last<3>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        const double gam = out[0], del = out[1], rr = out[2];
        sc->rr = rr;
        if (!finite(gam) || !finite(del) || !finite(rr)) {
            sc->done = 3;
        } else if (sqrt(rr) <= sc->tol * sqrt(sc->bb)) {
            sc->done = 1;
        } else if (sc->iter >= sc->max_iter) {
            sc->done = 2;
        } else {
            const bool first = (sc->iter == 0);
            const double beta = first ? 0.0 : gam / sc->rho;
            const double den = first ? del : del - beta * gam / sc->alpha;
            if (!(den > 0.0)) {
                sc->done = 4;
            } else {
                sc->beta = beta;
                sc->alpha = gam / den;
                sc->rho_prev = sc->rho;
                sc->rho = gam;
                sc->pq = den;
                sc->iter += 1;
                sc->total_iter += 1;
            }
        }
    }
}

// C2: p = r~ + beta p, s = w + beta s, x~ += alpha p, r~ -= alpha s (first iteration: p = r~,
// s = w, whatever the buffers held)
template <int NC>
__global__ void __launch_bounds__(kThreads) k_cg_update(Dims d, double* __restrict__ x, double* __restrict__ p,
                                                        double* __restrict__ s, double* __restrict__ r,
                                                        const double* __restrict__ w, const PcgScalars* sc) {
    if (sc->done) return;
    const double al = sc->alpha, be = sc->beta;
    const bool first = (sc->iter == 1);
    const unsigned int G = (unsigned int)(d.N / 2);
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const long long off = (long long)g * 2;
#pragma unroll
        for (int k = 0; k < NC; k++) {
            const long long o = k * d.N + off;
            double xv[2], pv[2], sv[2], rv[2], wv[2];
            ldv<double, 2>(r + o, rv);
            ldv<double, 2>(w + o, wv);
            ldv<double, 2>(x + o, xv);
            if (first) {
                pv[0] = rv[0]; pv[1] = rv[1];
                sv[0] = wv[0]; sv[1] = wv[1];
            } else {
                ldv<double, 2>(p + o, pv);
                ldv<double, 2>(s + o, sv);
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    pv[e] = fma(be, pv[e], rv[e]);
                    sv[e] = fma(be, sv[e], wv[e]);
                }
            }
#pragma unroll
            for (int e = 0; e < 2; e++) {
                xv[e] = fma(al, pv[e], xv[e]);
                rv[e] = fma(-al, sv[e], rv[e]);
            }
            stv<double, 2>(p + o, pv);
            stv<double, 2>(s + o, sv);
            stv<double, 2>(x + o, xv);
            stv<double, 2>(r + o, rv);
        }
    }
}

// ------------------------------------------------------------------------------------------
// FP64 solve: set-up and finish
// ------------------------------------------------------------------------------------------
// r = b - M x0 (unscaled tables), x~ = x0 / s, r~ = s r, p~ = r~; rho, ||r||^2, ||b||^2
__global__ void __launch_bounds__(kThreads) k_init64(Dims d, int nc, const double* __restrict__ b,
                                                     const double* __restrict__ x0, double* __restrict__ xs,
                                                     double* __restrict__ r, double* __restrict__ p,
                                                     OpTab<double> t, OpTab64u tu, PcgScalars* sc,
                                                     double* __restrict__ partials) {
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / 2);
    const long long plane = (long long)nt * d.np;
    double a_rho = 0.0, a_rr = 0.0, a_bb = 0.0;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<2>(d, g);
        const double s = t.s[c.ij];
        const double dg = tu.dg[c.ij];
        const double wl = tu.awr[c.i * nt + c.j], wh = tu.awr[(c.i + 1) * nt + c.j];
        const double tl = tu.awt[c.i * (nt + 1) + c.j], th = tu.awt[c.i * (nt + 1) + c.j + 1];
        const double wp = tu.awp[c.ij];
        for (int k = 0; k < nc; k++) {
            const double* u = x0 + k * d.N;
            double bv[2], rv[2], xv[2];
            ldv<double, 2>(b + k * d.N + c.base, bv);
            ldv<double, 2>(u + c.base, xv);
            const long long row = c.base - c.k0;
            const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
            const int kp = (c.k0 + 2 == d.np) ? 0 : c.k0 + 2;
            double n[2];
            double mx[2];
            mx[0] = dg * xv[0] - wp * (u[row + km] + xv[1]);
            mx[1] = dg * xv[1] - wp * (xv[0] + u[row + kp]);
            if (c.i > 0) { ldv<double, 2>(u + c.base - plane, n); mx[0] -= wl * n[0]; mx[1] -= wl * n[1]; }
            if (c.i < d.nr - 1) { ldv<double, 2>(u + c.base + plane, n); mx[0] -= wh * n[0]; mx[1] -= wh * n[1]; }
            if (c.j > 0) { ldv<double, 2>(u + c.base - d.np, n); mx[0] -= tl * n[0]; mx[1] -= tl * n[1]; }
            if (c.j < nt - 1) { ldv<double, 2>(u + c.base + d.np, n); mx[0] -= th * n[0]; mx[1] -= th * n[1]; }
            double xsv[2], rsv[2];
            const double si = sqrt(dg);
            for (int e = 0; e < 2; e++) {
                rv[e] = bv[e] - mx[e];
                rsv[e] = s * rv[e];
                xsv[e] = xv[e] * si;
                a_rho = fma(rsv[e], rsv[e], a_rho);
                a_rr = fma(rv[e], rv[e], a_rr);
                a_bb = fma(bv[e], bv[e], a_bb);
            }
            stv<double, 2>(xs + k * d.N + c.base, xsv);
            stv<double, 2>(r + k * d.N + c.base, rsv);
            stv<double, 2>(p + k * d.N + c.base, rsv);
        }
    }
    double val[3] = {a_rho, a_rr, a_bb}, out[3];
    if (reduce_last<3>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        sc->rho = out[0];
        sc->rr = out[1];
        sc->bb = out[2];
        sc->beta = 0.0;
        sc->iter = 0;
        sc->total_iter = 0;
        sc->outer = 0;
        sc->par = 0;
        sc->ax = 0.0;
        if (!finite(out[0]) || !finite(out[1]) || !finite(out[2])) sc->done = 3;
        else if (out[2] == 0.0) sc->done = 1;
        else if (sqrt(out[1]) <= sc->tol * sqrt(out[2])) sc->done = 1;
        else if (sc->max_iter <= 0) sc->done = 2;
        else sc->done = 0;
    }
}

// x = s (x~ + ax p~) (x = 0 when b = 0); ax is the deferred x update of the last iteration
__global__ void k_finish64(Dims d, int nc, const double* __restrict__ xs, const double* __restrict__ p,
                           double* __restrict__ x, const double* __restrict__ s, const PcgScalars* sc) {
    const bool zero = (sc->bb == 0.0);
    const double ax = sc->ax;
    const unsigned int G = (unsigned int)(d.N / 2);
    const unsigned int npv = d.np / 2;
    for (int k = 0; k < nc; k++)
        for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
            double v[2];
            ldv<double, 2>(xs + k * d.N + (long long)g * 2, v);
            if (ax != 0.0) {
                double pv[2];
                ldv<double, 2>(p + k * d.N + (long long)g * 2, pv);
                v[0] = fma(ax, pv[0], v[0]);
                v[1] = fma(ax, pv[1], v[1]);
            }
            const double sv = s[g / npv];
            v[0] = zero ? 0.0 : sv * v[0];
            v[1] = zero ? 0.0 : sv * v[1];
            stv<double, 2>(x + k * d.N + (long long)g * 2, v);
        }
}

// ------------------------------------------------------------------------------------------
// mixed precision: FP64 outer residual and correction around FP32 inner CG
// ------------------------------------------------------------------------------------------
// r = b - M x in FP64; r~32 = float(s r), x~32 = 0. With restart != 0 the FP32 CG starts afresh
// (beta = 0, so the next p update gives p~32 = r~32); otherwise the true residual replaces the
// recursive one and the CG recurrence continues with the same p~32 (reliable update, residual
// replacement): beta = <r~_true, r~_true> / rho of the previous iteration.
template <int V>
__global__ void __launch_bounds__(kThreads) k_outer_res(Dims d, int nc, const double* __restrict__ b,
                                                        const double* __restrict__ x, float* __restrict__ r32a,
                                                        float* __restrict__ r32b,
                                                        float* __restrict__ p32, float* __restrict__ x32,
                                                        OpTab<double> t, OpTab64u tu, PcgScalars* sc,
                                                        double* __restrict__ partials, int first, int restart,
                                                        int pc2, OpTab<float> t32) {
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / 2);
    // single-reduction FP32 pair (r32b non-null): <r~, A~ p~_old> of the replaced residual, in FP32
    // as its update kernel would have formed it, for the denominator of the next iteration
    const bool want_wp = (r32b != nullptr) && !first;
    const float* __restrict__ pold = p32 + (long long)(first ? 0 : sc->par) * 3 * d.N;
    double a_wp = 0.0;
    const long long plane = (long long)nt * d.np;
    // r~ goes to the half of a double-buffered r~ (r32b non-null) on the parity of p~
    float* __restrict__ r32 = (r32b && !first && sc->par) ? r32b : r32a;
    double a_rout = 0.0, a_bb = 0.0, a_rho = 0.0, a_rin = 0.0;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<2>(d, g);
        const double s = t.s[c.ij];
        const double dg = tu.dg[c.ij];
        const double wl = tu.awr[c.i * nt + c.j], wh = tu.awr[(c.i + 1) * nt + c.j];
        const double tl = tu.awt[c.i * (nt + 1) + c.j], th = tu.awt[c.i * (nt + 1) + c.j + 1];
        const double wp = tu.awp[c.ij];
        double cell_in = 0.0;
        for (int k = 0; k < nc; k++) {
            const double* u = x + k * d.N;
            double bv[2], xv[2], n[2], mx[2];
            ldv<double, 2>(b + k * d.N + c.base, bv);
            ldv<double, 2>(u + c.base, xv);
            const long long row = c.base - c.k0;
            const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
            const int kp = (c.k0 + 2 == d.np) ? 0 : c.k0 + 2;
            mx[0] = dg * xv[0] - wp * (u[row + km] + xv[1]);
            mx[1] = dg * xv[1] - wp * (xv[0] + u[row + kp]);
            if (c.i > 0) { ldv<double, 2>(u + c.base - plane, n); mx[0] -= wl * n[0]; mx[1] -= wl * n[1]; }
            if (c.i < d.nr - 1) { ldv<double, 2>(u + c.base + plane, n); mx[0] -= wh * n[0]; mx[1] -= wh * n[1]; }
            if (c.j > 0) { ldv<double, 2>(u + c.base - d.np, n); mx[0] -= tl * n[0]; mx[1] -= tl * n[1]; }
            if (c.j < nt - 1) { ldv<double, 2>(u + c.base + d.np, n); mx[0] -= th * n[0]; mx[1] -= th * n[1]; }
            float rs[2];
            for (int e = 0; e < 2; e++) {
                const double rv = bv[e] - mx[e];
                rs[e] = (float)(s * rv);
                a_rout = fma(rv, rv, a_rout);
                if (first) a_bb = fma(bv[e], bv[e], a_bb);
                const double rd = (double)rs[e];
                a_rho = fma(rd, rd, a_rho);
                cell_in = fma(rd, rd, cell_in);
            }
            *reinterpret_cast<float2*>(r32 + k * d.N + c.base) = make_float2(rs[0], rs[1]);
            if (want_wp) {
                const float* pk = pold + k * d.N;
                const float2 pc = *reinterpret_cast<const float2*>(pk + c.base);
                const float pm = pk[row + km], pp = pk[row + kp];
                const long long im = (c.i > 0) ? -plane : 0, ip = (c.i < d.nr - 1) ? plane : 0;
                const long long jm = (c.j > 0) ? -(long long)d.np : 0, jp = (c.j < nt - 1) ? (long long)d.np : 0;
                const float2 a = *reinterpret_cast<const float2*>(pk + c.base + im);
                const float2 bq = *reinterpret_cast<const float2*>(pk + c.base + ip);
                const float2 cq = *reinterpret_cast<const float2*>(pk + c.base + jm);
                const float2 eq = *reinterpret_cast<const float2*>(pk + c.base + jp);
                const float cr_lo = t32.ar[c.i * nt + c.j], cr_hi = t32.ar[(c.i + 1) * nt + c.j];
                const float ct_lo = t32.at[c.i * (nt + 1) + c.j], ct_hi = t32.at[c.i * (nt + 1) + c.j + 1];
                const float cp = t32.ap[c.ij];
                float o0 = fmaf(-cp, pm + pc.y, pc.x), o1 = fmaf(-cp, pc.x + pp, pc.y);
                o0 = fmaf(-cr_lo, a.x, o0);
                o1 = fmaf(-cr_lo, a.y, o1);
                o0 = fmaf(-cr_hi, bq.x, o0);
                o1 = fmaf(-cr_hi, bq.y, o1);
                o0 = fmaf(-ct_lo, cq.x, o0);
                o1 = fmaf(-ct_lo, cq.y, o1);
                o0 = fmaf(-ct_hi, eq.x, o0);
                o1 = fmaf(-ct_hi, eq.y, o1);
                a_wp = fma((double)rs[0], (double)o0, a_wp);
                a_wp = fma((double)rs[1], (double)o1, a_wp);
            }
            *reinterpret_cast<float2*>(x32 + k * d.N + c.base) = make_float2(0.f, 0.f);
            // first pass: p~32 = r~32 so no value left from an earlier solve can reach 0 * p
            if (first) *reinterpret_cast<float2*>(p32 + k * d.N + c.base) = make_float2(rs[0], rs[1]);
        }
        a_rin = fma(dg, cell_in, a_rin);
    }
    double val[4] = {a_rout, first ? a_bb : a_wp, a_rho, a_rin}, out[4];
    if (reduce_last<4>(val, partials, &sc->count, out) && threadIdx.x == 0) {
        if (want_wp) sc->wp = out[1];
        if (first) {
            sc->bb = out[1];
            sc->par = 0;
        }
        sc->rr_out = out[0];
        sc->ax = 0.0;   // k_correct has absorbed the deferred x update into x
        // keep the recurrence only while the replaced residual still agrees with the recursive
        // one (rho_true <= 4 rho_recursive); otherwise beta = 0 restarts it (p = r next)
        // (with PC2 the preconditioner pass that follows forms rho = <r, z> and takes this decision)
        if (!pc2) {
            const bool keep = !restart && sc->rho_prev > 0.0 && out[2] <= 4.0 * sc->rho;
            sc->beta = keep ? out[2] / sc->rho_prev : 0.0;
            sc->rho = out[2];
        }
        sc->rr = out[3];
        sc->iter = 0;
        const double bn = sqrt(sc->bb);
        if (!finite(out[0]) || !finite(out[2])) { sc->done = 3; sc->outer_done = 3; }
        else if (sc->bb == 0.0 || sqrt(out[0]) <= sc->tol * bn) { sc->done = 1; sc->outer_done = 1; }
        else {
            sc->outer_done = 0;
            sc->done = (sc->max_iter <= 0) ? 2 : 0;
        }
    }
}

// x += s (x~32 + ax p~32) (FP64 correction; ax p~32, formed in FP32, is the deferred x update of
// the last inner iteration)
__global__ void k_correct(Dims d, int nc, double* __restrict__ x, const float* __restrict__ xs,
                          const float* __restrict__ p, const double* __restrict__ s, PcgScalars* sc) {
    if (sc->outer_done) return;
    const float ax = (float)sc->ax;
    p += (long long)sc->par * 3 * d.N;   // the half of the p double buffer holding the current p~
    const unsigned int G = (unsigned int)(d.N / 2);
    const unsigned int npv = d.np / 2;
    for (int k = 0; k < nc; k++)
        for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
            double v[2];
            ldv<double, 2>(x + k * d.N + (long long)g * 2, v);
            float2 e = *reinterpret_cast<const float2*>(xs + k * d.N + (long long)g * 2);
            if (ax != 0.f) {
                const float2 pv = *reinterpret_cast<const float2*>(p + k * d.N + (long long)g * 2);
                e.x = fmaf(ax, pv.x, e.x);
                e.y = fmaf(ax, pv.y, e.y);
            }
            const double sv = s[g / npv];
            v[0] = fma(sv, (double)e.x, v[0]);
            v[1] = fma(sv, (double)e.y, v[1]);
            stv<double, 2>(x + k * d.N + (long long)g * 2, v);
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->outer += 1;
}

// q = M p (unscaled FP64), for the C-ABI operator call
__global__ void __launch_bounds__(kThreads) k_apply64(Dims d, int nc, const double* __restrict__ p,
                                                      double* __restrict__ q, OpTab64u tu) {
    const int nt = d.nt;
    const unsigned int G = (unsigned int)(d.N / 2);
    const long long plane = (long long)nt * d.np;
    for (unsigned int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const Cell c = decompose<2>(d, g);
        const double dg = tu.dg[c.ij];
        const double wl = tu.awr[c.i * nt + c.j], wh = tu.awr[(c.i + 1) * nt + c.j];
        const double tl = tu.awt[c.i * (nt + 1) + c.j], th = tu.awt[c.i * (nt + 1) + c.j + 1];
        const double wp = tu.awp[c.ij];
        for (int k = 0; k < nc; k++) {
            const double* u = p + k * d.N;
            double xv[2], n[2], mx[2];
            ldv<double, 2>(u + c.base, xv);
            const long long row = c.base - c.k0;
            const int km = (c.k0 == 0) ? d.np - 1 : c.k0 - 1;
            const int kp = (c.k0 + 2 == d.np) ? 0 : c.k0 + 2;
            mx[0] = dg * xv[0] - wp * (u[row + km] + xv[1]);
            mx[1] = dg * xv[1] - wp * (xv[0] + u[row + kp]);
            if (c.i > 0) { ldv<double, 2>(u + c.base - plane, n); mx[0] -= wl * n[0]; mx[1] -= wl * n[1]; }
            if (c.i < d.nr - 1) { ldv<double, 2>(u + c.base + plane, n); mx[0] -= wh * n[0]; mx[1] -= wh * n[1]; }
            if (c.j > 0) { ldv<double, 2>(u + c.base - d.np, n); mx[0] -= tl * n[0]; mx[1] -= tl * n[1]; }
            if (c.j < nt - 1) { ldv<double, 2>(u + c.base + d.np, n); mx[0] -= th * n[0]; mx[1] -= th * n[1]; }
            stv<double, 2>(q + k * d.N + c.base, mx);
        }
    }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
void build_tables(mhd_grid_s* g, const double* alpha_dev, bool fp32) {
    const int n = g->d.nr * g->d.nt;
    k_tables<<<(n + 255) / 256, 256, 0, g->stream>>>(g->d, g->geo, alpha_dev, g->t64, g->t32, g->tu,
                                                      fp32 ? 1 : 0);
}

void apply_operator(mhd_grid_s* g, const double* alpha_dev, int nc, const double* p, double* q) {
    build_tables(g, alpha_dev, false);
    const int blocks = grid_blocks(g, g->d.N / 2, 8);
    k_apply64<<<blocks, kThreads, 0, g->stream>>>(g->d, nc, p, q, g->tu);
}

namespace {

constexpr int kPerSmIter = 4;

bool use_v4(const mhd_grid_s* g) { return (g->d.np % 4) == 0; }

// enqueue one CG iteration (p update, stencil + <p,q>, update) of the given precision
template <typename T, int V, int NC>
void enqueue_split(mhd_grid_s* g, cudaStream_t st, T* x, T* r, T* p, T* q, const OpTab<T>& t, int blocks,
                   int prof0) {
    const Dims d = g->d;
    int s = prof_begin(g, st, prof0);
    k_pupdate<T, V, NC, true><<<blocks, kThreads, 0, st>>>(d, r, p, x, g->sc);
    prof_end(g, st, s);
    s = prof_begin(g, st, prof0 + 1);
    // the FP32 stencil is latency-bound: 6 CTAs per SM instead of 4 for more loads in flight
    const int bs = (sizeof(T) == 4) ? grid_blocks(g, d.N / V, 6) : blocks;
    k_spmv_dot<T, V, NC><<<bs, kThreads, 0, st>>>(d, p, q, t, g->sc, g->partials);
    prof_end(g, st, s);
    s = prof_begin(g, st, prof0 + 2);
    // FP32: one full wave of resident CTAs (measured 0.189 against 0.197 ms at 4 per SM); FP64:
    // 4 per SM (a full wave of 5 measured slower, 0.485 against 0.466 ms)
    const int bu = (sizeof(T) == 4) ? grid_blocks(g, d.N / V, resident_per_sm<k_update<T, V, NC, false, true>>())
                                    : blocks;
    k_update<T, V, NC, false, true><<<bu, kThreads, 0, st>>>(d, x, p, r, q, g->tu.dg, g->sc, g->partials);
    prof_end(g, st, s);
}

// FP64 iteration with the components overlapped: the stencil couples no components, so the HBM-bound
// p update of component c+1 (side stream) runs while the FP64-bound stencil of component c runs
// (grid stream); the stencils run at 3 CTAs per SM to leave the p update room on every SM. The
// stencils stay in order on one stream (they share the reduction buffers); the update follows.
template <int NC>
void enqueue_split64_ov(mhd_grid_s* g, cudaStream_t st, int p_per_sm) {
    const Dims d = g->d;
    const int bp = grid_blocks(g, d.N / 2, p_per_sm);
    const int bs = grid_blocks(g, d.N / 2, 3);
    cudaStream_t sd = g->side;
    cudaEventRecord(g->side_ev[0], st);   // fork: the side stream follows everything before
    cudaStreamWaitEvent(sd, g->side_ev[0], 0);
    for (int c = 0; c < NC; c++) {
        int s = prof_begin(g, sd, MHD_KERNEL_PUPDATE64);
        k_pupdate<double, 2, 1, true><<<bp, kThreads, 0, sd>>>(d, g->r64 + c * d.N, g->p64 + c * d.N,
                                                               g->x64 + c * d.N, g->sc);
        prof_end(g, sd, s);
        cudaEventRecord(g->side_ev[1 + c], sd);
        cudaStreamWaitEvent(st, g->side_ev[1 + c], 0);   // the last wait also joins the side stream
        s = prof_begin(g, st, MHD_KERNEL_SPMV64);
        k_spmv_dotc<2><<<bs, kThreads, 0, st>>>(d, c, c == NC - 1 ? 1 : 0, g->p64, g->q64, g->t64, g->sc, g->partials);
        prof_end(g, st, s);
    }
    k_alpha_from_parts<<<1, 1, 0, st>>>(g->sc, NC);
    const int s = prof_begin(g, st, MHD_KERNEL_UPDATE64);
    k_update<double, 2, NC, false, true><<<grid_blocks(g, d.N / 2, kPerSmIter), kThreads, 0, st>>>(
        d, g->x64, g->p64, g->r64, g->q64, g->tu.dg, g->sc, g->partials);
    prof_end(g, st, s);
}

// FP32 inner iteration with the p update folded into the stencil (p~ double-buffered)
template <int V, int NC>
void enqueue_fused32(mhd_grid_s* g, cudaStream_t st) {
    const Dims d = g->d;
    int s = prof_begin(g, st, MHD_KERNEL_PSPMV32);
    k_pspmv32<V, NC><<<grid_blocks(g, d.N / V, 4), kThreads, 0, st>>>(d, g->r32, g->p32, g->x32, g->q32, g->t32,
                                                                      g->sc, g->partials);
    prof_end(g, st, s);
    s = prof_begin(g, st, MHD_KERNEL_UPDATE32);
    k_update<float, V, NC, false, true><<<grid_blocks(g, d.N / V, resident_per_sm<k_update<float, V, NC, false, true>>()),
                                          kThreads, 0, st>>>(
        d, g->x32, g->p32, g->r32, g->q32, g->tu.dg, g->sc, g->partials);
    prof_end(g, st, s);
}

// FP32 inner iteration by the recompute pair (no q~ stored; x~ updated every second iteration); MINB:
// CTAs per SM the kernels are compiled for (registers per thread 65536 / (256 MINB))
template <int V, int NC, int MINB>
void enqueue_recompute32(mhd_grid_s* g, cudaStream_t st, bool rev) {
    const Dims d = g->d;
    int s = prof_begin(g, st, MHD_KERNEL_PFOLD32);
    k_pfold32<V, NC, MINB><<<grid_blocks(g, d.N / V, resident_per_sm<k_pfold32<V, NC, MINB>>()), kThreads, 0, st>>>(
        d, g->r32, g->p32, g->t32, g->sc, g->partials);
    prof_end(g, st, s);
    s = prof_begin(g, st, MHD_KERNEL_RUPD32);
    if (rev)
        k_rupd32<V, NC, true, MINB><<<grid_blocks(g, d.N / V, resident_per_sm<k_rupd32<V, NC, true, MINB>>()), kThreads,
                                      0, st>>>(d, g->x32, g->r32, g->p32, g->t32, g->tu.dg, g->sc, g->partials);
    else
        k_rupd32<V, NC, false, MINB><<<grid_blocks(g, d.N / V, resident_per_sm<k_rupd32<V, NC, false, MINB>>()),
                                       kThreads, 0, st>>>(d, g->x32, g->r32, g->p32, g->t32, g->tu.dg, g->sc,
                                                          g->partials);
    prof_end(g, st, s);
}

template <int V, int MINB>
void enqueue_recompute32_nc(mhd_grid_s* g, cudaStream_t st, int nc, bool rev) {
    if (nc == 3) enqueue_recompute32<V, 3, MINB>(g, st, rev);
    else if (nc == 2) enqueue_recompute32<V, 2, MINB>(g, st, rev);
    else enqueue_recompute32<V, 1, MINB>(g, st, rev);
}

// -3 / -4: 4 CTAs per SM (64 registers); -5: 6 CTAs per SM (40 registers), forwards. (L2 prefetches
// of the next component's centre lines were measured slower: 0.421 against 0.279 ms for the first
// kernel at 256x256x512.)
template <int V>
void enqueue_recompute32_var(mhd_grid_s* g, cudaStream_t st, int nc) {
    if (g->slab32 == -5) enqueue_recompute32_nc<V, 6>(g, st, nc, false);
    else enqueue_recompute32_nc<V, 4>(g, st, nc, g->slab32 == -4);
}

template <int V, int NC, int MINB_R, bool UNR, int MINB_U>
void enqueue_cgpair32_k(mhd_grid_s* g, cudaStream_t st) {
    const Dims d = g->d;
    int s = prof_begin(g, st, MHD_KERNEL_CGR32);
    k_cgr32<V, NC, MINB_R, UNR><<<grid_blocks(g, d.N / V, resident_per_sm<k_cgr32<V, NC, MINB_R, UNR>>()), kThreads,
                                  0, st>>>(d, g->r32, g->q32, g->t32, g->tu.dg, g->sc, g->partials);
    prof_end(g, st, s);
    s = prof_begin(g, st, MHD_KERNEL_CGU32);
    k_cgu32<V, NC, MINB_U><<<grid_blocks(g, d.N / V, resident_per_sm<k_cgu32<V, NC, MINB_U>>()), kThreads, 0, st>>>(
        d, g->x32, g->r32, g->q32, g->p32, g->t32, g->sc, g->partials);
    prof_end(g, st, s);
}

// -6: both kernels at 4 CTAs per SM; -7: the residual kernel unrolled over the components, both at 3;
// -8: unrolled residual kernel at 3, update kernel at 4. (Measured slower and removed: the cross
// term from the previous residual read by the residual kernel, its update kernel without a
// reduction: 0.286 + 0.355 ms; a plane-marching residual kernel: 0.208 against 0.165 ms.)
template <int V, int NC>
void enqueue_cgpair32(mhd_grid_s* g, cudaStream_t st) {
    switch (g->slab32) {
        case -7: enqueue_cgpair32_k<V, NC, 3, true, 3>(g, st); break;
        case -8: enqueue_cgpair32_k<V, NC, 3, true, 4>(g, st); break;
        default: enqueue_cgpair32_k<V, NC, 4, false, 4>(g, st); break;
    }
}

template <int V>
void enqueue_cgpair32_nc(mhd_grid_s* g, cudaStream_t st, int nc) {
    if (nc == 3) enqueue_cgpair32<V, 3>(g, st);
    else if (nc == 2) enqueue_cgpair32<V, 2>(g, st);
    else enqueue_cgpair32<V, 1>(g, st);
}

template <int V>
void enqueue_fused32_nc(mhd_grid_s* g, cudaStream_t st, int nc) {
    if (nc == 3) enqueue_fused32<V, 3>(g, st);
    else if (nc == 2) enqueue_fused32<V, 2>(g, st);
    else enqueue_fused32<V, 1>(g, st);
}

template <typename T, int V>
void enqueue_split_nc(mhd_grid_s* g, cudaStream_t st, int nc, T* x, T* r, T* p, T* q, const OpTab<T>& t,
                      int blocks, int prof0) {
    if (nc == 3) enqueue_split<T, V, 3>(g, st, x, r, p, q, t, blocks, prof0);
    else if (nc == 2) enqueue_split<T, V, 2>(g, st, x, r, p, q, t, blocks, prof0);
    else enqueue_split<T, V, 1>(g, st, x, r, p, q, t, blocks, prof0);
}

template <int NC>
void enqueue_cg(mhd_grid_s* g, cudaStream_t st, int blocks) {
    const Dims d = g->d;
    double* s_vec = g->p64 + 3 * (size_t)d.N;   // second half of the p double buffer
    int ps = prof_begin(g, st, MHD_KERNEL_SPMV64);
    k_cg_spmv<NC><<<blocks, kThreads, 0, st>>>(d, g->r64, g->q64, g->t64, g->tu.dg, g->sc, g->partials);
    prof_end(g, st, ps);
    ps = prof_begin(g, st, MHD_KERNEL_UPDATE64);
    k_cg_update<NC><<<blocks, kThreads, 0, st>>>(d, g->x64, g->p64, s_vec, g->r64, g->q64, g->sc);
    prof_end(g, st, ps);
}

// PC2 on the scaled system: p~ = z~ + beta p~, q~ = A~ p~ with <p~, q~>, then the phi-line kernel
template <int NC>
void enqueue_pc2(mhd_grid_s* g, cudaStream_t st, int blocks) {
    const Dims d = g->d;
    double* z = g->p64 + 3 * (size_t)d.N;
    int ps = prof_begin(g, st, MHD_KERNEL_PUPDATE64);
    k_pupdate<double, 2, NC><<<blocks, kThreads, 0, st>>>(d, z, g->p64, nullptr, g->sc);
    prof_end(g, st, ps);
    ps = prof_begin(g, st, MHD_KERNEL_SPMV64);
    k_spmv_dot<double, 2, NC><<<blocks, kThreads, 0, st>>>(d, g->p64, g->q64, g->t64, g->sc, g->partials);
    prof_end(g, st, ps);
    ps = prof_begin(g, st, MHD_KERNEL_PC2);
    pc2_enqueue_line(g, st, NC, false);
    prof_end(g, st, ps);
}

// the same for the FP32 inner solves of mixed precision; z~ lives in the PC2 workspace, and with
// the fused variant p~ alternates between the two halves of the p double buffer
template <typename T, int V, int NC>
void enqueue_pc2_32(mhd_grid_s* g, cudaStream_t st) {
    const Dims d = g->d;
    float* z = pc2_z32(g);
    if (g->pc2_fused32 > 0) {
        const int ps = prof_begin(g, st, MHD_KERNEL_PSPMV32);
        k_pspmv32<V, NC><<<grid_blocks(g, d.N / V, 4), kThreads, 0, st>>>(d, z, g->p32, g->x32, g->q32, g->t32, g->sc,
                                                                          g->partials);
        prof_end(g, st, ps);
    } else {
        int ps = prof_begin(g, st, MHD_KERNEL_PUPDATE32);
        k_pupdate<float, V, NC, true><<<grid_blocks(g, d.N / V, kPerSmIter), kThreads, 0, st>>>(d, z, g->p32, g->x32,
                                                                                                g->sc);
        prof_end(g, st, ps);
        ps = prof_begin(g, st, MHD_KERNEL_SPMV32);
        k_spmv_dot<float, V, NC><<<grid_blocks(g, d.N / V, 6), kThreads, 0, st>>>(d, g->p32, g->q32, g->t32, g->sc,
                                                                                  g->partials);
        prof_end(g, st, ps);
    }
    const int ps = prof_begin(g, st, MHD_KERNEL_PC2);
    pc2_enqueue_line(g, st, NC, true);
    prof_end(g, st, ps);
}

template <int V>
void enqueue_pc2_32_nc(mhd_grid_s* g, cudaStream_t st, int nc) {
    if (nc == 3) enqueue_pc2_32<float, V, 3>(g, st);
    else if (nc == 2) enqueue_pc2_32<float, V, 2>(g, st);
    else enqueue_pc2_32<float, V, 1>(g, st);
}

// kind: 0 FP64 Hestenes-Stiefel, 1 FP32 inner (Hestenes-Stiefel), 2 FP64 single-reduction,
// 3 FP64 with PC2, 4 FP32 inner with PC2
void enqueue_iteration(mhd_grid_s* g, cudaStream_t st, int prec, int nc) {
    const Dims d = g->d;
    if (prec == 4) {
        if (use_v4(g)) enqueue_pc2_32_nc<4>(g, st, nc);
        else enqueue_pc2_32_nc<2>(g, st, nc);
    } else if (prec == 3) {
        const int blocks = grid_blocks(g, d.N / 2, kPerSmIter);
        if (nc == 3) enqueue_pc2<3>(g, st, blocks);
        else if (nc == 2) enqueue_pc2<2>(g, st, blocks);
        else enqueue_pc2<1>(g, st, blocks);
    } else if (prec == 2) {
        const int blocks = grid_blocks(g, d.N / 2, kPerSmIter);
        if (nc == 3) enqueue_cg<3>(g, st, blocks);
        else if (nc == 2) enqueue_cg<2>(g, st, blocks);
        else enqueue_cg<1>(g, st, blocks);
    } else if (prec == 0 && g->slab64 == -2 && g->side) {
        // components overlapped (p updates launched for 4 CTAs per SM; 2 and 1 were measured
        // slower, 2.355 and 2.603 against 2.182 ms per iteration at 256x256x512)
        if (nc == 3) enqueue_split64_ov<3>(g, st, kPerSmIter);
        else if (nc == 2) enqueue_split64_ov<2>(g, st, kPerSmIter);
        else enqueue_split64_ov<1>(g, st, kPerSmIter);
    } else if (prec == 0 && nc == 3 && tiled32_ok(g) && g->slab64 > 0) {
        // fused p update + stencil (p double-buffered), then the update reading the new p
        const int blocks = grid_blocks(g, d.N / 2, kPerSmIter);
        enqueue_tiled64_a(g, st, g->slab64, MHD_KERNEL_SPMV64);
        const int s = prof_begin(g, st, MHD_KERNEL_UPDATE64);
        k_update<double, 2, 3, true><<<blocks, kThreads, 0, st>>>(d, g->x64, g->p64, g->r64, g->q64, g->tu.dg,
                                                                   g->sc, g->partials);
        prof_end(g, st, s);
    } else if (prec == 0) {
        enqueue_split_nc<double, 2>(g, st, nc, g->x64, g->r64, g->p64, g->q64, g->t64,
                                    grid_blocks(g, d.N / 2, kPerSmIter), MHD_KERNEL_PUPDATE64);
    } else if (g->slab32 <= -100) {
        // plane-marching pair with bulk-copy staging, when the autotuner measured it fastest
        enqueue_bulk32(g, st, nc, -100 - g->slab32);
    } else if (g->slab32 <= -6 && g->slab32 >= -8) {
        // single-reduction pair (residual kernel, then the update), when measured fastest
        if (use_v4(g)) enqueue_cgpair32_nc<4>(g, st, nc);
        else enqueue_cgpair32_nc<2>(g, st, nc);
    } else if (g->slab32 <= -3 && g->slab32 >= -5) {
        // recompute pair, when the autotuner measured it fastest (-4: the r update walks backwards,
        // -5: compiled for 6 CTAs per SM)
        if (use_v4(g)) enqueue_recompute32_var<4>(g, st, nc);
        else enqueue_recompute32_var<2>(g, st, nc);
    } else if (g->slab32 == -2) {
        // p update folded into the stencil, when the autotuner measured it fastest
        if (use_v4(g)) enqueue_fused32_nc<4>(g, st, nc);
        else enqueue_fused32_nc<2>(g, st, nc);
    } else if (tiled32_ok(g) && g->slab32 > 0) {
        // plane-marching pair, when the autotuner measured it faster than the split kernels
        enqueue_tiled32(g, st, nc, g->slab32, MHD_KERNEL_SPMV32, MHD_KERNEL_UPDATE32);
    } else if (use_v4(g)) {
        enqueue_split_nc<float, 4>(g, st, nc, g->x32, g->r32, g->p32, g->q32, g->t32,
                                   grid_blocks(g, d.N / 4, kPerSmIter), MHD_KERNEL_PUPDATE32);
    } else {
        enqueue_split_nc<float, 2>(g, st, nc, g->x32, g->r32, g->p32, g->q32, g->t32,
                                   grid_blocks(g, d.N / 2, kPerSmIter), MHD_KERNEL_PUPDATE32);
    }
}

// a CUDA graph of `graph_batch` iterations; every kernel returns at once after convergence
mhd_status_t iteration_graph(mhd_grid_s* g, int prec, int nc, cudaGraphExec_t* out) {
    cudaGraphExec_t& ge = g->iter_graph[prec][nc];
    if (ge) {
        *out = ge;
        return MHD_OK;
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return check_cuda(g, "iteration_graph: stream");
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return check_cuda(g, "iteration_graph: begin capture");
    }
    for (int it = 0; it < g->graph_batch; it++) enqueue_iteration(g, cs, prec, nc);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return set_error(g, MHD_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_error(g, MHD_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    *out = ge;
    return MHD_OK;
}

mhd_status_t read_scalars(mhd_grid_s* g) {
    if (cudaMemcpyAsync(g->h_sc, g->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess)
        return check_cuda(g, "read scalars");
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "sync");
    prof_flush(g);
    return MHD_OK;
}

// run batches of iterations until the device flags completion
mhd_status_t run_iterations(mhd_grid_s* g, int prec, int nc) {
    cudaGraphExec_t ge = nullptr;
    if (!g->prof) {
        mhd_status_t st = iteration_graph(g, prec, nc, &ge);
        if (st != MHD_OK) return st;
    }
    for (;;) {
        if (read_scalars(g) != MHD_OK) return MHD_ERR_CUDA;
        if (g->h_sc->done) return MHD_OK;
        if (g->prof) {
            // direct launches, each bracketed by events
            for (int it = 0; it < 2 * g->graph_batch; it++) enqueue_iteration(g, g->stream, prec, nc);
            if (check_cuda(g, "iteration launch") != MHD_OK) return MHD_ERR_CUDA;
            continue;
        }
        // launch two batches per poll to overlap the host round trip with device work
        if (cudaGraphLaunch(ge, g->stream) != cudaSuccess) return check_cuda(g, "graph launch");
        if (cudaGraphLaunch(ge, g->stream) != cudaSuccess) return check_cuda(g, "graph launch");
    }
}

// set the scalar block for a new solve (enqueued; no host sync)
__global__ void k_setup(PcgScalars* sc, double tol, double inner_tol, int max_iter) {
    sc->tol = tol;
    sc->inner_tol = inner_tol;
    sc->max_iter = max_iter;
    sc->done = 0;
    sc->iter = 0;
    sc->total_iter = 0;
    sc->outer = 0;
    sc->outer_done = 0;
    sc->rr_out = 0.0;
    sc->rho_prev = 0.0;
    sc->par = 0;
    sc->ax = 0.0;
    sc->count = 0u;
}

// mixed: the inner stop test reuses k_update's sqrt(rr) <= tol*sqrt(bb) by swapping in
// tol := inner_tol and bb := rr_out for the inner solve, then restoring them
__global__ void k_inner_begin(PcgScalars* sc, double* saved) {
    saved[0] = sc->tol;
    saved[1] = sc->bb;
    sc->tol = sc->inner_tol;
    sc->bb = sc->rr_out;
}
__global__ void k_inner_end(PcgScalars* sc, const double* saved) {
    sc->tol = saved[0];
    sc->bb = saved[1];
}

}  // namespace

namespace {
__global__ void k_tune_reset(PcgScalars* sc) {
    sc->done = 0;
    sc->alpha = 0.0;
    sc->beta = 0.0;
    sc->rho = 1.0;
    sc->tol = 0.0;
    sc->bb = 1.0;
    sc->iter = 0;
    sc->max_iter = 1 << 30;
    sc->par = 0;
    sc->ax = 0.0;
    sc->count = 0u;
}

// choose the r-slab length of the tiled FP32 kernels by timing a few iterations of each
// candidate (alpha = beta = 0, so the vectors are left as they are); run before a solve sets up
// its scalars
// Diagnostics: MHD_FORCE_SLAB=<n> skips the timing and uses slab n (-1: split kernels, -2 (FP32
// only): the p update folded into the stencil).
int forced_slab() {
    const char* f = std::getenv("MHD_FORCE_SLAB");
    return f ? (int)std::strtol(f, nullptr, 10) : 0;
}

mhd_status_t tune_slab32(mhd_grid_s* g, int nc) {
    if (g->slab32 != 0) return MHD_OK;
    if (const int f = forced_slab()) {
        if (f <= -2 && f >= -8) g->slab32 = f;
        else if (f <= -100) g->slab32 = (bulk32_ok(g) && f < -100) ? f : -1;
        else g->slab32 = (f > 0 && tiled32_ok(g) && tiled32_blocks(g, f) <= kMaxBlocks) ? f : -1;
        return MHD_OK;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return check_cuda(g, "tune events");
    int best = 0;
    float best_ms = 1e30f;
    const int prof = g->prof;
    g->prof = 0;
    // positive finite vectors (bytes 0x3F: 0.747f) so the timed iterations do real work and no
    // reduction trips a breakdown flag (the solve's set-up overwrites every vector afterwards)
    const size_t n3 = 3 * (size_t)g->d.N;
    // candidates -1: the split kernels (p update, stencil, update); -2: the p update folded into
    // the stencil, then the update; -3, -4, -5: the recompute pair (no q~ stored), forwards, with
    // the r update walking backwards, or at 6 CTAs per SM; -6, -7, -8: the single-reduction pair
    // (-7: its residual kernel unrolled over the components and both kernels at 3 CTAs per SM; -8:
    // the unrolled residual kernel with the update kernel at 4); -132,
    // -164: the recompute pair as plane-marching kernels staged by bulk copies (units of 32 or 64
    // planes). Four iterations each after one untimed: an even count, so each is timed with its
    // x updates.
    for (int cand : {-1, -2, -3, -4, -5, -6, -7, -8, -132, -164}) {
        if (cand <= -100 && !bulk32_ok(g)) continue;
        k_tune_reset<<<1, 1, 0, g->stream>>>(g->sc);
        g->slab32 = cand;
        cudaMemsetAsync(g->r32, 0x3F, sizeof(float) * n3, g->stream);
        cudaMemsetAsync(g->p32, 0x3F, sizeof(float) * 2 * n3, g->stream);
        cudaMemsetAsync(g->x32, 0, sizeof(float) * n3, g->stream);
        enqueue_iteration(g, g->stream, 1, nc);
        cudaEventRecord(e0, g->stream);
        for (int it = 0; it < 4; it++) enqueue_iteration(g, g->stream, 1, nc);
        cudaEventRecord(e1, g->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms *= 0.75f;   // per 3 iterations, as the tiled candidates below
        if (ms < best_ms) {
            best_ms = ms;
            best = cand;
        }
    }
    cudaMemsetAsync(g->r32, 0x3F, sizeof(float) * n3, g->stream);
    cudaMemsetAsync(g->p32, 0x3F, sizeof(float) * 2 * n3, g->stream);
    for (int slab : {8, 16, 32, 64}) {
        if (!tiled32_ok(g)) break;
        if (slab > 2 * g->d.nr && best > 0) break;
        if (tiled32_blocks(g, slab) > kMaxBlocks) continue;
        k_tune_reset<<<1, 1, 0, g->stream>>>(g->sc);
        enqueue_tiled32(g, g->stream, nc, slab, 0, 0);
        cudaEventRecord(e0, g->stream);
        for (int it = 0; it < 3; it++) enqueue_tiled32(g, g->stream, nc, slab, 0, 0);
        cudaEventRecord(e1, g->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = slab;
        }
    }
    g->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best == 0) return set_error(g, MHD_ERR_CUDA, "FP32 CG kernels: no launchable variant");
    g->slab32 = best;  // -1 split, -2 folded, -3/-4 recompute pair, <= -100 bulk-staged pair, > 0 tiled slab
    return check_cuda(g, "tune slab");
}
}  // namespace

namespace {
// FP64: time the split iteration against the fused tiled kernel A at each slab length (alpha =
// beta = 0 on positive finite vectors) and keep the fastest
mhd_status_t tune_slab64(mhd_grid_s* g) {
    if (g->slab64 != 0) return MHD_OK;
    if (const int f = forced_slab()) {
        g->slab64 = (f > 0 && tiled32_ok(g) && tiled32_blocks(g, f) <= kMaxBlocks) ? f : (f == -64 ? -2 : -1);
        return MHD_OK;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return check_cuda(g, "tune events");
    const int prof = g->prof;
    g->prof = 0;
    const size_t n3 = 3 * (size_t)g->d.N;
    cudaMemsetAsync(g->r64, 0x3F, sizeof(double) * n3, g->stream);
    cudaMemsetAsync(g->p64, 0x3F, sizeof(double) * 2 * n3, g->stream);
    int best = 0;
    float best_ms = 1e30f;
    for (int slab : {-1, -2, 8, 16, 32, 64}) {
        if (slab == -2 && !g->side) continue;
        if (slab > 0 && (!tiled32_ok(g) || tiled32_blocks(g, slab) > kMaxBlocks || (slab > 2 * g->d.nr && best != 0)))
            continue;
        g->slab64 = slab;
        k_tune_reset<<<1, 1, 0, g->stream>>>(g->sc);
        enqueue_iteration(g, g->stream, 0, 3);
        cudaEventRecord(e0, g->stream);
        for (int it = 0; it < 2; it++) enqueue_iteration(g, g->stream, 0, 3);
        cudaEventRecord(e1, g->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = slab;
        }
    }
    g->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g->slab64 = (best == 0) ? -1 : best;
    cudaMemsetAsync(g->p64, 0, sizeof(double) * 2 * n3, g->stream);
    return check_cuda(g, "tune slab64");
}
}  // namespace

namespace {
__global__ void k_set_unit(double* a) { *a = 1.0; }
}  // namespace

// kernel choices and CUDA graphs of 3-component solves, ahead of the first solve (mhd_grid_reserve);
// the tables are built for alpha = 1 so the timed trial iterations run on finite coefficients
mhd_status_t solver_reserve(mhd_grid_s* g, int features) {
    k_set_unit<<<1, 1, 0, g->stream>>>(&g->ss->alpha_user);
    build_tables(g, &g->ss->alpha_user, true);
    mhd_status_t st = check_cuda(g, "reserve: tables");
    if (st != MHD_OK) return st;
    cudaGraphExec_t ge = nullptr;
    if (features & MHD_RESERVE_PC1) {
        if (g->slab64 == 0 && (st = tune_slab64(g)) != MHD_OK) return st;
        if ((st = iteration_graph(g, 0, 3, &ge)) != MHD_OK) return st;
    }
    if (features & MHD_RESERVE_MIXED) {
        if (g->slab32 == 0 && (st = tune_slab32(g, 3)) != MHD_OK) return st;
        if ((st = iteration_graph(g, 1, 3, &ge)) != MHD_OK) return st;
    }
    if (features & MHD_RESERVE_CG) {
        if ((st = iteration_graph(g, 2, 3, &ge)) != MHD_OK) return st;
    }
    if (features & MHD_RESERVE_PC2) {
        if ((st = pc2_reserve(g)) != MHD_OK) return st;
        if ((st = iteration_graph(g, 3, 3, &ge)) != MHD_OK) return st;
        if (features & MHD_RESERVE_MIXED) {
            if (g->pc2_fused32 == 0) g->pc2_fused32 = (forced_slab() == -1) ? -1 : 1;
            if ((st = iteration_graph(g, 4, 3, &ge)) != MHD_OK) return st;
        }
    }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "reserve: sync");
    return MHD_OK;
}

mhd_status_t solve(mhd_grid_s* g, const double* alpha_dev, int nc, const double* b, double* x,
                   const double* x0, const mhd_params_t* prm, int* iters, int* outer, double* relres) {
    const Dims d = g->d;
    const bool mixed = (prm->precision == MHD_PREC_MIXED);
    build_tables(g, alpha_dev, mixed);
    const bool pc2 = (prm->preconditioner == 1);
    if (mixed && g->slab32 == 0 && !pc2) {
        mhd_status_t st = tune_slab32(g, 3);
        if (st != MHD_OK) return st;
    }
    if (!mixed && nc == 3 && g->slab64 == 0 && prm->pcg_variant == 0 && prm->preconditioner == 0) {
        mhd_status_t st = tune_slab64(g);
        if (st != MHD_OK) return st;
    }
    k_setup<<<1, 1, 0, g->stream>>>(g->sc, prm->tol, prm->inner_tol, prm->max_iter);
    const int blocks2 = grid_blocks(g, d.N / 2, kPerSmIter);
    if (!mixed) {
        k_init64<<<grid_blocks(g, d.N / 2, resident_per_sm<k_init64>()), kThreads, 0, g->stream>>>(
            d, nc, b, x0, g->x64, g->r64, g->p64, g->t64, g->tu, g->sc, g->partials);
        mhd_status_t st = check_cuda(g, "pcg init");
        if (st != MHD_OK) return st;
        if (pc2) {
            if ((st = pc2_factor(g)) != MHD_OK) return st;
            pc2_init64(g, nc);
        }
        st = run_iterations(g, pc2 ? 3 : (prm->pcg_variant == 1 ? 2 : 0), nc);
        if (st != MHD_OK) return st;
        k_finish64<<<blocks2, kThreads, 0, g->stream>>>(d, nc, g->x64, g->p64, x, g->t64.s, g->sc);
        if ((st = check_cuda(g, "pcg finish")) != MHD_OK) return st;
        if (read_scalars(g) != MHD_OK) return MHD_ERR_CUDA;
        const PcgScalars& h = *g->h_sc;
        if (iters) *iters = h.iter;
        if (outer) *outer = 0;
        if (relres) *relres = (h.bb > 0) ? std::sqrt(h.rr) / std::sqrt(h.bb) : 0.0;
        if (h.done == 1) return MHD_OK;
        if (h.done == 3) return set_error(g, MHD_ERR_NONFINITE, "pcg: non-finite value in a reduction");
        if (h.done == 4) return set_error(g, MHD_ERR_NOCONV, "pcg: breakdown (operator not positive definite)");
        return set_error(g, MHD_ERR_NOCONV, "pcg: no convergence within max_iter");
    }
    // mixed precision: x starts as x0 in FP64 (in place in the caller's x)
    if (x != x0)
        cudaMemcpyAsync(x, x0, sizeof(double) * nc * d.N, cudaMemcpyDeviceToDevice, g->stream);
    double* saved = g->partials + kMaxBlocks * kPartialsPerBlock;  // spare doubles past the partials
    if (pc2) {
        mhd_status_t st = pc2_factor(g);
        if (st != MHD_OK) return st;
        // the FP32 PC2 iteration folds the p update into the stencil unless the split kernels are
        // forced (MHD_FORCE_SLAB=-1): measured faster at every size tried
        if (g->pc2_fused32 == 0) g->pc2_fused32 = (forced_slab() == -1) ? -1 : 1;
    }
    int outer_done = 0;
    for (int o = 0; o <= prm->max_outer; o++) {
        const int ps = prof_begin(g, g->stream, MHD_KERNEL_OUTER_RES);
        const int restart = (o == 0 || prm->mixed_restart) ? 1 : 0;
        k_outer_res<2><<<grid_blocks(g, d.N / 2, resident_per_sm<k_outer_res<2>>()), kThreads, 0, g->stream>>>(
            d, nc, b, x, g->r32, (!pc2 && g->slab32 <= -6 && g->slab32 >= -8) ? g->q32 : nullptr, g->p32, g->x32, g->t64, g->tu, g->sc,
            g->partials, o == 0 ? 1 : 0, restart, pc2 ? 1 : 0, g->t32);
        if (pc2) pc2_reliable32(g, nc, restart);
        prof_end(g, g->stream, ps);
        mhd_status_t st = check_cuda(g, "outer residual");
        if (st != MHD_OK) return st;
        if (read_scalars(g) != MHD_OK) return MHD_ERR_CUDA;
        outer_done = g->h_sc->outer_done;
        if (outer_done || o == prm->max_outer) break;
        k_inner_begin<<<1, 1, 0, g->stream>>>(g->sc, saved);
        st = run_iterations(g, pc2 ? 4 : 1, nc);
        if (st != MHD_OK) return st;
        k_inner_end<<<1, 1, 0, g->stream>>>(g->sc, saved);
        if (g->h_sc->done == 6)
            return set_error(g, MHD_ERR_TIMEOUT, "pcg (mixed): a bounded wait for a bulk copy gave up");
        if (g->h_sc->done == 3) break;
        k_correct<<<blocks2, kThreads, 0, g->stream>>>(d, nc, x, g->x32, g->p32, g->t64.s, g->sc);
        if ((st = check_cuda(g, "correction")) != MHD_OK) return st;
    }
    if (read_scalars(g) != MHD_OK) return MHD_ERR_CUDA;
    const PcgScalars& h = *g->h_sc;
    if (iters) *iters = h.total_iter;
    if (outer) *outer = h.outer;
    if (relres) *relres = (h.bb > 0) ? std::sqrt(h.rr_out) / std::sqrt(h.bb) : 0.0;
    if (h.bb == 0.0) {
        cudaMemsetAsync(x, 0, sizeof(double) * nc * d.N, g->stream);
        return MHD_OK;
    }
    if (h.outer_done == 1) return MHD_OK;
    if (h.outer_done == 3 || h.done == 3) return set_error(g, MHD_ERR_NONFINITE, "pcg: non-finite value");
    return set_error(g, MHD_ERR_NOCONV, "pcg (mixed): no convergence within max_outer");
}

}  // namespace mhd
