// Grid object: metric tables of the staggered spherical grid and all solver workspace.
//
// Geometry (exact finite-volume quantities of spherical cells on the staggered, logically
// rectangular, non-uniform mesh of Sec. 2.2):
//   V_ij   = (r_{i+1}^3 - r_i^3)/3 (cos th_j - cos th_{j+1}) dphi
//   A^r_ij = r_i^2 (cos th_j - cos th_{j+1}) dphi
//   A^t_ij = sin th_j (r_{i+1}^2 - r_i^2)/2 dphi        (zero at the poles)
//   A^p_i  = (r_{i+1}^2 - r_i^2)/2 dtheta
// Stiffness weights of K (rho A / centre distance): radial faces use rho0 at the face radius,
// theta and phi faces rho at the cell-centre radius; the inner face carries the Dirichlet
// weight rho0(r0) A^r_0j / (rc_0 - r0).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "mhd_internal.cuh"

namespace mhd {

static std::mutex g_err_mu;
static std::string g_create_error;

mhd_status_t set_error(mhd_grid_s* g, mhd_status_t st, const std::string& msg) {
    if (g) g->last_error = msg;
    else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_create_error = msg;
    }
    return st;
}

mhd_status_t check_cuda(mhd_grid_s* g, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(g, MHD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return MHD_OK;
}

int grid_blocks(const mhd_grid_s* g, long long work, int per_sm) {
    long long b = (work + kThreads - 1) / kThreads;
    long long cap = (long long)g->num_sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    if (b > kMaxBlocks) b = kMaxBlocks;
    return (int)b;
}

int prof_begin(mhd_grid_s* g, cudaStream_t st, int kernel) {
    if (!g->prof) return -1;
    if (g->prof_nslot >= mhd_grid_s::kProfSlots) {
        cudaStreamSynchronize(st);
        if (g->side && st != g->side) cudaStreamSynchronize(g->side);   // slots recorded on the side stream
        if (st != g->stream) cudaStreamSynchronize(g->stream);
        prof_flush(g);
    }
    const int s = g->prof_nslot++;
    g->prof_kid[s] = kernel;
    cudaEventRecord(g->prof_ev[2 * s], st);
    return s;
}

void prof_end(mhd_grid_s* g, cudaStream_t st, int slot) {
    if (slot >= 0) cudaEventRecord(g->prof_ev[2 * slot + 1], st);
}

void prof_flush(mhd_grid_s* g) {
    for (int s = 0; s < g->prof_nslot; s++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->prof_ev[2 * s], g->prof_ev[2 * s + 1]) == cudaSuccess) {
            g->prof_ms[g->prof_kid[s]] += ms;
            g->prof_cnt[g->prof_kid[s]] += 1;
        }
    }
    cudaGetLastError();
    g->prof_nslot = 0;
}

}  // namespace mhd

using namespace mhd;

namespace {

struct HostGeo {
    std::vector<double> r, rc, sn, cn, sc, cc, rho, rhoV, kt2, wr, wt, wp;
    double max_kt2 = 0;
};

HostGeo make_geo(const mhd_grid_desc_t& d) {
    const int nr = d.nr, nt = d.nt, np = d.np;
    const double pi = 3.14159265358979323846;
    const double dth = pi / nt, dph = 2.0 * pi / np;
    HostGeo h;
    h.r.resize(nr + 1);
    h.rc.resize(nr);
    h.sn.resize(nt + 1);
    h.cn.resize(nt + 1);
    h.sc.resize(nt);
    h.cc.resize(nt);
    h.rho.resize(nr);
    h.rhoV.resize((size_t)nr * nt);
    h.kt2.resize((size_t)nr * nt);
    h.wr.assign((size_t)(nr + 1) * nt, 0.0);
    h.wt.assign((size_t)nr * (nt + 1), 0.0);
    h.wp.assign((size_t)nr * nt, 0.0);
    // radial nodes by repeated multiplication (identical bits on every host)
    double h0;
    if (d.stretch == 1.0) {
        h0 = (d.r1 - d.r0) / nr;
    } else {
        double snr = 1.0;
        for (int i = 0; i < nr; i++) snr *= d.stretch;
        h0 = (d.r1 - d.r0) * (d.stretch - 1.0) / (snr - 1.0);
    }
    h.r[0] = d.r0;
    double dr = h0;
    for (int i = 0; i < nr; i++) {
        h.r[i + 1] = h.r[i] + dr;
        dr *= d.stretch;
    }
    for (int i = 0; i < nr; i++) h.rc[i] = 0.5 * (h.r[i] + h.r[i + 1]);
    for (int j = 0; j <= nt; j++) {
        h.sn[j] = std::sin(j * dth);
        h.cn[j] = std::cos(j * dth);
    }
    h.sn[0] = 0.0;
    h.sn[nt] = 0.0;
    h.cn[0] = 1.0;
    h.cn[nt] = -1.0;
    for (int j = 0; j < nt; j++) {
        h.sc[j] = std::sin((j + 0.5) * dth);
        h.cc[j] = std::cos((j + 0.5) * dth);
    }
    auto rho0 = [&](double r) { return (d.r0 / r) * (d.r0 / r); };
    for (int i = 0; i < nr; i++) {
        const double ri = h.r[i], ro = h.r[i + 1];
        const double ring = 0.5 * (ro * ro - ri * ri);
        h.rho[i] = rho0(h.rc[i]);
        for (int j = 0; j < nt; j++) {
            const double band = h.cn[j] - h.cn[j + 1];
            const double vol = (ro * ro * ro - ri * ri * ri) / 3.0 * band * dph;
            h.rhoV[(size_t)i * nt + j] = h.rho[i] * vol;
            const double a = ro - ri, b = h.rc[i] * dth, c = h.rc[i] * h.sc[j] * dph;
            const double k2 = 1.0 / (a * a) + 1.0 / (b * b) + 1.0 / (c * c);
            h.kt2[(size_t)i * nt + j] = k2;
            if (k2 > h.max_kt2) h.max_kt2 = k2;
            h.wp[(size_t)i * nt + j] = h.rho[i] * (ring * dth) / c;
        }
        for (int j = 1; j < nt; j++)
            h.wt[(size_t)i * (nt + 1) + j] = h.rho[i] * (h.sn[j] * ring * dph) / (h.rc[i] * dth);
    }
    for (int j = 0; j < nt; j++) {
        const double band = h.cn[j] - h.cn[j + 1];
        h.wr[j] = rho0(d.r0) * (d.r0 * d.r0 * band * dph) / (h.rc[0] - d.r0);
        for (int i = 1; i < nr; i++)
            h.wr[(size_t)i * nt + j] =
                rho0(h.r[i]) * (h.r[i] * h.r[i] * band * dph) / (h.rc[i] - h.rc[i - 1]);
        h.wr[(size_t)nr * nt + j] = 0.0;
    }
    return h;
}

// geometric factors of the explicit kernels (ExTab), one row at a time from the 1-D metric tables
// (the ex_* row functions); each factor is evaluated once here instead of once per element
struct HostEx {
    std::vector<double> sh, ihp, cot, jr, jt, jp, fr, ft, fp;
};

HostEx make_ex(const HostGeo& h, const mhd_grid_desc_t& d) {
    const int nr = d.nr, nt = d.nt;
    const double pi = 3.14159265358979323846;
    GeoView g{h.r.data(), h.rc.data(), h.sn.data(), h.cn.data(), h.sc.data(), h.cc.data(), h.rho.data(),
              nr, nt, d.r0, pi / nt, 2.0 * pi / d.np};
    HostEx x;
    x.sh.assign(5 * (size_t)nr, 0.0);
    x.ihp.assign((size_t)nr * nt, 0.0);
    x.cot.assign(nt, 0.0);
    x.jr.assign(4 * (size_t)nr * (nt + 1), 0.0);
    x.jt.assign(3 * (size_t)(nr + 1) * nt, 0.0);
    x.jp.assign(3 * (size_t)(nr + 1) * (nt + 1), 0.0);
    x.fr.assign(3 * (size_t)(nr + 1) * nt, 0.0);
    x.ft.assign(3 * (size_t)nr * (nt + 1), 0.0);
    x.fp.assign(3 * (size_t)nr * nt, 0.0);
    for (int i = 0; i < nr; i++) {
        ex_shell(g, i, &x.sh[5 * (size_t)i]);
        for (int j = 0; j < nt; j++) x.ihp[(size_t)i * nt + j] = ex_ihp(g, i, j);
        for (int j = 0; j <= nt; j++) ex_jr(g, i, j, &x.jr[4 * ((size_t)i * (nt + 1) + j)]);
        for (int j = 0; j <= nt; j++) ex_ft(g, i, j, &x.ft[3 * ((size_t)i * (nt + 1) + j)]);
        for (int j = 0; j < nt; j++) ex_fp(g, i, j, &x.fp[3 * ((size_t)i * nt + j)]);
    }
    for (int j = 0; j < nt; j++) x.cot[j] = ex_cot(g, j);
    for (int i = 0; i <= nr; i++) {
        for (int j = 0; j < nt; j++) ex_jt(g, i, j, &x.jt[3 * ((size_t)i * nt + j)]);
        for (int j = 0; j <= nt; j++) ex_jp(g, i, j, &x.jp[3 * ((size_t)i * (nt + 1) + j)]);
        for (int j = 0; j < nt; j++) ex_fr(g, i, j, &x.fr[3 * ((size_t)i * nt + j)]);
    }
    return x;
}

template <typename T>
bool dalloc(T** p, size_t n, std::vector<void*>& owned) {
    void* m = nullptr;
    if (cudaMalloc(&m, n * sizeof(T) + 256) != cudaSuccess) return false;
    owned.push_back(m);
    *p = reinterpret_cast<T*>(m);
    return true;
}

// rows [i0, i1) of the global grid's tables (the whole grid when i0 = 0, i1 = nr)
HostGeo slice_geo(const HostGeo& a, int nr_global, int nt, int i0, int i1) {
    if (i0 == 0 && i1 == nr_global) return a;
    HostGeo h;
    const size_t t = (size_t)nt, t1 = (size_t)nt + 1;
    h.r.assign(a.r.begin() + i0, a.r.begin() + i1 + 1);
    h.rc.assign(a.rc.begin() + i0, a.rc.begin() + i1);
    h.rho.assign(a.rho.begin() + i0, a.rho.begin() + i1);
    h.sn = a.sn;
    h.cn = a.cn;
    h.sc = a.sc;
    h.cc = a.cc;
    h.rhoV.assign(a.rhoV.begin() + i0 * t, a.rhoV.begin() + i1 * t);
    h.kt2.assign(a.kt2.begin() + i0 * t, a.kt2.begin() + i1 * t);
    h.wr.assign(a.wr.begin() + i0 * t, a.wr.begin() + (i1 + 1) * t);
    h.wt.assign(a.wt.begin() + i0 * t1, a.wt.begin() + i1 * t1);
    h.wp.assign(a.wp.begin() + i0 * t, a.wp.begin() + i1 * t);
    h.max_kt2 = a.max_kt2;
    return h;
}

mhd_status_t create_grid(const mhd_grid_desc_t* desc, int i0, int i1, bool as_slab, void* cuda_stream, mhd_grid_t* out);

}  // namespace

extern "C" mhd_status_t mhd_grid_create(const mhd_grid_desc_t* desc, void* cuda_stream, mhd_grid_t* out) {
    if (!desc || !out) return set_error(nullptr, MHD_ERR_ARG, "mhd_grid_create: null argument");
    return create_grid(desc, 0, desc->nr, false, cuda_stream, out);
}

extern "C" mhd_status_t mhd_grid_create_slab(const mhd_grid_desc_t* desc, int i0, int i1, void* cuda_stream,
                                             mhd_grid_t* out) {
    if (!desc || !out) return set_error(nullptr, MHD_ERR_ARG, "mhd_grid_create_slab: null argument");
    if (i0 < 0 || i1 > desc->nr || i1 - i0 < 2)
        return set_error(nullptr, MHD_ERR_ARG, "mhd_grid_create_slab: need 0 <= i0, i1 <= nr, i1 - i0 >= 2");
    return create_grid(desc, i0, i1, true, cuda_stream, out);
}

namespace {
mhd_status_t create_grid(const mhd_grid_desc_t* desc, int i0, int i1, bool as_slab, void* cuda_stream,
                         mhd_grid_t* out) {
    *out = nullptr;
    const mhd_grid_desc_t dg = *desc;
    if (dg.nr < 2 || dg.nt < 2 || dg.np < 2 || (dg.np % 2) != 0)
        return set_error(nullptr, MHD_ERR_ARG, "mhd_grid_create: need nr>=2, nt>=2, np even >= 2");
    if (!(dg.r0 > 0) || !(dg.r1 > dg.r0) || !(dg.stretch > 0))
        return set_error(nullptr, MHD_ERR_ARG, "mhd_grid_create: need 0 < r0 < r1, stretch > 0");
    // a slab grid, even one holding every row (a decomposition over one rank), takes the slab calls
    const bool slab = as_slab;
    // a slab is described by its own rows: nr = i1 - i0, r0 and r1 its first and last radial nodes
    const HostGeo hg = make_geo(dg);
    mhd_grid_desc_t d = dg;
    if (slab) {
        d.nr = i1 - i0;
        d.r0 = hg.r[i0];
        d.r1 = hg.r[i1];
    }
    const long long N = (long long)d.nr * d.nt * d.np;
    // every flat index the kernels split (three face or edge families together) stays below 2^31
    if (N > (1LL << 30) || 3LL * (d.nr + 1) * (d.nt + 1) * d.np >= (1LL << 31))
        return set_error(nullptr, MHD_ERR_ARG, "mhd_grid_create: grid too large");

    mhd_grid_s* g = new mhd_grid_s();
    g->d.nr = d.nr;
    g->d.nt = d.nt;
    g->d.np = d.np;
    g->d.N = N;
    g->desc = d;
    g->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    g->graph_batch = 16;
    std::memset(g->iter_graph, 0, sizeof(g->iter_graph));
    if (cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking) != cudaSuccess) g->side = nullptr;
    for (int q = 0; q < 4; q++)
        if (cudaEventCreateWithFlags(&g->side_ev[q], cudaEventDisableTiming) != cudaSuccess) g->side_ev[q] = nullptr;
    cudaGetLastError();

    HostGeo h = slice_geo(hg, dg.nr, d.nt, i0, i1);
    HostEx hx = make_ex(h, d);
    g->max_kt2 = h.max_kt2;
    std::vector<void*> owned;
    const int nr = d.nr, nt = d.nt;
    const size_t n3 = 3 * (size_t)N;
    bool ok = true;
    double *r, *rc, *sn, *cn, *sc, *cc, *rho, *rhoV, *kt2, *wr, *wt, *wp;
    ok = ok && dalloc(&r, nr + 1, owned) && dalloc(&rc, nr, owned) && dalloc(&sn, nt + 1, owned) &&
         dalloc(&cn, nt + 1, owned) && dalloc(&sc, nt, owned) && dalloc(&cc, nt, owned) &&
         dalloc(&rho, nr, owned) && dalloc(&rhoV, (size_t)nr * nt, owned) &&
         dalloc(&kt2, (size_t)nr * nt, owned) && dalloc(&wr, (size_t)(nr + 1) * nt, owned) &&
         dalloc(&wt, (size_t)nr * (nt + 1), owned) && dalloc(&wp, (size_t)nr * nt, owned);
    double *x_sh, *x_ihp, *x_cot, *x_jr, *x_jt, *x_jp, *x_fr, *x_ft, *x_fp;
    ok = ok && dalloc(&x_sh, hx.sh.size(), owned) && dalloc(&x_ihp, hx.ihp.size(), owned) &&
         dalloc(&x_cot, hx.cot.size(), owned) && dalloc(&x_jr, hx.jr.size(), owned) &&
         dalloc(&x_jt, hx.jt.size(), owned) && dalloc(&x_jp, hx.jp.size(), owned) &&
         dalloc(&x_fr, hx.fr.size(), owned) && dalloc(&x_ft, hx.ft.size(), owned) && dalloc(&x_fp, hx.fp.size(), owned);
    ok = ok && dalloc(&g->t64.ar, (size_t)(nr + 1) * nt, owned) &&
         dalloc(&g->t64.at, (size_t)nr * (nt + 1), owned) && dalloc(&g->t64.ap, (size_t)nr * nt, owned) &&
         dalloc(&g->t64.s, (size_t)nr * nt, owned);
    ok = ok && dalloc(&g->t32.ar, (size_t)(nr + 1) * nt, owned) &&
         dalloc(&g->t32.at, (size_t)nr * (nt + 1), owned) && dalloc(&g->t32.ap, (size_t)nr * nt, owned) &&
         dalloc(&g->t32.s, (size_t)nr * nt, owned);
    ok = ok && dalloc(&g->tu.dg, (size_t)nr * nt, owned) && dalloc(&g->tu.awr, (size_t)(nr + 1) * nt, owned) &&
         dalloc(&g->tu.awt, (size_t)nr * (nt + 1), owned) && dalloc(&g->tu.awp, (size_t)nr * nt, owned);
    ok = ok && dalloc(&g->x64, n3, owned) && dalloc(&g->r64, n3, owned) && dalloc(&g->p64, 2 * n3, owned) &&
         dalloc(&g->q64, n3, owned);
    ok = ok && dalloc(&g->x32, n3, owned) && dalloc(&g->r32, n3, owned) && dalloc(&g->p32, 2 * n3, owned) &&
         dalloc(&g->q32, n3, owned);
    ok = ok && dalloc(&g->b0, n3, owned) && dalloc(&g->b1, n3, owned) && dalloc(&g->dlt, n3, owned);
    ok = ok && dalloc(&g->er, (size_t)nr * (nt + 1) * d.np, owned) &&
         dalloc(&g->et, (size_t)(nr + 1) * nt * d.np, owned) &&
         dalloc(&g->ep, (size_t)(nr + 1) * (nt + 1) * d.np, owned) && dalloc(&g->ec, n3, owned) &&
         dalloc(&g->ring, 2 * (size_t)nr, owned) && dalloc(&g->sts_tab, 8 * (size_t)nr * nt, owned);
    double* pcs = nullptr;
    ok = ok && dalloc(&pcs, 2 * (size_t)d.np, owned) && dalloc(&g->bharm, 8 * (size_t)nr, owned) &&
         dalloc(&g->slab_out, 8 + 2 * (size_t)nt, owned);
    g->slab_i0 = slab ? i0 : 0;
    g->slab_nr_global = slab ? dg.nr : 0;
    ok = ok && dalloc(&g->partials, (size_t)kMaxBlocks * kPartialsPerBlock + 16, owned) &&
         dalloc(&g->sc, 1, owned) && dalloc(&g->ss, 1, owned);
    if (!ok) {
        for (void* m : owned) cudaFree(m);
        if (g->side) cudaStreamDestroy(g->side);
        for (auto& e : g->side_ev)
            if (e) cudaEventDestroy(e);
        cudaGetLastError();
        delete g;
        return set_error(nullptr, MHD_ERR_OOM, "mhd_grid_create: device allocation failed");
    }
    if (cudaMallocHost(&g->h_sc, sizeof(PcgScalars)) != cudaSuccess ||
        cudaMallocHost(&g->h_ss, sizeof(StepScalars)) != cudaSuccess ||
        cudaMallocHost(&g->h_alpha, 8 * sizeof(double)) != cudaSuccess) {
        for (void* m : owned) cudaFree(m);
        if (g->side) cudaStreamDestroy(g->side);
        for (auto& e : g->side_ev)
            if (e) cudaEventDestroy(e);
        cudaGetLastError();
        delete g;
        return set_error(nullptr, MHD_ERR_OOM, "mhd_grid_create: pinned host allocation failed");
    }
    // the single block of device memory list is kept for destroy
    auto* keep = new std::vector<void*>(owned);
    g->geo_mem = keep;

    auto up = [&](double* dst, const std::vector<double>& src) {
        return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice,
                               g->stream) == cudaSuccess;
    };
    ok = up(r, h.r) && up(rc, h.rc) && up(sn, h.sn) && up(cn, h.cn) && up(sc, h.sc) && up(cc, h.cc) &&
         up(rho, h.rho) && up(rhoV, h.rhoV) && up(kt2, h.kt2) && up(wr, h.wr) && up(wt, h.wt) && up(wp, h.wp);
    ok = ok && up(x_sh, hx.sh) && up(x_ihp, hx.ihp) && up(x_cot, hx.cot) && up(x_jr, hx.jr) && up(x_jt, hx.jt) &&
         up(x_jp, hx.jp) && up(x_fr, hx.fr) && up(x_ft, hx.ft) && up(x_fp, hx.fp);
    std::vector<double> h_pcs(2 * (size_t)d.np);
    for (int k = 0; k < d.np; k++) {
        const double ph = (k + 0.5) * (2.0 * 3.14159265358979323846 / d.np);
        h_pcs[k] = std::cos(ph);
        h_pcs[d.np + k] = std::sin(ph);
    }
    ok = ok && up(pcs, h_pcs);
    ok = ok && cudaMemsetAsync(g->bharm, 0, sizeof(double) * 8 * nr, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->partials, 0, sizeof(double) * kMaxBlocks * kPartialsPerBlock, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->sc, 0, sizeof(PcgScalars), g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->ss, 0, sizeof(StepScalars), g->stream) == cudaSuccess;
    // zero the FP32 p buffers once so the first fused update never reads garbage
    // every solver vector starts finite (0 * garbage could otherwise be NaN)
    ok = ok && cudaMemsetAsync(g->p32, 0, sizeof(float) * 2 * n3, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->x32, 0, sizeof(float) * n3, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->r32, 0, sizeof(float) * n3, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->q32, 0, sizeof(float) * n3, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->p64, 0, sizeof(double) * 2 * n3, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->x64, 0, sizeof(double) * n3, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->r64, 0, sizeof(double) * n3, g->stream) == cudaSuccess;
    ok = ok && cudaMemsetAsync(g->q64, 0, sizeof(double) * n3, g->stream) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(g->stream) == cudaSuccess;
    if (!ok) {
        mhd_grid_destroy(g);
        return set_error(nullptr, MHD_ERR_CUDA, "mhd_grid_create: table upload failed");
    }
    Geo& G = g->geo;
    G.r = r; G.rc = rc; G.sn = sn; G.cn = cn; G.sc = sc; G.cc = cc; G.rho = rho; G.rhoV = rhoV;
    G.kt2 = kt2; G.wr = wr; G.wt = wt; G.wp = wp;
    G.r0 = d.r0;
    G.r1 = h.r[nr];
    G.dth = 3.14159265358979323846 / nt;
    G.dph = 2.0 * 3.14159265358979323846 / d.np;
    G.max_kt2 = h.max_kt2;
    G.pcs = pcs;
    G.pole_f = 2.0 / (d.np * std::cos(G.dth));
    ExTab& X = g->ex;
    X.sh = x_sh; X.ihp = x_ihp; X.cot = x_cot; X.jr = x_jr; X.jt = x_jt; X.jp = x_jp;
    X.fr = x_fr; X.ft = x_ft; X.fp = x_fp;
    // row sums of |D^-1 K| (the Dirichlet weight sits on the diagonal only)
    double lam = 0.0;
    for (int i = 0; i < nr; i++)
        for (int j = 0; j < nt; j++) {
            const double s = h.wr[(size_t)i * nt + j] + h.wr[(size_t)(i + 1) * nt + j] + h.wt[(size_t)i * (nt + 1) + j] +
                             h.wt[(size_t)i * (nt + 1) + j + 1] + 2.0 * h.wp[(size_t)i * nt + j];
            const double off = s - (i == 0 ? h.wr[j] : 0.0);
            lam = std::max(lam, (s + off) / h.rhoV[(size_t)i * nt + j]);
        }
    g->visc_lambda_unit = lam;
    *out = g;
    return MHD_OK;
}

}  // namespace

extern "C" mhd_status_t mhd_grid_reserve(mhd_grid_t g, int features) {
    if (!g) return MHD_ERR_ARG;
    if (g->slab_nr_global > 0) return set_error(g, MHD_ERR_ARG, "mhd_grid_reserve: not available on a slab grid");
    if (features & ~MHD_RESERVE_ALL) return set_error(g, MHD_ERR_ARG, "mhd_grid_reserve: unknown feature bit");
    mhd_status_t st = solver_reserve(g, features);
    if (st != MHD_OK) return st;
    if ((features & MHD_RESERVE_RESISTIVITY) && (st = res_reserve(g)) != MHD_OK) return st;
    if ((features & MHD_RESERVE_ADJOINT) && (st = adjoint_reserve(g)) != MHD_OK) return st;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "mhd_grid_reserve");
    return MHD_OK;
}

extern "C" mhd_status_t mhd_grid_destroy(mhd_grid_t g) {
    if (!g) return MHD_OK;
    cudaStreamSynchronize(g->stream);
    batched_forget(g);
    adjoint_free(g);
    res_free(g);
    pc2_free(g);
    for (auto& row : g->iter_graph)
        for (auto& ge : row)
            if (ge) cudaGraphExecDestroy(ge);
    if (g->geo_mem) {
        auto* keep = reinterpret_cast<std::vector<void*>*>(g->geo_mem);
        for (void* m : *keep) cudaFree(m);
        delete keep;
    }
    if (g->h_sc) cudaFreeHost(g->h_sc);
    if (g->h_ss) cudaFreeHost(g->h_ss);
    if (g->h_alpha) cudaFreeHost(g->h_alpha);
    if (g->prof_ev[0])
        for (auto& e : g->prof_ev) cudaEventDestroy(e);
    if (g->side) cudaStreamDestroy(g->side);
    for (auto& e : g->side_ev)
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    delete g;
    return MHD_OK;
}

extern "C" mhd_status_t mhd_grid_sizes(mhd_grid_t g, long long sizes[6]) {
    if (!g || !sizes) return MHD_ERR_ARG;
    const long long nr = g->d.nr, nt = g->d.nt, np = g->d.np;
    sizes[0] = (nr + 1) * nt * np;
    sizes[1] = nr * (nt + 1) * np;
    sizes[2] = nr * nt * np;
    sizes[3] = sizes[4] = sizes[5] = nr * nt * np;
    return MHD_OK;
}

extern "C" mhd_status_t mhd_profile_enable(mhd_grid_t g, int enable) {
    if (!g) return MHD_ERR_ARG;
    cudaStreamSynchronize(g->stream);
    if (enable && !g->prof_ev[0]) {
        for (auto& e : g->prof_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return check_cuda(g, "profile events");
    }
    g->prof = enable ? 1 : 0;
    g->prof_nslot = 0;
    for (int k = 0; k < MHD_KERNEL_COUNT; k++) {
        g->prof_ms[k] = 0.0;
        g->prof_cnt[k] = 0;
    }
    return MHD_OK;
}

extern "C" mhd_status_t mhd_profile_read(mhd_grid_t g, int kernel, double* total_ms, long long* launches) {
    if (!g || kernel < 0 || kernel >= MHD_KERNEL_COUNT) return MHD_ERR_ARG;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return check_cuda(g, "profile sync");
    prof_flush(g);
    if (total_ms) *total_ms = g->prof_ms[kernel];
    if (launches) *launches = g->prof_cnt[kernel];
    return MHD_OK;
}

extern "C" mhd_status_t mhd_grid_kernel_forms(mhd_grid_t g, int* fp64_form, int* fp32_form) {
    if (!g) return MHD_ERR_ARG;
    if (fp64_form) *fp64_form = g->slab64;
    if (fp32_form) *fp32_form = g->slab32;
    return MHD_OK;
}

extern "C" const char* mhd_last_error(mhd_grid_t g) {
    if (g) return g->last_error.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    return g_create_error.c_str();
}
