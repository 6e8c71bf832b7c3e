// mhd_force_noalloc: the momentum force without a grid object and without any allocation.
//
// Who needs it: code that may not allocate device memory after it starts. Examples are a host
// application that hands this library a fixed device-memory budget and owns every buffer, a
// real-time or latency-bound loop where cudaMalloc (which can synchronise the device) is not
// allowed, and plug-in code run under an allocator policy that forbids new device allocations.
// mhd_grid_create allocates the grid's tables and workspace, so those callers cannot use
// mhd_force; this entry point takes the grid description instead and keeps all its scratch
// (metric tables, current density on edges, polar ring sums and harmonics) in one file-scope
// device array.
//
// The scratch array is static device memory: every GPU that loads the library holds it until
// the process exits. Its address is looked up once per device with cudaGetSymbolAddress on the
// first call made with that device current; make that first call before any stream capture.
// All calls share the array and every call overwrites what it reads, so nothing needs clearing,
// but two calls whose work overlaps on the GPU (different streams, or different host threads)
// race on it.
#include <cmath>
#include <mutex>

#include "mhd_internal.cuh"

namespace {

// 10 MiB of FP64 scratch: tables plus the three edge arrays of J plus the ring sums.
constexpr long long kScratchDoubles = 1310720;
constexpr long long kMaxCells = 262144;  // e.g. 64 x 64 x 64
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// radial nodes by repeated multiplication, one thread (the recurrence is sequential)
__global__ void k_noalloc_radial(int nr, double r0, double r1, double s, double* r) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double h0;
    if (s == 1.0) {
        h0 = (r1 - r0) / nr;
    } else {
        double snr = 1.0;
        for (int i = 0; i < nr; i++) snr *= s;
        h0 = (r1 - r0) * (s - 1.0) / (snr - 1.0);
    }
    r[0] = r0;
    double dr = h0;
    for (int i = 0; i < nr; i++) {
        r[i + 1] = r[i] + dr;
        dr *= s;
    }
}

// the remaining tables the force kernels read
__global__ void k_noalloc_tables(int nr, int nt, int np, double r0, double dth, double dph, const double* r,
                                 double* rc, double* sn, double* cn, double* sc, double* cc, double* rho, double* rhoV,
                                 double* pcs) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < np) {
        pcs[idx] = cos((idx + 0.5) * dph);
        pcs[np + idx] = sin((idx + 0.5) * dph);
    }
    if (idx <= nt) {
        sn[idx] = (idx == 0 || idx == nt) ? 0.0 : sin(idx * dth);
        cn[idx] = (idx == 0) ? 1.0 : (idx == nt ? -1.0 : cos(idx * dth));
    }
    if (idx < nt) {
        sc[idx] = sin((idx + 0.5) * dth);
        cc[idx] = cos((idx + 0.5) * dth);
    }
    if (idx < nr) {
        const double c = 0.5 * (r[idx] + r[idx + 1]);
        rc[idx] = c;
        rho[idx] = (r0 / c) * (r0 / c);
    }
    if (idx < nr * nt) {
        const int i = idx / nt, j = idx - i * nt;
        const double ri = r[i], ro = r[i + 1];
        const double c = 0.5 * (ri + ro);
        const double bj = (j == 0 ? 1.0 : cos(j * dth)) - (j + 1 == nt ? -1.0 : cos((j + 1) * dth));
        rhoV[idx] = (r0 / c) * (r0 / c) * ((ro * ro * ro - ri * ri * ri) / 3.0 * bj * dph);
    }
}

// the explicit kernels' geometric factors (the force's per-shell, per-row and per-edge-row tables),
// one thread per (i, j) of the (nr + 1) x (nt + 1) node grid
__global__ void k_noalloc_ex(mhd::GeoView g, double* sh, double* ihp, double* cot, double* jr, double* jt, double* jp) {
    const int nr = g.nr, nt = g.nt;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (nr + 1) * (nt + 1)) return;
    const int i = idx / (nt + 1), j = idx - i * (nt + 1);
    if (i < nr && j == 0) mhd::ex_shell(g, i, sh + 5 * (size_t)i);
    if (i == 0 && j < nt) cot[j] = mhd::ex_cot(g, j);
    if (i < nr && j < nt) ihp[(size_t)i * nt + j] = mhd::ex_ihp(g, i, j);
    if (i < nr) mhd::ex_jr(g, i, j, jr + 4 * ((size_t)i * (nt + 1) + j));
    if (j < nt) mhd::ex_jt(g, i, j, jt + 3 * ((size_t)i * nt + j));
    mhd::ex_jp(g, i, j, jp + 3 * ((size_t)i * (nt + 1) + j));
}

double* scratch_for_current_device(int* dev_out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    *dev_out = dev;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    return g_scratch_addr[dev];
}

}  // namespace

extern "C" mhd_status_t mhd_force_noalloc(const mhd_grid_desc_t* desc, const mhd_fields_t* f, double dt,
                                          double* b, void* cuda_stream) {
    if (!desc || !f || !b || !f->br || !f->bt || !f->bp || !f->vr || !f->vt || !f->vp) return MHD_ERR_ARG;
    const mhd_grid_desc_t d = *desc;
    if (d.nr < 2 || d.nt < 2 || d.np < 2 || (d.np % 2) != 0) return MHD_ERR_ARG;
    if (!(d.r0 > 0) || !(d.r1 > d.r0) || !(d.stretch > 0)) return MHD_ERR_ARG;
    const long long N = (long long)d.nr * d.nt * d.np;
    const long long nr = d.nr, nt = d.nt, np = d.np;
    // scratch layout (doubles): r, rc, sn, cn, sc, cc, rho, rhoV, the explicit tables (shell, 1/(r sin
    // dph), cot, edge rows), jr, jt, jp, ring, cos / sin of the phi centres, polar B_theta harmonics
    const long long n_ex = 5 * nr + nr * nt + nt + 4 * nr * (nt + 1) + 3 * (nr + 1) * nt + 3 * (nr + 1) * (nt + 1);
    const long long n_tab = (nr + 1) + nr + 2 * (nt + 1) + 2 * nt + nr + nr * nt + n_ex;
    const long long n_edge = nr * (nt + 1) * np + (nr + 1) * nt * np + (nr + 1) * (nt + 1) * np;
    const long long need = n_tab + n_edge + 2 * nr + 2 * np + 4 * nr + 20 * 16;  // +16 doubles alignment slack per table
    if (N > kMaxCells || need > kScratchDoubles) return MHD_ERR_ARG;

    int dev = 0;
    double* base = scratch_for_current_device(&dev);
    if (!base) return MHD_ERR_CUDA;
    long long off = 0;
    auto take = [&](long long n) {
        double* p = base + off;
        off += (n + 15) / 16 * 16;  // keep each table 128-byte aligned (double2 loads)
        return p;
    };
    double* r = take(nr + 1);
    double* rc = take(nr);
    double* sn = take(nt + 1);
    double* cn = take(nt + 1);
    double* sc = take(nt);
    double* cc = take(nt);
    double* rho = take(nr);
    double* rhoV = take(nr * nt);
    double* x_sh = take(5 * nr);
    double* x_ihp = take(nr * nt);
    double* x_cot = take(nt);
    double* x_jr = take(4 * nr * (nt + 1));
    double* x_jt = take(3 * (nr + 1) * nt);
    double* x_jp = take(3 * (nr + 1) * (nt + 1));
    double* jr = take(nr * (nt + 1) * np);
    double* jt = take((nr + 1) * nt * np);
    double* jp = take((nr + 1) * (nt + 1) * np);
    double* ring = take(2 * nr);
    double* pcs = take(2 * np);
    double* bharm = take(4 * nr);   // north and south B_theta rings; the adjoint half is not used here
    if (off > kScratchDoubles) return MHD_ERR_ARG;

    // a grid view on the stack whose tables and workspace live in the static scratch
    mhd_grid_s v{};
    v.d.nr = d.nr;
    v.d.nt = d.nt;
    v.d.np = d.np;
    v.d.N = N;
    v.desc = d;
    v.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    v.device = dev;
    if (cudaDeviceGetAttribute(&v.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MHD_ERR_CUDA;
    const double pi = 3.14159265358979323846;
    const double dth = pi / d.nt, dph = 2.0 * pi / d.np;
    // r1 of the table as the recurrence produces it (the force uses the last node)
    double r_last = d.r0;
    {
        double h0;
        if (d.stretch == 1.0) {
            h0 = (d.r1 - d.r0) / d.nr;
        } else {
            double snr = 1.0;
            for (int i = 0; i < d.nr; i++) snr *= d.stretch;
            h0 = (d.r1 - d.r0) * (d.stretch - 1.0) / (snr - 1.0);
        }
        double dr = h0;
        for (int i = 0; i < d.nr; i++) {
            r_last += dr;
            dr *= d.stretch;
        }
    }
    v.geo.r = r;
    v.geo.rc = rc;
    v.geo.sn = sn;
    v.geo.cn = cn;
    v.geo.sc = sc;
    v.geo.cc = cc;
    v.geo.rho = rho;
    v.geo.rhoV = rhoV;
    v.geo.kt2 = nullptr;
    v.geo.wr = v.geo.wt = v.geo.wp = nullptr;
    v.geo.r0 = d.r0;
    v.geo.r1 = r_last;
    v.geo.dth = dth;
    v.geo.dph = dph;
    v.geo.pcs = pcs;
    v.geo.pole_f = 2.0 / (d.np * std::cos(dth));
    v.ex.sh = x_sh;
    v.ex.ihp = x_ihp;
    v.ex.cot = x_cot;
    v.ex.jr = x_jr;
    v.ex.jt = x_jt;
    v.ex.jp = x_jp;
    v.ex.fr = v.ex.ft = v.ex.fp = nullptr;   // CT face factors: not used by the force
    v.er = jr;
    v.et = jt;
    v.ep = jp;
    v.ring = ring;
    v.bharm = bharm;

    k_noalloc_radial<<<1, 1, 0, v.stream>>>(d.nr, d.r0, d.r1, d.stretch, r);
    long long nt_work = nr * nt > nt + 1 ? nr * nt : nt + 1;
    if (np > nt_work) nt_work = np;
    k_noalloc_tables<<<(int)((nt_work + 255) / 256), 256, 0, v.stream>>>(d.nr, d.nt, d.np, d.r0, dth, dph, r, rc, sn,
                                                                         cn, sc, cc, rho, rhoV, pcs);
    const mhd::GeoView gv{r, rc, sn, cn, sc, cc, rho, d.nr, d.nt, d.r0, dth, dph};
    const long long nodes = (nr + 1) * (nt + 1);
    k_noalloc_ex<<<(int)((nodes + 255) / 256), 256, 0, v.stream>>>(gv, x_sh, x_ihp, x_cot, x_jr, x_jt, x_jp);
    mhd::force(&v, f->vr, f->vt, f->vp, nullptr, 0.0, f->br, f->bt, f->bp, nullptr, dt, nullptr, b);
    if (cudaGetLastError() != cudaSuccess) return MHD_ERR_CUDA;
    return MHD_OK;
}
