// Internal declarations of the sm_103a zero-beta MHD library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>

#include "mhd.h"

namespace mhd {

constexpr int kThreads = 256;       // threads per CTA for every grid-stride kernel
constexpr int kMaxBlocks = 4096;    // capacity of the per-block partial-sum array
constexpr int kPartialsPerBlock = 4;

// Device-resident scalars of one PCG solve. Written only by the last CTA of a reducing
// kernel (fixed-order sum of the per-CTA partials, so results are deterministic).
struct PcgScalars {
    double rho;      // <r~, r~> (scaled residual, = <r, z> of the unscaled Jacobi PCG)
    double rr;       // ||r||_2^2 of the unscaled residual (stop test)
    double bb;       // ||b||_2^2
    double pq;       // <p~, A~ p~>
    double alpha, beta;
    double tol;      // stop when sqrt(rr) <= tol * sqrt(bb)   (FP64 solve / outer loop)
    double rr_out;   // mixed: squared norm of the current outer FP64 residual
    double inner_tol;
    double rho_prev; // rho of the previous CG iteration (residual replacement keeps the recurrence)
    int iter;        // iterations of the current (inner) solve
    int max_iter;
    int done;        // 0 running, 1 converged, 2 iteration cap, 3 non-finite, 4 breakdown, 6 device
                     // wait timeout (bulk-copy pipeline)
    int outer;       // mixed: outer passes done
    int outer_done;  // mixed: 0 running, 1 converged, 3 non-finite
    int total_iter;  // mixed: inner iterations summed over the outer passes
    unsigned int count;  // last-block ticket
    int par;         // FP32 tiled path: which of the two p buffers holds the current p
    double dte;      // implicit resistivity: dt eta of the current solve
    double ax;       // alpha of the last CG iteration whose alpha p~ has not yet been added to x~
    double pqc[3];   // per-component shares of <p~, q~> (FP64 iteration with the components overlapped)
    double wp;       // FP32 single-reduction pair: <r~, A~ p~_old> summed by the update kernel
};

// Device-resident scalars of one step.
struct StepScalars {
    double dt, cf, cw, alpha_si, alpha_nu;
    double max_kv2, max_kva2, max_kt2;
    double alpha_user;   // alpha of a direct operator/solver call
    int status;      // MHD_OK or MHD_ERR_ARG (C_f >= 1 / no dt)
    unsigned int count;
};

struct Dims {
    int nr, nt, np;
    int pad;
    long long N;
};

// flat indices of the field layouts: [nr(+1)][nt][np] (ix) and [nr][nt+1][np] (ixt); periodic phi
__device__ __forceinline__ long long ix(const Dims& d, int i, int j, int k) {
    return ((long long)i * d.nt + j) * d.np + k;
}
__device__ __forceinline__ long long ixt(const Dims& d, int i, int j, int k) {
    return ((long long)i * (d.nt + 1) + j) * d.np + k;
}
__device__ __forceinline__ int kp1(const Dims& d, int k) { return (k + 1 == d.np) ? 0 : k + 1; }
__device__ __forceinline__ int km1(const Dims& d, int k) { return (k == 0) ? d.np - 1 : k - 1; }
// (phi index, row) of a flat index of an array made of rows of np elements; every array of a grid
// has fewer than 2^31 elements (checked at grid creation), so 32-bit division suffices
__device__ __forceinline__ void split_np(const Dims& d, long long e, int& k, unsigned int& row) {
    const unsigned int u = (unsigned int)e;
    row = u / (unsigned int)d.np;
    k = (int)(u - row * (unsigned int)d.np);
}

// Per-grid FP64 metric tables (device). Built on the host from the grid definition.
struct Geo {
    const double* r;     // [nr+1] radial nodes
    const double* rc;    // [nr]   radial centres
    const double* sn;    // [nt+1] sin(theta_j), exact 0 at the poles
    const double* cn;    // [nt+1] cos(theta_j), exact +-1 at the poles
    const double* sc;    // [nt]   sin of theta centres
    const double* cc;    // [nt]   cos of theta centres
    const double* rho;   // [nr]   rho0 at radial centres
    const double* rhoV;  // [nr*nt] rho_c V_c
    const double* kt2;   // [nr*nt] k~^2 at cell centres
    const double* wr;    // [(nr+1)*nt] radial-face weights (wr[0] = Dirichlet weight at r0,
                         //             wr[nr] = 0: Neumann at r1)
    const double* wt;    // [nr*(nt+1)] theta-face weights (0 at the poles)
    const double* wp;    // [nr*nt] phi-face weight (each of the two faces)
    const double* pcs;   // [2*np] cos, then sin, of the phi centres (polar pole values)
    double r0, r1, dth, dph;
    double max_kt2;
    double pole_f;       // 2 / (np cos(dth)): first-harmonic pole value of the B_theta face ring
};

// B_theta at a cell centre of a polar ring (reading R4): the mean of the non-polar face value and
// of the pole value along the cell's meridian. The pole value is the first phi harmonic of the
// B_theta face ring next to the pole (h: that ring's sums of B_theta cos(phi_c) and B_theta
// sin(phi_c)), evaluated at phi_c_k and divided by cos(dth), the factor by which the horizontal
// part of the theta unit vector shrinks between the axis and the ring.
__device__ __forceinline__ double polar_btc(const Geo& G, int np, const double* __restrict__ h, int k,
                                            double face) {
    const double pole = (h[0] * G.pcs[k] + h[1] * G.pcs[np + k]) * G.pole_f;
    return 0.5 * (face + pole);
}

// Operator tables of M_alpha for one solve, in the Jacobi-scaled form
// A~ = S M S, S = diag(M)^(-1/2): unit diagonal, off-diagonals -a (a >= 0).
template <typename T>
struct OpTab {
    T* ar;   // [(nr+1)*nt] radial faces (0 at r0 and r1)
    T* at;   // [nr*(nt+1)] theta faces (0 at the poles)
    T* ap;   // [nr*nt]     phi faces
    T* s;    // [nr*nt]     diag^(-1/2)
};

// Geometric factors of the explicit kernels, formed once on the host at grid creation so that no
// explicit kernel divides (FP64 division is a long instruction sequence on this part, and these
// kernels are bound by the FP64 pipe). A row is the np elements of one (i, j).
struct ExTab {
    const double* sh;    // [5*nr] per shell: 1/(rc_i - rc_{i-1}) (at i = 0: 1/(2 (rc_0 - r0))),
                         //        1/(rc_{i+1} - rc_i) (0 at i = nr-1), 1/rc_i, 1/rho_i, 1/(rc_i dth)
    const double* ihp;   // [nr*nt] 1/(rc_i sin(theta_j) dph)
    const double* cot;   // [nt] cot of the theta centres
    const double* jr;    // [4*nr*(nt+1)] radial-edge rows: dual lengths / dual area (3), polar cap factor
    const double* jt;    // [3*(nr+1)*nt] theta-edge rows (ghost radii on r0 and r1)
    const double* jp;    // [3*(nr+1)*(nt+1)] phi-edge rows (0 on the polar rows)
    const double* fr;    // [3*(nr+1)*nt] r-face rows: edge lengths / face area
    const double* ft;    // [3*nr*(nt+1)] theta-face rows (0 on the polar rows)
    const double* fp;    // [3*nr*nt] phi-face rows
};

// The entries of ExTab from the 1-D metric tables, one row at a time; the host builds the grid's
// tables with these and the no-allocation force path builds its own on the device.
struct GeoView {
    const double *r, *rc, *sn, *cn, *sc, *cc, *rho;
    int nr, nt;
    double r0, dth, dph;   // r1 is r[nr]
};
__host__ __device__ inline void ex_shell(const GeoView& g, int i, double* o) {
    const double* rc = g.rc;
    o[0] = (i > 0) ? 1.0 / (rc[i] - rc[i - 1]) : 1.0 / (2.0 * (rc[0] - g.r0));
    o[1] = (i < g.nr - 1) ? 1.0 / (rc[i + 1] - rc[i]) : 0.0;
    o[2] = 1.0 / rc[i];
    o[3] = 1.0 / g.rho[i];
    o[4] = 1.0 / (rc[i] * g.dth);
}
__host__ __device__ inline double ex_ihp(const GeoView& g, int i, int j) {
    return 1.0 / (g.rc[i] * g.sc[j] * g.dph);
}
__host__ __device__ inline double ex_cot(const GeoView& g, int j) { return g.cc[j] / g.sc[j]; }
// radial edge (i, j), j in [0, nt]: interior rows {rc sin_j dph, rc sin_{j-1} dph, rc dth} / dual
// area; polar rows (j = 0, nt): the cap factor in o[3]
__host__ __device__ inline void ex_jr(const GeoView& g, int i, int j, double* o) {
    const double rc = g.rc[i], twopi = 6.283185307179586;
    o[0] = o[1] = o[2] = o[3] = 0.0;
    if (j == 0) {
        o[3] = (rc * g.sc[0] * g.dph) / (rc * rc * (1.0 - g.cc[0]) * twopi);
    } else if (j == g.nt) {
        o[3] = (rc * g.sc[g.nt - 1] * g.dph) / (rc * rc * (1.0 + g.cc[g.nt - 1]) * twopi);
    } else {
        const double area = rc * rc * (g.cc[j - 1] - g.cc[j]) * g.dph;
        o[0] = rc * g.sc[j] * g.dph / area;
        o[1] = rc * g.sc[j - 1] * g.dph / area;
        o[2] = rc * g.dth / area;
    }
}
// radii on either side of the node shell i in [0, nr] (ghost radii mirrored at r0 and r1)
__host__ __device__ inline void ex_rlohi(const GeoView& g, int i, double& rlo, double& rhi) {
    rlo = (i > 0) ? g.rc[i - 1] : 2.0 * g.r0 - g.rc[0];
    rhi = (i < g.nr) ? g.rc[i] : 2.0 * g.r[g.nr] - g.rc[g.nr - 1];
}
// theta edge (i, j), i in [0, nr]
__host__ __device__ inline void ex_jt(const GeoView& g, int i, int j, double* o) {
    double rlo, rhi;
    ex_rlohi(g, i, rlo, rhi);
    const double area = g.sc[j] * 0.5 * (rhi * rhi - rlo * rlo) * g.dph;
    o[0] = rlo * g.sc[j] * g.dph / area;
    o[1] = (rhi - rlo) / area;
    o[2] = rhi * g.sc[j] * g.dph / area;
}
// phi edge (i, j), i in [0, nr], j in [0, nt] (0 on the polar rows)
__host__ __device__ inline void ex_jp(const GeoView& g, int i, int j, double* o) {
    o[0] = o[1] = o[2] = 0.0;
    if (j == 0 || j == g.nt) return;
    double rlo, rhi;
    ex_rlohi(g, i, rlo, rhi);
    const double area = 0.5 * (rhi * rhi - rlo * rlo) * g.dth;
    o[0] = (rhi - rlo) / area;
    o[1] = rhi * g.dth / area;
    o[2] = rlo * g.dth / area;
}
// r face (i, j), i in [0, nr]: {r dth, r sin_{j+1} dph, r sin_j dph} / face area
__host__ __device__ inline void ex_fr(const GeoView& g, int i, int j, double* o) {
    const double ri = g.r[i];
    const double area = ri * ri * (g.cn[j] - g.cn[j + 1]) * g.dph;
    o[0] = ri * g.dth / area;
    o[1] = ri * g.sn[j + 1] * g.dph / area;
    o[2] = ri * g.sn[j] * g.dph / area;
}
// theta face (i, j), j in [0, nt] (0 on the polar rows): {ri sin_j dph, dr, ro sin_j dph} / area
__host__ __device__ inline void ex_ft(const GeoView& g, int i, int j, double* o) {
    o[0] = o[1] = o[2] = 0.0;
    if (j == 0 || j == g.nt) return;
    const double ri = g.r[i], ro = g.r[i + 1];
    const double area = g.sn[j] * 0.5 * (ro * ro - ri * ri) * g.dph;
    o[0] = ri * g.sn[j] * g.dph / area;
    o[1] = (ro - ri) / area;
    o[2] = ro * g.sn[j] * g.dph / area;
}
// phi face (i, j): {dr, ro dth, ri dth} / face area
__host__ __device__ inline void ex_fp(const GeoView& g, int i, int j, double* o) {
    const double ri = g.r[i], ro = g.r[i + 1];
    const double area = 0.5 * (ro * ro - ri * ri) * g.dth;
    o[0] = (ro - ri) / area;
    o[1] = ro * g.dth / area;
    o[2] = ri * g.dth / area;
}

// Unscaled FP64 tables of the same M_alpha (outer residual of mixed precision).
struct OpTab64u {
    double* dg;   // [nr*nt] diagonal
    double* awr;  // [(nr+1)*nt] alpha * wr with the Dirichlet face zeroed (it is in dg)
    double* awt;  // [nr*(nt+1)]
    double* awp;  // [nr*nt]
};

}  // namespace mhd

// The opaque grid object behind mhd_grid_t.
struct mhd_grid_s {
    mhd::Dims d;
    mhd_grid_desc_t desc;
    cudaStream_t stream;
    cudaStream_t side;      // second stream of the FP64 iteration that overlaps the components
    cudaEvent_t side_ev[4]; // its fork / join events (no timing)
    int device;
    int num_sms;
    // host copies of the metric tables
    double max_kt2;
    // device allocations
    void* geo_mem;
    mhd::Geo geo;
    mhd::ExTab ex;
    mhd::OpTab<double> t64;
    mhd::OpTab<float> t32;
    mhd::OpTab64u tu;
    // FP64 PCG workspace (stacked 3-component vectors, 3N each; p64 holds two buffers)
    double *x64, *r64, *p64, *q64;
    // FP32 PCG workspace
    float *x32, *r32, *p32, *q32;
    // step workspace
    double *b0, *b1, *dlt;
    double *er, *et, *ep;   // edge arrays (E or J)
    double *ec;             // cell-centred E (3N)
    double *ring;           // [2*nr] polar ring sums
    int slab_i0;            // slab grids (mhd_grid_create_slab): first global row; slab_nr_global is
    int slab_nr_global;     // the global row count (0 for an ordinary grid)
    double *slab_out;       // [8 + 2*nt] slab calls: reduction results, interface couplings
    double *bharm;          // [8*nr] first-harmonic sums of the rings next to the poles: [0, 4 nr) of
                            // the B_theta faces (north rows, then south; cos and sin per row), [4 nr,
                            // 8 nr) scratch of the adjoint's transpose
    double *sts_tab;        // [8*nr*nt] RKL2 stage coefficients (nu dt / (rho V) times K's weights)
    double* partials;       // [kMaxBlocks * kPartialsPerBlock]
    void* adj_mem;          // adjoint workspace, allocated by the first adjoint call
    void* res_mem;          // implicit-resistivity workspace, allocated by the first such step
    void* pc2_mem;          // PC2 workspace (1 / dt of the phi-line ILU(0)), allocated by the first PC2 solve
    mhd::PcgScalars* sc;    // device
    mhd::StepScalars* ss;   // device
    mhd::PcgScalars* h_sc;  // pinned host mirror
    mhd::StepScalars* h_ss; // pinned host mirror
    double* h_alpha;        // pinned host scalar staging
    // CUDA graphs of a batch of PCG iterations, keyed by kind (FP64, FP32 inner, FP64
    // single-reduction, FP64 PC2, FP32 inner PC2) and ncomp
    cudaGraphExec_t iter_graph[5][4];
    int graph_batch;
    int slab32;             // FP32 CG kernels: r-slab length of the tiled pair (> 0), split kernels (-1),
                            // p update folded into the stencil (-2), recompute pair (-3, -4 with the
                            // r update walking backwards), bulk-staged pair with units of L planes
                            // (-100 - L); 0: not tuned
    int slab64;             // same for the FP64 fused p-update + stencil kernel; -2: the split kernels
                            // with each component's p update overlapping the previous component's stencil
    int pc2_fused32;        // FP32 PC2 iteration: p update folded into the stencil (1) or split (-1); 0: unset
    double visc_lambda_unit; // Gershgorin bound on the spectral radius of D^-1 K (nu = 1)
    std::string last_error;
    // kernel timing (diagnostics)
    int prof;
    static constexpr int kProfSlots = 512;
    cudaEvent_t prof_ev[2 * kProfSlots];
    int prof_kid[kProfSlots];
    int prof_nslot;
    double prof_ms[MHD_KERNEL_COUNT];
    long long prof_cnt[MHD_KERNEL_COUNT];
};

namespace mhd {

// launch helpers
int grid_blocks(const mhd_grid_s* g, long long work, int per_sm = 4);

// CTAs of kThreads threads that one SM holds at once for kernel K (its registers and static
// shared memory permitting), looked up once per kernel. A grid-stride kernel launched with more
// CTAs than fit in one wave, but not a whole number of waves, leaves most SMs idle during the last
// partial wave; launching exactly one resident wave avoids that.
template <auto K>
int resident_per_sm() {
    static const int n = [] {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, kThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            b = 1;
        }
        return b > 0 ? b : 1;
    }();
    return n;
}

// explicit kernels (explicit.cu)
mhd_status_t coeffs(mhd_grid_s* g, const mhd_params_t* p, const double* vr, const double* vt,
                    const double* vp, const double* br, const double* bt, const double* bp);
void current_edges(mhd_grid_s* g, const double* br, const double* bt, const double* bp, bool walls_zero = false,
                   cudaStream_t st = nullptr);
// polar ring sums of a cell-centred array into the grid's ring buffer (north rows, then south)
void ring_sums(mhd_grid_s* g, const double* a, cudaStream_t st);
// first-harmonic sums (cos, sin of the phi centres) of the rows next to the poles of an array of
// np-element rows: out[2 b], out[2 b + 1] for b = i (row off_n + i stride_i) and b = nr + i (row
// off_s + i stride_i), i < nr
void ring_harmonics(mhd_grid_s* g, const double* a, long long stride_i, long long off_n, long long off_s,
                    double* out, cudaStream_t st);
// the B_theta face rings j = 1 and nt - 1 into g->bharm (read by every cell-centred B)
void bt_harmonics(mhd_grid_s* g, const double* bt, cudaStream_t st = nullptr);
// B -= dt curl_h E with E in the grid's edge arrays (dt from the device scalar)
void ct_apply(mhd_grid_s* g, const double* dt_dev, double* br, double* bt, double* bp);
void force(mhd_grid_s* g, const double* vr, const double* vt, const double* vp,
           const double* dlt, double dfac, const double* br, const double* bt, const double* bp,
           const double* dt_dev, double dt_host, const double* b_avg, double* b);
void induction(mhd_grid_s* g, const double* vr, const double* vt, const double* vp,
               const double* dlt, double dfac, double eta, const double* dt_dev, double dt_host,
               double* br, double* bt, double* bp);
void vstar_rhs(mhd_grid_s* g, double* vr, double* vt, double* vp, const double* dlt, double* b);
void diagnostics(mhd_grid_s* g, const double* vr, const double* vt, const double* vp, const double* br,
                 const double* bt, const double* bp, double* out);
int sts_stages(const mhd_grid_s* g, double nu, double dt);
mhd_status_t res_solve(mhd_grid_s* g, const double* dt_dev, double eta, double* br, double* bt, double* bp,
                       const mhd_params_t* p, int* iters, double* relres);
mhd_status_t res_transpose(mhd_grid_s* g, const double* dt_dev, double eta, double* lr, double* lt, double* lp,
                           const mhd_params_t* p);
void res_free(mhd_grid_s* g);
mhd_status_t pc2_factor(mhd_grid_s* g);
void pc2_init64(mhd_grid_s* g, int nc);
void pc2_reliable32(mhd_grid_s* g, int nc, int restart);
void pc2_enqueue_line(mhd_grid_s* g, cudaStream_t st, int nc, bool fp32);
void pc2_free(mhd_grid_s* g);
float* pc2_z32(mhd_grid_s* g);   // z~ of the FP32 PC2 iteration (3N floats, PC2 workspace)
int sts_advance(mhd_grid_s* g, double nu, const double* dt_dev, double dt_host, double* y);

// tiled FP32 CG kernels (tiled.cu)
bool tiled32_ok(const mhd_grid_s* g);
int tiled32_blocks(const mhd_grid_s* g, int slab);
void enqueue_tiled32(mhd_grid_s* g, cudaStream_t st, int nc, int slab, int prof_a, int prof_b);
void enqueue_tiled64_a(mhd_grid_s* g, cudaStream_t st, int slab, int prof_id);

// FP32 CG iteration as a bulk-copy-staged plane-marching pair (bulk.cu); slab: planes per work unit
bool bulk32_ok(const mhd_grid_s* g);
void enqueue_bulk32(mhd_grid_s* g, cudaStream_t st, int nc, int slab);

// PCG (pcg.cu). alpha is read from device memory (alpha_dev) so a step never syncs on it.
void build_tables(mhd_grid_s* g, const double* alpha_dev, bool fp32);
void apply_operator(mhd_grid_s* g, const double* alpha_dev, int nc, const double* p, double* q);
mhd_status_t solve(mhd_grid_s* g, const double* alpha_dev, int nc, const double* b, double* x,
                   const double* x0, const mhd_params_t* prm, int* iters, int* outer,
                   double* relres);

mhd_status_t set_error(mhd_grid_s* g, mhd_status_t st, const std::string& msg);
// allocations ahead of first use (mhd_grid_reserve)
mhd_status_t res_reserve(mhd_grid_s* g);
mhd_status_t pc2_reserve(mhd_grid_s* g);
mhd_status_t adjoint_reserve(mhd_grid_s* g);
mhd_status_t solver_reserve(mhd_grid_s* g, int features);
void batched_forget(mhd_grid_s* g);   // batched.cu: drop cached plans that use g
void adjoint_free(mhd_grid_s* g);     // adjoint.cu: release the adjoint workspace

// kernel timing: bracket a launch with events when profiling is on (returns the slot or -1)
int prof_begin(mhd_grid_s* g, cudaStream_t st, int kernel);
void prof_end(mhd_grid_s* g, cudaStream_t st, int slot);
void prof_flush(mhd_grid_s* g);   // after a stream sync: fold finished slots into the totals

// NVTX ranges on the host timeline of a profiler (a function-pointer test when none is attached):
// one named range per entry point, and `next` closes the current phase and opens the next one
class NvtxRange {
  public:
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
class NvtxPhase {
  public:
    NvtxPhase() = default;
    void next(const char* name) {
        if (open_) nvtxRangePop();
        nvtxRangePushA(name);
        open_ = true;
    }
    ~NvtxPhase() {
        if (open_) nvtxRangePop();
    }
    NvtxPhase(const NvtxPhase&) = delete;
    NvtxPhase& operator=(const NvtxPhase&) = delete;

  private:
    bool open_ = false;
};
mhd_status_t check_cuda(mhd_grid_s* g, const char* where);

}  // namespace mhd
