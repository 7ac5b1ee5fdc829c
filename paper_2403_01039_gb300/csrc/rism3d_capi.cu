// Host layer of the C ABI declared in include/rism3d.h: validation, device workspace layout,
// transform plans, the interpolation table of Eq. 13, and the CUDA-graph iteration loop.
// All arithmetic of the method runs in rism3d_kernels.cuh; this file only prepares inputs
// (unit conversion, table scaling, twiddle factors) and schedules launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rism3d.h"

#include <nvtx3/nvToolsExt.h>
#include "rism3d_internal.h"

using namespace rism;

// NVTX range around each public call, so that a timeline (Nsight Systems, ncu --nvtx)
// shows where the set-up, the iteration and the reductions of a solve begin and end; the
// header-only NVTX costs nothing unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

namespace {

constexpr double kKB = 0.0019872041;      // kcal / (mol K)
constexpr double kCoulomb = 332.0637;     // kcal A / (mol e^2)
constexpr double kPi = 3.14159265358979323846;
constexpr size_t kMaxSmem = 227 * 1024;
constexpr size_t kPencilSmemTarget = 64 * 1024;
constexpr size_t kSlabSmemTarget = 72 * 1024;   // row-chunk size when a plane does not fit
constexpr int kMaxLaunches = 12;                  // launches of one iteration at most
constexpr int kEventsPerIter = 2 * kMaxLaunches;  // an event pair around each

thread_local std::string g_create_error;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Factor L into radices 8/4/2 (powers of two, largest first, without a trailing 2 when a
// 4 can absorb it) and 3/5. Returns false if L has another prime factor.
bool make_plan(int L, FftPlan &p) {
    p.L = L;
    p.nst = 0;
    int n = L, twos = 0;
    while (n % 2 == 0) {
        n /= 2;
        ++twos;
    }
    std::vector<int> r;
    while (n % 3 == 0) {
        n /= 3;
        r.push_back(3);
    }
    while (n % 5 == 0) {
        n /= 5;
        r.push_back(5);
    }
    if (n != 1 || L < 1) return false;
    int eights = twos / 3, rem = twos % 3;
    std::vector<int> t;
    if (rem == 1 && eights > 0) {
        --eights;
        t.push_back(4);
        t.push_back(4);
    } else if (rem == 1) {
        t.push_back(2);
    } else if (rem == 2) {
        t.push_back(4);
    }
    for (int i = 0; i < eights; ++i) t.insert(t.begin(), 8);
    for (int v : r) t.push_back(v);
    if ((int)t.size() > kMaxRadixStages) return false;
    int ns = 1;
    for (size_t i = 0; i < t.size(); ++i) {
        p.radix[i] = t[i];
        p.dlr[i] = make_fastdiv(L / t[i]);
        p.dns[i] = make_fastdiv(ns);
        ns *= t[i];
    }
    p.nst = (int)t.size();
    return true;
}

// Sequences one warp can transform together while each lane holds at most maxc values in
// every stage (0 when a single sequence does not fit: the block-wide path is used).
int warp_seqs(const FftPlan &p, int maxc) {
    int cap = 1 << 30;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s];
        const int c = 32 * (maxc / R) * R;          // values one warp holds in this stage
        cap = c < cap ? c : cap;
    }
    return cap / p.L;
}

// Largest batch chunk for which every stage keeps at most MAXC / R butterflies per thread.
int fft_chunk(const FftPlan &p, int nthreads, int maxc) {
    int chunk = 1 << 30;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s];
        const int per = maxc / R;                  // butterflies a thread can hold
        const int lr = p.L / R;                    // butterflies per sequence
        const int c = (int)((long long)nthreads * per / lr);
        chunk = c < chunk ? c : chunk;
    }
    return chunk;
}

}  // namespace

namespace {
// element-kernel blocks per site for one half of the planes (as launch_split uses)
int split_elem_blocks_host(int nv) { return (kSplitBlocks + nv - 1) / nv; }
}  // namespace

struct rism3d_ctx {
    int device = 0;
    int precision = 32;
    rism3d_options opt{};
    int nv = 0, Nx = 0, Ny = 0, Nz = 0, Kz = 0;
    long long G = 0;
    double spacing[3] = {0, 0, 0}, origin[3] = {0, 0, 0};
    std::vector<double> q, sig, eps, rho;
    double temperature = 0, beta = 0, dV = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *ws = nullptr;
    bool own_ws = false;
    size_t ws_bytes = 0;
    // device pointers inside the workspace
    Ctrl *ctrl = nullptr;
    double *atoms = nullptr, *site_sig = nullptr, *site_eps = nullptr, *site_q = nullptr;
    double *site_rho_dV = nullptr;
    int n_atoms = 0;
    double *sfe_part = nullptr, *staging = nullptr;
    Fields<float> f32{};
    Fields<double> f64{};
    Ctrl *ctrl_host = nullptr;                 // pinned
    cudaGraphExec_t graph = nullptr;
    bool has_solute = false;
    bool offset_live = false;                  // the iterate may have a nonzero offset tau0
    int cur_slot = 0;
    int last_kind = kKH, last_order = 1;
    std::vector<double> atom_host;
    std::string err;
    rism3d_stats stats{};
    std::vector<cudaEvent_t> ev;               // [check_every][5] around the iteration kernels
    cudaEvent_t ev_aux[2] = {nullptr, nullptr};
    cudaEvent_t chunk_ev = nullptr;            // end of the last launched iteration chunk
    cudaStream_t side = nullptr;               // second branch of the split plane passes
    cudaEvent_t fork[4] = {nullptr, nullptr, nullptr, nullptr};
    // state of the solve in progress (rism3d_solve and the batch scheduler)
    int run_iter_before = 0, run_closure = kKH, run_order = 1;
    std::chrono::steady_clock::time_point run_t0;
    double *lr_buf = nullptr;                  // finite-size correction: FP64 partial sums (lazy)

    bool fp32() const { return precision == 32; }
};

namespace rism {
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace rism

static rism3d_status fail(rism3d_ctx *ctx, rism3d_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_error = buf;
    return st;
}

#define CUDA_TRY(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail((ctx), RISM3D_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                                     \
    } while (0)

// ------------------------------------------------------------------ layout
namespace {

struct Layout {
    size_t ctrl, bu, phi, w, wref, psi, spec, X, R, T, tau0, anchor, phase, table, tw, partials, sfe, atoms,
        sites, staging, total;
};

struct Geometry {
    int nv, Nx, Ny, Nz, Kz, M, nk, max_atoms, s;   // s = bytes per real
    long long G;
    FftPlan px, py, ph;
    int pitch, W, pencil_pitch, chunk_rows, chunk_cols, chunk_x;
    int slab_rows, nyc, Wy, ypitch, chunk_y;
    int cl, chunk_ys;                           // cluster y transform (0: y-pencil pass)
    FftPlan pys;
    size_t plane_smem, pencil_smem, ypencil_smem;
};

Layout make_layout(const Geometry &g) {
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t c = 2 * (size_t)g.s;
    const size_t specN = (size_t)g.Nx * g.Ny * g.Kz + (size_t)g.Nx * g.Ny;
    L.ctrl = take(sizeof(Ctrl));
    L.bu = take((size_t)g.nv * g.G * g.s);
    L.phi = take((size_t)g.G * g.s);
    L.w = take((size_t)g.nv * g.G * g.s);
    L.wref = take((size_t)g.nv * g.G * g.s);
    L.psi = take(specN * c);
    L.spec = take((size_t)g.nv * specN * c);
    L.X = take((size_t)g.M * g.nv * g.G * g.s);
    L.R = take((size_t)g.M * g.nv * g.G * g.s);
    L.T = take((size_t)g.nv * g.G * g.s);
    L.tau0 = take((size_t)g.nv * g.G * g.s);
    L.anchor = take((size_t)2 * g.nv * g.G * g.s);
    L.phase = take((size_t)kPhaseChunk * (g.Nx + g.Ny + g.Kz + 1) * c);
    L.table = take((size_t)g.nk * (g.nv + 1) * g.nv * g.s);
    L.tw = take((size_t)(g.Nx + g.Ny + g.Kz + g.Kz + 1 + g.Kz + g.Ny + g.Nx) * c);
    L.partials = take((size_t)std::max(g.nv * g.Nx * g.nyc, kSplitPartials) * (kMaxHist + 1) * sizeof(double));
    L.sfe = take((size_t)g.nv * kSfeBlocksPerSite * sizeof(double));
    L.atoms = take((size_t)g.max_atoms * kAtomStride * sizeof(double));
    L.sites = take((size_t)4 * kMaxSites * sizeof(double));
    L.staging = take((size_t)g.nv * g.G * sizeof(double));
    L.total = o;
    return L;
}

rism3d_status check_inputs(const rism3d_solvent *sv, const rism3d_grid *gr, const rism3d_options *op,
                           Geometry &g) {
    if (!sv || !gr || !op) return fail(nullptr, RISM3D_EINVAL, "null solvent, grid or options");
    if (sv->n_sites < 1 || sv->n_sites > kMaxSites)
        return fail(nullptr, RISM3D_EINVAL, "n_sites must be in 1..%d", kMaxSites);
    if (!sv->q || !sv->sigma || !sv->eps || !sv->rho || !sv->chi)
        return fail(nullptr, RISM3D_EINVAL, "null solvent array");
    for (int i = 0; i < sv->n_sites; ++i)
        if (!(sv->rho[i] > 0.0) || !std::isfinite(sv->rho[i]))
            return fail(nullptr, RISM3D_EINVAL, "rho[%d] must be positive", i);
    if (!(sv->temperature > 0.0)) return fail(nullptr, RISM3D_EINVAL, "temperature must be positive");
    if (sv->n_k < 2 || !(sv->dk > 0.0)) return fail(nullptr, RISM3D_EINVAL, "need n_k >= 2 and dk > 0");
    for (int d = 0; d < 3; ++d) {
        if (gr->n[d] < 2) return fail(nullptr, RISM3D_EINVAL, "grid n[%d] must be >= 2", d);
        if (!(gr->spacing[d] > 0.0)) return fail(nullptr, RISM3D_EINVAL, "spacing[%d] must be > 0", d);
    }
    if (gr->n[2] % 2) return fail(nullptr, RISM3D_EUNSUPPORTED, "Nz must be even");
    if (op->precision != 32 && op->precision != 64)
        return fail(nullptr, RISM3D_EINVAL, "precision must be 32 or 64");
    if (op->mdiis_nvec < 1 || op->mdiis_nvec > kMaxHist)
        return fail(nullptr, RISM3D_EINVAL, "mdiis_nvec must be in 1..%d", kMaxHist);
    if (!(op->mdiis_damp > 0.0 && op->mdiis_damp <= 2.0))
        return fail(nullptr, RISM3D_EINVAL, "mdiis_damp must be in (0, 2]");
    if (op->slab_rows < 0) return fail(nullptr, RISM3D_EINVAL, "slab_rows must be >= 0");
    if (op->kgrid != 0 && op->kgrid != 1) return fail(nullptr, RISM3D_EINVAL, "kgrid must be 0 or 1");
    if (op->ypencil_pass != 0 && op->ypencil_pass != 1)
        return fail(nullptr, RISM3D_EINVAL, "ypencil_pass must be 0 or 1");
    if (!(op->anchor_ratio >= 0.0 && op->anchor_ratio < 1.0))
        return fail(nullptr, RISM3D_EINVAL, "anchor_ratio must be in [0, 1) (0: the default 0.1)");
    if (op->split_passes != 0 && op->split_passes != 1) return fail(nullptr, RISM3D_EINVAL, "split_passes must be 0 or 1");
    if (op->timing < 0 || op->timing > 2) return fail(nullptr, RISM3D_EINVAL, "timing must be 0, 1 or 2");
    if (op->accelerator != 0 && op->accelerator != 1)
        return fail(nullptr, RISM3D_EINVAL, "accelerator must be 0 (MDIIS) or 1 (modified Anderson)");
    if (op->max_iter < 1 || op->check_every < 1 || op->max_atoms < 1)
        return fail(nullptr, RISM3D_EINVAL, "max_iter, check_every and max_atoms must be >= 1");
    g.nv = sv->n_sites;
    g.Nx = gr->n[0];
    g.Ny = gr->n[1];
    g.Nz = gr->n[2];
    g.Kz = g.Nz / 2;
    g.G = (long long)g.Nx * g.Ny * g.Nz;
    g.M = op->accelerator == 1 ? 3 : op->mdiis_nvec;   // Anderson keeps the last three pairs
    g.nk = sv->n_k;
    g.max_atoms = op->max_atoms;
    g.s = op->precision == 32 ? 4 : 8;
    if (!make_plan(g.Nx, g.px) || !make_plan(g.Ny, g.py) || !make_plan(g.Kz, g.ph))
        return fail(nullptr, RISM3D_EUNSUPPORTED, "Nx, Ny and Nz/2 must factor into 2, 3 and 5");
    const int maxc = 8;                         // complex values a thread holds per FFT stage
    const size_t c = 2 * (size_t)g.s;
    g.pitch = g.Kz + 1;
    if (g.pitch % 2 == 0) g.pitch += 1;        // odd pitch: column access without bank conflicts
    auto plane_bytes = [&](int rows) {   // rows, then twiddles (h, y, z, q), then reduction
        return c * ((size_t)rows * g.pitch + g.Kz + g.Ny + g.Kz + 1 + g.Kz) +
               (kMaxHist + 1) * (kThreadsPlane / 32) * sizeof(double) + 16;
    };
    // whole y-z planes when they fit in shared memory, else row chunks + a y-pencil pass
    g.slab_rows = g.Ny;
    if (op->slab_rows > 0) {
        g.slab_rows = op->slab_rows < g.Ny ? op->slab_rows : g.Ny;
    } else if (plane_bytes(g.Ny) > kMaxSmem) {
        int r = 1;
        while (2 * r <= g.Ny && plane_bytes(2 * r) <= kSlabSmemTarget) r *= 2;
        g.slab_rows = r;
    }
    g.nyc = (g.Ny + g.slab_rows - 1) / g.slab_rows;
    g.plane_smem = plane_bytes(g.slab_rows);
    // row chunks that split the plane evenly into 2, 4 or 8 form a cluster that does the y
    // transform (its local part needs a plan of the chunk length and S twiddles more)
    g.cl = 0;
    if (g.nyc > 1 && !op->ypencil_pass && op->kgrid == 0 && (g.nyc == 2 || g.nyc == 4 || g.nyc == 8) &&
        g.Ny == g.nyc * g.slab_rows && make_plan(g.slab_rows, g.pys) &&
        g.plane_smem + c * g.slab_rows <= kMaxSmem) {
        g.cl = g.nyc;
        g.plane_smem += c * g.slab_rows;
    }
    if (g.plane_smem > kMaxSmem)
        return fail(nullptr, RISM3D_EUNSUPPORTED,
                    "a row chunk of %d rows x %d needs %zu bytes of shared memory (limit %zu)", g.slab_rows,
                    g.Kz + 1, g.plane_smem, kMaxSmem);
    g.ypitch = g.Ny + 1;
    g.Wy = 1;
    for (int w = 16; w >= 1; w /= 2)
        if (c * ((size_t)g.nv * w * g.ypitch + g.Ny) <= kPencilSmemTarget || w == 1) {
            g.Wy = w;
            break;
        }
    g.ypencil_smem = c * ((size_t)g.nv * g.Wy * g.ypitch + g.Ny);
    if (g.nyc > 1 && g.ypencil_smem > kMaxSmem)
        return fail(nullptr, RISM3D_EUNSUPPORTED, "y pencils of %d points do not fit in shared memory", g.Ny);
    g.pencil_pitch = g.Nx + 1;
    g.W = 1;
    for (int w = 16; w >= 1; w /= 2) {
        size_t b = c * ((size_t)g.nv * w * g.pencil_pitch + g.Nx);
        if (b <= kPencilSmemTarget || w == 1) {
            g.W = w;
            break;
        }
    }
    g.pencil_smem = c * ((size_t)g.nv * g.W * g.pencil_pitch + g.Nx);
    if (g.pencil_smem > kMaxSmem)
        return fail(nullptr, RISM3D_EUNSUPPORTED, "x pencils of %d points do not fit in shared memory",
                    g.Nx);
    g.px.seq_per_warp = warp_seqs(g.px, maxc);
    g.py.seq_per_warp = warp_seqs(g.py, maxc);
    g.ph.seq_per_warp = warp_seqs(g.ph, maxc);
    g.chunk_rows = fft_chunk(g.ph, kThreadsPlane, maxc);
    g.chunk_ys = 1;
    if (g.cl) {
        g.pys.seq_per_warp = warp_seqs(g.pys, maxc);
        g.chunk_ys = fft_chunk(g.pys, kThreadsPlane, maxc);
    }
    g.chunk_cols = fft_chunk(g.py, kThreadsPlane, maxc);
    g.chunk_x = fft_chunk(g.px, kThreadsPencil, maxc);
    g.chunk_y = fft_chunk(g.py, kThreadsPencil, maxc);
    if (g.chunk_rows < 1 || g.chunk_cols < 1 || g.chunk_x < 1 || g.chunk_y < 1)
        return fail(nullptr, RISM3D_EUNSUPPORTED, "transform length too long for one block");
    return RISM3D_OK;
}

template <typename T>
void fill_fields(rism3d_ctx *ctx, const Geometry &g, const Layout &L, Fields<T> &f) {
    typedef typename Cx<T>::type C;
    char *b = static_cast<char *>(ctx->ws);
    f.nv = g.nv;
    f.Nx = g.Nx;
    f.Ny = g.Ny;
    f.Nz = g.Nz;
    f.Kz = g.Kz;
    f.M = g.M;
    f.G = g.G;
    f.specN = (long long)g.Nx * g.Ny * g.Kz;
    f.bu = reinterpret_cast<T *>(b + L.bu);
    f.phi = reinterpret_cast<T *>(b + L.phi);
    f.w = reinterpret_cast<T *>(b + L.w);
    f.wref = reinterpret_cast<T *>(b + L.wref);
    f.psi = reinterpret_cast<C *>(b + L.psi);
    f.psi_nyq = f.psi + f.specN;
    f.spec = reinterpret_cast<C *>(b + L.spec);
    f.spec_nyq = f.spec + (long long)g.nv * f.specN;
    f.X = reinterpret_cast<T *>(b + L.X);
    f.R = reinterpret_cast<T *>(b + L.R);
    f.Tc = reinterpret_cast<T *>(b + L.T);
    f.tau0 = reinterpret_cast<T *>(b + L.tau0);
    f.g_a = reinterpret_cast<T *>(b + L.anchor);
    f.h_a = f.g_a + (long long)g.nv * g.G;
    f.phase = reinterpret_cast<C *>(b + L.phase);
    f.table = reinterpret_cast<T *>(b + L.table);
    f.nk = g.nk;
    C *tw = reinterpret_cast<C *>(b + L.tw);
    f.tw_x = tw;
    f.tw_y = f.tw_x + g.Nx;
    f.tw_h = f.tw_y + g.Ny;
    f.tw_z = f.tw_h + g.Kz;
    f.tw_q = f.tw_z + g.Kz + 1;
    f.tw_ys = f.tw_q + g.Kz;
    f.tw_xs = f.tw_ys + g.Ny;
    f.half = ctx->opt.kgrid == 1;
    f.split = ctx->opt.split_passes != 0;
    f.px = g.px;
    f.py = g.py;
    f.ph = g.ph;
    f.chunk_rows = g.chunk_rows;
    f.chunk_cols_fwd = g.chunk_cols;
    f.chunk_x = g.chunk_x;
    f.pitch = g.pitch;
    f.slab_rows = g.slab_rows;
    f.nyc = g.nyc;
    f.cl = g.cl;
    f.pys = g.pys;
    f.chunk_ys = g.chunk_ys;
    f.dK1 = make_fastdiv(g.Kz + 1);
    f.Wy = g.Wy;
    f.ypitch = g.ypitch;
    f.ytiles_main = g.Nx * ((g.Kz + g.Wy - 1) / g.Wy);
    f.ytiles_nyq = f.half ? 0 : (g.Nx + g.Wy - 1) / g.Wy;   // the half grid has no Nyquist plane
    f.chunk_y = g.chunk_y;
    f.W = g.W;
    f.pencil_pitch = g.pencil_pitch;
    f.tiles_main = g.Ny * ((g.Kz + g.W - 1) / g.W);
    f.tiles_nyq = f.half ? 0 : (g.Ny + g.W - 1) / g.W;
    f.dKz = make_fastdiv(g.Kz);
    f.dKz1h = make_fastdiv(g.Kz / 2 + 1);
    f.dKzp = make_fastdiv((g.Kz + 1) / 2);
    f.dW = make_fastdiv(g.W);
    f.dNx = make_fastdiv(g.Nx);
    f.dWy = make_fastdiv(g.Wy > 0 ? g.Wy : 1);
    f.dNy = make_fastdiv(g.Ny);
    for (int i = 0; i < kMaxSites; ++i) f.bq[i] = i < g.nv ? ctx->beta * ctx->q[i] : 0.0;
    for (int d = 0; d < 3; ++d) {
        const int N = d == 0 ? g.Nx : (d == 1 ? g.Ny : g.Nz);
        f.ks[d] = 2.0 * kPi / (N * ctx->spacing[d]);
    }
    f.partials = reinterpret_cast<double *>(b + L.partials);
    f.ctrl = reinterpret_cast<Ctrl *>(b + L.ctrl);
    f.nparts = split_planes(f) ? 2 * split_elem_blocks_host(g.nv) * g.nv : g.nv * g.Nx * g.nyc;
}

// Interpolation table of Eq. 13 scaled for the unnormalised inverse transform:
// A[j][a][g] = X_ag(k_j) / (Nx Ny Nz) for a < n_v, and the charge row
// A[j][n_v][g] = -sum_a q_a X_ag(k_j) / (Nx Ny Nz), which multiplies beta Phi~ / dV.
template <typename T>
std::vector<T> make_table(const rism3d_solvent *sv, long long G) {
    const int nv = sv->n_sites, nk = sv->n_k;
    std::vector<T> A((size_t)nk * (nv + 1) * nv);
    const double inv = 1.0 / (double)G;
    for (int j = 0; j < nk; ++j) {
        for (int g = 0; g < nv; ++g) {
            double Q = 0.0;
            for (int a = 0; a < nv; ++a) {
                const double x = sv->chi[((size_t)a * nv + g) * nk + j];
                A[((size_t)j * (nv + 1) + a) * nv + g] = (T)(x * inv);
                Q += sv->q[a] * x;
            }
            A[((size_t)j * (nv + 1) + nv) * nv + g] = (T)(-Q * inv);
        }
    }
    return A;
}

// exp(-2 pi i m / L), m < L, from the host libm in FP64, rounded to the working precision.
template <typename T>
void push_twiddles(std::vector<typename Cx<T>::type> &v, int L, int count) {
    typedef typename Cx<T>::type C;
    for (int m = 0; m < count; ++m) {
        const double a = -2.0 * kPi * (double)m / (double)L;
        C c;
        c.x = (T)std::cos(a);
        c.y = (T)std::sin(a);
        v.push_back(c);
    }
}

template <typename T>
rism3d_status upload_tables(rism3d_ctx *ctx, const rism3d_solvent *sv, const Layout &L, Fields<T> &f) {
    typedef typename Cx<T>::type C;
    std::vector<T> A = make_table<T>(sv, ctx->G);
    char *b = static_cast<char *>(ctx->ws);
    CUDA_TRY(ctx, cudaMemcpy(b + L.table, A.data(), A.size() * sizeof(T), cudaMemcpyHostToDevice));
    std::vector<C> tw;
    push_twiddles<T>(tw, ctx->Nx, ctx->Nx);
    push_twiddles<T>(tw, ctx->Ny, ctx->Ny);
    push_twiddles<T>(tw, ctx->Kz, ctx->Kz);
    push_twiddles<T>(tw, ctx->Nz, ctx->Kz + 1);
    // half grid: exp(-i pi (2m + 1) / Nz) and the per-axis shifts exp(-i pi n / N)
    auto push_angle = [&](double a) {
        C c;
        c.x = (T)std::cos(a);
        c.y = (T)std::sin(a);
        tw.push_back(c);
    };
    for (int m = 0; m < ctx->Kz; ++m) push_angle(-kPi * (2.0 * m + 1.0) / ctx->Nz);
    for (int m = 0; m < ctx->Ny; ++m) push_angle(-kPi * (double)m / ctx->Ny);
    for (int m = 0; m < ctx->Nx; ++m) push_angle(-kPi * (double)m / ctx->Nx);
    CUDA_TRY(ctx, cudaMemcpy(b + L.tw, tw.data(), tw.size() * sizeof(C), cudaMemcpyHostToDevice));
    f.inv_dk = 1.0 / sv->dk;
    CUDA_TRY(ctx, prepare_kernels<T>(f));
    return RISM3D_OK;
}

void closure_stages(int kind, int order, double tol, Ctrl &c) {
    const double stage_tol = tol > 1e-4 ? tol : 1e-4;
    int n = 0;
    if (kind == kKH) {
        c.stage_kind[n] = kKH, c.stage_order[n++] = 1;
    } else if (kind == kHNC) {
        c.stage_kind[n] = kKH, c.stage_order[n++] = 1;
        c.stage_kind[n] = kHNC, c.stage_order[n++] = 0;
    } else {
        c.stage_kind[n] = kKH, c.stage_order[n++] = 1;
        for (int o = 2; o <= order && n < kMaxClosureStages; ++o) c.stage_kind[n] = kPSE, c.stage_order[n++] = o;
    }
    c.n_stages = n;
    for (int i = 0; i < n; ++i) c.stage_tol[i] = (i == n - 1) ? tol : stage_tol;
}

// One iteration as a list of launches. Fused form: plane_fwd (stats slot 0), [y pencils
// forward (8)], pencil (1), [y pencils inverse (9)], plane_inv (2), mdiis (3), all on the
// context's stream. Split form (FP32 whole planes, split_planes): the element and
// transform kernels of the two halves of the x planes on two branches,
//   main: fwd_elem(A) -> fft_fwd(A) -> [wait B] fft_fwd(B) -> pencil -> fft_inv(A) ->
//         fft_inv(B) -> inv_elem(B) -> [wait] mdiis
//   side: [after fwd_elem(A)] fwd_elem(B);   [after fft_inv(A)] inv_elem(A)
// so that each element kernel runs beside a transform kernel (slots 10-13 for fwd_elem,
// fft_fwd, fft_inv, inv_elem). tev (timing) receives an event pair around every launch
// on its stream and tslot the launch's stats slot; returns the number of launches.
struct Launch {
    int slot, which, stream, half;
};

int iteration_plan(const rism3d_ctx *ctx, bool with_mdiis, Launch *L) {
    const bool fp32 = ctx->fp32();
    const bool split = fp32 ? split_planes(ctx->f32) : false;
    const bool ysplit = fp32 ? (ctx->f32.nyc > 1 && ctx->f32.cl == 0) : (ctx->f64.nyc > 1 && ctx->f64.cl == 0);
    int n = 0;
    if (split) {
        L[n++] = {10, 0, 0, 0};
        L[n++] = {10, 0, 1, 1};
        L[n++] = {11, 1, 0, 0};
        L[n++] = {11, 1, 0, 1};
        L[n++] = {1, -1, 0, 0};
        L[n++] = {12, 2, 0, 0};
        L[n++] = {13, 3, 1, 0};
        L[n++] = {12, 2, 0, 1};
        L[n++] = {13, 3, 0, 1};
    } else {
        L[n++] = {0, -1, 0, 0};
        if (ysplit) L[n++] = {8, -1, 0, 0};
        L[n++] = {1, -1, 0, 0};
        if (ysplit) L[n++] = {9, -1, 0, 0};
        L[n++] = {2, -1, 0, 0};
    }
    if (with_mdiis) L[n++] = {3, -1, 0, 0};
    return n;
}

// launches per iteration and kernel slot (both halves of a split pass count)
int iteration_slots(const rism3d_ctx *ctx, bool with_mdiis, int *slots) {
    Launch L[kMaxLaunches];
    const int n = iteration_plan(ctx, with_mdiis, L);
    for (int i = 0; i < n; ++i) slots[i] = L[i].slot;
    return n;
}

template <typename T>
rism3d_status launch_one(rism3d_ctx *ctx, const Fields<T> &f, const Launch &l, cudaStream_t s) {
    const int half_x = f.Nx / 2;
    const int x0 = l.half ? half_x : 0, x1 = l.half ? f.Nx : half_x;
    switch (l.slot) {
        case 0: CUDA_TRY(ctx, launch_plane_fwd<T>(f, s)); break;
        case 8: CUDA_TRY(ctx, launch_ypencil<T>(f, -1, s)); break;
        case 1: CUDA_TRY(ctx, launch_pencil<T>(f, s)); break;
        case 9: CUDA_TRY(ctx, launch_ypencil<T>(f, +1, s)); break;
        case 2: CUDA_TRY(ctx, launch_plane_inv<T>(f, s)); break;
        case 3: CUDA_TRY(ctx, launch_mdiis<T>(f, s)); break;
        default: CUDA_TRY(ctx, launch_split<T>(f, l.which, x0, x1, l.half ? f.nparts / 2 : 0, s)); break;
    }
    return RISM3D_OK;
}

template <typename T>
rism3d_status run_iteration(rism3d_ctx *ctx, const Fields<T> &f, bool with_mdiis, cudaEvent_t *tev) {
    Launch L[kMaxLaunches];
    const int n = iteration_plan(ctx, with_mdiis, L);
    const unsigned ext = cudaEventRecordExternal;
    cudaStream_t st[2] = {ctx->stream, ctx->side};
    const bool split = n > 0 && L[0].slot == 10;
    if (split && (!ctx->side || !ctx->fork[0])) return fail(ctx, RISM3D_ESTATE, "split passes without side stream");
    for (int i = 0; i < n; ++i) {
        const Launch &l = L[i];
        if (split) {                                      // fork / join points of the plan
            if (i == 1 || i == 6) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->side, ctx->fork[i == 1 ? 0 : 2], 0));
            if (i == 3) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->fork[1], 0));
        }
        cudaStream_t s = st[l.stream];
        if (tev) CUDA_TRY(ctx, cudaEventRecordWithFlags(tev[2 * i], s, ext));
        rism3d_status r = launch_one<T>(ctx, f, l, s);
        if (r != RISM3D_OK) return r;
        if (tev) CUDA_TRY(ctx, cudaEventRecordWithFlags(tev[2 * i + 1], s, ext));
        if (split) {
            if (i == 0) CUDA_TRY(ctx, cudaEventRecord(ctx->fork[0], ctx->stream));   // fwd_elem(A) done
            if (i == 1) CUDA_TRY(ctx, cudaEventRecord(ctx->fork[1], ctx->side));     // fwd_elem(B) done
            if (i == 5) CUDA_TRY(ctx, cudaEventRecord(ctx->fork[2], ctx->stream));   // fft_inv(A) done
            if (i == 6) CUDA_TRY(ctx, cudaEventRecord(ctx->fork[3], ctx->side));     // inv_elem(A) done
            if (i == 8) CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->fork[3], 0));   // join
        }
    }
    return RISM3D_OK;
}

// The split plane passes' second stream and fork/join events (created once).
rism3d_status ensure_side(rism3d_ctx *ctx) {
    if (!(ctx->fp32() && split_planes(ctx->f32)) || ctx->side) return RISM3D_OK;
    CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    for (auto &e : ctx->fork) CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return RISM3D_OK;
}

rism3d_status iteration(rism3d_ctx *ctx, bool with_mdiis) {
    if (rism3d_status st = ensure_side(ctx)) return st;
    return ctx->fp32() ? run_iteration<float>(ctx, ctx->f32, with_mdiis, nullptr)
                       : run_iteration<double>(ctx, ctx->f64, with_mdiis, nullptr);
}

// Algorithmic HBM bytes of the iterations that ran (from the device counters): per
// site-point (P = n_v Nx Ny Nz of them, s bytes per real, z = (Kz + 1) / Kz for the half
// spectrum) plane_fwd moves the history it combines (Y_i per stored pair, R_i as well
// under dynamic damping, + 1 for the new tau, or 1 to load tau), w (1), the spectrum it
// writes (z) and the anchor g_a (1 read, 1 write on refresh; a refresh also reads and
// writes tau0, writes w and rewrites each stored Y it combines); pencil reads and writes the spectrum (2 z) plus Psi (z/n_v) until the first
// anchor; plane_inv reads the spectrum (z), tau and w (2), the history residuals, the
// anchor h_a, and writes R and Y (2) and h_a on refresh.
void account_iterations(rism3d_ctx *ctx, const Ctrl &c) {
    const double P = (double)ctx->nv * (double)ctx->G;
    const double s = ctx->fp32() ? 4.0 : 8.0;
    const double z = ctx->opt.kgrid == 1 ? 1.0 : (double)(ctx->Kz + 1) / (double)ctx->Kz;   // half spectrum per real
    const double it = (double)c.acc_iters;
    ctx->stats.iterations += c.acc_iters;
    ctx->stats.bytes[1] += P * s * z * (2.0 * it + (double)c.acc_psi / ctx->nv);
    if (ctx->fp32() && split_planes(ctx->f32)) {
        // split passes: the element kernels also write / read the transform input / output
        ctx->stats.bytes[10] += P * s * ((double)c.acc_fwd_units + (double)c.acc_upd_r + 2.0 * it +
                                         (double)c.acc_anchor + 4.0 * (double)c.acc_refresh +
                                         2.0 * (double)c.acc_shift);
        ctx->stats.bytes[11] += P * s * it * (1.0 + z);
        ctx->stats.bytes[12] += P * s * it * (z + 1.0);
        ctx->stats.bytes[13] += P * s * (it * 5.0 + (double)c.acc_hist + (double)c.acc_anchor +
                                         (double)c.acc_refresh);
    } else {
        ctx->stats.bytes[0] += P * s * ((double)c.acc_fwd_units + (double)c.acc_upd_r + it * (1.0 + z) +
                                        (double)c.acc_anchor + 4.0 * (double)c.acc_refresh +
                                        2.0 * (double)c.acc_shift);
        ctx->stats.bytes[2] += P * s * (it * (z + 4.0) + (double)c.acc_hist + (double)c.acc_anchor +
                                        (double)c.acc_refresh);
    }
    const int nyc = ctx->fp32() ? ctx->f32.nyc : ctx->f64.nyc;
    ctx->stats.bytes[3] += 8.0 * ctx->nv * ctx->Nx * nyc * (it + (double)c.acc_hist);
    const int cl = ctx->fp32() ? ctx->f32.cl : ctx->f64.cl;
    if (nyc > 1 && cl == 0) {         // y pencils read and write the spectrum
        ctx->stats.bytes[8] += P * s * z * 2.0 * it;
        ctx->stats.bytes[9] += P * s * z * 2.0 * it;
    }
}

// Event pair around a direct (non-graph) launch of kernel k, when timing is on.
struct AuxTimer {
    rism3d_ctx *ctx;
    int k;
    bool on;
    AuxTimer(rism3d_ctx *c, int kernel) : ctx(c), k(kernel), on(c->opt.timing != 0) {
        if (on) cudaEventRecord(ctx->ev_aux[0], ctx->stream);
    }
    void stop(double bytes) {
        ctx->stats.launches[k] += 1;
        ctx->stats.bytes[k] += bytes;
        if (!on) return;
        cudaEventRecord(ctx->ev_aux[1], ctx->stream);
        cudaEventSynchronize(ctx->ev_aux[1]);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev_aux[0], ctx->ev_aux[1]) == cudaSuccess) {
            ctx->stats.ms[k] += ms;
            ctx->stats.timed[k] += 1;
        }
    }
};

rism3d_status build_graph(rism3d_ctx *ctx) {
    if (ctx->graph) return RISM3D_OK;
    cudaGraph_t g = nullptr;
    const int K = ctx->opt.check_every;
    if (ctx->opt.timing && ctx->ev.empty()) {
        ctx->ev.assign((size_t)K * kEventsPerIter, nullptr);
        for (auto &e : ctx->ev) CUDA_TRY(ctx, cudaEventCreate(&e));
    }
    if (rism3d_status st0 = ensure_side(ctx)) return st0;
    CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    rism3d_status st = RISM3D_OK;
    for (int i = 0; i < K && st == RISM3D_OK; ++i) {
        // timing 1: every iteration of the graph; 2: its first iteration only
        const bool timed = ctx->opt.timing == 1 || (ctx->opt.timing == 2 && i == 0);
        cudaEvent_t *tev = timed ? &ctx->ev[(size_t)i * kEventsPerIter] : nullptr;
        st = ctx->fp32() ? run_iteration<float>(ctx, ctx->f32, true, tev)
                         : run_iteration<double>(ctx, ctx->f64, true, tev);
    }
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (st != RISM3D_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(ctx, RISM3D_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->graph = nullptr;
        return fail(ctx, RISM3D_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return RISM3D_OK;
}

void reset_ctrl(rism3d_ctx *ctx, Ctrl &c) {
    std::memset(&c, 0, sizeof(Ctrl));
    c.status = kRunning;
    c.max_iter = ctx->opt.max_iter;
    c.M = ctx->opt.accelerator == 1 ? 3 : ctx->opt.mdiis_nvec;
    c.accel = ctx->opt.accelerator;
    c.s1 = ctx->opt.anderson_s1;
    c.s2 = ctx->opt.anderson_s2;
    c.dynamic = ctx->opt.dynamic_damp ? 1 : 0;
    c.damp = ctx->opt.mdiis_damp;
    c.eta = ctx->opt.mdiis_damp;       // the first pair's Y uses the static damping
    c.inv_count = 1.0 / ((double)ctx->nv * (double)ctx->G);
    c.cur = ctx->cur_slot;
    c.anchor_valid = 0;
    c.refresh = 0;
    c.next_refresh = 1e-2;
    c.anchor_ratio = ctx->opt.anchor_ratio > 0.0 ? ctx->opt.anchor_ratio : 1e-1;
}

template <typename T> Fields<T> &fields(rism3d_ctx *ctx);
template <> Fields<float> &fields<float>(rism3d_ctx *ctx) { return ctx->f32; }
template <> Fields<double> &fields<double>(rism3d_ctx *ctx) { return ctx->f64; }

rism3d_status to_working(rism3d_ctx *ctx, const double *src, int on_device, int slot) {
    const long long n = (long long)ctx->nv * ctx->G;
    const double *dsrc = src;
    if (!on_device) {
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->staging, src, n * sizeof(double), cudaMemcpyHostToDevice,
                                      ctx->stream));
        dsrc = ctx->staging;
    }
    if (ctx->fp32())
        CUDA_TRY(ctx, launch_guess_from_t<float>(ctx->f32, slot, dsrc, ctx->stream));
    else
        CUDA_TRY(ctx, launch_guess_from_t<double>(ctx->f64, slot, dsrc, ctx->stream));
    ctx->offset_live = false;
    return RISM3D_OK;
}

rism3d_status field_out(rism3d_ctx *ctx, int field, int slot, int kind, int order, double *dst,
                        size_t count, int on_device) {
    const long long n = field == RISM3D_PHI ? ctx->G : (long long)ctx->nv * ctx->G;
    if ((long long)count < n) return fail(ctx, RISM3D_EINVAL, "dst holds %zu values, need %lld", count, n);
    double *d = on_device ? dst : ctx->staging;
    if (ctx->fp32())
        CUDA_TRY(ctx, launch_get_field<float>(ctx->f32, field, slot, kind, order, d, ctx->stream));
    else
        CUDA_TRY(ctx, launch_get_field<double>(ctx->f64, field, slot, kind, order, d, ctx->stream));
    if (!on_device)
        CUDA_TRY(ctx, cudaMemcpyAsync(dst, ctx->staging, n * sizeof(double), cudaMemcpyDeviceToHost,
                                      ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RISM3D_OK;
}

bool valid_closure(int kind, int order) {
    if (kind == kKH || kind == kHNC) return true;
    return kind == kPSE && order >= 1 && order < kMaxClosureStages;
}

}  // namespace

// ------------------------------------------------------------------ public entry points
// Finite-size correction of the SFE (see rism3d.h): Delta = -(beta / 2) [(1 / V) sum_{k != 0}
// Re(Phi~ conj(phi~_box)) S(k) - (1 / 2 pi^2) int k^2 |Phi~|^2 S(k) dk (orientation-averaged)].
constexpr double kLrKmax = 20.0;          // quadrature of the infinite-space integral: [0, 20] 1/A
constexpr int kLrQuad = 16385;            // trapezoid points (spacing 1.22e-3 1/A)
constexpr int kLrChunks = 64;             // atom-row chunks of the pair sums
constexpr int kLrBlocks = 304;            // blocks of the lattice sum and of the quadrature

template <typename T>
static rism3d_status lr_parts(rism3d_ctx *ctx, Fields<T> &f, double *lat, double *integ) {
    typedef typename Cx<T>::type C;
    FftPlan plans[3];
    const int n[3] = {ctx->Nx, ctx->Ny, ctx->Nz};
    for (int d = 0; d < 3; ++d)
        if (!make_plan(n[d], plans[d]))
            return fail(ctx, RISM3D_EUNSUPPORTED, "no transform plan for length %d", n[d]);
    double rq[kMaxSites];
    for (int g = 0; g < kMaxSites; ++g) rq[g] = g < ctx->nv ? ctx->rho[g] * ctx->q[g] : 0.0;
    double q2 = 0.0;
    for (int a = 0; a < ctx->n_atoms; ++a) q2 += ctx->atom_host[(size_t)a * kAtomStride + 3] * ctx->atom_host[(size_t)a * kAtomStride + 3];
    const size_t nbuf = (size_t)kLrChunks * kLrQuad + 2 * kLrBlocks;
    if (!ctx->lr_buf) CUDA_TRY(ctx, cudaMalloc(&ctx->lr_buf, nbuf * sizeof(double)));
    double *pairs = ctx->lr_buf, *lat_part = pairs + (size_t)kLrChunks * kLrQuad, *int_part = lat_part + kLrBlocks;
    const double c4 = (4.0 * kPi * kCoulomb) * (4.0 * kPi * kCoulomb);
    C *scratch = reinterpret_cast<C *>(f.spec);           // free between solves; nv >= 2 checked by the caller
    CUDA_TRY(ctx, launch_lr_parts<T>(f, scratch, plans, rq, ctx->atoms, ctx->n_atoms, kLrKmax, kLrQuad, kLrChunks,
                                     pairs, lat_part, kLrBlocks, int_part, kLrBlocks, c4, q2, ctx->stream));
    std::vector<double> h(2 * kLrBlocks);
    CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), lat_part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    double sl = 0.0, si = 0.0;
    for (int b = 0; b < kLrBlocks; ++b) sl += h[b];
    for (int b = 0; b < kLrBlocks; ++b) si += h[kLrBlocks + b];
    const double V = (double)ctx->G * ctx->dV;
    *lat = sl * ctx->dV * ctx->dV / (ctx->beta * V);       // Psi = beta Phi~ / dV, phi~_box = dV DFT(phi)
    *integ = si / (2.0 * kPi * kPi);
    return RISM3D_OK;
}

extern "C" {

const char *rism3d_version(void) { return "rism3d-gb300 0.1 (sm_103a)"; }

void rism3d_options_default(rism3d_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = 32;
    opt->mdiis_nvec = 5;
    opt->mdiis_damp = 0.7;
    opt->dynamic_damp = 0;
    opt->max_iter = 10000;
    opt->check_every = 8;
    opt->max_atoms = 100000;
    opt->accelerator = 0;
    opt->anderson_s1 = 0.2;
    opt->anderson_s2 = 0.0;
    opt->anchor_ratio = 1e-1;
}

rism3d_status rism3d_workspace_bytes(const rism3d_solvent *solvent, const rism3d_grid *grid,
                                     const rism3d_options *opt, size_t *bytes) {
    Geometry g{};
    rism3d_status st = check_inputs(solvent, grid, opt, g);
    if (st != RISM3D_OK) return st;
    if (!bytes) return fail(nullptr, RISM3D_EINVAL, "null bytes");
    *bytes = make_layout(g).total;
    return RISM3D_OK;
}

rism3d_status rism3d_create(const rism3d_solvent *sv, const rism3d_grid *gr, const rism3d_options *op,
                            rism3d_ctx **out) {
    NvtxRange nvtx_("rism3d_create");
    if (!out) return fail(nullptr, RISM3D_EINVAL, "null out");
    *out = nullptr;
    Geometry g{};
    rism3d_status st = check_inputs(sv, gr, op, g);
    if (st != RISM3D_OK) return st;
    Layout L = make_layout(g);
    if (op->workspace && op->workspace_bytes < L.total)
        return fail(nullptr, RISM3D_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed",
                    op->workspace_bytes, L.total);
    if (op->workspace && (reinterpret_cast<uintptr_t>(op->workspace) & 255))
        return fail(nullptr, RISM3D_EINVAL, "workspace must be 256-byte aligned");

    rism3d_ctx *ctx = new rism3d_ctx();
    cudaGetDevice(&ctx->device);
    ctx->precision = op->precision;
    ctx->opt = *op;
    ctx->nv = g.nv;
    ctx->Nx = g.Nx;
    ctx->Ny = g.Ny;
    ctx->Nz = g.Nz;
    ctx->Kz = g.Kz;
    ctx->G = g.G;
    for (int d = 0; d < 3; ++d) {
        ctx->spacing[d] = gr->spacing[d];
        ctx->origin[d] = gr->origin[d];
    }
    ctx->q.assign(sv->q, sv->q + g.nv);
    ctx->sig.assign(sv->sigma, sv->sigma + g.nv);
    ctx->eps.assign(sv->eps, sv->eps + g.nv);
    ctx->rho.assign(sv->rho, sv->rho + g.nv);
    ctx->temperature = sv->temperature;
    ctx->beta = 1.0 / (kKB * sv->temperature);
    ctx->dV = gr->spacing[0] * gr->spacing[1] * gr->spacing[2];
    auto bail = [&](rism3d_status s) {
        g_create_error = ctx->err;
        rism3d_destroy(ctx);
        return s;
    };
    if (op->cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(op->cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(fail(ctx, RISM3D_ECUDA, "stream: %s", cudaGetErrorString(e)));
        ctx->own_stream = true;
    }
    if (op->workspace) {
        ctx->ws = op->workspace;
        ctx->ws_bytes = op->workspace_bytes;
    } else {
        cudaError_t e = cudaMalloc(&ctx->ws, L.total);
        if (e != cudaSuccess) {
            ctx->ws = nullptr;
            return bail(fail(ctx, RISM3D_ENOMEM, "cudaMalloc(%zu): %s", L.total, cudaGetErrorString(e)));
        }
        ctx->own_ws = true;
        ctx->ws_bytes = L.total;
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&ctx->ctrl_host), sizeof(Ctrl)) != cudaSuccess) {
        ctx->ctrl_host = nullptr;
        return bail(fail(ctx, RISM3D_ENOMEM, "pinned host allocation failed"));
    }
    if (op->timing)
        for (auto &e : ctx->ev_aux)
            if (cudaEventCreate(&e) != cudaSuccess) {
                e = nullptr;
                return bail(fail(ctx, RISM3D_ECUDA, "event creation failed"));
            }
    char *b = static_cast<char *>(ctx->ws);
    ctx->ctrl = reinterpret_cast<Ctrl *>(b + L.ctrl);
    ctx->atoms = reinterpret_cast<double *>(b + L.atoms);
    ctx->site_sig = reinterpret_cast<double *>(b + L.sites);
    ctx->site_eps = ctx->site_sig + kMaxSites;
    ctx->site_q = ctx->site_eps + kMaxSites;
    ctx->site_rho_dV = ctx->site_q + kMaxSites;
    ctx->sfe_part = reinterpret_cast<double *>(b + L.sfe);
    ctx->staging = reinterpret_cast<double *>(b + L.staging);
    double sites[4 * kMaxSites] = {0};
    for (int i = 0; i < g.nv; ++i) {
        sites[i] = ctx->sig[i];
        sites[kMaxSites + i] = ctx->eps[i];
        sites[2 * kMaxSites + i] = ctx->q[i];
        sites[3 * kMaxSites + i] = ctx->rho[i] * ctx->dV;
    }
    if (cudaMemcpy(ctx->site_sig, sites, sizeof(sites), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(ctx, RISM3D_ECUDA, "upload of solvent sites failed"));
    if (ctx->fp32()) {
        fill_fields<float>(ctx, g, L, ctx->f32);
        st = upload_tables<float>(ctx, sv, L, ctx->f32);
    } else {
        fill_fields<double>(ctx, g, L, ctx->f64);
        st = upload_tables<double>(ctx, sv, L, ctx->f64);
    }
    if (st != RISM3D_OK) return bail(st);
    Ctrl c;
    reset_ctrl(ctx, c);
    c.status = kConverged;       // idle until a solve
    if (cudaMemcpy(ctx->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(ctx, RISM3D_ECUDA, "upload of the control block failed"));
    *out = ctx;
    return RISM3D_OK;
}

rism3d_status rism3d_set_solute(rism3d_ctx *ctx, int n_atoms, const double *xyz, const double *q,
                                const double *sigma, const double *eps) {
    NvtxRange nvtx_("rism3d_set_solute");
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (n_atoms < 1 || n_atoms > ctx->opt.max_atoms)
        return fail(ctx, RISM3D_EINVAL, "n_atoms must be in 1..%d", ctx->opt.max_atoms);
    if (!xyz || !q || !sigma || !eps) return fail(ctx, RISM3D_EINVAL, "null solute array");
    DeviceGuard dg(ctx->device);
    const double L[3] = {ctx->Nx * ctx->spacing[0], ctx->Ny * ctx->spacing[1], ctx->Nz * ctx->spacing[2]};
    // every atom is checked before anything of the context changes: bad arguments leave the
    // previous solute in place
    std::vector<double> atoms((size_t)n_atoms * kAtomStride, 0.0);
    for (int a = 0; a < n_atoms; ++a) {
        double *at = &atoms[(size_t)a * kAtomStride];
        for (int d = 0; d < 3; ++d) {
            at[d] = xyz[3 * a + d];
            at[6 + d] = (xyz[3 * a + d] - ctx->origin[d]) / L[d];
            if (!std::isfinite(at[d])) return fail(ctx, RISM3D_EINVAL, "atom %d has a non-finite position", a);
        }
        at[3] = q[a];
        at[4] = sigma[a];
        at[5] = eps[a];
        if (!(sigma[a] >= 0.0) || !(eps[a] >= 0.0) || !std::isfinite(q[a]))
            return fail(ctx, RISM3D_EINVAL, "atom %d: sigma, eps must be >= 0 and q finite", a);
    }
    // from here on the device fields are rewritten: a CUDA error part-way leaves no solute
    ctx->has_solute = false;
    ctx->atom_host.swap(atoms);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->atoms, ctx->atom_host.data(), ctx->atom_host.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, ctx->stream));
    const double amp0 = 4.0 * kPi * kCoulomb * ctx->beta / ctx->dV;
    const double P = (double)ctx->nv * ctx->G, sb = ctx->fp32() ? 4.0 : 8.0;
    const double z = ctx->opt.kgrid == 1 ? 1.0 : (double)(ctx->Kz + 1) / ctx->Kz;
    {
        AuxTimer tm(ctx, 4);
        if (ctx->fp32())
            CUDA_TRY(ctx, launch_potential<float>(ctx->f32, ctx->atoms, n_atoms, ctx->site_sig, ctx->site_eps,
                                                  ctx->site_q, ctx->beta, ctx->origin, ctx->spacing, ctx->stream));
        else
            CUDA_TRY(ctx, launch_potential<double>(ctx->f64, ctx->atoms, n_atoms, ctx->site_sig, ctx->site_eps,
                                                   ctx->site_q, ctx->beta, ctx->origin, ctx->spacing, ctx->stream));
        tm.stop((2.0 * P + ctx->G) * sb);
    }
    {
        AuxTimer tm(ctx, 5);
        if (ctx->fp32())
            CUDA_TRY(ctx, launch_longrange<float>(ctx->f32, ctx->atoms, n_atoms, amp0, ctx->stream));
        else
            CUDA_TRY(ctx, launch_longrange<double>(ctx->f64, ctx->atoms, n_atoms, amp0, ctx->stream));
        tm.stop(ctx->G * sb * z);
    }
    {
        AuxTimer tm(ctx, 7);
        if (ctx->fp32())
            CUDA_TRY(ctx, launch_init_guess<float>(ctx->f32, 0, ctx->stream));
        else
            CUDA_TRY(ctx, launch_init_guess<double>(ctx->f64, 0, ctx->stream));
        tm.stop(P * sb);
    }
    ctx->cur_slot = 0;
    ctx->offset_live = false;
    ctx->n_atoms = n_atoms;
    ctx->has_solute = true;
    ctx->last_kind = kKH;
    ctx->last_order = 1;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RISM3D_OK;
}

rism3d_status rism3d_set_guess(rism3d_ctx *ctx, const double *t, int on_device) {
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "set_guess before set_solute");
    if (!t) return fail(ctx, RISM3D_EINVAL, "null t");
    DeviceGuard dg(ctx->device);
    ctx->cur_slot = 0;
    rism3d_status st = to_working(ctx, t, on_device, 0);
    if (st != RISM3D_OK) return st;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RISM3D_OK;
}

// A solve in phases, so that the batch scheduler can interleave contexts: begin (graph,
// control block), launch a chunk of check_every iterations (graph + status read-back +
// event), take a finished chunk's accounting, finish (final control block, report).
static rism3d_status solve_begin(rism3d_ctx *ctx, int closure, int pse_order, double tol) {
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "solve before set_solute");
    if (!valid_closure(closure, pse_order)) return fail(ctx, RISM3D_EINVAL, "bad closure %d / order %d", closure, pse_order);
    if (!(tol > 0.0)) return fail(ctx, RISM3D_EINVAL, "tol must be positive");
    ctx->run_t0 = std::chrono::steady_clock::now();
    rism3d_status st = build_graph(ctx);
    if (st != RISM3D_OK) return st;
    if (!ctx->chunk_ev) CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->chunk_ev, cudaEventDisableTiming));
    if (ctx->offset_live) {              // restart from the last iterate with tau0 = 0
        if (ctx->fp32())
            CUDA_TRY(ctx, launch_flatten<float>(ctx->f32, ctx->stream));
        else
            CUDA_TRY(ctx, launch_flatten<double>(ctx->f64, ctx->stream));
    }
    ctx->offset_live = true;
    Ctrl &c = *ctx->ctrl_host;
    reset_ctrl(ctx, c);
    closure_stages(closure, pse_order, tol, c);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, ctx->stream));
    ctx->run_iter_before = 0;
    ctx->run_closure = closure;
    ctx->run_order = pse_order;
    return RISM3D_OK;
}

static rism3d_status solve_launch_chunk(rism3d_ctx *ctx) {
    CUDA_TRY(ctx, cudaGraphLaunch(ctx->graph, ctx->stream));
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctrl_host, ctx->ctrl, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaEventRecord(ctx->chunk_ev, ctx->stream));
    return RISM3D_OK;
}

// After the chunk's event has completed: launch counts and kernel times; *running tells
// whether the solve needs another chunk.
static rism3d_status solve_chunk_done(rism3d_ctx *ctx, bool *running) {
    const Ctrl &c = *ctx->ctrl_host;
    const int K = ctx->opt.check_every;
    const int ran = c.iter - ctx->run_iter_before;
    ctx->run_iter_before = c.iter;
    int slots[kMaxLaunches];
    const int nk = iteration_slots(ctx, true, slots);
    for (int k = 0; k < nk; ++k) ctx->stats.launches[slots[k]] += K;
    if (ctx->opt.timing) {
        const int timed_its = ctx->opt.timing == 2 ? 1 : K;
        for (int i = 0; i < ran && i < timed_its; ++i)
            for (int k = 0; k < nk; ++k) {
                float ms = 0.f;
                const size_t e0 = (size_t)i * kEventsPerIter + 2 * k;   // pair around launch k
                CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev[e0], ctx->ev[e0 + 1]));
                ctx->stats.ms[slots[k]] += ms;
                ctx->stats.timed[slots[k]] += 1;
            }
    }
    *running = c.status == kRunning;
    return RISM3D_OK;
}

// stop = true ends a running solve early (batch time limit): the device control block is
// marked stopped so that kernels still queued return at once.
static rism3d_status solve_finish(rism3d_ctx *ctx, rism3d_report *rep, bool stop) {
    Ctrl &c = *ctx->ctrl_host;
    if (stop) {
        c.status = kStopped;
        CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctrl, &c, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    }
    CUDA_TRY(ctx, cudaMemcpyAsync(&c, ctx->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    auto t1 = std::chrono::steady_clock::now();
    account_iterations(ctx, c);
    ctx->stats.solves += 1;
    ctx->cur_slot = c.cur;
    ctx->last_kind = ctx->run_closure;
    ctx->last_order = ctx->run_closure == kPSE ? ctx->run_order : (ctx->run_closure == kKH ? 1 : 0);
    if (rep) {
        rep->iterations = c.iter;
        rep->converged = c.status == kConverged;
        rep->rms_residual = c.rms;
        rep->seconds_iter = std::chrono::duration<double>(t1 - ctx->run_t0).count();
    }
    if (c.status == kStopped)
        return fail(ctx, RISM3D_ETIMEOUT, "stopped by the time limit at iteration %d (rms %.3e)", c.iter, c.rms);
    if (c.status == kDiverged) return fail(ctx, RISM3D_EDIVERGED, "non-finite residual at iteration %d", c.iter);
    if (c.status == kMaxIter)
        return fail(ctx, RISM3D_ENOTCONV, "not converged after %d iterations (rms %.3e)", c.iter, c.rms);
    return RISM3D_OK;
}

rism3d_status rism3d_solve(rism3d_ctx *ctx, int closure, int pse_order, double tol, rism3d_report *rep) {
    NvtxRange nvtx_("rism3d_solve");
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    DeviceGuard dg(ctx->device);
    rism3d_status st = solve_begin(ctx, closure, pse_order, tol);
    if (st != RISM3D_OK) return st;
    for (;;) {
        if ((st = solve_launch_chunk(ctx)) != RISM3D_OK) return st;
        CUDA_TRY(ctx, cudaEventSynchronize(ctx->chunk_ev));
        bool running = false;
        if ((st = solve_chunk_done(ctx, &running)) != RISM3D_OK) return st;
        if (!running) break;
    }
    return solve_finish(ctx, rep, false);
}

rism3d_status rism3d_solve_batch(rism3d_batch_job *jobs, int n_jobs, int max_inflight, double time_limit_s) {
    NvtxRange nvtx_("rism3d_solve_batch");
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(nullptr, RISM3D_EINVAL, "bad job list");
    if (max_inflight < 1) return fail(nullptr, RISM3D_EINVAL, "max_inflight must be >= 1");
    for (int j = 0; j < n_jobs; ++j) {    // a job that never starts reports ESTATE
        jobs[j].status = RISM3D_ESTATE;
        jobs[j].sfe = 0.0;
        jobs[j].report = rism3d_report{};
    }
    int device = -1;
    for (int j = 0; j < n_jobs; ++j) {
        rism3d_ctx *c = jobs[j].ctx;
        if (!c) return fail(nullptr, RISM3D_EINVAL, "job %d has no context", j);
        if (device < 0) device = c->device;
        if (c->device != device) return fail(nullptr, RISM3D_EINVAL, "jobs span more than one device");
        for (int i = 0; i < j; ++i)
            if (jobs[i].ctx == c) return fail(nullptr, RISM3D_EINVAL, "jobs %d and %d share a context", i, j);
    }
    if (n_jobs == 0) return RISM3D_OK;
    DeviceGuard dg(device);
    using clock = std::chrono::steady_clock;
    std::vector<int> active;
    std::vector<clock::time_point> started(n_jobs);
    int next = 0, done = 0;
    auto end_job = [&](int j, rism3d_status st) {
        rism3d_batch_job &J = jobs[j];
        if (J.sfe_kind && (st == RISM3D_OK || st == RISM3D_ENOTCONV)) {
            const rism3d_status s2 = rism3d_get_sfe(J.ctx, J.sfe_kind, J.pse_order, &J.sfe, nullptr);
            if (st == RISM3D_OK) st = s2;
        }
        J.status = st;
        ++done;
    };
    auto start_job = [&](int j) {
        rism3d_batch_job &J = jobs[j];
        started[j] = clock::now();
        rism3d_status st = RISM3D_OK;
        if (J.n_atoms > 0) st = rism3d_set_solute(J.ctx, J.n_atoms, J.xyz, J.q, J.sigma, J.eps);
        if (st == RISM3D_OK) st = solve_begin(J.ctx, J.closure, J.pse_order, J.tol);
        if (st == RISM3D_OK) st = solve_launch_chunk(J.ctx);
        if (st != RISM3D_OK) {
            end_job(j, st);
            return;
        }
        active.push_back(j);
    };
    while (done < n_jobs) {
        while ((int)active.size() < max_inflight && next < n_jobs) start_job(next++);
        bool progressed = false;
        for (size_t a = 0; a < active.size();) {
            const int j = active[a];
            rism3d_ctx *c = jobs[j].ctx;
            const cudaError_t q = cudaEventQuery(c->chunk_ev);
            if (q == cudaErrorNotReady) {
                ++a;
                continue;
            }
            progressed = true;
            rism3d_status st = q == cudaSuccess ? RISM3D_OK
                                                : fail(c, RISM3D_ECUDA, "chunk: %s", cudaGetErrorString(q));
            bool running = false;
            if (st == RISM3D_OK) st = solve_chunk_done(c, &running);
            const bool late = time_limit_s > 0.0 &&
                              std::chrono::duration<double>(clock::now() - started[j]).count() > time_limit_s;
            if (st == RISM3D_OK && running && !late) {
                st = solve_launch_chunk(c);
                if (st == RISM3D_OK) {
                    ++a;
                    continue;
                }
            }
            if (st == RISM3D_OK) st = solve_finish(c, &jobs[j].report, running && late);
            active.erase(active.begin() + a);
            end_job(j, st);
            if (next < n_jobs) start_job(next++);
        }
        if (!progressed) std::this_thread::yield();
    }
    for (int j = 0; j < n_jobs; ++j)
        if (jobs[j].status != RISM3D_OK) return jobs[j].status;
    return RISM3D_OK;
}

// ------------------------------------------------------------------ batch as one graph launch
// Loop test at the end of one body pass of a job's device loop: the first pass sets the
// deadline (%globaltimer + limit_ns; limit_ns = 0: none); a running solve past its deadline
// is marked stopped; the loop goes on while the solve runs.
static __global__ void k_loop_ctl(Ctrl *c, cudaGraphConditionalHandle h, unsigned long long limit_ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    if (limit_ns && c->deadline == 0ULL) c->deadline = now + limit_ns;
    if (c->status == kRunning && c->deadline != 0ULL && now > c->deadline) c->status = kStopped;
    cudaGraphSetConditional(h, c->status == kRunning ? 1u : 0u);
}

// Adds to g one conditional while node whose body is check_every iterations of ctx followed
// by the loop test (captured on the context's own streams).
static rism3d_status add_device_loop(rism3d_ctx *ctx, cudaGraph_t g, unsigned long long limit_ns) {
    cudaGraphConditionalHandle h;
    CUDA_TRY(ctx, cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(ctx, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (rism3d_status st0 = ensure_side(ctx)) return st0;
    CUDA_TRY(ctx, cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    rism3d_status st = RISM3D_OK;
    for (int i = 0; i < ctx->opt.check_every && st == RISM3D_OK; ++i)
        st = ctx->fp32() ? run_iteration<float>(ctx, ctx->f32, true, nullptr)
                         : run_iteration<double>(ctx, ctx->f64, true, nullptr);
    if (st == RISM3D_OK) {
        k_loop_ctl<<<1, 32, 0, ctx->stream>>>(ctx->ctrl, h, limit_ns);
        if (cudaGetLastError() != cudaSuccess) st = fail(ctx, RISM3D_ECUDA, "loop test launch");
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &out);
    if (st != RISM3D_OK) return st;
    if (e != cudaSuccess) return fail(ctx, RISM3D_ECUDA, "device loop capture: %s", cudaGetErrorString(e));
    return RISM3D_OK;
}

rism3d_status rism3d_solve_batch_graph(rism3d_batch_job *jobs, int n_jobs, double time_limit_s) {
    NvtxRange nvtx_("rism3d_solve_batch_graph");
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(nullptr, RISM3D_EINVAL, "bad job list");
    if (!(time_limit_s >= 0.0)) return fail(nullptr, RISM3D_EINVAL, "time_limit_s must be >= 0");
    for (int j = 0; j < n_jobs; ++j) {
        jobs[j].status = RISM3D_ESTATE;
        jobs[j].sfe = 0.0;
        jobs[j].report = rism3d_report{};
    }
    int device = -1;
    for (int j = 0; j < n_jobs; ++j) {
        rism3d_ctx *c = jobs[j].ctx;
        if (!c) return fail(nullptr, RISM3D_EINVAL, "job %d has no context", j);
        if (device < 0) device = c->device;
        if (c->device != device) return fail(nullptr, RISM3D_EINVAL, "jobs span more than one device");
        for (int i = 0; i < j; ++i)
            if (jobs[i].ctx == c) return fail(nullptr, RISM3D_EINVAL, "jobs %d and %d share a context", i, j);
    }
    if (n_jobs == 0) return RISM3D_OK;
    DeviceGuard dg(device);
    const unsigned long long limit_ns =
        time_limit_s > 0.0 ? (unsigned long long)std::max(1.0, time_limit_s * 1e9) : 0ULL;
    std::vector<char> live(n_jobs, 0);
    cudaStream_t ls = nullptr;
    cudaEvent_t done = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    rism3d_status rc = RISM3D_OK;
    auto cleanup = [&]() {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        if (done) cudaEventDestroy(done);
        if (ls) cudaStreamDestroy(ls);
    };
    if (cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess || cudaGraphCreate(&g, 0) != cudaSuccess) {
        cleanup();
        return fail(nullptr, RISM3D_ECUDA, "batch graph: stream, event or graph creation failed");
    }
    // per job: solute, control block, and its device loop in the graph
    for (int j = 0; j < n_jobs; ++j) {
        rism3d_batch_job &J = jobs[j];
        rism3d_status st = RISM3D_OK;
        if (J.n_atoms > 0) st = rism3d_set_solute(J.ctx, J.n_atoms, J.xyz, J.q, J.sigma, J.eps);
        if (st == RISM3D_OK) st = solve_begin(J.ctx, J.closure, J.pse_order, J.tol);
        if (st == RISM3D_OK) st = add_device_loop(J.ctx, g, limit_ns);
        if (st == RISM3D_OK && (cudaEventRecord(J.ctx->chunk_ev, J.ctx->stream) != cudaSuccess ||
                                cudaStreamWaitEvent(ls, J.ctx->chunk_ev, 0) != cudaSuccess))
            st = fail(J.ctx, RISM3D_ECUDA, "batch graph: ordering after the job's set-up");
        if (st != RISM3D_OK) {
            J.status = st;
            cleanup();
            return st;
        }
        live[j] = 1;
    }
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, ls);
    if (e == cudaSuccess) e = cudaEventRecord(done, ls);
    if (e != cudaSuccess) {
        cleanup();
        return fail(nullptr, RISM3D_ECUDA, "batch graph: %s", cudaGetErrorString(e));
    }
    for (int j = 0; j < n_jobs; ++j) {
        rism3d_batch_job &J = jobs[j];
        rism3d_status st = RISM3D_OK;
        if (cudaStreamWaitEvent(J.ctx->stream, done, 0) != cudaSuccess)
            st = fail(J.ctx, RISM3D_ECUDA, "batch graph: ordering before the read-back");
        if (st == RISM3D_OK) st = solve_finish(J.ctx, &J.report, false);
        if (st == RISM3D_OK || st == RISM3D_ETIMEOUT || st == RISM3D_ENOTCONV) {
            // launches: every body pass runs check_every iterations' kernels
            int slots[kMaxLaunches];
            const int nk = iteration_slots(J.ctx, true, slots);
            const int K = J.ctx->opt.check_every;
            const long long passes = std::max(1, (J.report.iterations + K - 1) / K);
            for (int k = 0; k < nk; ++k) J.ctx->stats.launches[slots[k]] += passes * K;
        }
        if (J.sfe_kind && (st == RISM3D_OK || st == RISM3D_ENOTCONV)) {
            const rism3d_status s2 = rism3d_get_sfe(J.ctx, J.sfe_kind, J.pse_order, &J.sfe, nullptr);
            if (st == RISM3D_OK) st = s2;
        }
        J.status = st;
        if (st != RISM3D_OK && rc == RISM3D_OK) rc = st;
    }
    cudaEventSynchronize(done);
    cleanup();
    return rc;
}

rism3d_status rism3d_residual(rism3d_ctx *ctx, int closure, int pse_order, const double *t, double *R,
                              int on_device) {
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "residual before set_solute");
    if (!valid_closure(closure, pse_order)) return fail(ctx, RISM3D_EINVAL, "bad closure");
    if (!t || !R) return fail(ctx, RISM3D_EINVAL, "null t or R");
    DeviceGuard dg(ctx->device);
    ctx->cur_slot = 0;
    rism3d_status st = to_working(ctx, t, on_device, 0);
    if (st != RISM3D_OK) return st;
    Ctrl &c = *ctx->ctrl_host;
    reset_ctrl(ctx, c);
    c.n_stages = 1;
    c.stage_kind[0] = closure;
    c.stage_order[0] = closure == kPSE ? pse_order : (closure == kKH ? 1 : 0);
    c.stage_tol[0] = 0.0;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, ctx->stream));
    st = iteration(ctx, false);
    if (st != RISM3D_OK) return st;
    {
        int slots[kMaxLaunches];
        const int nk = iteration_slots(ctx, false, slots);
        for (int kk = 0; kk < nk; ++kk) ctx->stats.launches[slots[kk]] += 1;
    }
    const int k = c.stage_kind[0], o = c.stage_order[0];
    st = field_out(ctx, RISM3D_R, 0, k, o, R, (size_t)ctx->nv * ctx->G, on_device);
    // leave the device idle
    c.status = kConverged;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctrl, &c, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return st;
}

rism3d_status rism3d_get(rism3d_ctx *ctx, int field, double *dst, size_t count, int on_device) {
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (field < RISM3D_G || field > RISM3D_R) return fail(ctx, RISM3D_EINVAL, "bad field %d", field);
    if (!dst) return fail(ctx, RISM3D_EINVAL, "null dst");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "get before set_solute");
    DeviceGuard dg(ctx->device);
    return field_out(ctx, field, ctx->cur_slot, ctx->last_kind, ctx->last_order, dst, count, on_device);
}

rism3d_status rism3d_get_sfe(rism3d_ctx *ctx, int kind, int pse_order, double *total, double *per_site) {
    NvtxRange nvtx_("rism3d_get_sfe");
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (kind < RISM3D_SFE_KH || kind > RISM3D_SFE_PSE) return fail(ctx, RISM3D_EINVAL, "bad SFE kind %d", kind);
    if (kind == RISM3D_SFE_PSE && pse_order < 1) return fail(ctx, RISM3D_EINVAL, "PSE order must be >= 1");
    if (!total) return fail(ctx, RISM3D_EINVAL, "null total");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "get_sfe before set_solute");
    DeviceGuard dg(ctx->device);
    {
        AuxTimer tm(ctx, 6);
        if (ctx->fp32())
            CUDA_TRY(ctx, launch_sfe<float>(ctx->f32, ctx->cur_slot, ctx->last_kind, ctx->last_order, kind,
                                            pse_order, ctx->sfe_part, kSfeBlocksPerSite, ctx->stream));
        else
            CUDA_TRY(ctx, launch_sfe<double>(ctx->f64, ctx->cur_slot, ctx->last_kind, ctx->last_order, kind,
                                             pse_order, ctx->sfe_part, kSfeBlocksPerSite, ctx->stream));
        tm.stop(2.0 * ctx->nv * ctx->G * (ctx->fp32() ? 4.0 : 8.0));
    }
    std::vector<double> part((size_t)ctx->nv * kSfeBlocksPerSite);
    CUDA_TRY(ctx, cudaMemcpyAsync(part.data(), ctx->sfe_part, part.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const double kT = kKB * ctx->temperature;
    double tot = 0.0;
    for (int g = 0; g < ctx->nv; ++g) {
        double s = 0.0;
        for (int b = 0; b < kSfeBlocksPerSite; ++b) s += part[(size_t)g * kSfeBlocksPerSite + b];
        const double v = kT * ctx->rho[g] * ctx->dV * s;
        if (per_site) per_site[g] = v;
        tot += v;
    }
    *total = tot;
    return RISM3D_OK;
}

rism3d_status rism3d_get_sfe_finite_size(rism3d_ctx *ctx, double *delta) {
    NvtxRange nvtx_("rism3d_get_sfe_finite_size");
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (!delta) return fail(ctx, RISM3D_EINVAL, "null delta");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "finite-size correction before set_solute");
    if (ctx->opt.kgrid != 0)
        return fail(ctx, RISM3D_EUNSUPPORTED, "the finite-size correction is defined on the periodic (integer) k grid");
    if (ctx->nv < 2) return fail(ctx, RISM3D_EUNSUPPORTED, "the finite-size correction needs at least two solvent sites");
    DeviceGuard dg(ctx->device);
    double lat = 0.0, integ = 0.0;
    rism3d_status st = ctx->fp32() ? lr_parts<float>(ctx, ctx->f32, &lat, &integ)
                                   : lr_parts<double>(ctx, ctx->f64, &lat, &integ);
    if (st != RISM3D_OK) return st;
    *delta = -0.5 * ctx->beta * (lat - integ);
    return RISM3D_OK;
}

static rism3d_status guess_crop(rism3d_ctx *ctx, int mode, const int *corner, int crop, float *out,
                                const float *in) {
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "learned-guess crop before set_solute");
    if (!corner || crop < 1 || (mode == 2 ? !in : !out)) return fail(ctx, RISM3D_EINVAL, "bad crop arguments");
    const int N[3] = {ctx->Nx, ctx->Ny, ctx->Nz};
    for (int d = 0; d < 3; ++d)
        if (corner[d] < 0 || (long long)corner[d] + crop > N[d])
            return fail(ctx, RISM3D_EINVAL, "crop [%d, %d) outside the grid on axis %d", corner[d], corner[d] + crop, d);
    DeviceGuard dg(ctx->device);
    const int slot = mode == 2 ? 0 : ctx->cur_slot;
    if (ctx->fp32())
        CUDA_TRY(ctx, launch_guess_crop<float>(ctx->f32, mode, slot, corner, crop, out, in, ctx->stream));
    else
        CUDA_TRY(ctx, launch_guess_crop<double>(ctx->f64, mode, slot, corner, crop, out, in, ctx->stream));
    if (mode == 2) {
        ctx->cur_slot = 0;
        ctx->offset_live = false;
    }
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return RISM3D_OK;
}

rism3d_status rism3d_guess_input(rism3d_ctx *ctx, const int *corner, int crop, float *x) {
    return guess_crop(ctx, 0, corner, crop, x, nullptr);
}

rism3d_status rism3d_guess_target(rism3d_ctx *ctx, const int *corner, int crop, float *tau) {
    return guess_crop(ctx, 1, corner, crop, tau, nullptr);
}

rism3d_status rism3d_set_guess_crop(rism3d_ctx *ctx, const int *corner, int crop, const float *tau) {
    return guess_crop(ctx, 2, corner, crop, nullptr, tau);
}

rism3d_status rism3d_get_pmv(rism3d_ctx *ctx, double kT_chi_T, double *pmv, double *c_integral) {
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (!pmv || !(kT_chi_T > 0.0)) return fail(ctx, RISM3D_EINVAL, "need pmv and kT_chi_T > 0");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "get_pmv before set_solute");
    DeviceGuard dg(ctx->device);
    {
        AuxTimer tm(ctx, 6);
        if (ctx->fp32())
            CUDA_TRY(ctx, launch_sfe<float>(ctx->f32, ctx->cur_slot, ctx->last_kind, ctx->last_order, 5, 1,
                                            ctx->sfe_part, kSfeBlocksPerSite, ctx->stream));
        else
            CUDA_TRY(ctx, launch_sfe<double>(ctx->f64, ctx->cur_slot, ctx->last_kind, ctx->last_order, 5, 1,
                                             ctx->sfe_part, kSfeBlocksPerSite, ctx->stream));
        tm.stop(2.0 * ctx->nv * ctx->G * (ctx->fp32() ? 4.0 : 8.0));
    }
    std::vector<double> part((size_t)ctx->nv * kSfeBlocksPerSite);
    CUDA_TRY(ctx, cudaMemcpyAsync(part.data(), ctx->sfe_part, part.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    double rc = 0.0;
    for (int g = 0; g < ctx->nv; ++g) {
        double sum = 0.0;
        for (int b = 0; b < kSfeBlocksPerSite; ++b) sum += part[(size_t)g * kSfeBlocksPerSite + b];
        const double ci = ctx->dV * sum;
        if (c_integral) c_integral[g] = ci;
        rc += ctx->rho[g] * ci;
    }
    *pmv = kT_chi_T * (1.0 - rc);
    return RISM3D_OK;
}

rism3d_status rism3d_get_sfe_gradient(rism3d_ctx *ctx, double *grad) {
    NvtxRange nvtx_("rism3d_get_sfe_gradient");
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (!grad) return fail(ctx, RISM3D_EINVAL, "null grad");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "get_sfe_gradient before set_solute");
    DeviceGuard dg(ctx->device);
    // partial sums and results in the FP64 staging field, atoms taken in chunks that fit
    const long long cap = (long long)ctx->nv * ctx->G;
    const long long per_atom = 3LL * kGradBlocks + 3;
    int chunk = (int)std::min<long long>(ctx->n_atoms, cap / per_atom);
    if (chunk < 1) return fail(ctx, RISM3D_EUNSUPPORTED, "grid too small for the gradient scratch");
    for (int a0 = 0; a0 < ctx->n_atoms; a0 += chunk) {
        const int na = std::min(chunk, ctx->n_atoms - a0);
        double *part = ctx->staging;
        double *out = ctx->staging + (long long)na * 3 * kGradBlocks;
        const double *atoms = ctx->atoms + (long long)a0 * kAtomStride;
        AuxTimer tm(ctx, 7);
        if (ctx->fp32())
            CUDA_TRY(ctx, launch_sfe_gradient<float>(ctx->f32, ctx->cur_slot, ctx->last_kind, ctx->last_order,
                                                     ctx->site_rho_dV, atoms, na, ctx->site_sig, ctx->site_eps,
                                                     ctx->site_q, ctx->origin, ctx->spacing, part, out,
                                                     ctx->stream));
        else
            CUDA_TRY(ctx, launch_sfe_gradient<double>(ctx->f64, ctx->cur_slot, ctx->last_kind, ctx->last_order,
                                                      ctx->site_rho_dV, atoms, na, ctx->site_sig, ctx->site_eps,
                                                      ctx->site_q, ctx->origin, ctx->spacing, part, out,
                                                      ctx->stream));
        tm.stop((double)ctx->nv * ctx->G * (ctx->fp32() ? 4.0 : 8.0));
        CUDA_TRY(ctx, cudaMemcpyAsync(grad + (size_t)a0 * 3, out, (size_t)na * 3 * sizeof(double),
                                      cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return RISM3D_OK;
}

}  // extern "C"

// Pencil tile width W chosen by measurement: the x-transform pass is timed on this
// context's own buffers for every W whose tile fits in shared memory, and the fastest is
// kept (the captured graph is rebuilt on the next solve).
template <typename T>
static rism3d_status tune_pencil(rism3d_ctx *ctx, Fields<T> &f, int *chosen, double *ms_out) {
    typedef typename Cx<T>::type C;
    Ctrl &c = *ctx->ctrl_host;
    const int saved_status = c.status;
    c.status = kRunning;                      // the pass runs only for a running solve
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctrl, &c, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(ctx, cudaEventCreate(&e0));
    CUDA_TRY(ctx, cudaEventCreate(&e1));
    int best_w = f.W;
    float best = 1e30f;
    rism3d_status st = RISM3D_OK;
    for (int w = 1; w <= 32 && st == RISM3D_OK; w *= 2) {
        const size_t smem = sizeof(C) * ((size_t)f.nv * w * f.pencil_pitch + f.Nx);
        if (smem > kMaxSmem - 1024) break;
        f.W = w;
        f.tiles_main = f.Ny * ((f.Kz + w - 1) / w);
        f.tiles_nyq = f.half ? 0 : (f.Ny + w - 1) / w;
        f.dW = make_fastdiv(w);
        cudaError_t e = launch_pencil<T>(f, ctx->stream);            // warm-up
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            if (r == 1) e = cudaEventRecord(e0, ctx->stream);
            if (e == cudaSuccess) e = launch_pencil<T>(f, ctx->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            st = fail(ctx, RISM3D_ECUDA, "pencil tuning (W = %d): %s", w, cudaGetErrorString(e));
            break;
        }
        if (ms < best) {
            best = ms;
            best_w = w;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    f.W = best_w;
    f.tiles_main = f.Ny * ((f.Kz + best_w - 1) / best_w);
    f.tiles_nyq = f.half ? 0 : (f.Ny + best_w - 1) / best_w;
    f.dW = make_fastdiv(best_w);
    c.status = saved_status;
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ctrl, &c, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    if (chosen) *chosen = best_w;
    if (ms_out) *ms_out = best / 2.0;
    return st;
}

extern "C" {

rism3d_status rism3d_tune_planes(const rism3d_solvent *sv, const rism3d_grid *gr, const rism3d_options *op,
                                 int iters, rism3d_options *best, double *ms_per_iter) {
    NvtxRange nvtx_("rism3d_tune_planes");
    if (!sv || !gr || !op || !best) return fail(nullptr, RISM3D_EINVAL, "null argument");
    if (iters < 2) return fail(nullptr, RISM3D_EINVAL, "iters must be >= 2");
    struct Cand {
        int slab, ypencil;
    };
    std::vector<Cand> cands = {{0, 0}};
    const int Ny = gr->n[1];
    for (int d : {2, 4, 8})
        if (Ny % d == 0) {
            cands.push_back({Ny / d, 0});
            cands.push_back({Ny / d, 1});
        }
    double best_ms = 1e300;
    bool found = false;
    rism3d_options chosen = *op;
    for (const Cand &c : cands) {
        rism3d_options o = *op;
        o.slab_rows = c.slab;
        o.ypencil_pass = c.ypencil;
        o.max_iter = iters;
        o.timing = 0;
        o.workspace = nullptr;          // each candidate allocates its own workspace
        o.workspace_bytes = 0;
        rism3d_ctx *ctx = nullptr;
        if (rism3d_create(sv, gr, &o, &ctx) != RISM3D_OK) continue;   // shape not available here
        double xyz[3];
        for (int d = 0; d < 3; ++d) xyz[d] = gr->origin[d] + 0.5 * gr->n[d] * gr->spacing[d];
        const double q = 0.0, sig = 3.5, eps = 0.2;
        double ms = 1e300;
        if (rism3d_set_solute(ctx, 1, xyz, &q, &sig, &eps) == RISM3D_OK) {
            rism3d_report rep{};
            rism3d_solve(ctx, RISM3D_KH, 1, 1e-300, &rep);          // graph capture and warm-up
            const rism3d_status st = rism3d_solve(ctx, RISM3D_KH, 1, 1e-300, &rep);
            if ((st == RISM3D_OK || st == RISM3D_ENOTCONV) && rep.iterations > 0)
                ms = rep.seconds_iter * 1e3 / rep.iterations;
        }
        rism3d_destroy(ctx);
        if (ms < best_ms) {
            best_ms = ms;
            chosen.slab_rows = c.slab;
            chosen.ypencil_pass = c.ypencil;
            found = true;
        }
    }
    if (!found) return fail(nullptr, RISM3D_EUNSUPPORTED, "no plane tile shape could be created and timed");
    *best = chosen;
    if (ms_per_iter) *ms_per_iter = best_ms;
    return RISM3D_OK;
}

rism3d_status rism3d_tune(rism3d_ctx *ctx, int *pencil_width, double *pencil_ms) {
    NvtxRange nvtx_("rism3d_tune");
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    if (!ctx->has_solute) return fail(ctx, RISM3D_ESTATE, "tune before set_solute");
    DeviceGuard dg(ctx->device);
    return ctx->fp32() ? tune_pencil<float>(ctx, ctx->f32, pencil_width, pencil_ms)
                       : tune_pencil<double>(ctx, ctx->f64, pencil_width, pencil_ms);
}

rism3d_status rism3d_get_stats(const rism3d_ctx *ctx, rism3d_stats *out) {
    if (!ctx || !out) return fail(nullptr, RISM3D_EINVAL, "null context or stats");
    *out = ctx->stats;
    return RISM3D_OK;
}

rism3d_status rism3d_reset_stats(rism3d_ctx *ctx) {
    if (!ctx) return fail(nullptr, RISM3D_EINVAL, "null context");
    std::memset(&ctx->stats, 0, sizeof(ctx->stats));
    return RISM3D_OK;
}

const char *rism3d_last_error(const rism3d_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void rism3d_destroy(rism3d_ctx *ctx) {
    if (!ctx) return;
    {
        DeviceGuard dg(ctx->device);
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
        for (auto e : ctx->ev)
            if (e) cudaEventDestroy(e);
        for (auto e : ctx->ev_aux)
            if (e) cudaEventDestroy(e);
        if (ctx->chunk_ev) cudaEventDestroy(ctx->chunk_ev);
        for (auto e : ctx->fork)
            if (e) cudaEventDestroy(e);
        if (ctx->side) cudaStreamDestroy(ctx->side);
        if (ctx->own_ws && ctx->ws) cudaFree(ctx->ws);
        if (ctx->lr_buf) cudaFree(ctx->lr_buf);
        if (ctx->ctrl_host) cudaFreeHost(ctx->ctrl_host);
        if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    }
    delete ctx;
}

}  // extern "C"
