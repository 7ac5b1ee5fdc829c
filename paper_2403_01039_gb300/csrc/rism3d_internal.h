// Internal declarations shared by the kernels (rism3d_kernels.cuh) and the host layer
// (rism3d_capi.cu). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rism {

constexpr int kMaxSites = 8;      // solvent sites n_v
constexpr int kMaxHist = 16;      // MDIIS vectors M
constexpr int kMaxRadixStages = 10;
constexpr int kMaxClosureStages = 12;
constexpr int kThreadsPlane = 256;
constexpr int kThreadsPencil = 256;
constexpr int kThreadsMdiis = 32 * (kMaxHist + 1);   // at least one warp per Gram value
constexpr int kSplitBlocks = 608;                     // element-kernel blocks per half (split passes)
constexpr int kSplitPartials = 2 * (kSplitBlocks + kMaxSites);   // Gram partial slots they need

// Solver status words written by the device (Ctrl::status).
enum { kRunning = 0, kConverged = 1, kDiverged = 2, kMaxIter = 3, kStopped = 4 };
enum { kKH = 1, kHNC = 2, kPSE = 3 };

// Mixed-radix plan of one transform length: L = prod(radix[0..nst)).
// Division by a run-time constant d (1 <= d < 2^31) for 0 <= n < 2^31 with one high
// multiply: q = (umulhi(n, mul) + n) >> l, l = ceil(log2 d), mul = floor(2^32 (2^l - d) / d) + 1
// (the round-up method of Granlund and Montgomery). Used in the index arithmetic of the
// element loops, where a hardware-less integer division costs tens of instructions.
struct FastDiv {
    unsigned d, mul, l;
};
inline FastDiv make_fastdiv(unsigned d) {
    FastDiv f;
    f.d = d;
    f.l = 0;
    while ((1ull << f.l) < d) ++f.l;
    f.mul = (unsigned)((((1ull << 32) * ((1ull << f.l) - d)) / d) + 1);
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ int fdiv(int n, const FastDiv &f) {
    return (int)((__umulhi((unsigned)n, f.mul) + (unsigned)n) >> f.l);
}
#endif

struct FftPlan {
    int L;
    int nst;
    int radix[kMaxRadixStages];
    int seq_per_warp;               // > 0: warp-cooperative transform of this many sequences
    FastDiv dlr[kMaxRadixStages];   // per stage: L / radix (butterflies per sequence)
    FastDiv dns[kMaxRadixStages];   // per stage: product of the earlier radices
};

// Device-resident solver state. The iteration kernels read it on every launch, so one
// captured CUDA graph serves every iteration; the MDIIS kernel rewrites it.
struct Ctrl {
    int status;
    int iter;                       // iterations done (all stages)
    int max_iter;
    int n_stages;
    int stage;
    int stage_kind[kMaxClosureStages];
    int stage_order[kMaxClosureStages];
    double stage_tol[kMaxClosureStages];
    int M;                          // history capacity
    int dynamic;
    double damp;
    int accel;                      // 0 MDIIS (Eq. 40), 1 modified Anderson (Eqs. 34-39)
    double s1, s2;                  // Anderson shifts
    double inv_count;               // 1 / (n_v * Nx * Ny * Nz)
    int n_partials;                 // blocks that wrote Gram partials
    // iterate bookkeeping
    int cur;                        // ring slot that receives the pair (Y, R) of the current t
    int do_update;                  // plane_fwd forms t = sum c_i Y_i + sum d_i R_i into Tc
    int upd_n;
    int upd_slot[kMaxHist];
    double upd_coef[kMaxHist];      // c_i of Eq. 40
    double upd_dcoef[kMaxHist];     // d_i = c_i (eta - eta_i): nonzero only if the damping changed
    int upd_r;                      // 1 if some d_i != 0 (the update then also reads R_i)
    double eta;                     // damping of the next update; plane_inv stores Y = t + eta R
    double eta_slot[kMaxHist];      // the eta each slot's Y was stored with
    int hist_n;                     // history slots (oldest first) paired with R_cur in the Gram
    int hist_slot[kMaxHist];
    double rms;                     // RMS of the last residual
    // defect-correction anchor: h = h_a + L(c^sr - c^sr_a) with L the linear map of
    // steps 3-5; refreshed (g_a = g, h_a = h and the iterate offset tau0 moved to the current
    // iterate) whenever the RMS falls below next_refresh
    int anchor_valid;
    int refresh;
    double next_refresh;
    // work counters for the byte model, summed over the iterations that ran
    long long acc_iters;
    long long acc_fwd_units;        // fields read + written by plane_fwd's t (update or load)
    long long acc_upd_r;            // history residuals read by plane_fwd (dynamic damping)
    long long acc_hist;             // history residuals read by plane_inv
    long long acc_anchor;           // iterations that read the anchor (plane_fwd and plane_inv)
    long long acc_refresh;          // iterations that wrote the anchor
    long long acc_shift;            // stored Y fields rewritten in the new offset on refresh
    long long acc_psi;              // iterations whose pencil pass read Psi
    double B[kMaxHist * kMaxHist];  // Gram matrix indexed by ring slot
    double anchor_ratio;            // re-anchor when the RMS has fallen by this factor
    unsigned long long deadline;    // device-loop solves: %globaltimer value past which the
                                    // loop stops (0 until the first loop test sets it)
};

template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 type; };
template <> struct Cx<double> { typedef double2 type; };

// Everything one iteration kernel needs, passed by value.
template <typename T>
struct Fields {
    typedef typename Cx<T>::type C;
    int nv, Nx, Ny, Nz, Kz;         // Kz = Nz / 2
    int M;                          // MDIIS ring capacity
    long long G;                    // Nx * Ny * Nz
    long long specN;                // Nx * Ny * Kz complex values per site (kz < Kz)
    T *bu;                          // [nv][G] beta * u (outputs and SFE)
    T *phi;                         // [G] long-range field phi (f_g = beta q_g phi)
    T *w;                           // [nv][G] f - beta*u + tau0; the iteration uses d = w + delta
    T *wref;                        // [nv][G] f - beta*u (w with tau0 = 0)
    C *psi, *psi_nyq;               // beta Phi~ / dV on [Nx][Ny][Kz] and the kz = Kz plane [Nx][Ny]
    C *spec, *spec_nyq;             // [nv][Nx][Ny][Kz], [nv][Nx][Ny]
    T *X, *R;                       // ring [M][nv][G]: X holds Y = tau + eta R, R the residual
    T *Tc;                          // [nv][G] the current iterate offset delta = tau - tau0
    T *tau0;                        // [nv][G] iterate offset: tau = t - f = tau0 + delta
    T *g_a, *h_a;                   // anchor fields [nv][G]: g and h at the anchor point
    C *phase;                       // per-atom axis phase tables [kPhaseChunk][Nx + Ny + Kz + 1]
    T *table;                       // [nk][nv + 1][nv]: X_ag / G and the charge row -Q_g / G
    int nk;
    double inv_dk;
    C *tw_x, *tw_y, *tw_h, *tw_z;   // exp(-2 pi i m / L) for L = Nx, Ny, Kz, Nz
    int half;                       // 1: half-integer k grid
    int split;                      // 1: split plane passes requested
    C *tw_q;                        // half grid: exp(-i pi (2m + 1) / Nz), m < Kz
    C *tw_ys, *tw_xs;               // half grid: exp(-i pi n / N) for N = Ny, Nx
    FftPlan px, py, ph;
    int chunk_rows, chunk_cols_fwd, chunk_x;   // batch chunk sizes of the in-place FFTs
    int pitch;                      // complex row pitch of a plane in shared memory
    int slab_rows, nyc;             // rows per plane block and row chunks per plane (1: whole)
    int cl;                         // > 1: the nyc row chunks of a plane form a thread-block
                                    // cluster that does the y transform (no y-pencil pass)
    FftPlan pys;                    // cluster y transform: local length slab_rows
    int chunk_ys;
    FastDiv dK1;                    // Kz + 1
    int Wy, ypitch, ytiles_main, ytiles_nyq, chunk_y;   // y-pencil pass (split planes only)
    int W;                          // columns per pencil tile
    int tiles_main, tiles_nyq;
    int pencil_pitch;
    FastDiv dKz, dKz1h, dKzp, dW, dNx, dWy, dNy;   // Kz, Kz/2 + 1, (Kz + 1)/2, W, Nx, Wy, Ny
    double bq[kMaxSites];           // beta * q_gamma
    double ks[3];                   // 2 pi / (N d) per axis
    double *partials;               // [kMaxHist + 1][nparts] (value-major)
    int nparts;                     // Gram partial sums per value (blocks that write them)
    Ctrl *ctrl;
};

// ---- launchers (explicitly instantiated for float and double) ----
// Sets the dynamic shared-memory limits of the iteration kernels; call before launching or
// capturing them.
template <typename T> cudaError_t prepare_kernels(const Fields<T> &f);
template <typename T> size_t plane_smem_bytes(const Fields<T> &f);
template <typename T> size_t pencil_smem_bytes(const Fields<T> &f);
template <typename T> cudaError_t launch_plane_fwd(const Fields<T> &f, cudaStream_t s);
template <typename T> cudaError_t launch_pencil(const Fields<T> &f, cudaStream_t s);
template <typename T> cudaError_t launch_plane_inv(const Fields<T> &f, cudaStream_t s);
template <typename T> cudaError_t launch_ypencil(const Fields<T> &f, int sign, cudaStream_t s);
template <typename T> cudaError_t launch_mdiis(const Fields<T> &f, cudaStream_t s);
// atoms: [n][8] doubles: x, y, z (absolute), q, sigma, eps, ux, uy, uz with u = (R - r0) / L
template <typename T>
cudaError_t launch_potential(const Fields<T> &f, const double *atoms, int n_atoms,
                             const double *site_sig, const double *site_eps, const double *site_q,
                             double beta, const double *origin, const double *spacing,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_longrange(const Fields<T> &f, const double *atoms, int n_atoms, double amp0,
                             cudaStream_t s);
template <typename T> cudaError_t launch_init_guess(const Fields<T> &f, int slot, cudaStream_t s);
template <typename T>
cudaError_t launch_guess_from_t(const Fields<T> &f, int slot, const double *src, cudaStream_t s);
// tau = tau0 + delta -> delta, tau0 = 0, w = wref (before a solve restarts from its iterate)
template <typename T> cudaError_t launch_flatten(const Fields<T> &f, cudaStream_t s);
// field: 1 g, 2 c, 3 h, 4 t, 5 beta u, 6 phi, 7 R
template <typename T>
cudaError_t launch_get_field(const Fields<T> &f, int field, int slot, int kind, int order,
                             double *dst, cudaStream_t s);
template <typename T>
cudaError_t launch_sfe(const Fields<T> &f, int slot, int kind, int order, int sfe_kind,
                       int sfe_order, double *partials, int blocks_per_site, cudaStream_t s);

// Message returned by rism3d_last_error(NULL) (thread-local).
void set_global_error(const char *msg);

// d(SFE)/dR of every atom (second Eq. 21); rho_dV[g] = rho_g dV (device); partials needs
// n_atoms * 3 * kGradBlocks doubles; out receives [n_atoms][3] (device).
// Learned-guess crops: mode 0 network input, 1 iterate of `slot` (both to out), 2 iterate of
// `slot` from `in` (zero outside the crop).
template <typename T>
cudaError_t launch_guess_crop(const Fields<T> &f, int mode, int slot, const int *corner, int n, float *out,
                              const float *in, cudaStream_t s);
// Split plane passes: which = 0 fwd_elem, 1 fft_fwd, 2 fft_inv, 3 inv_elem over x planes
// [x0, x1); inv_elem writes its Gram partials from slot part0.
template <typename T> bool split_planes(const Fields<T> &f);
template <typename T>
cudaError_t launch_split(const Fields<T> &f, int which, int x0, int x1, int part0, cudaStream_t s);
template <typename T>
cudaError_t launch_sfe_gradient(const Fields<T> &f, int slot, int kind, int order, const double *rho_dV,
                                const double *atoms, int n_atoms, const double *site_sig,
                                const double *site_eps, const double *site_q, const double *origin,
                                const double *spacing, double *partials, double *out, cudaStream_t s);

// Finite-size correction of a charged solute's SFE: phi is transformed into scratch (a
// complex [Nx][Ny][Nz] array), plans[0..2] are the axis transforms of lengths Nx, Ny, Nz;
// rq[g] = rho_g q_g (host); atoms [n][kAtomStride] (device); pairs [chunks][nq], lat_part
// [lat_blocks], int_part [int_blocks] (device, FP64).
template <typename T>
cudaError_t launch_lr_parts(const Fields<T> &f, typename Cx<T>::type *scratch, const FftPlan *plans,
                            const double *rq, const double *atoms, int n_atoms, double k_max, int nq, int chunks,
                            double *pairs, double *lat_part, int lat_blocks, double *int_part, int int_blocks,
                            double c4, double q2, cudaStream_t s);

constexpr int kSfeBlocksPerSite = 152;
constexpr int kGradBlocks = 304;
constexpr int kPhaseChunk = 256;  // atoms per long-range pass (phase-table capacity)
constexpr size_t kAtomStride = 9;

}  // namespace rism
