/*
 * rism3d.h - C ABI of the GB300 3D-RISM solver (RISMiCal, arXiv 2403.01039).
 *
 * The library solves the 3D-RISM equation h_g = sum_a c_a * X_ag (Eq. 13) closed by
 * KH (Eqs. 15-16, read as the Kovalenko-Hirata form), HNC (Eq. 14) or PSE-n, with the
 * long-range Coulomb split of Eqs. 29-32, by the fixed-point procedure of the
 * "Numerical procedure" section (steps 1-7) accelerated by MDIIS (Eq. 40), and reports
 * the solvation free energy (Eqs. 17-18, GF, PSE-n). Every step runs in the library's
 * own CUDA kernels on one GPU; the host side only validates, marshals and schedules.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: Angstrom, kcal/mol, elementary charges, Kelvin.
 * Grid: point (i, j, k) sits at origin + (i dx, j dy, k dz); fields are C-ordered
 *   [site][i][j][k] with k fastest. Nz must be even; Nx, Ny and Nz/2 must factor into
 *   2, 3 and 5.
 * Transform: c~(k) = dV sum_n c(r_n) exp(-i k.(r_n - r0)) on the periodic integer grid
 *   k_m = 2 pi m / (N d), m in [-N/2, N/2) (the paper does not fix a discrete convention).
 * Ownership: the library copies every input array during the call; the caller keeps its
 *   arrays. Outputs go to caller buffers. A context is owned by the library until
 *   rism3d_destroy.
 * Errors: every call returns a status; nothing throws across the ABI. After a failure
 *   rism3d_last_error(ctx) (or rism3d_last_error(NULL) when no context exists) gives a
 *   one-line message. RISM3D_ENOTCONV and RISM3D_EDIVERGED leave the last iterate readable.
 *   Common to every call: RISM3D_EINVAL for a NULL context or required pointer, an
 *   argument out of its stated range, or an output buffer smaller than stated;
 *   RISM3D_ESTATE for a call that needs a solute before rism3d_set_solute has succeeded;
 *   RISM3D_ECUDA when a CUDA runtime call fails (the message names it). Nothing is
 *   written to outputs when a call fails before its device work.
 * Threads: one context per host thread; every kernel of a context runs on its stream.
 * Pointers: "host" arrays are ordinary host memory; "device" arrays are device memory of
 *   the current CUDA device (for example a torch CUDA tensor's data_ptr()).
 */
#ifndef RISM3D_PUBLIC_API_H_
#define RISM3D_PUBLIC_API_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rism3d_ctx rism3d_ctx;

typedef enum {
    RISM3D_OK = 0,
    RISM3D_EINVAL = 1,      /* bad argument (size, pointer, non-positive rho or T, ...) */
    RISM3D_ENOMEM = 2,      /* device allocation failed or workspace too small */
    RISM3D_ECUDA = 3,       /* a CUDA runtime call failed */
    RISM3D_ESTATE = 4,      /* call out of order (e.g. solve before set_solute) */
    RISM3D_ENOTCONV = 5,    /* max_iter reached before the tolerance */
    RISM3D_EDIVERGED = 6,   /* a non-finite residual appeared */
    RISM3D_ETIMEOUT = 7,    /* a bounded device wait expired */
    RISM3D_EUNSUPPORTED = 8 /* grid or option outside what the kernels implement */
} rism3d_status;

/* Closures: KH (Eqs. 15-16, read g = exp(d) for d <= 0, 1 + d for d > 0), HNC (Eq. 14),
 * PSE-n (partial series expansion of order n; PSE-1 is KH). PSE-n and HNC are reached by
 * closure continuation: KH, PSE-2, ..., PSE-n (or KH, HNC), each stage started from the
 * previous solution and converged to 1e-4 (or the requested tolerance if looser), the last
 * stage to the requested tolerance. */
enum { RISM3D_KH = 1, RISM3D_HNC = 2, RISM3D_PSE = 3 };

/* SFE expressions: KH (Eq. 18), HNC (Eq. 17), GF (Gaussian fluctuation), PSE-n. */
enum { RISM3D_SFE_KH = 1, RISM3D_SFE_HNC = 2, RISM3D_SFE_GF = 3, RISM3D_SFE_PSE = 4 };

/* Fields readable with rism3d_get. G, H = g - 1 and C = h - t come from the closure of the
 * current iterate t; U is beta*u (Eq. 22); PHI is the shared long-range field
 * phi(r) = 332.0637 sum_a q_a (1 - exp(-r_a)) / r_a so that f_g = beta q_g phi (Eq. 29);
 * R is the residual t' - t of the last iteration (Eq. 33). */
enum { RISM3D_G = 1, RISM3D_C = 2, RISM3D_H = 3, RISM3D_T = 4, RISM3D_U = 5,
       RISM3D_PHI = 6, RISM3D_R = 7 };

typedef struct {
    int n_sites;              /* solvent sites n_v, 1..8 */
    const double *q;          /* [n_sites] partial charges (host) */
    const double *sigma;      /* [n_sites] LJ sigma (host) */
    const double *eps;        /* [n_sites] LJ epsilon (host) */
    const double *rho;        /* [n_sites] site number densities, > 0 (host) */
    double temperature;       /* > 0 */
    int n_k;                  /* >= 2 entries of the susceptibility table */
    double dk;                /* table spacing; entry j is at k = j * dk */
    const double *chi;        /* [n_sites][n_sites][n_k] X_ag(k_j) = omega_ag + rho_a h_ag
                                 (the solvent susceptibility defined under Eq. 8), host.
                                 Linearly interpolated in |k|; past the end the last entry
                                 is used. */
} rism3d_solvent;

typedef struct {
    int n[3];                 /* Nx, Ny, Nz */
    double spacing[3];        /* dx, dy, dz > 0 */
    double origin[3];         /* position of grid point (0, 0, 0) */
} rism3d_grid;

typedef struct {
    int precision;            /* 64: every step in FP64. 32: FFTs, contraction, closure and
                                 the stored fields in FP32; Gram matrix, MDIIS solve, SFE and
                                 the Coulomb/long-range sums accumulated in FP64. */
    int mdiis_nvec;           /* M, stored iterates, 1..16 (1 = damped Picard) */
    double mdiis_damp;        /* eta of t_new = sum c_i (t_i + eta R_i), in (0, 2] */
    int dynamic_damp;         /* 1: eta = clamp(-0.2 log10(RMS), 0.1, 1) (Modified DIIS
                                 passage, log base read as 10) */
    int max_iter;             /* iteration limit over all closure stages, >= 1 */
    int check_every;          /* iterations per CUDA-graph launch between status polls */
    int max_atoms;            /* capacity for rism3d_set_solute */
    int timing;               /* 1: record CUDA events around every kernel of the solve so
                                 rism3d_get_stats reports measured per-kernel device time;
                                 2: the same for the first iteration of each check_every
                                 chunk only (a sample with less recording overhead) */
    int accelerator;          /* 0: MDIIS (Eq. 40, mdiis_nvec vectors); 1: the modified
                                 Anderson method with two histories (Eqs. 34-39; Picard for
                                 the first two steps; mdiis_damp is its mixing b) */
    double anderson_s1;       /* Anderson shift s_1 (paper's value 0.2) */
    double anderson_s2;       /* Anderson shift s_2 (paper's value 0.0) */
    int slab_rows;            /* 0: whole y-z planes per block when they fit in shared memory,
                                 else row chunks plus a y-pencil pass (automatic); > 0 forces
                                 chunks of this many rows */
    int split_passes;         /* 1: run the plane passes as streaming element kernels and
                                 transform kernels on two graph branches (FP32, whole planes,
                                 Nz/2 of 64 or 128, integer k grid; otherwise ignored);
                                 0 (default): the fused plane kernels. Same results within
                                 rounding. */
    int kgrid;                /* 0: periodic integer k grid (the convention above); 1:
                                 half-integer grid k_m = 2 pi (m + 1/2) / (N d) on every axis
                                 (the placement of k in the "Numerical procedure" section): no
                                 k is zero, the transform carries the factor
                                 exp(-i pi sum_d n_d / N_d) and the fields are antiperiodic
                                 over the box */
    int ypencil_pass;         /* row-chunked planes only. 0 (default): when a plane's chunks
                                 number 2, 4 or 8 and split it evenly (integer k grid), they
                                 run as one thread-block cluster that does the y transform
                                 through distributed shared memory; 1: the y transform as a
                                 separate y-pencil pass over the spectrum. Same results
                                 within rounding. */
    double anchor_ratio;      /* the transform re-anchors (h = h_a + L(c^sr - c^sr_a), iterate
                                 offset moved to the current iterate) when the RMS first falls
                                 below 1e-2 and then whenever it has fallen by this factor
                                 since the last anchor; in (0, 1), default 0.1 (0 also
                                 selects it) */
    void *cuda_stream;        /* cudaStream_t to run on; NULL: the library creates one */
    void *workspace;          /* device buffer of >= rism3d_workspace_bytes bytes, 256-byte
                                 aligned, owned by the caller and kept alive until
                                 rism3d_destroy; NULL: the library allocates it */
    size_t workspace_bytes;
} rism3d_options;

typedef struct {
    int iterations;           /* iterations over all closure stages */
    int converged;            /* 1 if the final stage reached the tolerance */
    double rms_residual;      /* RMS of R = t' - t of the last iteration, read of Eq. 41 */
    double seconds_iter;      /* wall time of the solve call */
} rism3d_report;

/* Per-kernel counters of a context, accumulated since creation or the last
 * rism3d_reset_stats. Kernel index: 0 plane_fwd (MDIIS update + closure + forward z/y FFT),
 * 1 pencil (x FFT + Eq. 13 contraction + inverse x FFT), 2 plane_inv (inverse y/z FFT +
 * residual + Gram partials), 3 mdiis (Gram reduction + bordered solve), 4 potential
 * (Eqs. 22, 29), 5 long_range (Eq. 30), 6 sfe, 7 other (guess, conversions, field output),
 * 8 and 9 the forward and inverse y-pencil passes (planes split into row chunks only),
 * 10-13 the split form of the plane passes (FP32, whole planes, Nz/2 of 64 or 128): 10
 * fwd_elem (update + closure), 11 fft_fwd (forward z/y FFT), 12 fft_inv (inverse y/z FFT),
 * 13 inv_elem (residual + Gram partials), each launched for two halves of the x planes. */
#define RISM3D_N_KERNELS 14
typedef struct {
    long long launches[RISM3D_N_KERNELS];   /* kernels launched (including ones that found the
                                               solve finished and returned at once) */
    long long timed[RISM3D_N_KERNELS];      /* launches that did work and were timed */
    double ms[RISM3D_N_KERNELS];            /* summed CUDA-event time of the timed launches */
    double bytes[RISM3D_N_KERNELS];         /* algorithmic HBM bytes of the launches that did
                                               work (the byte model of the kernel's docs) */
    long long iterations;
    long long solves;
} rism3d_stats;

/* Library version string, static storage. */
const char *rism3d_version(void);

/* Fill *opt with the defaults: precision 32, MDIIS with M = 5, eta = 0.7, static damping,
 * max_iter 10000, check_every 8, max_atoms 100000, timing off, Anderson shifts 0.2 / 0.0,
 * NULL stream and workspace. */
void rism3d_options_default(rism3d_options *opt);

/* Bytes of device workspace a context with these inputs needs. EINVAL on bad input,
 * EUNSUPPORTED if the grid cannot be handled. */
rism3d_status rism3d_workspace_bytes(const rism3d_solvent *solvent, const rism3d_grid *grid,
                                     const rism3d_options *opt, size_t *bytes);

/* Create a context for one solvent and one grid (the solvent's 1D part is computed once
 * per solvent and reused, Package Features section). Copies the susceptibility table to
 * the device as the interpolation table of Eq. 13. On success *out is a new context, else
 * *out is NULL: EINVAL (bad solvent, grid or options), EUNSUPPORTED (a grid the kernels do
 * not implement), ENOMEM (a caller workspace smaller than rism3d_workspace_bytes, or the
 * device allocation failed). */
rism3d_status rism3d_create(const rism3d_solvent *solvent, const rism3d_grid *grid,
                            const rism3d_options *opt, rism3d_ctx **out);

/* Set the solute (the paper's "initialization"): builds beta*u_g (Eq. 22, Lorentz-Berthelot
 * mixing, r^2 floored at 1e-8 A^2, beta*u capped above at 1e4), the long-range field phi
 * (Eq. 29) and its analytic transform (Eq. 30, zero at k = 0 and on Nyquist planes), and
 * sets the initial guess t = f (step 1). xyz is [n_atoms][3], q/sigma/eps are [n_atoms],
 * all host arrays. 1 <= n_atoms <= max_atoms. EINVAL (a bad count, a null array, a
 * non-finite position or charge, a negative sigma or eps) leaves the previous solute in
 * place; a CUDA error after the checks leaves the context without a solute (ESTATE from
 * the calls that need one until a later rism3d_set_solute succeeds). */
rism3d_status rism3d_set_solute(rism3d_ctx *ctx, int n_atoms, const double *xyz,
                                const double *q, const double *sigma, const double *eps);

/* Replace the initial guess of step 1 (t = f) by a caller field t [n_sites][Nx][Ny][Nz]
 * of FP64, host memory (on_device = 0) or device memory (on_device = 1), for a warm start.
 * The next rism3d_solve starts from it with an empty MDIIS history. */
rism3d_status rism3d_set_guess(rism3d_ctx *ctx, const double *t, int on_device);

/* Run steps 2-7 from the current guess until RMS(R) < tol (read of Eq. 41), max_iter, or a
 * non-finite residual. closure is RISM3D_KH / RISM3D_HNC / RISM3D_PSE, pse_order >= 1 for
 * PSE. Returns OK, ENOTCONV or EDIVERGED (the report is filled in every case), or an
 * error. The converged iterate replaces the guess, so a second call continues from it. */
rism3d_status rism3d_solve(rism3d_ctx *ctx, int closure, int pse_order, double tol,
                           rism3d_report *report);

/* One application of steps 2-5 to a caller field t (FP64, [n_sites][Nx][Ny][Nz]):
 * writes R = t' - t = h + 1 - g (Eq. 33) into R. Both arrays host or both device
 * (on_device). Overwrites the context's iterate and history. */
rism3d_status rism3d_residual(rism3d_ctx *ctx, int closure, int pse_order, const double *t,
                              double *R, int on_device);

/* Copy one field (see RISM3D_G ...) of every site, converted to FP64, into dst
 * ([n_sites][Nx][Ny][Nz], or [Nx][Ny][Nz] for PHI; host or device memory by on_device).
 * count is the capacity of dst in elements (EINVAL when smaller than the field). G, H and
 * C use the closure of the last solve (KH before any solve), Eqs. 14-16 and 31. */
rism3d_status rism3d_get(rism3d_ctx *ctx, int field, double *dst, size_t count, int on_device);

/* Solvation free energy in kcal/mol of the current iterate: k_B T sum_g rho_g dV
 * sum_grid (integrand of kind), Eqs. 17-18, GF and PSE-n (pse_order >= 1). Accumulated in
 * FP64. per_site ([n_sites], host) may be NULL. */
rism3d_status rism3d_get_sfe(rism3d_ctx *ctx, int kind, int pse_order, double *total,
                             double *per_site);

/* Learned initial guess (next row of the method; the paper starts every solve from t = f):
 * crops of side `crop` at grid index corner[3] (inside the grid, else EINVAL), FP32 device
 * arrays of exactly n_sites * crop^3 values [n_sites][crop][crop][crop], for the network
 * of unet3d.h. */
/* Network input: tanh(beta u_g / 4) on the crop (after rism3d_set_solute). */
rism3d_status rism3d_guess_input(rism3d_ctx *ctx, const int *corner, int crop, float *x);
/* Training target: the current iterate tau = t - f on the crop (after a solve). */
rism3d_status rism3d_guess_target(rism3d_ctx *ctx, const int *corner, int crop, float *tau);
/* Start the next rism3d_solve from tau = the given values on the crop and 0 elsewhere
 * (step 1 otherwise uses tau = 0, i.e. t = f). */
rism3d_status rism3d_set_guess_crop(rism3d_ctx *ctx, const int *corner, int crop, const float *tau);

/* One job of rism3d_solve_batch. Inputs: ctx (a context of its own; the grid may differ from
 * job to job; jobs run concurrently when their contexts have different streams and in turn
 * when they share one), an optional solute (n_atoms > 0: set with
 * rism3d_set_solute when the job starts; 0: keep the context's current solute), the closure,
 * PSE order and tolerance as for rism3d_solve, and sfe_kind (0 = none, else as
 * rism3d_get_sfe, evaluated when the solve ends). Outputs: report, sfe (kcal/mol) and the
 * job's status. */
typedef struct {
    rism3d_ctx *ctx;
    int n_atoms;
    const double *xyz, *q, *sigma, *eps;   /* host, as rism3d_set_solute */
    int closure, pse_order;
    double tol;
    int sfe_kind;
    rism3d_report report;     /* out */
    double sfe;               /* out */
    rism3d_status status;     /* out */
} rism3d_batch_job;

/* Solve many independent problems concurrently on one GPU (next row of the method: the
 * batched form for many solutes on uneven grids; the paper solves one problem at a time).
 * A host scheduler keeps up to max_inflight jobs in flight, each advancing check_every
 * iterations per graph launch on its own stream, and starts the next job as soon as one
 * ends, so small grids that cannot fill the GPU alone share it. Each job computes exactly
 * what rism3d_solve would (bit-identical results). time_limit_s > 0 bounds each job's wall
 * time: a job still running past it is stopped after its current chunk and reports
 * RISM3D_ETIMEOUT with its last iterate readable; 0 means no limit. Returns RISM3D_OK when
 * every job succeeded, else the first failing job's status (each job's own is in its
 * record); RISM3D_EINVAL for a bad list (a context in two jobs, several devices). */
rism3d_status rism3d_solve_batch(rism3d_batch_job *jobs, int n_jobs, int max_inflight,
                                 double time_limit_s);

/* The same jobs as rism3d_solve_batch as ONE launch of one CUDA graph (no counterpart in the
 * paper; the batched form for many solutes on uneven grids): each job is a device-side loop
 * (a conditional while node) whose body runs the job's check_every iterations and a loop
 * test that keeps the loop going while the job's device control block says "running", so
 * no host round trip happens between iterations and the jobs' loops run side by side on the
 * GPU. Set-up (solute, control block, capture of every job's loop) runs on the host before
 * the launch; the call returns when the graph has finished. time_limit_s > 0 bounds each
 * job on the device: the loop test compares the GPU's global timer with the job's deadline
 * (set by its first loop test) and stops the job, which reports RISM3D_ETIMEOUT with its
 * last iterate readable; 0 means no limit. Results are those of rism3d_solve (the same
 * kernels in the same order). Status as rism3d_solve_batch. */
rism3d_status rism3d_solve_batch_graph(rism3d_batch_job *jobs, int n_jobs, double time_limit_s);

/* Partial molar volume of Eq. 19, V = k_B T chi_T (1 - sum_g rho_g int c_g(r) dr), in A^3 per
 * molecule, from the current iterate; kT_chi_T (A^3) is the solvent's k_B T times its
 * isothermal compressibility (rism1d_xrism_ex reports it). c_integral ([n_sites], host) may
 * be NULL; it receives int c_g(r) dr as grid sums. The pressure correction of Eq. 21 is
 * -P * V with the bulk pressure P of Eq. 20 (rism1d_xrism_ex). */
rism3d_status rism3d_get_pmv(rism3d_ctx *ctx, double kT_chi_T, double *pmv, double *c_integral);

/* Finite-size error of the SFE of a charged solute on the periodic grid (next row of the
 * method: thermodynamics; the paper evaluates Eqs. 17-18 as box sums and gives no
 * correction). The long-range field of Eq. 30 has no k = 0 term, so the box holds the
 * solvent's response only at the lattice wave vectors; at long range that response is
 * linear, with the solvent's charge response S(k) = sum_{a,g} q_a X_ag(k) rho_g q_g. delta
 * (kcal/mol) is half the energy of that response in the solute's Eq. 29 potential on the
 * box minus the same energy in infinite space:
 *   delta = -(beta / 2) [ (1/V) sum_{k != 0} Re(Phi~(k) conj(phi~_box(k))) S(|k|)
 *                        - int d^3k / (2 pi)^3 |Phi~(k)|^2 S(|k|) ],
 * Phi~ the Eq. 30 field (without beta q_g), phi~_box the DFT of the grid field phi times dV,
 * the integral in its orientation-averaged radial form (pair sums over the atoms,
 * trapezoidal rule on [0, 20] 1/A, 16385 points); S below the first table point is
 * continued as S(k_1) (k / k_1)^2. The infinite-dilution SFE is rism3d_get_sfe's total minus
 * delta (delta grows as Q^2 / L for net charge Q and box side L; about 0.8 x the Ewald-Wigner
 * value for a cation in water). Depends on the solute and solvent only; uses the spectrum
 * buffer as scratch (no state a later solve or rism3d_get needs) and allocates 8.4 MB of
 * partial sums on the first call. Cost: O(N^3 log N) plus O(n_atoms^2) pair sums (about 0.2 s
 * for 2000 atoms). EUNSUPPORTED on the half-integer grid or with one solvent site. */
rism3d_status rism3d_get_sfe_finite_size(rism3d_ctx *ctx, double *delta);

/* Derivative of the SFE with respect to every solute atom position (the second "Eq. 21",
 * Hybrid implementation section): grad[a][k] = sum_g rho_g dV sum_grid g_g(r) du_g(r)/dR_a,k
 * in kcal/mol/A, with du/dR the analytic derivative of Eq. 22's pair terms (Lorentz-Berthelot
 * mixing, r^2 floored at 1e-8 A^2). grad is host [n_atoms][3]. For a neutral solute this is the
 * exact derivative of the KH/HNC SFE on the grid; for a charged one it omits the dependence of
 * the long-range split (Eqs. 29-30) on the atom positions. EUNSUPPORTED when the grid is too
 * small to hold the FP64 partial sums of one atom (n_sites * Nx * Ny * Nz below 915). */
rism3d_status rism3d_get_sfe_gradient(rism3d_ctx *ctx, double *grad);

/* Autotune the transform tiles of this context by measurement: the x-pencil pass (x
 * transforms, contraction of Eq. 13, inverse x transforms) is timed on the context's own
 * buffers for every tile width W = 1, 2, 4, ... columns that fits in shared memory, and the
 * fastest W is kept for later solves (results do not depend on W). Call after
 * rism3d_set_solute and outside a solve; it overwrites the spectrum buffer (no state a
 * later solve needs). pencil_width and pencil_ms (time of one pass at the chosen W) may be
 * NULL. No counterpart in the paper. */
rism3d_status rism3d_tune(rism3d_ctx *ctx, int *pencil_width, double *pencil_ms);

/* Autotune the plane-pass tile before creating a context (no counterpart in the paper):
 * for each row-chunk shape the grid admits - whole y-z planes or automatic chunks
 * (slab_rows = 0), and chunks of Ny/2, Ny/4 and Ny/8 rows, each as a thread-block cluster
 * that does the y transform (ypencil_pass = 0) and with the separate y-pencil pass (1) - a
 * context is created with opt's other options, given a neutral LJ sphere at the grid centre,
 * and timed over `iters` iterations (after a first solve that captures its graph). *best
 * receives opt with the fastest slab_rows and ypencil_pass; ms_per_iter (may be NULL) its
 * time per iteration. Shapes that cannot be created (shared memory, cluster limits) are
 * skipped. Every candidate allocates and frees its own workspace, so the call needs the
 * memory of one context at a time. Results of solves do not depend on the shape beyond
 * rounding. EINVAL for bad arguments or iters < 2; EUNSUPPORTED when no shape works. */
rism3d_status rism3d_tune_planes(const rism3d_solvent *solvent, const rism3d_grid *grid, const rism3d_options *opt,
                                 int iters, rism3d_options *best, double *ms_per_iter);

/* Copy the counters; timing fields are zero unless the context was created with timing = 1. */
rism3d_status rism3d_get_stats(const rism3d_ctx *ctx, rism3d_stats *out);

/* Zero the counters. */
rism3d_status rism3d_reset_stats(rism3d_ctx *ctx);

/* Solvation free energy (same integrands as rism3d_get_sfe) from caller fields, without
 * allocating device memory. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate - a host framework that owns every device allocation (a
 * memory pool holding the whole device), or a latency-critical loop in which cudaMalloc
 * or cudaFree would synchronise the device - and needs no context. h, c and (for
 * RISM3D_SFE_PSE only, else may be NULL) d = -beta u + t are arrays [n_sites][n_points] of
 * FP64 in device (or managed) memory of the current device, checked before any launch:
 * other pointers give RISM3D_EINVAL. rho is host [n_sites]; per_site (host [n_sites]) may
 * be NULL. Runs on cuda_stream (NULL = default stream) and synchronises that stream before
 * it returns. Its scratch is a static device array of 8 x 152 + 8 doubles that every GPU
 * that loads the library keeps until the process exits: n_sites above 8 is rejected with
 * RISM3D_EINVAL. The first call on each device looks up that array's device address, so
 * make it before any stream capture. Every call shares the array (each call rewrites all it
 * reads, so nothing needs clearing); calls that overlap on the GPU race on it. Launch
 * failures give RISM3D_ECUDA before anything is copied back. */
rism3d_status rism3d_sfe_noalloc(int n_sites, long long n_points, const double *h, const double *c,
                                 const double *d, const double *rho, double temperature, double dV,
                                 int kind, int pse_order, double *total, double *per_site,
                                 void *cuda_stream);

/* FP32 (precision 32) or FP64 (64) fused multiply-add throughput of the current device in
 * flop/s (2 per FMA), measured with CUDA events around a kernel of independent FMA chains
 * on every SM (best of five runs). A measurement of the machine for the roofline of the
 * arithmetic-bound FP64 form, not part of the method: the paper has no counterpart.
 * RISM3D_EINVAL for another precision or a NULL pointer, RISM3D_ECUDA on a CUDA error. */
rism3d_status rism3d_fma_rate(int precision, double *flops_per_s);

/* Message of the last failure on ctx (or of the last failed create when ctx is NULL). */
const char *rism3d_last_error(const rism3d_ctx *ctx);

/* Free the context and everything the library allocated for it. NULL is accepted. */
void rism3d_destroy(rism3d_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* RISM3D_PUBLIC_API_H_ */
