/*
 * rism1d.h - solvent preparation for the 3D-RISM solver: the 1D RISM equation of a pure
 * (multi-component) molecular solvent, Eq. 4 of RISMiCal (arXiv 2403.01039), whose solution
 * gives the solvent susceptibility X_ag = omega_ag + rho_a h_ag defined under Eq. 8. The
 * paper computes it once per solvent and reuses it (Package Features section); this is
 * host code (small radial problem, run once), not part of the GPU hot path.
 *
 * Readings (the paper defers the 1D method to Kinoshita and is silent on details):
 *  - radial grid r_i = i dr, k_j = j dk with dk = pi / (n_r dr), i, j = 1..n_r-1, and the
 *    radial transform pair F(k) = (4 pi dr / k) sum_i r_i f(r_i) sin(k r_i),
 *    f(r) = (dk / (2 pi^2 r)) sum_j k_j F(k_j) sin(k_j r), evaluated with a radix-2 FFT
 *    (n_r must be a power of two);
 *  - pair potential: LJ (Lorentz-Berthelot mixing) + 332.0637 q_a q_b / r; the Coulomb long
 *    range split with the function of Eq. 29, u_L = 332.0637 q_a q_b (1 - e^{-r}) / r, whose
 *    transform 4 pi 332.0637 q_a q_b / (k^2 (k^2 + 1)) is Eq. 30; the closure acts on
 *    d = -beta u_s + tau with tau = h - c_s, c = c_s - beta u_L;
 *  - omega_ab(k) = sin(k l_ab) / (k l_ab) within a molecule (species), 1 on the diagonal,
 *    0 between molecules;
 *  - X_ab(0) = omega_ab(0) + rho_a 4 pi dr sum_i r_i^2 h_ab(r_i);
 *  - MDIIS (Eq. 40 read as the bordered DIIS system) with the charges switched on in
 *    charge_steps equal steps, each solve starting from the previous tau;
 *  - DRISM (option dielectric > 0; the dielectrically consistent RISM of Perkyns and
 *    Pettitt): the equation above is solved with omega' = omega + rho zeta in place of
 *    omega for h' = h - zeta, the physical h being h' + zeta, so X = omega' + rho h'.
 *    zeta_ab(k) = d_a d_b h_c(k) couples the sites of molecules with a dipole:
 *    d_a = j0(k x_a) j0(k y_a) j1(k z_a), (x, y, z) the site in its molecule's frame
 *    (origin at the centroid of the molecule's sites, z along the dipole, x along the
 *    component normal to z of the site farthest from the z axis, the first on a tie,
 *    y = z cross x), h_c(k) = h_c0 exp(-a^2 k^2 / 4) with a = drism_damping and
 *    h_c0 = (dielectric - 1 - 3 y) / sum_s rho_s y_s, y_s = 4 pi beta 332.0637 rho_s mu_s^2 / 9
 *    per polar species s and y = sum_s y_s. This amplitude makes the k -> 0 limit of
 *    4 pi beta S_qq(k) / k^2 equal 1 - 1/dielectric (XRISM gives 3y / (1 + 3y)).
 * Errors: every call returns a status (0 = OK, see rism1d_status); rism1d_last_error() gives
 * a one-line message for the calling thread. All arrays are host memory owned by the caller.
 */
#ifndef RISM1D_PUBLIC_API_H_
#define RISM1D_PUBLIC_API_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RISM1D_OK = 0,
    RISM1D_EINVAL = 1,     /* bad argument */
    RISM1D_ENOTCONV = 2,   /* max_iter reached in some charge step (chi is still written) */
    RISM1D_EDIVERGED = 3   /* a non-finite residual appeared */
} rism1d_status;

typedef struct {
    int n_sites;             /* 1..16 */
    const double *q;         /* [n_sites] charges (e) */
    const double *sigma;     /* [n_sites] LJ sigma (Angstrom) */
    const double *eps;       /* [n_sites] LJ epsilon (kcal/mol) */
    const double *rho;       /* [n_sites] site number density (1/A^3), > 0; equal within a
                                molecule */
    const int *species;      /* [n_sites] molecule index of each site */
    const double *coords;    /* [n_sites][3] site positions inside their molecule (A) */
    double temperature;      /* K */
} rism1d_solvent;

typedef struct {
    int n_r;                 /* radial points, power of two (default 2048) */
    double dr;               /* radial spacing (default 0.05 A) */
    int closure;             /* 1 KH (default), 2 HNC */
    double tol;              /* RMS residual tolerance per charge step (default 1e-10) */
    int max_iter;            /* per charge step (default 5000) */
    int mdiis_nvec;          /* default 5 */
    double mdiis_damp;       /* default 0.3 */
    int charge_steps;        /* default 10 */
    double dielectric;       /* 0 (default): XRISM; > 0: DRISM with this dielectric constant,
                                which must exceed 1 + 3y (the XRISM value); needs a solvent
                                molecule with a dipole */
    double drism_damping;    /* DRISM damping length a (A), > 0 (default 1.0) */
} rism1d_options;

void rism1d_options_default(rism1d_options *opt);

/* Solve Eq. 4 and write chi[a][b][j] = X_ab(j dk), j = 0..n_r-1 ([n_sites][n_sites][n_r]),
 * *dk = pi / (n_r dr). iterations (total) and rms (last) may be NULL. */
rism1d_status rism1d_xrism(const rism1d_solvent *solvent, const rism1d_options *opt, double *chi,
                           double *dk, int *iterations, double *rms);

/* As rism1d_xrism, and also (each may be NULL): c_r ([n_sites][n_sites][n_r - 1], the full
 * direct correlation c = c_s - beta u_L at r_i = i dr, i = 1..n_r-1), the bulk pressure of
 * Eq. 20, P = sum_G rho_G (n_G + 1) k_B T / 2 - 2 pi k_B T sum_ab rho_a rho_b int c_ab r^2 dr
 * (kcal/mol/A^3; G runs over species, n_G their site counts), and k_B T chi_T = X_00(0) / rho_0
 * (A^3; the structure factor of the first site, the molecular centre for water). */
rism1d_status rism1d_xrism_ex(const rism1d_solvent *solvent, const rism1d_options *opt, double *chi,
                              double *dk, double *c_r, double *pressure, double *kT_chi_T,
                              int *iterations, double *rms);

const char *rism1d_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RISM1D_PUBLIC_API_H_ */
