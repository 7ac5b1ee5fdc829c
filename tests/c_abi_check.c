/*
 * A plain C99 client of the library (compiled with gcc -std=c99 -pedantic -Werror and run by
 * test_c_abi.py on any host, no GPU needed). It shows that the declarations of
 * include/rism3d.h, rism1d.h and unet3d.h are C, that the library links from C, and that
 * the calls which need no device behave as declared: option defaults, workspace sizes, the
 * solvent preparation of Eq. 4 (host code), and argument validation.
 * Prints one line per check group and "OK" at the end; exit status 0 on success.
 */
#include "rism1d.h"
#include "rism3d.h"
#include "unet3d.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>

static int failures = 0;

#define CHECK(cond)                                                           \
    do {                                                                      \
        if (!(cond)) {                                                        \
            printf("FAIL line %d: %s\n", __LINE__, #cond);                    \
            ++failures;                                                       \
        }                                                                     \
    } while (0)

int main(void) {
    /* 3-site water: O, H1, H2 (OH 1.0 A, HOH 109.47 deg), one molecule species */
    const double q[3] = {-0.8476, 0.4238, 0.4238};
    const double sigma[3] = {3.166, 1.0, 1.0};
    const double eps[3] = {0.1553, 0.046, 0.046};
    const double rho[3] = {0.0334, 0.0334, 0.0334};
    const int species[3] = {0, 0, 0};
    const double coords[9] = {0.0, 0.0, 0.0, 1.0, 0.0, 0.0, -0.33331324756823727, 0.9428161427317179, 0.0};
    const double pi = 3.14159265358979323846;

    printf("version %s\n", rism3d_version());

    /* 1. solvent susceptibility from the host 1D solver (Eq. 4) */
    rism1d_solvent s1;
    s1.n_sites = 3;
    s1.q = q;
    s1.sigma = sigma;
    s1.eps = eps;
    s1.rho = rho;
    s1.species = species;
    s1.coords = coords;
    s1.temperature = 298.15;
    rism1d_options o1;
    rism1d_options_default(&o1);
    o1.n_r = 1024;
    o1.tol = 1e-8;
    double *chi = (double *)malloc(sizeof(double) * 9 * (size_t)o1.n_r);
    double dk = 0.0, rms = 1.0;
    int its = 0;
    rism1d_status st1 = rism1d_xrism(&s1, &o1, chi, &dk, &its, &rms);
    CHECK(st1 == RISM1D_OK);
    CHECK(rms < 1e-8 && its > 0);
    CHECK(fabs(dk - pi / (o1.n_r * o1.dr)) < 1e-15);
    {
        /* equal densities within the molecule: X = omega + rho h is symmetric, and the two
           hydrogens are interchangeable */
        double asym = 0.0, hh = 0.0;
        for (int j = 0; j < o1.n_r; ++j) {
            asym = fmax(asym, fabs(chi[(0 * 3 + 1) * o1.n_r + j] - chi[(1 * 3 + 0) * o1.n_r + j]));
            hh = fmax(hh, fabs(chi[(0 * 3 + 1) * o1.n_r + j] - chi[(0 * 3 + 2) * o1.n_r + j]));
        }
        CHECK(asym < 1e-9 && hh < 1e-9);
        CHECK(chi[0] > 0.0);              /* X_OO(0) = S_OO(0) > 0 */
    }
    printf("rism1d: %d iterations, rms %.2e\n", its, rms);
    s1.n_sites = 0;
    CHECK(rism1d_xrism(&s1, &o1, chi, &dk, NULL, NULL) == RISM1D_EINVAL);
    CHECK(rism1d_last_error() != NULL);
    s1.n_sites = 3;

    /* 2. options and workspace sizes of a 3D context (host arithmetic only) */
    rism3d_options opt;
    rism3d_options_default(&opt);
    CHECK(opt.precision == 32 && opt.mdiis_nvec == 5 && fabs(opt.mdiis_damp - 0.7) < 1e-15);
    rism3d_solvent s3;
    s3.n_sites = 3;
    s3.q = q;
    s3.sigma = sigma;
    s3.eps = eps;
    s3.rho = rho;
    s3.temperature = 298.15;
    s3.n_k = o1.n_r;
    s3.dk = dk;
    s3.chi = chi;
    rism3d_grid grid = {{32, 32, 32}, {0.5, 0.5, 0.5}, {-8.0, -8.0, -8.0}};
    size_t b32 = 0, b64 = 0;
    CHECK(rism3d_workspace_bytes(&s3, &grid, &opt, &b32) == RISM3D_OK);
    opt.precision = 64;
    CHECK(rism3d_workspace_bytes(&s3, &grid, &opt, &b64) == RISM3D_OK);
    CHECK(b32 > 0 && b32 < b64);
    /* at least beta*u, 2M history fields and the staging field per site-point */
    CHECK(b64 >= (size_t)3 * 32 * 32 * 32 * 8 * (1 + 2 * 5 + 1));
    printf("workspace: %zu B (FP32), %zu B (FP64)\n", b32, b64);

    /* 3. validation before any device work */
    const double bad_rho[3] = {0.0334, -1.0, 0.0334};
    s3.rho = bad_rho;
    size_t b = 0;
    CHECK(rism3d_workspace_bytes(&s3, &grid, &opt, &b) == RISM3D_EINVAL);
    s3.rho = rho;
    grid.n[2] = 31;                       /* odd Nz: no real-to-complex half spectrum */
    CHECK(rism3d_workspace_bytes(&s3, &grid, &opt, &b) == RISM3D_EUNSUPPORTED);
    grid.n[2] = 32;
    rism3d_report rep;
    CHECK(rism3d_solve(NULL, RISM3D_KH, 1, 1e-6, &rep) == RISM3D_EINVAL);
    CHECK(rism3d_set_solute(NULL, 1, q, q, q, q) == RISM3D_EINVAL);
    CHECK(rism3d_last_error(NULL) != NULL);
    CHECK(rism3d_create(&s3, &grid, &opt, NULL) == RISM3D_EINVAL);
    unet3d *net = NULL;
    CHECK(unet3d_create(5, 5, 6, 16, 32, 64, NULL, &net) == 1 && net == NULL);   /* crop % 4 */
    CHECK(unet3d_param_count(NULL) == 0);
    printf("validation checked\n");

    free(chi);
    printf("%s\n", failures ? "FAILED" : "OK");
    return failures != 0;
}
