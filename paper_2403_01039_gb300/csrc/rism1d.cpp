// Solvent preparation: 1D XRISM for a pure molecular solvent (Eq. 4) giving the solvent
// susceptibility X_ag = omega_ag + rho_a h_ag (defined under Eq. 8), the input table of the
// 3D-RISM solve. Host code: a radial problem of n_r points solved once per solvent.
// Conventions and readings are listed in include/rism1d.h.
#include "rism1d.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

namespace {

constexpr double kKB = 0.0019872041;    // kcal / (mol K)
constexpr double kCoulomb = 332.0637;   // kcal A / (mol e^2)
constexpr double kPi = 3.14159265358979323846;
constexpr double kCap = 1.0e4;          // cap of beta*u
constexpr double kPivotMin = 1.0e-12;

thread_local std::string g_err;

rism1d_status fail(rism1d_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

typedef std::complex<double> cd;

// Sine transform S_j = sum_{i=1}^{N-1} f_i sin(pi i j / N), j = 1..N-1, through a complex FFT of
// length 2N of the odd extension (x_i = f_i, x_{2N-i} = -f_i): X_j = -2 i S_j.
class SineTransform {
  public:
    explicit SineTransform(int N) : N_(N), L_(2 * N), buf_(2 * N) {
        tw_.resize(L_ / 2);
        for (int m = 0; m < L_ / 2; ++m) tw_[m] = std::polar(1.0, -2.0 * kPi * m / L_);
    }
    void run(const double *f, double *S) {
        std::fill(buf_.begin(), buf_.end(), cd(0.0, 0.0));
        for (int i = 1; i < N_; ++i) {
            buf_[i] = f[i - 1];
            buf_[L_ - i] = -f[i - 1];
        }
        fft();
        for (int j = 1; j < N_; ++j) S[j - 1] = -0.5 * buf_[j].imag();
    }

  private:
    void fft() {   // iterative radix-2, forward sign
        const int n = L_;
        for (int i = 1, j = 0; i < n; ++i) {
            int bit = n >> 1;
            for (; j & bit; bit >>= 1) j ^= bit;
            j ^= bit;
            if (i < j) std::swap(buf_[i], buf_[j]);
        }
        // butterflies in real arithmetic: the same products as the complex operator for
        // finite values, without its inf/nan recovery path
        double *z = reinterpret_cast<double *>(buf_.data());
        const double *w = reinterpret_cast<const double *>(tw_.data());
        for (int len = 2; len <= n; len <<= 1) {
            const int half = len / 2, stride = n / len;
            for (int i = 0; i < n; i += len)
                for (int k = 0; k < half; ++k) {
                    double *pu = z + 2 * (i + k), *pv = z + 2 * (i + k + half);
                    const double wr = w[2 * k * stride], wi = w[2 * k * stride + 1];
                    const double vr = pv[0] * wr - pv[1] * wi, vi = pv[0] * wi + pv[1] * wr;
                    const double ur = pu[0], ui = pu[1];
                    pu[0] = ur + vr;
                    pu[1] = ui + vi;
                    pv[0] = ur - vr;
                    pv[1] = ui - vi;
                }
        }
    }
    int N_, L_;
    std::vector<cd> buf_, tw_;
};

// Solve A x = b (dense n x n, row-major) by Gaussian elimination with partial pivoting.
bool gauss(std::vector<double> &A, std::vector<double> &b, int n, double pivot_min) {
    for (int col = 0; col < n; ++col) {
        int p = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[r * n + col]) > std::fabs(A[p * n + col])) p = r;
        if (std::fabs(A[p * n + col]) < pivot_min) return false;
        if (p != col) {
            for (int j = 0; j < n; ++j) std::swap(A[col * n + j], A[p * n + j]);
            std::swap(b[col], b[p]);
        }
        for (int r = col + 1; r < n; ++r) {
            const double f = A[r * n + col] / A[col * n + col];
            for (int j = col; j < n; ++j) A[r * n + j] -= f * A[col * n + j];
            b[r] -= f * b[col];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * b[j];
        b[r] = s / A[r * n + r];
    }
    return true;
}

// Same linear system with several right-hand sides (columns of B, n x m row-major).
bool gauss_multi(std::vector<double> &A, std::vector<double> &B, int n, int m) {
    for (int col = 0; col < n; ++col) {
        int p = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[r * n + col]) > std::fabs(A[p * n + col])) p = r;
        if (A[p * n + col] == 0.0) return false;
        if (p != col) {
            for (int j = 0; j < n; ++j) std::swap(A[col * n + j], A[p * n + j]);
            for (int j = 0; j < m; ++j) std::swap(B[col * m + j], B[p * m + j]);
        }
        for (int r = col + 1; r < n; ++r) {
            const double f = A[r * n + col] / A[col * n + col];
            for (int j = col; j < n; ++j) A[r * n + j] -= f * A[col * n + j];
            for (int j = 0; j < m; ++j) B[r * m + j] -= f * B[col * m + j];
        }
    }
    for (int r = n - 1; r >= 0; --r)
        for (int j = 0; j < m; ++j) {
            double s = B[r * m + j];
            for (int c = r + 1; c < n; ++c) s -= A[r * n + c] * B[c * m + j];
            B[r * m + j] = s / A[r * n + r];
        }
    return true;
}

double sph_j0(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }
double sph_j1(double x) { return x == 0.0 ? 0.0 : std::sin(x) / (x * x) - std::cos(x) / x; }

// DRISM zeta_ab(k_j) (header), written into Z [n][n][P]; false when no molecule has a
// dipole or the dielectric constant is not above the XRISM value 1 + 3y.
bool drism_zeta(const rism1d_solvent *sv, double beta, double dielectric, double a, const std::vector<double> &k,
                std::vector<double> &Z, std::string &why) {
    const int n = sv->n_sites, P = (int)k.size();
    std::vector<double> d((size_t)n * P, 0.0);
    double y_tot = 0.0, rho_y = 0.0;
    std::vector<int> done;
    for (int s0 = 0; s0 < n; ++s0) {
        const int sp = sv->species[s0];
        if (std::find(done.begin(), done.end(), sp) != done.end()) continue;
        done.push_back(sp);
        std::vector<int> idx;
        for (int b = 0; b < n; ++b)
            if (sv->species[b] == sp) idx.push_back(b);
        double cen[3] = {0.0, 0.0, 0.0};
        for (int b : idx)
            for (int c = 0; c < 3; ++c) cen[c] += sv->coords[3 * b + c] / (double)idx.size();
        std::vector<double> pos(3 * idx.size());
        double mu[3] = {0.0, 0.0, 0.0};
        for (size_t i = 0; i < idx.size(); ++i)
            for (int c = 0; c < 3; ++c) {
                pos[3 * i + c] = sv->coords[3 * idx[i] + c] - cen[c];
                mu[c] += sv->q[idx[i]] * pos[3 * i + c];
            }
        const double m = std::sqrt(mu[0] * mu[0] + mu[1] * mu[1] + mu[2] * mu[2]);
        if (m < 1e-12) continue;
        const double z[3] = {mu[0] / m, mu[1] / m, mu[2] / m};
        // x along the normal-to-z part of the site farthest from the z axis
        double x[3] = {0.0, 0.0, 0.0}, best = -1.0;
        for (size_t i = 0; i < idx.size(); ++i) {
            const double *p = &pos[3 * i];
            const double pz = p[0] * z[0] + p[1] * z[1] + p[2] * z[2];
            const double v[3] = {p[0] - pz * z[0], p[1] - pz * z[1], p[2] - pz * z[2]};
            const double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (nv > best) {
                best = nv;
                for (int c = 0; c < 3; ++c) x[c] = nv > 0.0 ? v[c] / nv : 0.0;
            }
        }
        if (!(best > 1e-12)) {        // all sites on the dipole axis: any x normal to z
            const double e[3] = {std::fabs(z[0]) < 0.9 ? 1.0 : 0.0, std::fabs(z[0]) < 0.9 ? 0.0 : 1.0, 0.0};
            double c3[3] = {z[1] * e[2] - z[2] * e[1], z[2] * e[0] - z[0] * e[2], z[0] * e[1] - z[1] * e[0]};
            const double nc = std::sqrt(c3[0] * c3[0] + c3[1] * c3[1] + c3[2] * c3[2]);
            for (int c = 0; c < 3; ++c) x[c] = c3[c] / nc;
        }
        const double yv[3] = {z[1] * x[2] - z[2] * x[1], z[2] * x[0] - z[0] * x[2], z[0] * x[1] - z[1] * x[0]};
        const double rho_s = sv->rho[idx[0]];
        const double ys = 4.0 * kPi * beta * kCoulomb * rho_s * m * m / 9.0;
        y_tot += ys;
        rho_y += rho_s * ys;
        for (size_t i = 0; i < idx.size(); ++i) {
            const double *p = &pos[3 * i];
            const double px = p[0] * x[0] + p[1] * x[1] + p[2] * x[2];
            const double py = p[0] * yv[0] + p[1] * yv[1] + p[2] * yv[2];
            const double pz = p[0] * z[0] + p[1] * z[1] + p[2] * z[2];
            for (int j = 0; j < P; ++j)
                d[(size_t)idx[i] * P + j] = sph_j0(k[j] * px) * sph_j0(k[j] * py) * sph_j1(k[j] * pz);
        }
    }
    if (rho_y == 0.0) {
        why = "DRISM needs a solvent molecule with a dipole";
        return false;
    }
    if (!(dielectric > 1.0 + 3.0 * y_tot)) {
        why = "DRISM dielectric constant must exceed the XRISM value 1 + 3y = " + std::to_string(1.0 + 3.0 * y_tot);
        return false;
    }
    const double hc0 = (dielectric - 1.0 - 3.0 * y_tot) / rho_y;
    Z.assign((size_t)n * n * P, 0.0);
    for (int a0 = 0; a0 < n; ++a0)
        for (int b = 0; b < n; ++b)
            for (int j = 0; j < P; ++j)
                Z[((size_t)a0 * n + b) * P + j] =
                    d[(size_t)a0 * P + j] * d[(size_t)b * P + j] * hc0 * std::exp(-(a * k[j]) * (a * k[j]) / 4.0);
    return true;
}

// HNC (closure 2): exp(d); KH (closure 1): exp(d) for d <= 0, 1 + d otherwise.
double closure_g(double d, int closure) {
    if (closure == 2 || d <= 0.0) return std::exp(d);
    return 1.0 + d;
}

}  // namespace

extern "C" {

void rism1d_options_default(rism1d_options *o) {
    if (!o) return;
    o->n_r = 2048;
    o->dr = 0.05;
    o->closure = 1;
    o->tol = 1e-10;
    o->max_iter = 5000;
    o->mdiis_nvec = 5;
    o->mdiis_damp = 0.3;
    o->charge_steps = 10;
    o->dielectric = 0.0;
    o->drism_damping = 1.0;
}

rism1d_status rism1d_xrism(const rism1d_solvent *sv, const rism1d_options *op, double *chi, double *dk_out,
                           int *iterations, double *rms_out) {
    return rism1d_xrism_ex(sv, op, chi, dk_out, nullptr, nullptr, nullptr, iterations, rms_out);
}

rism1d_status rism1d_xrism_ex(const rism1d_solvent *sv, const rism1d_options *op, double *chi, double *dk_out,
                              double *c_r, double *pressure, double *kT_chi_T, int *iterations,
                              double *rms_out) {
    if (!sv || !op || !chi || !dk_out) return fail(RISM1D_EINVAL, "null argument");
    const int n = sv->n_sites, N = op->n_r;
    if (n < 1 || n > 16) return fail(RISM1D_EINVAL, "n_sites must be in 1..16");
    if (N < 8 || (N & (N - 1))) return fail(RISM1D_EINVAL, "n_r must be a power of two >= 8");
    if (!(op->dr > 0.0) || !(sv->temperature > 0.0)) return fail(RISM1D_EINVAL, "dr and T must be positive");
    if (op->closure != 1 && op->closure != 2) return fail(RISM1D_EINVAL, "closure must be 1 (KH) or 2 (HNC)");
    if (!(op->dielectric >= 0.0) || !(op->drism_damping > 0.0) || !std::isfinite(op->dielectric))
        return fail(RISM1D_EINVAL, "dielectric must be >= 0 (0: XRISM) and drism_damping > 0");
    if (op->mdiis_nvec < 1 || op->mdiis_nvec > 32 || op->charge_steps < 1 || op->max_iter < 1 || !(op->tol > 0))
        return fail(RISM1D_EINVAL, "bad MDIIS / charge-step options");
    if (!sv->q || !sv->sigma || !sv->eps || !sv->rho || !sv->species || !sv->coords)
        return fail(RISM1D_EINVAL, "null solvent array");
    for (int a = 0; a < n; ++a) {
        if (!(sv->rho[a] > 0.0)) return fail(RISM1D_EINVAL, "rho must be positive");
        if (!(sv->sigma[a] >= 0.0) || !(sv->eps[a] >= 0.0) || !std::isfinite(sv->q[a]) ||
            !std::isfinite(sv->sigma[a]) || !std::isfinite(sv->eps[a]))
            return fail(RISM1D_EINVAL, "site sigma and eps must be finite and >= 0, q finite");
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(sv->coords[3 * a + d])) return fail(RISM1D_EINVAL, "non-finite site position");
        for (int b = 0; b < a; ++b) {
            if (sv->species[a] != sv->species[b]) continue;
            const double dx = sv->coords[3 * a] - sv->coords[3 * b];
            const double dy = sv->coords[3 * a + 1] - sv->coords[3 * b + 1];
            const double dz = sv->coords[3 * a + 2] - sv->coords[3 * b + 2];
            if (!(dx * dx + dy * dy + dz * dz > 0.0))        // omega = sin(kl)/(kl) needs l > 0
                return fail(RISM1D_EINVAL, "two sites of one molecule at the same position");
        }
    }

    const int P = N - 1;                     // radial points i = 1..N-1
    const double dr = op->dr, dk = kPi / (N * dr);
    const double beta = 1.0 / (kKB * sv->temperature);
    std::vector<double> r(P), k(P);
    for (int i = 0; i < P; ++i) {
        r[i] = (i + 1) * dr;
        k[i] = (i + 1) * dk;
    }
    const size_t F = (size_t)n * n * P;       // one field over all pairs
    auto at = [P, n](int a, int b) { return ((size_t)a * n + b) * P; };
    // intramolecular correlation omega_ab(k)
    std::vector<double> W(F, 0.0);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            if (a == b) {
                for (int j = 0; j < P; ++j) W[at(a, b) + j] = 1.0;
            } else if (sv->species[a] == sv->species[b]) {
                const double dx = sv->coords[3 * a] - sv->coords[3 * b];
                const double dy = sv->coords[3 * a + 1] - sv->coords[3 * b + 1];
                const double dz = sv->coords[3 * a + 2] - sv->coords[3 * b + 2];
                const double l = std::sqrt(dx * dx + dy * dy + dz * dz);
                for (int j = 0; j < P; ++j) W[at(a, b) + j] = std::sin(k[j] * l) / (k[j] * l);
            }
        }
    // DRISM: omega' = omega + rho_a zeta_ab replaces omega in the RISM equation (Z = 0: XRISM)
    std::vector<double> Z(F, 0.0), Wp(W);
    if (op->dielectric > 0.0) {
        std::string why;
        if (!drism_zeta(sv, beta, op->dielectric, op->drism_damping, k, Z, why)) return fail(RISM1D_EINVAL, why);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                for (int j = 0; j < P; ++j) Wp[at(a, b) + j] += sv->rho[a] * Z[at(a, b) + j];
    }
    SineTransform dst(N);
    std::vector<double> tmp(P), out(P);
    auto forward = [&](const double *f, double *Fk) {
        for (int i = 0; i < P; ++i) tmp[i] = r[i] * f[i];
        dst.run(tmp.data(), out.data());
        for (int j = 0; j < P; ++j) Fk[j] = 4.0 * kPi * dr / k[j] * out[j];
    };
    auto inverse = [&](const double *Fk, double *f) {
        for (int j = 0; j < P; ++j) tmp[j] = k[j] * Fk[j];
        dst.run(tmp.data(), out.data());
        for (int i = 0; i < P; ++i) f[i] = dk / (2.0 * kPi * kPi * r[i]) * out[i];
    };

    std::vector<double> tau(F, 0.0), bus(F), bUL(F), h(F), cs(F), Cs(F), H(F), R(F), tnew(F);
    std::vector<double> A((size_t)n * n), Bm((size_t)n * n), WC((size_t)n * n);
    const int M = op->mdiis_nvec;
    int total = 0;
    double rms = 0.0;
    rism1d_status status = RISM1D_OK;

    for (int step = 1; step <= op->charge_steps; ++step) {
        const double scale = (double)step / op->charge_steps;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                const double s = 0.5 * (sv->sigma[a] + sv->sigma[b]);
                const double e = std::sqrt(sv->eps[a] * sv->eps[b]);
                const double qq = sv->q[a] * scale * sv->q[b] * scale;
                for (int i = 0; i < P; ++i) {
                    const double r2 = std::max(r[i] * r[i], 1e-8);
                    const double sr6 = std::pow(s * s / r2, 3);
                    const double u = 4.0 * e * (sr6 * sr6 - sr6) + kCoulomb * qq * std::exp(-r[i]) / r[i];
                    bus[at(a, b) + i] = std::min(beta * u, kCap);
                }
                for (int j = 0; j < P; ++j)
                    bUL[at(a, b) + j] = beta * 4.0 * kPi * kCoulomb * qq / (k[j] * k[j] * (k[j] * k[j] + 1.0));
            }
        std::vector<std::vector<double>> hist_t, hist_R, gram;
        bool converged = false;
        for (int it = 1; it <= op->max_iter; ++it) {
            ++total;
            // closure on d = -beta u_s + tau; pair functions are symmetric (ab = ba), so the
            // upper triangle is computed and mirrored
            for (size_t x = 0; x < F; ++x) {
                const double g = closure_g(-bus[x] + tau[x], op->closure);
                h[x] = g - 1.0;
                cs[x] = h[x] - tau[x];
            }
            for (int a = 0; a < n; ++a)
                for (int b = a; b < n; ++b) {
                    forward(&cs[at(a, b)], &Cs[at(a, b)]);
                    if (b != a) std::copy(&Cs[at(a, b)], &Cs[at(a, b)] + P, &Cs[at(b, a)]);
                }
            // RISM equation per k: (I - W' C rho) H' = W' C W' with C = C_s - beta U_L, and
            // H = H' + zeta (W' = W and zeta = 0 for XRISM)
            for (int j = 0; j < P; ++j) {
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b) {
                        double s = 0.0;
                        for (int c = 0; c < n; ++c)
                            s += Wp[at(a, c) + j] * (Cs[at(c, b) + j] - bUL[at(c, b) + j]);
                        WC[a * n + b] = s;
                    }
                for (int a = 0; a < n; ++a)
                    for (int b = 0; b < n; ++b) {
                        A[a * n + b] = (a == b ? 1.0 : 0.0) - WC[a * n + b] * sv->rho[b];
                        double s = 0.0;
                        for (int c = 0; c < n; ++c) s += WC[a * n + c] * Wp[at(c, b) + j];
                        Bm[a * n + b] = s;
                    }
                if (!gauss_multi(A, Bm, n, n)) return fail(RISM1D_EDIVERGED, "singular RISM matrix");
                // H is symmetric (omega rho = rho omega within a molecule): keep its upper
                // triangle, mirrored, so that tau stays exactly symmetric
                for (int a = 0; a < n; ++a)
                    for (int b = a; b < n; ++b) {
                        const double v = Bm[a * n + b] + Z[at(a, b) + j];
                        H[at(a, b) + j] = v;
                        H[at(b, a) + j] = v;
                    }
            }
            std::vector<double> tk(P);
            for (int a = 0; a < n; ++a)
                for (int b = a; b < n; ++b) {
                    for (int j = 0; j < P; ++j) tk[j] = H[at(a, b) + j] - Cs[at(a, b) + j];
                    inverse(tk.data(), &tnew[at(a, b)]);
                    if (b != a) std::copy(&tnew[at(a, b)], &tnew[at(a, b)] + P, &tnew[at(b, a)]);
                }
            double ss = 0.0;
            for (size_t x = 0; x < F; ++x) {
                R[x] = tnew[x] - tau[x];
                ss += R[x] * R[x];
            }
            rms = std::sqrt(ss / (double)F);
            if (!std::isfinite(rms)) return fail(RISM1D_EDIVERGED, "non-finite residual in 1D RISM");
            if (rms < op->tol) {
                converged = true;
                break;
            }
            // MDIIS: minimise |sum c_i R_i| with sum c_i = 1 (bordered Gram system). The Gram
            // entries of stored pairs do not change, so only the new row is computed.
            hist_t.push_back(tau);
            hist_R.push_back(R);
            {
                const int m0 = (int)hist_R.size();
                std::vector<double> row(m0);
                for (int p = 0; p < m0; ++p) {
                    double s = 0.0;
                    for (size_t x = 0; x < F; ++x) s += hist_R[p][x] * hist_R[m0 - 1][x];
                    row[p] = s;
                }
                for (int p = 0; p < m0 - 1; ++p) gram[p].push_back(row[p]);
                gram.push_back(row);
            }
            auto drop_oldest = [&]() {
                hist_t.erase(hist_t.begin());
                hist_R.erase(hist_R.begin());
                gram.erase(gram.begin());
                for (auto &g : gram) g.erase(g.begin());
            };
            if ((int)hist_R.size() > M) drop_oldest();
            std::vector<double> coef;
            for (;;) {
                const int m = (int)hist_R.size();
                if (m == 1) {
                    coef.assign(1, 1.0);
                    break;
                }
                std::vector<double> Gm((size_t)m * m);
                double dmax = 0.0;
                for (int p = 0; p < m; ++p)
                    for (int q = 0; q < m; ++q) Gm[p * m + q] = gram[p][q];
                for (int p = 0; p < m; ++p) dmax = std::max(dmax, Gm[p * m + p]);
                const int dim = m + 1;
                std::vector<double> Ab((size_t)dim * dim, 0.0), rhs(dim, 0.0);
                for (int p = 0; p < m; ++p) {
                    for (int q = 0; q < m; ++q) Ab[p * dim + q] = dmax > 0 ? Gm[p * m + q] / dmax : Gm[p * m + q];
                    Ab[p * dim + m] = 1.0;
                    Ab[m * dim + p] = 1.0;
                }
                rhs[m] = 1.0;
                if (gauss(Ab, rhs, dim, kPivotMin)) {
                    coef.assign(rhs.begin(), rhs.begin() + m);
                    break;
                }
                drop_oldest();
            }
            std::fill(tau.begin(), tau.end(), 0.0);
            for (size_t p = 0; p < coef.size(); ++p)
                for (size_t x = 0; x < F; ++x) tau[x] += coef[p] * (hist_t[p][x] + op->mdiis_damp * hist_R[p][x]);
        }
        if (!converged) status = RISM1D_ENOTCONV;
    }
    // final fields at the converged tau (full charges)
    for (size_t x = 0; x < F; ++x) h[x] = closure_g(-bus[x] + tau[x], op->closure) - 1.0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            double h0 = 0.0;
            for (int i = 0; i < P; ++i) h0 += r[i] * r[i] * h[at(a, b) + i];
            h0 *= 4.0 * kPi * dr;
            const double w0 = (a == b || sv->species[a] == sv->species[b]) ? 1.0 : 0.0;
            double *row = chi + ((size_t)a * n + b) * N;
            row[0] = w0 + sv->rho[a] * h0;
            for (int j = 0; j < P; ++j) row[j + 1] = W[at(a, b) + j] + sv->rho[a] * H[at(a, b) + j];
        }
    // full direct correlation c = c_s - beta u_L (Coulomb tail of Eq. 29's form) at full charge
    if (c_r || pressure) {
        std::vector<double> cfull(F);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) {
                const double qq = sv->q[a] * sv->q[b];
                for (int i = 0; i < P; ++i) {
                    const double x = at(a, b) + i;
                    (void)x;
                    cfull[at(a, b) + i] = cs[at(a, b) + i] - beta * kCoulomb * qq * (-std::expm1(-r[i])) / r[i];
                }
            }
        if (c_r) std::copy(cfull.begin(), cfull.end(), c_r);
        if (pressure) {
            const double kT = 1.0 / beta;
            double ideal = 0.0;
            std::vector<int> seen;
            for (int a = 0; a < n; ++a) {
                if (std::find(seen.begin(), seen.end(), sv->species[a]) != seen.end()) continue;
                seen.push_back(sv->species[a]);
                int nsites = 0;
                for (int b = 0; b < n; ++b) nsites += sv->species[b] == sv->species[a];
                ideal += sv->rho[a] * (nsites + 1) * kT / 2.0;
            }
            double ex = 0.0;
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) {
                    double integ = 0.0;
                    for (int i = 0; i < P; ++i) integ += r[i] * r[i] * cfull[at(a, b) + i];
                    ex += sv->rho[a] * sv->rho[b] * integ * dr;
                }
            *pressure = ideal - 2.0 * kPi * kT * ex;
        }
    }
    if (kT_chi_T) *kT_chi_T = chi[0] / sv->rho[0];
    *dk_out = dk;
    if (iterations) *iterations = total;
    if (rms_out) *rms_out = rms;
    if (status != RISM1D_OK) return fail(status, "1D RISM did not reach the tolerance in every charge step");
    return RISM1D_OK;
}

const char *rism1d_last_error(void) { return g_err.c_str(); }

}  // extern "C"
