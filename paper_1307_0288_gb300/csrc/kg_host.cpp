// Host-side parts of the library: error reporting, the lattice/neighbour table,
// Bessel coefficients, Jackson damping, the Chebyshev energy sums and the running
// conductivities.  None of this needs a GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "kg_internal.h"

namespace kg {

static thread_local std::string g_last_error;

kg_status fail(kg_status code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

void clear_error() { g_last_error.clear(); }

// ---------------------------------------------------------------------------------
// Lattice (Sec. 2).  Site (i, j), n = j*nx + i.  The three bonds of a site are its two
// neighbours along the zigzag chain, (i-1, j) and (i+1, j), and one neighbour on the
// adjacent chain: (i, j+1) when i + j is odd, (i, j-1) when it is even.
// ---------------------------------------------------------------------------------

static bool periodic_x(int kind) { return kind == KG_SHEET || kind == KG_ZGNR; }
static bool periodic_y(int kind) { return kind == KG_SHEET || kind == KG_AGNR || kind == KG_SHEET_OPEN_X; }

kg_status build_host_lattice(const kg_lattice* lat, const int64_t* vacancies, int64_t n_vac,
                             HostLattice* out) {
    if (!lat) return fail(KG_EINVAL, "lattice is NULL");
    if (lat->kind < KG_SHEET || lat->kind > KG_SHEET_OPEN_X) return fail(KG_EINVAL, "unknown lattice kind");
    if (lat->reserved != 0) return fail(KG_EINVAL, "kg_lattice.reserved must be 0");
    const int kind = lat->kind;
    const int64_t nx = lat->nx, ny = lat->ny;
    if (nx < 1 || ny < 1) return fail(KG_EINVAL, "nx and ny must be positive");
    if (periodic_x(kind) && (nx < 4 || nx % 2))
        return fail(KG_EINVAL, "a periodic x direction needs an even nx >= 4");
    if (periodic_y(kind) && (ny < 2 || ny % 2))
        return fail(KG_EINVAL, "a periodic y direction needs an even ny >= 2");
    if (!periodic_x(kind) && nx < 2) return fail(KG_EINVAL, "an open x direction needs nx >= 2");
    const int64_t n = nx * ny;
    if (n >= (int64_t)INT32_MAX - 1) return fail(KG_EINVAL, "too many sites for 32-bit indices");
    if (!(lat->gamma0_ev > 0) || !(lat->bond_nm > 0) || !(lat->emax_ev > 0))
        return fail(KG_EINVAL, "gamma0_ev, bond_nm and emax_ev must be positive");
    if (!(3.0 * lat->gamma0_ev < lat->emax_ev))
        return fail(KG_EINVAL, "emax_ev must exceed the band edge 3 gamma0");
    if (n_vac < 0 || n_vac > n) return fail(KG_EINVAL, "n_vacancies out of range");
    if (n_vac > 0 && !vacancies) return fail(KG_EINVAL, "vacancies is NULL");

    out->kind = kind;
    out->nx = nx;
    out->ny = ny;
    out->n = n;
    out->removed.assign((size_t)n, 0);
    for (int64_t k = 0; k < n_vac; k++) {
        const int64_t v = vacancies[k];
        if (v < 0 || v >= n) return fail(KG_EINVAL, "vacancy site out of range");
        if (out->removed[(size_t)v]) return fail(KG_EINVAL, "duplicate vacancy site");
        out->removed[(size_t)v] = 1;
    }
    out->n_active = n - n_vac;
    out->idx.assign((size_t)(3 * n), -1);
    out->parity.assign((size_t)n, 0);
    const bool px = periodic_x(kind), py = periodic_y(kind);
    for (int64_t j = 0; j < ny; j++) {
        for (int64_t i = 0; i < nx; i++) {
            const int64_t site = j * nx + i;
            const int odd = (int)((i + j) & 1);
            out->parity[(size_t)site] = (uint8_t)odd;
            if (out->removed[(size_t)site]) continue;
            const int64_t cand_i[3] = {i - 1, i + 1, i};
            const int64_t cand_j[3] = {j, j, odd ? j + 1 : j - 1};
            for (int k = 0; k < 3; k++) {
                int64_t ii = cand_i[k], jj = cand_j[k];
                if (ii < 0 || ii >= nx) {
                    if (!px) continue;
                    ii = (ii + nx) % nx;
                }
                if (jj < 0 || jj >= ny) {
                    if (!py) continue;
                    jj = (jj + ny) % ny;
                }
                const int64_t m = jj * nx + ii;
                if (out->removed[(size_t)m]) continue;
                out->idx[(size_t)(k * n + site)] = (int32_t)m;
            }
        }
    }
    return KG_OK;
}

double slot_displacement(int kind, double a, int parity, int slot) {
    if (kind != KG_AGNR) {
        // transport along x: the chain neighbours sit at -+ sqrt(3) a / 2, the
        // neighbour on the adjacent chain straight above or below.
        const double d = std::sqrt(3.0) * a / 2.0;
        return slot == 0 ? d : (slot == 1 ? -d : 0.0);
    }
    // transport along y: an odd site sits a/2 above its chain neighbours and a
    // below its partner on chain j+1; an even site the mirror image.
    if (slot < 2) return parity ? 0.5 * a : -0.5 * a;
    return parity ? -a : a;
}

// ---------------------------------------------------------------------------------
// Bessel coefficients J_m(tau) for Eqs. 36-37.
// For orders m >= tau^2/4 + 1 the power series (A&S 9.1.10)
//   J_m(x) = sum_k (-x^2/4)^k (x/2)^m / (k! (m+k)!)
// has decreasing terms from the start, so it is evaluated directly (full relative
// accuracy for the small tail coefficients that decide the truncation).  Lower orders
// use Bessel's integral (A&S 9.1.21) J_m(x) = (1/2pi) int_0^{2pi} cos(m t - x sin t) dt
// with the periodic trapezoidal rule on K points, which converges geometrically
// (Trefethen and Weideman, SIAM Review 56 (2014)); K exceeds m + |x| by a wide margin.
// ---------------------------------------------------------------------------------

static double bessel_series_term_sum(int m, double x) {
    const double q = -0.25 * x * x;
    double term = 1.0;
    for (int k = 1; k <= m; k++) term *= (0.5 * x) / k;   // (x/2)^m / m!
    double sum = term;
    for (int k = 1; k < 200; k++) {
        term *= q / ((double)k * (double)(m + k));
        sum += term;
        if (std::fabs(term) < 1e-18 * std::fabs(sum)) break;
    }
    return sum;
}

static double bessel_trapezoid(int m, double x) {
    const int K = 2 * (m + (int)std::fabs(x) + 64);
    double s = 0.0, c = 0.0;   // Neumaier-compensated sum
    for (int k = 0; k < K; k++) {
        const double mt = 2.0 * kPi * (double)((int64_t)m * k % K) / K;
        const double t = 2.0 * kPi * k / K;
        const double v = std::cos(mt - x * std::sin(t));
        const double u = s + v;
        c += (std::fabs(s) >= std::fabs(v)) ? (s - u) + v : (v - u) + s;
        s = u;
    }
    return (s + c) / K;
}

static double bessel_j(int m, double x) {
    if (x == 0.0) return m == 0 ? 1.0 : 0.0;
    if ((double)m >= 0.25 * x * x + 1.0) return bessel_series_term_sum(m, x);
    return bessel_trapezoid(m, x);
}

kg_status bessel_series(double tau, double tol, int max_terms, double* j, int* n_terms) {
    if (!(tau >= 0.0) || !(tol > 0.0) || !std::isfinite(tau))
        return fail(KG_EINVAL, "bessel_series: need tau >= 0 and tol > 0");
    if (!j || !n_terms || max_terms < 1) return fail(KG_EINVAL, "bessel_series: bad output");
    int np = -1;
    for (int m = 0; m < max_terms + 1; m++) {
        const double v = bessel_j(m, tau);
        if ((double)m > tau && std::fabs(v) < tol) {
            np = m;
            break;
        }
        if (m < max_terms) j[m] = v;
    }
    if (np < 0) return fail(KG_EINVAL, "bessel_series: max_terms too small for tau");
    *n_terms = np;
    return KG_OK;
}

}  // namespace kg

using namespace kg;

extern "C" {

const char* kg_last_error(void) { return g_last_error.c_str(); }

int kg_abi_version(void) { return KG_ABI_VERSION; }

kg_status kg_lattice_neighbors(const kg_lattice* lattice, const int64_t* vacancies,
                               int64_t n_vacancies, int32_t* idx_out) {
    if (!idx_out) return fail(KG_EINVAL, "idx_out is NULL");
    HostLattice hl;
    KG_TRY(build_host_lattice(lattice, vacancies, n_vacancies, &hl));
    std::memcpy(idx_out, hl.idx.data(), hl.idx.size() * sizeof(int32_t));
    return KG_OK;
}

kg_status kg_bessel_series(double tau, double tol, int max_terms, double* j_out, int* n_terms) {
    return bessel_series(tau, tol, max_terms, j_out, n_terms);
}

// Jackson damping (Eq. 35): g_n = (1 - n a) cos(pi n a) + a sin(pi n a) cot(pi a),
// a = 1 / (M + 1).
kg_status kg_jackson(int n_moments, double* g_out) {
    if (n_moments < 1 || !g_out) return fail(KG_EINVAL, "kg_jackson: bad arguments");
    const double a = 1.0 / (n_moments + 1.0);
    const double cot = std::cos(kPi * a) / std::sin(kPi * a);
    for (int n = 0; n < n_moments; n++)
        g_out[n] = (1.0 - n * a) * std::cos(kPi * n * a) + a * std::sin(kPi * n * a) * cot;
    return KG_OK;
}

// Eqs. 29-31 with T_n(E~) generated by the three-term recurrence T_{n+1} = 2E~T_n - T_{n-1}.
kg_status kg_kpm_sum(const double* mu, int n_sets, int n_moments, const double* energies_ev,
                     int n_e, double emax_ev, double area_nm2, double* out) {
    if (!mu || !energies_ev || !out || n_sets < 1 || n_moments < 1 || n_e < 1 ||
        !(emax_ev > 0) || !(area_nm2 > 0))
        return fail(KG_EINVAL, "kg_kpm_sum: bad arguments");
    std::vector<double> g((size_t)n_moments), w((size_t)n_moments);
    kg_jackson(n_moments, g.data());
    for (int n = 0; n < n_moments; n++) w[(size_t)n] = g[(size_t)n] * (n == 0 ? 1.0 : 2.0);
    for (int e = 0; e < n_e; e++) {
        const double x = energies_ev[e] / emax_ev;
        if (!(std::fabs(x) < 1.0)) return fail(KG_EINVAL, "kg_kpm_sum: |E| must be below E_max");
        const double pref = 2.0 / (kPi * area_nm2 * emax_ev * std::sqrt(1.0 - x * x));
        for (int s = 0; s < n_sets; s++) {
            const double* m = mu + (size_t)s * n_moments;
            double t0 = 1.0, t1 = x;
            double acc = w[0] * m[0];
            if (n_moments > 1) acc += w[1] * x * m[1];
            for (int n = 2; n < n_moments; n++) {
                const double t2 = 2.0 * x * t1 - t0;
                acc += w[(size_t)n] * t2 * m[n];
                t0 = t1;
                t1 = t2;
            }
            out[(size_t)s * n_e + e] = pref * acc;
        }
    }
    return KG_OK;
}

// Eq. 22 with the Hanning window of Eq. 28 and the scaled step dtau = pi hbar / E_max:
// rho(E) = 1 / (E_max Omega) sum_{n=-N_m}^{N_m} w_n Re[exp(i pi n E / E_max) F_n].
kg_status kg_ftm_sum(const double* f, int n_sets, int n_m, const double* energies_ev, int n_e,
                     double emax_ev, double area_nm2, double* out) {
    if (!f || !energies_ev || !out || n_sets < 1 || n_m < 0 || n_e < 1 || !(emax_ev > 0) || !(area_nm2 > 0))
        return fail(KG_EINVAL, "kg_ftm_sum: bad arguments");
    const int width = 2 * n_m + 1;
    for (int s = 0; s < n_sets; s++) {
        const double* fs = f + (size_t)s * width * 2;
        for (int e = 0; e < n_e; e++) {
            const double x = energies_ev[e] / emax_ev;
            double acc = 0.0;
            for (int k = -n_m; k <= n_m; k++) {
                const double w = 0.5 * (1.0 + std::cos(kPi * k / (n_m + 1.0)));
                const double ph = kPi * k * x;
                const double re = fs[2 * (k + n_m)], im = fs[2 * (k + n_m) + 1];
                acc += w * (std::cos(ph) * re - std::sin(ph) * im);
            }
            out[(size_t)s * n_e + e] = acc / (emax_ev * area_nm2);
        }
    }
    return KG_OK;
}

// Ballistic length and conductance (Eqs. 50-51): DX^2 = (rho DX^2) / rho (Eq. 10),
// L = 2 sqrt(DX^2), G = (W / L) sigma^E1, sigma^E1 from Eq. 9 (central differences).
kg_status kg_ballistic(const double* rho, const double* rho_dx2, int n_times, int n_e, double dt_fs,
                       double width_nm, double* length_out, double* g_out) {
    if (!rho || !rho_dx2 || !length_out || !g_out || n_times < 2 || n_e < 1 || !(dt_fs > 0) || !(width_nm > 0))
        return fail(KG_EINVAL, "kg_ballistic: bad arguments");
    std::vector<double> s1((size_t)n_times * n_e);
    KG_TRY(kg_conductivity(KG_SIGMA_E1, rho_dx2, n_times, n_e, dt_fs, s1.data()));
    for (int t = 0; t < n_times; t++)
        for (int e = 0; e < n_e; e++) {
            const size_t k = (size_t)t * n_e + e;
            const double dx2 = rho[e] > 0 ? rho_dx2[k] / rho[e] : 0.0;
            const double len = dx2 > 0 ? 2.0 * std::sqrt(dx2) : 0.0;
            length_out[k] = len;
            g_out[k] = len > 0 ? width_nm / len * s1[k] : 0.0;
        }
    return KG_OK;
}

// Semi-classical conductivity (Sec. 5.2): the maximum over t > 0 (Eq. 53) and the average
// over the block t1 <= t <= t2 (Eq. 54, trapezoid over the grid points in the block).
kg_status kg_sigma_sc(const double* sigma, int n_times, int n_e, double dt_fs, double t1_fs, double t2_fs,
                      double* max_out, double* avg_out) {
    if (!sigma || n_times < 2 || n_e < 1 || !(dt_fs > 0) || !(t2_fs > t1_fs))
        return fail(KG_EINVAL, "kg_sigma_sc: bad arguments");
    const int k1 = std::max(0, (int)std::ceil(t1_fs / dt_fs - 1e-9));
    const int k2 = std::min(n_times - 1, (int)std::floor(t2_fs / dt_fs + 1e-9));
    if (avg_out && k2 <= k1) return fail(KG_EINVAL, "kg_sigma_sc: the block holds fewer than two times");
    for (int e = 0; e < n_e; e++) {
        if (max_out) {
            double m = sigma[(size_t)1 * n_e + e];
            for (int t = 2; t < n_times; t++) m = std::fmax(m, sigma[(size_t)t * n_e + e]);
            max_out[e] = m;
        }
        if (avg_out) {
            double acc = 0.0;
            for (int t = k1; t < k2; t++)
                acc += 0.5 * dt_fs * (sigma[(size_t)t * n_e + e] + sigma[(size_t)(t + 1) * n_e + e]);
            avg_out[e] = acc / ((k2 - k1) * dt_fs);
        }
    }
    return KG_OK;
}

// Pade [m/n] fit (Eq. 58; reading: the denominator sum starts at k = 1):
//   y(t) = sum_{j<=m} a_j t^j / (1 + sum_{1<=k<=n} b_k t^k),
// linearised as sum_j a_j t^j - y sum_k b_k t^k = y and solved in the least-squares sense
// with Householder QR on the columns scaled to unit norm.  coef_out = (a_0..a_m, b_1..b_n).
// Least squares min |A x - rhs| over the columns listed in cols (the others are 0), with
// Householder QR on those columns scaled to unit norm.  A is row-major [rows][p].
static kg_status ls_columns(const std::vector<double>& A, const double* rhs, int rows, int p,
                            const std::vector<int>& cols, double* x_out) {
    const int q = (int)cols.size();
    std::vector<double> M((size_t)rows * q), b(rhs, rhs + rows), scale(q, 0.0), x(q, 0.0);
    for (int i = 0; i < rows; i++)
        for (int c = 0; c < q; c++) M[(size_t)i * q + c] = A[(size_t)i * p + cols[c]];
    for (int c = 0; c < q; c++) {
        double s = 0.0;
        for (int i = 0; i < rows; i++) s += M[(size_t)i * q + c] * M[(size_t)i * q + c];
        scale[c] = s > 0 ? std::sqrt(s) : 1.0;
        for (int i = 0; i < rows; i++) M[(size_t)i * q + c] /= scale[c];
    }
    for (int c = 0; c < q; c++) {
        double norm = 0.0;
        for (int i = c; i < rows; i++) norm += M[(size_t)i * q + c] * M[(size_t)i * q + c];
        norm = std::sqrt(norm);
        if (norm == 0.0) return fail(KG_EINVAL, "kg_pade_fit: rank-deficient system");
        const double alpha = M[(size_t)c * q + c] > 0 ? -norm : norm;
        std::vector<double> v(rows - c);
        for (int i = c; i < rows; i++) v[i - c] = M[(size_t)i * q + c];
        v[0] -= alpha;
        double vv = 0.0;
        for (double w : v) vv += w * w;
        if (vv == 0.0) continue;
        for (int cc = c; cc < q; cc++) {
            double d = 0.0;
            for (int i = c; i < rows; i++) d += v[i - c] * M[(size_t)i * q + cc];
            d = 2.0 * d / vv;
            for (int i = c; i < rows; i++) M[(size_t)i * q + cc] -= d * v[i - c];
        }
        double d = 0.0;
        for (int i = c; i < rows; i++) d += v[i - c] * b[i];
        d = 2.0 * d / vv;
        for (int i = c; i < rows; i++) b[i] -= d * v[i - c];
    }
    for (int c = q - 1; c >= 0; c--) {
        double s = b[c];
        for (int cc = c + 1; cc < q; cc++) s -= M[(size_t)c * q + cc] * x[cc];
        x[c] = s / M[(size_t)c * q + c];
    }
    for (int c = 0; c < p; c++) x_out[c] = 0.0;
    for (int c = 0; c < q; c++) x_out[cols[c]] = x[c] / scale[c];
    return KG_OK;
}

// The linearised system of Eq. 58: row i is (t^0..t^m, -y t^1..-y t^n), right-hand side y.
static std::vector<double> pade_system(const double* t, const double* y, int n_points, int m, int n) {
    const int p = m + 1 + n;
    std::vector<double> A((size_t)n_points * p);
    for (int i = 0; i < n_points; i++) {
        double tp = 1.0;
        for (int j = 0; j <= m; j++, tp *= t[i]) A[(size_t)i * p + j] = tp;
        tp = t[i];
        for (int k = 1; k <= n; k++, tp *= t[i]) A[(size_t)i * p + m + k] = -y[i] * tp;
    }
    return A;
}

kg_status kg_pade_fit(const double* t, const double* y, int n_points, int m, int n, double* coef_out) {
    const int p = m + 1 + n;
    if (!t || !y || !coef_out || m < 0 || n < 0 || n_points < p) return fail(KG_EINVAL, "kg_pade_fit: bad arguments");
    const std::vector<double> A = pade_system(t, y, n_points, m, n);
    std::vector<int> cols(p);
    for (int c = 0; c < p; c++) cols[c] = c;
    return ls_columns(A, y, n_points, p, cols, coef_out);
}

// Bounded least squares min |W (A x - y)| with every b_k >= 0 (W = diag(w)).  The problem is
// convex; its minimiser solves the unconstrained problem with some set of b_k held at 0, so
// all 2^n such sets are solved and the feasible solution with the smallest residual kept.
static kg_status pade_bounded(const std::vector<double>& A, const double* y, const std::vector<double>& w,
                              int n_points, int m, int n, double* x_out) {
    const int p = m + 1 + n;
    std::vector<double> Aw(A.size()), yw(n_points), x(p);
    for (int i = 0; i < n_points; i++) {
        yw[i] = w[i] * y[i];
        for (int c = 0; c < p; c++) Aw[(size_t)i * p + c] = w[i] * A[(size_t)i * p + c];
    }
    double best_r = -1.0;
    for (unsigned mask = 0; mask < (1u << n); mask++) {   // bit k set: b_{k+1} held at 0
        std::vector<int> cols;
        for (int j = 0; j <= m; j++) cols.push_back(j);
        for (int k = 0; k < n; k++)
            if (!(mask & (1u << k))) cols.push_back(m + 1 + k);
        if (ls_columns(Aw, yw.data(), n_points, p, cols, x.data()) != KG_OK) continue;
        bool feasible = true;
        for (int k = 0; k < n; k++) feasible &= x[m + 1 + k] >= 0.0;
        if (!feasible) continue;
        double r = 0.0;
        for (int i = 0; i < n_points; i++) {
            double e = -yw[i];
            for (int c = 0; c < p; c++) e += Aw[(size_t)i * p + c] * x[c];
            r += e * e;
        }
        if (best_r < 0 || r < best_r) {
            best_r = r;
            for (int c = 0; c < p; c++) x_out[c] = x[c];
        }
    }
    clear_error();
    return best_r < 0 ? fail(KG_EINVAL, "kg_pade_fit_positive: no solvable column set") : KG_OK;
}

// Residuals R(t_i) - y_i of the approximant x = (a_0..a_m, b_1..b_n) and, when J is not null,
// their Jacobian [n_points][p]: dR/da_j = t^j / D, dR/db_k = -R t^k / D.  Returns sum r^2.
static double pade_residuals(const double* t, const double* y, int n_points, int m, int n, const double* x,
                             double* r, double* J) {
    const int p = m + 1 + n;
    double sum = 0.0;
    for (int i = 0; i < n_points; i++) {
        double num = 0.0, den = 1.0, tp = 1.0;
        for (int j = 0; j <= m; j++, tp *= t[i]) num += x[j] * tp;
        tp = t[i];
        for (int k = 1; k <= n; k++, tp *= t[i]) den += x[m + k] * tp;
        const double R = num / den, e = R - y[i];
        if (r) r[i] = e;
        sum += e * e;
        if (J) {
            tp = 1.0;
            for (int j = 0; j <= m; j++, tp *= t[i]) J[(size_t)i * p + j] = tp / den;
            tp = t[i];
            for (int k = 1; k <= n; k++, tp *= t[i]) J[(size_t)i * p + m + k] = -R * tp / den;
        }
    }
    return sum;
}

// Projected Levenberg-Marquardt (Levenberg 1944, Marquardt 1963) on sum (R(t_i) - y_i)^2
// with b_k >= 0, from x (updated in place).  A b_k at 0 whose gradient points below 0 is held
// fixed for the step; every trial point is projected onto b >= 0.  Returns the final sum.
static double pade_refine(const double* t, const double* y, int n_points, int m, int n, double* x) {
    const int p = m + 1 + n;
    std::vector<double> r(n_points), J((size_t)n_points * p), xt(p);
    double f = pade_residuals(t, y, n_points, m, n, x, r.data(), J.data());
    double lambda = 1e-3;
    for (int it = 0; it < 500 && lambda < 1e16; it++) {
        std::vector<double> H((size_t)p * p, 0.0), g(p, 0.0);
        for (int i = 0; i < n_points; i++)
            for (int c = 0; c < p; c++) {
                g[c] += J[(size_t)i * p + c] * r[i];
                for (int d = 0; d < p; d++) H[(size_t)c * p + d] += J[(size_t)i * p + c] * J[(size_t)i * p + d];
            }
        std::vector<int> fr;   // free parameters of this step
        for (int c = 0; c < p; c++)
            if (!(c > m && x[c] <= 0.0 && g[c] >= 0.0)) fr.push_back(c);
        const int q = (int)fr.size();
        // (H + lambda diag H) d = -g on the free set, in Jacobi-scaled variables, by Gaussian elimination
        std::vector<double> S(q), M((size_t)q * (q + 1));
        for (int c = 0; c < q; c++) S[c] = H[(size_t)fr[c] * p + fr[c]] > 0 ? 1.0 / std::sqrt(H[(size_t)fr[c] * p + fr[c]]) : 1.0;
        for (int c = 0; c < q; c++) {
            for (int d = 0; d < q; d++) M[(size_t)c * (q + 1) + d] = H[(size_t)fr[c] * p + fr[d]] * S[c] * S[d];
            M[(size_t)c * (q + 1) + c] *= 1.0 + lambda;
            M[(size_t)c * (q + 1) + q] = -g[fr[c]] * S[c];
        }
        bool singular = false;
        for (int c = 0; c < q && !singular; c++) {
            int piv = c;
            for (int d = c + 1; d < q; d++)
                if (std::fabs(M[(size_t)d * (q + 1) + c]) > std::fabs(M[(size_t)piv * (q + 1) + c])) piv = d;
            if (M[(size_t)piv * (q + 1) + c] == 0.0) { singular = true; break; }
            if (piv != c)
                for (int e = 0; e <= q; e++) std::swap(M[(size_t)c * (q + 1) + e], M[(size_t)piv * (q + 1) + e]);
            for (int d = c + 1; d < q; d++) {
                const double fct = M[(size_t)d * (q + 1) + c] / M[(size_t)c * (q + 1) + c];
                for (int e = c; e <= q; e++) M[(size_t)d * (q + 1) + e] -= fct * M[(size_t)c * (q + 1) + e];
            }
        }
        if (singular) { lambda *= 10.0; continue; }
        std::vector<double> d(q);
        for (int c = q - 1; c >= 0; c--) {
            double v = M[(size_t)c * (q + 1) + q];
            for (int e = c + 1; e < q; e++) v -= M[(size_t)c * (q + 1) + e] * d[e];
            d[c] = v / M[(size_t)c * (q + 1) + c];
        }
        for (int c = 0; c < p; c++) xt[c] = x[c];
        for (int c = 0; c < q; c++) xt[fr[c]] += d[c] * S[c];
        for (int k = 1; k <= n; k++) xt[m + k] = std::max(xt[m + k], 0.0);
        const double ft = pade_residuals(t, y, n_points, m, n, xt.data(), nullptr, nullptr);
        if (std::isfinite(ft) && ft < f) {
            const bool tiny = f - ft <= 1e-15 * f;
            for (int c = 0; c < p; c++) x[c] = xt[c];
            f = pade_residuals(t, y, n_points, m, n, x, r.data(), J.data());
            lambda = std::max(lambda * 0.1, 1e-12);
            if (tiny) break;
        } else {
            lambda *= 10.0;
        }
    }
    return f;
}

// Eq. 58 with every b_k >= 0 (no pole for t >= 0), fitted to the true residual
// sum (R(t_i) - y_i)^2.  Starting points: Sanathanan-Koerner reweighting of the linearised
// problem (the linearised residual of point i is the true one times the denominator D(t_i),
// so each pass divides row i by D(t_i) of the previous pass, until the weights change by
// less than 1e-12, at most 100 passes), begun from four weight profiles
// w_i = (1 + |t_i| / s)^-n, s = infinity, t_max, t_max / 10, t_max / 100.  Each start is
// refined by projected Levenberg-Marquardt; the one with the smallest residual is returned.
kg_status kg_pade_fit_positive(const double* t, const double* y, int n_points, int m, int n, double* coef_out) {
    const int p = m + 1 + n;
    if (!t || !y || !coef_out || m < 0 || n < 0 || n > 8 || n_points < p)
        return fail(KG_EINVAL, "kg_pade_fit_positive: bad arguments (n <= 8, n_points >= m + 1 + n)");
    const std::vector<double> A = pade_system(t, y, n_points, m, n);
    double t_max = 0.0;
    for (int i = 0; i < n_points; i++) t_max = std::max(t_max, std::fabs(t[i]));
    std::vector<double> x(p), best(p);
    double best_r = -1.0;
    for (int start = 0; start < 4; start++) {
        std::vector<double> w(n_points, 1.0);
        if (start > 0 && t_max > 0) {
            const double sc = t_max / std::pow(10.0, start - 1);
            for (int i = 0; i < n_points; i++) w[i] = std::pow(1.0 + std::fabs(t[i]) / sc, -n);
        }
        bool solved = false;
        for (int pass = 0; pass < 100; pass++) {
            if (pade_bounded(A, y, w, n_points, m, n, x.data()) != KG_OK) break;
            solved = true;
            double change = 0.0;
            for (int i = 0; i < n_points; i++) {
                double den = 1.0, tp = t[i];
                for (int k = 1; k <= n; k++, tp *= t[i]) den += x[m + k] * tp;
                const double wn = 1.0 / den;
                change = std::max(change, std::fabs(wn - w[i]) / w[i]);
                w[i] = wn;
            }
            if (change < 1e-12) break;
        }
        if (!solved) continue;
        const double r = pade_refine(t, y, n_points, m, n, x.data());
        if (std::isfinite(r) && (best_r < 0 || r < best_r)) {
            best_r = r;
            best = x;
        }
    }
    clear_error();
    if (best_r < 0) return fail(KG_EINVAL, "kg_pade_fit_positive: no solvable column set");
    for (int c = 0; c < p; c++) coef_out[c] = best[c];
    return KG_OK;
}

// Value and t-derivative of the fitted Pade approximant at n_points times.
kg_status kg_pade_eval(const double* coef, int m, int n, const double* t, int n_points, double* value_out,
                       double* deriv_out) {
    if (!coef || !t || m < 0 || n < 0 || n_points < 1) return fail(KG_EINVAL, "kg_pade_eval: bad arguments");
    for (int i = 0; i < n_points; i++) {
        double num = 0.0, dnum = 0.0, den = 1.0, dden = 0.0, tp = 1.0;
        for (int j = 0; j <= m; j++, tp *= t[i]) {
            num += coef[j] * tp;
            if (j > 0) dnum += j * coef[j] * tp / t[i];
        }
        tp = t[i];
        for (int k = 1; k <= n; k++, tp *= t[i]) {
            den += coef[m + k] * tp;
            dden += k * coef[m + k] * tp / t[i];
        }
        if (value_out) value_out[i] = num / den;
        if (deriv_out) deriv_out[i] = (dnum * den - num * dden) / (den * den);
    }
    return KG_OK;
}

kg_status kg_conductivity(int formula, const double* density, int n_times, int n_e,
                          double dt_fs, double* out) {
    if (!density || !out || n_times < 1 || n_e < 1 || !(dt_fs > 0))
        return fail(KG_EINVAL, "kg_conductivity: bad arguments");
    const double h_ev_fs = 2.0 * kPi * kHbarEvFs;
    auto at = [&](const double* a, int t, int e) { return a[(size_t)t * n_e + e]; };
    for (int e = 0; e < n_e; e++) {
        if (formula == KG_SIGMA_GK) {
            // Eq. 6, trapezoid rule: sigma(t_m) = h sum_{k<m} dt (f_k + f_{k+1}) / 2
            double acc = 0.0;
            out[e] = 0.0;
            for (int t = 1; t < n_times; t++) {
                acc += 0.5 * dt_fs * (at(density, t - 1, e) + at(density, t, e));
                out[(size_t)t * n_e + e] = h_ev_fs * acc;
            }
        } else if (formula == KG_SIGMA_E1) {
            // Eq. 9: (h/2) d/dt, central differences inside, one-sided at both ends
            for (int t = 0; t < n_times; t++) {
                double d;
                if (n_times == 1) d = 0.0;
                else if (t == 0) d = (at(density, 1, e) - at(density, 0, e)) / dt_fs;
                else if (t == n_times - 1) d = (at(density, t, e) - at(density, t - 1, e)) / dt_fs;
                else d = (at(density, t + 1, e) - at(density, t - 1, e)) / (2.0 * dt_fs);
                out[(size_t)t * n_e + e] = 0.5 * h_ev_fs * d;
            }
        } else if (formula == KG_SIGMA_E2) {
            // Eq. 11: h f / (2 t), zero at t = 0
            out[e] = 0.0;
            for (int t = 1; t < n_times; t++)
                out[(size_t)t * n_e + e] = h_ev_fs * at(density, t, e) / (2.0 * t * dt_fs);
        } else {
            return fail(KG_EINVAL, "kg_conductivity: unknown formula");
        }
    }
    return KG_OK;
}

}  // extern "C"
