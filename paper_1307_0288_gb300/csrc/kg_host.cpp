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
static bool periodic_y(int kind) { return kind == KG_SHEET || kind == KG_AGNR; }

kg_status build_host_lattice(const kg_lattice* lat, const int64_t* vacancies, int64_t n_vac,
                             HostLattice* out) {
    if (!lat) return fail(KG_EINVAL, "lattice is NULL");
    if (lat->kind < KG_SHEET || lat->kind > KG_AGNR) return fail(KG_EINVAL, "unknown lattice kind");
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
kg_status kg_pade_fit(const double* t, const double* y, int n_points, int m, int n, double* coef_out) {
    const int p = m + 1 + n;
    if (!t || !y || !coef_out || m < 0 || n < 0 || n_points < p) return fail(KG_EINVAL, "kg_pade_fit: bad arguments");
    std::vector<double> A((size_t)n_points * p), b(y, y + n_points), scale(p, 0.0);
    for (int i = 0; i < n_points; i++) {
        double tp = 1.0;
        for (int j = 0; j <= m; j++, tp *= t[i]) A[(size_t)i * p + j] = tp;
        tp = t[i];
        for (int k = 1; k <= n; k++, tp *= t[i]) A[(size_t)i * p + m + k] = -y[i] * tp;
    }
    for (int c = 0; c < p; c++) {
        double s = 0.0;
        for (int i = 0; i < n_points; i++) s += A[(size_t)i * p + c] * A[(size_t)i * p + c];
        scale[c] = s > 0 ? std::sqrt(s) : 1.0;
        for (int i = 0; i < n_points; i++) A[(size_t)i * p + c] /= scale[c];
    }
    // Householder QR: A = Q R, then R x = Q^T b
    for (int c = 0; c < p; c++) {
        double norm = 0.0;
        for (int i = c; i < n_points; i++) norm += A[(size_t)i * p + c] * A[(size_t)i * p + c];
        norm = std::sqrt(norm);
        if (norm == 0.0) return fail(KG_EINVAL, "kg_pade_fit: rank-deficient system");
        const double alpha = A[(size_t)c * p + c] > 0 ? -norm : norm;
        std::vector<double> v(n_points - c);
        for (int i = c; i < n_points; i++) v[i - c] = A[(size_t)i * p + c];
        v[0] -= alpha;
        double vv = 0.0;
        for (double q : v) vv += q * q;
        if (vv == 0.0) continue;
        for (int cc = c; cc < p; cc++) {
            double d = 0.0;
            for (int i = c; i < n_points; i++) d += v[i - c] * A[(size_t)i * p + cc];
            d = 2.0 * d / vv;
            for (int i = c; i < n_points; i++) A[(size_t)i * p + cc] -= d * v[i - c];
        }
        double d = 0.0;
        for (int i = c; i < n_points; i++) d += v[i - c] * b[i];
        d = 2.0 * d / vv;
        for (int i = c; i < n_points; i++) b[i] -= d * v[i - c];
    }
    for (int c = p - 1; c >= 0; c--) {
        double s = b[c];
        for (int cc = c + 1; cc < p; cc++) s -= A[(size_t)c * p + cc] * coef_out[cc];
        coef_out[c] = s / A[(size_t)c * p + c];
    }
    for (int c = 0; c < p; c++) coef_out[c] /= scale[c];
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
