// Seeded synthetic inputs of the method, reproducible from C.
//
// The method consumes random numbers in three places: which atoms are removed
// (random single vacancies, Sec. 2), the Anderson on-site energies (uniform in
// [-W/2, W/2]), and the random phases of the trace-estimator vectors (Sec. 3.1.1:
// phi_n = exp(i theta_n), theta_n uniform in [0, 2 pi)).  This file draws them from
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) in counter mode, one stream per kind of draw:
//   key = mix64(seed + stream * G),  x_k = mix64(key + (k + 1) * G),  G = 0x9E3779B97F4A7C15,
// with mix64 the SplitMix64 output finaliser (shifts 30, 27, 31; multipliers
// 0xBF58476D1CE4E5B9, 0x94D049BB133111EB), all modulo 2^64.  Uniform doubles are the
// top 53 bits of a word times 2^-53.  Streams: 0 vacancies, 1 Anderson energies,
// 16 + r random vector r.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "kg_internal.h"

namespace kg {

static constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
static constexpr uint64_t kStreamVacancy = 0, kStreamAnderson = 1, kStreamVector0 = 16;

static inline uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

struct Stream {
    uint64_t key;
    Stream(uint64_t seed, uint64_t stream) : key(mix64(seed + stream * kGolden)) {}
    uint64_t word(uint64_t k) const { return mix64(key + (k + 1) * kGolden); }
    double uniform(uint64_t k) const { return (double)(word(k) >> 11) * 0x1.0p-53; }
};

}  // namespace kg

using namespace kg;

extern "C" {

kg_status kg_splitmix64(uint64_t seed, uint64_t stream, int64_t start, int64_t count, uint64_t* out) {
    clear_error();
    if (start < 0 || count < 0 || (count > 0 && !out)) return fail(KG_EINVAL, "kg_splitmix64: bad range or null output");
    const Stream s(seed, stream);
    for (int64_t k = 0; k < count; k++) out[k] = s.word((uint64_t)(start + k));
    return KG_OK;
}

kg_status kg_n_vacancies(int64_t n_sites, double concentration, int64_t* n_vac) {
    clear_error();
    if (!n_vac || n_sites < 0 || !(concentration >= 0.0 && concentration <= 1.0))
        return fail(KG_EINVAL, "kg_n_vacancies: need n_sites >= 0 and 0 <= concentration <= 1");
    // round half to even (the default rounding mode)
    *n_vac = (int64_t)std::nearbyint(concentration * (double)n_sites);
    return KG_OK;
}

kg_status kg_vacancy_sites(int64_t n_sites, int64_t n_vac, uint64_t seed, int64_t* out) {
    clear_error();
    if (n_sites < 0 || n_sites > (int64_t)INT32_MAX - 1 || n_vac < 0 || n_vac > n_sites)
        return fail(KG_EINVAL, "kg_vacancy_sites: need 0 <= n_vac <= n_sites < 2^31 - 1");
    if (n_vac == 0) return KG_OK;
    if (!out) return fail(KG_EINVAL, "kg_vacancy_sites: null output");
    // partial Fisher-Yates shuffle: step k swaps positions k and k + floor(w_k (N - k) / 2^32),
    // w_k the top 32 bits of word k (w_k (N - k) < 2^63: no overflow)
    std::vector<int64_t> perm((size_t)n_sites);
    for (int64_t i = 0; i < n_sites; i++) perm[(size_t)i] = i;
    const Stream s(seed, kStreamVacancy);
    for (int64_t k = 0; k < n_vac; k++) {
        const uint64_t w = s.word((uint64_t)k) >> 32;
        const uint64_t m = (uint64_t)(n_sites - k);
        const int64_t j = k + (int64_t)((w * m) >> 32);
        std::swap(perm[(size_t)k], perm[(size_t)j]);
    }
    std::vector<int64_t> v(perm.begin(), perm.begin() + n_vac);
    std::sort(v.begin(), v.end());
    for (int64_t k = 0; k < n_vac; k++) out[k] = v[(size_t)k];
    return KG_OK;
}

kg_status kg_anderson_onsite(int64_t n_sites, double w_ev, uint64_t seed, double* out_ev) {
    clear_error();
    if (n_sites < 0 || !(w_ev >= 0.0) || (n_sites > 0 && !out_ev))
        return fail(KG_EINVAL, "kg_anderson_onsite: need n_sites >= 0, W >= 0 and an output");
    const Stream s(seed, kStreamAnderson);
    for (int64_t n = 0; n < n_sites; n++) {
        const double u = s.uniform((uint64_t)n);
        const double centred = u - 0.5;
        out_ev[n] = w_ev * centred;
    }
    return KG_OK;
}

kg_status kg_random_phase_vectors(int64_t n_sites, int n_vectors, uint64_t seed, const int64_t* vacancies,
                                  int64_t n_vacancies, double* out) {
    clear_error();
    if (n_sites < 0 || n_vectors < 1 || n_vacancies < 0 || (n_vacancies > 0 && !vacancies) ||
        (n_sites > 0 && !out))
        return fail(KG_EINVAL, "kg_random_phase_vectors: bad sizes or null pointers");
    for (int64_t k = 0; k < n_vacancies; k++)
        if (vacancies[k] < 0 || vacancies[k] >= n_sites)
            return fail(KG_EINVAL, "kg_random_phase_vectors: vacancy out of range");
    const double two_pi = 2.0 * kPi;
    for (int r = 0; r < n_vectors; r++) {
        const Stream s(seed, kStreamVector0 + (uint64_t)r);
        for (int64_t n = 0; n < n_sites; n++) {
            const double theta = two_pi * s.uniform((uint64_t)n);
            double* o = out + ((size_t)n * n_vectors + r) * 2;
            o[0] = std::cos(theta);
            o[1] = std::sin(theta);
        }
    }
    for (int64_t k = 0; k < n_vacancies; k++)
        for (int r = 0; r < n_vectors; r++) {
            double* o = out + ((size_t)vacancies[k] * n_vectors + r) * 2;
            o[0] = 0.0;
            o[1] = 0.0;
        }
    return KG_OK;
}

}  // extern "C"
