// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "kg.h"

namespace kg {

// hbar in eV fs (CODATA 2018) and h = 2 pi hbar.
constexpr double kHbarEvFs = 0.6582119569;
constexpr double kPi = 3.14159265358979323846;

// Thread-local error message + status helpers.
kg_status fail(kg_status code, const std::string& msg);
void clear_error();

#define KG_CUDA_TRY(expr)                                                              \
    do {                                                                               \
        cudaError_t kg_e_ = (expr);                                                    \
        if (kg_e_ != cudaSuccess)                                                      \
            return ::kg::fail(KG_ECUDA, std::string(#expr) + ": " +                    \
                                            cudaGetErrorString(kg_e_));               \
    } while (0)

#define KG_TRY(expr)                    \
    do {                                \
        kg_status kg_s_ = (expr);       \
        if (kg_s_ != KG_OK) return kg_s_; \
    } while (0)

// ---------------------------------------------------------------------------------
// Host-side lattice (built once per Hamiltonian, then uploaded)
// ---------------------------------------------------------------------------------

struct HostLattice {
    int kind = 0;
    int64_t nx = 0, ny = 0, n = 0, n_active = 0;
    std::vector<int32_t> idx;       // [3][n], -1 = no neighbour
    std::vector<uint8_t> removed;   // [n]
    std::vector<uint8_t> parity;    // [n] (i + j) & 1
};

// Validates the lattice description and fills the slot-major neighbour table.
kg_status build_host_lattice(const kg_lattice* lat, const int64_t* vacancies, int64_t n_vac,
                             HostLattice* out);

// Displacement X_n - X_m (nm) of the bond in slot k of a site with parity p, along the
// transport direction of the lattice kind.
double slot_displacement(int kind, double bond_nm, int parity, int slot);

// Bessel coefficients (host, FP64).
kg_status bessel_series(double tau, double tol, int max_terms, double* j, int* n_terms);

// ---------------------------------------------------------------------------------
// Device-side description of H~ passed to every kernel launcher
// ---------------------------------------------------------------------------------

struct DevH {
    const int32_t* idx = nullptr;   // [3][istride], sentinel = n (the zero row)
    int64_t istride = 0;
    int64_t n = 0;                  // sites; vectors have n + 1 rows (row n is zero)
    const double* onsite = nullptr; // eps_n / E_max, or null
    const double* onsite2 = nullptr;// 2 eps_n / E_max (the factor of the steps after the first), or null
                                    // (then formed from onsite)
    const uint8_t* parity = nullptr;// only for transport along y (AGNR)
    double h = 0.0;                 // H~ hopping  -gamma0 / E_max
    double dh[2][3] = {{0}};        // (X_n - X_m) * h per parity and slot (nm)
    bool ytransport = false;
};

// Number of SMs of the current device.
int sm_count();

// Device description of a built Hamiltonian (defined with the handle in kg_api.cu).
const DevH& hamiltonian_dev(const kg_hamiltonian* h);
cudaStream_t hamiltonian_stream(const kg_hamiltonian* h);

// Complex vector element of each precision.
template <typename T>
struct Vec2;
template <>
struct Vec2<double> { using type = double2; };
template <>
struct Vec2<float> { using type = float2; };
template <typename T>
using vec2_t = typename Vec2<T>::type;

// ----- launchers (kg_kernels.cu); all return cudaError_t of the launch -----
// T = double: complex128 vectors (KG_FP64); T = float: complex64 vectors (KG_C64).
// Partial sums and moments are FP64 in both.

// KPM step with phi_L = phi_R (Chebyshev doubling): out = c H~ cur - prev (prev may be
// null on the first step, then c = 1), partial[g][r][2] = (sum |cur|^2, sum Re conj(out) cur).
template <typename T>
cudaError_t launch_kpm_sym(const DevH& H, int R, bool first, const vec2_t<T>* cur,
                           const vec2_t<T>* prev, vec2_t<T>* out, double* partial, int grid,
                           cudaStream_t s);

// KPM step with a separate phi_L: out = c H~ cur - prev; partial[g][r][2] = <L|out>.
// On the first step partial[g][r][4] = (<L|out>, <L|cur>).
template <typename T>
cudaError_t launch_kpm_gen(const DevH& H, int R, bool first, const vec2_t<T>* L,
                           const vec2_t<T>* cur, const vec2_t<T>* prev, vec2_t<T>* out,
                           double* partial, int grid, cudaStream_t s);

// One full resident wave of the (non-first) KPM step kernel for this H and R.
template <typename T>
int kpm_grid(const DevH& H, int R, bool sym);

// Small instances: the moment recursion of an H with at most 16 CTAs of work per step
// runs as one thread-block cluster per chunk of steps, vectors in shared memory.
constexpr int kClusterMaxChunk = 256;   // steps per launch at most (one ring of partial slabs)
struct ClusterPlan {
    int grid = 0;        // CTAs = cluster size (0: the cluster path is not available)
    int log_nt = 0;      // threads per CTA = 1 << log_nt, one item per thread
    int chunk = 0;       // recursion steps per launch at most (<= kClusterMaxChunk)
    size_t smem = 0;     // dynamic shared memory per CTA
};

// Chooses the cluster plan for this H, R and mode (cached per device); false when the
// instance is too large (more than 16 CTAs of work or R > 16) or no such cluster fits.
template <typename T>
bool kpm_cluster_plan(const DevH& H, int R, bool sym, ClusterPlan* plan);

// KPM steps n0 .. n0 + nsteps - 1 in one cluster launch: the per-step kernels' vectors
// (bitwise), and per step k the per-CTA partial sums in ring slab k, laid out
// [k][plan.grid][R][2] like theirs.  phi_n and phi_{n-1} of step n0 are read from src_cur
// and src_prev; after the last step phi_n and phi_{n-1} are written to dst_cur and
// dst_prev.  first: step n0 = 0 is the first step (src_prev unused); the general
// recursion then also writes <L|phi_0> to slab nsteps (nsteps + 1 <= plan.chunk).
template <typename T>
cudaError_t launch_kpm_cluster(const DevH& H, int R, bool sym, const ClusterPlan& plan,
                               const vec2_t<T>* L, const vec2_t<T>* src_cur, const vec2_t<T>* src_prev,
                               vec2_t<T>* dst_cur, vec2_t<T>* dst_prev, double* ring, int nsteps, bool first,
                               cudaStream_t s);

// Reduce per-block partials of a KPM run into moments mu[r * r_stride + n].
//   first: partial [grid][R][A] of the first step (A = 2 sym, 4 gen)
//   ring:  partial slabs [ring][grid][R][2]; slab (slab0 + b) % ring belongs to step n0 + b
cudaError_t launch_reduce_first(const double* partial, int grid, int R, bool sym,
                                double2* mu, int64_t r_stride, int M, cudaStream_t s);
cudaError_t launch_reduce_ring(const double* ring, int slab0, int nslab, int ring_size,
                               int grid, int R, bool sym, int n0, double2* mu,
                               int64_t r_stride, int M, cudaStream_t s, bool first = false);

template <typename T>
struct ChainsT {
    using V2 = vec2_t<T>;
    const V2* cur[3] = {nullptr, nullptr, nullptr};
    const V2* prev[3] = {nullptr, nullptr, nullptr};
    V2* nxt[3] = {nullptr, nullptr, nullptr};
    V2* acc[3] = {nullptr, nullptr, nullptr};
    // commutator chain [X, T_m(H~)] applied to chain nch-1
    const V2* qcur = nullptr;
    const V2* qprev = nullptr;
    V2* qnxt = nullptr;
    V2* qacc = nullptr;             // null: accumulate into acc[0]
};

// Small instances: a whole Chebyshev-Bessel series (terms m = 1 .. nterms) in one
// cluster launch.  cr[m], ci[m] are the coefficients 2 J_m (s i)^m of term m (index 0
// unused); j0 = J_0.  Series longer than kClusterMaxTerms take the per-term launches.
constexpr int kClusterMaxTerms = 96;
struct SeriesCoef {
    double j0 = 0.0;
    double cr[kClusterMaxTerms + 1] = {0};
    double ci[kClusterMaxTerms + 1] = {0};
    int nterms = 0;
    int norm_chain = 0;             // chain whose result's squared norm is formed
    double2* norm_out = nullptr;    // [R] (||acc_r||^2, 0), or null for none
};

// Chooses the cluster plan of the series kernel for this H, R, nch and xc (cached per
// device); false when the instance is too large or no such cluster fits.
template <typename T>
bool evolve_cluster_plan(const DevH& H, int R, int nch, bool xc, ClusterPlan* plan);

// The series on the chains ch.cur[k] (inputs, not modified) into ch.acc[k] (and the
// commutator chain into ch.qacc, or into ch.acc[0] when null), in one cluster launch.
template <typename T>
cudaError_t launch_evolve_cluster(const DevH& H, int R, int nch, bool xc, const ClusterPlan& plan,
                                  const SeriesCoef& cf, const ChainsT<T>& ch, cudaStream_t s);

// One term m of the Chebyshev-Bessel series on nch plain chains (+ the commutator
// chain when xc).  first = the m = 1 step (also adds the J_0 term).  The grid is one
// resident wave of the selected kernel.
template <typename T>
cudaError_t launch_evolve(const DevH& H, int R, int nch, bool xc, bool first, double j0,
                          double cr, double ci, const ChainsT<T>& ch, cudaStream_t s);

// out = op(in): 0 H~, 1 [X, H~], 2 V = -(i E_max / hbar)[X, H~] (scale = E_max / hbar).
template <typename T>
cudaError_t launch_apply(const DevH& H, int R, int op, double scale, const vec2_t<T>* in,
                         vec2_t<T>* out, cudaStream_t s);

// out[r * r_stride] = <L_r|X_r> for the R vectors (partial: [grid][R][2] scratch).
template <typename T>
cudaError_t launch_dot(int64_t n_items, int R, const vec2_t<T>* L, const vec2_t<T>* X, double* partial,
                       int grid, double2* out, int64_t r_stride, cudaStream_t s);

// complex128 -> complex64, element-wise.
cudaError_t launch_to_c64(const double2* in, float2* out, int64_t n_items, cudaStream_t s);
cudaError_t launch_to_c128(const float2* in, double2* out, int64_t n_items, cudaStream_t s);

// Grid size (CTAs) for a streaming kernel over n_items = n * R complex items.
int stream_grid(int64_t n_items);

// Sets *flag (device int, cleared by the caller) when one of the n doubles at p is
// NaN or infinite; one kernel launch on stream s.
cudaError_t launch_nonfinite(const double* p, int64_t n, int* flag, cudaStream_t s);

// FP64 FMA throughput probe: grid size (CTAs), FMA instructions per launch, and one
// launch writing grid x 256 doubles to out.
int fp64_probe_grid();
double fp64_probe_fmas();
cudaError_t launch_fp64_probe(double* out, cudaStream_t s);

}  // namespace kg
