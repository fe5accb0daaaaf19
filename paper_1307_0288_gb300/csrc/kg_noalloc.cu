// DOS moments through an entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host framework that
// owns all device memory through its own allocator, processes that must not allocate
// once they are serving, or plug-ins whose device memory budget is fixed up front.
// kg_dos_moments_noalloc serves them: its scratch space is one file-scope device
// array of fixed size, reserved when the library's device code is loaded and held by
// every GPU that loads it until the process exits.  The caller provides inputs and
// outputs in device memory it already owns.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "kg_internal.h"

namespace kg {

static_assert(KG_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size must be a multiple of 256");

// The scratch array.  In host code this name is only a host-side stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress (see below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[KG_NOALLOC_SCRATCH_BYTES];

static constexpr int kNoallocRing = 32;   // partial-sum slabs reduced per launch
static constexpr int kMaxDevices = 64;

static std::mutex g_scratch_mutex;
static void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up once per
// device, with that device current.
static kg_status scratch_address(void** out) {
    int dev = 0;
    KG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(KG_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(KG_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return KG_OK;
}

// Neighbour table with "absent" (-1) redirected to the zero row n.
__global__ void sentinel_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t count,
                                int32_t n) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        const int32_t v = in[k];
        out[k] = (v < 0 || v >= n) ? n : v;
    }
}

// max |onsite[k]| over k < n as the bit pattern of a non-negative double (which orders
// like the value), NaN counted as +infinity; *out must start at 0.
__global__ void onsite_absmax_kernel(const double* __restrict__ onsite, int64_t n,
                                     unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double m = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const double a = fabs(onsite[k]);
        m = (a == a) ? fmax(m, a) : INFINITY;
    }
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace kg

using namespace kg;

extern "C" kg_status kg_dos_moments_noalloc(const int32_t* idx_dev, const double* onsite_dev,
                                            int64_t n_sites, double hopping, int n_vectors,
                                            int n_moments, const double* phi_dev, double* mu_dev,
                                            void* cuda_stream) {
    clear_error();
    const int R = n_vectors, M = n_moments;
    if (!idx_dev || !phi_dev || !mu_dev) return fail(KG_EINVAL, "idx_dev, phi_dev and mu_dev are required");
    if (n_sites < 1 || n_sites >= (int64_t)INT32_MAX - 1) return fail(KG_EINVAL, "n_sites out of range");
    if (R < 1 || R > 64 || (R & (R - 1))) return fail(KG_EINVAL, "n_vectors must be a power of two in 1..64");
    if (M < 1) return fail(KG_EINVAL, "n_moments must be >= 1");
    if (!(hopping != 0.0) || !(std::fabs(hopping) < 1.0 / 3.0))
        return fail(KG_EINVAL, "hopping must be the scaled value -gamma0/E_max, 0 < |hopping| < 1/3");
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t n = n_sites;
    const int grid = stream_grid(n * R);
    // scratch layout: neighbour table, three vector blocks of n+1 rows, partial sums
    const size_t b_idx = align256((size_t)3 * n * sizeof(int32_t));
    const size_t b_vec = align256((size_t)(n + 1) * R * sizeof(double2));
    const size_t b_first = align256((size_t)grid * R * 4 * sizeof(double));
    const size_t b_ring = align256((size_t)kNoallocRing * grid * R * 2 * sizeof(double));
    const size_t b_check = 256;   // max |onsite| and the non-finite flag
    const size_t need = b_idx + 3 * b_vec + b_first + b_ring + b_check;
    if (need > KG_NOALLOC_SCRATCH_BYTES)
        return fail(KG_EINVAL, "kg_dos_moments_noalloc: n_sites x n_vectors too large for the fixed scratch (" +
                                   std::to_string(need) + " bytes needed, " +
                                   std::to_string((size_t)KG_NOALLOC_SCRATCH_BYTES) + " available)");
    void* base = nullptr;
    KG_TRY(scratch_address(&base));
    char* p = (char*)base;
    int32_t* idx = (int32_t*)p;
    double2* phi0 = (double2*)(p + b_idx);
    double2* b0 = (double2*)(p + b_idx + b_vec);
    double2* b1 = (double2*)(p + b_idx + 2 * b_vec);
    double* first = (double*)(p + b_idx + 3 * b_vec);
    double* ring = (double*)(p + b_idx + 3 * b_vec + b_first);
    unsigned long long* onsite_max = (unsigned long long*)(p + b_idx + 3 * b_vec + b_first + b_ring);
    int* bad_flag = (int*)(onsite_max + 1);

    // The Chebyshev expansion needs the spectrum of H~ inside [-1, 1] (Eqs. 32-34); by
    // Gershgorin's theorem 3|h| + max|eps_n / E_max| < 1 guarantees it.
    if (onsite_dev) {
        KG_CUDA_TRY(cudaMemsetAsync(onsite_max, 0, sizeof(*onsite_max), s));
        onsite_absmax_kernel<<<stream_grid(n), 256, 0, s>>>(onsite_dev, n, onsite_max);
        KG_CUDA_TRY(cudaGetLastError());
        unsigned long long bits = 0;
        KG_CUDA_TRY(cudaMemcpyAsync(&bits, onsite_max, sizeof(bits), cudaMemcpyDeviceToHost, s));
        KG_CUDA_TRY(cudaStreamSynchronize(s));
        double emax_onsite = 0.0;
        std::memcpy(&emax_onsite, &bits, sizeof(emax_onsite));
        if (!(3.0 * std::fabs(hopping) + emax_onsite < 1.0))
            return fail(KG_EINVAL, "kg_dos_moments_noalloc: 3|hopping| + max|onsite| = " +
                                       std::to_string(3.0 * std::fabs(hopping) + emax_onsite) +
                                       " must be < 1 (the spectrum of H~ must lie inside [-1, 1])");
    }

    DevH H;
    H.idx = idx;
    H.istride = n;
    H.n = n;
    H.onsite = onsite_dev;
    H.h = hopping;

    // The array keeps the previous call's contents: clear the zero rows.
    const size_t row = (size_t)R * sizeof(double2);
    for (double2* v : {phi0, b0, b1})
        KG_CUDA_TRY(cudaMemsetAsync((char*)v + (size_t)n * row, 0, row, s));
    sentinel_kernel<<<stream_grid(3 * n), 256, 0, s>>>(idx_dev, idx, 3 * n, (int32_t)n);
    KG_CUDA_TRY(cudaGetLastError());
    KG_CUDA_TRY(cudaMemcpyAsync(phi0, phi_dev, (size_t)n * row, cudaMemcpyDeviceToDevice, s));

    double2* mu = (double2*)mu_dev;
    KG_CUDA_TRY(launch_kpm_sym<double>(H, R, true, phi0, nullptr, b1, first, grid, s));
    KG_CUDA_TRY(launch_reduce_first(first, grid, R, true, mu, M, M, s));
    const int steps = (M - 1) / 2;
    const double2* cur = b1;
    const double2* prev = phi0;
    double2* out = b0;
    int pending = 0, first_pending = 1;
    for (int k = 1; k <= steps; k++) {
        double* slab = ring + (int64_t)((k - 1) % kNoallocRing) * grid * R * 2;
        KG_CUDA_TRY(launch_kpm_sym<double>(H, R, false, cur, prev, out, slab, grid, s));
        if (++pending == kNoallocRing || k == steps) {
            KG_CUDA_TRY(launch_reduce_ring(ring, (first_pending - 1) % kNoallocRing, pending, kNoallocRing,
                                           grid, R, true, first_pending, mu, M, M, s));
            first_pending = k + 1;
            pending = 0;
        }
        const double2* nc = out;
        prev = cur;
        out = const_cast<double2*>(cur);
        cur = nc;
    }
    // moments that are NaN or infinite (non-finite inputs, or entries beyond 2^63) fail
    KG_CUDA_TRY(cudaMemsetAsync(bad_flag, 0, sizeof(int), s));
    KG_CUDA_TRY(launch_nonfinite(mu_dev, (int64_t)R * M * 2, bad_flag, s));
    int bad = 0;
    KG_CUDA_TRY(cudaMemcpyAsync(&bad, bad_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    KG_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad)
        return fail(KG_ENUMERIC, "kg_dos_moments_noalloc: non-finite moments (NaN/Inf inputs, or vector "
                                 "entries of magnitude 2^63 or more)");
    return KG_OK;
}
