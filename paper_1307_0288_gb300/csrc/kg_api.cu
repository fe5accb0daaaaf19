// GPU entry points of the C ABI: Hamiltonian handle, workspace, and the moment and
// time-evolution drivers (Algorithms 2, 3, 5, 6, 7 of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kg_internal.h"

namespace kg {

// Test hook: workspace allocations above this many bytes fail as if the device were out
// of memory (0 = no cap).  Injects KG_ENOMEM on the host, without a real allocation failure.
static std::atomic<unsigned long long> g_alloc_cap{0};

// Small instances run their moment recursion as one cluster launch per chunk of up to
// 256 steps (kg_set_small_persistent); 0 = one launch per step everywhere.
static std::atomic<int> g_small_persistent{1};

// Device buffer owned by the handle.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // Grows to at least `want` bytes; new memory is zero-filled (the zero row of every
    // vector block relies on it).
    kg_status ensure(size_t want, cudaStream_t s) {
        if (bytes >= want) return KG_OK;
        const unsigned long long cap = g_alloc_cap.load();
        if (cap && want > cap)
            return fail(KG_ENOMEM, "workspace allocation of " + std::to_string(want) + " bytes exceeds the test cap");
        release();
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(KG_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed");
        }
        bytes = want;
        KG_CUDA_TRY(cudaMemsetAsync(p, 0, want, s));
        return KG_OK;
    }
};

struct TimedPhase {
    cudaEvent_t a, b;
    int kind;   // 0 kpm, 1 evolve
};

}  // namespace kg

struct kg_hamiltonian {
    int kind = 0;
    int64_t nx = 0, ny = 0, n = 0, n_active = 0;
    double gamma0 = 0, bond = 0, emax = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    kg::DevBuf idx, onsite, parity;
    kg::DevH dev;
    // workspace
    static constexpr int kNumVec = 10;
    kg::DevBuf vec[kNumVec];
    kg::DevBuf part_first, part_ring, moments, flag, norms, norm_part;
    // pinned host staging for the end-of-run checks (non-finite flag and the norms)
    void* host_stage = nullptr;
    size_t host_stage_bytes = 0;
    // timing
    bool timing = false;
    std::vector<kg::TimedPhase> phases;
    std::vector<cudaEvent_t> spare_events;
    kg_timing counters{};
};

namespace kg {

const DevH& hamiltonian_dev(const kg_hamiltonian* h) { return h->dev; }
cudaStream_t hamiltonian_stream(const kg_hamiltonian* h) { return h->stream; }

static constexpr int kRing = 256;   // partial-sum slabs reduced per launch

static kg_status check_device(kg_hamiltonian* h) {
    int cur = -1;
    KG_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != h->device) KG_CUDA_TRY(cudaSetDevice(h->device));
    return KG_OK;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static bool valid_r(int r) { return r >= 1 && r <= 64 && (r & (r - 1)) == 0; }

static cudaEvent_t take_event(kg_hamiltonian* h) {
    if (!h->spare_events.empty()) {
        cudaEvent_t e = h->spare_events.back();
        h->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct PhaseTimer {
    kg_hamiltonian* h;
    int kind;
    cudaEvent_t a = nullptr;
    PhaseTimer(kg_hamiltonian* h_, int kind_) : h(h_), kind(kind_) {
        if (h->timing) {
            a = take_event(h);
            cudaEventRecord(a, h->stream);
        }
    }
    ~PhaseTimer() {
        if (h->timing && a) {
            cudaEvent_t b = take_event(h);
            cudaEventRecord(b, h->stream);
            h->phases.push_back({a, b, kind});
        }
    }
};

static size_t vec_bytes(const kg_hamiltonian* h, int R) {
    return (size_t)(h->n + 1) * (size_t)R * sizeof(double2);
}

// Makes `count` vector blocks of R columns available.  Row n of every block (the
// zero row that absent neighbours point at) is cleared on each call, since a block
// may have been used with another R before.
static kg_status ensure_vectors(kg_hamiltonian* h, int R, int count) {
    if (count > kg_hamiltonian::kNumVec) return fail(KG_EINVAL, "internal: too many vectors");
    const size_t want = vec_bytes(h, R);
    for (int k = 0; k < count; k++) {
        KG_TRY(h->vec[k].ensure(want, h->stream));
        KG_CUDA_TRY(cudaMemsetAsync((char*)h->vec[k].p + (size_t)h->n * R * sizeof(double2), 0,
                                    (size_t)R * sizeof(double2), h->stream));
    }
    return KG_OK;
}

static double2* V(kg_hamiltonian* h, int k) { return (double2*)h->vec[k].p; }

// Copies N rows of R vectors from a host or device source into a device block.
static kg_status copy_in(kg_hamiltonian* h, const double* src, double2* dst, int R) {
    const size_t bytes = (size_t)h->n * R * sizeof(double2);
    KG_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                                is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                h->stream));
    return KG_OK;
}

static kg_status copy_out(kg_hamiltonian* h, const void* src, double* dst, size_t bytes) {
    KG_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes,
                                is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return KG_OK;
}

// KG_ENUMERIC when a result on the device is not finite: non-finite input entries, or
// FP64 vector entries beyond the range of the double-float inner products (2^63).
static kg_status check_finite(kg_hamiltonian* h, const void* dev, size_t n_doubles) {
    KG_TRY(h->flag.ensure(sizeof(int), h->stream));
    KG_CUDA_TRY(cudaMemsetAsync(h->flag.p, 0, sizeof(int), h->stream));
    KG_CUDA_TRY(launch_nonfinite((const double*)dev, (int64_t)n_doubles, (int*)h->flag.p, h->stream));
    h->counters.other_launches += 1;
    int bad = 0;
    KG_CUDA_TRY(cudaMemcpyAsync(&bad, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (bad)
        return fail(KG_ENUMERIC, "non-finite moments: the input vectors hold NaN/Inf entries or FP64 entries "
                                 "of magnitude 2^63 or more");
    return KG_OK;
}

static kg_status ensure_partials(kg_hamiltonian* h, int R, int grid) {
    KG_TRY(h->part_first.ensure((size_t)grid * R * 4 * sizeof(double), h->stream));
    KG_TRY(h->part_ring.ensure((size_t)kRing * grid * R * 2 * sizeof(double), h->stream));
    return KG_OK;
}

// ---------------------------------------------------------------------------------
// KPM moments (Algorithm 5) of one pair (phi_L, phi_R) block of R vectors.
//   sym: phi_L == phi_R, two moments per recursion step (Chebyshev doubling)
//   buffers b0, b1: scratch vector blocks; phi_r is not modified.
//   mu: device [R][r_stride] double2, moments written at mu[r*r_stride + n], n < M.
// ---------------------------------------------------------------------------------
template <typename T>
static kg_status kpm_moments(kg_hamiltonian* h, int R, int M, bool sym, const vec2_t<T>* phi_l,
                             const vec2_t<T>* phi_r, vec2_t<T>* b0, vec2_t<T>* b1, double2* mu,
                             int64_t r_stride) {
    using V2 = vec2_t<T>;
    PhaseTimer t(h, 0);
    const int grid = kpm_grid<T>(h->dev, R, sym);
    const int steps = sym ? (M - 1) / 2 : M - 2;   // recursion steps after the first
    ClusterPlan plan;
    const bool cluster = steps > 0 && g_small_persistent.load() && kpm_cluster_plan<T>(h->dev, R, sym, &plan);
    KG_TRY(ensure_partials(h, R, cluster ? std::max(grid, plan.grid) : grid));
    double* pf = (double*)h->part_first.p;
    double* ring = (double*)h->part_ring.p;
    cudaStream_t s = h->stream;
    if (cluster) {
        // small instance: the first step and up to a chunk of further steps per cluster launch,
        // vectors in shared memory.  The chunk's last phi_n and phi_{n-1} land where the
        // per-step loop's rotation would put them: after the first step (phi_1 into b1,
        // phi_0 staying in phi_r) every later step writes in place over phi_{n-1}.
        static_assert(kClusterMaxChunk <= kRing, "a chunk's partial slabs must fit the ring");
        const int total = steps + 1;   // the first step and the `steps` further ones
        const V2* cur = phi_r;
        const V2* prev = nullptr;
        V2* out = b1;
        for (int n0 = 0; n0 < total;) {
            const bool first = n0 == 0;
            const int room = plan.chunk - ((first && !sym) ? 1 : 0);
            const int cnt = std::min(room, total - n0);
            const V2* src_cur = cur;
            const V2* src_prev = prev;
            for (int k = 0; k < cnt; k++) {   // the per-step loop's rotation, replayed on the host
                const int n = n0 + k;
                const V2* new_cur = out;
                prev = cur;
                out = n == 0 ? b0 : const_cast<V2*>(cur);
                cur = new_cur;
            }
            // cnt >= 2 whenever the chunk starts with the first step (steps > 0), so its final
            // phi_n and phi_{n-1} are both in b0 / b1 and phi_r is never written
            KG_CUDA_TRY(launch_kpm_cluster<T>(h->dev, R, sym, plan, phi_l, src_cur, src_prev, const_cast<V2*>(cur),
                                              const_cast<V2*>(prev), ring, cnt, first, s));
            KG_CUDA_TRY(launch_reduce_ring(ring, 0, cnt + ((first && !sym) ? 1 : 0), kRing, plan.grid, R, sym, n0,
                                           mu, r_stride, M, s, first));
            h->counters.kpm_launches += 1;
            h->counters.other_launches += 1;
            h->counters.kpm_site_steps += (double)h->n * R * cnt;
            n0 += cnt;
        }
        return KG_OK;
    }
    // first step: phi_1 = H~ phi_0 (into b1), moments 0 and 1
    if (sym) KG_CUDA_TRY(launch_kpm_sym<T>(h->dev, R, true, phi_r, nullptr, b1, pf, grid, s));
    else KG_CUDA_TRY(launch_kpm_gen<T>(h->dev, R, true, phi_l, phi_r, nullptr, b1, pf, grid, s));
    KG_CUDA_TRY(launch_reduce_first(pf, grid, R, sym, mu, r_stride, M, s));
    h->counters.kpm_launches += 1;
    h->counters.other_launches += 1;
    h->counters.kpm_site_steps += (double)h->n * R;
    // remaining steps n = 1..S: phi_{n+1} = 2H~phi_n - phi_{n-1}
    const V2* cur = b1;
    const V2* prev = phi_r;
    V2* out = b0;
    int pending = 0, first_pending = 1;
    for (int n = 1; n <= steps; n++) {
        double* slab = ring + (int64_t)((n - 1) % kRing) * grid * R * 2;
        if (sym) KG_CUDA_TRY(launch_kpm_sym<T>(h->dev, R, false, cur, prev, out, slab, grid, s));
        else KG_CUDA_TRY(launch_kpm_gen<T>(h->dev, R, false, phi_l, cur, prev, out, slab, grid, s));
        h->counters.kpm_launches += 1;
        h->counters.kpm_site_steps += (double)h->n * R;
        pending++;
        if (pending == kRing || n == steps) {
            KG_CUDA_TRY(launch_reduce_ring(ring, (first_pending - 1) % kRing, pending, kRing, grid, R,
                                           sym, first_pending, mu, r_stride, M, s));
            h->counters.other_launches += 1;
            first_pending = n + 1;
            pending = 0;
        }
        // rotate: the new phi_n is `out`; phi_{n-1} becomes the next output (in place)
        const V2* new_cur = out;
        prev = cur;
        out = const_cast<V2*>(cur);
        cur = new_cur;
    }
    return KG_OK;
}

// Bessel coefficients of one time step and the (s i)^m phase factors (Eq. 36).
struct Series {
    std::vector<double> j;
    int np = 0;
};

static kg_status series_for_tau(double tau, double tol, Series* out) {
    if (!(tol > 0) || !(tol < 1)) return fail(KG_EINVAL, "bessel_tol must be in (0, 1)");
    const int cap = (int)tau + 400;
    out->j.assign((size_t)cap, 0.0);
    KG_TRY(bessel_series(tau, tol, cap, out->j.data(), &out->np));
    return KG_OK;
}

static kg_status series_for(kg_hamiltonian* h, double dt, double tol, Series* out) {
    if (!(dt > 0) || !std::isfinite(dt)) return fail(KG_EINVAL, "dt must be positive");
    if (!(tol > 0) || !(tol < 1)) return fail(KG_EINVAL, "bessel_tol must be in (0, 1)");
    const double tau = h->emax * dt / h->gamma0;   // tau = E_max dt / hbar, dt in hbar/gamma0
    const int cap = (int)tau + 400;
    out->j.assign((size_t)cap, 0.0);
    KG_TRY(bessel_series(tau, tol, cap, out->j.data(), &out->np));
    return KG_OK;
}

// 2 J_m (s i)^m as (cr, ci); s = -1 for U(+dt), +1 for U(-dt).
static void term_coef(const Series& ser, int m, int s, double* cr, double* ci) {
    const double f = 2.0 * ser.j[(size_t)m];
    switch (m & 3) {
        case 0: *cr = f; *ci = 0; break;
        case 1: *cr = 0; *ci = f * s; break;
        case 2: *cr = -f; *ci = 0; break;
        default: *cr = 0; *ci = -f * s; break;
    }
}

// Runs the Chebyshev-Bessel series over prepared chains; rotates chain pointers.
//   chains: nch plain chains with cur = input (p_0), nxt buffers for p_1 given in
//   p1[k], accumulators acc[k]; xc: commutator chain of the last plain chain with
//   buffers q1, q0 (q0 receives q_2), routed to qacc (null = acc[0]).
// The plain-chain inputs are overwritten from m = 2 on (p_m replaces p_{m-2}).
template <typename T>
static kg_status block_norms(kg_hamiltonian* h, int R, const vec2_t<T>* x, int slot);

// norm_slot >= 0: also records ||acc[norm_chain]||^2 per vector in slot norm_slot of
// h->norms (the unitarity check), inside the cluster launch when that path runs.
template <typename T>
static kg_status run_series(kg_hamiltonian* h, int R, const Series& ser, int s, int nch, bool xc,
                            vec2_t<T>* const* in, vec2_t<T>* const* p1, vec2_t<T>* const* acc,
                            vec2_t<T>* q1, vec2_t<T>* q0, vec2_t<T>* qacc, int norm_slot = -1,
                            int norm_chain = 0) {
    using V2 = vec2_t<T>;
    PhaseTimer t(h, 1);
    ChainsT<T> ch;
    const int nterms = std::max(ser.np - 1, 1);   // the m = 1 term runs even when N_p = 1 (with c_1 = 0)
    ClusterPlan plan;
    if (g_small_persistent.load() && nterms <= kClusterMaxTerms &&
        evolve_cluster_plan<T>(h->dev, R, nch, xc, &plan)) {
        // small instance: the whole series in one cluster launch, chains in shared memory;
        // the inputs are left unchanged
        SeriesCoef cf;
        cf.j0 = ser.j[0];
        cf.nterms = nterms;
        for (int m = 1; m <= nterms; m++)
            if (m < ser.np) term_coef(ser, m, s, &cf.cr[m], &cf.ci[m]);
        for (int k = 0; k < nch; k++) {
            ch.cur[k] = in[k];
            ch.acc[k] = acc[k];
        }
        if (xc) ch.qacc = qacc;
        if (norm_slot >= 0) {
            cf.norm_chain = norm_chain;
            cf.norm_out = (double2*)h->norms.p + (size_t)norm_slot * R;
        }
        KG_CUDA_TRY(launch_evolve_cluster<T>(h->dev, R, nch, xc, plan, cf, ch, h->stream));
        h->counters.evolve_launches += 1;
        h->counters.evolve_site_steps += (double)h->n * R * (nch + (xc ? 1 : 0)) * nterms;
        return KG_OK;
    }
    V2* cur[3];
    V2* prv[3];
    for (int k = 0; k < nch; k++) {
        ch.cur[k] = in[k];
        ch.nxt[k] = p1[k];
        ch.acc[k] = acc[k];
        cur[k] = p1[k];
        prv[k] = in[k];
    }
    if (xc) {
        ch.qnxt = q1;
        ch.qacc = qacc;
    }
    double cr = 0, ci = 0;
    if (ser.np > 1) term_coef(ser, 1, s, &cr, &ci);
    // first step: p_1 = H~ p_0, acc = J_0 p_0 + c_1 p_1 (c_1 = 0 when N_p = 1)
    KG_CUDA_TRY(launch_evolve<T>(h->dev, R, nch, xc, true, ser.j[0], cr, ci, ch, h->stream));
    h->counters.evolve_launches += 1;
    h->counters.evolve_site_steps += (double)h->n * R * (nch + (xc ? 1 : 0));
    V2* qc = q1;
    V2* qp = nullptr;
    V2* qn = q0;
    for (int m = 2; m < ser.np; m++) {
        term_coef(ser, m, s, &cr, &ci);
        for (int k = 0; k < nch; k++) {
            ch.cur[k] = cur[k];
            ch.prev[k] = prv[k];
            ch.nxt[k] = prv[k];   // in place: p_m overwrites p_{m-2}
        }
        if (xc) {
            ch.qcur = qc;
            ch.qprev = qp;
            ch.qnxt = qn;
        }
        KG_CUDA_TRY(launch_evolve<T>(h->dev, R, nch, xc, false, 0.0, cr, ci, ch, h->stream));
        h->counters.evolve_launches += 1;
        h->counters.evolve_site_steps += (double)h->n * R * (nch + (xc ? 1 : 0));
        for (int k = 0; k < nch; k++) {
            V2* t2 = prv[k];
            prv[k] = cur[k];
            cur[k] = t2;
        }
        if (xc) {
            // q_m now sits in qn; q_{m+1} will overwrite q_{m-1}
            V2* newc = qn;
            qp = qc;
            qc = newc;
            qn = qp;
        }
    }
    if (norm_slot >= 0) KG_TRY(block_norms<T>(h, R, acc[norm_chain], norm_slot));
    return KG_OK;
}

// Typed view of workspace vector block k.
template <typename T>
static vec2_t<T>* VT(kg_hamiltonian* h, int k) { return (vec2_t<T>*)h->vec[k].p; }

// Stages the caller's complex128 vectors (host or device) into block `dst` of
// precision T; `tmp` is a scratch block used for the complex64 conversion.
template <typename T>
static kg_status stage_input(kg_hamiltonian* h, const double* phi, int R, int dst, int tmp) {
    if constexpr (sizeof(T) == sizeof(double)) {
        (void)tmp;
        return copy_in(h, phi, V(h, dst), R);
    } else {
        KG_TRY(copy_in(h, phi, V(h, tmp), R));
        KG_CUDA_TRY(launch_to_c64(V(h, tmp), VT<float>(h, dst), h->n * R, h->stream));
        h->counters.other_launches += 1;
        // the zero row of the complex64 layout
        KG_CUDA_TRY(cudaMemsetAsync(VT<float>(h, dst) + h->n * R, 0, (size_t)R * sizeof(float2), h->stream));
        return KG_OK;
    }
}

// Zero rows of the complex64 layout for the listed blocks (ensure_vectors clears the
// complex128 position of row n, which is a different byte offset).
template <typename T>
static kg_status clear_zero_rows(kg_hamiltonian* h, int R, int count) {
    if constexpr (sizeof(T) != sizeof(double)) {
        for (int k = 0; k < count; k++)
            KG_CUDA_TRY(cudaMemsetAsync(VT<T>(h, k) + h->n * R, 0, (size_t)R * sizeof(vec2_t<T>), h->stream));
    }
    return KG_OK;
}

template <typename T>
static kg_status dos_impl(kg_hamiltonian* h, int R, int M, const double* phi) {
    KG_TRY(ensure_vectors(h, R, 4));
    KG_TRY(stage_input<T>(h, phi, R, 0, 3));
    KG_TRY(clear_zero_rows<T>(h, R, 4));   // after staging: it writes complex128 rows into block 3
    return kpm_moments<T>(h, R, M, true, VT<T>(h, 0), VT<T>(h, 0), VT<T>(h, 1), VT<T>(h, 2),
                          (double2*)h->moments.p, M);
}

// ||x_r||^2 of the R vectors of a block into norms[slot][r].x (device).
template <typename T>
static kg_status block_norms(kg_hamiltonian* h, int R, const vec2_t<T>* x, int slot) {
    const int grid = stream_grid(h->n * R);
    KG_TRY(h->norm_part.ensure((size_t)grid * R * 2 * sizeof(double), h->stream));
    KG_CUDA_TRY(launch_dot<T>(h->n * R, R, x, x, (double*)h->norm_part.p, grid,
                              (double2*)h->norms.p + (size_t)slot * R, 1, h->stream));
    h->counters.other_launches += 2;
    return KG_OK;
}

// U(dt) is unitary (Eq. 36): the norm of the evolved vector must not drift.  finish_run
// fails with KG_ENUMERIC when any of the recorded norms differs from slot 0 by more than
// 1e-10 (FP64) or 1e-3 (complex64) relative, e.g. for a Bessel truncation far too loose.
// End of a time loop with one synchronisation: the non-finite check of the moments, the
// copy of the norm record and of the flag into pinned host memory, and the copy of the
// moments to the caller's buffer are all queued, then the stream is synchronised once and
// the unitarity and finiteness conditions are evaluated (KG_ENUMERIC, as check_finite does
// for the other entry points; the caller's buffer then holds the offending moments).
template <typename T>
static kg_status finish_run(kg_hamiltonian* h, int R, int slots, double* mu_out, size_t n_doubles) {
    const size_t want = 64 + (size_t)slots * R * sizeof(double2);
    if (h->host_stage_bytes < want) {
        if (h->host_stage) cudaFreeHost(h->host_stage);
        h->host_stage = nullptr;
        h->host_stage_bytes = 0;
        KG_CUDA_TRY(cudaMallocHost(&h->host_stage, want));
        h->host_stage_bytes = want;
    }
    int* bad = (int*)h->host_stage;
    double2* nrm = (double2*)((char*)h->host_stage + 64);
    KG_TRY(h->flag.ensure(sizeof(int), h->stream));
    KG_CUDA_TRY(cudaMemsetAsync(h->flag.p, 0, sizeof(int), h->stream));
    KG_CUDA_TRY(launch_nonfinite((const double*)h->moments.p, (int64_t)n_doubles, (int*)h->flag.p, h->stream));
    h->counters.other_launches += 1;
    KG_CUDA_TRY(cudaMemcpyAsync(bad, h->flag.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    if (slots > 0)
        KG_CUDA_TRY(cudaMemcpyAsync(nrm, h->norms.p, (size_t)slots * R * sizeof(double2), cudaMemcpyDeviceToHost,
                                    h->stream));
    KG_CUDA_TRY(cudaMemcpyAsync(mu_out, h->moments.p, n_doubles * sizeof(double),
                                is_device_ptr(mu_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    const double tol = sizeof(T) == sizeof(double) ? 1e-10 : 1e-3;
    for (int r = 0; r < R; r++) {
        const double n0 = nrm[(size_t)r].x;
        for (int t = 1; t < slots; t++) {
            const double nt = nrm[(size_t)t * R + r].x;
            if (!std::isfinite(nt) || std::fabs(nt - n0) > tol * std::max(n0, 1e-300))
                return fail(KG_ENUMERIC, "norm drift of the evolved vector " + std::to_string(r) + ": |phi|^2 " +
                                             std::to_string(n0) + " -> " + std::to_string(nt) + " after " +
                                             std::to_string(t) + " steps (U(dt) must be unitary; bessel_tol?)");
        }
    }
    if (*bad)
        return fail(KG_ENUMERIC, "non-finite moments: the input vectors hold NaN/Inf entries or FP64 entries "
                                 "of magnitude 2^63 or more");
    return KG_OK;
}

// Writes block `src` (precision T) to the caller's complex128 buffer (host or device);
// complex64 goes through the scratch block `tmp`.
template <typename T>
static kg_status state_out(kg_hamiltonian* h, int R, const vec2_t<T>* src, int tmp, double* dst) {
    const size_t bytes = (size_t)h->n * R * sizeof(double2);
    const void* from = src;
    if constexpr (sizeof(T) != sizeof(double)) {
        KG_CUDA_TRY(launch_to_c128(src, V(h, tmp), h->n * R, h->stream));
        h->counters.other_launches += 1;
        from = V(h, tmp);
    }
    KG_CUDA_TRY(cudaMemcpyAsync(dst, from, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream));
    return KG_OK;
}

// VAC time loop (Algorithm 2, Eqs. 42-43) on the state (A, B), A = U^dagger(t) phi,
// B = U^dagger(t) V phi.  Fresh run (resume = false): A = phi, B = V phi, moments at
// t_0 .. t_{NC-1}.  Resume: the state (a_in, b_in; b_in null means V a_in) is advanced NC
// steps, with the moments after each step; the final state goes to (a_out, b_out) if given.
template <typename T>
static kg_status vac_impl(kg_hamiltonian* h, int R, int M, int NC, const Series& ser, const double* a_in,
                          const double* b_in, bool resume, double* a_out, double* b_out, double* mu_out) {
    using V2 = vec2_t<T>;
    // blocks: 0 A, 1 B, 2 A', 3 B', 4 L, 5 p1(A), 6 p1(B), 7 kpm b0, 8 kpm b1
    KG_TRY(ensure_vectors(h, R, 9));
    V2 *A = VT<T>(h, 0), *B = VT<T>(h, 1), *A2 = VT<T>(h, 2), *B2 = VT<T>(h, 3), *L = VT<T>(h, 4);
    const double vscale = h->emax / kHbarEvFs;
    KG_TRY(stage_input<T>(h, a_in, R, 0, 7));
    if (b_in) KG_TRY(stage_input<T>(h, b_in, R, 1, 7));
    KG_TRY(clear_zero_rows<T>(h, R, 9));   // after staging: it writes complex128 rows into block 7
    if (!b_in) {
        KG_CUDA_TRY(launch_apply<T>(h->dev, R, 2, vscale, A, B, h->stream));   // B = V phi
        h->counters.other_launches += 1;
    }
    const int steps = resume ? NC : NC - 1;
    KG_TRY(h->norms.ensure((size_t)(steps + 1) * R * sizeof(double2), h->stream));
    KG_TRY(block_norms<T>(h, R, A, 0));
    double2* mu = (double2*)h->moments.p;
    int slot = 0;
    for (int t = 0; t < NC; t++) {
        if (t > 0 || resume) {
            // A <- U(-dt) A, B <- U(-dt) B  (Eqs. 42-43)
            V2* in[2] = {A, B};
            V2* p1[2] = {VT<T>(h, 5), VT<T>(h, 6)};
            V2* acc[2] = {A2, B2};
            // A' = U(-dt) A is chain 0; its norm goes to the next slot
            KG_TRY(run_series<T>(h, R, ser, +1, 2, false, in, p1, acc, nullptr, nullptr, nullptr, ++slot, 0));
            std::swap(A, A2);
            std::swap(B, B2);
        }
        KG_CUDA_TRY(launch_apply<T>(h->dev, R, 2, vscale, A, L, h->stream));   // L = V A
        h->counters.other_launches += 1;
        KG_TRY(kpm_moments<T>(h, R, M, false, L, B, VT<T>(h, 7), VT<T>(h, 8), mu + (int64_t)t * M,
                              (int64_t)NC * M));
    }
    if (a_out) KG_TRY(state_out<T>(h, R, A, 7, a_out));
    if (b_out) KG_TRY(state_out<T>(h, R, B, 8, b_out));
    return finish_run<T>(h, R, slot + 1, mu_out, (size_t)R * NC * M * 2);
}

// MSD time loop (Algorithm 3, Eq. 44) on the state (psi, xi), psi = U(t) phi,
// xi = [X, U(t)] phi.  Fresh run: psi = phi, xi = 0, moments at t_0 (zero) .. t_{NC-1}.
// Resume: the state (psi_in, xi_in; xi_in null means 0) is advanced NC steps, with the
// moments after each step; the final state goes to (psi_out, xi_out) if given.
template <typename T>
static kg_status msd_impl(kg_hamiltonian* h, int R, int M, int NC, const Series& ser, const double* psi_in,
                          const double* xi_in, bool resume, double* psi_out, double* xi_out, double* mu_out) {
    using V2 = vec2_t<T>;
    // blocks: 0 psi, 1 xi, 2 psi', 3 xi', 4 p1(xi), 5 p1(psi), 6 q1, 7 q0
    KG_TRY(ensure_vectors(h, R, 8));
    V2 *psi = VT<T>(h, 0), *xi = VT<T>(h, 1), *psi2 = VT<T>(h, 2), *xi2 = VT<T>(h, 3);
    KG_TRY(stage_input<T>(h, psi_in, R, 0, 7));
    if (xi_in) KG_TRY(stage_input<T>(h, xi_in, R, 1, 7));
    KG_TRY(clear_zero_rows<T>(h, R, 8));   // after staging: it writes complex128 rows into block 7
    if (!xi_in) KG_CUDA_TRY(cudaMemsetAsync(xi, 0, vec_bytes(h, R), h->stream));   // [X, U(0)] = 0
    double2* mu = (double2*)h->moments.p;
    const int t0 = resume ? 0 : 1;
    if (!resume) KG_CUDA_TRY(cudaMemsetAsync(mu, 0, (size_t)R * NC * M * sizeof(double2), h->stream));
    KG_TRY(h->norms.ensure((size_t)(NC - t0 + 1) * R * sizeof(double2), h->stream));
    KG_TRY(block_norms<T>(h, R, psi, 0));
    for (int t = t0; t < NC; t++) {
        // xi <- U(dt) xi + [X, U(dt)] psi ;  psi <- U(dt) psi  (Eq. 44)
        V2* in[2] = {xi, psi};
        V2* p1[2] = {VT<T>(h, 4), VT<T>(h, 5)};
        V2* acc[2] = {xi2, psi2};
        // psi' = U(dt) psi is chain 1; its norm goes to slot t - t0 + 1
        KG_TRY(run_series<T>(h, R, ser, -1, 2, true, in, p1, acc, VT<T>(h, 6), VT<T>(h, 7), nullptr, t - t0 + 1, 1));
        std::swap(xi, xi2);
        std::swap(psi, psi2);
        // moments of xi; scratch: the now-free chain buffers 4 and 5
        KG_TRY(kpm_moments<T>(h, R, M, true, xi, xi, VT<T>(h, 4), VT<T>(h, 5), mu + (int64_t)t * M,
                              (int64_t)NC * M));
    }
    if (psi_out) KG_TRY(state_out<T>(h, R, psi, 6, psi_out));
    if (xi_out) KG_TRY(state_out<T>(h, R, xi, 7, xi_out));
    return finish_run<T>(h, R, NC - t0 + 1, mu_out, (size_t)R * NC * M * 2);
}

static kg_status check_run(const kg_hamiltonian* h, const kg_run* run, bool need_time) {
    if (!h) return fail(KG_EINVAL, "hamiltonian is NULL");
    if (!run) return fail(KG_EINVAL, "run is NULL");
    if (run->n_moments < 1) return fail(KG_EINVAL, "n_moments must be >= 1");
    if (!valid_r(run->n_vectors)) return fail(KG_EINVAL, "n_vectors must be a power of two in 1..64");
    if (run->precision != KG_FP64 && run->precision != KG_C64) return fail(KG_EINVAL, "unknown precision");
    if (need_time && run->n_times < 1) return fail(KG_EINVAL, "n_times must be >= 1");
    return KG_OK;
}

static kg_status ensure_moments(kg_hamiltonian* h, size_t count) {
    return h->moments.ensure(count * sizeof(double2), h->stream);
}

}  // namespace kg

using namespace kg;

extern "C" {

kg_status kg_build_hamiltonian(const kg_lattice* lattice, const int64_t* vacancies,
                               int64_t n_vacancies, const double* onsite_ev, void* cuda_stream,
                               kg_hamiltonian** out) {
    clear_error();
    if (!out) return fail(KG_EINVAL, "out is NULL");
    *out = nullptr;
    HostLattice hl;
    KG_TRY(build_host_lattice(lattice, vacancies, n_vacancies, &hl));
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(KG_ENODEV, "no CUDA device available");
    }
    const int64_t n = hl.n;
    double max_eps = 0.0;
    if (onsite_ev) {
        for (int64_t k = 0; k < n; k++) {
            if (!std::isfinite(onsite_ev[k])) return fail(KG_EINVAL, "onsite energy not finite");
            max_eps = std::fmax(max_eps, std::fabs(onsite_ev[k]));
        }
    }
    if (!(3.0 * lattice->gamma0_ev + max_eps < lattice->emax_ev))
        return fail(KG_EINVAL, "emax_ev must exceed 3 gamma0 + max |eps|");
    kg_hamiltonian* h = new (std::nothrow) kg_hamiltonian();
    if (!h) return fail(KG_ENOMEM, "host allocation failed");
    h->kind = hl.kind;
    h->nx = hl.nx;
    h->ny = hl.ny;
    h->n = n;
    h->n_active = hl.n_active;
    h->gamma0 = lattice->gamma0_ev;
    h->bond = lattice->bond_nm;
    h->emax = lattice->emax_ev;
    h->stream = (cudaStream_t)cuda_stream;
    auto bail = [&](kg_status st) {
        kg_destroy_hamiltonian(h);
        return st;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(fail(KG_ENODEV, "cudaGetDevice failed"));
    // neighbour table with the sentinel pointing at the zero row n
    std::vector<int32_t> idx(hl.idx.size());
    for (size_t k = 0; k < idx.size(); k++) idx[k] = hl.idx[k] < 0 ? (int32_t)n : hl.idx[k];
    kg_status st = h->idx.ensure(idx.size() * sizeof(int32_t), h->stream);
    if (st != KG_OK) return bail(st);
    if (cudaMemcpyAsync(h->idx.p, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                        h->stream) != cudaSuccess)
        return bail(fail(KG_ECUDA, "upload of the neighbour table failed"));
    h->dev.idx = (const int32_t*)h->idx.p;
    h->dev.istride = n;
    h->dev.n = n;
    h->dev.h = -lattice->gamma0_ev / lattice->emax_ev;
    for (int p = 0; p < 2; p++)
        for (int k = 0; k < 3; k++)
            h->dev.dh[p][k] = slot_displacement(hl.kind, lattice->bond_nm, p, k) * h->dev.h;
    h->dev.ytransport = (hl.kind == KG_AGNR);
    if (onsite_ev) {
        // eps_n / E_max and, after it, 2 eps_n / E_max (exact): the recursion steps after the
        // first read the doubled value instead of doubling it on the DP pipe
        std::vector<double> e(2 * ((size_t)n + 1), 0.0);
        for (int64_t k = 0; k < n; k++) {
            e[(size_t)k] = hl.removed[(size_t)k] ? 0.0 : onsite_ev[k] / lattice->emax_ev;
            e[(size_t)n + 1 + (size_t)k] = 2.0 * e[(size_t)k];
        }
        st = h->onsite.ensure(e.size() * sizeof(double), h->stream);
        if (st != KG_OK) return bail(st);
        if (cudaMemcpyAsync(h->onsite.p, e.data(), e.size() * sizeof(double), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
            return bail(fail(KG_ECUDA, "upload of on-site energies failed"));
        KG_CUDA_TRY(cudaStreamSynchronize(h->stream));   // the host array goes out of scope
        h->dev.onsite = (const double*)h->onsite.p;
        h->dev.onsite2 = (const double*)h->onsite.p + (n + 1);
    }
    if (h->dev.ytransport) {
        st = h->parity.ensure((size_t)n + 1, h->stream);
        if (st != KG_OK) return bail(st);
        if (cudaMemcpyAsync(h->parity.p, hl.parity.data(), (size_t)n, cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess)
            return bail(fail(KG_ECUDA, "upload of the parity table failed"));
        h->dev.parity = (const uint8_t*)h->parity.p;
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return bail(fail(KG_ECUDA, std::string("build: ") + cudaGetErrorString(cudaGetLastError())));
    *out = h;
    return KG_OK;
}

kg_status kg_hamiltonian_info(const kg_hamiltonian* h, int64_t* n_sites, int64_t* n_active,
                              double* emax_ev, double* area_nm2) {
    if (!h) return fail(KG_EINVAL, "hamiltonian is NULL");
    if (n_sites) *n_sites = h->n;
    if (n_active) *n_active = h->n_active;
    if (emax_ev) *emax_ev = h->emax;
    if (area_nm2) *area_nm2 = (std::sqrt(3.0) * h->nx * h->bond / 2.0) * (1.5 * h->ny * h->bond);
    return KG_OK;
}

void kg_destroy_hamiltonian(kg_hamiltonian* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->host_stage) cudaFreeHost(h->host_stage);
    h->host_stage = nullptr;
    h->idx.release();
    h->onsite.release();
    h->parity.release();
    for (auto& v : h->vec) v.release();
    h->part_first.release();
    h->part_ring.release();
    h->moments.release();
    h->flag.release();
    h->norms.release();
    h->norm_part.release();
    for (auto& p : h->phases) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : h->spare_events) cudaEventDestroy(e);
    delete h;
}

kg_status kg_dos_moments(kg_hamiltonian* h, const kg_run* run, const double* phi, double* mu_out) {
    clear_error();
    KG_TRY(check_run(h, run, false));
    if (!phi || !mu_out) return fail(KG_EINVAL, "phi and mu_out must not be NULL");
    KG_TRY(check_device(h));
    const int R = run->n_vectors, M = run->n_moments;
    KG_TRY(ensure_moments(h, (size_t)R * M));
    if (run->precision == KG_C64) KG_TRY(dos_impl<float>(h, R, M, phi));
    else KG_TRY(dos_impl<double>(h, R, M, phi));
    KG_TRY(check_finite(h, h->moments.p, (size_t)R * M * 2));
    return copy_out(h, h->moments.p, mu_out, (size_t)R * M * sizeof(double2));
}

kg_status kg_vac(kg_hamiltonian* h, const kg_run* run, const double* phi, double* mu_out) {
    clear_error();
    KG_TRY(check_run(h, run, true));
    if (!phi || !mu_out) return fail(KG_EINVAL, "phi and mu_out must not be NULL");
    KG_TRY(check_device(h));
    const int R = run->n_vectors, M = run->n_moments, NC = run->n_times;
    Series ser;
    if (NC > 1) KG_TRY(series_for(h, run->dt, run->bessel_tol, &ser));
    KG_TRY(ensure_moments(h, (size_t)R * NC * M));
    if (run->precision == KG_C64) return vac_impl<float>(h, R, M, NC, ser, phi, nullptr, false, nullptr, nullptr, mu_out);
    return vac_impl<double>(h, R, M, NC, ser, phi, nullptr, false, nullptr, nullptr, mu_out);
}

kg_status kg_msd(kg_hamiltonian* h, const kg_run* run, const double* phi, double* mu_out) {
    clear_error();
    KG_TRY(check_run(h, run, true));
    if (!phi || !mu_out) return fail(KG_EINVAL, "phi and mu_out must not be NULL");
    KG_TRY(check_device(h));
    const int R = run->n_vectors, M = run->n_moments, NC = run->n_times;
    Series ser;
    if (NC > 1) KG_TRY(series_for(h, run->dt, run->bessel_tol, &ser));
    KG_TRY(ensure_moments(h, (size_t)R * NC * M));
    if (run->precision == KG_C64) return msd_impl<float>(h, R, M, NC, ser, phi, nullptr, false, nullptr, nullptr, mu_out);
    return msd_impl<double>(h, R, M, NC, ser, phi, nullptr, false, nullptr, nullptr, mu_out);
}

kg_status kg_vac_resume(kg_hamiltonian* h, const kg_run* run, const double* a, const double* b, double* mu_out,
                        double* a_out, double* b_out) {
    clear_error();
    KG_TRY(check_run(h, run, true));
    if (!a || !mu_out) return fail(KG_EINVAL, "a and mu_out must not be NULL");
    if ((a_out == nullptr) != (b_out == nullptr)) return fail(KG_EINVAL, "a_out and b_out go together");
    KG_TRY(check_device(h));
    const int R = run->n_vectors, M = run->n_moments, NC = run->n_times;
    Series ser;
    KG_TRY(series_for(h, run->dt, run->bessel_tol, &ser));
    KG_TRY(ensure_moments(h, (size_t)R * NC * M));
    if (run->precision == KG_C64) return vac_impl<float>(h, R, M, NC, ser, a, b, true, a_out, b_out, mu_out);
    return vac_impl<double>(h, R, M, NC, ser, a, b, true, a_out, b_out, mu_out);
}

kg_status kg_msd_resume(kg_hamiltonian* h, const kg_run* run, const double* psi, const double* xi, double* mu_out,
                        double* psi_out, double* xi_out) {
    clear_error();
    KG_TRY(check_run(h, run, true));
    if (!psi || !mu_out) return fail(KG_EINVAL, "psi and mu_out must not be NULL");
    if ((psi_out == nullptr) != (xi_out == nullptr)) return fail(KG_EINVAL, "psi_out and xi_out go together");
    KG_TRY(check_device(h));
    const int R = run->n_vectors, M = run->n_moments, NC = run->n_times;
    Series ser;
    KG_TRY(series_for(h, run->dt, run->bessel_tol, &ser));
    KG_TRY(ensure_moments(h, (size_t)R * NC * M));
    if (run->precision == KG_C64) return msd_impl<float>(h, R, M, NC, ser, psi, xi, true, psi_out, xi_out, mu_out);
    return msd_impl<double>(h, R, M, NC, ser, psi, xi, true, psi_out, xi_out, mu_out);
}

kg_status kg_test_alloc_cap(uint64_t bytes) {
    clear_error();
    g_alloc_cap.store(bytes);
    return KG_OK;
}

kg_status kg_set_small_persistent(int enable) {
    clear_error();
    g_small_persistent.store(enable ? 1 : 0);
    return KG_OK;
}

kg_status kg_ftm_dos_moments(kg_hamiltonian* h, const kg_run* run, const double* phi, double* f_out) {
    clear_error();
    KG_TRY(check_run(h, run, false));
    if (run->precision != KG_FP64) return fail(KG_EINVAL, "kg_ftm_dos_moments: only KG_FP64");
    if (!phi || !f_out) return fail(KG_EINVAL, "phi and f_out must not be NULL");
    KG_TRY(check_device(h));
    const int R = run->n_vectors, NM = run->n_moments;
    const int64_t width = 2 * (int64_t)NM + 1;
    Series ser;
    KG_TRY(series_for_tau(kPi, run->bessel_tol, &ser));   // dtau = pi hbar for H~ (Sec. 4.2)
    // blocks: 0 phi (kept), 1 phi'_R, 2 p1 scratch, 3 series output
    KG_TRY(ensure_vectors(h, R, 4));
    KG_TRY(ensure_moments(h, (size_t)R * width));
    const int grid = stream_grid(h->n * R);
    KG_TRY(h->part_first.ensure((size_t)grid * R * 4 * sizeof(double), h->stream));
    double* part = (double*)h->part_first.p;
    double2* mu = (double2*)h->moments.p;
    KG_TRY(copy_in(h, phi, V(h, 0), R));
    // F_0 = <phi|phi>
    KG_CUDA_TRY(launch_dot<double>(h->n * R, R, V(h, 0), V(h, 0), part, grid, mu + NM, width, h->stream));
    h->counters.other_launches += 2;
    for (int dir = +1; dir >= -1; dir -= 2) {
        double2* p = V(h, 1);
        double2* q = V(h, 3);
        KG_CUDA_TRY(cudaMemcpyAsync(p, V(h, 0), vec_bytes(h, R), cudaMemcpyDeviceToDevice, h->stream));
        for (int k = 1; k <= NM; k++) {
            // |phi'_R> <- U(+-dtau)|phi'_R>  (Eq. 36: (-i)^m forward, (+i)^m backward)
            double2* in[1] = {p};
            double2* p1[1] = {V(h, 2)};
            double2* acc[1] = {q};
            KG_TRY(run_series<double>(h, R, ser, dir > 0 ? -1 : +1, 1, false, in, p1, acc, nullptr, nullptr,
                                      nullptr));
            std::swap(p, q);
            KG_CUDA_TRY(launch_dot<double>(h->n * R, R, V(h, 0), p, part, grid, mu + NM + dir * k, width,
                                           h->stream));
            h->counters.other_launches += 2;
        }
    }
    KG_TRY(check_finite(h, mu, (size_t)R * width * 2));
    return copy_out(h, mu, f_out, (size_t)R * width * sizeof(double2));
}

kg_status kg_apply(kg_hamiltonian* h, int op, const double* in_dev, double* out_dev, int n_vectors) {
    clear_error();
    if (!h) return fail(KG_EINVAL, "hamiltonian is NULL");
    if (op < KG_OP_H || op > KG_OP_V) return fail(KG_EINVAL, "unknown op");
    if (!valid_r(n_vectors)) return fail(KG_EINVAL, "n_vectors must be a power of two in 1..64");
    if (!in_dev || !out_dev || in_dev == out_dev) return fail(KG_EINVAL, "need distinct in/out");
    KG_TRY(check_device(h));
    const int R = n_vectors;
    KG_TRY(ensure_vectors(h, R, 2));
    KG_TRY(copy_in(h, in_dev, V(h, 0), R));
    KG_CUDA_TRY(launch_apply<double>(h->dev, R, op, h->emax / kHbarEvFs, V(h, 0), V(h, 1), h->stream));
    h->counters.other_launches += 1;
    return copy_out(h, V(h, 1), out_dev, (size_t)h->n * R * sizeof(double2));
}

kg_status kg_evolve(kg_hamiltonian* h, double dt, int which, double bessel_tol, const double* in_dev,
                    double* out_dev, int n_vectors) {
    clear_error();
    if (!h) return fail(KG_EINVAL, "hamiltonian is NULL");
    if (which < KG_U_FORWARD || which > KG_U_COMMUTATOR) return fail(KG_EINVAL, "unknown which");
    if (!valid_r(n_vectors)) return fail(KG_EINVAL, "n_vectors must be a power of two in 1..64");
    if (!in_dev || !out_dev || in_dev == out_dev) return fail(KG_EINVAL, "need distinct in/out");
    KG_TRY(check_device(h));
    const int R = n_vectors;
    Series ser;
    KG_TRY(series_for(h, dt, bessel_tol, &ser));
    // vectors: 0 p0 (copy of in), 1 p1, 2 acc, 3 q1, 4 q0, 5 qacc
    KG_TRY(ensure_vectors(h, R, 6));
    KG_TRY(copy_in(h, in_dev, V(h, 0), R));
    double2* in[1] = {V(h, 0)};
    double2* p1[1] = {V(h, 1)};
    double2* acc[1] = {V(h, 2)};
    if (which == KG_U_COMMUTATOR) {
        KG_TRY(run_series<double>(h, R, ser, -1, 1, true, in, p1, acc, V(h, 3), V(h, 4), V(h, 5)));
        return copy_out(h, V(h, 5), out_dev, (size_t)h->n * R * sizeof(double2));
    }
    KG_TRY(run_series<double>(h, R, ser, which == KG_U_FORWARD ? -1 : +1, 1, false, in, p1, acc, nullptr,
                              nullptr, nullptr));
    return copy_out(h, V(h, 2), out_dev, (size_t)h->n * R * sizeof(double2));
}

kg_status kg_timing_enable(kg_hamiltonian* h, int enable) {
    if (!h) return fail(KG_EINVAL, "hamiltonian is NULL");
    cudaStreamSynchronize(h->stream);
    for (auto& p : h->phases) {
        h->spare_events.push_back(p.a);
        h->spare_events.push_back(p.b);
    }
    h->phases.clear();
    h->counters = kg_timing{};
    h->timing = enable != 0;
    return KG_OK;
}

kg_status kg_fp64_fma_rate(int repeats, double* fma_per_s) {
    clear_error();
    if (!fma_per_s) return fail(KG_EINVAL, "fma_per_s is required");
    if (repeats < 1 || repeats > 100) return fail(KG_EINVAL, "repeats must be in 1..100");
    double* buf = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    auto cleanup = [&]() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (buf) cudaFree(buf);
    };
    const size_t bytes = (size_t)fp64_probe_grid() * 256 * sizeof(double);
    cudaError_t e = cudaMalloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) e = launch_fp64_probe(buf, nullptr);   // warm-up
    float best = 0.0f;
    for (int k = 0; k < repeats && e == cudaSuccess; k++) {
        e = cudaEventRecord(a, nullptr);
        if (e == cudaSuccess) e = launch_fp64_probe(buf, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(b, nullptr);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && ms > 0.0f && (best == 0.0f || ms < best)) best = ms;
    }
    cleanup();
    if (e != cudaSuccess) return fail(KG_ECUDA, std::string("kg_fp64_fma_rate: ") + cudaGetErrorString(e));
    if (best <= 0.0f) return fail(KG_ECUDA, "kg_fp64_fma_rate: no timed launch");
    *fma_per_s = fp64_probe_fmas() / (best * 1e-3);
    return KG_OK;
}

kg_status kg_timing_read(kg_hamiltonian* h, kg_timing* out) {
    if (!h || !out) return fail(KG_EINVAL, "NULL argument");
    KG_CUDA_TRY(cudaStreamSynchronize(h->stream));
    kg_timing t = h->counters;
    t.kpm_ms = 0;
    t.evolve_ms = 0;
    for (auto& p : h->phases) {
        float ms = 0;
        KG_CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
        (p.kind == 0 ? t.kpm_ms : t.evolve_ms) += ms;
    }
    *out = t;
    return KG_OK;
}

}  // extern "C"
