// Batched DOS moments over many uneven instances (e.g. ribbons of different widths,
// lengths and disorder) in one persistent launch.
//
// The instances are concatenated into one block-diagonal neighbour table (each keeps
// its own hopping -gamma0/E_max,i and scaled on-site energies).  R random vectors per
// instance are laid out [N_total + 1][R] (row N_total is the shared zero row).  CTAs
// are distributed over the instances in proportion to their site counts; each CTA
// owns one contiguous site range of one instance, so per-instance moment sums stay
// separable and the reduction is deterministic.
//
// Instead of one kernel launch (a grid-wide barrier) per Chebyshev step, the kernel
// is persistent: CTA c publishes "step n done" in flags[c] and starts step n + 1 once
// the CTAs holding the neighbours of its sites (a contiguous CTA range computed on the
// host) have published step n.  Neighbouring instances never wait on each other.
// Every wait is bounded: after kSpinLimit polls the CTA raises the error flag and
// returns, and every CTA that sees the flag returns too (the host reports
// KG_ETIMEOUT).  All CTAs are co-resident (grid = one occupancy-derived wave).
//
// The block width RB (vectors one thread group covers per pass: 8, 16, 32 or 64) is
// chosen by a measured autotuner; the device work of a call (flag reset, persistent
// kernel, reduction) is captured once per (RB, step count) in a CUDA graph and
// replayed.  The recursion is FP64 (6 DFMA per site-vector); the moments' inner
// products are double-float sums on the FP32 pipe (kg_dot.cuh).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "kg_dot.cuh"
#include "kg_internal.h"

namespace kg {

constexpr int kBThreads = 512;   // measured on the 16-ribbon batch: 7.05 against 7.19 ms per step with 256
constexpr int kBWarps = kBThreads / 32;
constexpr long long kSpinLimit = 1ll << 22;   // polls of ~100 ns before giving up

struct BatchArgs {
    const int32_t* idx;       // [3][n_total], sentinel = n_total
    int64_t n_total;
    const double* onsite;     // [n_total] scaled, or null
    const double* onsite2;    // [n_total] the same doubled (steps after the first), or null
    const double* hop;        // [n_inst] -gamma0 / E_max,i
    const int* cta_inst;      // [n_cta]
    const int64_t* cta_s0;    // [n_cta] first site
    const int64_t* cta_s1;    // [n_cta] one past the last site
    const int* dep_lo;        // [n_cta] first CTA this CTA waits on
    const int* dep_hi;        // [n_cta] last CTA this CTA waits on
    double2* A;               // phi_0, later phi_2, phi_4, ...
    double2* B;               // phi_1, phi_3, ...
    double* partial;          // [steps][n_cta][R][2]
    int* flags;               // [n_cta] completed steps
    int* error;               // 0 ok, 1 a wait gave up
    int n_cta;
    int steps;                // recursion steps: 0 (phi_1 = H~ phi_0) .. steps-1
    int stall_cta;            // test hook: this CTA never publishes steps >= 1 (-1: off)
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Per-chunk block reduction of (sum |x|^2, sum Re conj(y) x) for the RB vectors of
// chunk q; thread t holds vector q*RB + t % RB.  Writes dst[q*RB + r][2].
template <int RB>
__device__ __forceinline__ void chunk_reduce(double a0, double a1, double* __restrict__ dst) {
    __shared__ double sm[kBWarps][32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (RB < 32) {
#pragma unroll
        for (int off = 16; off >= RB; off >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, off);
            a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        }
    }
    constexpr int kLanes = RB < 32 ? RB : 32;
    if (lane < kLanes) {
        sm[warp][lane][0] = a0;
        sm[warp][lane][1] = a1;
    }
    __syncthreads();
    if (threadIdx.x < RB) {
        const int r = threadIdx.x;
        constexpr int kGroups = RB < 32 ? 1 : RB / 32;
        double s0 = 0.0, s1 = 0.0;
        for (int w = (RB < 32 ? 0 : (r >> 5)); w < kBWarps; w += kGroups) {
            s0 += sm[w][r & 31][0];
            s1 += sm[w][r & 31][1];
        }
        dst[r * 2] = s0;
        dst[r * 2 + 1] = s1;
    }
    __syncthreads();
}

template <int R, int RB, bool ONSITE>
__global__ void __launch_bounds__(kBThreads) batched_kpm_kernel(BatchArgs a) {
    constexpr int kChunks = R / RB;
    constexpr int kSitesPerPass = kBThreads / RB;
    const int cta = blockIdx.x;
    const int64_t s0 = a.cta_s0[cta], s1 = a.cta_s1[cta];
    const double h = a.hop[a.cta_inst[cta]];
    const int d0 = a.dep_lo[cta], d1 = a.dep_hi[cta];
    const int rl = threadIdx.x % RB, sl = threadIdx.x / RB;
    const int64_t n_total = a.n_total;
    for (int n = 0; n < a.steps; n++) {
        if (n > 0) {
            // wait until every CTA holding neighbours of our sites has finished step n-1
            for (int d = d0 + threadIdx.x; d <= d1; d += kBThreads) {
                long long spins = 0;
                while (ld_acquire(a.flags + d) < n) {
                    if (++spins > kSpinLimit || *(volatile int*)a.error) {
                        atomicExch(a.error, 1);
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __syncthreads();
            if (*(volatile int*)a.error) return;
        }
        const double2* cur = (n & 1) ? a.B : a.A;
        double2* out = (n & 1) ? a.A : a.B;   // in place over phi_{n-1} from n = 1 on
        const double c = n == 0 ? h : 2.0 * h;
        Dot64 acc0[kChunks], acc1[kChunks];
        // one thread covers kChunks vectors of a site, so the index loads are amortised over
        // them.  With one vector per thread (block width R) the next site's indices are
        // loaded one iteration ahead; at narrower widths the extra registers cost occupancy.
        constexpr bool kPrefetch = kChunks == 1;
        int64_t site = s0 + sl;
        int32_t j0 = 0, j1 = 0, j2 = 0;
        if constexpr (kPrefetch) {
            if (site < s1) {
                j0 = __ldg(a.idx + site);
                j1 = __ldg(a.idx + n_total + site);
                j2 = __ldg(a.idx + 2 * n_total + site);
            }
        }
        for (; site < s1; site += kSitesPerPass) {
            int32_t i0, i1, i2;
            if constexpr (kPrefetch) {
                i0 = j0;
                i1 = j1;
                i2 = j2;
                const int64_t nxt = site + kSitesPerPass;
                if (nxt < s1) {
                    j0 = __ldg(a.idx + nxt);
                    j1 = __ldg(a.idx + n_total + nxt);
                    j2 = __ldg(a.idx + 2 * n_total + nxt);
                }
            } else {
                i0 = __ldg(a.idx + site);
                i1 = __ldg(a.idx + n_total + site);
                i2 = __ldg(a.idx + 2 * n_total + site);
            }
            double e = 0.0;
            if constexpr (ONSITE) e = n == 0 ? __ldg(a.onsite + site) : __ldg(a.onsite2 + site);
#pragma unroll
            for (int q = 0; q < kChunks; q++) {
                const int r = q * RB + rl;
                // Vectors are rewritten by other CTAs during the kernel, so no read-only
                // (non-coherent) loads.  Plain cached loads are coherent here: every value read
                // in step n was written before a release (st.release.gpu of the writer's step
                // flag) that this CTA's ld.acquire.gpu observed before the barrier above, so by
                // the PTX memory model these weak loads cannot return older values (the
                // acquire invalidates the SM's L1), and nothing read in step n is rewritten
                // before this CTA publishes step n.  L1 then serves the in-chain neighbours
                // (adjacent rows) as in the per-step kernels.
                const double2 va = __ldca(cur + (int64_t)i0 * R + r);
                const double2 vb = __ldca(cur + (int64_t)i1 * R + r);
                const double2 vc = __ldca(cur + (int64_t)i2 * R + r);
                const double2 x = __ldca(cur + site * R + r);
                double2 z = make_double2(0.0, 0.0);
                if (n > 0) z = __ldca(out + site * R + r);
                const double tr = ONSITE ? fma(e, x.x, -z.x) : -z.x;
                const double ti = ONSITE ? fma(e, x.y, -z.y) : -z.y;
                const double yr = fma(c, va.x, fma(c, vb.x, fma(c, vc.x, tr)));
                const double yi = fma(c, va.y, fma(c, vb.y, fma(c, vc.y, ti)));
                __stcg(out + site * R + r, make_double2(yr, yi));
                acc0[q].add_prod(x.x, x.x);
                acc0[q].add_prod(x.y, x.y);
                acc1[q].add_prod(yr, x.x);
                acc1[q].add_prod(yi, x.y);
            }
        }
        double* dst = a.partial + ((int64_t)n * a.n_cta + cta) * R * 2;
#pragma unroll
        for (int q = 0; q < kChunks; q++) chunk_reduce<RB>(acc0[q].value(), acc1[q].value(), dst + q * RB * 2);
        // publish: all of this CTA's writes of step n before the flag
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (!(cta == a.stall_cta && n >= 1)) st_release(a.flags + cta, n + 1);
        }
    }
}

// Moments of instance i from the partial sums of its CTAs [c0_i, c1_i), fixed order:
// mu_0 = S0(0), mu_1 = S1(0), mu_{2n} = 2 S0(n) - mu_0, mu_{2n+1} = 2 S1(n) - mu_1.
__global__ void batched_reduce_kernel(const double* __restrict__ partial, const int* __restrict__ inst_c0,
                                      const int* __restrict__ inst_c1, int n_cta, int R, int M,
                                      double2* __restrict__ mu /* [n_inst][R][M] */) {
    const int n = blockIdx.x, i = blockIdx.y;
    const int c0 = inst_c0[i], c1 = inst_c1[i];
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        double s0 = 0, s1 = 0, m0 = 0, m1 = 0;
        for (int c = c0; c < c1; c++) {
            s0 += partial[(((int64_t)n * n_cta + c) * R + r) * 2];
            s1 += partial[(((int64_t)n * n_cta + c) * R + r) * 2 + 1];
            m0 += partial[((int64_t)c * R + r) * 2];
            m1 += partial[((int64_t)c * R + r) * 2 + 1];
        }
        double2* m = mu + ((int64_t)i * R + r) * M;
        if (n == 0) {
            m[0] = make_double2(s0, 0.0);
            if (M > 1) m[1] = make_double2(s1, 0.0);
        } else {
            if (2 * n < M) m[2 * n] = make_double2(2.0 * s0 - m0, 0.0);
            if (2 * n + 1 < M) m[2 * n + 1] = make_double2(2.0 * s1 - m1, 0.0);
        }
    }
}

// Re-bases one instance's neighbour table into the concatenated one.
__global__ void rebase_idx_kernel(const int32_t* __restrict__ in, int64_t n_i, int64_t offset,
                                  int32_t* __restrict__ out, int64_t n_total) {
    const int64_t count = 3 * n_i;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int slot = (int)(k / n_i);
        const int64_t site = k % n_i;
        const int32_t v = in[k];
        out[slot * n_total + offset + site] = (v >= n_i || v < 0) ? (int32_t)n_total : (int32_t)(v + offset);
    }
}

template <int R, int RB>
static cudaError_t launch_batched(const BatchArgs& a, bool onsite, cudaStream_t s) {
    if (onsite) batched_kpm_kernel<R, RB, true><<<a.n_cta, kBThreads, 0, s>>>(a);
    else batched_kpm_kernel<R, RB, false><<<a.n_cta, kBThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int R, int RB>
static int batched_occupancy(bool onsite) {
    int per_sm = 0;
    cudaError_t e = onsite
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kpm_kernel<R, RB, true>, kBThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kpm_kernel<R, RB, false>, kBThreads, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return per_sm < 1 ? 1 : per_sm;
}

#define KG_BATCH_DISPATCH(R_, RB_, ...)                                                    \
    do {                                                                                   \
        if (R_ == 64 && RB_ == 64) { constexpr int R = 64, RB = 64; __VA_ARGS__; }                \
        else if (R_ == 64 && RB_ == 32) { constexpr int R = 64, RB = 32; __VA_ARGS__; }           \
        else if (R_ == 64 && RB_ == 16) { constexpr int R = 64, RB = 16; __VA_ARGS__; }           \
        else if (R_ == 64 && RB_ == 8) { constexpr int R = 64, RB = 8; __VA_ARGS__; }             \
        else if (R_ == 32 && RB_ == 32) { constexpr int R = 32, RB = 32; __VA_ARGS__; }           \
        else if (R_ == 32 && RB_ == 16) { constexpr int R = 32, RB = 16; __VA_ARGS__; }           \
        else if (R_ == 32 && RB_ == 8) { constexpr int R = 32, RB = 8; __VA_ARGS__; }             \
        else if (R_ == 16 && RB_ == 16) { constexpr int R = 16, RB = 16; __VA_ARGS__; }           \
        else if (R_ == 16 && RB_ == 8) { constexpr int R = 16, RB = 8; __VA_ARGS__; }             \
        else if (R_ == 8 && RB_ == 8) { constexpr int R = 8, RB = 8; __VA_ARGS__; }               \
        else if (R_ == 4 && RB_ == 4) { constexpr int R = 4, RB = 4; __VA_ARGS__; }               \
        else if (R_ == 2 && RB_ == 2) { constexpr int R = 2, RB = 2; __VA_ARGS__; }               \
        else if (R_ == 1 && RB_ == 1) { constexpr int R = 1, RB = 1; __VA_ARGS__; }               \
    } while (0)

// ---------------------------------------------------------------------------------
// Host side: the batch (concatenated tables, CTA schedule, graphs, tuning)
// ---------------------------------------------------------------------------------

struct Batch {
    std::vector<const kg_hamiltonian*> members;
    int R = 0;
    int device = 0;
    cudaStream_t stream = nullptr;   // owned: graph capture needs a non-legacy stream
    int64_t n_total = 0;
    std::vector<int64_t> offset;     // site offset of each instance
    std::vector<int64_t> sizes;
    bool onsite = false;
    // device arrays
    void* mem = nullptr;
    int32_t* idx = nullptr;
    double* onsite_d = nullptr;
    double* onsite2_d = nullptr;
    double* hop = nullptr;
    double2* A = nullptr;
    double2* B = nullptr;
    int* flags = nullptr;
    int* error = nullptr;
    double* partial = nullptr;
    size_t partial_bytes = 0;
    double2* mu = nullptr;
    size_t mu_bytes = 0;
    // schedule (per RB: occupancy differs)
    struct Sched {
        int n_cta = 0;
        int* cta_inst = nullptr;
        int64_t* cta_s0 = nullptr;
        int64_t* cta_s1 = nullptr;
        int* dep_lo = nullptr;
        int* dep_hi = nullptr;
        int* inst_c0 = nullptr;
        int* inst_c1 = nullptr;
        void* mem = nullptr;
    };
    // A tuning configuration is (block width RB, CTA budget = one occupancy wave / split),
    // encoded as cfg = RB * 8 + split.
    std::map<int, Sched> sched;                                 // cfg -> schedule
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (cfg, M) -> graph
    int tuned_cfg = 0;
    double tuned_ms_per_step = 0.0;
    struct Trial {
        int rb, n_cta;
        double ms;
    };
    std::vector<Trial> tuning_log;
    int stall_cta = -1;   // test hook
    ~Batch() {
        for (auto& g : graphs) cudaGraphExecDestroy(g.second);
        for (auto& s : sched) cudaFree(s.second.mem);
        if (partial) cudaFree(partial);
        if (mu) cudaFree(mu);
        if (mem) cudaFree(mem);
        if (stream) cudaStreamDestroy(stream);
    }
};

// Host copy of one member's neighbour table (device -> host), for the schedule.
static kg_status member_table(const kg_hamiltonian* h, std::vector<int32_t>* out) {
    const DevH& d = hamiltonian_dev(h);
    out->resize((size_t)(3 * d.n));
    KG_CUDA_TRY(cudaMemcpy(out->data(), d.idx, out->size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return KG_OK;
}

static kg_status build_schedule(Batch* b, int rb, int split, Batch::Sched* s) {
    int per_sm = 0;
    KG_BATCH_DISPATCH(b->R, rb, per_sm = batched_occupancy<R, RB>(b->onsite));
    if (per_sm < 1) return fail(KG_EINVAL, "batched: no kernel for this (R, block width)");
    const int n_inst = (int)b->members.size();
    const int64_t wave = (int64_t)sm_count() * per_sm;
    // CTA budget: one occupancy wave (split 1) or a fraction of it (fewer, longer site
    // ranges: fewer step flags to wait on, less parallelism); never below one per member
    int64_t budget = std::max<int64_t>(wave / std::max(split, 1), n_inst);
    if (budget > wave) return fail(KG_EINVAL, "batched: more instances than co-resident CTAs");
    // CTAs per instance in proportion to its sites, at least one, at most one per 32 sites
    std::vector<int64_t> k(n_inst, 1);
    int64_t used = n_inst;
    std::vector<std::pair<double, int>> frac;
    for (int i = 0; i < n_inst; i++) {
        const double ideal = (double)budget * b->sizes[i] / (double)b->n_total;
        int64_t want = std::max<int64_t>(1, (int64_t)std::floor(ideal));
        want = std::min<int64_t>(want, std::max<int64_t>(1, b->sizes[i] / 32));
        used += want - 1;
        k[i] = want;
        frac.push_back({ideal - (double)want, i});
    }
    std::sort(frac.begin(), frac.end(), [](auto& x, auto& y) { return x.first > y.first; });
    for (auto& f : frac) {
        if (used >= budget) break;
        const int i = f.second;
        if (k[i] + 1 <= std::max<int64_t>(1, b->sizes[i] / 32)) {
            k[i]++;
            used++;
        }
    }
    std::vector<int> cta_inst, inst_c0(n_inst), inst_c1(n_inst);
    std::vector<int64_t> cs0, cs1;
    for (int i = 0; i < n_inst; i++) {
        inst_c0[i] = (int)cta_inst.size();
        for (int64_t j = 0; j < k[i]; j++) {
            cta_inst.push_back(i);
            cs0.push_back(b->offset[i] + b->sizes[i] * j / k[i]);
            cs1.push_back(b->offset[i] + b->sizes[i] * (j + 1) / k[i]);
        }
        inst_c1[i] = (int)cta_inst.size();
    }
    const int n_cta = (int)cta_inst.size();
    // dependency range: CTAs owning any neighbour of the CTA's sites (and itself)
    std::vector<int> lo(n_cta), hi(n_cta);
    for (int i = 0; i < n_inst; i++) {
        std::vector<int32_t> t;
        KG_TRY(member_table(b->members[i], &t));
        const int64_t ni = b->sizes[i];
        for (int c = inst_c0[i]; c < inst_c1[i]; c++) {
            int64_t mn = cs0[c], mx = cs1[c] - 1;
            for (int64_t site = cs0[c] - b->offset[i]; site < cs1[c] - b->offset[i]; site++) {
                for (int slot = 0; slot < 3; slot++) {
                    const int32_t v = t[(size_t)(slot * ni + site)];
                    if (v >= 0 && v < ni) {
                        mn = std::min<int64_t>(mn, v + b->offset[i]);
                        mx = std::max<int64_t>(mx, v + b->offset[i]);
                    }
                }
            }
            int a0 = c, a1 = c;
            while (a0 > inst_c0[i] && cs0[a0] > mn) a0--;
            while (a1 < inst_c1[i] - 1 && cs1[a1] <= mx) a1++;
            lo[c] = a0;
            hi[c] = a1;
        }
    }
    // symmetrise (a CTA that reads mine must be waited for before I overwrite)
    for (int c = 0; c < n_cta; c++)
        for (int d = lo[c]; d <= hi[c]; d++) {
            lo[d] = std::min(lo[d], c);
            hi[d] = std::max(hi[d], c);
        }
    const size_t bytes = n_cta * (sizeof(int) * 3 + sizeof(int64_t) * 2) + n_inst * sizeof(int) * 2 + 256;
    KG_CUDA_TRY(cudaMalloc(&s->mem, bytes));
    char* p = (char*)s->mem;
    auto take = [&](size_t n) { char* q = p; p += (n + 15) & ~(size_t)15; return q; };
    s->cta_s0 = (int64_t*)take(n_cta * sizeof(int64_t));
    s->cta_s1 = (int64_t*)take(n_cta * sizeof(int64_t));
    s->cta_inst = (int*)take(n_cta * sizeof(int));
    s->dep_lo = (int*)take(n_cta * sizeof(int));
    s->dep_hi = (int*)take(n_cta * sizeof(int));
    s->inst_c0 = (int*)take(n_inst * sizeof(int));
    s->inst_c1 = (int*)take(n_inst * sizeof(int));
    KG_CUDA_TRY(cudaMemcpy(s->cta_s0, cs0.data(), n_cta * sizeof(int64_t), cudaMemcpyHostToDevice));
    KG_CUDA_TRY(cudaMemcpy(s->cta_s1, cs1.data(), n_cta * sizeof(int64_t), cudaMemcpyHostToDevice));
    KG_CUDA_TRY(cudaMemcpy(s->cta_inst, cta_inst.data(), n_cta * sizeof(int), cudaMemcpyHostToDevice));
    KG_CUDA_TRY(cudaMemcpy(s->dep_lo, lo.data(), n_cta * sizeof(int), cudaMemcpyHostToDevice));
    KG_CUDA_TRY(cudaMemcpy(s->dep_hi, hi.data(), n_cta * sizeof(int), cudaMemcpyHostToDevice));
    KG_CUDA_TRY(cudaMemcpy(s->inst_c0, inst_c0.data(), n_inst * sizeof(int), cudaMemcpyHostToDevice));
    KG_CUDA_TRY(cudaMemcpy(s->inst_c1, inst_c1.data(), n_inst * sizeof(int), cudaMemcpyHostToDevice));
    s->n_cta = n_cta;
    return KG_OK;
}

static kg_status create_batch(kg_hamiltonian* const* hs, int n_h, int R, std::unique_ptr<Batch>* out) {
    auto b = std::make_unique<Batch>();
    b->R = R;
    KG_CUDA_TRY(cudaGetDevice(&b->device));
    KG_CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    int64_t total = 0;
    for (int i = 0; i < n_h; i++) {
        const DevH& d = hamiltonian_dev(hs[i]);
        b->members.push_back(hs[i]);
        b->offset.push_back(total);
        b->sizes.push_back(d.n);
        total += d.n;
        b->onsite = b->onsite || d.onsite != nullptr;
        if (d.ytransport) return fail(KG_EINVAL, "batched: armchair ribbons are not supported");
    }
    if (total >= (int64_t)INT32_MAX - 1) return fail(KG_EINVAL, "batched: too many sites in total");
    b->n_total = total;
    const size_t b_idx = ((size_t)3 * total * sizeof(int32_t) + 255) & ~(size_t)255;
    const size_t b_on = b->onsite ? (((size_t)(total + 1) * sizeof(double) + 255) & ~(size_t)255) : 0;
    const size_t b_hop = ((size_t)n_h * sizeof(double) + 255) & ~(size_t)255;
    const size_t b_vec = (((size_t)(total + 1) * R * sizeof(double2)) + 255) & ~(size_t)255;
    const size_t b_flags = 256 + (size_t)sm_count() * 64 * sizeof(int);
    const size_t bytes = b_idx + 2 * b_on + b_hop + 2 * b_vec + b_flags;
    if (cudaMalloc(&b->mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(KG_ENOMEM, "batched: device allocation failed");
    }
    char* p = (char*)b->mem;
    b->idx = (int32_t*)p; p += b_idx;
    if (b->onsite) {
        b->onsite_d = (double*)p;
        p += b_on;
        b->onsite2_d = (double*)p;
        p += b_on;
    }
    b->hop = (double*)p; p += b_hop;
    b->A = (double2*)p; p += b_vec;
    b->B = (double2*)p; p += b_vec;
    b->error = (int*)p;
    b->flags = (int*)p + 64;
    // every double2 block must sit on a 16-byte boundary
    for (const void* q : {(const void*)b->A, (const void*)b->B, (const void*)b->hop, (const void*)b->idx})
        if ((uintptr_t)q % 16 != 0) return fail(KG_EINVAL, "batched: internal layout misaligned");
    KG_CUDA_TRY(cudaMemsetAsync(b->mem, 0, bytes, b->stream));
    std::vector<double> hop(n_h);
    for (int i = 0; i < n_h; i++) {
        const DevH& d = hamiltonian_dev(hs[i]);
        hop[i] = d.h;
        rebase_idx_kernel<<<stream_grid(3 * d.n), 256, 0, b->stream>>>(d.idx, d.n, b->offset[i], b->idx, total);
        KG_CUDA_TRY(cudaGetLastError());
        if (d.onsite) {
            KG_CUDA_TRY(cudaMemcpyAsync(b->onsite_d + b->offset[i], d.onsite, d.n * sizeof(double),
                                        cudaMemcpyDeviceToDevice, b->stream));
            if (d.onsite2) {
                KG_CUDA_TRY(cudaMemcpyAsync(b->onsite2_d + b->offset[i], d.onsite2, d.n * sizeof(double),
                                            cudaMemcpyDeviceToDevice, b->stream));
            } else {
                return fail(KG_EINVAL, "batched: member without doubled on-site energies");
            }
        }
    }
    KG_CUDA_TRY(cudaMemcpyAsync(b->hop, hop.data(), n_h * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(b->stream));
    *out = std::move(b);
    return KG_OK;
}

static kg_status ensure_batch_buffers(Batch* b, int steps, int M) {
    int max_cta = 0;
    for (auto& s : b->sched) max_cta = std::max(max_cta, s.second.n_cta);
    const size_t pb = (size_t)steps * max_cta * b->R * 2 * sizeof(double);
    if (pb > b->partial_bytes) {
        if (b->partial) cudaFree(b->partial);
        b->partial = nullptr;
        b->partial_bytes = 0;
        // graphs refer to the old buffer
        for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
        b->graphs.clear();
        KG_CUDA_TRY(cudaMalloc(&b->partial, pb));
        b->partial_bytes = pb;
    }
    const size_t mb = b->members.size() * (size_t)b->R * M * sizeof(double2);
    if (mb > b->mu_bytes) {
        if (b->mu) cudaFree(b->mu);
        b->mu = nullptr;
        b->mu_bytes = 0;
        for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
        b->graphs.clear();
        KG_CUDA_TRY(cudaMalloc(&b->mu, mb));
        b->mu_bytes = mb;
    }
    return KG_OK;
}

static kg_status get_sched(Batch* b, int cfg, Batch::Sched** out) {
    auto it = b->sched.find(cfg);
    if (it == b->sched.end()) {
        Batch::Sched s;
        KG_TRY(build_schedule(b, cfg / 8, cfg % 8, &s));
        it = b->sched.emplace(cfg, s).first;
    }
    *out = &it->second;
    return KG_OK;
}

// Enqueues (and on first use captures into a graph) the device work for M moments.
static kg_status run_graph(Batch* b, int cfg, int M) {
    const int rb = cfg / 8;
    Batch::Sched* s = nullptr;
    KG_TRY(get_sched(b, cfg, &s));
    const int steps = std::max(1, (M + 1) / 2);   // step n yields moments 2n and 2n+1
    KG_TRY(ensure_batch_buffers(b, steps, M));
    const auto key = std::make_pair(cfg, M);
    auto it = b->graphs.find(key);
    const bool direct = b->stall_cta >= 0;   // test hook runs are never cached as graphs
    if (it == b->graphs.end() || direct) {
        BatchArgs a{};
        a.idx = b->idx;
        a.n_total = b->n_total;
        a.onsite = b->onsite_d;
        a.onsite2 = b->onsite2_d;
        a.hop = b->hop;
        a.cta_inst = s->cta_inst;
        a.cta_s0 = s->cta_s0;
        a.cta_s1 = s->cta_s1;
        a.dep_lo = s->dep_lo;
        a.dep_hi = s->dep_hi;
        a.A = b->A;
        a.B = b->B;
        a.partial = b->partial;
        a.flags = b->flags;
        a.error = b->error;
        a.n_cta = s->n_cta;
        a.steps = steps;
        a.stall_cta = b->stall_cta;
        if (direct) {
            KG_CUDA_TRY(cudaMemsetAsync(b->error, 0, 64 * sizeof(int) + (size_t)s->n_cta * sizeof(int), b->stream));
            cudaError_t e = cudaErrorInvalidConfiguration;   // no instantiation for (R, RB)
            KG_BATCH_DISPATCH(b->R, rb, e = (launch_batched<R, RB>(a, b->onsite, b->stream)));
            KG_CUDA_TRY(e);
            batched_reduce_kernel<<<dim3(steps, (unsigned)b->members.size()), 64, 0, b->stream>>>(
                b->partial, s->inst_c0, s->inst_c1, s->n_cta, b->R, M, b->mu);
            KG_CUDA_TRY(cudaGetLastError());
            return KG_OK;
        }
        cudaGraph_t g = nullptr;
        KG_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemsetAsync(b->error, 0, 64 * sizeof(int) + (size_t)s->n_cta * sizeof(int), b->stream);
        cudaError_t e2 = cudaErrorInvalidConfiguration;   // no instantiation for (R, RB)
        KG_BATCH_DISPATCH(b->R, rb, e2 = (launch_batched<R, RB>(a, b->onsite, b->stream)));
        batched_reduce_kernel<<<dim3(steps, (unsigned)b->members.size()), 64, 0, b->stream>>>(
            b->partial, s->inst_c0, s->inst_c1, s->n_cta, b->R, M, b->mu);
        cudaError_t e3 = cudaGetLastError();
        cudaError_t e4 = cudaStreamEndCapture(b->stream, &g);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(KG_ECUDA, "batched: graph capture failed");
        }
        cudaGraphExec_t ex = nullptr;
        cudaError_t e5 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e5 != cudaSuccess) return fail(KG_ECUDA, std::string("batched: graph instantiate: ") + cudaGetErrorString(e5));
        if (it != b->graphs.end()) cudaGraphExecDestroy(it->second);
        it = b->graphs.insert_or_assign(key, ex).first;
    }
    KG_CUDA_TRY(cudaGraphLaunch(it->second, b->stream));
    return KG_OK;
}

static kg_status check_error_flag(Batch* b) {
    int err = 0;
    KG_CUDA_TRY(cudaMemcpyAsync(&err, b->error, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (err) return fail(KG_ETIMEOUT, "batched: a CTA gave up waiting for its neighbours' step flags");
    return KG_OK;
}

static std::vector<int> candidate_widths(int R) {
    std::vector<int> c;
    for (int rb : {8, 16, 32, 64})
        if (rb <= R && R % rb == 0) c.push_back(rb);
    if (c.empty()) c.push_back(R);
    return c;
}

// Measures every block width on a short run (same batch, 24 moments) and keeps the fastest.
static kg_status autotune(Batch* b) {
    if (b->tuned_cfg) return KG_OK;
    const int probe_m = 24;
    cudaEvent_t e0, e1;
    KG_CUDA_TRY(cudaEventCreate(&e0));
    KG_CUDA_TRY(cudaEventCreate(&e1));
    double best = 1e300;
    int best_cfg = 0;
    for (int rb : candidate_widths(b->R))
        for (int split : {1, 2}) {
            const int cfg = rb * 8 + split;
            KG_TRY(run_graph(b, cfg, probe_m));   // warm-up and capture
            KG_CUDA_TRY(cudaEventRecord(e0, b->stream));
            for (int k = 0; k < 3; k++) KG_TRY(run_graph(b, cfg, probe_m));
            KG_CUDA_TRY(cudaEventRecord(e1, b->stream));
            KG_TRY(check_error_flag(b));
            float ms = 0;
            KG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            const double per_step = ms / 3.0 / (probe_m / 2);
            b->tuning_log.push_back({rb, b->sched[cfg].n_cta, per_step});
            if (per_step < best) {
                best = per_step;
                best_cfg = cfg;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->tuned_cfg = best_cfg;
    b->tuned_ms_per_step = best;
    return KG_OK;
}

// One cached batch per process (keyed by the member handles and R).
static std::unique_ptr<Batch> g_batch;

static kg_status get_batch(kg_hamiltonian* const* hs, int n_h, int R, Batch** out) {
    bool same = g_batch && g_batch->R == R && (int)g_batch->members.size() == n_h;
    if (same) {
        int dev = 0;
        KG_CUDA_TRY(cudaGetDevice(&dev));
        same = dev == g_batch->device;
        for (int i = 0; same && i < n_h; i++) same = g_batch->members[i] == hs[i];
    }
    if (!same) {
        g_batch.reset();
        KG_TRY(create_batch(hs, n_h, R, &g_batch));
    }
    *out = g_batch.get();
    return KG_OK;
}

}  // namespace kg

using namespace kg;

extern "C" {

kg_status kg_batched_dos_moments(kg_hamiltonian* const* hs, int n_h, const kg_run* run,
                                 const double* const* phis, double* mu_out) {
    clear_error();
    if (!hs || n_h < 1 || !run || !phis || !mu_out) return fail(KG_EINVAL, "batched: NULL or empty argument");
    const int R = run->n_vectors, M = run->n_moments;
    if (R < 1 || R > 64 || (R & (R - 1))) return fail(KG_EINVAL, "n_vectors must be a power of two in 1..64");
    if (M < 1) return fail(KG_EINVAL, "n_moments must be >= 1");
    if (run->precision != KG_FP64) return fail(KG_EINVAL, "batched: only KG_FP64");
    for (int i = 0; i < n_h; i++)
        if (!hs[i] || !phis[i]) return fail(KG_EINVAL, "batched: NULL member");
    Batch* b = nullptr;
    KG_TRY(get_batch(hs, n_h, R, &b));
    // The batch runs on its own capture-capable (non-blocking) stream: order it after
    // the work already queued on the legacy default stream and on the members' stream.
    {
        cudaEvent_t ev[2];
        KG_CUDA_TRY(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        KG_CUDA_TRY(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        KG_CUDA_TRY(cudaEventRecord(ev[0], (cudaStream_t)0));
        KG_CUDA_TRY(cudaEventRecord(ev[1], hamiltonian_stream(hs[0])));
        KG_CUDA_TRY(cudaStreamWaitEvent(b->stream, ev[0], 0));
        KG_CUDA_TRY(cudaStreamWaitEvent(b->stream, ev[1], 0));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    KG_TRY(autotune(b));
    // stage the inputs: instance i's [N_i][R] block at rows offset_i ..
    for (int i = 0; i < n_h; i++)
        KG_CUDA_TRY(cudaMemcpyAsync(b->A + b->offset[i] * R, phis[i], (size_t)b->sizes[i] * R * sizeof(double2),
                                    cudaMemcpyDefault, b->stream));
    KG_CUDA_TRY(cudaMemsetAsync(b->A + b->n_total * R, 0, (size_t)R * sizeof(double2), b->stream));
    KG_CUDA_TRY(cudaMemsetAsync(b->B + b->n_total * R, 0, (size_t)R * sizeof(double2), b->stream));
    KG_TRY(run_graph(b, b->tuned_cfg, M));
    KG_TRY(check_error_flag(b));
    // error[1]: non-finite moments (cleared with the wait flags by every graph replay)
    KG_CUDA_TRY(launch_nonfinite((const double*)b->mu, (int64_t)n_h * R * M * 2, b->error + 1, b->stream));
    int bad = 0;
    KG_CUDA_TRY(cudaMemcpyAsync(&bad, b->error + 1, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    KG_CUDA_TRY(cudaMemcpyAsync(mu_out, b->mu, (size_t)n_h * R * M * sizeof(double2), cudaMemcpyDefault,
                                b->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (bad)
        return fail(KG_ENUMERIC, "batched: non-finite moments (input vectors with NaN/Inf entries or entries "
                                 "of magnitude 2^63 or more)");
    return KG_OK;
}

kg_status kg_batched_tuning(int* block_width, double* ms_per_step, int* n_ctas, int max_log, int* log_width,
                            int* log_ctas, double* log_ms) {
    clear_error();
    if (!g_batch || !g_batch->tuned_cfg) return fail(KG_EINVAL, "batched: no tuned batch yet");
    if (block_width) *block_width = g_batch->tuned_cfg / 8;
    if (ms_per_step) *ms_per_step = g_batch->tuned_ms_per_step;
    if (n_ctas) *n_ctas = g_batch->sched[g_batch->tuned_cfg].n_cta;
    for (int k = 0; k < max_log && k < (int)g_batch->tuning_log.size(); k++) {
        if (log_width) log_width[k] = g_batch->tuning_log[k].rb;
        if (log_ctas) log_ctas[k] = g_batch->tuning_log[k].n_cta;
        if (log_ms) log_ms[k] = g_batch->tuning_log[k].ms;
    }
    return KG_OK;
}

kg_status kg_batched_release(void) {
    g_batch.reset();
    return KG_OK;
}

kg_status kg_batched_test_stall(int cta) {
    if (!g_batch) return fail(KG_EINVAL, "batched: no batch yet");
    g_batch->stall_cta = cta;
    return KG_OK;
}

}  // extern "C"
