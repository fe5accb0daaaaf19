// Kernels of the Chebyshev recursion for sm_103a, in two precisions:
//   T = double: complex128 vectors, FP64 recursion, inner products in double-float
//               arithmetic on the FP32 pipe (kg_dot.cuh), combined in FP64;
//   T = float:  complex64 vectors, FP32 recursion, inner products accumulated per
//               thread with exact FP32 products and compensated (TwoSum) sums, then
//               combined across threads and blocks in FP64.
//
// Every kernel streams over the N*R complex items of a block of R vectors laid out
// [N+1][R] (row N is a permanent zero row; the neighbour table points removed or
// missing neighbours at it, so the gather needs no branch).  One thread owns items
// w = n*R + r with a fixed r, so per-vector partial sums stay in registers; the
// R vectors of a site share one load of the site's three neighbour indices.
//
// The GB300 executes FP64 at 1/64 of the FP32 rate (about 0.6e12 DFMA/s, and DADD
// slower than DFMA), so the FP64 recursion is limited by the DP pipe, not by HBM.
// FP64 operations are therefore all fused multiply-adds: the neighbour sum and the
// "- T_{n-1}" fold into the hopping multiply (3 FMA per real component), and the inner
// products of the moments run on the FP32 and integer pipes (Acc<double> below), so a
// site-vector update costs 6 DFMA.  The FP32 kernels are HBM-bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <unordered_map>

#include "kg_dot.cuh"
#include "kg_internal.h"

namespace kg {

// Threads per block: 256 for the streaming, reduction and complex64 kernels; 512 for the
// FP64 recursion kernels (measured on the 2.1M-site sheet: 98 against 102 us per KPM step;
// the FP64 step at 42 registers runs two 512-thread blocks per SM, and capping it at 40
// registers for a third block measured slower, 106 us; the complex64 step is faster with 256).
constexpr int kThreads = 256;
template <typename T>
constexpr int kBlock = sizeof(T) == sizeof(double) ? 512 : 256;

// --------------------------------------------------------------------------------
// Inner-product accumulators
// --------------------------------------------------------------------------------

template <typename T>
struct Acc;

// FP64: double-float products and sums on the FP32 and integer pipes (kg_dot.cuh).
template <>
struct Acc<double> : Dot64 {};

// FP32 products are split exactly into p + e (e = fma(a, b, -p)); p is added with
// Knuth's TwoSum, whose rounding error joins e in the compensation term c.  The
// explicit-rounding intrinsics keep the compiler from contracting or reassociating.
template <>
struct Acc<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = fmaf(a, b, -p);
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        c = __fadd_rn(c, __fadd_rn(err, e));
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// --------------------------------------------------------------------------------
// Block reduction of NACC per-thread FP64 partials belonging to vector r = tid % R.
// Deterministic: fixed shuffle tree, then a fixed-order sum over warps.
// dst receives [R][NACC] doubles for this block.
// --------------------------------------------------------------------------------
template <int R, int NACC, int NT>
__device__ __forceinline__ void block_reduce(double (&acc)[NACC], double* __restrict__ dst) {
    constexpr int kWarps = NT / 32;
    constexpr int kLanesUsed = R < 32 ? R : 32;
    // only the lanes that hold a distinct vector store (the smallest table: the rest of
    // the SM's unified L1/shared storage stays L1 for the neighbour gathers)
    __shared__ double sm[kWarps][kLanesUsed][NACC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (R < 32) {
#pragma unroll
        for (int off = 16; off >= R; off >>= 1) {
#pragma unroll
            for (int q = 0; q < NACC; q++) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        }
    }
    if (lane < kLanesUsed) {
#pragma unroll
        for (int q = 0; q < NACC; q++) sm[warp][lane][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        constexpr int kGroups = R < 32 ? 1 : R / 32;
        double s[NACC];
#pragma unroll
        for (int q = 0; q < NACC; q++) s[q] = 0.0;
        for (int w = (R < 32 ? 0 : (r >> 5)); w < kWarps; w += kGroups) {
#pragma unroll
            for (int q = 0; q < NACC; q++) s[q] += sm[w][r & (kLanesUsed - 1)][q];
        }
#pragma unroll
        for (int q = 0; q < NACC; q++) dst[r * NACC + q] = s[q];
    }
}

template <typename T>
struct Nbr {
    vec2_t<T> a, b, c, x;   // the three neighbours and the site itself
};

struct Idx3 {
    int32_t i0, i1, i2;
};

__device__ __forceinline__ Idx3 load_idx(const int32_t* __restrict__ idx, int64_t istride, int64_t n) {
    return Idx3{__ldg(idx + n), __ldg(idx + istride + n), __ldg(idx + 2 * istride + n)};
}

template <typename T, int R>
__device__ __forceinline__ Nbr<T> gather_at(Idx3 j, int64_t n, int r, const vec2_t<T>* __restrict__ v) {
    Nbr<T> g;
    g.a = __ldg(v + (int64_t)j.i0 * R + r);
    g.b = __ldg(v + (int64_t)j.i1 * R + r);
    g.c = __ldg(v + (int64_t)j.i2 * R + r);
    g.x = __ldg(v + n * R + r);
    return g;
}

template <typename T, int R>
__device__ __forceinline__ Nbr<T> gather(const int32_t* __restrict__ idx, int64_t istride, int64_t n,
                                         int r, const vec2_t<T>* __restrict__ v) {
    return gather_at<T, R>(load_idx(idx, istride, n), n, r, v);
}

// y = c * (a + b + c3) + e * x - z   as a chain of fused multiply-adds (z may be 0).
template <typename T>
__device__ __forceinline__ T hop(T c, T a, T b, T c3, T e, T x, T z, bool onsite) {
    T t = onsite ? fma(e, x, -z) : -z;
    return fma(c, a, fma(c, b, fma(c, c3, t)));
}

// (s i)^m is real for even m and imaginary for odd m, so ODD selects the two FMAs that
// the non-zero part of the coefficient needs: acc += cr * y  or  acc += i ci * y.
template <typename T>
__device__ __forceinline__ void add_term(vec2_t<T>& a, bool odd, T cr, T ci, T yr, T yi) {
    if (odd) {
        a.x = fma(-ci, yi, a.x);
        a.y = fma(ci, yr, a.y);
    } else {
        a.x = fma(cr, yr, a.x);
        a.y = fma(cr, yi, a.y);
    }
}

// On-site factor of a recursion step: eps_n / E_max on the first step, 2 eps_n / E_max on the
// later ones (read pre-doubled when the Hamiltonian carries it: no DP multiply per item).
template <bool FIRST>
__device__ __forceinline__ double onsite_factor(const DevH& H, int64_t n) {
    if (FIRST) return __ldg(H.onsite + n);
    return H.onsite2 ? __ldg(H.onsite2 + n) : 2.0 * __ldg(H.onsite + n);
}

template <typename T>
__device__ __forceinline__ vec2_t<T> mk(T x, T y);
template <>
__device__ __forceinline__ double2 mk<double>(double x, double y) { return make_double2(x, y); }
template <>
__device__ __forceinline__ float2 mk<float>(float x, float y) { return make_float2(x, y); }

// Programmatic dependent launch.  The per-step kernels of a recursion are launched with
// programmatic stream serialisation, so the CTAs of step n+1 may become resident while
// step n still runs.  Each such kernel reads only constant data (the neighbour table,
// the on-site energies) before pdl_wait(), which returns once the previous grid has
// completed and its memory operations are visible; every read of a vector and every
// write comes after it.  pdl_trigger() right after the wait lets the next step's CTAs
// be scheduled as early as resources allow (they wait in turn), so the launch latency
// and the CTA ramp of step n+1 overlap the tail of step n.  Launched without the
// attribute, the wait returns at once and the trigger has no effect.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// --------------------------------------------------------------------------------
// KPM step with phi_L = phi_R (DOS and MSD moments).  Uses the Chebyshev product
// identity 2 T_m T_n = T_{m+n} + T_{|m-n|}, so one recursion step n yields two moments:
//   mu_{2n} = 2 <phi_n|phi_n> - mu_0,   mu_{2n+1} = 2 <phi_{n+1}|phi_n> - mu_1
// (both real for Hermitian H~).  The kernel computes phi_{n+1} = 2H~phi_n - phi_{n-1}
// (first step: phi_1 = H~ phi_0) and the two per-block partial sums.
// --------------------------------------------------------------------------------
// Every kernel below loads the neighbour indices of its next item one iteration
// ahead: an iteration then waits only for its gathers, not for an index load followed
// by the gathers.  (Measured on the 2.1M-site sheet: FP64 KPM step 113 -> 103 us,
// complex64 95 -> 80 us; a second item per thread in flight adds registers and no
// speed once the indices are prefetched.)

template <typename T, int R, bool ONSITE, bool FIRST>
__global__ void __launch_bounds__(kBlock<T>) kpm_sym_kernel(DevH H, const vec2_t<T>* __restrict__ cur,
                                                            const vec2_t<T>* prev, vec2_t<T>* out,
                                                            double* __restrict__ partial) {
    constexpr int NT = kBlock<T>;
    const int64_t n_items = H.n * R;
    const int64_t stride = (int64_t)gridDim.x * NT;
    const int r = threadIdx.x & (R - 1);
    const T c = (T)(FIRST ? H.h : 2.0 * H.h);
    Acc<T> a0, a1;
    int64_t w = (int64_t)blockIdx.x * NT + threadIdx.x;
    Idx3 nid;
    if (w < n_items) nid = load_idx(H.idx, H.istride, w / R);
    pdl_wait();
    pdl_trigger();
    for (; w < n_items; w += stride) {
        const int64_t n = w / R;
        const Nbr<T> g = gather_at<T, R>(nid, n, r, cur);
        T e = 0;
        if constexpr (ONSITE) e = (T)onsite_factor<FIRST>(H, n);
        vec2_t<T> z = mk<T>(0, 0);
        if constexpr (!FIRST) z = prev[w];
        if (w + stride < n_items) nid = load_idx(H.idx, H.istride, (w + stride) / R);
        const T yr = hop<T>(c, g.a.x, g.b.x, g.c.x, e, g.x.x, z.x, ONSITE);
        const T yi = hop<T>(c, g.a.y, g.b.y, g.c.y, e, g.x.y, z.y, ONSITE);
        out[w] = mk<T>(yr, yi);
        a0.add_prod(g.x.x, g.x.x);
        a0.add_prod(g.x.y, g.x.y);
        a1.add_prod(yr, g.x.x);
        a1.add_prod(yi, g.x.y);
    }
    double acc[2] = {a0.value(), a1.value()};
    block_reduce<R, 2, NT>(acc, partial + (int64_t)blockIdx.x * R * 2);
}

// --------------------------------------------------------------------------------
// KPM step with a separate phi_L (VAC moments, Algorithm 5):
//   phi_{n+1} = 2H~phi_n - phi_{n-1};  C_{n+1} = <phi_L|phi_{n+1}>
// First step: phi_1 = H~ phi_0 and partials (<L|phi_1>, <L|phi_0>).
// --------------------------------------------------------------------------------
template <typename T, int R, bool ONSITE, bool FIRST>
__global__ void __launch_bounds__(kBlock<T>) kpm_gen_kernel(DevH H, const vec2_t<T>* __restrict__ L,
                                                           const vec2_t<T>* __restrict__ cur,
                                                           const vec2_t<T>* prev, vec2_t<T>* out,
                                                           double* __restrict__ partial) {
    constexpr int NACC = FIRST ? 4 : 2;
    constexpr int NT = kBlock<T>;
    const int64_t n_items = H.n * R;
    const int64_t stride = (int64_t)gridDim.x * NT;
    const int r = threadIdx.x & (R - 1);
    const T c = (T)(FIRST ? H.h : 2.0 * H.h);
    Acc<T> a[NACC];
    int64_t w = (int64_t)blockIdx.x * NT + threadIdx.x;
    Idx3 nid;
    if (w < n_items) nid = load_idx(H.idx, H.istride, w / R);
    pdl_wait();
    pdl_trigger();
    for (; w < n_items; w += stride) {
        const int64_t n = w / R;
        const Nbr<T> g = gather_at<T, R>(nid, n, r, cur);
        T e = 0;
        if constexpr (ONSITE) e = (T)onsite_factor<FIRST>(H, n);
        vec2_t<T> z = mk<T>(0, 0);
        if constexpr (!FIRST) z = prev[w];
        const vec2_t<T> l = __ldg(L + w);
        if (w + stride < n_items) nid = load_idx(H.idx, H.istride, (w + stride) / R);
        const T yr = hop<T>(c, g.a.x, g.b.x, g.c.x, e, g.x.x, z.x, ONSITE);
        const T yi = hop<T>(c, g.a.y, g.b.y, g.c.y, e, g.x.y, z.y, ONSITE);
        out[w] = mk<T>(yr, yi);
        // <L|y> = (l.x y.x + l.y y.y) + i (l.x y.y - l.y y.x)
        a[0].add_prod(l.x, yr);
        a[0].add_prod(l.y, yi);
        a[1].add_prod(l.x, yi);
        a[1].add_prod(-l.y, yr);
        if constexpr (FIRST) {
            a[2].add_prod(l.x, g.x.x);
            a[2].add_prod(l.y, g.x.y);
            a[3].add_prod(l.x, g.x.y);
            a[3].add_prod(-l.y, g.x.x);
        }
    }
    double acc[NACC];
#pragma unroll
    for (int q = 0; q < NACC; q++) acc[q] = a[q].value();
    block_reduce<R, NACC, NT>(acc, partial + (int64_t)blockIdx.x * R * NACC);
}

// --------------------------------------------------------------------------------
// Small instances: many KPM steps in one launch of one thread-block cluster, with the
// vectors resident in the cluster's shared memory.
// A 4096-site sheet with one vector is a few CTAs of work per step; one launch per step
// then costs several times the step, and so do global-memory round trips between steps.
// Here one cluster of G <= 16 CTAs of nt threads (one item w = n R + r per thread, CTA
// b owning items b nt .. b nt + nt - 1) runs the recursion steps of a chunk:
//   * each CTA keeps its items of phi_n and phi_{n-1} in shared memory (two buffers of
//     nt + 1 entries; entry nt is a permanent zero, the stand-in for the zero row N);
//   * a step reads the three neighbours through distributed shared memory (the owner
//     CTA of item j R + r is (j R + r) / nt), forms phi_{n+1} = 2 H~ phi_n - phi_{n-1}
//     with the per-step kernels' arithmetic (so the vectors are bitwise theirs) and
//     writes it in place over phi_{n-1};
//   * the two inner products are formed per thread (Acc<T>), merged across the lanes
//     that hold the same vector by double-float additions (TwoSum), and stored per warp
//     in a shared-memory table [step][warp][r]; the cross-warp sums, in a fixed order,
//     are done once at the end of the chunk and written to the ring slabs [step][G][R][2]
//     that the moment reduction reads;
//   * steps are separated by the cluster's hardware barrier (arrive.release /
//     wait.acquire at cluster scope), which every thread of every CTA reaches once per
//     step (and once before the first step, so no CTA reads a peer that has not started):
//     no spin loop.  After the last step each CTA writes its phi_n and phi_{n-1} back to
//     the global blocks that the per-step loop's pointer rotation would leave them in.
// --------------------------------------------------------------------------------
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// The two halves of the cluster barrier, for work between them that peers do not read.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

__device__ __forceinline__ uint32_t map_cluster_rank(uint32_t local_smem, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(local_smem), "r"(rank));
    return a;
}

__device__ __forceinline__ void ld_cluster(uint32_t a, double2& v) {
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
}
__device__ __forceinline__ void ld_cluster(uint32_t a, float2& v) {
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
}

// (s, c) += (s2, c2) for double-float pairs: Knuth's TwoSum of the heads, the tails and
// the rounding error summed, then renormalised (FastTwoSum).  Exact roundings throughout.
__device__ __forceinline__ void df_merge(float& s, float& c, float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    const float cc = __fadd_rn(__fadd_rn(c, c2), err);
    s = __fadd_rn(t, cc);
    c = __fsub_rn(cc, __fsub_rn(s, t));
}

constexpr int kClusterMaxR = 16;   // vectors per block the cluster path takes

// first = 1: the chunk starts with the first recursion step (phi_1 = H~ phi_0 with the
// hopping h, no phi_{-1} term: the per-step kernels' FIRST arithmetic), whose partial sums
// go to ring slab 0 like any step's (for the general recursion, <L|phi_0> goes to the
// extra slab nsteps).  The chunk reads its phi_n and phi_{n-1} from src_cur / src_prev
// (src_prev unused when first) and leaves its last phi_n and phi_{n-1} in dst_cur /
// dst_prev, the blocks the per-step loop's pointer rotation would leave them in.
template <typename T, int R, bool ONSITE, bool SYM>
__global__ void __launch_bounds__(512) kpm_cluster_kernel(DevH H, const vec2_t<T>* __restrict__ L,
                                                         const vec2_t<T>* src_cur, const vec2_t<T>* src_prev,
                                                         vec2_t<T>* dst_cur, vec2_t<T>* dst_prev,
                                                         double* __restrict__ ring, int nsteps, int log_nt,
                                                         int first) {
    static_assert(R <= kClusterMaxR, "cluster path: at most 16 vectors per block");
    using V2 = vec2_t<T>;
    extern __shared__ __align__(16) unsigned char kg_cluster_smem[];
    const int nt = 1 << log_nt;
    const int nwarps = nt >> 5;
    V2* sv = reinterpret_cast<V2*>(kg_cluster_smem);                    // [2][nt + 1]
    float4* wp = reinterpret_cast<float4*>(sv + 2 * (nt + 1));          // [nsteps (+1)][nwarps][R]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int r = t & (R - 1);
    const int64_t n_items = H.n * R;
    const int64_t w = ((int64_t)blockIdx.x << log_nt) + t;
    const bool valid = w < n_items;
    const V2 zero = mk<T>(0, 0);

    // own items of phi_n (buffer 0) and phi_{n-1} (buffer 1), and the zero entries
    sv[t] = valid ? src_cur[w] : zero;
    sv[nt + 1 + t] = (valid && !first) ? src_prev[w] : zero;
    if (t == 0) {
        sv[nt] = zero;
        sv[2 * nt + 1] = zero;
    }
    // cluster addresses of the three neighbours in buffer 0 (buffer 1 is boff bytes on)
    const int64_t n = valid ? w / R : H.n;
    uint32_t na[3];
    {
        const Idx3 j = valid ? load_idx(H.idx, H.istride, n) : Idx3{(int32_t)H.n, (int32_t)H.n, (int32_t)H.n};
        const int32_t jj[3] = {j.i0, j.i1, j.i2};
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(sv);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const int64_t item = (int64_t)jj[q] * R + r;
            const bool zr = jj[q] >= H.n;   // removed or missing neighbour: the zero entry
            const uint32_t rank = zr ? blockIdx.x : (uint32_t)(item >> log_nt);
            const uint32_t slot = zr ? (uint32_t)nt : (uint32_t)(item & (nt - 1));
            na[q] = map_cluster_rank(base + slot * (uint32_t)sizeof(V2), rank);
        }
    }
    T e1 = 0, e2 = 0;
    if constexpr (ONSITE) {
        const double o = valid ? __ldg(H.onsite + n) : 0.0;
        e1 = (T)(1.0 * o);
        e2 = (T)(2.0 * o);
    }
    V2 l = zero;
    if constexpr (!SYM) l = valid ? __ldg(L + w) : zero;
    const T c1 = (T)H.h, c2 = (T)(2.0 * H.h);
    const uint32_t boff = (uint32_t)((nt + 1) * sizeof(V2));
    cluster_barrier();   // every CTA's buffers are filled before any peer reads them

    int cb = 0;   // buffer holding phi_n
    for (int k = 0; k < nsteps; k++) {
        const bool fs = first && k == 0;
        const T c = fs ? c1 : c2;
        const T e = fs ? e1 : e2;
        const uint32_t o = cb ? boff : 0u;
        V2 ga, gb, gc;
        ld_cluster(na[0] + o, ga);
        ld_cluster(na[1] + o, gb);
        ld_cluster(na[2] + o, gc);
        V2* curb = sv + cb * (nt + 1);
        V2* prvb = sv + (cb ^ 1) * (nt + 1);
        const V2 x = curb[t];
        const V2 z = fs ? zero : prvb[t];
        const T yr = hop<T>(c, ga.x, gb.x, gc.x, e, x.x, z.x, ONSITE);
        const T yi = hop<T>(c, ga.y, gb.y, gc.y, e, x.y, z.y, ONSITE);
        if (valid) prvb[t] = mk<T>(yr, yi);
        // phi_{n+1} is written: release it to the peers now, and form this step's inner
        // products (registers and this CTA's own table only) while the barrier completes
        cluster_arrive();
        Acc<T> a0, a1;   // padding threads hold zeros and add nothing
        if constexpr (SYM) {
            a0.add_prod(x.x, x.x);
            a0.add_prod(x.y, x.y);
            a1.add_prod(yr, x.x);
            a1.add_prod(yi, x.y);
        } else {
            a0.add_prod(l.x, yr);
            a0.add_prod(l.y, yi);
            a1.add_prod(l.x, yi);
            a1.add_prod(-l.y, yr);
        }
        float s0 = a0.s, c0 = a0.c, s1 = a1.s, c1s = a1.c;
#pragma unroll
        for (int off = 16; off >= R; off >>= 1) {
            const float s0o = __shfl_xor_sync(0xffffffffu, s0, off), c0o = __shfl_xor_sync(0xffffffffu, c0, off);
            const float s1o = __shfl_xor_sync(0xffffffffu, s1, off), c1o = __shfl_xor_sync(0xffffffffu, c1s, off);
            df_merge(s0, c0, s0o, c0o);
            df_merge(s1, c1s, s1o, c1o);
        }
        if (lane < R) wp[((int64_t)k * nwarps + warp) * R + lane] = make_float4(s0, c0, s1, c1s);
        if constexpr (!SYM) {
            if (fs) {
                // <L|phi_0> of the first step, kept as step nsteps
                Acc<T> b0, b1;
                b0.add_prod(l.x, x.x);
                b0.add_prod(l.y, x.y);
                b1.add_prod(l.x, x.y);
                b1.add_prod(-l.y, x.x);
                float u0 = b0.s, v0 = b0.c, u1 = b1.s, v1 = b1.c;
#pragma unroll
                for (int off = 16; off >= R; off >>= 1) {
                    const float u0o = __shfl_xor_sync(0xffffffffu, u0, off), v0o = __shfl_xor_sync(0xffffffffu, v0, off);
                    const float u1o = __shfl_xor_sync(0xffffffffu, u1, off), v1o = __shfl_xor_sync(0xffffffffu, v1, off);
                    df_merge(u0, v0, u0o, v0o);
                    df_merge(u1, v1, u1o, v1o);
                }
                if (lane < R) wp[((int64_t)nsteps * nwarps + warp) * R + lane] = make_float4(u0, v0, u1, v1);
            }
        }
        cluster_wait();   // every peer's phi_{n+1} is visible before the next step's gathers
        cb ^= 1;
    }
    // no peer reads this CTA's buffers any more; write phi_n and phi_{n-1} back
    if (valid) {
        dst_cur[w] = sv[cb * (nt + 1) + t];
        dst_prev[w] = sv[(cb ^ 1) * (nt + 1) + t];
    }
    __syncthreads();   // the last step's per-warp sums (written after its arrive) are in wp
    // cross-warp sums per (step, vector, product), fixed order, into ring slab k
    const int nslab = nsteps + ((!SYM && first) ? 1 : 0);
    for (int i = t; i < nslab * R * 2; i += nt) {
        const int k = i / (2 * R), rr = (i >> 1) & (R - 1), q = i & 1;
        float s = 0.0f, cc = 0.0f;
        for (int wi = 0; wi < nwarps; wi++) {
            const float4 v = wp[((int64_t)k * nwarps + wi) * R + rr];
            if (q == 0) df_merge(s, cc, v.x, v.y);
            else df_merge(s, cc, v.z, v.w);
        }
        ring[(((int64_t)k * gridDim.x + blockIdx.x) * R + rr) * 2 + q] = (double)s + (double)cc;
    }
}

// --------------------------------------------------------------------------------
// Small instances: the whole Chebyshev-Bessel series of one time step (Algorithms 6
// and 7, Eqs. 36-39) in one launch of one thread-block cluster.
// Per term the per-term kernel below (evolve_kernel) is a few microseconds of launch
// for a few microseconds of work; here the cluster's CTAs keep, for every chain, the two
// latest terms p_{m-1} and p_{m-2} in shared memory (two buffers of nt + 1 entries per
// chain, entry nt a permanent zero), read the neighbours of p_{m-1} through distributed
// shared memory, write p_m in place over p_{m-2}, and keep the series accumulators in
// registers.  The commutator chain q_m of the last plain chain (Eq. 39) is a third
// chain with its own two buffers.  One cluster barrier separates the terms.  The
// arithmetic of a term (hop, add_term and their order) is that of evolve_kernel, so the
// results are bitwise those of the per-term launches.
// --------------------------------------------------------------------------------
// With cf.norm_out set, the kernel also forms ||acc_{cf.norm_chain}||^2 of each vector (the
// unitarity check of the time loops, Eq. 36): per thread in the inner-product arithmetic
// of the per-step kernels (Acc<T>), merged across lanes by double-float additions, per CTA
// over its warps in a fixed order, and over the cluster's CTAs by CTA 0 through
// distributed shared memory in rank order; written as (||x||^2, 0).
template <typename T, int R, int NCH, bool XC, bool ONSITE, bool YPAR>
__global__ void __launch_bounds__(512) evolve_cluster_kernel(DevH H, ChainsT<T> ch, SeriesCoef cf, int log_nt) {
    static_assert(R <= kClusterMaxR, "cluster path: at most 16 vectors per block");
    using V2 = vec2_t<T>;
    constexpr int NB = NCH + (XC ? 1 : 0);   // chains held in shared memory
    extern __shared__ __align__(16) unsigned char kg_cluster_smem[];
    const int nt = 1 << log_nt;
    V2* sv = reinterpret_cast<V2*>(kg_cluster_smem);   // [NB][2][nt + 1]
    const int t = threadIdx.x;
    const int r = t & (R - 1);
    const int64_t n_items = H.n * R;
    const int64_t w = ((int64_t)blockIdx.x << log_nt) + t;
    const bool valid = w < n_items;
    const V2 zero = mk<T>(0, 0);
    auto buf = [&](int k, int b) { return sv + (k * 2 + b) * (nt + 1); };

#pragma unroll
    for (int k = 0; k < NCH; k++) {
        buf(k, 0)[t] = valid ? ch.cur[k][w] : zero;
        buf(k, 1)[t] = zero;
    }
    if constexpr (XC) {
        buf(NCH, 0)[t] = zero;
        buf(NCH, 1)[t] = zero;
    }
    if (t == 0) {
        for (int k = 0; k < NB; k++) {
            buf(k, 0)[nt] = zero;
            buf(k, 1)[nt] = zero;
        }
    }
    // cluster addresses of the three neighbours in buffer (0, 0); buffer (k, b) is
    // (2 k + b)(nt + 1) entries further on
    const int64_t n = valid ? w / R : H.n;
    uint32_t na[3];
    {
        const Idx3 j = valid ? load_idx(H.idx, H.istride, n) : Idx3{(int32_t)H.n, (int32_t)H.n, (int32_t)H.n};
        const int32_t jj[3] = {j.i0, j.i1, j.i2};
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(sv);
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const int64_t item = (int64_t)jj[q] * R + r;
            const bool zr = jj[q] >= H.n;
            const uint32_t rank = zr ? blockIdx.x : (uint32_t)(item >> log_nt);
            const uint32_t slot = zr ? (uint32_t)nt : (uint32_t)(item & (nt - 1));
            na[q] = map_cluster_rank(base + slot * (uint32_t)sizeof(V2), rank);
        }
    }
    T e1 = 0, e2 = 0;
    if constexpr (ONSITE) {
        const double o = valid ? __ldg(H.onsite + n) : 0.0;
        e1 = (T)(1.0 * o);
        e2 = (T)(2.0 * o);
    }
    double d0d = 0, d1d = 0, d2d = 0;
    if constexpr (XC) {
        if constexpr (YPAR) {
            const int p = valid ? __ldg(H.parity + n) : 0;
            d0d = H.dh[p][0]; d1d = H.dh[p][1]; d2d = H.dh[p][2];
        } else {
            d0d = H.dh[0][0]; d1d = H.dh[0][1]; d2d = H.dh[0][2];
        }
    }
    const bool q_into_0 = (ch.qacc == nullptr);
    const T j0 = (T)cf.j0;
    const uint32_t bstride = (uint32_t)((nt + 1) * sizeof(V2));
    V2 acc[NCH];
    V2 qa = zero;
    cluster_barrier();   // every CTA's buffers are filled before any peer reads them

    int cb = 0;   // buffer holding p_{m-1}
    for (int m = 1; m <= cf.nterms; m++) {
        const bool first = m == 1;
        const T c = first ? (T)H.h : (T)(2.0 * H.h);
        const T e = first ? e1 : e2;
        const T cr = (T)cf.cr[m], ci = (T)cf.ci[m];
        const bool odd = first || cf.cr[m] == 0.0;
        V2 q_add = zero;
        V2 gsa = zero, gsb = zero, gsc = zero;
#pragma unroll
        for (int k = 0; k < NCH; k++) {
            const uint32_t off = (uint32_t)(k * 2 + cb) * bstride;
            V2 ga, gb, gc;
            ld_cluster(na[0] + off, ga);
            ld_cluster(na[1] + off, gb);
            ld_cluster(na[2] + off, gc);
            const V2 x = buf(k, cb)[t];
            const V2 z = first ? zero : buf(k, cb ^ 1)[t];
            const T yr = hop<T>(c, ga.x, gb.x, gc.x, e, x.x, z.x, ONSITE);
            const T yi = hop<T>(c, ga.y, gb.y, gc.y, e, x.y, z.y, ONSITE);
            if (valid) buf(k, cb ^ 1)[t] = mk<T>(yr, yi);
            V2 a = first ? mk<T>(j0 * x.x, j0 * x.y) : acc[k];
            add_term<T>(a, odd, cr, ci, yr, yi);
            if (k == 0) q_add = a;
            else acc[k] = a;
            if (k == NCH - 1) {
                gsa = ga;
                gsb = gb;
                gsc = gc;
            }
        }
        if constexpr (XC) {
            const T cx = first ? (T)1 : (T)2;
            const T d0 = cx * (T)d0d, d1 = cx * (T)d1d, d2 = cx * (T)d2d;
            T qr, qi;
            if (first) {
                if constexpr (YPAR) {
                    qr = fma(d0, gsa.x, fma(d1, gsb.x, d2 * gsc.x));
                    qi = fma(d0, gsa.y, fma(d1, gsb.y, d2 * gsc.y));
                } else {
                    qr = fma(d0, gsa.x, d1 * gsb.x);
                    qi = fma(d0, gsa.y, d1 * gsb.y);
                }
            } else {
                const uint32_t off = (uint32_t)(NCH * 2 + cb) * bstride;
                V2 qa0, qb0, qc0;
                ld_cluster(na[0] + off, qa0);
                ld_cluster(na[1] + off, qb0);
                ld_cluster(na[2] + off, qc0);
                const V2 qx = buf(NCH, cb)[t];
                const V2 qz = buf(NCH, cb ^ 1)[t];   // zero at m = 2 (q_0 = 0)
                qr = hop<T>(c, qa0.x, qb0.x, qc0.x, e, qx.x, qz.x, ONSITE);
                qi = hop<T>(c, qa0.y, qb0.y, qc0.y, e, qx.y, qz.y, ONSITE);
                if constexpr (YPAR) {
                    qr = fma(d0, gsa.x, fma(d1, gsb.x, fma(d2, gsc.x, qr)));
                    qi = fma(d0, gsa.y, fma(d1, gsb.y, fma(d2, gsc.y, qi)));
                } else {
                    qr = fma(d0, gsa.x, fma(d1, gsb.x, qr));
                    qi = fma(d0, gsa.y, fma(d1, gsb.y, qi));
                }
            }
            if (valid) buf(NCH, cb ^ 1)[t] = mk<T>(qr, qi);
            if (q_into_0) {
                add_term<T>(q_add, odd, cr, ci, qr, qi);
            } else {
                if (first) qa = zero;
                add_term<T>(qa, odd, cr, ci, qr, qi);
            }
        }
        acc[0] = q_add;
        cluster_barrier();
        cb ^= 1;
    }
    if (valid) {
#pragma unroll
        for (int k = 0; k < NCH; k++) ch.acc[k][w] = acc[k];
        if constexpr (XC) {
            if (!q_into_0) ch.qacc[w] = qa;
        }
    }
    if (cf.norm_out != nullptr) {
        // after the chain buffers: [nwarps][R] float2 per-warp sums, then [R] doubles per CTA
        const int lane = t & 31, warp = t >> 5, nwarps = nt >> 5;
        float2* wsum = reinterpret_cast<float2*>(sv + NB * 2 * (nt + 1));
        double* csum = reinterpret_cast<double*>(wsum + nwarps * R);
        V2 xv = zero;
#pragma unroll
        for (int k = 0; k < NCH; k++)
            if (k == cf.norm_chain) xv = acc[k];
        Acc<T> a;   // invalid threads hold zeros
        a.add_prod(xv.x, xv.x);
        a.add_prod(xv.y, xv.y);
        float sn = a.s, cn = a.c;
#pragma unroll
        for (int off = 16; off >= R; off >>= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, sn, off), co = __shfl_xor_sync(0xffffffffu, cn, off);
            df_merge(sn, cn, so, co);
        }
        if (lane < R) wsum[warp * R + lane] = make_float2(sn, cn);
        __syncthreads();
        if (t < R) {
            float s2 = 0.0f, c2 = 0.0f;
            for (int wi = 0; wi < nwarps; wi++) df_merge(s2, c2, wsum[wi * R + t].x, wsum[wi * R + t].y);
            csum[t] = (double)s2 + (double)c2;
        }
        cluster_barrier();   // every CTA's sums are written
        if (blockIdx.x == 0 && t < R) {
            const uint32_t local = (uint32_t)__cvta_generic_to_shared(csum + t);
            double tot = 0.0;
            for (uint32_t b = 0; b < gridDim.x; b++) {
                double v;
                asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(map_cluster_rank(local, b)));
                tot += v;
            }
            cf.norm_out[t] = make_double2(tot, 0.0);
        }
        cluster_barrier();   // no CTA exits while CTA 0 still reads its sums
    }
}

// --------------------------------------------------------------------------------
// complex64 KPM steps with 128-bit accesses: for R >= 2 one thread owns the two adjacent
// vectors (2 r2, 2 r2 + 1) of a site and moves them as one float4, halving the load and
// store instructions per byte of the HBM-bound FP32 step.  Per-vector partial sums are
// kept separately, in the [R][NACC] order the reductions expect.
// --------------------------------------------------------------------------------
struct Nbr4 {
    float4 a, b, c, x;
};

template <int R2>
__device__ __forceinline__ Nbr4 gather_pair(Idx3 j, int64_t n, int r2, const float4* __restrict__ v) {
    Nbr4 g;
    g.a = __ldg(v + (int64_t)j.i0 * R2 + r2);
    g.b = __ldg(v + (int64_t)j.i1 * R2 + r2);
    g.c = __ldg(v + (int64_t)j.i2 * R2 + r2);
    g.x = __ldg(v + n * R2 + r2);
    return g;
}

template <int R, bool ONSITE, bool FIRST>
__global__ void __launch_bounds__(kThreads) kpm_sym_pair_kernel(DevH H, const float4* __restrict__ cur,
                                                                const float4* prev, float4* out,
                                                                double* __restrict__ partial) {
    constexpr int R2 = R / 2;
    const int64_t n_items = H.n * R2;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int r2 = threadIdx.x & (R2 - 1);
    const float c = (float)(FIRST ? H.h : 2.0 * H.h);
    Acc<float> s0, s1, t0, t1;   // <x|x>, <y|x> of vectors 2 r2 and 2 r2 + 1
    int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    Idx3 nid;
    if (w < n_items) nid = load_idx(H.idx, H.istride, w / R2);
    pdl_wait();
    pdl_trigger();
    for (; w < n_items; w += stride) {
        const int64_t n = w / R2;
        const Nbr4 g = gather_pair<R2>(nid, n, r2, cur);
        float e = 0.0f;
        if constexpr (ONSITE) e = (float)onsite_factor<FIRST>(H, n);
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (!FIRST) z = prev[w];
        if (w + stride < n_items) nid = load_idx(H.idx, H.istride, (w + stride) / R2);
        float4 y;
        y.x = hop<float>(c, g.a.x, g.b.x, g.c.x, e, g.x.x, z.x, ONSITE);
        y.y = hop<float>(c, g.a.y, g.b.y, g.c.y, e, g.x.y, z.y, ONSITE);
        y.z = hop<float>(c, g.a.z, g.b.z, g.c.z, e, g.x.z, z.z, ONSITE);
        y.w = hop<float>(c, g.a.w, g.b.w, g.c.w, e, g.x.w, z.w, ONSITE);
        out[w] = y;
        s0.add_prod(g.x.x, g.x.x);
        s0.add_prod(g.x.y, g.x.y);
        s1.add_prod(y.x, g.x.x);
        s1.add_prod(y.y, g.x.y);
        t0.add_prod(g.x.z, g.x.z);
        t0.add_prod(g.x.w, g.x.w);
        t1.add_prod(y.z, g.x.z);
        t1.add_prod(y.w, g.x.w);
    }
    double acc[4] = {s0.value(), s1.value(), t0.value(), t1.value()};
    block_reduce<R2, 4, kThreads>(acc, partial + (int64_t)blockIdx.x * R * 2);
}

template <int R, bool ONSITE, bool FIRST>
__global__ void __launch_bounds__(kThreads) kpm_gen_pair_kernel(DevH H, const float4* __restrict__ L,
                                                                const float4* __restrict__ cur,
                                                                const float4* prev, float4* out,
                                                                double* __restrict__ partial) {
    constexpr int NACC = FIRST ? 4 : 2;
    constexpr int R2 = R / 2;
    const int64_t n_items = H.n * R2;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int r2 = threadIdx.x & (R2 - 1);
    const float c = (float)(FIRST ? H.h : 2.0 * H.h);
    Acc<float> a[2 * NACC];   // vector 2 r2: a[0..NACC), vector 2 r2 + 1: a[NACC..2 NACC)
    int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    Idx3 nid;
    if (w < n_items) nid = load_idx(H.idx, H.istride, w / R2);
    pdl_wait();
    pdl_trigger();
    for (; w < n_items; w += stride) {
        const int64_t n = w / R2;
        const Nbr4 g = gather_pair<R2>(nid, n, r2, cur);
        float e = 0.0f;
        if constexpr (ONSITE) e = (float)onsite_factor<FIRST>(H, n);
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (!FIRST) z = prev[w];
        const float4 l = __ldg(L + w);
        if (w + stride < n_items) nid = load_idx(H.idx, H.istride, (w + stride) / R2);
        float4 y;
        y.x = hop<float>(c, g.a.x, g.b.x, g.c.x, e, g.x.x, z.x, ONSITE);
        y.y = hop<float>(c, g.a.y, g.b.y, g.c.y, e, g.x.y, z.y, ONSITE);
        y.z = hop<float>(c, g.a.z, g.b.z, g.c.z, e, g.x.z, z.z, ONSITE);
        y.w = hop<float>(c, g.a.w, g.b.w, g.c.w, e, g.x.w, z.w, ONSITE);
        out[w] = y;
        // <L|y> = (l.x y.x + l.y y.y) + i (l.x y.y - l.y y.x), per vector of the pair
        a[0].add_prod(l.x, y.x);
        a[0].add_prod(l.y, y.y);
        a[1].add_prod(l.x, y.y);
        a[1].add_prod(-l.y, y.x);
        a[NACC].add_prod(l.z, y.z);
        a[NACC].add_prod(l.w, y.w);
        a[NACC + 1].add_prod(l.z, y.w);
        a[NACC + 1].add_prod(-l.w, y.z);
        if constexpr (FIRST) {
            a[2].add_prod(l.x, g.x.x);
            a[2].add_prod(l.y, g.x.y);
            a[3].add_prod(l.x, g.x.y);
            a[3].add_prod(-l.y, g.x.x);
            a[NACC + 2].add_prod(l.z, g.x.z);
            a[NACC + 2].add_prod(l.w, g.x.w);
            a[NACC + 3].add_prod(l.z, g.x.w);
            a[NACC + 3].add_prod(-l.w, g.x.z);
        }
    }
    double acc[2 * NACC];
#pragma unroll
    for (int q = 0; q < 2 * NACC; q++) acc[q] = a[q].value();
    block_reduce<R2, 2 * NACC, kThreads>(acc, partial + (int64_t)blockIdx.x * R * NACC);
}

// --------------------------------------------------------------------------------
// Reductions of per-block partials into moments (fixed order => deterministic).
// --------------------------------------------------------------------------------

// Sum over g of part[g][R][A] for (r, q) -> out[r][q].  256 threads; pairs are
// assigned round-robin, each pair's threads sum a strided subset then combine in a
// fixed order through shared memory.
__device__ void reduce_blocks(const double* __restrict__ part, int grid, int R, int A,
                              double* __restrict__ out_rq) {
    __shared__ double sm[kThreads];
    const int pairs = R * A;
    const int tpp = kThreads / pairs;   // threads per pair (>= 1, pairs <= 256)
    const int t = threadIdx.x;
    const int pair = t / tpp, sub = t % tpp;
    double s = 0.0;
    if (pair < pairs) {
        const int r = pair / A, q = pair % A;
        for (int g = sub; g < grid; g += tpp) s += part[((int64_t)g * R + r) * A + q];
    }
    sm[t] = s;
    __syncthreads();
    if (t < pairs) {
        double v = 0.0;
        for (int k = 0; k < tpp; k++) v += sm[t * tpp + k];
        out_rq[t] = v;
    }
    __syncthreads();
}

__global__ void reduce_first_kernel(const double* __restrict__ part, int grid, int R, int sym,
                                    double2* mu, int64_t r_stride, int M) {
    __shared__ double res[kThreads];
    const int A = sym ? 2 : 4;
    reduce_blocks(part, grid, R, A, res);
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        double2* m = mu + r * r_stride;
        if (sym) {
            m[0] = make_double2(res[r * 2 + 0], 0.0);
            if (M > 1) m[1] = make_double2(res[r * 2 + 1], 0.0);
        } else {
            m[0] = make_double2(res[r * 4 + 2], res[r * 4 + 3]);
            if (M > 1) m[1] = make_double2(res[r * 4 + 0], res[r * 4 + 1]);
        }
    }
}

// first = 1 (slab slab0 holds the first step, n0 = 0): the first step's sums are the
// moments themselves (mu_0 = S0(0), mu_1 = S1(0) with doubling; mu_1 = <L|phi_1>), every
// block re-reduces slab slab0 for mu_0 and mu_1 instead of reading them back (no order
// between the blocks of one launch), and for the general recursion the last block's
// slab holds <L|phi_0> = mu_0.
__global__ void reduce_ring_kernel(const double* __restrict__ ring, int slab0, int ring_size,
                                   int grid, int R, int sym, int n0, double2* mu, int64_t r_stride,
                                   int M, int first) {
    __shared__ double res[kThreads];
    __shared__ double res0[kThreads];
    const int slab = (slab0 + blockIdx.x) % ring_size;
    const int n = n0 + blockIdx.x;   // recursion step that produced this slab
    reduce_blocks(ring + (int64_t)slab * grid * R * 2, grid, R, 2, res);
    if (first && sym) reduce_blocks(ring + (int64_t)(slab0 % ring_size) * grid * R * 2, grid, R, 2, res0);
    if (threadIdx.x < R) {
        const int r = threadIdx.x;
        double2* m = mu + r * r_stride;
        if (sym) {
            if (first && n == 0) {
                m[0] = make_double2(res[r * 2], 0.0);
                if (M > 1) m[1] = make_double2(res[r * 2 + 1], 0.0);
            } else {
                const double mu0 = first ? res0[r * 2] : m[0].x, mu1 = first ? res0[r * 2 + 1] : m[1].x;
                if (2 * n < M) m[2 * n] = make_double2(2.0 * res[r * 2] - mu0, 0.0);
                if (2 * n + 1 < M) m[2 * n + 1] = make_double2(2.0 * res[r * 2 + 1] - mu1, 0.0);
            }
        } else if (first && blockIdx.x == gridDim.x - 1) {
            m[0] = make_double2(res[r * 2], res[r * 2 + 1]);   // <L|phi_0>
        } else {
            if (n + 1 < M) m[n + 1] = make_double2(res[r * 2], res[r * 2 + 1]);
        }
    }
}

// --------------------------------------------------------------------------------
// One term of the Chebyshev-Bessel series (Algorithms 6 and 7) on NCH chains.
// Plain chain k:   p_m = 2H~p_{m-1} - p_{m-2}  (first: p_1 = H~p_0)
//                  acc_k += (cr + i ci) p_m    (first: acc_k = J_0 p_0 + (cr + i ci) p_1)
// Commutator chain of the last plain chain s (Eq. 39):
//                  q_m = 2[X,H~]p_{m-1} + 2H~q_{m-1} - q_{m-2}  (first: q_1 = [X,H~]p_0)
//                  qacc += (cr + i ci) q_m  (into acc_0 when qacc is null)
// [X,H~] has the same sparsity as H~ with per-slot factors (X_n - X_m) H~_nm, so it
// reuses the gathered neighbours of chain s.
// --------------------------------------------------------------------------------

template <typename T, int R, int NCH, bool XC, bool FIRST, bool ONSITE, bool YPAR, bool ODD>
__global__ void __launch_bounds__(kBlock<T>) evolve_kernel(DevH H, double j0d, double crd, double cid,
                                                          ChainsT<T> ch) {
    using V2 = vec2_t<T>;
    const int64_t n_items = H.n * R;
    const int64_t stride = (int64_t)gridDim.x * kBlock<T>;
    const int r = threadIdx.x & (R - 1);
    const T c = (T)(FIRST ? H.h : 2.0 * H.h);
    const T cx = FIRST ? (T)1 : (T)2;
    const T j0 = (T)j0d, cr = (T)crd, ci = (T)cid;
    const bool q_into_0 = (ch.qacc == nullptr);
    int64_t w = (int64_t)blockIdx.x * kBlock<T> + threadIdx.x;
    Idx3 nid;
    if (w < n_items) nid = load_idx(H.idx, H.istride, w / R);
    pdl_wait();
    pdl_trigger();
    for (; w < n_items; w += stride) {
        const int64_t n = w / R;
        const Idx3 id = nid;
        if (w + stride < n_items) nid = load_idx(H.idx, H.istride, (w + stride) / R);
        T e = 0;
        if constexpr (ONSITE) e = (T)onsite_factor<FIRST>(H, n);
        V2 q_add = mk<T>(0, 0);   // chain-0 accumulator, finished after the commutator chain
        Nbr<T> gs;
#pragma unroll
        for (int k = 0; k < NCH; k++) {
            const Nbr<T> g = gather_at<T, R>(id, n, r, ch.cur[k]);
            if (k == NCH - 1) gs = g;
            V2 z = mk<T>(0, 0);
            if constexpr (!FIRST) z = ch.prev[k][w];
            const T yr = hop<T>(c, g.a.x, g.b.x, g.c.x, e, g.x.x, z.x, ONSITE);
            const T yi = hop<T>(c, g.a.y, g.b.y, g.c.y, e, g.x.y, z.y, ONSITE);
            ch.nxt[k][w] = mk<T>(yr, yi);
            V2 a;
            if constexpr (FIRST) {
                a = mk<T>(j0 * g.x.x, j0 * g.x.y);
            } else {
                a = ch.acc[k][w];
            }
            add_term<T>(a, ODD, cr, ci, yr, yi);
            if (k == 0) {
                q_add = a;
            } else {
                ch.acc[k][w] = a;
            }
        }
        if constexpr (XC) {
            // [X,H~] p_{m-1}: sum over slots of (X_n - X_m) H~_nm p[nbr]
            double d0d, d1d, d2d;
            if constexpr (YPAR) {
                const int p = __ldg(H.parity + n);
                d0d = H.dh[p][0]; d1d = H.dh[p][1]; d2d = H.dh[p][2];
            } else {
                d0d = H.dh[0][0]; d1d = H.dh[0][1]; d2d = H.dh[0][2];
            }
            const T d0 = cx * (T)d0d, d1 = cx * (T)d1d, d2 = cx * (T)d2d;
            T qr, qi;
            // transport along x: the bond to the adjacent chain is vertical, (X_n - X_m) = 0,
            // so its term is dropped (d2 = 0); along y all three slots contribute
            if constexpr (FIRST) {
                if constexpr (YPAR) {
                    qr = fma(d0, gs.a.x, fma(d1, gs.b.x, d2 * gs.c.x));
                    qi = fma(d0, gs.a.y, fma(d1, gs.b.y, d2 * gs.c.y));
                } else {
                    qr = fma(d0, gs.a.x, d1 * gs.b.x);
                    qi = fma(d0, gs.a.y, d1 * gs.b.y);
                }
            } else {
                const Nbr<T> gq = gather_at<T, R>(id, n, r, ch.qcur);
                V2 qz = mk<T>(0, 0);
                if (ch.qprev) qz = ch.qprev[w];
                qr = hop<T>(c, gq.a.x, gq.b.x, gq.c.x, e, gq.x.x, qz.x, ONSITE);
                qi = hop<T>(c, gq.a.y, gq.b.y, gq.c.y, e, gq.x.y, qz.y, ONSITE);
                if constexpr (YPAR) {
                    qr = fma(d0, gs.a.x, fma(d1, gs.b.x, fma(d2, gs.c.x, qr)));
                    qi = fma(d0, gs.a.y, fma(d1, gs.b.y, fma(d2, gs.c.y, qi)));
                } else {
                    qr = fma(d0, gs.a.x, fma(d1, gs.b.x, qr));
                    qi = fma(d0, gs.a.y, fma(d1, gs.b.y, qi));
                }
            }
            ch.qnxt[w] = mk<T>(qr, qi);
            if (q_into_0) {
                add_term<T>(q_add, ODD, cr, ci, qr, qi);
            } else {
                V2 a = FIRST ? mk<T>(0, 0) : ch.qacc[w];
                add_term<T>(a, ODD, cr, ci, qr, qi);
                ch.qacc[w] = a;
            }
        }
        ch.acc[0][w] = q_add;
    }
}

// --------------------------------------------------------------------------------
// out = H~ in, [X,H~] in, or V in = -(i E_max/hbar) [X,H~] in (Eq. 15).
// --------------------------------------------------------------------------------
template <typename T, int R, int OP, bool ONSITE, bool YPAR>
__global__ void __launch_bounds__(kThreads) apply_kernel(DevH H, double scaled,
                                                         const vec2_t<T>* __restrict__ in,
                                                         vec2_t<T>* __restrict__ out) {
    const int64_t n_items = H.n * R;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int r = threadIdx.x & (R - 1);
    const T scale = (T)scaled;
    for (int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x; w < n_items; w += stride) {
        const int64_t n = w / R;
        const Nbr<T> g = gather<T, R>(H.idx, H.istride, n, r, in);
        if constexpr (OP == 0) {
            T e = 0;
            if constexpr (ONSITE) e = (T)__ldg(H.onsite + n);
            const T h = (T)H.h;
            out[w] = mk<T>(hop<T>(h, g.a.x, g.b.x, g.c.x, e, g.x.x, 0, ONSITE),
                           hop<T>(h, g.a.y, g.b.y, g.c.y, e, g.x.y, 0, ONSITE));
        } else {
            double d0d, d1d, d2d;
            if constexpr (YPAR) {
                const int p = __ldg(H.parity + n);
                d0d = H.dh[p][0]; d1d = H.dh[p][1]; d2d = H.dh[p][2];
            } else {
                d0d = H.dh[0][0]; d1d = H.dh[0][1]; d2d = H.dh[0][2];
            }
            const T d0 = (T)d0d, d1 = (T)d1d, d2 = (T)d2d;
            const T qr = fma(d0, g.a.x, fma(d1, g.b.x, d2 * g.c.x));
            const T qi = fma(d0, g.a.y, fma(d1, g.b.y, d2 * g.c.y));
            if constexpr (OP == 1) out[w] = mk<T>(qr, qi);
            else out[w] = mk<T>(scale * qi, -scale * qr);   // -(i s)(qr + i qi)
        }
    }
}

// complex128 -> complex64 (rounded to nearest), n_items elements.
__global__ void to_c64_kernel(const double2* __restrict__ in, float2* __restrict__ out, int64_t n_items) {
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x; w < n_items; w += stride) {
        const double2 v = in[w];
        out[w] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
    }
}

// --------------------------------------------------------------------------------
// Inner products <L|X> of R vector pairs (Fourier moments, Algorithm 4).
// --------------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(kThreads) dot_kernel(int64_t n_items, const vec2_t<T>* __restrict__ L,
                                                       const vec2_t<T>* __restrict__ X,
                                                       double* __restrict__ partial) {
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    Acc<T> a0, a1;
    for (int64_t w = (int64_t)blockIdx.x * kThreads + threadIdx.x; w < n_items; w += stride) {
        const vec2_t<T> l = __ldg(L + w), x = __ldg(X + w);
        a0.add_prod(l.x, x.x);
        a0.add_prod(l.y, x.y);
        a1.add_prod(l.x, x.y);
        a1.add_prod(-l.y, x.x);
    }
    double acc[2] = {a0.value(), a1.value()};
    block_reduce<R, 2, kThreads>(acc, partial + (int64_t)blockIdx.x * R * 2);
}

__global__ void reduce_dot_kernel(const double* __restrict__ part, int grid, int R, double2* out, int64_t r_stride) {
    __shared__ double res[kThreads];
    reduce_blocks(part, grid, R, 2, res);
    if (threadIdx.x < R) out[threadIdx.x * r_stride] = make_double2(res[threadIdx.x * 2], res[threadIdx.x * 2 + 1]);
}

// --------------------------------------------------------------------------------
// Launchers: runtime (R, flags) -> template instantiation.
// --------------------------------------------------------------------------------

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    return sms;
}

int stream_grid(int64_t n_items) {
    const int64_t need = (n_items + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)sm_count() * 6;   // a few resident waves worth of CTAs
    int64_t g = need < cap ? need : cap;
    return (int)(g < 1 ? 1 : g);
}

// Exactly one resident wave of a grid-stride kernel: SMs x co-resident CTAs per SM,
// capped by the work.  A partial second wave would leave most SMs idle at the end of
// every launch (the DP pipe is the bottleneck, so the tail costs its full share).
template <typename K>
static int one_wave_grid(K kernel, int64_t n_items, int threads = kThreads) {
    static thread_local std::unordered_map<const void*, int> cache;
    int per_sm = 0;
    auto it = cache.find((const void*)kernel);
    if (it != cache.end()) {
        per_sm = it->second;
    } else {
        // The grid-stride kernels keep at most a few KB in shared memory: give the rest of the
        // unified L1/shared storage to L1, which serves the in-chain neighbour gathers, but no
        // less shared memory than the CTAs that the registers allow need (static table + the
        // 1 KB the system reserves per CTA), so the carve-out never caps the occupancy.
        int by_regs = 0;
        cudaFuncAttributes fa{};
        int dev = 0, smem_sm = 0;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&by_regs, kernel, threads, 0) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
            smem_sm > 0) {
            const double need = (double)by_regs * ((double)fa.sharedSizeBytes + 1024.0);
            const int pct = std::min(100, std::max(0, (int)std::ceil(100.0 * need / smem_sm)));
            if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct) != cudaSuccess)
                cudaGetLastError();
        } else {
            cudaGetLastError();
        }
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        cache[(const void*)kernel] = per_sm;
    }
    const int64_t need = (n_items + threads - 1) / threads;
    const int64_t wave = (int64_t)sm_count() * per_sm;
    const int64_t g = need < wave ? need : wave;
    return (int)(g < 1 ? 1 : g);
}

// Launch with programmatic stream serialisation (see pdl_wait): used for the steps of a
// recursion after the first, whose predecessor in the stream is the previous step (or a
// reduction of partial sums), never a kernel that writes the neighbour table.
template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, int threads, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Launch of a recursion step: the first step plainly, later steps with PDL.
template <typename... KArgs, typename... Args>
static void launch_step(bool first, void (*kernel)(KArgs...), int grid, int threads, cudaStream_t s,
                        Args... args) {
    if (first) kernel<<<grid, threads, 0, s>>>(args...);
    else launch_pdl(kernel, grid, threads, s, args...);
}

#define KG_DISPATCH_R(R_, ...)                                   \
    switch (R_) {                                                \
        case 1: { constexpr int RR = 1; __VA_ARGS__; } break;    \
        case 2: { constexpr int RR = 2; __VA_ARGS__; } break;    \
        case 4: { constexpr int RR = 4; __VA_ARGS__; } break;    \
        case 8: { constexpr int RR = 8; __VA_ARGS__; } break;    \
        case 16: { constexpr int RR = 16; __VA_ARGS__; } break;  \
        case 32: { constexpr int RR = 32; __VA_ARGS__; } break;  \
        case 64: { constexpr int RR = 64; __VA_ARGS__; } break;  \
        default: return cudaErrorInvalidValue;                   \
    }

#define KG_BOOL(b_, NAME, ...)                         \
    if (b_) { constexpr bool NAME = true; __VA_ARGS__; } \
    else { constexpr bool NAME = false; __VA_ARGS__; }

// complex64 blocks of R >= 2 vectors use the paired (float4) kernels.
template <typename T>
constexpr bool kPaired = sizeof(T) == sizeof(float);

template <typename T>
cudaError_t launch_kpm_sym(const DevH& H, int R, bool first, const vec2_t<T>* cur, const vec2_t<T>* prev,
                           vec2_t<T>* out, double* partial, int grid, cudaStream_t s) {
    const bool ons = H.onsite != nullptr;
    if constexpr (kPaired<T>) {
        if (R >= 2) {
            const float4* c4 = reinterpret_cast<const float4*>(cur);
            const float4* p4 = reinterpret_cast<const float4*>(prev);
            float4* o4 = reinterpret_cast<float4*>(out);
            KG_DISPATCH_R(R, if constexpr (RR >= 2) { KG_BOOL(ons, ON, KG_BOOL(first, FI,
                launch_step(FI, kpm_sym_pair_kernel<RR, ON, FI>, grid, kThreads, s, H, c4, p4, o4, partial))) });
            return cudaGetLastError();
        }
    }
    KG_DISPATCH_R(R, KG_BOOL(ons, ON, KG_BOOL(first, FI,
        launch_step(FI, kpm_sym_kernel<T, RR, ON, FI>, grid, kBlock<T>, s, H, cur, prev, out, partial))));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kpm_gen(const DevH& H, int R, bool first, const vec2_t<T>* L, const vec2_t<T>* cur,
                           const vec2_t<T>* prev, vec2_t<T>* out, double* partial, int grid,
                           cudaStream_t s) {
    const bool ons = H.onsite != nullptr;
    if constexpr (kPaired<T>) {
        if (R >= 2) {
            const float4* l4 = reinterpret_cast<const float4*>(L);
            const float4* c4 = reinterpret_cast<const float4*>(cur);
            const float4* p4 = reinterpret_cast<const float4*>(prev);
            float4* o4 = reinterpret_cast<float4*>(out);
            KG_DISPATCH_R(R, if constexpr (RR >= 2) { KG_BOOL(ons, ON, KG_BOOL(first, FI,
                launch_step(FI, kpm_gen_pair_kernel<RR, ON, FI>, grid, kThreads, s, H, l4, c4, p4, o4,
                            partial))) });
            return cudaGetLastError();
        }
    }
    KG_DISPATCH_R(R, KG_BOOL(ons, ON, KG_BOOL(first, FI,
        launch_step(FI, kpm_gen_kernel<T, RR, ON, FI>, grid, kBlock<T>, s, H, L, cur, prev, out, partial))));
    return cudaGetLastError();
}

// One launch of `kernel` as a single cluster of `grid` CTAs of `threads` threads with
// `smem` bytes of dynamic shared memory (above the portable cluster size of 8 the kernel
// is allowed the non-portable size).  query = only check that such a cluster can be
// resident (cudaErrorNotSupported when not).
constexpr int kMaxCluster = 16;
constexpr size_t kClusterSmemBudget = 96 * 1024;   // shared memory per CTA of the cluster path

template <typename... KArgs, typename... Args>
static cudaError_t launch_single_cluster(void (*kernel)(KArgs...), int grid, int threads, size_t smem,
                                         bool query, cudaStream_t s, Args... args) {
    if (grid < 1 || grid > kMaxCluster) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (grid > 8) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)grid;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (query) {
        int clusters = 0;
        e = cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg);
        if (e != cudaSuccess) return e;
        return clusters >= 1 ? cudaSuccess : cudaErrorNotSupported;
    }
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

#define KG_DISPATCH_R16(R_, ...)                                 \
    switch (R_) {                                                \
        case 1: { constexpr int RR = 1; __VA_ARGS__; } break;    \
        case 2: { constexpr int RR = 2; __VA_ARGS__; } break;    \
        case 4: { constexpr int RR = 4; __VA_ARGS__; } break;    \
        case 8: { constexpr int RR = 8; __VA_ARGS__; } break;    \
        case 16: { constexpr int RR = 16; __VA_ARGS__; } break;  \
        default: return cudaErrorNotSupported;                   \
    }

template <typename T>
static cudaError_t kpm_cluster_dispatch(const DevH& H, int R, bool sym, const ClusterPlan& p, bool query,
                                        const vec2_t<T>* L, const vec2_t<T>* src_cur, const vec2_t<T>* src_prev,
                                        vec2_t<T>* dst_cur, vec2_t<T>* dst_prev, double* ring, int nsteps,
                                        bool first, cudaStream_t s) {
    const bool ons = H.onsite != nullptr;
    cudaError_t e = cudaErrorNotSupported;
    KG_DISPATCH_R16(R, KG_BOOL(ons, ON, KG_BOOL(sym, SY,
        e = launch_single_cluster(kpm_cluster_kernel<T, RR, ON, SY>, p.grid, 1 << p.log_nt, p.smem, query, s, H,
                                  L, src_cur, src_prev, dst_cur, dst_prev, ring, nsteps, p.log_nt,
                                  first ? 1 : 0))));
    return e;
}

template <typename T>
bool kpm_cluster_plan(const DevH& H, int R, bool sym, ClusterPlan* plan) {
    if (R < 1 || R > kClusterMaxR || (R & (R - 1))) return false;
    int dev = 0;
    cudaGetDevice(&dev);
    struct Key {
        int dev, tsize, R, sym, ons;
        int64_t n;
        bool operator==(const Key& o) const {
            return dev == o.dev && tsize == o.tsize && R == o.R && sym == o.sym && ons == o.ons && n == o.n;
        }
    };
    struct KeyHash {
        size_t operator()(const Key& k) const {
            return std::hash<int64_t>()(k.n) ^ ((size_t)k.dev << 48) ^ ((size_t)k.tsize << 40) ^
                   ((size_t)k.R << 32) ^ ((size_t)k.sym << 31) ^ ((size_t)k.ons << 30);
        }
    };
    static thread_local std::unordered_map<Key, ClusterPlan, KeyHash> cache;
    const Key key{dev, (int)sizeof(T), R, sym ? 1 : 0, H.onsite ? 1 : 0, H.n};
    auto it = cache.find(key);
    if (it == cache.end()) {
        ClusterPlan best;   // grid 0: not available
        const int64_t items = H.n * R;
        // the smallest CTAs that keep the cluster within 16 CTAs: the FP64 work spreads over the most SMs
        for (int log_nt = 7; log_nt <= 9 && best.grid == 0; log_nt++) {
            const int64_t nt = (int64_t)1 << log_nt;
            const int64_t grid = (items + nt - 1) / nt;
            if (grid < 1 || grid > kMaxCluster) continue;
            const size_t vec = 2 * (size_t)(nt + 1) * sizeof(vec2_t<T>);
            const size_t per_step = (size_t)(nt / 32) * R * sizeof(float4);
            if (vec + per_step > kClusterSmemBudget) continue;
            ClusterPlan p;
            p.log_nt = log_nt;
            p.grid = (int)grid;
            p.chunk = (int)std::min<size_t>(kClusterMaxChunk, (kClusterSmemBudget - vec) / per_step);
            p.smem = vec + (size_t)p.chunk * per_step;
            const cudaError_t e = kpm_cluster_dispatch<T>(H, R, sym, p, true, nullptr, nullptr, nullptr, nullptr,
                                                          nullptr, nullptr, 0, false, nullptr);
            if (e != cudaSuccess) cudaGetLastError();   // a refused query must not leak into later launch checks
            else best = p;
        }
        it = cache.emplace(key, best).first;
    }
    *plan = it->second;
    return plan->grid > 0;
}

template <typename T>
cudaError_t launch_kpm_cluster(const DevH& H, int R, bool sym, const ClusterPlan& p, const vec2_t<T>* L,
                               const vec2_t<T>* src_cur, const vec2_t<T>* src_prev, vec2_t<T>* dst_cur,
                               vec2_t<T>* dst_prev, double* ring, int nsteps, bool first, cudaStream_t s) {
    if (nsteps <= 0) return cudaSuccess;
    // the general recursion's first chunk keeps <L|phi_0> as one more step's partial sums
    if (nsteps + ((first && !sym) ? 1 : 0) > p.chunk || p.grid < 1) return cudaErrorInvalidValue;
    return kpm_cluster_dispatch<T>(H, R, sym, p, false, L, src_cur, src_prev, dst_cur, dst_prev, ring, nsteps,
                                   first, s);
}

template <typename T>
static cudaError_t evolve_cluster_dispatch(const DevH& H, int R, int nch, bool xc, const ClusterPlan& p,
                                           bool query, const SeriesCoef& cf, const ChainsT<T>& ch,
                                           cudaStream_t s) {
    const bool ons = H.onsite != nullptr, ypar = H.ytransport;
    cudaError_t e = cudaErrorNotSupported;
    const int nt = 1 << p.log_nt;
    KG_DISPATCH_R16(R, KG_BOOL(ons, ON, KG_BOOL(ypar, YP,
        if (nch == 1 && !xc) e = launch_single_cluster(evolve_cluster_kernel<T, RR, 1, false, ON, YP>, p.grid, nt,
                                                       p.smem, query, s, H, ch, cf, p.log_nt);
        else if (nch == 1) e = launch_single_cluster(evolve_cluster_kernel<T, RR, 1, true, ON, YP>, p.grid, nt,
                                                     p.smem, query, s, H, ch, cf, p.log_nt);
        else if (!xc) e = launch_single_cluster(evolve_cluster_kernel<T, RR, 2, false, ON, YP>, p.grid, nt,
                                                p.smem, query, s, H, ch, cf, p.log_nt);
        else e = launch_single_cluster(evolve_cluster_kernel<T, RR, 2, true, ON, YP>, p.grid, nt, p.smem,
                                       query, s, H, ch, cf, p.log_nt))));
    return e;
}

template <typename T>
bool evolve_cluster_plan(const DevH& H, int R, int nch, bool xc, ClusterPlan* plan) {
    if (R < 1 || R > kClusterMaxR || (R & (R - 1)) || nch < 1 || nch > 2) return false;
    int dev = 0;
    cudaGetDevice(&dev);
    struct Key {
        int dev, tsize, R, nch, xc, ons, ypar;
        int64_t n;
        bool operator==(const Key& o) const {
            return dev == o.dev && tsize == o.tsize && R == o.R && nch == o.nch && xc == o.xc && ons == o.ons &&
                   ypar == o.ypar && n == o.n;
        }
    };
    struct KeyHash {
        size_t operator()(const Key& k) const {
            return std::hash<int64_t>()(k.n) ^ ((size_t)k.dev << 48) ^ ((size_t)k.tsize << 40) ^
                   ((size_t)k.R << 32) ^ ((size_t)k.nch << 28) ^ ((size_t)k.xc << 27) ^ ((size_t)k.ons << 26) ^
                   ((size_t)k.ypar << 25);
        }
    };
    static thread_local std::unordered_map<Key, ClusterPlan, KeyHash> cache;
    const Key k{dev, (int)sizeof(T), R, nch, xc ? 1 : 0, H.onsite ? 1 : 0, H.ytransport ? 1 : 0, H.n};
    auto it = cache.find(k);
    if (it == cache.end()) {
        ClusterPlan best;
        const int64_t items = H.n * R;
        const int nb = nch + (xc ? 1 : 0);
        for (int log_nt = 7; log_nt <= 9 && best.grid == 0; log_nt++) {
            const int64_t nt = (int64_t)1 << log_nt;
            const int64_t grid = (items + nt - 1) / nt;
            if (grid < 1 || grid > kMaxCluster) continue;
            const size_t smem = (size_t)nb * 2 * (size_t)(nt + 1) * sizeof(vec2_t<T>) +
                                (size_t)(nt / 32) * R * sizeof(float2) + (size_t)R * sizeof(double);
            if (smem > kClusterSmemBudget) continue;
            ClusterPlan p;
            p.log_nt = log_nt;
            p.grid = (int)grid;
            p.chunk = kClusterMaxTerms;
            p.smem = smem;
            SeriesCoef none;
            const cudaError_t e = evolve_cluster_dispatch<T>(H, R, nch, xc, p, true, none, ChainsT<T>{}, nullptr);
            if (e != cudaSuccess) cudaGetLastError();   // a refused query must not leak into later launch checks
            else best = p;
        }
        it = cache.emplace(k, best).first;
    }
    *plan = it->second;
    return plan->grid > 0;
}

template <typename T>
cudaError_t launch_evolve_cluster(const DevH& H, int R, int nch, bool xc, const ClusterPlan& p,
                                  const SeriesCoef& cf, const ChainsT<T>& ch, cudaStream_t s) {
    if (cf.nterms < 1 || cf.nterms > kClusterMaxTerms || p.grid < 1) return cudaErrorInvalidValue;
    return evolve_cluster_dispatch<T>(H, R, nch, xc, p, false, cf, ch, s);
}

template <typename T>
int kpm_grid(const DevH& H, int R, bool sym) {
    const bool ons = H.onsite != nullptr;
    if constexpr (kPaired<T>) {
        if (R >= 2) {
            const int64_t pairs = H.n * (R / 2);
            int g = stream_grid(pairs);
            auto pick = [&](auto k) { g = one_wave_grid(k, pairs); };
            switch (R) {
#define KG_PAIR_GRID_CASE(RV)                                                                  \
                case RV:                                                                      \
                    if (sym) {                                                                \
                        if (ons) pick(kpm_sym_pair_kernel<RV, true, false>);                  \
                        else pick(kpm_sym_pair_kernel<RV, false, false>);                     \
                    } else {                                                                  \
                        if (ons) pick(kpm_gen_pair_kernel<RV, true, false>);                  \
                        else pick(kpm_gen_pair_kernel<RV, false, false>);                     \
                    }                                                                         \
                    break;
                KG_PAIR_GRID_CASE(2) KG_PAIR_GRID_CASE(4) KG_PAIR_GRID_CASE(8)
                KG_PAIR_GRID_CASE(16) KG_PAIR_GRID_CASE(32) KG_PAIR_GRID_CASE(64)
#undef KG_PAIR_GRID_CASE
                default: break;
            }
            return g;
        }
    }
    const int64_t items = H.n * R;
    int g = stream_grid(items);
    auto pick = [&](auto k) { g = one_wave_grid(k, items, kBlock<T>); };
    switch (R) {
#define KG_KPM_GRID_CASE(RV)                                                                   \
        case RV:                                                                              \
            if (sym) {                                                                        \
                if (ons) pick(kpm_sym_kernel<T, RV, true, false>);                            \
                else pick(kpm_sym_kernel<T, RV, false, false>);                               \
            } else {                                                                          \
                if (ons) pick(kpm_gen_kernel<T, RV, true, false>);                            \
                else pick(kpm_gen_kernel<T, RV, false, false>);                               \
            }                                                                                 \
            break;
        KG_KPM_GRID_CASE(1) KG_KPM_GRID_CASE(2) KG_KPM_GRID_CASE(4) KG_KPM_GRID_CASE(8)
        KG_KPM_GRID_CASE(16) KG_KPM_GRID_CASE(32) KG_KPM_GRID_CASE(64)
#undef KG_KPM_GRID_CASE
        default: break;
    }
    return g;
}

cudaError_t launch_reduce_first(const double* partial, int grid, int R, bool sym, double2* mu,
                                int64_t r_stride, int M, cudaStream_t s) {
    reduce_first_kernel<<<1, kThreads, 0, s>>>(partial, grid, R, sym ? 1 : 0, mu, r_stride, M);
    return cudaGetLastError();
}

cudaError_t launch_reduce_ring(const double* ring, int slab0, int nslab, int ring_size, int grid,
                               int R, bool sym, int n0, double2* mu, int64_t r_stride, int M,
                               cudaStream_t s, bool first) {
    if (nslab <= 0) return cudaSuccess;
    reduce_ring_kernel<<<nslab, kThreads, 0, s>>>(ring, slab0, ring_size, grid, R, sym ? 1 : 0,
                                                  n0, mu, r_stride, M, first ? 1 : 0);
    return cudaGetLastError();
}

template <typename T, int R, int NCH, bool XC>
static void evolve_dispatch(const DevH& H, bool first, double j0, double cr, double ci,
                            const ChainsT<T>& ch, cudaStream_t s) {
    const bool ons = H.onsite != nullptr, ypar = H.ytransport;
    const bool odd = first || cr == 0.0;   // the first step is the m = 1 term
    KG_BOOL(first, FI, KG_BOOL(ons, ON, KG_BOOL(ypar, YP, KG_BOOL(odd, OD,
        if constexpr (!FI || OD) {
            const int g = one_wave_grid(evolve_kernel<T, R, NCH, XC, FI, ON, YP, OD>, H.n * R, kBlock<T>);
            launch_step(FI, evolve_kernel<T, R, NCH, XC, FI, ON, YP, OD>, g, kBlock<T>, s, H, j0, cr, ci, ch);
        }))));
}

template <typename T>
cudaError_t launch_evolve(const DevH& H, int R, int nch, bool xc, bool first, double j0, double cr,
                          double ci, const ChainsT<T>& ch, cudaStream_t s) {
    if (nch < 1 || nch > 2) return cudaErrorInvalidValue;
    KG_DISPATCH_R(R,
        if (nch == 1 && !xc) evolve_dispatch<T, RR, 1, false>(H, first, j0, cr, ci, ch, s);
        else if (nch == 1) evolve_dispatch<T, RR, 1, true>(H, first, j0, cr, ci, ch, s);
        else if (!xc) evolve_dispatch<T, RR, 2, false>(H, first, j0, cr, ci, ch, s);
        else evolve_dispatch<T, RR, 2, true>(H, first, j0, cr, ci, ch, s));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(const DevH& H, int R, int op, double scale, const vec2_t<T>* in,
                         vec2_t<T>* out, cudaStream_t s) {
    const bool ons = H.onsite != nullptr, ypar = H.ytransport;
    const int grid = stream_grid(H.n * R);
    KG_DISPATCH_R(R, KG_BOOL(ons, ON, KG_BOOL(ypar, YP,
        if (op == 0) apply_kernel<T, RR, 0, ON, YP><<<grid, kThreads, 0, s>>>(H, scale, in, out);
        else if (op == 1) apply_kernel<T, RR, 1, ON, YP><<<grid, kThreads, 0, s>>>(H, scale, in, out);
        else apply_kernel<T, RR, 2, ON, YP><<<grid, kThreads, 0, s>>>(H, scale, in, out))));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dot(int64_t n_items, int R, const vec2_t<T>* L, const vec2_t<T>* X, double* partial, int grid,
                       double2* out, int64_t r_stride, cudaStream_t s) {
    KG_DISPATCH_R(R, dot_kernel<T, RR><<<grid, kThreads, 0, s>>>(n_items, L, X, partial));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_dot_kernel<<<1, kThreads, 0, s>>>(partial, grid, R, out, r_stride);
    return cudaGetLastError();
}

__global__ void to_c128_kernel(const float2* __restrict__ in, double2* __restrict__ out, int64_t n_items) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_items; k += stride) {
        const float2 v = in[k];
        out[k] = make_double2((double)v.x, (double)v.y);
    }
}

cudaError_t launch_to_c128(const float2* in, double2* out, int64_t n_items, cudaStream_t s) {
    to_c128_kernel<<<stream_grid(n_items), kThreads, 0, s>>>(in, out, n_items);
    return cudaGetLastError();
}

cudaError_t launch_to_c64(const double2* in, float2* out, int64_t n_items, cudaStream_t s) {
    to_c64_kernel<<<stream_grid(n_items), kThreads, 0, s>>>(in, out, n_items);
    return cudaGetLastError();
}

#define KG_INSTANTIATE(T)                                                                          \
    template cudaError_t launch_kpm_sym<T>(const DevH&, int, bool, const vec2_t<T>*,               \
                                           const vec2_t<T>*, vec2_t<T>*, double*, int, cudaStream_t); \
    template cudaError_t launch_kpm_gen<T>(const DevH&, int, bool, const vec2_t<T>*,               \
                                           const vec2_t<T>*, const vec2_t<T>*, vec2_t<T>*, double*,   \
                                           int, cudaStream_t);                                      \
    template int kpm_grid<T>(const DevH&, int, bool);                                              \
    template bool kpm_cluster_plan<T>(const DevH&, int, bool, ClusterPlan*);                       \
    template cudaError_t launch_kpm_cluster<T>(const DevH&, int, bool, const ClusterPlan&,         \
                                               const vec2_t<T>*, const vec2_t<T>*, const vec2_t<T>*, \
                                               vec2_t<T>*, vec2_t<T>*, double*, int, bool, cudaStream_t); \
    template bool evolve_cluster_plan<T>(const DevH&, int, int, bool, ClusterPlan*);                \
    template cudaError_t launch_evolve_cluster<T>(const DevH&, int, int, bool, const ClusterPlan&,   \
                                                  const SeriesCoef&, const ChainsT<T>&, cudaStream_t); \
    template cudaError_t launch_evolve<T>(const DevH&, int, int, bool, bool, double, double, double, \
                                          const ChainsT<T>&, cudaStream_t);                        \
    template cudaError_t launch_apply<T>(const DevH&, int, int, double, const vec2_t<T>*,           \
                                         vec2_t<T>*, cudaStream_t);                                  \
    template cudaError_t launch_dot<T>(int64_t, int, const vec2_t<T>*, const vec2_t<T>*, double*, int, \
                                       double2*, int64_t, cudaStream_t);

KG_INSTANTIATE(double)
KG_INSTANTIATE(float)

// --------------------------------------------------------------------------------
// Sets *flag when any of the n doubles is NaN or infinite (flag cleared by the caller).
// --------------------------------------------------------------------------------
__global__ void nonfinite_kernel(const double* __restrict__ p, int64_t n, int* __restrict__ flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) bad |= !isfinite(p[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) *flag = 1;
}

// --------------------------------------------------------------------------------
// FP64 FMA throughput probe: eight independent chains a <- a b + c per thread (the DP
// pipe's latency is covered by the chains and the resident warps), one store per
// thread so that nothing is dropped.  b and c arrive as arguments (no constant folding);
// with b < 1 the chains converge to c / (1 - b) and stay normal.
// --------------------------------------------------------------------------------
constexpr int kFmaChains = 8;
constexpr int kFmaIters = 2048;
constexpr int kFmaThreads = 256;
constexpr int kFmaCtasPerSm = 4;

__global__ void __launch_bounds__(kFmaThreads) fp64_fma_probe_kernel(double b, double c, double* __restrict__ out) {
    double a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; k++) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < kFmaIters; i++) {
#pragma unroll
        for (int k = 0; k < kFmaChains; k++) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kFmaChains; k++) s += a[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int fp64_probe_grid() { return sm_count() * kFmaCtasPerSm; }

double fp64_probe_fmas() {
    return (double)fp64_probe_grid() * kFmaThreads * kFmaChains * kFmaIters;
}

cudaError_t launch_fp64_probe(double* out, cudaStream_t s) {
    fp64_fma_probe_kernel<<<fp64_probe_grid(), kFmaThreads, 0, s>>>(0.9999999, 1e-3, out);
    return cudaGetLastError();
}

cudaError_t launch_nonfinite(const double* p, int64_t n, int* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 4);
    nonfinite_kernel<<<grid, 256, 0, s>>>(p, n, flag);
    return cudaGetLastError();
}

}  // namespace kg
