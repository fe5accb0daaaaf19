// Surrogate MLP for sigma(E, t): 3 -> 256 -> 256 -> 256 -> 256 -> 1, GELU (tanh form), BF16 weights
// and activations at the matrix-multiply inputs, FP32 accumulation, FP32 master weights
// and Adam.  The surrogate is not part of the paper; it is trained on sigma(E, t) curves
// the method generates.
//
// Batch inference runs the whole network in one persistent kernel (mlp_fused_kernel,
// below): activations stay in shared memory and TMEM, weights stream from L2.
//
// Training: the three 256 x 256 layers are dense contractions and run on the 5th-generation
// tensor cores: one hand-written tcgen05 GEMM kernel D[128 x 256] = A[128 x K] B[256 x K]^T with
// BF16 operands staged (by all threads, 16-byte vector loads) in shared memory in the
// 128-byte-swizzled K-major layout, the FP32 accumulator in tensor memory (TMEM, 256
// columns), a two-stage pipeline whose stages are released by tcgen05.commit arrivals
// on mbarriers, and fused epilogues read back with tcgen05.ld:
//   forward:        z = D + b, a = GELU(z)  -> z (FP32), a (BF16), a^T (BF16)
//   backward data:  dz = D * GELU'(z_prev)   -> dz (BF16), dz^T (BF16)
//   weight grads:   D (FP32), split over the batch (K) dimension
// Only K-major operands are used: the backward GEMMs read the transposed copies the
// epilogues write.  The 3-wide input layer, the 1-wide output layer, the bias and
// small reductions and Adam run on the CUDA cores.  Every wait is bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kg_internal.h"

namespace kg {
namespace mlp {

constexpr int H = 256;
constexpr int BM = 128, BN = 256, BK = 64;   // BK bf16 = one 128-byte swizzle row
constexpr int kGemmThreads = 128;
constexpr int kStageA = BM * BK * 2;         // 16 KB
constexpr int kStageB = BN * BK * 2;         // 32 KB
constexpr int kStages = 2;
constexpr int kGemmSmem = kStages * (kStageA + kStageB) + 1024 + 64;
constexpr long long kWaitLimit = 1ll << 22;   // try_wait polls before giving up
constexpr int kParams = H * 3 + H + 3 * (H * H + H) + H + 1;   // 198657

// offsets into the flat parameter vector (W1 [H][3], b1, W2, b2, W3, b3, W4, b4, W5, b5)
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + H * 3;
constexpr int64_t kOffW2 = kOffB1 + H;
__host__ __device__ constexpr int64_t layer_w(int l) { return kOffW2 + (int64_t)(l - 2) * (H * H + H); }   // l = 2..4
__host__ __device__ constexpr int64_t layer_b(int l) { return layer_w(l) + H * H; }
constexpr int64_t kOffW5 = layer_w(5), kOffB5 = kOffW5 + H;
static_assert(kOffB5 + 1 == kParams, "parameter layout");

enum Epi { EPI_F32 = 0, EPI_FWD = 1, EPI_FWD_INFER = 2, EPI_BWD = 3 };

struct GemmArgs {
    const __nv_bfloat16* A;   // [rows][lda], K-major
    int64_t lda, a_rows;      // rows >= a_rows read as zero
    const __nv_bfloat16* B;   // [256][ldb], K-major
    int64_t ldb;
    int k_atoms;              // 64-wide K blocks per CTA (blockIdx.y selects the block range)
    const float* bias;        // [256] (forward)
    float* d_f32;             // EPI_F32: partial [split][rows][256]; EPI_FWD: z [rows][256]
    int64_t split_stride;
    __nv_bfloat16* out;       // [rows][256]
    __nv_bfloat16* out_t;     // [256][ldot] (transposed), may be null
    int64_t ldot;
    const float* zprev;       // EPI_BWD: [rows][256]
    int64_t m_valid;          // EPI_BWD: rows >= m_valid get dz = 0
    int* error;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// GELU in its tanh form (Hendrycks and Gimpel, 2016):
//   GELU(z) = z/2 (1 + tanh(u)),  u = sqrt(2/pi) (z + 0.044715 z^3),
//   GELU'(z) = (1 + tanh u)/2 + z/2 (1 - tanh^2 u) sqrt(2/pi) (1 + 3 * 0.044715 z^2),
// with the hardware tanh.approx.f32 (about 2^-11 relative error, far below the BF16
// rounding of the activations).  One SFU instruction replaces the erf evaluation that
// made the GEMM epilogues issue-bound.
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kGeluK = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluC = 0.044715f;

__device__ __forceinline__ float gelu(float z) {
    const float u = z * fmaf(kGeluK * kGeluC, z * z, kGeluK);   // sqrt(2/pi) (z + 0.044715 z^3)
    const float hz = 0.5f * z;
    return fmaf(hz, tanh_hw(u), hz);
}

// Packed FP32 instructions of sm_100 and later (mul/fma .f32x2: one instruction, two IEEE
// round-to-nearest results), for two values at about half the issue slots.
__device__ __forceinline__ uint64_t f2_pack(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// 2 GELU(z) = z + z tanh(u) for two values (low half = z0), u as in gelu(): one FMA fewer
// than 0.5 z + 0.5 z tanh(u).  The fused inference kernel stores 2 GELU(z) and streams the
// following layer's weights halved (W/2, an exact power-of-two scaling in BF16), so every
// product (W/2)(2a) = W a and every FP32 sum of the next layer are bitwise those of W and
// GELU(z) (RN(2x) = 2 RN(x) for normal x).
__device__ __forceinline__ uint64_t gelu2_twice(uint64_t z) {
    const uint64_t kc = f2_pack(kGeluK * kGeluC, kGeluK * kGeluC), k = f2_pack(kGeluK, kGeluK);
    const uint64_t u = f2_mul(z, f2_fma(kc, f2_mul(z, z), k));
    const float2 uu = f2_unpack(u);
    return f2_fma(z, f2_pack(tanh_hw(uu.x), tanh_hw(uu.y)), z);
}
__device__ __forceinline__ uint32_t gelu2_twice_bf16(float z0, float z1) {
    const float2 g = f2_unpack(gelu2_twice(f2_pack(z0, z1)));
    const __nv_bfloat162 b2 = __floats2bfloat162_rn(g.x, g.y);
    return *(const uint32_t*)&b2;
}

__device__ __forceinline__ float gelu_grad(float z) {
    const float z2 = z * z;
    const float t = tanh_hw(kGeluK * fmaf(kGeluC * z, z2, z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * kGeluK * fmaf(3.0f * kGeluC, z2, 1.0f);
}

// SM100 shared-memory matrix descriptor: start >> 4 [0,14), leading byte offset >> 4
// [16,30) (unused for swizzled K-major), stride byte offset >> 4 [32,46) = 1024 B between
// 8-row groups, version 1 [46,48), layout 2 = 128-byte swizzle [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12
// = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; i++) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

// The dynamic shared memory limit is a per-device function attribute: set it once per
// (kernel, device), the devices done kept as bits of `done`.
template <typename K>
static kg_status set_smem_once(K kernel, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    KG_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load() & bit)) {
        KG_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
        done.fetch_or(bit);
    }
    return KG_OK;
}

#define KG_TMEM_LD32(taddr, v)                                                                       \
    asm volatile(                                                                                    \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14," \
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"              \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),        \
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),   \
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), \
          "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), \
          "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                                         \
        : "r"(taddr))

#define KG_TMEM_LD16(taddr, v)                                                                       \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"  \
                 "%14,%15}, [%16];"                                                                    \
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),  \
                   "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), \
                   "=r"(v[14]), "=r"(v[15])                                                            \
                 : "r"(taddr))

// Waits for this thread's TMEM loads; the registers of v are in-out operands, so no use of
// them can be scheduled before the wait.
#define KG_TMEM_WAIT16(v)                                                                            \
    asm volatile("tcgen05.wait::ld.sync.aligned;"                                                    \
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),  \
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), \
                   "+r"(v[14]), "+r"(v[15])                                                            \
                 :                                                                                     \
                 : "memory")

#define KG_TMEM_ST16(taddr, v)                                                                       \
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"  \
                 "%14,%15,%16};" ::"r"(taddr),                                                          \
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),  \
                 "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]) \
                 : "memory")

template <int EPI>
__global__ void __launch_bounds__(kGemmThreads, 1) umma_gemm_kernel(GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;   // swizzle atoms need 1024-byte alignment
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t bars = base + kStages * (kStageA + kStageB);
    uint32_t* tmem_slot = (uint32_t*)(base_ptr + kStages * (kStageA + kStageB) + 16);
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * BM;
    const int atom0 = blockIdx.y * g.k_atoms;
    const int na = g.k_atoms;

    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < kStages; s++) mbar_init(bars + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    for (int a = 0; a < na; a++) {
        const int s = a & 1;
        if (a >= 2) {
            // the MMAs that read this stage two blocks ago must be done
            if (!mbar_wait(bars + 8 * s, ((a - 2) >> 1) & 1)) {
                atomicExch(g.error, 1);
                s_fail = 1;
            }
            __syncthreads();
            if (s_fail) break;
        }
        const uint32_t sA = base + s * (kStageA + kStageB), sB = sA + kStageA;
        const int64_t kcol = (int64_t)(atom0 + a) * BK;
#pragma unroll
        for (int i = 0; i < (BM * 8) / kGemmThreads; i++) {
            const int q = tid + i * kGemmThreads, r = q >> 3, c = q & 7;
            const int64_t row = m0 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (row < g.a_rows) v = __ldg((const uint4*)(g.A + row * g.lda + kcol + c * 8));
            st_shared_v4(sA + r * 128 + ((c ^ (r & 7)) << 4), v);
        }
#pragma unroll
        for (int i = 0; i < (BN * 8) / kGemmThreads; i++) {
            const int q = tid + i * kGemmThreads, r = q >> 3, c = q & 7;
            const uint4 v = __ldg((const uint4*)(g.B + (int64_t)r * g.ldb + kcol + c * 8));
            st_shared_v4(sB + r * 128 + ((c ^ (r & 7)) << 4), v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < BK / 16; ks++) {
                const uint64_t ad = sw128_desc(sA + ks * 32), bd = sw128_desc(sB + ks * 32);
                const uint32_t acc = (a > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bars + 8 * s)
                         : "memory");
        }
        issued = a + 1;
    }
    // the last commit covers every MMA issued before it
    if (issued > 0) {
        if (!mbar_wait(bars + 8 * ((issued - 1) & 1), ((issued - 1) >> 1) & 1)) {
            atomicExch(g.error, 1);
            s_fail = 1;
        }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!s_fail) {
        const int rl = warp * 32 + lane;
        const int64_t row = m0 + rl;
#pragma unroll 1
        for (int cb = 0; cb < BN / 32; cb++) {
            uint32_t v[32];
            KG_TMEM_LD32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cb * 32), v);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; j++) {
                const int col = cb * 32 + j;
                const float acc = __uint_as_float(v[j]);
                if constexpr (EPI == EPI_F32) {
                    if (row < g.a_rows) g.d_f32[(int64_t)blockIdx.y * g.split_stride + row * BN + col] = acc;
                } else if constexpr (EPI == EPI_FWD || EPI == EPI_FWD_INFER) {
                    const float z = acc + g.bias[col];
                    const __nv_bfloat16 a = __float2bfloat16_rn(gelu(z));
                    if constexpr (EPI == EPI_FWD) g.d_f32[row * BN + col] = z;
                    g.out[row * BN + col] = a;
                    if (g.out_t) g.out_t[(int64_t)col * g.ldot + row] = a;
                } else {
                    const float dz = row < g.m_valid ? acc * gelu_grad(g.zprev[row * BN + col]) : 0.0f;
                    const __nv_bfloat16 b = __float2bfloat16_rn(dz);
                    g.out[row * BN + col] = b;
                    g.out_t[(int64_t)col * g.ldot + row] = b;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// ------------------------------------------------------------------- inference layout
//
// The weights of layers 2-4 are kept for inference in a core-matrix-tiled layout,
// [32 k-chunks][256 rows][8 values] per layer: a 64-wide K block is one contiguous 32 KB
// run that a single cp.async.bulk copies into the canonical K-major no-swizzle
// shared-memory layout (core matrix = 8 rows x 16 B; LBO = distance between core matrices
// along K, SBO = between 8-row groups).  Activation tiles in shared memory use the same
// layout with 128 rows, [32 k-chunks][128 rows][8], so that every store of 8 values of a
// row is one 16-byte word and a warp's 32 rows are conflict-free.

constexpr int kFCW = 16;                          // compute warps of the fused kernel
constexpr int kFGroups = kFCW / 4;                // column groups: 4 warps cover the 128 TMEM lanes
constexpr int kFCols = BN / kFGroups;             // accumulator columns per compute warp
constexpr int kPThreads = (kFCW + 2) * 32;        // + one load warp + one MMA / TMEM warp
static_assert(kFCols % 32 == 0 && 32 % kFCW == 0, "compute warp split");
static_assert(kFGroups * 4 <= 16, "output partial sums fit one k-chunk of a tile");

// No-swizzle K-major descriptor (layout type 0) with the given LBO / SBO in bytes.
__device__ __forceinline__ uint64_t ns_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool pwait(uint32_t bar, uint32_t parity, volatile int* abort) {
    for (long long i = 0; i < kWaitLimit; i++) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// ------------------------------------------------------------------- fused inference
//
// The whole network for batch inference in one persistent kernel, so activations never
// leave the SM.  A CTA takes 128-row tiles in pairs (X, Y).  Shared memory holds the two
// tiles' BF16 activations (2 x 64 KB, the canonical K-major no-swizzle layout of the
// tiled format) and a ring of three 32 KB weight blocks (64 K values of one 256 x 256
// layer); TMEM holds one 128 x 256 FP32 accumulator per tile (all 512 columns).  Every
// layer runs on the tensor cores:
//   layer 1   one K = 16 MMA: the tile's rows [xh, xt, xh, xt, 1, 1, 1, 0] (x = xh + xt in
//             BF16, written into the tile's first two k-chunks) against the block
//             [Wh, Wh, Wt, Wt, bh, bt, bu, 0] (W1 = Wh + Wt, b1 = bh + bt + bu), i.e.
//             W1 x + b1 to about 2^-16 relative, bias included;
//   layers 2-4  16 MMAs over the layer's four K blocks accumulate W a onto the layer's
//             bias, which the previous epilogue stored into the accumulator (FP32, exact).
//   warps 0-15  write the layer-1 rows (column groups 0 and 1, inputs loaded a pair ahead)
//               and run every epilogue: GELU from TMEM back into the tile buffer as the next
//               layer's operand, and the next layer's bias into each accumulator chunk once
//               it is read (tcgen05.st); after layer 4 the fused 256 -> 1 output.  Warp w reads TMEM
//               lanes 32 (w % 4) .. + 31 (the rule for tcgen05.ld) and 64 columns; four warps
//               per scheduler hide the TMEM, SFU and shared latencies;
//   warp 16     streams the blocks with cp.async.bulk (from L2 after the first tiles), in the
//               order the MMAs use them: per pair the layer-1 block (read by both tiles), then
//               per layer X's four weight blocks, then Y's (a ring entry costs a fixed
//               round trip, so few large blocks are faster than many small ones);
//   warp 17     issues the tcgen05 MMAs and owns the TMEM.
// Per pair the order is M1(X) M1(Y) | M2(X) M2(Y) M3(X) M3(Y) M4(X) M4(Y); the epilogue of
// one tile overlaps the other tile's MMAs, and a tile's next layer-1 rows are written right
// after its layer-4 epilogue.  Every wait is bounded.
constexpr int kFKB = 64;                                 // K values per weight block
constexpr int kFBlocks = H / kFKB;                       // weight blocks per layer
constexpr int kFSlots = 3;                               // ring slots
constexpr int kFWAtom = BN * kFKB * 2;                   // 32 KB: 8 k-chunks x 256 rows x 16 B
constexpr int kFBars = (16 * kFSlots + 32 + 127) / 128 * 128;   // w_full, w_empty, a_ready, acc_full
constexpr int kFXAtom = BN * 16 * 2;                     // 8 KB: a K = 16 block, 2 k-chunks x 256 rows x 16 B
constexpr int kFTile = BM * H * 2;                       // 64 KB
// tiles, ring, barriers, TMEM address (padded to 128 B), alignment slack
constexpr int kFSmem = 2 * kFTile + kFSlots * kFWAtom + kFBars + 128 + 128;
static_assert(kFSmem <= 232448, "fused kernel shared memory");
static_assert(kFXAtom <= kFWAtom && kFKB % 16 == 0, "ring slot size");

struct FArgs {
    const float* x;                  // [rows][3], rows >= n_valid read as zero
    int64_t n_valid;
    int64_t n_tiles;                 // 128-row tiles (pairs run past an odd count on zeros)
    const float* params;             // flat FP32 parameters (W1, b1, ..., w5, b5)
    const __nv_bfloat16* w_tiled;    // [3][32][256][8] BF16 weights of layers 2..4 (halved)
    const __nv_bfloat16* w_extra;    // [2][256][8] the K = 16 block of layer 1
    float* y;                        // [n_valid]
    int* error;
};

__global__ void __launch_bounds__(kPThreads, 1) mlp_fused_kernel(FArgs p) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 127u) & ~127u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t sA = base;                                   // tile t at sA + t * kFTile
    const uint32_t sW = base + 2 * kFTile;                      // slot k at sW + k * kFWAtom
    const uint32_t bars = base + 2 * kFTile + kFSlots * kFWAtom;
    const uint32_t w_full = bars, w_empty = bars + 8 * kFSlots, a_ready = bars + 16 * kFSlots,
                   acc_full = bars + 16 * kFSlots + 16;
    uint32_t* tmem_slot = (uint32_t*)(base_ptr + 2 * kFTile + kFSlots * kFWAtom + kFBars);
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_pairs = (p.n_tiles + 1) / 2;

    if (tid == 0) {
        s_abort = 0;
        for (int k = 0; k < kFSlots; k++) {
            mbar_init(w_full + 8 * k, 1);
            mbar_init(w_empty + 8 * k, 1);
        }
        for (int t = 0; t < 2; t++) {
            mbar_init(a_ready + 8 * t, kFCW);
            mbar_init(acc_full + 8 * t, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kFCW + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    auto give_up = [&]() {
        atomicExch(p.error, 1);
        s_abort = 1;
    };

    if (warp == kFCW && lane == 0) {
        // blocks in MMA order: per pair the layer-1 block, then per layer and tile the weight
        // K blocks
        int64_t g = 0;
        auto fill = [&](const void* src, uint32_t bytes) -> bool {
            const int slot = (int)(g % kFSlots);
            const int64_t use = g / kFSlots;
            if (use > 0 && !pwait(w_empty + 8 * slot, (uint32_t)((use - 1) & 1), &s_abort)) {
                give_up();
                return false;
            }
            expect_tx(w_full + 8 * slot, bytes);
            bulk_g2s(sW + slot * kFWAtom, src, bytes, w_full + 8 * slot);
            g++;
            return true;
        };
        const uint8_t* extra = (const uint8_t*)p.w_extra;
        bool ok = true;
        for (int64_t pr = blockIdx.x; pr < n_pairs && ok && !s_abort; pr += gridDim.x) {
            ok = fill(extra, kFXAtom);
            for (int l = 0; l < 3 && ok; l++)
                for (int t = 0; t < 2 && ok; t++) {
                    for (int k = 0; k < kFBlocks && ok; k++)
                        ok = fill((const uint8_t*)p.w_tiled + ((size_t)l * kFBlocks + k) * kFWAtom, kFWAtom);
                }
        }
        // no copy may still be landing when the CTA exits (bounded, ignores the abort flag)
        volatile int never = 0;
        for (int64_t q = (g > kFSlots ? g - kFSlots : 0); q < g; q++)
            if (!pwait(w_full + 8 * (int)(q % kFSlots), (uint32_t)((q / kFSlots) & 1), &never)) atomicExch(p.error, 1);
    } else if (warp == kFCW + 1 && lane == 0) {
        int64_t g = 0, job[2] = {0, 0};
        uint32_t last_bar = 0, last_parity = 0;
        auto mma = [&](int t, uint64_t ad, uint64_t bd, uint32_t accum) {
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + t * BN),
                "l"(ad), "l"(bd), "r"(kIdesc), "r"(accum)
                : "memory");
        };
        auto commit = [&](uint32_t bar, uint32_t parity) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                         : "memory");
            last_bar = bar;
            last_parity = parity;
        };
        // the block of ring use g has landed
        auto block_ready = [&]() -> bool {
            if (!pwait(w_full + 8 * (int)(g % kFSlots), (uint32_t)((g / kFSlots) & 1), &s_abort)) {
                give_up();
                return false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            return true;
        };
        // the tile's operand for its next layer is written and its accumulator drained
        auto operand_ready = [&](int t) -> bool {
            if (!pwait(a_ready + 8 * t, (uint32_t)(job[t] & 1), &s_abort)) {
                give_up();
                return false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            return true;
        };
        // K = 16 descriptors: A = two k-chunks of a tile (LBO = 128 rows x 16 B), B = two k-chunks
        // of the 256-row block in a ring slot (LBO = 256 rows x 16 B)
        bool ok = true;
        for (int64_t pr = blockIdx.x; pr < n_pairs && ok && !s_abort; pr += gridDim.x) {
            // layer 1: both tiles read the one layer-1 block
            ok = block_ready();
            const uint32_t slot1 = sW + (uint32_t)(g % kFSlots) * kFWAtom;
            for (int t = 0; t < 2 && ok; t++) {
                ok = operand_ready(t);
                if (!ok) break;
                mma(t, ns_desc(sA + t * kFTile, BM * 16, 128), ns_desc(slot1, BN * 16, 128), 0u);
                commit(acc_full + 8 * t, (uint32_t)(job[t] & 1));
                job[t]++;
            }
            if (!ok) break;
            commit(w_empty + 8 * (int)(g % kFSlots), (uint32_t)((g / kFSlots) & 1));
            g++;
            for (int l = 0; l < 3 && ok; l++)
                for (int t = 0; t < 2 && ok; t++) {
                    // (the accumulator holds the layer's bias, stored by the epilogue)
                    ok = operand_ready(t);
                    for (int k = 0; k < kFBlocks && ok; k++) {
                        ok = block_ready();
                        if (!ok) break;
                        const uint32_t slot = sW + (uint32_t)(g % kFSlots) * kFWAtom;
#pragma unroll
                        for (int st = 0; st < kFKB / 16; st++)
                            // A: k-chunks (kFKB / 8) k + 2st, +1 of the tile; B: k-chunks 2st, +1 of the block
                            mma(t, ns_desc(sA + t * kFTile + (k * (kFKB / 8) + 2 * st) * BM * 16, BM * 16, 128),
                                ns_desc(slot + 2 * st * BN * 16, BN * 16, 128), 1u);
                        commit(w_empty + 8 * (int)(g % kFSlots), (uint32_t)((g / kFSlots) & 1));
                        g++;
                    }
                    if (!ok) break;
                    commit(acc_full + 8 * t, (uint32_t)(job[t] & 1));
                    job[t]++;
                }
        }
        // every MMA issued must be complete before the TMEM is freed (bounded)
        volatile int never = 0;
        if (last_bar && !pwait(last_bar, last_parity, &never)) atomicExch(p.error, 1);
    } else if (warp < kFCW) {
        // warp w: TMEM lanes (tile rows) 32 (w % 4) .. + 31, accumulator columns of group w / 4
        const int quarter = warp & 3, grp = warp >> 2;
        const int rl = quarter * 32 + lane;
        const float* w5 = p.params + kOffW5;
        const float b5 = __ldg(p.params + kOffB5);
        int64_t job[2] = {0, 0};
        // all compute warps have written the tile's operand: publish
        // (and its reads of the tile's accumulator are complete: the next MMA overwrites it)
        auto publish = [&](int t) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(a_ready + 8 * t);
        };
        // the inputs of row rl of both tiles of a pair (column groups 0 and 1 write the layer-1
        // rows); the next pair's are loaded while this pair runs
        float xin[2][3];
        auto load_x = [&](int64_t pr) {
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const int64_t grow = (2 * pr + t) * BM + rl;
                const bool in = grp < 2 && pr < n_pairs && grow < p.n_valid;
#pragma unroll
                for (int i = 0; i < 3; i++) xin[t][i] = in ? __ldg(p.x + grow * 3 + i) : 0.0f;
            }
        };
        // layer-1 rows of tile t from xin[t]: k-chunk 0 = [xh0 xh1 xh2 xt0 xt1 xt2 xh0 xh1],
        // k-chunk 1 = [xh2 xt0 xt1 xt2 1 1 1 0]   (x = xh + xt in BF16)
        auto write_layer1 = [&](int t) {
                if (grp < 2) {
                    __nv_bfloat16 xh[3], xt[3];
#pragma unroll
                    for (int i = 0; i < 3; i++) {
                        xh[i] = __float2bfloat16_rn(xin[t][i]);
                        xt[i] = __float2bfloat16_rn(xin[t][i] - __bfloat162float(xh[i]));
                    }
                    auto pk = [](__nv_bfloat16 lo, __nv_bfloat16 hi) {
                        return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
                    };
                    const uint32_t one2 = 0x3F803F80u, one_zero = 0x00003F80u;
                    const uint4 row = grp == 0 ? make_uint4(pk(xh[0], xh[1]), pk(xh[2], xt[0]), pk(xt[1], xt[2]), pk(xh[0], xh[1]))
                                               : make_uint4(pk(xh[2], xt[0]), pk(xt[1], xt[2]), one2, one_zero);
                    st_shared_v4(sA + t * kFTile + (uint32_t)((grp * BM + rl) * 16), row);
                }
                publish(t);
        };
        // a tile's next layer-1 rows are written as soon as its layer-4 epilogue is done, so the
        // next pair's first MMA runs while the other tile's layer-4 epilogue does
        load_x(blockIdx.x);
        write_layer1(0);
        write_layer1(1);
        load_x(blockIdx.x + gridDim.x);
        for (int64_t pr = blockIdx.x; pr < n_pairs; pr += gridDim.x) {
            // epilogues of layers 1-4.  After an abort every wait returns at once, but all compute
            // warps still run every iteration, so each reaches every named barrier below.
            for (int l = 0; l < 4; l++)
                for (int t = 0; t < 2; t++) {
                    const bool ok = pwait(acc_full + 8 * t, (uint32_t)(job[t] & 1), &s_abort);
                    job[t]++;
                    if (!ok) {
                        give_up();
                        if (l == 3) asm volatile("bar.sync 1, %0;" ::"n"(kFCW * 32) : "memory");
                        continue;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // 16-column chunks; the next chunk's TMEM load is in flight while this one's
                    // GELU runs.  The epilogue stores 2 GELU(z) (layers 2-4 stream W/2) and puts
                    // the next layer's bias into the accumulator columns it has read, so that the
                    // next layer's MMAs accumulate onto it; the output layer sums w5 . 2 GELU(z4)
                    // in four partial sums and halves the total.
                    const float4* bias4 = (const float4*)(p.params + layer_b(l < 3 ? l + 2 : 4));
                    float ys[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    const uint32_t trow = tmem + t * BN + ((uint32_t)(quarter * 32) << 16);
                    constexpr int kChunk16 = kFCols / 16;
                    uint32_t va[16], vb[16];
                    KG_TMEM_LD16(trow + (uint32_t)(grp * kFCols), va);
                    KG_TMEM_WAIT16(va);
#pragma unroll
                    for (int cb = 0; cb < kChunk16; cb++) {
                        const int col0 = grp * kFCols + cb * 16;
                        uint32_t* v = (cb & 1) ? vb : va;
                        uint32_t* vn = (cb & 1) ? va : vb;
                        if (cb + 1 < kChunk16) KG_TMEM_LD16(trow + (uint32_t)(col0 + 16), vn);
                        if (l == 3) {
                            const float4* w54 = (const float4*)(w5 + col0);
#pragma unroll
                            for (int q = 0; q < 4; q++) {
                                const float4 f = __ldg(w54 + q);
                                const float2 g0 = f2_unpack(gelu2_twice(f2_pack(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]))));
                                const float2 g1 =
                                    f2_unpack(gelu2_twice(f2_pack(__uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]))));
                                ys[0] = fmaf(g0.x, f.x, ys[0]);
                                ys[1] = fmaf(g0.y, f.y, ys[1]);
                                ys[2] = fmaf(g1.x, f.z, ys[2]);
                                ys[3] = fmaf(g1.y, f.w, ys[3]);
                            }
                        } else {
                            // next layer's bias (warp-uniform loads, in flight during the GELUs)
                            float4 bq[4];
#pragma unroll
                            for (int q = 0; q < 4; q++) bq[q] = __ldg(bias4 + col0 / 4 + q);
#pragma unroll
                            for (int c8 = 0; c8 < 2; c8++) {
                                uint32_t packed[4];
#pragma unroll
                                for (int e = 0; e < 8; e += 2)
                                    packed[e >> 1] = gelu2_twice_bf16(__uint_as_float(v[c8 * 8 + e]), __uint_as_float(v[c8 * 8 + e + 1]));
                                const int chunk = (col0 >> 3) + c8;
                                st_shared_v4(sA + t * kFTile + (uint32_t)((chunk * BM + rl) * 16),
                                             make_uint4(packed[0], packed[1], packed[2], packed[3]));
                            }
                            uint32_t bv[16];
#pragma unroll
                            for (int q = 0; q < 4; q++) {
                                bv[4 * q] = __float_as_uint(bq[q].x);
                                bv[4 * q + 1] = __float_as_uint(bq[q].y);
                                bv[4 * q + 2] = __float_as_uint(bq[q].z);
                                bv[4 * q + 3] = __float_as_uint(bq[q].w);
                            }
                            KG_TMEM_ST16(trow + (uint32_t)col0, bv);
                        }
                        if (cb + 1 < kChunk16) KG_TMEM_WAIT16(vn);
                    }
                    const float ysum = 0.5f * ((ys[0] + ys[1]) + (ys[2] + ys[3]));
                    if (l < 3) {
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        publish(t);
                    } else {
                        // The column groups' partial sums meet in k-chunk 2 of the tile's operand
                        // buffer, which the completed layer-4 MMAs no longer read.  The next pair's
                        // layer-1 rows (k-chunks 0, 1) do not touch it, and its layer-1 epilogue
                        // writes there only after every warp, group 0 included (having read the
                        // sums), has published those rows.
                        float* ypart = (float*)(base_ptr + t * kFTile + 2 * BM * 16);   // [kFGroups][128]
                        ypart[grp * BM + rl] = ysum;
                        asm volatile("bar.sync 1, %0;" ::"n"(kFCW * 32) : "memory");
                        const int64_t grow = (2 * pr + t) * BM + rl;
                        if (grp == 0 && grow < p.n_valid) {
                            float yv = b5;
#pragma unroll
                            for (int q = 0; q < kFGroups; q++) yv += ypart[q * BM + rl];
                            p.y[grow] = yv;
                        }
                        if (pr + gridDim.x < n_pairs) write_layer1(t);
                    }
                }
            load_x(pr + 2 * (int64_t)gridDim.x);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == kFCW + 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
    }
}

// ------------------------------------------------------------------- CUDA-core kernels

// Layer 1 (K = 3): z = W1 x + b1, a = GELU(z); rows >= n_valid use x = 0.
__global__ void layer1_kernel(const float* __restrict__ x, int64_t n_valid, int64_t rows,
                              const float* __restrict__ p, float* __restrict__ z,
                              __nv_bfloat16* __restrict__ a, __nv_bfloat16* __restrict__ at) {
    const int64_t total = rows * H;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = k / H;
        const int c = (int)(k % H);
        float v = p[kOffB1 + c];
        if (r < n_valid) {
            v = fmaf(p[kOffW1 + c * 3 + 0], x[r * 3 + 0], v);
            v = fmaf(p[kOffW1 + c * 3 + 1], x[r * 3 + 1], v);
            v = fmaf(p[kOffW1 + c * 3 + 2], x[r * 3 + 2], v);
        }
        const __nv_bfloat16 g = __float2bfloat16_rn(gelu(v));
        if (z) z[k] = v;
        a[k] = g;
        if (at) at[(int64_t)c * rows + r] = g;
    }
}

// Output layer: one warp per row.  y = w5 . a + b5.  With targets (training):
// loss partial per block, dy = 2 (y - t) / n_valid, dz4 = dy w5 GELU'(z4) (BF16, both
// layouts), and per-block partials of dW5 (sum_rows dy a) and db5.
__global__ void out_kernel(const __nv_bfloat16* __restrict__ a4, const float* __restrict__ z4,
                           int64_t n_valid, int64_t rows, const float* __restrict__ p,
                           const float* __restrict__ t, float* __restrict__ y,
                           __nv_bfloat16* __restrict__ dz, __nv_bfloat16* __restrict__ dzt,
                           float* __restrict__ part /* [grid][H + 2] */) {
    __shared__ float s_w[H];
    __shared__ float s_dw[8][H];
    __shared__ float s_aux[8][2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = threadIdx.x; c < H; c += blockDim.x) s_w[c] = p[kOffW5 + c];
    for (int c = lane; c < H; c += 32) s_dw[warp][c] = 0.0f;
    float loss = 0.0f, db = 0.0f;
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * nw + warp; r < rows; r += (int64_t)gridDim.x * nw) {
        float acc = 0.0f;
        for (int c = lane; c < H; c += 32) acc = fmaf(__bfloat162float(a4[r * H + c]), s_w[c], acc);
        for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        const float yr = acc + p[kOffB5];
        if (lane == 0 && r < n_valid) y[r] = yr;
        if (t) {
            const float diff = r < n_valid ? yr - t[r] : 0.0f;
            const float dy = 2.0f * diff / (float)n_valid;
            if (lane == 0) {
                loss += diff * diff;
                db += dy;
            }
            for (int c = lane; c < H; c += 32) {
                const float d = dy * s_w[c] * gelu_grad(z4[r * H + c]);
                const __nv_bfloat16 b = __float2bfloat16_rn(d);
                dz[r * H + c] = b;
                dzt[(int64_t)c * rows + r] = b;
                s_dw[warp][c] += dy * __bfloat162float(a4[r * H + c]);
            }
        }
    }
    if (!t) return;
    if (lane == 0) {
        s_aux[warp][0] = loss;
        s_aux[warp][1] = db;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < H; c += blockDim.x) {
        float s = 0.0f;
        for (int w = 0; w < nw; w++) s += s_dw[w][c];
        part[(int64_t)blockIdx.x * (H + 2) + c] = s;
    }
    if (threadIdx.x == 0) {
        float l = 0.0f, d = 0.0f;
        for (int w = 0; w < nw; w++) {
            l += s_aux[w][0];
            d += s_aux[w][1];
        }
        part[(int64_t)blockIdx.x * (H + 2) + H] = l;
        part[(int64_t)blockIdx.x * (H + 2) + H + 1] = d;
    }
}

// Sums the out_kernel partials [nblk][H + 2] in a fixed order: columns 0..H-1 -> dW5,
// column H -> loss (times loss_scale), column H + 1 -> db5.
__global__ void out_partials_kernel(const float* __restrict__ part, int nblk, float* __restrict__ dw5,
                                    float* __restrict__ db5, double* __restrict__ loss_out, double loss_scale) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < H + 2; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; b++) s += part[(int64_t)b * (H + 2) + c];
        if (c < H) dw5[c] = (float)s;
        else if (c == H) *loss_out = s * loss_scale;
        else *db5 = (float)s;
    }
}

// Row sums of a transposed activation gradient: out[c] = sum_r dzt[c][r] (bias gradient),
// and for layer 1 also out_w[c][k] = sum_r dzt[c][r] x[r][k].  One block per c.
__global__ void grad_rows_kernel(const __nv_bfloat16* __restrict__ dzt, int64_t rows, int64_t n_valid,
                                 const float* __restrict__ x, float* __restrict__ db,
                                 float* __restrict__ dw1) {
    __shared__ float sm[4][256];
    const int c = blockIdx.x;
    float s[4] = {0, 0, 0, 0};
    for (int64_t r = threadIdx.x; r < n_valid; r += blockDim.x) {
        const float d = __bfloat162float(dzt[(int64_t)c * rows + r]);
        s[0] += d;
        if (x) {
            s[1] = fmaf(d, x[r * 3 + 0], s[1]);
            s[2] = fmaf(d, x[r * 3 + 1], s[2]);
            s[3] = fmaf(d, x[r * 3 + 2], s[3]);
        }
    }
    for (int q = 0; q < 4; q++) sm[q][threadIdx.x] = s[q];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int q = 0; q < 4; q++) sm[q][threadIdx.x] += sm[q][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        db[c] = sm[0][0];
        if (dw1) {
            dw1[c * 3 + 0] = sm[1][0];
            dw1[c * 3 + 1] = sm[2][0];
            dw1[c * 3 + 2] = sm[3][0];
        }
    }
}

// dst[i] = sum over splits of src[s][i] (weight gradient of a 256 x 256 layer).
__global__ void splitk_sum_kernel(const float* __restrict__ src, int splits, int64_t stride,
                                  float* __restrict__ dst) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)H * H;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int k = 0; k < splits; k++) s += src[k * stride + i];
        dst[i] = s;
    }
}

// Adam (Kingma and Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr mh / (sqrt(vh) + eps).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// The i-th of three BF16 terms whose sum is v exactly (FP32 has 24 significand bits, BF16 8):
// h = bf16(v), t = bf16(v - h), u = v - h - t (exact in BF16).
__device__ __forceinline__ float bf16_term(float v, int i) {
    const float h = __bfloat162float(__float2bfloat16_rn(v));
    const float r = v - h;
    const float t = __bfloat162float(__float2bfloat16_rn(r));
    return i == 0 ? h : i == 1 ? t : r - t;
}

// BF16 copies of W2..W4 ([out][in]) and their transposes ([in][out]), and the blocks of the
// fused inference kernel.
__global__ void cast_weights_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ w,
                                    __nv_bfloat16* __restrict__ wt, __nv_bfloat16* __restrict__ wtile,
                                    __nv_bfloat16* __restrict__ wextra) {
    // The layer-1 block of the fused kernel, K = 16, [2 k-chunks][256 rows][8], row = output
    // unit o: k 0-2 Wh, 3-5 Wh, 6-8 Wt, 9-11 Wt (W1 = Wh + Wt), 12-14 the three terms of b1,
    // 15 zero -- against the rows [xh, xt, xh, xt, 1, 1, 1, 0].
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < H * 16; k += gridDim.x * blockDim.x) {
        const int o = k / 16, kk = k % 16;
        float v = 0.0f;
        if (kk < 12) {
            const float wv = p[kOffW1 + o * 3 + kk % 3];
            v = kk < 6 ? bf16_term(wv, 0) : wv - bf16_term(wv, 0);
        } else if (kk < 15) {
            v = bf16_term(p[kOffB1 + o], kk - 12);
        }
        wextra[((kk >> 3) * H + o) * 8 + (kk & 7)] = __float2bfloat16_rn(v);
    }
    const int64_t total = 3 * (int64_t)H * H;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(k / (H * H));
        const int rem = (int)(k % (H * H));
        const int o = rem / H, i = rem % H;
        const __nv_bfloat16 b = __float2bfloat16_rn(p[layer_w(l + 2) + rem]);
        w[k] = b;
        wt[(int64_t)l * H * H + (int64_t)i * H + o] = b;
        // tiled: [32 k-chunks][256 rows][8], row = output unit o, k = input i.  Halved (exactly):
        // the fused inference kernel feeds these layers 2 GELU(z) (gelu2_twice)
        wtile[(int64_t)l * H * H + ((int64_t)(i >> 3) * H + o) * 8 + (i & 7)] =
            __float2bfloat16_rn(0.5f * p[layer_w(l + 2) + rem]);
    }
}

}  // namespace mlp
}  // namespace kg

// ------------------------------------------------------------------------- host side

using namespace kg;
using namespace kg::mlp;

struct kg_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;   // FP32 master [kParams]
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* w = nullptr;    // [3][H][H]
    __nv_bfloat16* wt = nullptr;   // [3][H][H]
    __nv_bfloat16* wtile = nullptr;   // [3][32][H][8] (tiled for the persistent kernel)
    __nv_bfloat16* wextra = nullptr;  // [2][H][8] (its layer-1 block)
    int* error = nullptr;
    double* loss = nullptr;
    int* error_host = nullptr;     // pinned copy of *error (one synchronisation per forward)
    int64_t step = 0;
    // batch buffers
    int64_t cap = 0;               // padded rows
    float* x = nullptr;            // [cap][3]
    float* t = nullptr;            // [cap]
    float* y = nullptr;            // [cap]
    float* z[4] = {nullptr, nullptr, nullptr, nullptr};                     // [cap][H]
    __nv_bfloat16* a[4] = {nullptr, nullptr, nullptr, nullptr};             // [cap][H]
    __nv_bfloat16* at[4] = {nullptr, nullptr, nullptr, nullptr};            // [H][cap]
    __nv_bfloat16* dz[2] = {nullptr, nullptr};
    __nv_bfloat16* dzt[2] = {nullptr, nullptr};
    float* part = nullptr;         // out-kernel partials / split-K partials
    size_t part_bytes = 0;
    std::vector<void*> batch_allocs;
    int64_t launches = 0;
    // CUDA-event timing of the tensor-core GEMM launches
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gemm_events;
    double gemm_flop = 0.0;
    int64_t gemm_launches = 0;
};

namespace {

kg_status mlp_free_batch(kg_mlp* m) {
    for (void* p : m->batch_allocs) cudaFree(p);
    m->batch_allocs.clear();
    m->cap = 0;
    return KG_OK;
}

kg_status mlp_alloc(kg_mlp* m, void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(KG_ENOMEM, "mlp: device allocation failed");
    }
    m->batch_allocs.push_back(*p);
    return KG_OK;
}

kg_status mlp_ensure(kg_mlp* m, int64_t rows, bool train) {
    if (rows <= m->cap && (!train || m->z[0])) return KG_OK;
    mlp_free_batch(m);
    for (auto& q : m->z) q = nullptr;
    for (auto& q : m->at) q = nullptr;
    for (auto& q : m->dz) q = nullptr;
    for (auto& q : m->dzt) q = nullptr;
    for (auto& q : m->a) q = nullptr;
    KG_TRY(mlp_alloc(m, (void**)&m->x, rows * 3 * sizeof(float)));
    KG_TRY(mlp_alloc(m, (void**)&m->t, rows * sizeof(float)));
    KG_TRY(mlp_alloc(m, (void**)&m->y, rows * sizeof(float)));
    // the per-layer activations only for training (the fused inference kernel keeps them on chip)
    if (train)
        for (int l = 0; l < 4; l++) KG_TRY(mlp_alloc(m, (void**)&m->a[l], rows * H * sizeof(__nv_bfloat16)));
    if (train) {
        for (int l = 0; l < 4; l++) {
            KG_TRY(mlp_alloc(m, (void**)&m->z[l], rows * H * sizeof(float)));
            KG_TRY(mlp_alloc(m, (void**)&m->at[l], rows * H * sizeof(__nv_bfloat16)));
        }
        for (int k = 0; k < 2; k++) {
            KG_TRY(mlp_alloc(m, (void**)&m->dz[k], rows * H * sizeof(__nv_bfloat16)));
            KG_TRY(mlp_alloc(m, (void**)&m->dzt[k], rows * H * sizeof(__nv_bfloat16)));
        }
    }
    if (train) {
        // out-kernel partials [<= 1024][H + 2] and split-K partials [rows / 64][H][H]
        const size_t pb = std::max<size_t>((size_t)1024 * (H + 2) * sizeof(float),
                                           (size_t)(rows / BK) * H * H * sizeof(float));
        KG_TRY(mlp_alloc(m, (void**)&m->part, pb));
        m->part_bytes = pb;
    } else {
        m->part = nullptr;
        m->part_bytes = 0;
    }
    m->cap = rows;
    return KG_OK;
}

bool is_dev(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <int EPI>
kg_status launch_gemm(kg_mlp* m, const GemmArgs& g, int64_t m_tiles, int splits) {
    static std::atomic<unsigned long long> configured{0};
    KG_TRY(set_smem_once(umma_gemm_kernel<EPI>, kGemmSmem, configured));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (m->timing) {
        KG_CUDA_TRY(cudaEventCreate(&e0));
        KG_CUDA_TRY(cudaEventCreate(&e1));
        KG_CUDA_TRY(cudaEventRecord(e0, m->stream));
    }
    umma_gemm_kernel<EPI><<<dim3((unsigned)m_tiles, (unsigned)splits), kGemmThreads, kGemmSmem, m->stream>>>(g);
    KG_CUDA_TRY(cudaGetLastError());
    if (m->timing) {
        KG_CUDA_TRY(cudaEventRecord(e1, m->stream));
        m->gemm_events.push_back({e0, e1});
        // 2 M N K per CTA tile (M = 128, N = 256, K = 64 per block)
        m->gemm_flop += 2.0 * BM * BN * (double)BK * g.k_atoms * (double)m_tiles * splits;
        m->gemm_launches++;
    }
    m->launches++;
    return KG_OK;
}

// Forward pass over `rows` (multiple of 128) rows, n_valid real samples; train keeps z, a^T.
kg_status mlp_forward(kg_mlp* m, int64_t n_valid, int64_t rows, bool train) {
    const int grid = std::max(1, std::min<int>(sm_count() * 8, (int)((rows * H + 255) / 256)));
    layer1_kernel<<<grid, 256, 0, m->stream>>>(m->x, n_valid, rows, m->params, train ? m->z[0] : nullptr,
                                               m->a[0], train ? m->at[0] : nullptr);
    KG_CUDA_TRY(cudaGetLastError());
    m->launches++;
    for (int l = 2; l <= 4; l++) {
        GemmArgs g{};
        g.A = m->a[l - 2];
        g.lda = H;
        g.a_rows = rows;
        g.B = m->w + (int64_t)(l - 2) * H * H;
        g.ldb = H;
        g.k_atoms = H / BK;
        g.bias = m->params + layer_b(l);
        g.d_f32 = train ? m->z[l - 1] : nullptr;
        g.out = m->a[l - 1];
        g.out_t = (train && l < 4) ? m->at[l - 1] : nullptr;
        g.ldot = rows;
        g.error = m->error;
        if (train) KG_TRY(launch_gemm<EPI_FWD>(m, g, rows / BM, 1));
        else KG_TRY(launch_gemm<EPI_FWD_INFER>(m, g, rows / BM, 1));
    }
    return KG_OK;
}

// Inference: the fused kernel over x [n_valid][3] into y [n_valid] (device pointers; rows
// up to the padded count read as zero).
kg_status mlp_infer(kg_mlp* m, const float* x, float* y, int64_t n_valid, int64_t rows) {
    static std::atomic<unsigned long long> configured{0};
    KG_TRY(set_smem_once(mlp_fused_kernel, kFSmem, configured));
    FArgs fa{};
    fa.x = x;
    fa.n_valid = n_valid;
    fa.n_tiles = rows / BM;
    fa.params = m->params;
    fa.w_tiled = m->wtile;
    fa.w_extra = m->wextra;
    fa.y = y;
    fa.error = m->error;
    const int64_t n_pairs = (fa.n_tiles + 1) / 2;
    const int grid = (int)std::min<int64_t>(n_pairs, sm_count());
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (m->timing) {
        KG_CUDA_TRY(cudaEventCreate(&e0));
        KG_CUDA_TRY(cudaEventCreate(&e1));
        KG_CUDA_TRY(cudaEventRecord(e0, m->stream));
    }
    mlp_fused_kernel<<<grid, kPThreads, kFSmem, m->stream>>>(fa);
    KG_CUDA_TRY(cudaGetLastError());
    if (m->timing) {
        KG_CUDA_TRY(cudaEventRecord(e1, m->stream));
        m->gemm_events.push_back({e0, e1});
        // tensor-core work: the three 256 x 256 layers on every (padded) tile of every pair
        m->gemm_flop += 3.0 * 2.0 * BM * BN * (double)H * (double)(2 * n_pairs);
        m->gemm_launches++;
    }
    m->launches++;
    return KG_OK;
}

kg_status check_mlp_error(kg_mlp* m) {
    int err = 0;
    KG_CUDA_TRY(cudaMemcpyAsync(&err, m->error, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (err) return fail(KG_ETIMEOUT, "mlp: a tensor-core wait gave up");
    return KG_OK;
}

// Loss and the full gradient into m->grad (FP32) for the batch already in m->x, m->t.
kg_status mlp_backward(kg_mlp* m, int64_t n_valid, int64_t rows) {
    const int oblocks = (int)std::min<int64_t>(1024, (rows + 7) / 8);
    out_kernel<<<oblocks, 256, 0, m->stream>>>(m->a[3], m->z[3], n_valid, rows, m->params, m->t, m->y, m->dz[0],
                                               m->dzt[0], m->part);
    KG_CUDA_TRY(cudaGetLastError());
    out_partials_kernel<<<2, 256, 0, m->stream>>>(m->part, oblocks, m->grad + kOffW5, m->grad + kOffB5, m->loss,
                                                  1.0 / (double)n_valid);
    KG_CUDA_TRY(cudaGetLastError());
    m->launches += 2;
    int cur = 0;
    for (int l = 4; l >= 2; l--) {
        // weight gradient dW_l = dz_l^T a_{l-1}, split over the batch (K) dimension
        const int atoms = (int)(rows / BK);
        int per = 1;
        for (int d : {8, 4, 2})
            if (atoms % d == 0) {
                per = d;
                break;
            }
        const int splits = atoms / per;
        if ((size_t)splits * H * H * sizeof(float) > m->part_bytes) return fail(KG_EINVAL, "mlp: internal split buffer");
        GemmArgs gw{};
        gw.A = m->dzt[cur];
        gw.lda = rows;
        gw.a_rows = H;
        gw.B = m->at[l - 2];
        gw.ldb = rows;
        gw.k_atoms = per;
        gw.d_f32 = m->part;
        gw.split_stride = (int64_t)H * H;
        gw.error = m->error;
        KG_TRY(launch_gemm<EPI_F32>(m, gw, H / BM, splits));
        splitk_sum_kernel<<<64, 256, 0, m->stream>>>(m->part, splits, (int64_t)H * H, m->grad + layer_w(l));
        KG_CUDA_TRY(cudaGetLastError());
        grad_rows_kernel<<<H, 256, 0, m->stream>>>(m->dzt[cur], rows, n_valid, nullptr, m->grad + layer_b(l),
                                                    nullptr);
        KG_CUDA_TRY(cudaGetLastError());
        m->launches += 2;
        // data gradient dz_{l-1} = (dz_l W_l) * GELU'(z_{l-1})
        GemmArgs gd{};
        gd.A = m->dz[cur];
        gd.lda = H;
        gd.a_rows = rows;
        gd.B = m->wt + (int64_t)(l - 2) * H * H;
        gd.ldb = H;
        gd.k_atoms = H / BK;
        gd.out = m->dz[cur ^ 1];
        gd.out_t = m->dzt[cur ^ 1];
        gd.ldot = rows;
        gd.zprev = m->z[l - 2];
        gd.m_valid = n_valid;
        gd.error = m->error;
        KG_TRY(launch_gemm<EPI_BWD>(m, gd, rows / BM, 1));
        cur ^= 1;
    }
    // layer 1: dW1 = dz1^T x, db1 = sum dz1
    grad_rows_kernel<<<H, 256, 0, m->stream>>>(m->dzt[cur], rows, n_valid, m->x, m->grad + kOffB1,
                                                m->grad + kOffW1);
    KG_CUDA_TRY(cudaGetLastError());
    m->launches++;
    return KG_OK;
}

kg_status stage_batch(kg_mlp* m, const float* x, const float* t, int64_t n, int64_t rows, bool train) {
    KG_TRY(mlp_ensure(m, rows, train));
    KG_CUDA_TRY(cudaMemcpyAsync(m->x, x, n * 3 * sizeof(float),
                                is_dev(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
    if (rows > n) KG_CUDA_TRY(cudaMemsetAsync(m->x + n * 3, 0, (rows - n) * 3 * sizeof(float), m->stream));
    if (t)
        KG_CUDA_TRY(cudaMemcpyAsync(m->t, t, n * sizeof(float),
                                    is_dev(t) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream));
    KG_CUDA_TRY(cudaMemsetAsync(m->error, 0, sizeof(int), m->stream));
    return KG_OK;
}

int64_t padded(int64_t n) { return (n + BM - 1) / BM * BM; }

}  // namespace

extern "C" {

kg_status kg_mlp_create(const float* params, void* cuda_stream, kg_mlp** out) {
    clear_error();
    if (!params || !out) return fail(KG_EINVAL, "mlp: NULL argument");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return fail(KG_ENODEV, "no CUDA device available");
    }
    kg_mlp* m = new (std::nothrow) kg_mlp();
    if (!m) return fail(KG_ENOMEM, "host allocation failed");
    m->stream = (cudaStream_t)cuda_stream;
    cudaGetDevice(&m->device);
    auto bail = [&](kg_status s) {
        kg_mlp_destroy(m);
        return s;
    };
    const size_t pb = kParams * sizeof(float);
    void* p = nullptr;
    if (cudaMalloc(&p, 4 * pb + (3 * 3 * H * H + 16 * H) * sizeof(__nv_bfloat16) + 256) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(KG_ENOMEM, "mlp: device allocation failed"));
    }
    char* c = (char*)p;
    m->params = (float*)c;
    m->grad = (float*)(c + pb);
    m->adam_m = (float*)(c + 2 * pb);
    m->adam_v = (float*)(c + 3 * pb);
    m->w = (__nv_bfloat16*)(c + ((4 * pb + 255) & ~(size_t)255));
    m->wt = m->w + 3 * H * H;
    m->wtile = m->wt + 3 * H * H;
    m->wextra = m->wtile + 3 * H * H;
    void* q = nullptr;
    if (cudaMalloc(&q, 256) != cudaSuccess) return bail(fail(KG_ENOMEM, "mlp: device allocation failed"));
    m->error = (int*)q;
    m->loss = (double*)((char*)q + 128);
    if (cudaMallocHost((void**)&m->error_host, sizeof(int)) != cudaSuccess)
        return bail(fail(KG_ENOMEM, "mlp: pinned host allocation failed"));
    *m->error_host = 0;
    cudaMemsetAsync(p, 0, 4 * pb, m->stream);
    cudaMemsetAsync(q, 0, 256, m->stream);
    if (cudaMemcpyAsync(m->params, params, pb, is_dev(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        m->stream) != cudaSuccess)
        return bail(fail(KG_ECUDA, "mlp: parameter upload failed"));
    cast_weights_kernel<<<256, 256, 0, m->stream>>>(m->params, m->w, m->wt, m->wtile, m->wextra);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess)
        return bail(fail(KG_ECUDA, std::string("mlp: ") + cudaGetErrorString(cudaGetLastError())));
    *out = m;
    return KG_OK;
}

void kg_mlp_destroy(kg_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    mlp_free_batch(m);
    if (m->params) cudaFree(m->params);
    if (m->error) cudaFree(m->error);
    if (m->error_host) cudaFreeHost(m->error_host);
    delete m;
}

kg_status kg_mlp_get_params(kg_mlp* m, float* params) {
    if (!m || !params) return fail(KG_EINVAL, "mlp: NULL argument");
    KG_CUDA_TRY(cudaMemcpyAsync(params, m->params, kParams * sizeof(float), cudaMemcpyDefault, m->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return KG_OK;
}

kg_status kg_mlp_forward(kg_mlp* m, const float* x, int64_t n, float* y) {
    clear_error();
    if (!m || !x || !y || n < 1) return fail(KG_EINVAL, "mlp: bad arguments");
    const int64_t rows = padded(n);
    // device inputs and outputs are read and written in place (the kernel reads rows >= n
    // as zero and writes only rows < n); host ones go through the handle's buffers
    const bool x_dev = is_dev(x), y_dev = is_dev(y);
    KG_TRY(mlp_ensure(m, rows, false));
    if (!x_dev)
        KG_CUDA_TRY(cudaMemcpyAsync(m->x, x, n * 3 * sizeof(float), cudaMemcpyHostToDevice, m->stream));
    KG_CUDA_TRY(cudaMemsetAsync(m->error, 0, sizeof(int), m->stream));
    KG_TRY(mlp_infer(m, x_dev ? x : m->x, y_dev ? y : m->y, n, rows));
    // one synchronisation for the wait flag and (host y) the outputs
    KG_CUDA_TRY(cudaMemcpyAsync(m->error_host, m->error, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    if (!y_dev) KG_CUDA_TRY(cudaMemcpyAsync(y, m->y, n * sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(m->stream));
    if (*m->error_host) return fail(KG_ETIMEOUT, "mlp: a tensor-core wait gave up");
    return KG_OK;
}

kg_status kg_mlp_gradients(kg_mlp* m, const float* x, const float* t, int64_t n, float* grad, double* loss) {
    clear_error();
    if (!m || !x || !t || n < 1) return fail(KG_EINVAL, "mlp: bad arguments");
    const int64_t rows = padded(n);
    KG_TRY(stage_batch(m, x, t, n, rows, true));
    KG_TRY(mlp_forward(m, n, rows, true));
    KG_TRY(mlp_backward(m, n, rows));
    KG_TRY(check_mlp_error(m));
    if (grad) KG_CUDA_TRY(cudaMemcpyAsync(grad, m->grad, kParams * sizeof(float), cudaMemcpyDefault, m->stream));
    if (loss) KG_CUDA_TRY(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    KG_CUDA_TRY(cudaStreamSynchronize(m->stream));
    return KG_OK;
}

kg_status kg_mlp_train_step(kg_mlp* m, const float* x, const float* t, int64_t n, float lr, double* loss) {
    clear_error();
    if (!m || !x || !t || n < 1 || !(lr > 0)) return fail(KG_EINVAL, "mlp: bad arguments");
    const int64_t rows = padded(n);
    KG_TRY(stage_batch(m, x, t, n, rows, true));
    KG_TRY(mlp_forward(m, n, rows, true));
    KG_TRY(mlp_backward(m, n, rows));
    m->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    adam_kernel<<<256, 256, 0, m->stream>>>(m->params, m->grad, m->adam_m, m->adam_v, kParams, lr, b1, b2, 1e-8f,
                                            c1, c2);
    KG_CUDA_TRY(cudaGetLastError());
    cast_weights_kernel<<<256, 256, 0, m->stream>>>(m->params, m->w, m->wt, m->wtile, m->wextra);
    KG_CUDA_TRY(cudaGetLastError());
    m->launches += 2;
    KG_TRY(check_mlp_error(m));
    if (loss) {
        KG_CUDA_TRY(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        KG_CUDA_TRY(cudaStreamSynchronize(m->stream));
    }
    return KG_OK;
}

kg_status kg_mlp_launches(kg_mlp* m, int64_t* launches) {
    if (!m || !launches) return fail(KG_EINVAL, "mlp: NULL argument");
    *launches = m->launches;
    return KG_OK;
}

kg_status kg_mlp_timing_enable(kg_mlp* m, int enable) {
    if (!m) return fail(KG_EINVAL, "mlp: NULL argument");
    cudaStreamSynchronize(m->stream);
    for (auto& e : m->gemm_events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    m->gemm_events.clear();
    m->gemm_flop = 0.0;
    m->gemm_launches = 0;
    m->timing = enable != 0;
    return KG_OK;
}

kg_status kg_mlp_timing_read(kg_mlp* m, double* gemm_ms, int64_t* gemm_launches, double* gemm_flop) {
    if (!m) return fail(KG_EINVAL, "mlp: NULL argument");
    KG_CUDA_TRY(cudaStreamSynchronize(m->stream));
    double ms = 0.0;
    for (auto& e : m->gemm_events) {
        float t = 0;
        KG_CUDA_TRY(cudaEventElapsedTime(&t, e.first, e.second));
        ms += t;
    }
    if (gemm_ms) *gemm_ms = ms;
    if (gemm_launches) *gemm_launches = m->gemm_launches;
    if (gemm_flop) *gemm_flop = m->gemm_flop;
    return KG_OK;
}

kg_status kg_mlp_gemm_test(const void* a_dev, const void* b_dev, int64_t rows, int k, float* d_dev) {
    clear_error();
    if (!a_dev || !b_dev || !d_dev || rows < 1 || k < BK || k % BK) return fail(KG_EINVAL, "gemm: bad sizes");
    kg_mlp tmp;
    int* err = nullptr;
    KG_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    KG_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
    GemmArgs g{};
    g.A = (const __nv_bfloat16*)a_dev;
    g.lda = k;
    g.a_rows = rows;
    g.B = (const __nv_bfloat16*)b_dev;
    g.ldb = k;
    g.k_atoms = k / BK;
    g.d_f32 = d_dev;
    g.split_stride = 0;
    g.error = err;
    kg_status s = launch_gemm<EPI_F32>(&tmp, g, (rows + BM - 1) / BM, 1);
    int h_err = 0;
    cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(err);
    tmp.batch_allocs.clear();
    if (s != KG_OK) return s;
    if (e != cudaSuccess) return fail(KG_ECUDA, std::string("gemm: ") + cudaGetErrorString(e));
    if (h_err) return fail(KG_ETIMEOUT, "gemm: a tensor-core wait gave up");
    return KG_OK;
}

}  // extern "C"
