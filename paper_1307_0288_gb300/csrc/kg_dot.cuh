// FP64 inner products evaluated on the FP32 and integer pipes.
//
// The GB300 executes FP64 at 1/64 of the FP32 rate, so the Chebyshev recursion is
// limited by the DP pipe.  The recursion itself stays in FP64 (6 DFMA per complex
// site-vector update); the moments' inner products, which would cost another 4 DFMA,
// are formed here in double-float arithmetic instead:
//   * each FP64 factor x is split by integer bit operations (no DP instruction, no
//     conversion) into a float head h (the top 24 significand bits) and a float tail l
//     (the next 23 bits), so |x - h - l| < 2^-46 |x|.  The tail is formed exactly as
//     (2^p (1 + m 2^-23)) - 2^p with its 23 bits m placed in a float's mantissa;
//   * a product a b is the exact TwoProduct of the heads, p + e with e = fma(ah, bh, -p)
//     (Dekker's splitting replaced by the FMA), plus the cross terms ah bl + al bh in
//     FP32; al bl (< 2^-46 |a b|) is dropped;
//   * the per-thread sum is a double-float pair (s, c): Knuth's TwoSum adds p to s, its
//     rounding error and the low part of the product join c, and FastTwoSum renormalises
//     the pair after every term, so |c| stays below one unit in the last place of s.
// Each term is accurate to about 2^-45 relative, and the per-thread sum to about
// k 2^-48 of the sum of |terms| after k terms; the pair is handed to the FP64 block
// reduction as s + c.  Range: factors of magnitude in [2^-63, 2^63) and zero are
// handled at that accuracy (the Chebyshev vectors of random-phase inputs are O(1));
// smaller factors lose their tail below 2^-103 and count as 0 below 2^-126, and
// non-finite or huge factors give non-finite sums.  The explicit-rounding intrinsics keep the
// compiler from contracting or reassociating the compensated steps.
#pragma once

#include <cuda_runtime.h>

namespace kg {

__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(bits >> 32), lw = (unsigned)bits;
    const unsigned sign = hw & 0x80000000u;
    const int ed = (int)((hw >> 20) & 0x7FF);
    const int eh = min(ed - 896, 255);                    // biased float exponent of the head
    const unsigned mh = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    hi = eh >= 1 ? __uint_as_float(sign | ((unsigned)eh << 23) | mh) : 0.0f;
    // tail bits 28..6 of the low word, weight 2^(e - 46) for bit 6: as 2^p (1 + m 2^-23) - 2^p
    // with p = e - 23, i.e. biased float exponent ed - 919
    const int et = min(ed - 919, 254);
    const unsigned eb = et >= 1 ? (unsigned)et << 23 : 0u;
    const float t = et >= 1 ? __fsub_rn(__uint_as_float(eb | ((lw & 0x1FFFFFFFu) >> 6)), __uint_as_float(eb))
                            : 0.0f;
    lo = __uint_as_float(__float_as_uint(t) | sign);
}

struct Dot64 {
    float s = 0.0f, c = 0.0f;
    // Adds a b, with the heads and tails of both factors already split.
    __device__ __forceinline__ void add_split(float ah, float al, float bh, float bl) {
        const float p = __fmul_rn(ah, bh);
        const float lo = fmaf(ah, bl, fmaf(al, bh, fmaf(ah, bh, -p)));
        const float t = __fadd_rn(s, p);
        const float bp = __fsub_rn(t, s);
        const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
        const float cc = __fadd_rn(c, __fadd_rn(err, lo));
        s = __fadd_rn(t, cc);
        c = __fsub_rn(cc, __fsub_rn(s, t));
    }
    __device__ __forceinline__ void add_prod(double a, double b) {
        float ah, al, bh, bl;
        split_f64(a, ah, al);
        split_f64(b, bh, bl);
        add_split(ah, al, bh, bl);
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace kg
