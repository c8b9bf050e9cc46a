// Device helpers shared by the dense sliced contractions on the bf16 tensor
// cores (the 2-RDM's Gram matrix and the FP64 same-spin sigma terms): operand
// staging by bulk copies, and the exact conversion of the per-weight FP32
// accumulators of six 8-bit digit slices (Ozaki splitting) into one 64-bit
// integer.
//
// Digit scheme: an operand value x is written in fixed point relative to a
// power of two 2^e that bounds it, X = round(x 2^(46 - e)) (|X| < 2^46), cut
// into six balanced 8-bit digits d_s (X = sum_s d_s 2^(40 - 8 s), top digit in
// [-64, 64], the others in [-128, 128]) held exactly by bf16 as d_s 2^(-8 s).
// The product of two values is the sum of the 36 digit products of weight
// s + t; the 21 of weight <= 5 are accumulated, one FP32 accumulator per
// weight 0..3 (exact integers in units 2^(-8 (s + t)): at most 3 2^22 units
// for 256 products, and FP32 holds integers up to 2^24) and one for weights
// 4 and 5 (plain FP32: terms 2^-32 below the leading ones).  The products of
// weight >= 6 are left out (below 2^-46 of the leading product, zero mean).
#pragma once
#include "sigma_wide_kernel.cuh"

namespace fci {
namespace sm {

// x 2^k for k >= 0, else x / 2^-k rounded to nearest, ties to even: the
// rounding is applied once per flush, hundreds of thousands of times per
// element, so it must not lean either way
__device__ __forceinline__ long long shl_round(long long x, int k) {
    if (k >= 0) return (long long)((unsigned long long)x << k);
    const int r = -k;
    const long long q = x >> r;                      // floor
    const long long rem = x - (long long)((unsigned long long)q << r);  // in [0, 2^r)
    const long long half = 1ll << (r - 1);
    return q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
}

// The integer x = v 2^k of an FP32 value holding an exact integer in units
// 2^-k, |x| <= 2^24: split as round(x 2^-12) 2^12 + rest by FP32 magic-number
// rounding (both parts exact), without conversion instructions.
__device__ __forceinline__ int exact_int24(float v, float two_k) {
    constexpr float M = 12582912.0f;  // 1.5 2^23
    constexpr int MB = 0x4B400000;
    const float x = v * two_k;                     // exact (power of two)
    const float t = fmaf(x, 0x1p-12f, M);
    const int h = __float_as_int(t) - MB;          // round(x 2^-12), |.| <= 2^12
    const float rest = fmaf(-(t - M), 4096.f, x);  // x - h 2^12, exact, |.| <= 2^11
    return h * 4096 + (__float_as_int(rest + M) - MB);
}

// round(2^f (acc0 + ... + acc4)) of one element from its five accumulator
// words: weights 0-3 hold exact integers in units 2^-8L (|.| <= 2^24 units);
// 2^24 (acc0 + ... + acc3) = 2^16 (2^8 (acc0 + acc1)) + 2^24 (acc2 + acc3) is
// then an exact integer.  acc4 is split into round(2^18 acc4), round(2^36 rest)
// and the remainder (|.| <= 2^-37), each exact and each within the FP32
// magic-number rounding.  16 <= f <= 52.
__device__ __forceinline__ long long levels_to_int_f(float v0, float v1, float v2, float v3, float a4, int f,
                                                     float two_f) {
    constexpr float M = 12582912.0f;  // 1.5 2^23
    constexpr int MB = 0x4B400000;
    const long long hi = (long long)exact_int24(v0, 1.f) * 256 + exact_int24(v1, 256.f);
    const long long mid = (long long)exact_int24(v2, 65536.f) * 256 + exact_int24(v3, 16777216.f);
    const float t1 = fmaf(a4, 262144.f, M);
    const int h1 = __float_as_int(t1) - MB;
    const float q1 = fmaf(-(t1 - M), 0x1p-18f, a4);  // a4 - h1 2^-18, exact
    const float t2 = fmaf(q1, 0x1p36f, M);
    const int h2 = __float_as_int(t2) - MB;
    const float q2 = fmaf(-(t2 - M), 0x1p-36f, q1);  // q1 - h2 2^-36, exact
    const int h3 = __float_as_int(fmaf(q2, two_f, M)) - MB;
    const long long lead = (hi << 16) + mid;         // 2^24 (acc0 + ... + acc3)
    const int low = h1 * 262144 + h2;                // 2^36 (acc4 - remainder), |.| < 2^28
    return shl_round(lead, f - 24) + shl_round(low, f - 36) + h3;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}


}  // namespace sm
}  // namespace fci
