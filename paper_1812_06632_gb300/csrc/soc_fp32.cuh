// soc_fp32.cuh -- the FP32 arithmetic of the package tracer on the device.
//
// Every operation is one IEEE binary32 operation with round-to-nearest-even,
// written with the _rn intrinsics; multiply-adds are fused only where an
// explicit __fmaf_rn says so (one rounding, as C99 fmaf), and the
// translation unit is compiled with -fmad=false so that the compiler fuses
// nothing else.  The results are therefore fixed by the operation sequence
// alone, which is what lets the counters be compared bit for bit with an
// independent CPU evaluation.
//
// 1 - exp and log are this project's own: Cody-Waite reduction with a Taylor
// polynomial, and the atanh series; the constants are 1/n!, 1/k, ln 2 split
// into a 16-bit head and its remainder, 1/ln 2 and sqrt 2, each rounded to
// binary32.
#pragma once
#include <cstdint>

namespace soc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies with a Weyl
// sequence on the key.
// ---------------------------------------------------------------------------
struct U4 { uint32_t a, b, c, d; };

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;   // bump after the round (unused after the last)
    }
    return U4{c0, c1, c2, c3};
}

// Odd multiples of 2^-24 in (0, 1): ((x >> 8) | 1) * 2^-24 (exact).
__device__ __forceinline__ float u01(uint32_t x)
{
    return __fmul_rn(__uint2float_rn((x >> 8) | 1u), 0x1p-24f);
}

// ---------------------------------------------------------------------------
// 1 - exp(-tau), tau >= 0, with full relative accuracy at every tau and no
// branch on tau (lanes of a warp in thin and thick cells stay converged):
// x = max(-tau, -87) = k ln2 + r (Cody-Waite: k = rint(x / ln 2), r by two
// fused multiply-adds, |r| <= ln2/2); e^r - 1 = r P(r), P the Taylor series
// of (e^r - 1)/r to degree 6 with coefficients RN(1/n!) in Horner form with
// fused multiply-adds; 1 - e^x = (1 - 2^k) - 2^k (e^r - 1) as one fused
// multiply-add.  Below tau = ln2/2 (k = 0) the result is -(e^r - 1) itself.
// tau <= 0 (or NaN) gives 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float one_minus_exp(float tau)
{
    const float x = fmaxf(-tau, -87.0f);
    const int k = __float2int_rn(__fmul_rn(x, 0x1.715476p+0f));         // rint(x / ln 2)
    const float t = __int2float_rn(k);
    float r = __fmaf_rn(-t, 0x1.62e4p-1f, x);                           // x - k ln2_hi
    r = __fmaf_rn(-t, 0x1.7f7d1cp-20f, r);                              //   - k ln2_lo
    float p = 0x1.a01a02p-13f;                                          // 1/7!
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);                               // 1/6!
    p = __fmaf_rn(p, r, 0x1.111112p-7f);                                // 1/5!
    p = __fmaf_rn(p, r, 0x1.555556p-5f);                                // 1/4!
    p = __fmaf_rn(p, r, 0x1.555556p-3f);                                // 1/3!
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    const float em1 = __fmul_rn(r, p);                                  // e^r - 1
    const float sc = __uint_as_float((uint32_t)(k + 127) << 23);         // 2^k
    const float q = __fmaf_rn(-sc, em1, __fsub_rn(1.0f, sc));
    return tau > 0.0f ? q : 0.0f;
}

// ln(u), u positive and normal.  u = m 2^e with m in (sqrt(1/2), sqrt 2];
// ln m = 2s + 2s z (1/3 + z/5 + z^2/7 + z^3/9), s = (m-1)/(m+1), z = s^2.
__device__ __forceinline__ float log_pos(float u)
{
    const uint32_t b = __float_as_uint(u);
    int e = (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > 0x1.6a09e6p+0f) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(s, s);
    float q = 0x1.c71c72p-4f;                                            // 1/9
    q = __fadd_rn(__fmul_rn(q, z), 0x1.24924ap-3f);                      // 1/7
    q = __fadd_rn(__fmul_rn(q, z), 0x1.99999ap-3f);                      // 1/5
    q = __fadd_rn(__fmul_rn(q, z), 0x1.555556p-2f);                      // 1/3
    const float s2 = __fadd_rn(s, s);
    const float lm = __fadd_rn(s2, __fmul_rn(__fmul_rn(s2, z), q));
    const float t = __int2float_rn(e);
    return __fadd_rn(__fadd_rn(__fmul_rn(t, 0x1.7f7d1cp-20f), lm), __fmul_rn(t, 0x1.62e4p-1f));
}

__device__ __forceinline__ float clamp01(float v) { return fminf(fmaxf(v, 0.0f), 1.0f); }

}  // namespace soc
