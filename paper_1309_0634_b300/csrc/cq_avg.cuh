/*
 * cq_avg.cuh -- AVG = SUM / COUNT as the correctly rounded double.
 *
 * The published AVG of a group is the IEEE quotient of its SUM, converted to
 * double, by its COUNT: RN(RN(s) / c), round to nearest even (the
 * aggregate's definition, Section 2; the oracle divides in fp64 the same
 * way).  Every finalisation computes one per touched group, and FP64
 * arithmetic is scarce on this part, so the quotient is taken with integer
 * long division instead:
 *
 *   for |s| < 2^53 (so RN(s) = s) and 1 <= c < 2^31, let k = floor(log2(|s|/c))
 *   be the exponent of the quotient; then T = |s| * 2^(52-k) / c lies in
 *   [2^52, 2^53), and its integer part Q with the remainder R of the division
 *   gives the rounded significand: Q + 1 when 2R > c, or when 2R = c and Q is
 *   odd, else Q.  The double is assembled from the sign, k and that
 *   significand (a carry to 2^53 raises the exponent by one).
 *
 * N = |s| * 2^(52-k) is below 2^84; when it fits 64 bits (counts below
 * about 2^11) it is divided by c at once, else as two 64-by-32-bit steps of
 * schoolbook long division (its high part, then the remainder followed by
 * its low 32 bits).  A sum of magnitude 2^53 or more falls back
 * to the FP64 division, whose input is then itself rounded.
 *
 * cq_check_avg (cq_check.cu) compares this against the FP64 division on the
 * device.
 */
#pragma once
#include <stdint.h>

namespace cq {

/* RN(RN(s) / c) for c >= 1. */
__device__ __forceinline__ double avg_rn(long long s, int32_t c) {
    const bool neg = s < 0;
    const unsigned long long a = neg ? 0ull - (unsigned long long)s : (unsigned long long)s;
    if (a >= (1ull << 53)) return __ddiv_rn(__ll2double_rn(s), (double)c);
    if (a == 0) return 0.0;
    const uint32_t cu = (uint32_t)c;
    const int la = 63 - __clzll((long long)a), lc = 31 - __clz((int)cu);
    const int d = la - lc;
    /* k is d when |s| >= c * 2^d, else d - 1 */
    const bool ge = d >= 0 ? (a >> d) >= cu : (a << (-d)) >= cu;
    const int k = ge ? d : d - 1;   /* -31 .. 52 */
    const int e = 52 - k;           /* 0 .. 83 */
    unsigned long long q, r;
    if (la + e <= 63) {   /* N < 2^64 (small counts): one division */
        const unsigned long long nn = a << e;
        q = nn / cu;
        r = nn - q * cu;
    } else {
        unsigned long long nh;
        uint32_t nl;
        if (e >= 32) {
            nh = a << (e - 32);
            nl = 0u;
        } else {
            nh = a >> (32 - e);
            nl = (uint32_t)(a << e);
        }
        const unsigned long long qh = nh / cu, rh = nh - qh * cu;
        const unsigned long long t = (rh << 32) | nl;
        const unsigned long long ql = t / cu;
        r = t - ql * cu;
        q = (qh << 32) + ql;
    }
    /* q in [2^52, 2^53) */
    const unsigned long long twice = r << 1;
    if (twice > cu || (twice == cu && (q & 1ull))) q += 1ull;
    const unsigned long long expo = (unsigned long long)(k + 1023) + (q >> 53);
    const unsigned long long bits = ((unsigned long long)neg << 63) | (expo << 52) | (q & ((1ull << 52) - 1ull));
    return __longlong_as_double((long long)bits);
}

}  // namespace cq
