// Counter-based normals for the LRS residual and the random-gamma mode.
//
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 4 x 64-bit counter,
// 2 x 64-bit key, ten rounds of two 64x64->128 multiplies mixed with the other
// words and the key, key bumped by two Weyl constants between rounds.
// Stream layout: key = (seed, member), counter = (step, block, stream_id, 0).
//
// Box-Muller on word pairs (2k, 2k+1): u1 = ((w >> 11) + 1) 2^-53,
// u2 = (w >> 11) 2^-53, z = sqrt(-2 ln u1) (cos, sin)(2 pi u2).  ln, cos and
// sin are evaluated here from their series with explicitly rounded IEEE
// operations (no contraction into FMA), so every normal is reproducible bit
// for bit on any IEEE double implementation evaluating the same sequence:
//   ln x  = e ln2 + 2 atanh(s), x = m 2^e, m in [sqrt2/2, sqrt2],
//           s = (m-1)/(m+1), atanh(s) = sum_{k<12} s^{2k+1}/(2k+1)
//   2 pi u = q pi/2 + theta (4u = q + r exactly, theta = r pi/2), Taylor series
//           of sin and cos in theta with 13 terms each, then the quadrant turn.
#pragma once
#include <stdint.h>

namespace lbm {

constexpr int kStreamLrs = 1;
constexpr int kStreamGamma = 2;

__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const unsigned long long hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

__device__ __forceinline__ unsigned long long philox_word(unsigned long long seed, unsigned long long member,
                                                          long long step, int stream, int word) {
    unsigned long long c[4] = {(unsigned long long)step, (unsigned long long)(word >> 2), (unsigned long long)stream, 0ULL};
    philox4x64_10(c, seed, member);
    return c[word & 3];
}

__device__ __forceinline__ double series_log(double x) {
    const double LN2 = 0.6931471805599453;
    const double SQRT2 = 1.4142135623730951;
    const int K = 12;
    long long b = __double_as_longlong(x);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    if (m > SQRT2) {
        m = __dmul_rn(m, 0.5);
        e += 1;
    }
    const double s = __ddiv_rn(__dadd_rn(m, -1.0), __dadd_rn(m, 1.0));
    const double s2 = __dmul_rn(s, s);
    double p = __ddiv_rn(1.0, (double)(2 * (K - 1) + 1));
    for (int k = K - 2; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, s2), __ddiv_rn(1.0, (double)(2 * k + 1)));
    const double t = __dmul_rn(s, p);
    return __dadd_rn(__dmul_rn((double)e, LN2), __dadd_rn(t, t));
}

__device__ __forceinline__ void series_cos_sin_2pi(double u, double* c, double* s) {
    const double HALF_PI = 1.5707963267948966;
    const int K = 13;
    double invf[2 * K + 2];
    invf[0] = 1.0;
    for (int k = 1; k < 2 * K + 2; ++k) invf[k] = __ddiv_rn(invf[k - 1], (double)k);
    const double v = __dmul_rn(u, 4.0);
    const double qf = floor(v);
    const int q = (int)qf;
    const double r = __dadd_rn(v, -qf);
    const double th = __dmul_rn(r, HALF_PI);
    const double t2 = __dmul_rn(th, th);
    double cs = ((K - 1) % 2 == 0) ? invf[2 * (K - 1)] : -invf[2 * (K - 1)];
    double sn = ((K - 1) % 2 == 0) ? invf[2 * (K - 1) + 1] : -invf[2 * (K - 1) + 1];
    for (int k = K - 2; k >= 0; --k) {
        const double ck = (k % 2 == 0) ? invf[2 * k] : -invf[2 * k];
        const double sk = (k % 2 == 0) ? invf[2 * k + 1] : -invf[2 * k + 1];
        cs = __dadd_rn(__dmul_rn(cs, t2), ck);
        sn = __dadd_rn(__dmul_rn(sn, t2), sk);
    }
    sn = __dmul_rn(sn, th);
    if (q == 0) { *c = cs; *s = sn; }
    else if (q == 1) { *c = -sn; *s = cs; }
    else if (q == 2) { *c = -cs; *s = -sn; }
    else { *c = sn; *s = -cs; }
}

// normal number j of (seed, member, step, stream)
__device__ __forceinline__ double philox_normal(unsigned long long seed, unsigned long long member, long long step,
                                                int stream, int j) {
    const int k = j >> 1;
    const unsigned long long w1 = philox_word(seed, member, step, stream, 2 * k);
    const unsigned long long w2 = philox_word(seed, member, step, stream, 2 * k + 1);
    const double u1 = __dmul_rn((double)((w1 >> 11) + 1ULL), 1.1102230246251565e-16);
    const double u2 = __dmul_rn((double)(w2 >> 11), 1.1102230246251565e-16);
    const double r = __dsqrt_rn(__dmul_rn(-2.0, series_log(u1)));
    double c, s;
    series_cos_sin_2pi(u2, &c, &s);
    return __dmul_rn(r, (j & 1) ? s : c);
}

}  // namespace lbm
