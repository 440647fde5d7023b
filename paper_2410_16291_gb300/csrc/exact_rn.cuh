// Correctly rounded (round-to-nearest-even) double results of the window
// statistics without the FP64 divide and square-root sequences, whose
// throughput on GB300 is ~60 G/s per GPU (measured) against ~37 T/s for FP32.
//
//   mean = RN( RN(Sw) / n )
//   std  = RN( RN( sqrt( RN(D) ) ) / n ),   D = n*Qw - Sw^2 (exact, 128-bit)
//
// which is, operation for operation, (double)Sw / (double)n and
// sqrt((double)D) / (double)n in IEEE double arithmetic.  Every step below
// produces the exactly rounded result from integer arithmetic:
//   - integer -> double: keep the top 53 bits, round on the guard bit with
//     the OR of the discarded bits as sticky bit;
//   - division by the window area n (a launch constant, n < 2^32): an 86-bit
//     numerator divided by n with two 2-word-by-1-word steps of Moller and
//     Granlund's division by invariant integers ("Improved division by
//     invariant integers", IEEE Trans. Computers 60(2), 2011, Algorithm 4),
//     giving a 54- or 55-bit quotient and an exact remainder for the sticky
//     bit;
//   - square root: an FP32 reciprocal-square-root seed, two Newton
//     corrections computed from exact integer residuals N - R^2 (32 of their
//     bits at a fixed position, converted with 32-bit conversions; the
//     second correction rounded to the nearest integer, which leaves R
//     within 0.51 of sqrt(N)), then one exact step to the nearest integer: R
//     is nearest iff -R < N - R^2 <= R (sqrt(N) is an integer or irrational,
//     never a half-integer).
// The functions are __host__ __device__ so a CPU test can compare them with
// the host's IEEE arithmetic bit for bit.
#pragma once

#include <stdint.h>
#include <math.h>

#if defined(__CUDACC__)
#define SWA_HD __host__ __device__ __forceinline__
#else
#define SWA_HD static inline
#endif

namespace swa {
namespace rn {

SWA_HD int clz64(uint64_t x)
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

SWA_HD int clz32(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

SWA_HD double bits_to_double(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    __builtin_memcpy(&d, &b, 8);
    return d;
#endif
}

SWA_HD float bits_to_float(uint32_t b)
{
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float f;
    __builtin_memcpy(&f, &b, 4);
    return f;
#endif
}

// Reciprocal square root seed: rsqrtf on the device (within 2 ulp); on the
// host the correctly rounded value, which host tests may push by
// SWA_RSQRT_TEST_ULPS ulp (a compile-time define) to cover the device's
// error.
SWA_HD float approx_rsqrt(float x)
{
#if defined(__CUDA_ARCH__)
    return rsqrtf(x);
#elif defined(SWA_RSQRT_TEST_ULPS)
    return (1.0f / sqrtf(x)) * (1.0f + (float)(SWA_RSQRT_TEST_ULPS) * 1.1920929e-7f);
#else
    return 1.0f / sqrtf(x);
#endif
}

// 32-bit conversions between integers and float, IEEE-rounded as named, on
// the device by the conversion instructions and on the host by C's
// conversions (which round the same way).  The square root below uses only
// these: GB300 runs 64-bit integer conversions at its FP64 rate, about two
// per SM per clock.
SWA_HD float i32_to_float_rn(int32_t v)
{
#if defined(__CUDA_ARCH__)
    return __int2float_rn(v);
#else
    return (float)v;
#endif
}

// |x| < 2^31, truncated toward zero.
SWA_HD int32_t float_to_i32_rz(float x)
{
#if defined(__CUDA_ARCH__)
    return __float2int_rz(x);
#else
    return (int32_t)x;
#endif
}

// |x| < 2^31, to the nearest integer (ties to even).
SWA_HD int32_t float_to_i32_rn(float x)
{
#if defined(__CUDA_ARCH__)
    return __float2int_rn(x);
#else
    return (int32_t)nearbyintf(x);
#endif
}

// 0 <= x < 2^32, truncated toward zero.
SWA_HD uint32_t float_to_u32_rz(float x)
{
#if defined(__CUDA_ARCH__)
    return __float2uint_rz(x);
#else
    return (uint32_t)x;
#endif
}

// A value sig * 2^exp with sig < 2^53 (sig == 0 means zero).
struct Fp {
    uint64_t sig;
    int exp;
};

// RN of a 64-bit integer to a 53-bit significand.
SWA_HD Fp round_u64(uint64_t x)
{
    const int L = 64 - clz64(x);
    if (L <= 53) return Fp{x, 0};
    const int sh = L - 53;
    uint64_t m = x >> sh;
    const uint64_t g = (x >> (sh - 1)) & 1u;
    const uint64_t st = (x & ((1ull << (sh - 1)) - 1)) != 0;
    m += g & (st | (m & 1u));
    int e = sh;
    if (m >> 53) { m >>= 1; ++e; }
    return Fp{m, e};
}

// RN of the 128-bit integer hi*2^64 + lo to a 53-bit significand.
SWA_HD Fp round_u128(uint64_t hi, uint64_t lo)
{
    if (hi == 0) return round_u64(lo);
    const int L = 128 - clz64(hi);                 // 65..128
    const int sh = L - 53;                          // 12..75
    uint64_t m, g, st;
    if (sh < 64) {
        m = (hi << (64 - sh)) | (lo >> sh);
        g = (lo >> (sh - 1)) & 1u;
        st = (lo & ((1ull << (sh - 1)) - 1)) != 0;
    } else {
        const int s2 = sh - 64;                     // 0..11
        m = hi >> s2;
        g = s2 ? (hi >> (s2 - 1)) & 1u : lo >> 63;
        st = s2 ? (((hi & ((1ull << (s2 - 1)) - 1)) | lo) != 0)
                : ((lo << 1) != 0);
    }
    m += g & (st | (m & 1u));
    int e = sh;
    if (m >> 53) { m >>= 1; ++e; }
    return Fp{m, e};
}

// Divisor n in [1, 2^32): normalized d = n << z (top bit set) and
// v = floor((2^64 - 1) / d) - 2^32.
// pow2: n is a power of two, so a/n is exact (an exponent shift by 31 - z).
struct Divisor {
    uint32_t d, v;
    int z;
    int pow2;
};

static inline Divisor make_divisor(uint32_t n)
{
    Divisor D;
    D.z = n ? __builtin_clz(n) : 0;
    D.d = n << D.z;
    D.v = (uint32_t)(0xffffffffffffffffull / D.d - (1ull << 32));
    D.pow2 = n && (n & (n - 1)) == 0;
    return D;
}

// (u1*2^32 + u0) / d for u1 < d: quotient word, remainder in *r.
SWA_HD uint32_t div_2by1(uint32_t u1, uint32_t u0, const Divisor &D, uint32_t *r)
{
    const uint64_t p = (uint64_t)D.v * u1 + (((uint64_t)u1 << 32) | u0);
    uint32_t q1 = (uint32_t)(p >> 32) + 1u;
    const uint32_t q0 = (uint32_t)p;
    uint32_t rr = u0 - q1 * D.d;
    if (rr > q0) { --q1; rr += D.d; }
    if (rr >= D.d) { ++q1; rr -= D.d; }
    *r = rr;
    return q1;
}

// Bits of RN(a * 2^aexp / n), 1 <= a < 2^53, n < 2^32 as a Divisor.
SWA_HD uint64_t div_rn(uint64_t a, int aexp, const Divisor &D)
{
    if (a == 0) return 0;
    const int la = 64 - clz64(a);
    if (D.pow2) {                                  // exact: a * 2^(aexp - log2 n)
        const uint64_t M = a << (53 - la);         // [2^52, 2^53)
        const int E = la - 1 + aexp - (31 - D.z);
        return ((uint64_t)(E + 1023) << 52) | (M & ((1ull << 52) - 1));
    }
    const int s = 86 - la;                         // a << s has 86 bits
    uint64_t hi, lo;
    if (s >= 64) { hi = a << (s - 64); lo = 0; }
    else { hi = a >> (64 - s); lo = a << s; }
    uint32_t r = (uint32_t)hi;                     // < 2^22 < d
    const uint32_t q1 = div_2by1(r, (uint32_t)(lo >> 32), D, &r);
    const uint32_t q0 = div_2by1(r, (uint32_t)lo, D, &r);
    uint64_t Q = ((uint64_t)q1 << 32) | q0;        // in [2^53, 2^55)
    uint64_t sticky = r != 0;
    int e = 0;
    if (Q >> 54) { sticky |= Q & 1u; Q >>= 1; e = 1; }
    uint64_t M = Q >> 1;
    const uint64_t g = Q & 1u;
    M += g & (sticky | (M & 1u));
    if (M >> 53) { M >>= 1; ++e; }
    const int sh = s - D.z;                        // value = Q * 2^(aexp - sh)
    const int E = 53 + e - sh + aexp;              // unbiased exponent
    return ((uint64_t)(E + 1023) << 52) | (M & ((1ull << 52) - 1));
}

// div_rn for a significand of exactly 53 bits (2^52 <= a < 2^53, the square
// root's result): the 86-bit numerator is a << 33, with no search for the
// leading bit.
SWA_HD uint64_t div_rn53(uint64_t a, int aexp, const Divisor &D)
{
    if (D.pow2) {                                  // exact: a * 2^(aexp - log2 n)
        const int E = 52 + aexp - (31 - D.z);
        return ((uint64_t)(E + 1023) << 52) | (a & ((1ull << 52) - 1));
    }
    uint32_t r = (uint32_t)(a >> 31);              // < 2^22 < d
    const uint32_t q1 = div_2by1(r, (uint32_t)(a << 1), D, &r);
    const uint32_t q0 = div_2by1(r, 0u, D, &r);
    uint64_t Q = ((uint64_t)q1 << 32) | q0;        // in [2^53, 2^55)
    uint64_t sticky = r != 0;
    int e = 0;
    if (Q >> 54) { sticky |= Q & 1u; Q >>= 1; e = 1; }
    uint64_t M = Q >> 1;
    const uint64_t g = Q & 1u;
    M += g & (sticky | (M & 1u));
    if (M >> 53) { M >>= 1; ++e; }
    const int E = 53 + e - (33 - D.z) + aexp;      // value = Q * 2^(aexp - 33 + z)
    return ((uint64_t)(E + 1023) << 52) | (M & ((1ull << 52) - 1));
}

// 128-bit N - R*R for R < 2^54, as (hi, lo) two's complement.
SWA_HD void residual(uint64_t Nhi, uint64_t Nlo, uint64_t R, int64_t *rhi, uint64_t *rlo)
{
    const uint32_t l = (uint32_t)R, h = (uint32_t)(R >> 32);
    const uint64_t ll = (uint64_t)l * l, hl = (uint64_t)h * l, hh = (uint64_t)h * h;
    // R^2 = hh*2^64 + 2*hl*2^32 + ll
    const uint64_t mid_lo = hl << 33, mid_hi = hl >> 31;
    uint64_t sq_lo = ll + mid_lo;
    uint64_t sq_hi = hh + mid_hi + (sq_lo < ll);
    const uint64_t lo = Nlo - sq_lo;
    const uint64_t hi = Nhi - sq_hi - (Nlo < sq_lo);
    *rhi = (int64_t)hi;
    *rlo = lo;
}

// RN(sqrt(sig * 2^exp)) for 1 <= sig < 2^53.
//
// Error budget.  N = Mx * 2^52 with 2^52 <= Mx < 2^54, so 2^52 <= sqrt(N) <
// 2^53.  The seed R0 = fx * rsqrt(fx) * 2^26 has relative error below 2^-21
// (24-bit truncation of Mx, rsqrtf within 2 ulp, one float rounding), so
// e0 = R0 - sqrt(N) has |e0| < 2^32.  A correction R += c * (N - R^2) with
// c = y * 2^-27 ~ 1/(2 sqrt(N)) leaves R - sqrt(N) = -e * (eps + e/(2 sqrt(N))
// + eps * e/(2 sqrt(N))), where eps < 2^-21 is the relative error of the
// float quotient (y, the residual's conversion and one product).
//   First: the residual |N - R0^2| < 2^86.01 enters as its bits 56..87
//   (an int32, floor), and the step is truncated to a multiple of 4; these
//   add below 8 + 4, so |e1| < 2^11 + 2^11 + 12.
//   Second: |N - R1^2| < 2^66.01 enters as its bits 36..67 (an int32;
//   floor, below 2^-17 in the step), and the step is rounded to the
//   nearest integer, so |e2| < 1/2 + 2^-9 + 2^-17 + 2^-28 < 0.51.
// Hence N - R2^2 lies within (2 sqrt(N) + 1) * 0.51 < 2^54 of zero: its low
// 64 bits, read as a signed integer, are its value, and the nearest integer
// to sqrt(N) is R2 - 1, R2 or R2 + 1.
SWA_HD Fp sqrt_rn(uint64_t sig, int exp)
{
    // Mx = sig shifted to 53 bits, and one bit further when that leaves an
    // odd exponent: Mx in [2^52, 2^54) with 53 + odd bits, E even.
    const int t = 53 - (64 - clz64(sig));
    const int odd = (exp - t) & 1;
    const uint64_t Mx = sig << (t + odd);
    const int E = exp - t - odd;
    const uint64_t Nhi = Mx >> 12, Nlo = Mx << 52; // N = Mx * 2^52
    // FP32 seed: y ~ 1/sqrt(Mx); R0 ~ sqrt(N) = sqrt(Mx) * 2^26.
    const float fx = bits_to_float(((uint32_t)(52 + odd + 127) << 23) |
                                   ((uint32_t)(Mx >> (29 + odd)) & 0x7fffffu));
    const float y = approx_rsqrt(fx);
    // fx * y * 16 lies in [2^30, 2^31) up to the seed's error: a float whose
    // integer part is itself, so R0 = that integer * 2^22 exactly.
    uint64_t R = (uint64_t)float_to_u32_rz(fx * y * 16.0f) << 22;
    int64_t rh;
    uint64_t rl;
    residual(Nhi, Nlo, R, &rh, &rl);
    const int32_t t1 = (int32_t)(uint32_t)(((uint64_t)rh << 8) | (rl >> 56));
    // step / 4 = t1 * 2^56 * y * 2^-27 / 4 = t1 * y * 2^27, |.| < 2^30.01
    R = (uint64_t)((int64_t)R +
                   4 * (int64_t)float_to_i32_rz(i32_to_float_rn(t1) * y * 134217728.0f));
    residual(Nhi, Nlo, R, &rh, &rl);
    const int32_t t2 = (int32_t)(uint32_t)(((uint64_t)rh << 28) | (rl >> 36));
    // step = t2 * 2^36 * y * 2^-27 = t2 * y * 2^9, |.| < 2^12.01
    R = (uint64_t)((int64_t)R + float_to_i32_rn(i32_to_float_rn(t2) * y * 512.0f));
    const int64_t rem = (int64_t)(Nlo - R * R);    // N - R^2, |.| < 2^54
    if (rem > (int64_t)R) ++R;
    else if (rem <= -(int64_t)R) --R;
    int e = E / 2 - 26;
    if (R >> 53) { R >>= 1; ++e; }
    return Fp{R, e};
}

// The double sig * 2^exp exactly (sig < 2^53; the exponent stays normal).
SWA_HD double fp_to_double(Fp f)
{
    if (!f.sig) return 0.0;
    const int L = 64 - clz64(f.sig);
    const uint64_t M = f.sig << (53 - L);
    const int E = L - 1 + f.exp;
    return bits_to_double(((uint64_t)(E + 1023) << 52) | (M & ((1ull << 52) - 1)));
}

// mean and std of one window from its exact moments (n < 2^32, n >= 1).
// The integer path serves areas n < 2^32 of pixels up to 65535, so
// Sw < 2^48: converting it to double is exact and RN(Sw) = Sw.
SWA_HD double mean_rn(uint64_t sw, const Divisor &D)
{
    return bits_to_double(div_rn(sw, 0, D));
}

SWA_HD double std_rn(uint64_t n, uint64_t sw, uint64_t qw, const Divisor &D)
{
    // D = n*qw - sw^2 (exact, >= 0)
    const uint64_t a_lo = n * qw;
#if defined(__CUDA_ARCH__)
    const uint64_t a_hi = __umul64hi(n, qw);
    const uint64_t b_lo = sw * sw, b_hi = __umul64hi(sw, sw);
#else
    const unsigned __int128 A = (unsigned __int128)n * qw, B = (unsigned __int128)sw * sw;
    const uint64_t a_hi = (uint64_t)(A >> 64), b_lo = (uint64_t)B, b_hi = (uint64_t)(B >> 64);
#endif
    const uint64_t d_lo = a_lo - b_lo;
    const uint64_t d_hi = a_hi - b_hi - (a_lo < b_lo);
    if ((d_hi | d_lo) == 0) return 0.0;
    const Fp d = round_u128(d_hi, d_lo);
    const Fp s = sqrt_rn(d.sig, d.exp);
    return bits_to_double(div_rn53(s.sig, s.exp, D));
}

// std_rn for windows whose products n*qw and sw*sw both stay below 2^64
// (n times the largest pixel value below 2^32): D is formed in 64 bits, the
// roundings are std_rn's.  n and sw are then below 2^32, so each product
// takes one 32 x 64 (n * qw) or 32 x 32 (sw * sw) multiplication.
SWA_HD double std_rn64(uint64_t n, uint64_t sw, uint64_t qw, const Divisor &D)
{
    const uint32_t n32 = (uint32_t)n, s32 = (uint32_t)sw;
    const uint64_t d = (uint64_t)n32 * qw - (uint64_t)s32 * s32;
    if (d == 0) return 0.0;
    const Fp r = round_u64(d);
    const Fp s = sqrt_rn(r.sig, r.exp);
    return bits_to_double(div_rn53(s.sig, s.exp, D));
}

}  // namespace rn
}  // namespace swa
