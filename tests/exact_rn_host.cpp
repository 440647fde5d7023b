// Host build of the CUDA path's exact-rounding helpers, for CPU tests.
#include <stdint.h>
#include "exact_rn.cuh"

extern "C" {

void rn_stats_bulk(const uint64_t *n, const uint64_t *sw, const uint64_t *qw, int64_t count,
                   double *mean, double *stdv)
{
    for (int64_t i = 0; i < count; ++i) {
        const swa::rn::Divisor D = swa::rn::make_divisor((uint32_t)n[i]);
        mean[i] = swa::rn::mean_rn(sw[i], D);
        stdv[i] = swa::rn::std_rn(n[i], sw[i], qw[i], D);
    }
}

// std through the 64-bit-D variant (valid when n * max pixel < 2^32).
void rn_std64_bulk(const uint64_t *n, const uint64_t *sw, const uint64_t *qw, int64_t count,
                   double *stdv)
{
    for (int64_t i = 0; i < count; ++i) {
        const swa::rn::Divisor D = swa::rn::make_divisor((uint32_t)n[i]);
        stdv[i] = swa::rn::std_rn64(n[i], sw[i], qw[i], D);
    }
}

double rn_u128(uint64_t hi, uint64_t lo)
{
    const swa::rn::Fp f = swa::rn::round_u128(hi, lo);
    if (!f.sig) return 0.0;
    return __builtin_ldexp((double)f.sig, f.exp);
}

double rn_sqrt(double x)
{
    uint64_t b;
    __builtin_memcpy(&b, &x, 8);
    const int e = (int)((b >> 52) & 0x7ff);
    const uint64_t sig = (b & ((1ull << 52) - 1)) | (1ull << 52);
    const swa::rn::Fp r = swa::rn::sqrt_rn(sig, e - 1075);
    return __builtin_ldexp((double)r.sig, r.exp);
}

double rn_div(uint64_t a, uint32_t n)
{
    const swa::rn::Divisor D = swa::rn::make_divisor(n);
    const swa::rn::Fp f = swa::rn::round_u64(a);
    return swa::rn::bits_to_double(swa::rn::div_rn(f.sig, f.exp, D));
}
}
