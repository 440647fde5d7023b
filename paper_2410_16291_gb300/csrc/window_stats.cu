// Window statistics by four corner lookups (Section II-B: a rectangle's sum is
// read at its corners, subtracting the intermediate points; Section III-B's
// 4(r*c) lookup term) with the average and standard deviation the paper's
// Section II-A mentions.
//
// For the window with top-left (y0, x0) and bottom-right (y1, x1):
//   Sw = S[y1][x1] - S[y0-1][x1] - S[y1][x0-1] + S[y0-1][x0-1]   (mod 2^64,
//        exact because the true value is below 2^64), index -1 reading as 0;
//   Qw likewise on Q;
//   mean = Sw / n;  D = n*Qw - Sw^2 (exact, 128-bit);  std = sqrt(D) / n.
// Both the integer path (exact_rn.cuh: the same roundings done in integer
// arithmetic, used when n < 2^32) and the FP64 path (the 128-bit integer
// rounded to double with a sticky bit, then the IEEE-rounded square root and
// divisions) give the correctly rounded IEEE results of (double)Sw/(double)n
// and sqrt((double)D)/(double)n, bit for bit.  The integer path exists
// because GB300's FP64 divide and square root run at ~60 G/s per GPU.
#include <cuda_runtime.h>
#include <stdint.h>

#include "exact_rn.cuh"
#include "swa_internal.h"

namespace swa {
namespace {

// Round-to-nearest-even conversion of hi*2^64 + lo to double: keep the top 64
// significant bits, fold every lower bit into bit 0 as a sticky bit (the
// rounding point of a 64-bit value with its top bit set lies at bit 10, so
// the sticky bit decides ties exactly as the discarded bits would), convert
// that 64-bit value with the correctly rounded conversion, and scale by an
// exact power of two.
__device__ __forceinline__ double u128_to_double_rn(uint64_t hi, uint64_t lo)
{
    if (hi == 0) return __ull2double_rn(lo);
    const int lz = __clzll((long long)hi);                  // 0..63
    const uint64_t top = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
    const uint64_t rest = lo << lz;                           // bits below `top`
    const double t = __ull2double_rn(top | (rest != 0));
    const int e = 64 - lz;                                    // value = top * 2^e
    return t * __longlong_as_double((long long)(1023 + e) << 52);
}

struct WinArgs {
    const uint64_t *S, *Q;
    int64_t ld;
    WinDesc w;
    double n_d;
    uint64_t n;
    rn::Divisor div;      // n as an invariant divisor (integer path)
    int64_t nbx;          // blocks per output row
};

template <bool DO_SUM, bool DO_MEAN, bool DO_STD, bool INT_RN>
__global__ void __launch_bounds__(256) k_windows(WinArgs a)
{
    const int64_t i = blockIdx.x / a.nbx;
    const int64_t j = (blockIdx.x % a.nbx) * 256 + threadIdx.x;
    if (j >= a.w.C) return;
    const int64_t y0 = i * a.w.sy, x0 = j * a.w.sx;
    const int64_t y1 = y0 + a.w.wh - 1, x1 = x0 + a.w.ww - 1;
    const int64_t ld = a.ld;
    const bool top = y0 > 0, left = x0 > 0;
    const int64_t rt = (y0 - 1) * ld, rb = y1 * ld;
    uint64_t sw = __ldg(a.S + rb + x1);
    if (top) sw -= __ldg(a.S + rt + x1);
    if (left) sw -= __ldg(a.S + rb + x0 - 1);
    if (top && left) sw += __ldg(a.S + rt + x0 - 1);
    const int64_t o = i * a.w.out_ld + j;
    if (DO_SUM) a.w.sum[o] = sw;
    if (DO_MEAN)
        a.w.mean[o] = INT_RN ? rn::mean_rn(sw, a.div) : __ddiv_rn(__ull2double_rn(sw), a.n_d);
    if (DO_STD) {
        uint64_t qw = __ldg(a.Q + rb + x1);
        if (top) qw -= __ldg(a.Q + rt + x1);
        if (left) qw -= __ldg(a.Q + rb + x0 - 1);
        if (top && left) qw += __ldg(a.Q + rt + x0 - 1);
        if (INT_RN) {
            a.w.std[o] = rn::std_rn(a.n, sw, qw, a.div);
        } else {
            const unsigned __int128 D =
                (unsigned __int128)a.n * qw - (unsigned __int128)sw * sw;
            const double d = u128_to_double_rn((uint64_t)(D >> 64), (uint64_t)D);
            a.w.std[o] = __ddiv_rn(__dsqrt_rn(d), a.n_d);
        }
    }
}

template <bool A, bool B, bool C>
void launch_one(const WinArgs &a, unsigned blocks, cudaStream_t s)
{
    LaunchScope ls("window_stats", s);
    if (a.n < (1ull << 32))
        k_windows<A, B, C, true><<<blocks, 256, 0, s>>>(a);
    else
        k_windows<A, B, C, false><<<blocks, 256, 0, s>>>(a);
}

}  // namespace

swa_status launch_windows(const uint64_t *S, const uint64_t *Q, int64_t ld, const WinDesc *w,
                          int n, cudaStream_t s)
{
    for (int k = 0; k < n; ++k) {
        WinArgs a;
        a.S = S;
        a.Q = Q;
        a.ld = ld;
        a.w = w[k];
        a.n = (uint64_t)(w[k].wh * w[k].ww);
        a.n_d = (double)a.n;
        a.div = rn::make_divisor(a.n < (1ull << 32) ? (uint32_t)a.n : 1u);
        a.nbx = (w[k].C + 255) / 256;
        const int64_t blocks = a.nbx * w[k].R;
        if (blocks <= 0) continue;
        if (blocks > 0x7fffffffLL) {
            set_error("window grid too large (%lld blocks)", (long long)blocks);
            return SWA_EINVAL;
        }
        const uint32_t o = w[k].outputs;
        const bool ds = o & SWA_OUT_SUM, dm = o & SWA_OUT_MEAN, dd = o & SWA_OUT_STD;
        const unsigned nb = (unsigned)blocks;
        if (ds && dm && dd) launch_one<true, true, true>(a, nb, s);
        else if (ds && dm) launch_one<true, true, false>(a, nb, s);
        else if (ds && dd) launch_one<true, false, true>(a, nb, s);
        else if (dm && dd) launch_one<false, true, true>(a, nb, s);
        else if (ds) launch_one<true, false, false>(a, nb, s);
        else if (dm) launch_one<false, true, false>(a, nb, s);
        else if (dd) launch_one<false, false, true>(a, nb, s);
        else continue;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("window launch failed: %s", cudaGetErrorString(e));
            return SWA_ECUDA;
        }
    }
    return SWA_OK;
}

}  // namespace swa
