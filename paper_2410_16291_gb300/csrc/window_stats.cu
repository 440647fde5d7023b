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

// One window query of a launch.
struct WinQ {
    WinDesc w;
    uint64_t n;           // window area
    double n_d;
    rn::Divisor div;      // n as an invariant divisor (integer path)
    int64_t nbx;          // blocks per output row
    int64_t first_block;  // first block of this query in the launch
};

constexpr int kQPerLaunch = 16;

struct WinArgs {
    const uint64_t *S, *Q;
    int64_t ld;
    int nq;
    WinQ q[kQPerLaunch];
};

// Every block covers 256 consecutive windows of one output row of one query;
// the query is found from the launch's block offsets (at most 16 entries).
template <bool DO_SUM, bool DO_MEAN, bool DO_STD, bool INT_RN>
__global__ void __launch_bounds__(256) k_windows(const __grid_constant__ WinArgs a)
{
    int k = 0;
#pragma unroll 1
    while (k + 1 < a.nq && (int64_t)blockIdx.x >= a.q[k + 1].first_block) ++k;
    const WinQ &q = a.q[k];
    const int64_t blk = (int64_t)blockIdx.x - q.first_block;
    const int64_t i = blk / q.nbx;
    const int64_t j = (blk % q.nbx) * 256 + threadIdx.x;
    if (j >= q.w.C) return;
    const int64_t y0 = i * q.w.sy, x0 = j * q.w.sx;
    const int64_t y1 = y0 + q.w.wh - 1, x1 = x0 + q.w.ww - 1;
    const int64_t ld = a.ld;
    const bool top = y0 > 0, left = x0 > 0;
    const int64_t rt = (y0 - 1) * ld, rb = y1 * ld;
    uint64_t sw = __ldg(a.S + rb + x1);
    if (top) sw -= __ldg(a.S + rt + x1);
    if (left) sw -= __ldg(a.S + rb + x0 - 1);
    if (top && left) sw += __ldg(a.S + rt + x0 - 1);
    const int64_t o = i * q.w.out_ld + j;
    if (DO_SUM) q.w.sum[o] = sw;
    if (DO_MEAN)
        q.w.mean[o] = INT_RN ? rn::mean_rn(sw, q.div) : __ddiv_rn(__ull2double_rn(sw), q.n_d);
    if (DO_STD) {
        uint64_t qw = __ldg(a.Q + rb + x1);
        if (top) qw -= __ldg(a.Q + rt + x1);
        if (left) qw -= __ldg(a.Q + rb + x0 - 1);
        if (top && left) qw += __ldg(a.Q + rt + x0 - 1);
        if (INT_RN) {
            q.w.std[o] = rn::std_rn(q.n, sw, qw, q.div);
        } else {
            const unsigned __int128 D =
                (unsigned __int128)q.n * qw - (unsigned __int128)sw * sw;
            const double d = u128_to_double_rn((uint64_t)(D >> 64), (uint64_t)D);
            q.w.std[o] = __ddiv_rn(__dsqrt_rn(d), q.n_d);
        }
    }
}

template <bool A, bool B, bool C, bool I>
void launch_one(const WinArgs &a, unsigned blocks, cudaStream_t s)
{
    LaunchScope ls("window_stats", s);
    k_windows<A, B, C, I><<<blocks, 256, 0, s>>>(a);
}

swa_status flush(WinArgs &a, int64_t blocks, uint32_t o, bool int_rn, cudaStream_t s)
{
    if (a.nq == 0 || blocks == 0) return SWA_OK;
    if (blocks > 0x7fffffffLL) {
        set_error("window grid too large (%lld blocks)", (long long)blocks);
        return SWA_EINVAL;
    }
    const bool ds = o & SWA_OUT_SUM, dm = o & SWA_OUT_MEAN, dd = o & SWA_OUT_STD;
    const unsigned nb = (unsigned)blocks;
#define SWA_L(A, B, C)                                                   \
    (int_rn ? launch_one<A, B, C, true>(a, nb, s) : launch_one<A, B, C, false>(a, nb, s))
    if (ds && dm && dd) SWA_L(true, true, true);
    else if (ds && dm) SWA_L(true, true, false);
    else if (ds && dd) SWA_L(true, false, true);
    else if (dm && dd) SWA_L(false, true, true);
    else if (ds) SWA_L(true, false, false);
    else if (dm) SWA_L(false, true, false);
    else if (dd) SWA_L(false, false, true);
#undef SWA_L
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("window launch failed: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    return SWA_OK;
}

}  // namespace

// Queries sharing an output selection and arithmetic path go into one launch
// (up to 16 per launch); the others follow in launches of their own.
swa_status launch_windows(const uint64_t *S, const uint64_t *Q, int64_t ld, const WinDesc *w,
                          int n, cudaStream_t s)
{
    bool done[SWA_MAX_WINDOWS] = {false};
    for (int k0 = 0; k0 < n; ++k0) {
        if (done[k0]) continue;
        const uint32_t o = w[k0].outputs;
        const bool int_rn = (uint64_t)(w[k0].wh * w[k0].ww) < (1ull << 32);
        WinArgs a;
        a.S = S;
        a.Q = Q;
        a.ld = ld;
        a.nq = 0;
        int64_t blocks = 0;
        for (int k = k0; k < n; ++k) {
            const uint64_t area = (uint64_t)(w[k].wh * w[k].ww);
            if (done[k] || w[k].outputs != o || (area < (1ull << 32)) != int_rn) continue;
            done[k] = true;
            const int64_t nbx = (w[k].C + 255) / 256;
            if (w[k].R * nbx == 0) continue;
            WinQ &q = a.q[a.nq++];
            q.w = w[k];
            q.n = area;
            q.n_d = (double)area;
            q.div = rn::make_divisor(int_rn ? (uint32_t)area : 1u);
            q.nbx = nbx;
            q.first_block = blocks;
            blocks += w[k].R * nbx;
            if (a.nq == kQPerLaunch) {
                swa_status st = flush(a, blocks, o, int_rn, s);
                if (st != SWA_OK) return st;
                a.nq = 0;
                blocks = 0;
            }
        }
        swa_status st = flush(a, blocks, o, int_rn, s);
        if (st != SWA_OK) return st;
    }
    return SWA_OK;
}

}  // namespace swa
