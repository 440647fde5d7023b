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

// Windows per thread: 4 (256 apart) where the arithmetic dominates, i.e.
// dense column strides whose corner loads mostly hit the same sectors; 1
// where the gather dominates (column stride >= kSparseStride: every corner
// load touches its own sector, and more resident warps hide more latency).
constexpr int kSparseStride = 4;
inline int wins_per_thread(int64_t sx) { return sx >= kSparseStride ? 1 : 4; }

// Every block covers 256*WPT consecutive windows of one output row of one
// query (thread t: windows t, t + 256, ... of the block, so every load and
// store instruction stays coalesced); the query is found from the launch's
// block offsets (at most 16 entries).  Block indices fit 32 bits.
template <bool DO_SUM, bool DO_MEAN, bool DO_STD, bool INT_RN, int WPT>
__global__ void __launch_bounds__(256) k_windows(const __grid_constant__ WinArgs a)
{
    constexpr int kWinPerThread = WPT;
    constexpr int kWinPerBlock = 256 * WPT;
    const uint32_t bid = blockIdx.x;
    int k = 0;
#pragma unroll 1
    while (k + 1 < a.nq && bid >= (uint32_t)a.q[k + 1].first_block) ++k;
    const WinQ &q = a.q[k];
    const uint32_t blk = bid - (uint32_t)q.first_block;
    const uint32_t nbx = (uint32_t)q.nbx;
    const uint32_t i = blk / nbx;
    const int64_t jb = (int64_t)(blk - i * nbx) * kWinPerBlock + threadIdx.x;
    const int64_t y0 = q.w.row0 + (int64_t)i * q.w.sy, y1 = y0 + q.w.wh - 1;
    const int64_t ld = a.ld;
    const bool top = y0 > 0;
    const uint64_t *St = a.S + (y0 - 1) * ld, *Sb = a.S + y1 * ld;
    const uint64_t *Qt = a.Q + (y0 - 1) * ld, *Qb = a.Q + y1 * ld;
    const int64_t orow = (int64_t)i * q.w.out_ld;
    // All corner loads of the thread's windows first (independent, so they
    // are in flight together), then the arithmetic.
    uint64_t sw[kWinPerThread], qw[kWinPerThread];
#pragma unroll
    for (int m = 0; m < kWinPerThread; ++m) {
        const int64_t j = jb + 256 * m;
        sw[m] = 0;
        qw[m] = 0;
        if (j < q.w.C) {
            const int64_t x0 = j * q.w.sx, x1 = x0 + q.w.ww - 1;
            const bool left = x0 > 0;
            sw[m] = __ldg(Sb + x1);
            if (top) sw[m] -= __ldg(St + x1);
            if (left) sw[m] -= __ldg(Sb + x0 - 1);
            if (top && left) sw[m] += __ldg(St + x0 - 1);
            if (DO_STD) {
                qw[m] = __ldg(Qb + x1);
                if (top) qw[m] -= __ldg(Qt + x1);
                if (left) qw[m] -= __ldg(Qb + x0 - 1);
                if (top && left) qw[m] += __ldg(Qt + x0 - 1);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < kWinPerThread; ++m) {
        const int64_t j = jb + 256 * m;
        if (j >= q.w.C) break;
        const int64_t o = orow + j;
        if (DO_SUM) q.w.sum[o] = sw[m];
        if (DO_MEAN)
            q.w.mean[o] =
                INT_RN ? rn::mean_rn(sw[m], q.div) : __ddiv_rn(__ull2double_rn(sw[m]), q.n_d);
        if (DO_STD) {
            if (INT_RN) {
                q.w.std[o] = rn::std_rn(q.n, sw[m], qw[m], q.div);
            } else {
                const unsigned __int128 D =
                    (unsigned __int128)q.n * qw[m] - (unsigned __int128)sw[m] * sw[m];
                const double d = u128_to_double_rn((uint64_t)(D >> 64), (uint64_t)D);
                q.w.std[o] = __ddiv_rn(__dsqrt_rn(d), q.n_d);
            }
        }
    }
}

template <bool A, bool B, bool C, bool I>
void launch_one(const WinArgs &a, unsigned blocks, int wpt, cudaStream_t s)
{
    LaunchScope ls("window_stats", s);
    if (wpt == 1) k_windows<A, B, C, I, 1><<<blocks, 256, 0, s>>>(a);
    else k_windows<A, B, C, I, 4><<<blocks, 256, 0, s>>>(a);
}

swa_status flush(WinArgs &a, int64_t blocks, uint32_t o, bool int_rn, int wpt, cudaStream_t s)
{
    if (a.nq == 0 || blocks == 0) return SWA_OK;
    if (blocks > 0x7fffffffLL) {
        set_error("window grid too large (%lld blocks)", (long long)blocks);
        return SWA_EINVAL;
    }
    const bool ds = o & SWA_OUT_SUM, dm = o & SWA_OUT_MEAN, dd = o & SWA_OUT_STD;
    const unsigned nb = (unsigned)blocks;
#define SWA_L(A, B, C)                                                   \
    (int_rn ? launch_one<A, B, C, true>(a, nb, wpt, s) : launch_one<A, B, C, false>(a, nb, wpt, s))
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

// Queries sharing an output selection, arithmetic path and windows per
// thread go into one launch (up to 16 per launch); the others follow in
// launches of their own.
swa_status launch_windows(const uint64_t *S, const uint64_t *Q, int64_t ld, const WinDesc *w,
                          int n, cudaStream_t s)
{
    bool done[SWA_MAX_WINDOWS] = {false};
    for (int k0 = 0; k0 < n; ++k0) {
        if (done[k0]) continue;
        const uint32_t o = w[k0].outputs;
        const bool int_rn = (uint64_t)(w[k0].wh * w[k0].ww) < (1ull << 32);
        const int wpt = wins_per_thread(w[k0].sx);
        WinArgs a;
        a.S = S;
        a.Q = Q;
        a.ld = ld;
        a.nq = 0;
        int64_t blocks = 0;
        for (int k = k0; k < n; ++k) {
            const uint64_t area = (uint64_t)(w[k].wh * w[k].ww);
            if (done[k] || w[k].outputs != o || (area < (1ull << 32)) != int_rn ||
                wins_per_thread(w[k].sx) != wpt)
                continue;
            done[k] = true;
            const int64_t nbx = (w[k].C + 256 * wpt - 1) / (256 * wpt);
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
                swa_status st = flush(a, blocks, o, int_rn, wpt, s);
                if (st != SWA_OK) return st;
                a.nq = 0;
                blocks = 0;
            }
        }
        swa_status st = flush(a, blocks, o, int_rn, wpt, s);
        if (st != SWA_OK) return st;
    }
    return SWA_OK;
}

}  // namespace swa
