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
    int32_t kw;           // ww / sx when that is a whole number below 256,
                          // else 0: a window's right corners are the left
                          // corners of the window kw positions further along
};

// Queries of a launch evaluated together: every thread computes, for each
// query of the group, the window at its own grid position (i, j), so
// queries with one stride read their corners from the same table rows in
// the same sweep (a window of w = k*s rows shares its corner rows with the
// windows k grid rows further down).  The group's grid is the union of its
// queries' output grids; blocks walk it row by row, or in column panels of
// `panel` blocks so that the rows a panel's sweep keeps reusing stay in L2.
struct WinGroup {
    int64_t R, C;         // rows and columns of the union grid
    int64_t nbx;          // blocks per union-grid row
    int64_t first_block;  // first block of this group in the launch
    int32_t q0, nq;       // queries q[q0, q0 + nq)
    int32_t panel;        // blocks per column panel (0: row-major order)
    int32_t share_tl;     // 1: all queries start at the same table row, so
                          //    at grid position (i, j) they share the
                          //    top-left corner (y0 - 1, x0 - 1)
};

constexpr int kQPerLaunch = 16;

struct WinArgs {
    const uint64_t *S, *Q;
    int64_t ld;
    int nq, ng;
    WinQ q[kQPerLaunch];
    WinGroup g[kQPerLaunch];
};

// Windows per thread: 2 (256 apart) where the arithmetic dominates, i.e.
// dense column strides whose corner loads mostly hit the same sectors; 1
// where the gather dominates (column stride >= kSparseStride: neighbouring
// threads' corners lie 24 bytes or more apart, so most corner loads touch
// their own sector, and more resident warps hide more latency).  Measured
// on 20,000^2 with windows 50 and 100 (with 4 dense windows per thread):
// stride 2 runs faster dense (3.09 vs 3.24 ms), stride 3 sparse (1.46 vs
// 1.65 ms), stride 6 sparse (0.56 vs 0.70 ms).  Two dense windows per thread
// instead of four fit the 64-bit-D path in 32 registers (8 blocks per SM
// instead of 6): workload 1's windows 15.21 -> 14.61 ms.
constexpr int kSparseStride = 3;
constexpr int kDenseWpt = 2;
inline int wins_per_thread(int64_t sx) { return sx >= kSparseStride ? 1 : kDenseWpt; }

// Column panel width (blocks of 256 windows) of sparse-stride groups.  With
// about 1,200 resident blocks a 4-block panel keeps ~300 grid rows in
// flight; their corner rows (4 x 256 + w/s points, S and Q, one 64-byte
// line each) stay well inside L2, while row-major order over a wide image
// (tens of blocks per row) pushes the rows a window's top corners need out
// of L2 before they are read.
constexpr int kPanelBlocks = 4;

// A corner of a sparse-stride window.  The default fill brings 128 bytes
// into L2 per miss, of which such a load uses 8; a 64-byte fill halves the
// DRAM reads once corners lie 128 bytes or more apart (one 64-byte line per
// corner point and table), and reads about the same bytes as the 128-byte
// fill for strides of 3 to 8.  The tables are read-only while a window kernel
// runs.
__device__ __forceinline__ uint64_t ld_corner_sparse(const uint64_t *p)
{
    uint64_t v;
    asm("ld.global.nc.L2::64B.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}

template <int WPT>
__device__ __forceinline__ uint64_t ld_corner(const uint64_t *p)
{
    if constexpr (WPT == 1) return ld_corner_sparse(p);
    else return __ldg(p);
}

// Rounding paths of mean and std: FP64 division and square root (window
// areas of 2^32 or more), the integer path on a 128-bit D, the integer path
// on a 64-bit D.
constexpr int kRnFp64 = 0, kRnInt128 = 1, kRnInt64 = 2;

// Sum, mean and std of the window at output index o from its moments.  The
// results leave with streaming stores (st.global.cs): nothing reads them
// back in the launch, so they should not push out of L2 the table rows and
// lattice entries that later windows' corners read.
template <bool DO_SUM, bool DO_MEAN, bool DO_STD, int RN>
__device__ __forceinline__ void store_stats(const WinQ &q, int64_t o, uint64_t sw, uint64_t qw)
{
    if (DO_SUM) __stcs(reinterpret_cast<unsigned long long *>(q.w.sum) + o, sw);
    if (DO_MEAN)
        __stcs(q.w.mean + o,
               RN != kRnFp64 ? rn::mean_rn(sw, q.div) : __ddiv_rn(__ull2double_rn(sw), q.n_d));
    if (DO_STD) {
        double sd;
        if (RN == kRnInt64) {
            sd = rn::std_rn64(q.n, sw, qw, q.div);
        } else if (RN == kRnInt128) {
            sd = rn::std_rn(q.n, sw, qw, q.div);
        } else {
            const unsigned __int128 D = (unsigned __int128)q.n * qw - (unsigned __int128)sw * sw;
            const double d = u128_to_double_rn((uint64_t)(D >> 64), (uint64_t)D);
            sd = __ddiv_rn(__dsqrt_rn(d), q.n_d);
        }
        __stcs(q.w.std + o, sd);
    }
}

// The WPT windows (i, jb), (i, jb + 256), ... of one query: all corner loads
// first (independent, so they are in flight together), then the arithmetic.
// With TL, the top-left corner's S and Q entries are given (tl_s, tl_q:
// WPT == 1, loaded once for all queries of a group).
template <bool DO_SUM, bool DO_MEAN, bool DO_STD, int RN, int WPT, bool TL = false>
__device__ __forceinline__ void window_row(const WinArgs &a, const WinQ &q, int64_t i, int64_t jb,
                                           uint64_t tl_s = 0, uint64_t tl_q = 0)
{
    static_assert(!TL || WPT == 1, "a given top-left corner serves one window per thread");
    const int64_t y0 = q.w.row0 + i * q.w.sy, y1 = y0 + q.w.wh - 1;
    const int64_t ld = a.ld;
    const bool top = y0 > 0;
    const uint64_t *St = a.S + (y0 - 1) * ld, *Sb = a.S + y1 * ld;
    const uint64_t *Qt = a.Q + (y0 - 1) * ld, *Qb = a.Q + y1 * ld;
    const int64_t orow = i * q.w.out_ld;
    uint64_t sw[WPT], qw[WPT];
#pragma unroll
    for (int m = 0; m < WPT; ++m) {
        const int64_t j = jb + 256 * m;
        sw[m] = 0;
        qw[m] = 0;
        if (j < q.w.C) {
            const int64_t x0 = j * q.w.sx, x1 = x0 + q.w.ww - 1;
            const bool left = x0 > 0;
            sw[m] = ld_corner<WPT>(Sb + x1);
            if (top) sw[m] -= ld_corner<WPT>(St + x1);
            if (left) sw[m] -= ld_corner<WPT>(Sb + x0 - 1);
            if constexpr (TL) sw[m] += tl_s;
            else if (top && left) sw[m] += ld_corner<WPT>(St + x0 - 1);
            if (DO_STD) {
                qw[m] = ld_corner<WPT>(Qb + x1);
                if (top) qw[m] -= ld_corner<WPT>(Qt + x1);
                if (left) qw[m] -= ld_corner<WPT>(Qb + x0 - 1);
                if constexpr (TL) qw[m] += tl_q;
                else if (top && left) qw[m] += ld_corner<WPT>(Qt + x0 - 1);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < WPT; ++m) {
        const int64_t j = jb + 256 * m;
        if (j >= q.w.C) break;
        store_stats<DO_SUM, DO_MEAN, DO_STD, RN>(q, orow + j, sw[m], qw[m]);
    }
}

// The group of block `bid`, found from the launch's block offsets (at most
// 16 entries).  Block indices fit 32 bits.
__device__ __forceinline__ const WinGroup &group_of(const WinArgs &a, uint32_t bid)
{
    int g = 0;
#pragma unroll 1
    while (g + 1 < a.ng && bid >= (uint32_t)a.g[g + 1].first_block) ++g;
    return a.g[g];
}

// One window per thread of a sparse-stride query with kw > 0 in a group
// that shares the top-left corner.  The block's 256 threads hold 256
// consecutive grid positions; a window's right corners are the left corners
// of the position kw further along, so every thread publishes its left
// corners in shared memory (the top-left one once per block, the bottom-left
// one per query) and takes its right corners from thread + kw, loading them
// itself only where that thread lies past the block.  Left corners are
// loaded wherever they lie inside the table row, so every thread that serves
// as a partner has them.  Called by every thread of the block (barriers).
template <bool DO_SUM, bool DO_MEAN, bool DO_STD, int RN>
__device__ __forceinline__ void window_shared(const WinArgs &a, const WinQ &q, int64_t i,
                                              int64_t jb, const uint64_t *sh_tl,
                                              uint64_t *sh_bl)
{
    const int t = threadIdx.x, p = t + q.kw;
    const int64_t y0 = q.w.row0 + i * q.w.sy, y1 = y0 + q.w.wh - 1;
    const int64_t ld = a.ld;
    const bool top = y0 > 0;
    const int64_t x0 = jb * q.w.sx, x1 = x0 + q.w.ww - 1;
    const uint64_t *Sb = a.S + y1 * ld, *Qb = a.Q + y1 * ld;
    uint64_t bl_s = 0, bl_q = 0;
    if (x0 > 0 && x0 - 1 < ld) {
        bl_s = ld_corner_sparse(Sb + x0 - 1);
        if (DO_STD) bl_q = ld_corner_sparse(Qb + x0 - 1);
    }
    sh_bl[t] = bl_s;
    if (DO_STD) sh_bl[256 + t] = bl_q;
    __syncthreads();
    const bool valid = jb < q.w.C;
    uint64_t tr_s = 0, tr_q = 0, br_s = 0, br_q = 0;
    if (valid) {
        if (p < 256) {
            tr_s = sh_tl[p];
            br_s = sh_bl[p];
            if (DO_STD) {
                tr_q = sh_tl[256 + p];
                br_q = sh_bl[256 + p];
            }
        } else {                                       // partner past the block
            const uint64_t *St = a.S + (y0 - 1) * ld, *Qt = a.Q + (y0 - 1) * ld;
            br_s = ld_corner_sparse(Sb + x1);
            tr_s = top ? ld_corner_sparse(St + x1) : 0;
            if (DO_STD) {
                br_q = ld_corner_sparse(Qb + x1);
                tr_q = top ? ld_corner_sparse(Qt + x1) : 0;
            }
        }
    }
    __syncthreads();                                   // sh_bl is reused by the next query
    if (!valid) return;
    const uint64_t tl_s = sh_tl[t], tl_q = DO_STD ? sh_tl[256 + t] : 0;
    const uint64_t sw = br_s - tr_s - bl_s + tl_s;
    const uint64_t qw = DO_STD ? br_q - tr_q - bl_q + tl_q : 0;
    store_stats<DO_SUM, DO_MEAN, DO_STD, RN>(q, i * q.w.out_ld + jb, sw, qw);
}

// Blocks per SM the dense kernel asks the compiler to fit (at most 65,536 /
// (256 x blocks) registers a thread): 8 on the 64-bit-D path, which needs no
// more than 32 registers for two windows a thread (ptxas: 27-32, no spills);
// 6 where the 128-bit path or the FP64 sequence need more, and for std
// alone, which would spill at 32.
template <bool DO_SUM, bool DO_MEAN, int RN>
constexpr int dense_min_blocks()
{
    return RN == kRnInt64 && (DO_SUM || DO_MEAN) ? 8 : 6;
}

// Dense column strides: every group holds one query; a block covers 512
// consecutive windows of one output row (thread t: windows t and t + 256,
// so every load and store instruction stays coalesced).
template <bool DO_SUM, bool DO_MEAN, bool DO_STD, int RN>
__global__ void __launch_bounds__(256, (dense_min_blocks<DO_SUM, DO_MEAN, RN>()))
    k_windows_dense(const __grid_constant__ WinArgs a)
{
    const uint32_t bid = blockIdx.x;
    const WinGroup &G = group_of(a, bid);
    const uint32_t blk = bid - (uint32_t)G.first_block;
    const uint32_t nbx = (uint32_t)G.nbx;
    const uint32_t i = blk / nbx;
    const int64_t jb = (int64_t)(blk - i * nbx) * (256 * kDenseWpt) + threadIdx.x;
    window_row<DO_SUM, DO_MEAN, DO_STD, RN, kDenseWpt>(a, a.q[G.q0], i, jb);
}

// Sparse column strides: a block covers 256 consecutive positions of one
// union-grid row of a group and evaluates each of the group's queries there
// (one window per thread and query).
template <bool DO_SUM, bool DO_MEAN, bool DO_STD, int RN>
__global__ void __launch_bounds__(256, 8) k_windows_sparse(const __grid_constant__ WinArgs a)
{
    const uint32_t bid = blockIdx.x;
    const WinGroup &G = group_of(a, bid);
    const uint32_t blk = bid - (uint32_t)G.first_block;
    const uint32_t nbx = (uint32_t)G.nbx;
    const uint32_t pw = (uint32_t)G.panel;
    uint32_t i, bx;
    if (pw == 0) {
        i = blk / nbx;
        bx = blk - i * nbx;
    } else {
        // Full panels of pw blocks first (each R rows deep), then the
        // remaining nbx mod pw columns of blocks as one narrower panel.
        const uint32_t R = (uint32_t)G.R;
        const uint32_t full = nbx / pw, per_panel = pw * R;
        if (blk < full * per_panel) {
            const uint32_t p = blk / per_panel, r = blk - p * per_panel;
            i = r / pw;
            bx = p * pw + (r - i * pw);
        } else {
            const uint32_t rest = nbx - full * pw, r = blk - full * per_panel;
            i = r / rest;
            bx = full * pw + (r - i * rest);
        }
    }
    const int64_t jb = (int64_t)bx * 256 + threadIdx.x;
    __shared__ uint64_t sh_tl[2 * 256], sh_bl[2 * 256];   // corners: S, then Q
    if (G.share_tl) {
        // One load of the shared top-left corner (zero on the table's first
        // row or column) for all queries: 7 of 8 corner loads per window
        // with two queries, 13 of 16 with four.
        const WinQ &q0 = a.q[G.q0];
        const int64_t y0 = q0.w.row0 + (int64_t)i * q0.w.sy, x0 = jb * q0.w.sx;
        uint64_t tl_s = 0, tl_q = 0;
        if (y0 > 0 && x0 > 0 && x0 - 1 < a.ld) {       // inside the table row
            const int64_t off = (y0 - 1) * a.ld + x0 - 1;
            tl_s = ld_corner_sparse(a.S + off);
            if (DO_STD) tl_q = ld_corner_sparse(a.Q + off);
        }
        sh_tl[threadIdx.x] = tl_s;
        if (DO_STD) sh_tl[256 + threadIdx.x] = tl_q;
        __syncthreads();
#pragma unroll 1
        for (int k = G.q0; k < G.q0 + G.nq; ++k) {
            const WinQ &q = a.q[k];
            if ((int64_t)i >= q.w.R) continue;         // uniform over the block
            if (q.kw)                                  // uniform over the block
                window_shared<DO_SUM, DO_MEAN, DO_STD, RN>(a, q, i, jb, sh_tl, sh_bl);
            else
                window_row<DO_SUM, DO_MEAN, DO_STD, RN, 1, true>(a, q, i, jb, tl_s, tl_q);
        }
    } else {
        // Queries with their own top-left corner (a single query of its
        // strides, or banded queries starting at different table rows): a
        // query with kw > 0 publishes its own top-left corners first.
#pragma unroll 1
        for (int k = G.q0; k < G.q0 + G.nq; ++k) {
            const WinQ &q = a.q[k];
            if ((int64_t)i >= q.w.R) continue;         // uniform over the block
            if (q.kw) {                                // uniform over the block
                const int64_t y0 = q.w.row0 + (int64_t)i * q.w.sy, x0 = jb * q.w.sx;
                uint64_t tl_s = 0, tl_q = 0;
                if (y0 > 0 && x0 > 0 && x0 - 1 < a.ld) {
                    const int64_t off = (y0 - 1) * a.ld + x0 - 1;
                    tl_s = ld_corner_sparse(a.S + off);
                    if (DO_STD) tl_q = ld_corner_sparse(a.Q + off);
                }
                sh_tl[threadIdx.x] = tl_s;             // own slot: read back by this
                if (DO_STD) sh_tl[256 + threadIdx.x] = tl_q;   // thread after the barriers
                __syncthreads();
                window_shared<DO_SUM, DO_MEAN, DO_STD, RN>(a, q, i, jb, sh_tl, sh_bl);
            } else {
                window_row<DO_SUM, DO_MEAN, DO_STD, RN, 1>(a, q, i, jb);
            }
        }
    }
}

template <bool A, bool B, bool C, int RN>
void launch_one(const WinArgs &a, unsigned blocks, int wpt, cudaStream_t s)
{
    LaunchScope ls("window_stats", s);
    if (wpt == 1) k_windows_sparse<A, B, C, RN><<<blocks, 256, 0, s>>>(a);
    else k_windows_dense<A, B, C, RN><<<blocks, 256, 0, s>>>(a);
}

swa_status flush(WinArgs &a, int64_t blocks, uint32_t o, int mode, int wpt, cudaStream_t s)
{
    if (a.ng == 0 || blocks == 0) return SWA_OK;
    if (blocks > 0x7fffffffLL) {
        set_error("window grid too large (%lld blocks)", (long long)blocks);
        return SWA_EINVAL;
    }
    const bool ds = o & SWA_OUT_SUM, dm = o & SWA_OUT_MEAN, dd = o & SWA_OUT_STD;
    const unsigned nb = (unsigned)blocks;
#define SWA_L(A, B, C)                                                              \
    (mode == kRnFp64     ? launch_one<A, B, C, kRnFp64>(a, nb, wpt, s)                   \
     : mode == kRnInt128 ? launch_one<A, B, C, kRnInt128>(a, nb, wpt, s)                 \
                       : launch_one<A, B, C, kRnInt64>(a, nb, wpt, s))
// Without std the 64-bit variant is never asked for (mode_of folds it).
#define SWA_L2(A, B, C)                                                             \
    (mode == kRnFp64 ? launch_one<A, B, C, kRnFp64>(a, nb, wpt, s)                      \
                   : launch_one<A, B, C, kRnInt128>(a, nb, wpt, s))
    if (ds && dm && dd) SWA_L(true, true, true);
    else if (ds && dm) SWA_L2(true, true, false);
    else if (ds && dd) SWA_L(true, false, true);
    else if (dm && dd) SWA_L(false, true, true);
    else if (ds) SWA_L2(true, false, false);
    else if (dm) SWA_L2(false, true, false);
    else if (dd) SWA_L(false, false, true);
#undef SWA_L
#undef SWA_L2
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
// launches of their own.  Within a launch, sparse-stride queries with the
// same strides form one group (one sweep over their union grid); every
// other query is a group of its own.
swa_status launch_windows(const uint64_t *S, const uint64_t *Q, int64_t ld, const WinDesc *w,
                          int n, cudaStream_t s)
{
    bool done[SWA_MAX_WINDOWS] = {false};
    // Rounding path of query k: the integer one for areas below 2^32, with
    // D in 64 bits when n times the largest pixel value stays below 2^32
    // (and std is asked for); FP64 for larger areas.
    auto area_of = [&](int k) {
        return w[k].area ? w[k].area : (uint64_t)(w[k].wh * w[k].ww);
    };
    auto mode_of = [&](int k) {
        const uint64_t area = area_of(k);
        if (area >= (1ull << 32)) return kRnFp64;
        const bool d64 = (w[k].outputs & SWA_OUT_STD) && w[k].vmax &&
                         area * (uint64_t)w[k].vmax < (1ull << 32);
        return d64 ? kRnInt64 : kRnInt128;
    };
    for (int k0 = 0; k0 < n; ++k0) {
        if (done[k0]) continue;
        const uint32_t o = w[k0].outputs;
        const int mode = mode_of(k0);
        const int wpt = wins_per_thread(w[k0].sx);
        auto fits = [&](int k) {
            return !done[k] && w[k].outputs == o && mode_of(k) == mode &&
                   wins_per_thread(w[k].sx) == wpt;
        };
        WinArgs a;
        a.S = S;
        a.Q = Q;
        a.ld = ld;
        a.nq = 0;
        a.ng = 0;
        int64_t blocks = 0;
        for (int k1 = k0; k1 < n; ++k1) {
            if (!fits(k1)) continue;
            // The group led by k1: k1 and, for sparse strides, every later
            // fitting query with its strides (at most one launch's worth).
            int members[kQPerLaunch], m = 0;
            int64_t R = 0, C = 0;
            for (int k = k1; k < n && m < kQPerLaunch; ++k) {
                if (!fits(k)) continue;
                if (k != k1 && (wpt != 1 || w[k].sy != w[k1].sy || w[k].sx != w[k1].sx))
                    continue;
                done[k] = true;
                if (w[k].R == 0 || w[k].C == 0) continue;   // nothing to evaluate
                members[m++] = k;
                R = w[k].R > R ? w[k].R : R;
                C = w[k].C > C ? w[k].C : C;
            }
            if (m == 0) continue;
            if (a.nq + m > kQPerLaunch || a.ng == kQPerLaunch) {
                swa_status st = flush(a, blocks, o, mode, wpt, s);
                if (st != SWA_OK) return st;
                a.nq = 0;
                a.ng = 0;
                blocks = 0;
            }
            bool same_row0 = true;
            for (int t = 1; t < m; ++t) same_row0 &= w[members[t]].row0 == w[members[0]].row0;
            WinGroup &g = a.g[a.ng++];
            g.R = R;
            g.C = C;
            g.share_tl = wpt == 1 && m > 1 && same_row0;
            g.nbx = (C + 256 * wpt - 1) / (256 * wpt);
            g.first_block = blocks;
            g.q0 = a.nq;
            g.nq = m;
            g.panel = (wpt == 1 && g.nbx > kPanelBlocks) ? kPanelBlocks : 0;
            blocks += R * g.nbx;
            for (int t = 0; t < m; ++t) {
                const int k = members[t];
                const uint64_t area = area_of(k);
                WinQ &q = a.q[a.nq++];
                q.w = w[k];
                q.n = area;
                q.n_d = (double)area;
                q.div = rn::make_divisor(mode != kRnFp64 ? (uint32_t)area : 1u);
                q.kw = (wpt == 1 && w[k].ww % w[k].sx == 0 && w[k].ww / w[k].sx < 256)
                           ? (int32_t)(w[k].ww / w[k].sx) : 0;
            }
        }
        swa_status st = flush(a, blocks, o, mode, wpt, s);
        if (st != SWA_OK) return st;
    }
    return SWA_OK;
}

}  // namespace swa
