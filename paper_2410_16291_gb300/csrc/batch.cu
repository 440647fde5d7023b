// Batched engine: many images of uneven sizes and dtypes, each with its own
// window queries, in two launches that replay as one CUDA graph:
//
//  1. k_batch: ONE persistent launch builds every image's tables.  Its work
//     is a single ticket queue over the SAT tiles of all images (image after
//     image; within an image along the anti-diagonals of its tile grid, or
//     row by row), each processed by the single-pass tile routine with
//     decoupled look-back inside its image.
//  2. k_batch_windows: one launch evaluates every query of every image; a
//     block covers 1024 consecutive windows of one output row of one query,
//     taken from a schedule that walks each image's queries down its tables
//     together (output rows merged by their first table row).
//
// The windows run in a launch of their own because the build's tiles need
// 25 KB of shared memory per warp (9 warps per SM), while the window
// arithmetic is ALU-bound and wants full occupancy.  A run (zeroing the
// ticket and flags, then the two kernels) allocates nothing, so it can be
// replayed from a CUDA graph.  Every image's tables stay in device memory
// until swa_batch_free.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "exact_rn.cuh"
#include "sat_tile.cuh"
#include "swa_internal.h"

namespace swa {
namespace {

struct alignas(128) BImg {
    CUtensorMap tmS, tmQ;             // TMA views of this image's tables
    const char *img;
    int64_t pitch, rows, cols, nby, nsx, ld;
    uint64_t *S, *Q;
    uint32_t *flag_v, *flag_h, *flag_c;
    uint64_t *agg_v, *inc_v, *agg_h, *inc_h, *corner;
    uint32_t tile_base, ntiles;
    int32_t dtype, vec, th, corner_mode;
};

struct BQuery {
    WinDesc w;
    uint64_t n;
    double n_d;
    rn::Divisor div;
    int32_t img, int_rn;
    int32_t d64;                      // std from a 64-bit D (n * max pixel < 2^32)
    int64_t nbx;                      // blocks per output row
    uint32_t item_base, nitems;       // first block, blocks
};

// One block of the query launch: its query and its block within the query
// (output row blk / nbx, column block blk % nbx).
struct BItem {
    uint32_t q, blk;
};

struct BatchArgs {
    const BImg *imgs;
    const BQuery *qs;
    const BItem *sched;               // the query launch's blocks, in launch order
    const uint2 *tick;                // build ticket -> (image, ticket within the image);
                                      // null: image after image
    int32_t nimg, nq;
    uint32_t total_tiles, total_items;
    uint32_t *ticket, *err;
    uint32_t diag;                    // each image's tiles in anti-diagonal order
};

// Warps per build block: 9 (as many as the SM's shared memory holds) or 8;
// a configuration choice the autotuner may make.
constexpr int kBatchWarpsMax = 9;
// Images of one kind whose tiles share the build's work queue at a time
// (their tickets merged by progress) unless the configuration says
// otherwise.  Measured on the batched workload (256 mixed images): build
// 21.28 ms image after image, 19.47 ms in groups of 4, 19.39 ms in groups of
// 16, 20.67 ms all at once; 48 equal 4096^2 uint8 images 2.60 -> 2.21 ms.
constexpr int32_t kBatchInterleave = 8;
// uint16 tiles: 64 rows, staged in two 32-row parts (see onepass_tile).
constexpr int kBatchU16Rows = 64;
// Shared memory per warp: the larger of the uint8 (64-row) and uint16 tile
// routines, so warps working on different dtypes never overlap.
constexpr int kBatchWarpBytes =
    onepass_warp_bytes<uint8_t, 64>() > onepass_warp_bytes<uint16_t, kBatchU16Rows>()
        ? onepass_warp_bytes<uint8_t, 64>() : onepass_warp_bytes<uint16_t, kBatchU16Rows>();

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *tm)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(tm))
                 : "memory");
}

// Largest index i in [0, n) with base(i) <= t (bases ascending).
template <typename F>
__device__ __forceinline__ int find_base(int n, uint32_t t, F base)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base(mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T, bool VEC, int TH>
__device__ __forceinline__ bool batch_tile(const BImg &im, uint32_t t, uint32_t *err,
                                           WarpRes &w)
{
    TileCtx c;
    c.img = im.img;
    c.pitch = im.pitch;
    c.rows = im.rows;
    c.cols = im.cols;
    c.nby = im.nby;
    c.nsx = im.nsx;
    c.flag_v = im.flag_v;
    c.flag_h = im.flag_h;
    c.flag_c = im.flag_c;
    c.corner = im.corner;
    c.corner_mode = im.corner_mode != 0;
    c.agg_v = im.agg_v;
    c.inc_v = im.inc_v;
    c.agg_h = im.agg_h;
    c.inc_h = im.inc_h;
    c.tmS = &im.tmS;
    c.tmQ = &im.tmQ;
    return onepass_tile<T, true, VEC, TH>(c, t, err, w);
}

constexpr int kBWinPerThread = 4;
constexpr int kBWinPerBlock = 256 * kBWinPerThread;

// Queries of all images: block -> (query, block within the query) from the
// launch's schedule, then 1024 consecutive windows of one output row (thread
// t: t, t+256, t+512, t+768).  Results leave with streaming stores
// (st.global.cs): nothing reads them back in this launch, so they should not
// push the table rows that the image's other queries read next out of L2.
// Launch bounds ask for 8 blocks per SM (32 registers a thread): ptxas fits
// the kernel, all three rounding paths included, without spills (left to
// itself it took 40 registers, 6 blocks per SM: 35.3 ms of queries on the
// batched workload, against 34.1 ms at 8 blocks).
__global__ void __launch_bounds__(256, 8) k_batch_windows(const BQuery *__restrict__ qs,
                                                       const BItem *__restrict__ sched,
                                                       const BImg *__restrict__ imgs)
{
    const BItem item = sched[blockIdx.x];
    const BQuery &q = qs[item.q];
    const BImg &im = imgs[q.img];
    const uint32_t blk = item.blk;
    const uint32_t nbx = (uint32_t)q.nbx;
    const uint32_t i = blk / nbx;
    const int64_t jb = (int64_t)(blk - i * nbx) * kBWinPerBlock + threadIdx.x;
    const int64_t ld = im.ld;
    const int64_t y0 = (int64_t)i * q.w.sy, y1 = y0 + q.w.wh - 1;
    const bool top = y0 > 0;
    const uint64_t *St = im.S + (y0 - 1) * ld, *Sb = im.S + y1 * ld;
    const uint64_t *Qt = im.Q + (y0 - 1) * ld, *Qb = im.Q + y1 * ld;
    const uint32_t o = q.w.outputs;
    const int64_t orow = (int64_t)i * q.w.out_ld;
#pragma unroll
    for (int m = 0; m < kBWinPerThread; ++m) {
        const int64_t j = jb + 256 * m;
        if (j >= q.w.C) break;
        const int64_t x0 = j * q.w.sx, x1 = x0 + q.w.ww - 1;
        const bool left = x0 > 0;
        uint64_t sw = __ldg(Sb + x1);
        if (top) sw -= __ldg(St + x1);
        if (left) sw -= __ldg(Sb + x0 - 1);
        if (top && left) sw += __ldg(St + x0 - 1);
        const int64_t oi = orow + j;
        if (o & SWA_OUT_SUM) __stcs(reinterpret_cast<unsigned long long *>(q.w.sum) + oi, sw);
        if (o & SWA_OUT_MEAN)
            __stcs(q.w.mean + oi, q.int_rn ? rn::mean_rn(sw, q.div)
                                           : __ddiv_rn(__ull2double_rn(sw), q.n_d));
        if (o & SWA_OUT_STD) {
            uint64_t qw = __ldg(Qb + x1);
            if (top) qw -= __ldg(Qt + x1);
            if (left) qw -= __ldg(Qb + x0 - 1);
            if (top && left) qw += __ldg(Qt + x0 - 1);
            double sd;
            if (q.int_rn) {
                sd = q.d64 ? rn::std_rn64(q.n, sw, qw, q.div) : rn::std_rn(q.n, sw, qw, q.div);
            } else {
                const unsigned __int128 D =
                    (unsigned __int128)q.n * qw - (unsigned __int128)sw * sw;
                const double dd =
                    rn::fp_to_double(rn::round_u128((uint64_t)(D >> 64), (uint64_t)D));
                sd = __ddiv_rn(__dsqrt_rn(dd), q.n_d);
            }
            __stcs(q.w.std + oi, sd);
        }
    }
}

// Builds: one persistent launch over the tiles of every image.
template <int TH8, int W>
__global__ void __launch_bounds__(W * 32, 1) k_batch(const __grid_constant__ BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    // The warp's ring and staging area persist across tiles and images (the
    // ring's slot order carries over, so no tile waits for the previous
    // tile's stores to finish).
    WarpRes w = warp_res<uint8_t, TH8>(smem_raw, kBatchWarpBytes);
    // Image after image, a warp's tickets only increase, so it caches the
    // ticket range of its current image and searches only past it; with
    // interleaved images the ticket table names the image and the ticket
    // within it.  The image's tensor maps (written by the host before the
    // launch) are acquired for the tensor-map proxy whenever the warp moves
    // to another image.
    int k = 0;
    uint32_t lo = a.imgs[0].tile_base, hi = lo + a.imgs[0].ntiles;
    bool acquired = false;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1u);
        t = __shfl_sync(kFull, t, 0);
        if (t >= a.total_tiles || *(volatile uint32_t *)a.err) break;
        uint32_t local;
        if (a.tick) {
            const uint2 e = a.tick[t];
            if ((int)e.x != k) {
                k = (int)e.x;
                acquired = false;
            }
            local = e.y;
        } else {
            if (t < lo || t >= hi) {
                k += find_base(a.nimg - k, t, [&](int i) { return a.imgs[k + i].tile_base; });
                lo = a.imgs[k].tile_base;
                hi = lo + a.imgs[k].ntiles;
                acquired = false;
            }
            local = t - lo;
        }
        const BImg &im = a.imgs[k];
        const uint32_t tl = a.diag ? diag_tile(local, im.nby, im.nsx) : local;
        if (!acquired) {
            tensormap_acquire(&im.tmS);
            tensormap_acquire(&im.tmQ);
            acquired = true;
        }
        bool ok;
        if (im.dtype == SWA_U8)
            ok = im.vec ? batch_tile<uint8_t, true, TH8>(im, tl, a.err, w)
                        : batch_tile<uint8_t, false, TH8>(im, tl, a.err, w);
        else
            ok = im.vec ? batch_tile<uint16_t, true, kBatchU16Rows>(im, tl, a.err, w)
                        : batch_tile<uint16_t, false, kBatchU16Rows>(im, tl, a.err, w);
        if (!ok) break;
    }
    cp_async_wait_all();
    if (lane == 0) bulk_wait_all();
    __syncwarp();
}

int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

}  // namespace
}  // namespace swa

using namespace swa;

struct swa_batch {
    uint64_t tag;
    int device;
    int32_t nimg, nq, th8, warps;
    uint32_t total_tiles, total_items;
    char *mem;                        // one allocation: descriptors, state, scratch, tables
    int64_t mem_bytes;
    int64_t zero_off, zero_bytes;     // ticket, error word, flags
    BatchArgs args;
    std::vector<int64_t> table_off;   // per image: S offset (Q follows)
    std::vector<int64_t> ld, rows, cols;
    cudaStream_t stream;
};

static const uint64_t kBatchTag = 0x5357414241544348ULL;   // "SWABATCH"

extern "C" {

swa_status swa_batch_create(const swa_batch_item *items, int32_t n, const swa_batch_config *cfg,
                            swa_stream stream, swa_batch **out)
{
    if (out) *out = nullptr;
    if (!items || n <= 0 || !out) {
        set_error("bad batch arguments");
        return SWA_EINVAL;
    }
    const int th8 = cfg && cfg->u8_tile_rows ? cfg->u8_tile_rows : 64;
    if (th8 != 32 && th8 != 64) {
        set_error("u8_tile_rows must be 32 or 64");
        return SWA_EINVAL;
    }
    const int warps = cfg && cfg->warps ? cfg->warps : kBatchWarpsMax;
    if (cfg && (cfg->order < 0 || cfg->order > 1 || cfg->ticket_order < 0 ||
                cfg->ticket_order > 1 || cfg->lookback < 0 || cfg->lookback > 1 ||
                (warps != 9 && warps != 8) || cfg->interleave < 0 || cfg->reserved[0] ||
                cfg->reserved[1])) {
        set_error("bad batch configuration");
        return SWA_EINVAL;
    }
    const bool corner_all = cfg && cfg->lookback == 1;
    const int32_t group = std::min(cfg && cfg->interleave ? cfg->interleave : kBatchInterleave, n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Image order: as given, or largest first.
    std::vector<int32_t> order(n);
    for (int32_t i = 0; i < n; ++i) order[i] = i;
    if (cfg && cfg->order == 1)
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
            return items[a].rows * items[a].cols > items[b].rows * items[b].cols;
        });
    // Interleaved images are grouped by the tile routine they run (pixel
    // type, rows aligned for vector loads or not), keeping the order above
    // within each kind.
    auto kind = [&](int32_t i) {
        const int64_t vb = items[i].dtype == SWA_U8 ? 8 : 16;
        const bool v = ((uintptr_t)items[i].image % vb == 0) && (items[i].pitch_bytes % vb == 0);
        return (items[i].dtype == SWA_U8 ? 0 : 2) + (v ? 0 : 1);
    };
    if (group > 1)
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return kind(a) < kind(b); });
    // Validate and size.
    int64_t nq = 0, tiles = 0, items_w = 0;
    for (int32_t i = 0; i < n; ++i) {
        const swa_batch_item &it = items[i];
        const int64_t pb = it.dtype == SWA_U16 ? 2 : 1;
        if (!it.image || it.rows <= 0 || it.cols <= 0 ||
            (it.dtype != SWA_U8 && it.dtype != SWA_U16) || it.pitch_bytes < it.cols * pb ||
            it.n_windows < 0 || (it.n_windows && !it.windows) ||
            (it.dtype == SWA_U16 && (((uintptr_t)it.image & 1) || (it.pitch_bytes & 1)))) {
            set_error("batch item %d: bad image arguments", i);
            return SWA_EINVAL;
        }
        const unsigned __int128 px = (unsigned __int128)it.rows * (unsigned __int128)it.cols;
        const unsigned __int128 mx = it.dtype == SWA_U8 ? 255 : 65535;
        if (px * mx * mx >= ((unsigned __int128)1 << 64)) {
            set_error("batch item %d: a table entry could exceed 2^64-1", i);
            return SWA_EOVERFLOW;
        }
        const int th = it.dtype == SWA_U8 ? th8 : kBatchU16Rows;
        tiles += ((it.rows + th - 1) / th) * ((it.cols + kSliceCols - 1) / kSliceCols);
        for (int32_t k = 0; k < it.n_windows; ++k) {
            const swa_window &w = it.windows[k];
            if (w.wh <= 0 || w.ww <= 0 || w.sy <= 0 || w.sx <= 0 || w.wh > it.rows ||
                w.ww > it.cols || !w.outputs || (w.outputs & ~7u) ||
                ((w.outputs & SWA_OUT_SUM) && !w.sum) || ((w.outputs & SWA_OUT_MEAN) && !w.mean) ||
                ((w.outputs & SWA_OUT_STD) && !w.std)) {
                set_error("batch item %d window %d: bad query", i, k);
                return SWA_EINVAL;
            }
            const int64_t R = (it.rows - w.wh) / w.sy + 1, C = (it.cols - w.ww) / w.sx + 1;
            if (w.out_ld < C) {
                set_error("batch item %d window %d: out_ld < %lld", i, k, (long long)C);
                return SWA_EINVAL;
            }
            items_w += R * ((C + kBWinPerBlock - 1) / kBWinPerBlock);
            ++nq;
        }
    }
    if (tiles >= 0xffffffffLL || items_w >= 0x7fffffffLL) {
        set_error("batch too large: %lld work items", (long long)(tiles + items_w));
        return SWA_EINVAL;
    }
    // Layout of the single allocation.
    int64_t off = 0;
    const int64_t off_imgs = off;
    off = align256(off + (int64_t)sizeof(BImg) * n);
    const int64_t off_qs = off;
    off = align256(off + (int64_t)sizeof(BQuery) * (nq ? nq : 1));
    const int64_t off_sched = off;
    off = align256(off + (int64_t)sizeof(BItem) * (items_w ? items_w : 1));
    const int64_t off_tick = off;
    if (group > 1) off = align256(off + (int64_t)sizeof(uint2) * tiles);
    const int64_t zero_off = off;                      // ticket, err, flags
    const int64_t off_ticket = off, off_err = off + 4;
    const int64_t off_flags = off + 256;
    off = off_flags + 3 * 4 * tiles;
    const int64_t zero_bytes = off - zero_off;
    off = align256(off);
    std::vector<BImg> himg(n);
    std::vector<BQuery> hq(nq ? nq : 1);
    swa_batch *b = new (std::nothrow) swa_batch();
    if (!b) return SWA_ENOMEM;
    b->tag = kBatchTag;
    b->nimg = n;
    b->nq = (int32_t)nq;
    b->th8 = th8;
    b->warps = warps;
    b->table_off.resize(n);
    b->ld.resize(n);
    b->rows.resize(n);
    b->cols.resize(n);
    b->stream = s;
    // Records and tables: offsets first, pointers after the allocation.
    std::vector<int64_t> off_flag(n), off_rec_v(n), off_rec_h(n), off_rec_c(n), off_tab(n);
    uint32_t tile_base = 0, flag_i = 0;
    for (int32_t pos = 0; pos < n; ++pos) {
        const int32_t i = order[pos];
        const swa_batch_item &it = items[i];
        const int th = it.dtype == SWA_U8 ? th8 : kBatchU16Rows;
        BImg &m = himg[pos];
        memset(&m, 0, sizeof(m));
        m.rows = it.rows;
        m.cols = it.cols;
        m.pitch = it.pitch_bytes;
        m.img = static_cast<const char *>(it.image);
        m.dtype = it.dtype;
        m.th = th;
        const int64_t vb = it.dtype == SWA_U8 ? 8 : 16;
        m.vec = ((uintptr_t)it.image % vb == 0) && (it.pitch_bytes % vb == 0);
        m.nby = (it.rows + th - 1) / th;
        m.nsx = (it.cols + kSliceCols - 1) / kSliceCols;
        m.corner_mode = (corner_all || corner_mode_for(m.nsx, it.dtype)) ? 1 : 0;
        m.ld = (it.cols + kLdAlign - 1) / kLdAlign * kLdAlign;
        m.ntiles = (uint32_t)(m.nby * m.nsx);
        m.tile_base = tile_base;
        tile_base += m.ntiles;
        off_flag[pos] = off_flags + 4 * (int64_t)flag_i;
        flag_i += 3 * m.ntiles;
        off_rec_v[pos] = off;
        off = align256(off + 2 * (int64_t)m.ntiles * 512 * 8);
        off_rec_h[pos] = off;
        off = align256(off + 2 * (int64_t)m.ntiles * (2 * th + 2) * 8);
        off_rec_c[pos] = off;
        off = align256(off + (int64_t)m.ntiles * 2 * 8);
    }
    for (int32_t pos = 0; pos < n; ++pos) {
        off_tab[pos] = off;
        off = align256(off + 2 * himg[pos].rows * himg[pos].ld * 8);
    }
    b->mem_bytes = off;
    swa_status st = SWA_OK;
    void *mem = nullptr;
    if (dev_alloc(&mem, off, s, &st) != cudaSuccess) {
        delete b;
        return st;
    }
    b->mem = static_cast<char *>(mem);
    cudaGetDevice(&b->device);
    char *base = b->mem;
    for (int32_t pos = 0; pos < n; ++pos) {
        BImg &m = himg[pos];
        const int th = m.th;
        m.flag_v = reinterpret_cast<uint32_t *>(base + off_flag[pos]);
        m.flag_h = m.flag_v + m.ntiles;
        m.flag_c = m.flag_h + m.ntiles;
        m.agg_v = reinterpret_cast<uint64_t *>(base + off_rec_v[pos]);
        m.inc_v = m.agg_v + (size_t)m.ntiles * 512;
        m.agg_h = reinterpret_cast<uint64_t *>(base + off_rec_h[pos]);
        m.inc_h = m.agg_h + (size_t)m.ntiles * (2 * th + 2);
        m.corner = reinterpret_cast<uint64_t *>(base + off_rec_c[pos]);
        m.S = reinterpret_cast<uint64_t *>(base + off_tab[pos]);
        m.Q = m.S + m.rows * m.ld;
        if (!table_tensor_map(&m.tmS, m.S, m.rows, m.ld) ||
            !table_tensor_map(&m.tmQ, m.Q, m.rows, m.ld)) {
            set_error("cuTensorMapEncodeTiled failed for batch image %d", order[pos]);
            dev_free(b->mem, b->mem_bytes, s);
            delete b;
            return SWA_ECUDA;
        }
        b->table_off[order[pos]] = off_tab[pos];
        b->ld[order[pos]] = m.ld;
        b->rows[order[pos]] = m.rows;
        b->cols[order[pos]] = m.cols;
    }
    // Queries in image order.
    uint32_t item_base = 0;
    int64_t qk = 0;
    std::vector<int64_t> q_first(n + 1, 0);           // image pos: queries [q_first[pos], q_first[pos+1])
    for (int32_t pos = 0; pos < n; ++pos) {
        const swa_batch_item &it = items[order[pos]];
        q_first[pos] = qk;
        for (int32_t k = 0; k < it.n_windows; ++k) {
            const swa_window &w = it.windows[k];
            BQuery &q = hq[qk++];
            memset(&q, 0, sizeof(q));
            q.w.wh = w.wh;
            q.w.ww = w.ww;
            q.w.sy = w.sy;
            q.w.sx = w.sx;
            q.w.R = (it.rows - w.wh) / w.sy + 1;
            q.w.C = (it.cols - w.ww) / w.sx + 1;
            q.w.out_ld = w.out_ld;
            q.w.outputs = w.outputs;
            q.w.sum = w.sum;
            q.w.mean = w.mean;
            q.w.std = w.std;
            q.n = (uint64_t)(w.wh * w.ww);
            q.n_d = (double)q.n;
            q.int_rn = q.n < (1ull << 32);
            q.d64 = q.int_rn && q.n * (it.dtype == SWA_U8 ? 255ull : 65535ull) < (1ull << 32);
            q.div = rn::make_divisor(q.int_rn ? (uint32_t)q.n : 1u);
            q.img = pos;
            q.nbx = (q.w.C + kBWinPerBlock - 1) / kBWinPerBlock;
            q.item_base = item_base;
            q.nitems = (uint32_t)(q.w.R * q.nbx);
            item_base += q.nitems;
        }
    }
    q_first[n] = qk;
    // Launch order of the query blocks: image by image; within an image, its
    // queries' output rows merged by the table row their windows start at
    // (y0 = i * sy), so all of the image's queries move down its tables
    // together and read each table row while the others' reads keep it in
    // L2, instead of each query sweeping the whole tables on its own.
    std::vector<BItem> hs(item_base ? item_base : 1);
    {
        struct RowKey {
            int64_t y0;
            uint32_t q, i;
        };
        std::vector<RowKey> rows;
        size_t o = 0;
        for (int32_t pos = 0; pos < n; ++pos) {
            rows.clear();
            for (int64_t k = q_first[pos]; k < q_first[pos + 1]; ++k)
                for (int64_t i = 0; i < hq[k].w.R; ++i)
                    rows.push_back(RowKey{i * hq[k].w.sy, (uint32_t)k, (uint32_t)i});
            std::stable_sort(rows.begin(), rows.end(),
                             [](const RowKey &x, const RowKey &y) { return x.y0 < y.y0; });
            for (const RowKey &r : rows) {
                const uint32_t nbx = (uint32_t)hq[r.q].nbx;
                for (uint32_t bx = 0; bx < nbx; ++bx) hs[o++] = BItem{r.q, r.i * nbx + bx};
            }
        }
    }
    // Build tickets with interleaved images: groups of up to `group`
    // consecutive images (in plan order) that run the same tile routine
    // (pixel type, aligned rows or not); within a group every tile gets the key
    // (i + 1/2) / N for its ticket i of the N of its image, and the group's
    // tiles are claimed in key order (ties: plan order).  Each image's
    // tickets keep their order, so every tile's predecessors still hold
    // smaller tickets; the images of a group advance together, so a tile's
    // predecessors are usually done when it starts.
    std::vector<uint2> ht(group > 1 ? tile_base : 0);
    if (group > 1) {
        struct TK {
            double key;
            uint32_t img, i;
        };
        std::vector<TK> g;
        size_t o = 0;
        for (int32_t p0 = 0, p1 = 0; p0 < n; p0 = p1) {
            p1 = p0 + 1;
            while (p1 < n && p1 - p0 < group && himg[p1].dtype == himg[p0].dtype &&
                   himg[p1].vec == himg[p0].vec)
                ++p1;
            g.clear();
            for (int32_t pos = p0; pos < p1; ++pos) {
                const uint32_t N = himg[pos].ntiles;
                for (uint32_t i = 0; i < N; ++i)
                    g.push_back(TK{(i + 0.5) / N, (uint32_t)pos, i});
            }
            std::stable_sort(g.begin(), g.end(),
                             [](const TK &x, const TK &y) { return x.key < y.key; });
            for (const TK &x : g) ht[o++] = make_uint2(x.img, x.i);
        }
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(base + off_imgs, himg.data(), sizeof(BImg) * n,
                             cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (group > 1 && (e = cudaMemcpyAsync(base + off_tick, ht.data(), sizeof(uint2) * tile_base,
                                           cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
        (nq && (e = cudaMemcpyAsync(base + off_qs, hq.data(), sizeof(BQuery) * nq,
                                    cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
        (item_base && (e = cudaMemcpyAsync(base + off_sched, hs.data(),
                                           sizeof(BItem) * item_base, cudaMemcpyHostToDevice,
                                           s)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        set_error("uploading batch descriptors: %s", cudaGetErrorString(e));
        dev_free(b->mem, b->mem_bytes, s);
        delete b;
        return SWA_ECUDA;
    }
    b->zero_off = zero_off;
    b->zero_bytes = zero_bytes;
    b->total_tiles = tile_base;
    b->total_items = item_base;
    BatchArgs &a = b->args;
    a.imgs = reinterpret_cast<const BImg *>(base + off_imgs);
    a.qs = reinterpret_cast<const BQuery *>(base + off_qs);
    a.sched = reinterpret_cast<const BItem *>(base + off_sched);
    a.tick = group > 1 ? reinterpret_cast<const uint2 *>(base + off_tick) : nullptr;
    a.nimg = n;
    a.nq = (int32_t)nq;
    a.total_tiles = tile_base;
    a.total_items = item_base;
    a.ticket = reinterpret_cast<uint32_t *>(base + off_ticket);
    a.err = reinterpret_cast<uint32_t *>(base + off_err);
    a.diag = (ticket_order_diag() && !(cfg && cfg->ticket_order == 1)) ? 1u : 0u;
    *out = b;
    return SWA_OK;
}

swa_status swa_batch_run(swa_batch *b, swa_stream stream)
{
    if (!b || b->tag != kBatchTag) return SWA_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(b->mem + b->zero_off, 0, (size_t)b->zero_bytes, s);
    if (e != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    const int W = b->warps;
    const size_t smem = 1024 + (size_t)W * kBatchWarpBytes;
    auto kern = W == 9 ? (b->th8 == 64 ? k_batch<64, 9> : k_batch<32, 9>)
                       : (b->th8 == 64 ? k_batch<64, 8> : k_batch<32, 8>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess) {
        set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    int64_t blocks = std::min<int64_t>(sms, ((int64_t)b->total_tiles + W - 1) / W);
    if (blocks < 1) blocks = 1;
    {
        LaunchScope ls("batch_build", s);
        kern<<<(unsigned)blocks, W * 32, smem, s>>>(b->args);
    }
    if (b->total_items) {
        LaunchScope ls("batch_windows", s);
        k_batch_windows<<<b->total_items, 256, 0, s>>>(b->args.qs, b->args.sched, b->args.imgs);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("batch launch failed: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    return SWA_OK;
}

swa_status swa_batch_sync(swa_batch *b)
{
    if (!b || b->tag != kBatchTag) return SWA_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        set_error("synchronize: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    uint32_t err = 0;
    if ((e = cudaMemcpy(&err, b->args.err, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) {
        set_error("reading the batch error word: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    if (err) {
        set_error("a batch wait exceeded its limit (0x%x)", err);
        return SWA_ETIMEOUT;
    }
    return SWA_OK;
}

swa_status swa_batch_tables(const swa_batch *b, int32_t item, const uint64_t **d_S,
                            const uint64_t **d_Q, int64_t *ld)
{
    if (!b || b->tag != kBatchTag || item < 0 || item >= b->nimg) return SWA_EINVAL;
    const uint64_t *S = reinterpret_cast<const uint64_t *>(b->mem + b->table_off[item]);
    if (d_S) *d_S = S;
    if (d_Q) *d_Q = S + b->rows[item] * b->ld[item];
    if (ld) *ld = b->ld[item];
    return SWA_OK;
}

int64_t swa_batch_bytes(const swa_batch *b)
{
    return (b && b->tag == kBatchTag) ? b->mem_bytes : -1;
}

void swa_batch_free(swa_batch *b)
{
    if (!b || b->tag != kBatchTag) return;
    dev_free(b->mem, b->mem_bytes, b->stream);
    b->tag = 0;
    delete b;
}

}  // extern "C"
