// Device building blocks of the SAT build shared by the one-image kernels
// (sat_build.cu) and the batched engine (batch.cu): pixel loads, warp scans,
// the TMA row output ring and the single-pass tile routine with decoupled
// look-back.  See sat_build.cu for the decomposition of a table entry.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "swa_internal.h"
#include "tile_order.cuh"

namespace swa {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 8;                 // warps per block in tile kernels

// Tile-local accumulator of squared pixels: 32 bits hold 256 x 128 x 255^2,
// but uint16 squares need 64 bits.
template <typename T> struct QAcc { using type = uint32_t; };
template <> struct QAcc<uint16_t> { using type = uint64_t; };

// Load 8 consecutive pixels of row y starting at column x, packed (2 words
// for uint8, 4 for uint16) until used; pixels at or past `cols` read as 0.
// VEC: the image base and pitch are aligned to 8 pixels' bytes, so a full
// chunk is one 8- (uint8) or 16-byte (uint16) load.
template <typename T> struct Raw8 { uint32_t w[sizeof(T) * 2]; };

template <typename T, bool VEC>
__device__ __forceinline__ Raw8<T> load_raw8(const char *__restrict__ img, int64_t pitch,
                                             int64_t y, int64_t x, int64_t cols)
{
    Raw8<T> r;
    const T *row = reinterpret_cast<const T *>(img + y * pitch);
    if (VEC && x + 8 <= cols) {
        if (sizeof(T) == 1) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(row + x));
            r.w[0] = v.x; r.w[1] = v.y;
        } else {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(row + x));
            r.w[0] = v.x; r.w[1] = v.y; r.w[2 % (sizeof(T) * 2)] = v.z;
            r.w[3 % (sizeof(T) * 2)] = v.w;
        }
    } else {
        // Any (even, for uint16) byte alignment: the 8-byte-aligned words that
        // cover the chunk, shifted by its misalignment, when they lie inside
        // the row; byte by byte near the row's ends.
        const char *rowc = img + y * pitch;
        const int64_t rowbytes = cols * (int64_t)sizeof(T);
        const int64_t cb = x * (int64_t)sizeof(T);
        const int m = (int)(reinterpret_cast<uintptr_t>(rowc + cb) & 7u);
        constexpr int NW = sizeof(T) == 1 ? 2 : 3;
        if (cb - m >= 0 && cb - m + 8 * NW <= rowbytes) {
            const unsigned long long *wp =
                reinterpret_cast<const unsigned long long *>(rowc + cb - m);
            uint64_t wv[NW];
#pragma unroll
            for (int i = 0; i < NW; ++i) wv[i] = __ldg(wp + i);
#pragma unroll
            for (int i = 0; i < NW - 1; ++i) {
                const uint64_t v = m ? (wv[i] >> (8 * m)) | (wv[i + 1] << (64 - 8 * m)) : wv[i];
                r.w[(2 * i) % (sizeof(T) * 2)] = (uint32_t)v;
                r.w[(2 * i + 1) % (sizeof(T) * 2)] = (uint32_t)(v >> 32);
            }
        } else {
#pragma unroll
            for (int i = 0; i < (int)sizeof(T) * 2; ++i) r.w[i] = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t v = (x + k < cols) ? (uint32_t)__ldg(row + x + k) : 0u;
                if (sizeof(T) == 1) r.w[k >> 2] |= v << (8 * (k & 3));
                else r.w[(k >> 1) % (sizeof(T) * 2)] |= v << (16 * (k & 1));
            }
        }
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void unpack8(const Raw8<T> &r, uint32_t px[8])
{
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (sizeof(T) == 1) px[k] = (r.w[k >> 2] >> (8 * (k & 3))) & 0xffu;
        else px[k] = (r.w[(k >> 1) % (sizeof(T) * 2)] >> (16 * (k & 1))) & 0xffffu;
    }
}

template <typename U>
__device__ __forceinline__ U warp_incl_scan(U v, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        U t = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += t;
    }
    return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) { return __reduce_add_sync(kFull, v); }
__device__ __forceinline__ uint64_t warp_sum(uint64_t v)
{
#pragma unroll
    for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
    return v;
}

// The lane's 8 consecutive staged pixels of one row.
template <typename T>
__device__ __forceinline__ void smem8(const T *row, int lane, uint32_t px[8])
{
    if (sizeof(T) == 1) {
        const uint2 v = *reinterpret_cast<const uint2 *>(row + lane * 8);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            px[k] = (v.x >> (8 * k)) & 0xffu;
            px[k + 4] = (v.y >> (8 * k)) & 0xffu;
        }
    } else {
        const uint4 v = *reinterpret_cast<const uint4 *>(row + lane * 8);
        px[0] = v.x & 0xffffu; px[1] = v.x >> 16;
        px[2] = v.y & 0xffffu; px[3] = v.y >> 16;
        px[4] = v.z & 0xffffu; px[5] = v.z >> 16;
        px[6] = v.w & 0xffffu; px[7] = v.w >> 16;
    }
}

// Bytes per staged tile row: the slice's pixels plus one 16-byte chunk, so
// an unaligned row can be staged as the 16-byte-aligned chunks covering it.
template <typename T>
constexpr int tile_row_bytes() { return kSliceCols * (int)sizeof(T) + 16; }

// Rows of a TH-row tile staged at a time: all of them while they hold at most
// 16 KB of pixels (256 columns of uint8 up to 64 rows) and the build writes
// S and Q, else 32-row parts.  A build of S alone (count tables, sum-only
// tables) writes half the bytes per tile for about the same work per tile,
// so it trades the second staging of a part for more warps per SM.
template <typename T, int TH, bool WQ = true>
constexpr int staged_rows() { return (TH * (int)sizeof(T) <= 64 && WQ) ? TH : 32; }

// The lane's 8 pixels of one staged row.  VEC rows hold the slice's pixels
// from byte 0; other rows hold the 16-byte-aligned chunks covering the
// slice, whose pixels start m bytes in (m = the row's misalignment, 0..15).
template <typename T, bool VEC>
__device__ __forceinline__ void staged8(const unsigned char *row, int lane, int m, uint32_t px[8])
{
    if (VEC) {
        smem8<T>(reinterpret_cast<const T *>(row), lane, px);
        return;
    }
    // The lane's bytes start at m + 8*sizeof(T)*lane: word j = that / 8,
    // shifted right by sh bits across the following word(s).
    const uint64_t *w = reinterpret_cast<const uint64_t *>(row) + (m >> 3) + lane * sizeof(T);
    const int sh = (m & 7) * 8;
    if (sizeof(T) == 1) {
        const uint64_t lo = w[0], hi = w[1];
        const uint64_t v = sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
#pragma unroll
        for (int k = 0; k < 8; ++k) px[k] = (uint32_t)(v >> (8 * k)) & 0xffu;
    } else {
        const uint64_t w0 = w[0], w1 = w[1], w2 = w[2];
        const uint64_t v0 = sh ? (w0 >> sh) | (w1 << (64 - sh)) : w0;
        const uint64_t v1 = sh ? (w1 >> sh) | (w2 << (64 - sh)) : w1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            px[k] = (uint32_t)(v0 >> (16 * k)) & 0xffffu;
            px[k + 4] = (uint32_t)(v1 >> (16 * k)) & 0xffffu;
        }
    }
}

// ------------------------------------------------------ TMA row output --
// Rows of S and Q leave through shared memory by TMA tensor stores
// (cp.async.bulk.tensor) from a two-slot ring per warp.  The ring holds each
// 2 KB row segment (256 uint64) as 16 "rows" of 128 bytes in the 128-byte
// swizzled layout the tensor map declares; with lane l owning columns
// 8l..8l+7 that layout makes the warp's 16-byte shared stores free of bank
// conflicts.  The bulk stores do not occupy the load/store unit, carry an
// L2 evict-first hint (the tables stream out at 16 bytes per pixel and are
// not re-read soon), and are not waited for by generic-proxy memory fences.
constexpr int kRing = 2;                           // output row slots per warp
constexpr int kRowBytes = kSliceCols * 8;          // one table row segment (2 KB)

// Ring bytes per warp: each slot holds an S row segment, and a Q one when
// the build writes Q.
template <bool WQ> constexpr int ring_bytes() { return kRing * (WQ ? 2 : 1) * kRowBytes; }

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t l2_evict_last_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// TMA tensor store of one 16 x 16 box of uint64 (a 256-column row segment)
// at coordinates (0, x0/16, y), in the current bulk group.
__device__ __forceinline__ void tma_store_row_hint(const CUtensorMap *tm, const void *smem,
                                                   int c1, int c2, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group.L2::cache_hint"
        " [%0, {%1, %2, %3}], [%4], %5;" ::"l"(reinterpret_cast<uint64_t>(tm)),
        "r"(0), "r"(c1), "r"(c2), "r"(smem_addr(smem)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void bulk_commit()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Wait until at most kRing-1 bulk groups still read their shared source.
__device__ __forceinline__ void bulk_wait_ring()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(kRing - 1) : "memory");
}

__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Byte offset, inside a 1024-aligned 2 KB row buffer in the tensor map's
// 128-byte swizzle, of the 16-byte chunk j (elements 8l+2j, 8l+2j+1) of lane
// l: box row l/2, chunk (4(l%2) + j) XOR (row mod 8).
__device__ __forceinline__ int swz_off(int lane, int j)
{
    const int r = lane >> 1;
    return r * 128 + ((((lane & 1) << 2) + j) ^ (r & 7)) * 16;
}

// One output row: the warp writes its 8 S (and Q) values per lane into the
// ring slot, then lane 0 issues the tensor stores.  Values are
// base + pre[k] + lp[k] (uint64 + uint64 + tile-local partial).
template <bool WQ, typename QA>
__device__ __forceinline__ void emit_row(unsigned char *ring, int &slot, const int sw[4],
                                         uint64_t base_s, const uint64_t vs[8],
                                         const uint32_t lp[8], uint64_t base_q,
                                         const uint64_t vq[8], const QA lq[8],
                                         const CUtensorMap *tmS, const CUtensorMap *tmQ,
                                         int c1, int y, uint64_t pol)
{
    const int lane = threadIdx.x & 31;
    unsigned char *rs = ring + slot * ((WQ ? 2 : 1) * kRowBytes);
    unsigned char *rq = rs + kRowBytes;
    if (lane == 0) bulk_wait_ring();     // the slot's previous copy has read it
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j)
        *reinterpret_cast<ulonglong2 *>(rs + sw[j]) =
            make_ulonglong2(base_s + vs[2 * j] + lp[2 * j], base_s + vs[2 * j + 1] + lp[2 * j + 1]);
    if (WQ) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            *reinterpret_cast<ulonglong2 *>(rq + sw[j]) =
                make_ulonglong2(base_q + vq[2 * j] + (uint64_t)lq[2 * j],
                                base_q + vq[2 * j + 1] + (uint64_t)lq[2 * j + 1]);
    }
    fence_async_smem();
    __syncwarp();
    if (lane == 0) {
        tma_store_row_hint(tmS, rs, c1, y, pol);
        if (WQ) tma_store_row_hint(tmQ, rq, c1, y, pol);
        bulk_commit();
    }
    slot = (slot + 1) % kRing;
}

// ------------------------------------------------------------- one pass --
// Single-pass build with decoupled look-back.  Warps take tiles in ticket
// order (an atomic counter, so every smaller ticket belongs to a warp that is
// already running), along the anti-diagonals of the tile grid (diag_tile) or
// row by row; either way a tile's predecessors in both chains hold smaller
// tickets.  A warp stages its tile in shared memory, reduces
// it, and publishes two aggregates at once:
//   vertical   (per tile column slice): the tile's 256 column sums;
//   horizontal (per tile band): the tile's row sums.
// It then looks back up its slice for the column carries V and left along
// its band for the row carries LR (32 predecessors' flags per round trip,
// summing aggregates down to the nearest inclusive record), publishes its
// inclusive records, takes the corner term K from the corner record of the
// tile above-left, publishes its own corner, and finally scans the staged
// tile and writes S and Q through the ring.  Every wait is bounded by a time
// limit; on expiry the warp sets the error word and all warps stop.
constexpr uint32_t kAgg = 1u, kInc = 2u;
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per wait

struct OnePass {
    const char *img;
    int64_t pitch, rows, cols, ld, nby, nsx;
    uint32_t *ticket, *err;
    uint32_t *flag_v, *flag_h, *flag_c;   // [tiles]
    uint64_t *agg_v, *inc_v;          // [tiles][2][256]
    uint64_t *agg_h, *inc_h;          // [tiles][2*TH + 2]
    uint64_t *corner;                 // [tiles][2]
    uint32_t stall_tile0;             // test hook: ticket 0 publishes nothing
    uint32_t diag;                    // tickets along anti-diagonals (diag_tile)
    uint32_t thr;                     // count tables: pixels > thr count 1, others 0
    uint32_t corner_mode;             // K from corner records (else edge mode)
    // Corner lattice (builds with a lattice stride st): the entries of S and Q
    // at rows y and columns x with y + 1 and x + 1 multiples of st, as
    // lat_s[(y + 1) / st - 1][(x + 1) / st - 1] (leading dimension lat_ld).
    uint64_t *lat_s, *lat_q;
    int64_t lat_ld;
    int32_t lat_stride;
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Warp-wide look-back window over the chain of predecessors first, first-1,
// ..., 0 (tile p's flag at flags[p * stride]): lane l polls predecessor
// first - l, so one round trip reads 32 flags.  Waits (bounded) until every
// predecessor up to the nearest inclusive one in the window has published,
// then returns n | (inclusive << 8): add the records of predecessors first
// .. first-n+1, the last one's inclusive record if `inclusive`, otherwise
// n = 32 aggregates and the caller continues 32 further on.  Returns -1 if
// the error word is set (by this wait timing out or by another warp).  The
// warp barrier after the polls orders every lane's record loads after the
// acquiring lane's load of the flag.
__device__ __forceinline__ int lookback32(const uint32_t *flags, int64_t stride, int64_t first,
                                          uint32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = first - lane;
    const uint32_t *fp = flags + (p >= 0 ? p : 0) * stride;
    uint64_t t0 = 0;
    unsigned ns = 64;
    for (;;) {
        // Lanes past the chain's start count as inclusive; tile 0 of a chain
        // always publishes an inclusive record, so they are never used.
        const uint32_t f = p >= 0 ? ld_acquire(fp) : kInc;
        const unsigned ready = __ballot_sync(kFull, f != 0);
        const unsigned incm = __ballot_sync(kFull, f == kInc);
        const unsigned need = incm ? (incm & (0u - incm)) * 2u - 1u : kFull;
        if ((ready & need) == need) {
            __syncwarp();
            return incm ? (__ffs(incm) | 256) : 32;
        }
        if (*(volatile uint32_t *)err) return -1;
        if (!t0) {
            t0 = global_ns();
        } else if (global_ns() - t0 > kWaitLimitNs) {
            if (lane == 0) atomicOr(err, kErrTimeout);
            __syncwarp();
            return -1;
        }
        __nanosleep(ns);
        if (ns < 2048) ns <<= 1;
    }
}

// Every lane has written its part of the records; make them visible, then
// raise up to two flags (an acquire-release fence followed by relaxed stores
// is a release; the readers' ld.acquire pairs with it).
__device__ __forceinline__ void publish(uint32_t *f1, uint32_t v1, uint32_t *f2 = nullptr,
                                        uint32_t v2 = 0)
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        st_relaxed(f1, v1);
        if (f2) st_relaxed(f2, v2);
    }
}

__device__ __forceinline__ void cp_async8(void *smem, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(g)
                 : "memory");
}

__device__ __forceinline__ void cp_async8_hint(void *smem, const void *g, uint64_t pol)
{
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" ::"r"(
                     smem_addr(smem)), "l"(g), "l"(pol)
                 : "memory");
}

// cp_async16 with an L2 cache policy (evict-last for lines read again soon,
// evict-first for their last read).
__device__ __forceinline__ void cp_async16_hint(void *smem, const void *g, uint64_t pol)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(
                     smem_addr(smem)), "l"(g), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(g)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// One image's view for the tile routine.
struct TileCtx {
    const char *img;
    int64_t pitch, rows, cols, nby, nsx;
    uint32_t *flag_v, *flag_h, *flag_c;   // [tiles]
    uint64_t *agg_v, *inc_v;          // [tiles][2][256]
    uint64_t *agg_h, *inc_h;          // [tiles][2*TH + 2]
    uint64_t *corner;                 // [tiles][2]: S, Q at the tile's bottom-right
    const CUtensorMap *tmS, *tmQ;
    uint32_t thr;                     // with THR: the threshold of the count table
    bool corner_mode;                 // K from corner records (else edge mode)
    uint64_t *lat_s, *lat_q;          // with LAT: the corner lattice (see OnePass)
    int64_t lat_ld;
    int32_t lat_stride;               // 8..255
};

// Per-warp resources of the tile routine (the same for every pixel type, so
// one warp can move between images of different types and keep its ring).
struct WarpRes {
    unsigned char *tile;              // staged rows of tile_row_bytes<T>()
    unsigned char *ring;              // [kRing][S, Q][2 KB]
    int slot;
    int sw[4];
    uint64_t pol;                     // L2 evict-first (table rows, last reads)
    uint64_t pol_keep;                // L2 evict-last (pixels staged twice)
};

// Adds the column records (S, and Q with WQ) of the n tiles first, first-1,
// ... of slice s above the current tile, the last one's inclusive record if
// `inc`, two records at a time so their loads overlap.
template <bool WQ>
__device__ __forceinline__ void add_vertical(const TileCtx &a, int64_t first, int64_t s, int n,
                                             bool inc, uint64_t vs[8], uint64_t vq[8])
{
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < n; k += 2) {
        const bool two = k + 1 < n;
        const int64_t u0 = (first - k) * a.nsx + s, u1 = two ? u0 - a.nsx : u0;
        const uint64_t *s0 = (inc && k == n - 1 ? a.inc_v : a.agg_v) + (size_t)u0 * 512 + lane * 8;
        const uint64_t *s1 =
            (inc && k + 1 == n - 1 ? a.inc_v : a.agg_v) + (size_t)u1 * 512 + lane * 8;
        ulonglong2 x0[4], x1[4], z0[4], z1[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x0[i] = __ldcg(reinterpret_cast<const ulonglong2 *>(s0 + 2 * i));
            x1[i] = __ldcg(reinterpret_cast<const ulonglong2 *>(s1 + 2 * i));
            if (WQ) {
                z0[i] = __ldcg(reinterpret_cast<const ulonglong2 *>(s0 + 256 + 2 * i));
                z1[i] = __ldcg(reinterpret_cast<const ulonglong2 *>(s1 + 256 + 2 * i));
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            vs[2 * i] += x0[i].x + (two ? x1[i].x : 0);
            vs[2 * i + 1] += x0[i].y + (two ? x1[i].y : 0);
            if (WQ) {
                vq[2 * i] += z0[i].x + (two ? z1[i].x : 0);
                vq[2 * i + 1] += z0[i].y + (two ? z1[i].y : 0);
            }
        }
    }
}

// With row-major tickets, images at least this many column slices wide take
// the corner term K from the tile above-left (corner mode); narrower ones
// from the horizontal records (edge mode).  In a narrow image the tile
// above-left is only a few tickets older, so chains of corner waits would run
// along the diagonals.  Measured crossover on GB300 (build throughput, both
// modes forced): uint8 from 96 slices, uint16 (half as many rows per tile, so
// tickets pass twice as fast) from 128.  With diagonal tickets (the default)
// edge mode wins at every width.  The build's host side decides and passes
// the mode in.
constexpr int64_t kCornerMinSlicesU8 = 96;
constexpr int64_t kCornerMinSlicesU16 = 128;

// The look-back of tile t = (b, s) after its reduction (column sums cs/cq,
// row sums rs_s/rs_q with lane l holding rows l + 32 j).  It finds the column
// carries V (looking back up the slice), the row carries LR (looking back
// left along the band) and the corner term K, the sum of everything above
// and to the left of the tile, in one of two ways (kCornerMinSlices):
//
// corner mode -- three releases:
//   1. the vertical aggregate (column sums) and the horizontal aggregate (row
//      sums), inclusive records directly for a chain's first tile;
//   2. after both look-backs, the inclusive records;
//   3. the tile's corner, the table's value at its bottom-right pixel:
//      corner(b, s) = K + sum(V) + sum(LR) + the tile's total, with
//      K = corner(b-1, s-1) (0 in the first band or slice).
//   The horizontal aggregate needs nothing but the tile itself, so a band's
//   row-carry chain never waits on the vertical look-backs of its tiles.
// edge mode -- three releases:
//   1. the vertical aggregate;
//   2. after the vertical look-back, the inclusive column prefix and the
//      horizontal aggregate: row sums and sum(V), the corner term of the
//      tiles to the right;
//   3. after the horizontal look-back (which also sums K), the inclusive row
//      prefix.
// On return vs/vq hold K + V*[x] (V prefix-summed across the slice) and
// lr_s/lr_q the row carries; false if a wait gave up.
template <bool WQ, int TH>
__device__ __forceinline__ bool lookback_tile(const TileCtx &a, uint32_t t, int64_t b, int64_t s,
                                              const uint64_t cs[8], const uint64_t cq[8],
                                              const uint64_t rs_s[TH / 32],
                                              const uint64_t rs_q[TH / 32], uint32_t *err,
                                              uint64_t vs[8], uint64_t vq[8],
                                              uint64_t lr_s[TH / 32], uint64_t lr_q[TH / 32])
{
    constexpr int RPL = TH / 32;
    constexpr int HREC = 2 * TH + 2;                   // row sums S, Q; then sum(V) S, Q
    const int lane = threadIdx.x & 31;
    const bool cm = a.corner_mode;
#pragma unroll
    for (int k = 0; k < 8; ++k) { vs[k] = 0; vq[k] = 0; }
#pragma unroll
    for (int j = 0; j < RPL; ++j) { lr_s[j] = 0; lr_q[j] = 0; }
    uint64_t K_s = 0, K_q = 0;

    auto write_vertical = [&](uint64_t *rec, bool with_v) {
        uint64_t *r = rec + (size_t)t * 512 + lane * 8;
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            *reinterpret_cast<ulonglong2 *>(r + k) =
                make_ulonglong2(cs[k] + (with_v ? vs[k] : 0), cs[k + 1] + (with_v ? vs[k + 1] : 0));
            if (WQ)
                *reinterpret_cast<ulonglong2 *>(r + 256 + k) = make_ulonglong2(
                    cq[k] + (with_v ? vq[k] : 0), cq[k + 1] + (with_v ? vq[k + 1] : 0));
        }
    };
    auto write_rows = [&](uint64_t *rec, bool with_lr) {
        uint64_t *r = rec + (size_t)t * HREC;
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            r[lane + 32 * j] = rs_s[j] + (with_lr ? lr_s[j] : 0);
            if (WQ) r[TH + lane + 32 * j] = rs_q[j] + (with_lr ? lr_q[j] : 0);
        }
    };
    auto look_up = [&]() -> bool {                     // V, from the slice above
        for (int64_t bb = b - 1;; bb -= 32) {
            const int lb = lookback32(a.flag_v + s, a.nsx, bb, err);
            if (lb < 0) return false;
            add_vertical<WQ>(a, bb, s, lb & 255, lb >> 8, vs, vq);
            if (lb >> 8) return true;
        }
    };
    auto look_left = [&]() -> bool {                   // LR (and K in edge mode)
        for (int64_t ss = s - 1;; ss -= 32) {
            const int lb = lookback32(a.flag_h + b * a.nsx, 1, ss, err);
            if (lb < 0) return false;
            const int n = lb & 255;
            for (int k = 0; k < n; ++k) {
                const int64_t u = b * a.nsx + ss - k;
                const uint64_t *src =
                    ((lb >> 8) && k == n - 1 ? a.inc_h : a.agg_h) + (size_t)u * HREC;
#pragma unroll
                for (int j = 0; j < RPL; ++j) {
                    lr_s[j] += __ldcg(src + lane + 32 * j);
                    if (WQ) lr_q[j] += __ldcg(src + TH + lane + 32 * j);
                }
                if (!cm) {
                    K_s += __ldcg(src + 2 * TH);
                    if (WQ) K_q += __ldcg(src + 2 * TH + 1);
                }
            }
            if (lb >> 8) return true;
        }
    };

    if (cm) {
        // 1. Both aggregates (inclusive for a chain's first tile), one release.
        write_vertical(b > 0 ? a.agg_v : a.inc_v, false);
        write_rows(s > 0 ? a.agg_h : a.inc_h, false);
        publish(a.flag_v + t, b > 0 ? kAgg : kInc, a.flag_h + t, s > 0 ? kAgg : kInc);
        // 2. Both look-backs, then the inclusive records.
        if (b > 0) {
            if (!look_up()) return false;
            write_vertical(a.inc_v, true);
        }
        if (s > 0) {
            if (!look_left()) return false;
            write_rows(a.inc_h, true);
        }
        if (b > 0 || s > 0)
            publish(b > 0 ? a.flag_v + t : a.flag_h + t, kInc,
                    (b > 0 && s > 0) ? a.flag_h + t : nullptr, kInc);
        // 3. K from the tile above-left; this tile's corner.
        if (b > 0 && s > 0) {
            const int64_t u = (b - 1) * a.nsx + (s - 1);
            if (lookback32(a.flag_c + u, 1, 0, err) < 0) return false;
            K_s = __ldcg(a.corner + 2 * u);
            if (WQ) K_q = __ldcg(a.corner + 2 * u + 1);
        }
        uint64_t ps = 0, pq = 0;               // this lane's share of V + LR + the tile
#pragma unroll
        for (int k = 0; k < 8; ++k) { ps += vs[k] + cs[k]; pq += vq[k] + cq[k]; }
#pragma unroll
        for (int j = 0; j < RPL; ++j) { ps += lr_s[j]; pq += lr_q[j]; }
        ps = warp_sum(ps);
        if (WQ) pq = warp_sum(pq);
        if (lane == 0) {
            a.corner[2 * (size_t)t] = K_s + ps;
            a.corner[2 * (size_t)t + 1] = WQ ? K_q + pq : 0;
        }
        publish(a.flag_c + t, kInc);
    } else {
        // 1. The vertical aggregate.
        if (b > 0) {
            write_vertical(a.agg_v, false);
            publish(a.flag_v + t, kAgg);
            if (!look_up()) return false;
        }
        // 2. The inclusive column prefix and the horizontal aggregate (row
        //    sums and sum(V)); inclusive for the band's first tile.
        write_vertical(a.inc_v, true);
        uint64_t vt_s = 0, vt_q = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) { vt_s += vs[k]; vt_q += vq[k]; }
        vt_s = warp_sum(vt_s);
        if (WQ) vt_q = warp_sum(vt_q);
        {
            uint64_t *rec = (s > 0 ? a.agg_h : a.inc_h);
            write_rows(rec, false);
            if (lane == 0) {
                rec[(size_t)t * HREC + 2 * TH] = vt_s;
                rec[(size_t)t * HREC + 2 * TH + 1] = vt_q;
            }
            publish(a.flag_v + t, kInc, a.flag_h + t, s > 0 ? kAgg : kInc);
        }
        // 3. Row carries and K from the left; the inclusive row prefix.
        if (s > 0) {
            if (!look_left()) return false;
            write_rows(a.inc_h, true);
            if (lane == 0) {
                a.inc_h[(size_t)t * HREC + 2 * TH] = K_s + vt_s;
                a.inc_h[(size_t)t * HREC + 2 * TH + 1] = K_q + vt_q;
            }
            publish(a.flag_h + t, kInc);
        }
    }

    // For the scan S = K + H[y] + V*[x] + lp: vs/vq become K + V*.
#pragma unroll
    for (int k = 1; k < 8; ++k) { vs[k] += vs[k - 1]; if (WQ) vq[k] += vq[k - 1]; }
    {
        const uint64_t is = warp_incl_scan(vs[7], lane), es = is - vs[7];
        const uint64_t iq = WQ ? warp_incl_scan(vq[7], lane) : 0, eq = iq - vq[7];
#pragma unroll
        for (int k = 0; k < 8; ++k) { vs[k] += es + K_s; if (WQ) vq[k] += eq + K_q; }
    }
    return true;
}

// Process tile t of one image (single pass): stage, reduce, publish, look
// back, publish, scan, write.  With LAT the scan also writes the tile's
// entries of the corner lattice (rows and columns one below a multiple of
// the lattice stride, which is at least 8, so a lane's 8 columns hold at most
// one lattice column).  Returns false if a wait gave up (the error word is
// then set).
template <typename T, bool WQ, bool VEC, int TH, bool THR = false, bool LAT = false>
__device__ __forceinline__ bool onepass_tile(const TileCtx &a, uint32_t t, uint32_t *err,
                                             WarpRes &w)
{
    using QA = typename QAcc<T>::type;
    constexpr int RPL = TH / 32;                       // rows each lane keeps
    const int lane = threadIdx.x & 31;
    constexpr int RB = tile_row_bytes<T>();
    // Rows staged at a time: the whole tile, or 32-row parts of it when its
    // pixels exceed 16 KB (uint16 64-row tiles), so the staging buffer and
    // the warps per SM stay those of the uint8 tile.  Parts are staged and
    // reduced bottom part first, so the top part is still staged when the
    // scan begins; the other parts are staged again for their scan (from L2,
    // which has just read them).
    constexpr int SR = staged_rows<T, TH, WQ>();
    constexpr int GPP = SR / 32;                       // 32-row groups per staged part
    static_assert(SR % 32 == 0 && TH % SR == 0, "staged parts are whole 32-row groups");
    unsigned char *tile = w.tile;
    const int64_t b = t / a.nsx, s = t % a.nsx;
    const int64_t y0 = b * TH;
    const int nr = (int)min((int64_t)TH, a.rows - y0);
    const int64_t x = s * kSliceCols + lane * kPxPerLane;
    const int64_t rowbytes = a.cols * (int64_t)sizeof(T);
    const int64_t xb = s * kSliceCols * (int64_t)sizeof(T);     // slice start in a row
    // Misalignment (mod 16) of the slice's first pixel in row r of the tile;
    // 0 with VEC.  32-bit arithmetic: only the low four bits matter.
    const uint32_t m0 = (uint32_t)reinterpret_cast<uintptr_t>(a.img + y0 * a.pitch + xb);
    const uint32_t pm = (uint32_t)a.pitch;
    auto mis = [&](int r) -> int { return VEC ? 0 : (int)((m0 + (uint32_t)r * pm) & 15u); };
    // THR: the table of the 0/1 indicator "pixel > a.thr" (a count table).
    auto px_of = [&](const unsigned char *row, int r, uint32_t px[8]) {
        staged8<T, VEC>(row, lane, mis(r), px);
        if (THR) {
#pragma unroll
            for (int k = 0; k < 8; ++k) px[k] = px[k] > a.thr ? 1u : 0u;
        }
    };

    // Stage rows r0 .. min(nr, r0 + SR) - 1 of the tile into buffer rows 0, 1,
    // ... (columns past the image read as 0).  With
    // VEC every lane copies its 8 pixels with one cp.async.  Otherwise a row
    // may start at any (even, for uint16) byte address: the warp copies the
    // 16-byte-aligned chunks covering the slice (uint8: 17 chunks, lanes
    // 0..16; uint16: 33 chunks, lane l chunk l and lane 0 chunk 32), and
    // staged8 shifts by the row's misalignment.  Pieces that lie wholly past
    // the row are zero-filled here; pieces that straddle an end of the row
    // are left for the pass below, which loads their bytes one row per lane.
    constexpr int NCH = kSliceCols * (int)sizeof(T) / 16 + 1;
    // hint: 0 none; 1 the part is staged again later (keep its lines in L2);
    // 2 the part's second staging (their last read).
    auto stage = [&](int r0, int hint) {
    const int r1 = min(nr, r0 + SR);
    for (int r = r0; r < r1; ++r) {
        unsigned char *drow = tile + (r - r0) * RB;
        const char *row = a.img + (y0 + r) * a.pitch;
        if (VEC) {
            T *dst = reinterpret_cast<T *>(drow) + lane * 8;
            const T *src = reinterpret_cast<const T *>(row) + x;
            if (x + 8 <= a.cols) {
                if (sizeof(T) == 1) {
                    if (hint) cp_async8_hint(dst, src, hint == 1 ? w.pol_keep : w.pol);
                    else cp_async8(dst, src);
                } else if (hint) cp_async16_hint(dst, src, hint == 1 ? w.pol_keep : w.pol);
                else cp_async16(dst, src);
            } else if (x >= a.cols) {
#pragma unroll
                for (int k = 0; k < 8; ++k) dst[k] = (T)0;
            }
        } else {
            const int m = mis(r);
#pragma unroll
            for (int i = 0; i < (NCH + 31) / 32; ++i) {
                const int k = lane + 32 * i;                  // chunk index
                if (k >= NCH) break;
                const int64_t off = xb - m + 16 * k;          // chunk's offset in the row
                uint4 *d = reinterpret_cast<uint4 *>(drow + 16 * k);
                if (off >= 0 && off + 16 <= rowbytes) {
                    if (hint) cp_async16_hint(d, row + off, hint == 1 ? w.pol_keep : w.pol);
                    else cp_async16(d, row + off);
                }
                else if (off >= rowbytes) *d = make_uint4(0u, 0u, 0u, 0u);
            }
        }
    }
    // Pieces that straddle an end of a row: lane l fills rows l, l+32, ...,
    // so their byte loads overlap across rows instead of costing one round
    // trip per row.  They occur only in the first slice (row start) and in
    // the last two (the row end; the second-to-last slice's extra chunk
    // reaches up to 15 bytes into the last slice).
    if (s == 0 || s + 2 >= a.nsx) {
        for (int r = r0 + lane; r < r1; r += 32) {
            unsigned char *drow = tile + (r - r0) * RB;
            const char *row = a.img + (y0 + r) * a.pitch;
            if (VEC) {
                const int64_t xl = (a.cols - s * kSliceCols) & ~(int64_t)7;   // partial lane's x
                if (s == a.nsx - 1 && (a.cols & 7)) {
                    T *dst = reinterpret_cast<T *>(drow) + xl;
                    const T *src = reinterpret_cast<const T *>(row) + s * kSliceCols + xl;
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        dst[k] = (s * kSliceCols + xl + k < a.cols) ? src[k] : (T)0;
                }
            } else {
                const int64_t off0 = xb - mis(r);              // offset of chunk 0
                const int64_t kend = (rowbytes - off0) / 16;   // chunk holding the row's end
                const bool end_cut = kend < NCH && (rowbytes - off0) % 16 != 0;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int64_t k = e == 0 ? 0 : kend;
                    if (e == 0 ? off0 >= 0 : (!end_cut || (kend == 0 && off0 < 0))) continue;
                    const int64_t off = off0 + 16 * k;
                    unsigned char *d = drow + 16 * k;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int64_t o = off + j;
                        d[j] = (o >= 0 && o < rowbytes) ? (unsigned char)row[o] : 0u;
                    }
                }
            }
        }
    }
    cp_async_wait_all();
    __syncwarp();
    };

    // Reduce: column sums (8 per lane), row sums (lane keeps rows lane + 32 j).
    uint64_t cs[8], cq[8];
    uint64_t rs_s[RPL], rs_q[RPL];
    {
        uint32_t c32[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        QA cqa[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        // Rows go in groups of 32 (group j unrolled, so rs_s[j] and rs_q[j]
        // have compile-time indices and stay in registers), staged parts from
        // the bottom one up (sums do not depend on the order).
#pragma unroll
        for (int jj = 0; jj < RPL; ++jj) {
            const int j = (RPL / GPP - 1 - jj / GPP) * GPP + jj % GPP;
            const int base = j / GPP * SR;             // first row of j's staged part
            if (jj % GPP == 0) {
                if (jj) __syncwarp();                  // the previous part is read
                if (base < nr) stage(base, base ? 1 : 0);
            }
            rs_s[j] = 0;
            rs_q[j] = 0;
            const int rend = min(nr, 32 * (j + 1));
            for (int r = 32 * j; r < rend; ++r) {
                uint32_t px[8];
                px_of(tile + (r - base) * RB, r, px);
                uint32_t rs = 0;
                QA rq = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    c32[k] += px[k];
                    rs += px[k];
                    if (WQ) {
                        const QA p2 = (QA)px[k] * (QA)px[k];
                        cqa[k] += p2;
                        rq += p2;
                    }
                }
                const uint64_t row_s = warp_sum(rs);
                const uint64_t row_q = WQ ? (uint64_t)warp_sum(rq) : 0;
                if ((r & 31) == lane) { rs_s[j] = row_s; rs_q[j] = row_q; }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) { cs[k] = c32[k]; cq[k] = cqa[k]; }
    }

    // Publish, look back, publish: V (as K + V* prefix), row carries, K.
    uint64_t vs[8], vq[8], lr_s[RPL], lr_q[RPL];
    if (!lookback_tile<WQ, TH>(a, t, b, s, cs, cq, rs_s, rs_q, err, vs, vq, lr_s, lr_q))
        return false;

    // Corner lattice: the tile's first lattice row lat_y, the offset of the
    // lane's entry in that lattice row, and lat_k, the lane's lattice column
    // among its 8 columns (-1 if none).  Row and column indices are below
    // 2^31 for lattice builds, so 32-bit divisions find them (two per tile).
    uint32_t lat_y = 0;
    int64_t lat_off = 0;
    int lat_k = -1;
    if (LAT) {
        const uint32_t st = (uint32_t)a.lat_stride;
        const uint32_t qy = ((uint32_t)y0 + st) / st;         // first y >= y0 with st | y + 1
        lat_y = qy * st - 1;
        const uint32_t qx = ((uint32_t)x + st) / st;          // first column >= x likewise
        const int64_t xn = (int64_t)qx * st - 1;
        if (xn < x + kPxPerLane && xn < a.cols) lat_k = (int)(xn - x);
        lat_off = (int64_t)(qy - 1) * a.lat_ld + (qx - 1);
    }
    // Writes the lane's lattice entry of row y (values as emit_row forms them).
    auto lat_row = [&](int64_t y, uint64_t base_s, const uint32_t *lp, uint64_t base_q,
                       const QA *lq) {
        if (!LAT || (uint32_t)y != lat_y) return;
        if (lat_k >= 0) {
            uint64_t vS = 0, vQ = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k == lat_k) {
                    vS = base_s + vs[k] + lp[k];
                    if (WQ) vQ = base_q + vq[k] + (uint64_t)lq[k];
                }
            a.lat_s[lat_off] = vS;
            if (WQ) a.lat_q[lat_off] = vQ;
        }
        lat_y += (uint32_t)a.lat_stride;
        lat_off += a.lat_ld;
    };

    // Rows go in pairs: the two rows' prefix and warp-scan chains are
    // independent, which gives the scheduler two chains to interleave.
    uint32_t cp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    QA cqa[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t H_s = 0, H_q = 0;
    const int c1 = (int)(s * (kSliceCols / 16));
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        // Group j of 32 rows (unrolled: lr_s[j] has a compile-time index).
        const uint64_t ls = lr_s[j], lq = lr_q[j];
        const int base = j / GPP * SR;                 // first row of j's staged part
        if (j && j % GPP == 0 && base < nr) {          // parts below the top one
            __syncwarp();                              // the previous part is read
            stage(base, 2);
        }
        const int rend = min(nr, 32 * (j + 1));
        for (int r = 32 * j; r < rend; r += 2) {
            uint32_t pa[8], pb[8];
            px_of(tile + (r - base) * RB, r, pa);
            // Row r+1 of the part exists in the buffer (stale when r+1 == nr, unused).
            px_of(tile + (r + 1 - base) * RB, r + 1, pb);
            // r is even, so rows r and r+1 lie in the same group of 32.
            const uint64_t ha_s = H_s + __shfl_sync(kFull, ls, r & 31);
            const uint64_t hb_s = ha_s + __shfl_sync(kFull, ls, (r + 1) & 31);
            uint64_t ha_q = 0, hb_q = 0;
            if (WQ) {
                ha_q = H_q + __shfl_sync(kFull, lq, r & 31);
                hb_q = ha_q + __shfl_sync(kFull, lq, (r + 1) & 31);
            }
            H_s = hb_s;
            H_q = hb_q;
            uint32_t la[8], lb[8];
            QA qa[8], qb[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                cp[k] += pa[k];
                la[k] = cp[k] + (k ? la[k - 1] : 0u);
                cp[k] += pb[k];
                lb[k] = cp[k] + (k ? lb[k - 1] : 0u);
                if (WQ) {
                    cqa[k] += (QA)pa[k] * (QA)pa[k];
                    qa[k] = cqa[k] + (k ? qa[k - 1] : (QA)0);
                    cqa[k] += (QA)pb[k] * (QA)pb[k];
                    qb[k] = cqa[k] + (k ? qb[k - 1] : (QA)0);
                }
            }
            const uint32_t isa = warp_incl_scan(la[7], lane);
            const uint32_t isb = warp_incl_scan(lb[7], lane);
            const uint64_t base_as = ha_s + (uint64_t)(isa - la[7]);
            const uint64_t base_bs = hb_s + (uint64_t)(isb - lb[7]);
            uint64_t base_aq = 0, base_bq = 0;
            if (WQ) {
                const QA iqa = warp_incl_scan(qa[7], lane);
                const QA iqb = warp_incl_scan(qb[7], lane);
                base_aq = ha_q + (uint64_t)(iqa - qa[7]);
                base_bq = hb_q + (uint64_t)(iqb - qb[7]);
            }
            emit_row<WQ, QA>(w.ring, w.slot, w.sw, base_as, vs, la, base_aq, vq, qa, a.tmS,
                             a.tmQ, c1, (int)(y0 + r), w.pol);
            lat_row(y0 + r, base_as, la, base_aq, qa);
            if (r + 1 < nr) {
                emit_row<WQ, QA>(w.ring, w.slot, w.sw, base_bs, vs, lb, base_bq, vq, qb, a.tmS, a.tmQ,
                                 c1, (int)(y0 + r + 1), w.pol);
                lat_row(y0 + r + 1, base_bs, lb, base_bq, qb);
            }
        }
    }
    __syncwarp();     // the tile buffer is reused by the next ticket
    return true;
}

// Shared-memory bytes per warp of the single-pass tile routine (a build
// without Q keeps a ring of S rows only, so more warps fit on an SM).
template <typename T, int TH, bool WQ = true>
constexpr int onepass_warp_bytes()
{
    return (ring_bytes<WQ>() + staged_rows<T, TH, WQ>() * tile_row_bytes<T>() + 1023) / 1024 *
           1024;
}

// The warp's ring and tile inside the block's dynamic shared memory; warps
// are `stride` bytes apart (a multiple of 1024, at least the routine's need).
template <typename T, int TH, bool WQ = true>
__device__ __forceinline__ WarpRes warp_res(unsigned char *smem_raw,
                                            int stride = onepass_warp_bytes<T, TH, WQ>())
{
    static_assert(onepass_warp_bytes<T, TH, WQ>() % 1024 == 0,
                  "ring slots stay 1024-byte aligned");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    WarpRes w;
    w.ring = base + (size_t)warp * stride;
    w.tile = w.ring + ring_bytes<WQ>();
    w.slot = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) w.sw[j] = swz_off(lane, j);
    w.pol = l2_evict_first_policy();
    w.pol_keep = l2_evict_last_policy();
    return w;
}

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Tensor map of a table (rows x ld uint64, ld a multiple of 16) as a 3-D
// tensor [rows][ld/16][16] with 16 x 16 x 1 boxes in the 128-byte swizzle.
bool table_tensor_map(CUtensorMap *tm, uint64_t *T, int64_t rows, int64_t ld)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {16, (cuuint64_t)(ld / 16), (cuuint64_t)rows};
    const cuuint64_t strides[2] = {128, (cuuint64_t)ld * 8};
    const cuuint32_t box[3] = {16, 16, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, T, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

}  // namespace
}  // namespace swa
