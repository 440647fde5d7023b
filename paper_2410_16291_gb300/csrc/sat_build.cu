// Summed-area table build on the GPU (Section II-B's table; Section III-B's
// O(r*c)/p parallel cost).
//
// Decomposition.  The image is cut into warp tiles of TH rows x 256 columns
// (one 256-column "slice" per warp, 8 pixels per lane).  For a tile whose
// top-left pixel is (y0, xs0), every entry of the inclusive table splits into
// three carries and one tile-local part:
//
//   S[y][x] = K + H[y] + V*[x] + lp[y][x]
//     K     = sum of I over rows < y0, columns < xs0 (the tiles above-left),
//     H[y]  = sum of I over rows y0..y, columns < xs0 (left row sums, summed
//             down the tile),
//     V*[x] = sum over columns xs0..x of V[j], V[j] = sum of I over rows < y0
//             in column j (the column sums above the tile),
//     lp    = the tile's own 2-D inclusive prefix sum.
//
// The default build is a single pass with decoupled look-back (k_onepass
// below).  The two-pass build obtains the carries by reading the image twice:
// a reduce kernel writes per-tile column sums, row sums and totals; a carry
// kernel turns them into exclusive scans; the scan kernel re-reads the image
// and writes S (and Q, the same for I^2).  Table entries are exact uint64;
// tile-local parts use 32-bit integers where their bounds allow.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "swa_internal.h"

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
#pragma unroll
        for (int i = 0; i < (int)sizeof(T) * 2; ++i) r.w[i] = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t v = (x + k < cols) ? (uint32_t)__ldg(row + x + k) : 0u;
            if (sizeof(T) == 1) r.w[k >> 2] |= v << (8 * (k & 3));
            else r.w[(k >> 1) % (sizeof(T) * 2)] |= v << (16 * (k & 1));
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

struct Carries {
    uint64_t *cs_s, *cs_q;   // [nby][ld]  column sums per band -> V (exclusive over bands)
    uint64_t *rs_s, *rs_q;   // [nsx][rows] row sums per slice -> LR (exclusive over slices)
    uint64_t *tt_s, *tt_q;   // [nby][nsx] tile totals; then [nsx][nby] exclusive over slices
    uint64_t *tk_s, *tk_q;   // [nsx][nby] row-scanned tile totals (transposed)
};

// ---------------------------------------------------------------- reduce --
// One warp per tile: column sums (per lane, 8 columns), row sums (warp
// reductions, kept by lane (row mod 32) and stored 32 rows at a time) and the
// tile total.
template <typename T, bool WQ, bool VEC, int TH>
__global__ void __launch_bounds__(kWarps * 32)
k_reduce(const char *__restrict__ img, int64_t pitch, int64_t rows, int64_t cols,
         int64_t ld, int64_t nby, int64_t nsx, Carries c)
{
    using QA = typename QAcc<T>::type;
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (t >= nby * nsx) return;
    const int64_t b = t / nsx, s = t % nsx;
    const int64_t y0 = b * TH, y1 = min(rows, y0 + TH);
    const int64_t x = s * kSliceCols + lane * kPxPerLane;

    uint32_t cs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    QA cq[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t keep_s = 0, keep_q = 0, tot_s = 0, tot_q = 0;
    constexpr int PF = 8;
    for (int64_t ya = y0; ya < y1; ya += PF) {
      Raw8<T> raw[PF];
#pragma unroll
      for (int i = 0; i < PF; ++i)
          if (ya + i < y1) raw[i] = load_raw8<T, VEC>(img, pitch, ya + i, x, cols);
#pragma unroll
      for (int i = 0; i < PF; ++i) {
        const int64_t y = ya + i;
        if (y >= y1) break;
        uint32_t px[8];
        unpack8<T>(raw[i], px);
        uint32_t rs = 0;
        QA rq = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cs[k] += px[k];
            rs += px[k];
            if (WQ) {
                QA p2 = (QA)px[k] * (QA)px[k];
                cq[k] += p2;
                rq += p2;
            }
        }
        uint64_t row_s = warp_sum(rs);
        uint64_t row_q = WQ ? (uint64_t)warp_sum(rq) : 0;
        const int r = (int)(y - y0) & 31;
        if (lane == r) { keep_s = row_s; keep_q = row_q; }
        tot_s += row_s;
        tot_q += row_q;
        if (r == 31 || y == y1 - 1) {
            const int64_t yy = y - r + lane;
            if (yy <= y) {
                c.rs_s[s * rows + yy] = keep_s;
                if (WQ) c.rs_q[s * rows + yy] = keep_q;
            }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (x + k < cols) {
            c.cs_s[b * ld + x + k] = cs[k];
            if (WQ) c.cs_q[b * ld + x + k] = cq[k];
        }
    }
    if (lane == 0) {
        c.tt_s[b * nsx + s] = tot_s;
        if (WQ) c.tt_q[b * nsx + s] = tot_q;
    }
}

// ---------------------------------------------------------------- carries --
// Three independent groups of blocks:
//   A: per column, exclusive scan of the band column sums down the bands (V);
//   B: per row, exclusive scan of the slice row sums along the slices (LR);
//   C: per band, exclusive scan of the tile totals along the slices, written
//      transposed so the scan kernel can sum it down the bands coalesced.
// Loads are batched 8 at a time ahead of the dependent running sum.
template <bool WQ>
__device__ __forceinline__ void excl_scan_strided(uint64_t *__restrict__ a,
                                                  uint64_t *__restrict__ q,
                                                  int64_t n, int64_t stride)
{
    uint64_t run_s = 0, run_q = 0;
    int64_t i = 0;
    for (; i + 8 <= n; i += 8) {
        uint64_t vs[8], vq[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            vs[k] = a[(i + k) * stride];
            if (WQ) vq[k] = q[(i + k) * stride];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a[(i + k) * stride] = run_s;
            run_s += vs[k];
            if (WQ) { q[(i + k) * stride] = run_q; run_q += vq[k]; }
        }
    }
    for (; i < n; ++i) {
        uint64_t vs = a[i * stride];
        a[i * stride] = run_s;
        run_s += vs;
        if (WQ) { uint64_t vq = q[i * stride]; q[i * stride] = run_q; run_q += vq; }
    }
}

template <bool WQ>
__global__ void __launch_bounds__(256)
k_carry(int64_t rows, int64_t cols, int64_t ld, int64_t nby, int64_t nsx,
        int64_t nA, int64_t nB, Carries c)
{
    const int64_t blk = blockIdx.x;
    if (blk < nA) {
        const int64_t x = blk * 256 + threadIdx.x;
        if (x < cols) excl_scan_strided<WQ>(c.cs_s + x, c.cs_q + x, nby, ld);
    } else if (blk < nA + nB) {
        const int64_t y = (blk - nA) * 256 + threadIdx.x;
        if (y < rows) excl_scan_strided<WQ>(c.rs_s + y, c.rs_q + y, nsx, rows);
    } else {
        const int64_t b = (blk - nA - nB) * 256 + threadIdx.x;
        if (b >= nby) return;
        uint64_t run_s = 0, run_q = 0;
        for (int64_t s = 0; s < nsx; ++s) {
            uint64_t vs = c.tt_s[b * nsx + s];
            c.tk_s[s * nby + b] = run_s;
            run_s += vs;
            if (WQ) {
                uint64_t vq = c.tt_q[b * nsx + s];
                c.tk_q[s * nby + b] = run_q;
                run_q += vq;
            }
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

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
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
    unsigned char *rs = ring + slot * (2 * kRowBytes);
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

// ------------------------------------------------------------------ scan --
// Two-pass build, second pass: one warp per tile; assemble the carries, then
// walk the tile's rows keeping per-column running sums, scan each row across
// the warp and write S (and Q) through the ring.
template <typename T, bool WQ, bool VEC, int TH>
__global__ void __launch_bounds__(kWarps * 32)
k_scan(const char *__restrict__ img, int64_t pitch, int64_t rows, int64_t cols,
       int64_t ld, int64_t nby, int64_t nsx, Carries c,
       const __grid_constant__ CUtensorMap tmS, const __grid_constant__ CUtensorMap tmQ)
{
    using QA = typename QAcc<T>::type;
    constexpr int RING_BYTES = kRing * 2 * kRowBytes;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    unsigned char *ring = base + (size_t)warp * RING_BYTES;
    const int64_t t = (int64_t)blockIdx.x * kWarps + warp;
    if (t >= nby * nsx) return;
    const int64_t b = t / nsx, s = t % nsx;
    const int64_t y0 = b * TH, y1 = min(rows, y0 + TH);
    const int64_t x = s * kSliceCols + lane * kPxPerLane;
    const uint64_t pol = l2_evict_first_policy();

    // K: exclusive 2-D sum of tile totals above-left = sum over bands < b of
    // the (already slice-scanned) totals.
    uint64_t K_s = 0, K_q = 0;
    for (int64_t bb = lane; bb < b; bb += 32) {
        K_s += c.tk_s[s * nby + bb];
        if (WQ) K_q += c.tk_q[s * nby + bb];
    }
    K_s = warp_sum(K_s);
    if (WQ) K_q = warp_sum(K_q);

    // V*: inclusive scan of the column sums above the tile across the slice.
    uint64_t vs[8], vq[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const bool in = x + k < cols;
        vs[k] = in ? c.cs_s[b * ld + x + k] : 0;
        vq[k] = (WQ && in) ? c.cs_q[b * ld + x + k] : 0;
    }
#pragma unroll
    for (int k = 1; k < 8; ++k) { vs[k] += vs[k - 1]; if (WQ) vq[k] += vq[k - 1]; }
    {
        uint64_t is = warp_incl_scan(vs[7], lane), es = is - vs[7];
        uint64_t iq = WQ ? warp_incl_scan(vq[7], lane) : 0, eq = iq - vq[7];
#pragma unroll
        for (int k = 0; k < 8; ++k) { vs[k] += es + K_s; if (WQ) vq[k] += eq + K_q; }
    }

    int sw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) sw[j] = swz_off(lane, j);
    const int c1 = (int)(s * (kSliceCols / 16));
    int slot = 0;
    uint32_t cp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    QA cq[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t H_s = 0, H_q = 0, lr_s = 0, lr_q = 0;
    Raw8<T> pa = load_raw8<T, VEC>(img, pitch, y0, x, cols), pb = pa;
    if (y0 + 1 < y1) pb = load_raw8<T, VEC>(img, pitch, y0 + 1, x, cols);
    for (int64_t y = y0; y < y1; ++y) {
        uint32_t px[8];
        unpack8<T>(pa, px);
        pa = pb;
        if (y + 2 < y1) pb = load_raw8<T, VEC>(img, pitch, y + 2, x, cols);
        const int r = (int)(y - y0) & 31;
        if (r == 0) {
            const int64_t yy = y + lane;
            lr_s = yy < y1 ? c.rs_s[s * rows + yy] : 0;
            lr_q = (WQ && yy < y1) ? c.rs_q[s * rows + yy] : 0;
        }
        H_s += __shfl_sync(kFull, lr_s, r);
        if (WQ) H_q += __shfl_sync(kFull, lr_q, r);

        uint32_t lp[8];
        QA lq[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            cp[k] += px[k];
            lp[k] = cp[k] + (k ? lp[k - 1] : 0u);
            if (WQ) {
                cq[k] += (QA)px[k] * (QA)px[k];
                lq[k] = cq[k] + (k ? lq[k - 1] : (QA)0);
            }
        }
        const uint32_t is = warp_incl_scan(lp[7], lane);
        const uint64_t base_s = H_s + (uint64_t)(is - lp[7]);
        uint64_t base_q = 0;
        if (WQ) {
            const QA iq = warp_incl_scan(lq[7], lane);
            base_q = H_q + (uint64_t)(iq - lq[7]);
        }
        emit_row<WQ, QA>(ring, slot, sw, base_s, vs, lp, base_q, vq, lq, &tmS, &tmQ, c1, (int)y,
                         pol);
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
}

// ------------------------------------------------------------- one pass --
// Single-pass build with decoupled look-back.  Warps take tiles in row-major
// ticket order (an atomic counter, so every smaller ticket belongs to a warp
// that is already running).  A warp stages its tile in shared memory, reduces
// it, and publishes two aggregates:
//   vertical   (per tile column slice): the tile's 256 column sums;
//   horizontal (per tile band): the tile's row sums and the total of the
//              column sums above it (the corner term K of the tiles to its
//              right).
// It then looks back up its slice for the column carries V (summing
// aggregates until a tile with an inclusive prefix is found), publishes its
// own inclusive column prefix together with its horizontal aggregate, looks
// back left along its band for the row carries LR and K the same way,
// publishes its inclusive row prefix, and finally scans the staged tile and
// writes S and Q through the ring.  Every wait is bounded by a time limit; on
// expiry the warp sets the error word and all warps stop.
constexpr uint32_t kAgg = 1u, kInc = 2u;
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per wait
constexpr int kOpWarps = 8;                        // warps per block (independent tiles)

struct OnePass {
    const char *img;
    int64_t pitch, rows, cols, ld, nby, nsx;
    uint32_t *ticket, *err;
    uint32_t *flag_v, *flag_h;        // [tiles]
    uint64_t *agg_v, *inc_v;          // [tiles][2][256]
    uint64_t *agg_h, *inc_h;          // [tiles][2*TH + 2]
    uint32_t stall_tile0;             // test hook: ticket 0 publishes nothing
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

// Wait until *flag is non-zero in every lane; returns it, or 0 if the error
// word is set (by this wait timing out or by another warp).
__device__ __noinline__ uint32_t wait_flag(const uint32_t *flag, uint32_t *err)
{
    uint32_t v = ld_acquire(flag);
    if (__all_sync(kFull, v != 0)) return __shfl_sync(kFull, v, 0);
    const uint64_t t0 = global_ns();
    unsigned ns = 64;
    for (;;) {
        __nanosleep(ns);
        if (ns < 2048) ns <<= 1;
        v = ld_acquire(flag);
        if (__all_sync(kFull, v != 0)) return __shfl_sync(kFull, v, 0);
        if (*(volatile uint32_t *)err) return 0;
        if (global_ns() - t0 > kWaitLimitNs) {
            if ((threadIdx.x & 31) == 0) atomicOr(err, kErrTimeout);
            __syncwarp();
            return 0;
        }
    }
}

// Every lane has written its part of the records; make them visible, then
// raise up to two flags (a fence followed by relaxed stores is a release).
__device__ __forceinline__ void publish(uint32_t *f1, uint32_t v1, uint32_t *f2 = nullptr,
                                        uint32_t v2 = 0)
{
    __threadfence();
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

__device__ __forceinline__ void cp_async16(void *smem, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(g)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <typename T, bool WQ, bool VEC, int TH>
__global__ void __launch_bounds__(kOpWarps * 32, 1)
k_onepass(OnePass a, const __grid_constant__ CUtensorMap tmS,
          const __grid_constant__ CUtensorMap tmQ)
{
    using QA = typename QAcc<T>::type;
    static_assert(TH == 32 || TH == 64, "rows per tile");
    constexpr int RPL = TH / 32;                       // rows each lane keeps
    constexpr int HREC = 2 * TH + 2;                   // horizontal record length
    constexpr int TILE_BYTES = TH * kSliceCols * (int)sizeof(T);
    constexpr int RING_BYTES = kRing * 2 * kRowBytes;
    constexpr int WARP_BYTES = RING_BYTES + TILE_BYTES;
    static_assert(WARP_BYTES % 1024 == 0, "ring slots stay 1024-byte aligned");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *base = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    unsigned char *ring = base + (size_t)warp * WARP_BYTES;     // [kRing][S, Q][2 KB]
    T *tile = reinterpret_cast<T *>(ring + RING_BYTES);
    const int64_t ntiles = a.nby * a.nsx;
    const uint64_t pol = l2_evict_first_policy();
    int sw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) sw[j] = swz_off(lane, j);
    int slot = 0;

    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1u);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= ntiles || *(volatile uint32_t *)a.err) break;
        if (t == 0 && a.stall_tile0) continue;
        const int64_t b = t / a.nsx, s = t % a.nsx;
        const int64_t y0 = b * TH;
        const int nr = (int)min((int64_t)TH, a.rows - y0);
        const int64_t x = s * kSliceCols + lane * kPxPerLane;

        // Stage the tile (rows 0..nr-1; columns past the image read as 0).
        for (int r = 0; r < nr; ++r) {
            T *dst = tile + r * kSliceCols + lane * 8;
            const T *src = reinterpret_cast<const T *>(a.img + (y0 + r) * a.pitch) + x;
            if (VEC && x + 8 <= a.cols) {
                if (sizeof(T) == 1) cp_async8(dst, src);
                else cp_async16(dst, src);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) dst[k] = (x + k < a.cols) ? src[k] : (T)0;
            }
        }
        cp_async_wait_all();
        __syncwarp();

        // Reduce: column sums (8 per lane), row sums (lane keeps rows lane + 32 j).
        uint64_t cs[8], cq[8];
        uint64_t rs_s[RPL], rs_q[RPL];
        {
            uint32_t c32[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            QA cqa[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < RPL; ++j) { rs_s[j] = 0; rs_q[j] = 0; }
            for (int r = 0; r < nr; ++r) {
                uint32_t px[8];
                smem8<T>(tile + r * kSliceCols, lane, px);
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
                if ((r & 31) == lane) { rs_s[r >> 5] = row_s; rs_q[r >> 5] = row_q; }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) { cs[k] = c32[k]; cq[k] = cqa[k]; }
        }

        // Vertical: publish the column sums, look back up the slice for V.
        uint64_t vs[8] = {0, 0, 0, 0, 0, 0, 0, 0}, vq[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        uint64_t *inv = a.inc_v + (size_t)t * 512 + lane * 8;
        if (b > 0) {
            uint64_t *ag = a.agg_v + (size_t)t * 512 + lane * 8;
#pragma unroll
            for (int k = 0; k < 8; k += 2) {
                *reinterpret_cast<ulonglong2 *>(ag + k) = make_ulonglong2(cs[k], cs[k + 1]);
                if (WQ)
                    *reinterpret_cast<ulonglong2 *>(ag + 256 + k) =
                        make_ulonglong2(cq[k], cq[k + 1]);
            }
            publish(a.flag_v + t, kAgg);
            bool ok = true;
            for (int64_t bb = b - 1; bb >= 0; --bb) {
                const int64_t u = bb * a.nsx + s;
                const uint32_t f = wait_flag(a.flag_v + u, a.err);
                if (!f) { ok = false; break; }
                const uint64_t *src =
                    (f == kInc ? a.inc_v : a.agg_v) + (size_t)u * 512 + lane * 8;
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                    const ulonglong2 w = __ldcg(reinterpret_cast<const ulonglong2 *>(src + k));
                    vs[k] += w.x;
                    vs[k + 1] += w.y;
                    if (WQ) {
                        const ulonglong2 z =
                            __ldcg(reinterpret_cast<const ulonglong2 *>(src + 256 + k));
                        vq[k] += z.x;
                        vq[k + 1] += z.y;
                    }
                }
                if (f == kInc) break;
            }
            if (!ok) break;
        }
#pragma unroll
        for (int k = 0; k < 8; k += 2) {
            *reinterpret_cast<ulonglong2 *>(inv + k) =
                make_ulonglong2(vs[k] + cs[k], vs[k + 1] + cs[k + 1]);
            if (WQ)
                *reinterpret_cast<ulonglong2 *>(inv + 256 + k) =
                    make_ulonglong2(vq[k] + cq[k], vq[k + 1] + cq[k + 1]);
        }

        // Horizontal record = (row sums, total of V over the slice); published
        // with the inclusive vertical record (as inclusive when s == 0).
        uint64_t vt_s = 0, vt_q = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) { vt_s += vs[k]; vt_q += vq[k]; }
        vt_s = warp_sum(vt_s);
        if (WQ) vt_q = warp_sum(vt_q);
        uint64_t lr_s[RPL], lr_q[RPL], K_s = 0, K_q = 0;
#pragma unroll
        for (int j = 0; j < RPL; ++j) { lr_s[j] = 0; lr_q[j] = 0; }
        {
            uint64_t *rec = (s > 0 ? a.agg_h : a.inc_h) + (size_t)t * HREC;
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                rec[lane + 32 * j] = rs_s[j];
                if (WQ) rec[TH + lane + 32 * j] = rs_q[j];
            }
            if (lane == 0) { rec[2 * TH] = vt_s; rec[2 * TH + 1] = vt_q; }
            publish(a.flag_v + t, kInc, a.flag_h + t, s > 0 ? kAgg : kInc);
        }
        if (s > 0) {
            bool ok = true;
            for (int64_t ss = s - 1; ss >= 0; --ss) {
                const int64_t u = b * a.nsx + ss;
                const uint32_t f = wait_flag(a.flag_h + u, a.err);
                if (!f) { ok = false; break; }
                const uint64_t *src = (f == kInc ? a.inc_h : a.agg_h) + (size_t)u * HREC;
#pragma unroll
                for (int j = 0; j < RPL; ++j) {
                    lr_s[j] += __ldcg(src + lane + 32 * j);
                    if (WQ) lr_q[j] += __ldcg(src + TH + lane + 32 * j);
                }
                K_s += __ldcg(src + 2 * TH);
                if (WQ) K_q += __ldcg(src + 2 * TH + 1);
                if (f == kInc) break;
            }
            if (!ok) break;
            uint64_t *in = a.inc_h + (size_t)t * HREC;
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                in[lane + 32 * j] = lr_s[j] + rs_s[j];
                if (WQ) in[TH + lane + 32 * j] = lr_q[j] + rs_q[j];
            }
            if (lane == 0) { in[2 * TH] = K_s + vt_s; in[2 * TH + 1] = K_q + vt_q; }
            publish(a.flag_h + t, kInc);
        }

        // Scan the staged tile: S = K + H[y] + V*[x] + lp.  vs/vq become K + V*.
#pragma unroll
        for (int k = 1; k < 8; ++k) { vs[k] += vs[k - 1]; if (WQ) vq[k] += vq[k - 1]; }
        {
            const uint64_t is = warp_incl_scan(vs[7], lane), es = is - vs[7];
            const uint64_t iq = WQ ? warp_incl_scan(vq[7], lane) : 0, eq = iq - vq[7];
#pragma unroll
            for (int k = 0; k < 8; ++k) { vs[k] += es + K_s; if (WQ) vq[k] += eq + K_q; }
        }
        uint32_t cp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        QA cqa[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        uint64_t H_s = 0, H_q = 0;
        const int c1 = (int)(s * (kSliceCols / 16));
        for (int r = 0; r < nr; ++r) {
            uint32_t px[8];
            smem8<T>(tile + r * kSliceCols, lane, px);
            uint64_t ls = lr_s[0], lq = lr_q[0];
#pragma unroll
            for (int j = 1; j < RPL; ++j)
                if ((r >> 5) == j) { ls = lr_s[j]; lq = lr_q[j]; }
            H_s += __shfl_sync(kFull, ls, r & 31);
            if (WQ) H_q += __shfl_sync(kFull, lq, r & 31);
            uint32_t lp[8];
            QA lq8[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                cp[k] += px[k];
                lp[k] = cp[k] + (k ? lp[k - 1] : 0u);
                if (WQ) {
                    cqa[k] += (QA)px[k] * (QA)px[k];
                    lq8[k] = cqa[k] + (k ? lq8[k - 1] : (QA)0);
                }
            }
            const uint32_t is = warp_incl_scan(lp[7], lane);
            const uint64_t base_s = H_s + (uint64_t)(is - lp[7]);
            uint64_t base_q = 0;
            if (WQ) {
                const QA iq = warp_incl_scan(lq8[7], lane);
                base_q = H_q + (uint64_t)(iq - lq8[7]);
            }
            emit_row<WQ, QA>(ring, slot, sw, base_s, vs, lp, base_q, vq, lq8, &tmS, &tmQ, c1,
                             (int)(y0 + r), pol);
        }
        __syncwarp();     // the tile buffer is reused by the next ticket
    }
    cp_async_wait_all();
    if (lane == 0) bulk_wait_all();
    __syncwarp();
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

// ------------------------------------------------------------ launchers --
constexpr int kTH = 128;   // two-pass rows per tile (u8 tile-local Q sums stay below 2^32)

swa_status launch_error(const char *what, cudaError_t e)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SWA_ECUDA;
}

template <typename T, bool WQ, bool VEC>
swa_status launch_twopass(const BuildPlan &p, const char *img, uint64_t *S, uint64_t *Q,
                          char *scratch, cudaStream_t st)
{
    Carries c;
    const int64_t nb = p.nby, ns = p.nsx;
    c.cs_s = reinterpret_cast<uint64_t *>(scratch + p.off_cs);
    c.cs_q = c.cs_s + nb * p.ld;
    c.rs_s = reinterpret_cast<uint64_t *>(scratch + p.off_rs);
    c.rs_q = c.rs_s + ns * p.rows;
    c.tt_s = reinterpret_cast<uint64_t *>(scratch + p.off_bt);
    c.tt_q = c.tt_s + nb * ns;
    c.tk_s = c.tt_q + nb * ns;
    c.tk_q = c.tk_s + nb * ns;
    const int64_t tiles = nb * ns;
    const int64_t blocks = (tiles + kWarps - 1) / kWarps;
    CUtensorMap tmS, tmQ;
    if (!table_tensor_map(&tmS, S, p.rows, p.ld) ||
        !table_tensor_map(&tmQ, WQ ? Q : S, p.rows, p.ld)) {
        set_error("cuTensorMapEncodeTiled failed for a %lldx%lld table", (long long)p.rows,
                  (long long)p.ld);
        return SWA_ECUDA;
    }
    const size_t smem = 1024 + (size_t)kWarps * kRing * 2 * kRowBytes;
    auto scan = k_scan<T, WQ, VEC, kTH>;
    cudaError_t e = cudaFuncSetAttribute(scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return launch_error("cudaFuncSetAttribute", e);
    {
        LaunchScope ls("sat_reduce", st);
        k_reduce<T, WQ, VEC, kTH><<<(unsigned)blocks, kWarps * 32, 0, st>>>(
            img, p.pitch, p.rows, p.cols, p.ld, nb, ns, c);
    }
    const int64_t nA = (p.cols + 255) / 256, nB = (p.rows + 255) / 256, nC = (nb + 255) / 256;
    {
        LaunchScope ls("sat_carry", st);
        k_carry<WQ><<<(unsigned)(nA + nB + nC), 256, 0, st>>>(p.rows, p.cols, p.ld, nb, ns,
                                                              nA, nB, c);
    }
    {
        LaunchScope ls("sat_scan", st);
        scan<<<(unsigned)blocks, kWarps * 32, smem, st>>>(img, p.pitch, p.rows, p.cols, p.ld,
                                                           nb, ns, c, tmS, tmQ);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return launch_error("SAT build launch failed", e);
    return SWA_OK;
}

template <typename T>
swa_status dispatch_twopass(const BuildPlan &p, const char *img, uint64_t *S, uint64_t *Q,
                            char *scratch, cudaStream_t st)
{
    if (p.with_q)
        return p.vec ? launch_twopass<T, true, true>(p, img, S, Q, scratch, st)
                     : launch_twopass<T, true, false>(p, img, S, Q, scratch, st);
    return p.vec ? launch_twopass<T, false, true>(p, img, S, Q, scratch, st)
                 : launch_twopass<T, false, false>(p, img, S, Q, scratch, st);
}

template <typename T> constexpr int onepass_rows() { return sizeof(T) == 1 ? 64 : 32; }

template <typename T, bool WQ, bool VEC>
swa_status launch_onepass(const BuildPlan &p, const char *img, uint64_t *S, uint64_t *Q,
                          char *scratch, uint32_t *err, cudaStream_t st)
{
    constexpr int TH = onepass_rows<T>();
    OnePass a;
    a.img = img;
    a.pitch = p.pitch;
    a.rows = p.rows;
    a.cols = p.cols;
    a.ld = p.ld;
    a.nby = p.nby;
    a.nsx = p.nsx;
    a.err = err;
    a.ticket = reinterpret_cast<uint32_t *>(scratch + p.off_ticket);
    a.flag_v = reinterpret_cast<uint32_t *>(scratch + p.off_stat);
    a.flag_h = a.flag_v + p.nby * p.nsx;
    a.agg_v = reinterpret_cast<uint64_t *>(scratch + p.off_cs);
    a.inc_v = a.agg_v + (size_t)p.nby * p.nsx * 512;
    a.agg_h = reinterpret_cast<uint64_t *>(scratch + p.off_rs);
    a.inc_h = a.agg_h + (size_t)p.nby * p.nsx * (2 * TH + 2);
    a.stall_tile0 = (test_hooks() & SWA_HOOK_STALL_TILE0) ? 1u : 0u;
    CUtensorMap tmS, tmQ;
    if (!table_tensor_map(&tmS, S, p.rows, p.ld) ||
        !table_tensor_map(&tmQ, WQ ? Q : S, p.rows, p.ld)) {
        set_error("cuTensorMapEncodeTiled failed for a %lldx%lld table", (long long)p.rows,
                  (long long)p.ld);
        return SWA_ECUDA;
    }
    const size_t smem =
        1024 + (size_t)kOpWarps * (kRing * 2 * kRowBytes + TH * kSliceCols * sizeof(T));
    auto kern = k_onepass<T, WQ, VEC, TH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return launch_error("cudaFuncSetAttribute", e);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kOpWarps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = p.nby * p.nsx;
    int64_t blocks = (int64_t)sms * per_sm;
    const int64_t need = (tiles + kOpWarps - 1) / kOpWarps;
    if (blocks > need) blocks = need;
    if ((e = cudaMemsetAsync(scratch + p.off_ticket, 0, p.off_cs - p.off_ticket, st)) !=
        cudaSuccess)
        return launch_error("cudaMemsetAsync", e);
    {
        LaunchScope ls("sat_build", st);
        kern<<<(unsigned)blocks, kOpWarps * 32, smem, st>>>(a, tmS, tmQ);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return launch_error("SAT build launch failed", e);
    return SWA_OK;
}

template <typename T>
swa_status dispatch_onepass(const BuildPlan &p, const char *img, uint64_t *S, uint64_t *Q,
                            char *scratch, uint32_t *err, cudaStream_t st)
{
    if (p.with_q)
        return p.vec ? launch_onepass<T, true, true>(p, img, S, Q, scratch, err, st)
                     : launch_onepass<T, true, false>(p, img, S, Q, scratch, err, st);
    return p.vec ? launch_onepass<T, false, true>(p, img, S, Q, scratch, err, st)
                 : launch_onepass<T, false, false>(p, img, S, Q, scratch, err, st);
}

int64_t align256(int64_t v) { return (v + 255) & ~(int64_t)255; }

}  // namespace

BuildPlan make_plan(int64_t rows, int64_t cols, int64_t pitch, int dtype, uint32_t flags,
                    const void *image)
{
    BuildPlan p{};
    p.rows = rows;
    p.cols = cols;
    p.pitch = pitch;
    p.dtype = dtype;
    p.with_q = (flags & SWA_WITH_SQ) != 0;
    p.twopass = (flags & SWA_TWOPASS) != 0;
    p.ld = (cols + kLdAlign - 1) / kLdAlign * kLdAlign;
    // 8-pixel vector loads (8 bytes for uint8, 16 for uint16) need the base
    // address and the pitch aligned to the vector size.
    const int64_t vbytes = dtype == SWA_U8 ? 8 : 16;
    p.vec = ((uintptr_t)image % vbytes == 0) && (pitch % vbytes == 0);
    p.th = p.twopass ? kTH : (dtype == SWA_U8 ? onepass_rows<uint8_t>()
                                              : onepass_rows<uint16_t>());
    p.nby = (rows + p.th - 1) / p.th;
    p.nsx = (cols + kSliceCols - 1) / kSliceCols;
    int64_t off = 0;
    if (p.twopass) {
        p.off_err = off;
        off = align256(off + 16);
        p.off_cs = off;
        off = align256(off + 2 * p.nby * p.ld * 8);
        p.off_rs = off;
        off = align256(off + 2 * p.nsx * rows * 8);
        p.off_bt = off;
        off = align256(off + 4 * p.nby * p.nsx * 8);
        p.off_stat = off;
        p.off_ticket = off;
    } else {
        // ticket, then the two flag arrays (zeroed per build), then records.
        const int64_t tiles = p.nby * p.nsx;
        p.off_err = 0;
        p.off_ticket = 0;
        p.off_stat = 256;
        off = align256(256 + 2 * tiles * 4);
        p.off_cs = off;                                   // vertical records
        off = align256(off + 2 * tiles * 512 * 8);
        p.off_rs = off;                                   // horizontal records
        off = align256(off + 2 * tiles * (2 * p.th + 2) * 8);
        p.off_bt = off;
    }
    p.scratch_bytes = off;
    return p;
}

swa_status launch_build(const BuildPlan &p, const void *image, uint64_t *S, uint64_t *Q,
                        char *scratch, uint32_t *err, cudaStream_t st)
{
    const char *img = static_cast<const char *>(image);
    if (p.twopass) {
        if (p.dtype == SWA_U8) return dispatch_twopass<uint8_t>(p, img, S, Q, scratch, st);
        return dispatch_twopass<uint16_t>(p, img, S, Q, scratch, st);
    }
    if (p.dtype == SWA_U8) return dispatch_onepass<uint8_t>(p, img, S, Q, scratch, err, st);
    return dispatch_onepass<uint16_t>(p, img, S, Q, scratch, err, st);
}

}  // namespace swa

// ------------------------------------------------ allocation-free build --
// swa_build_sat_noalloc runs the single-pass build with its scratch (tile
// tickets, flags and look-back records) in this fixed device array instead of
// memory allocated per call.  The array exists once per device that loads the
// library and stays allocated until the process exits.  All calls share it,
// so calls whose builds overlap on the GPU race; each call clears the parts
// that must start at zero (the ticket and the flags) before its kernel runs.
namespace swa {
namespace {
constexpr int64_t kNoAllocScratchBytes = 64ll << 20;          // 64 MiB
constexpr int64_t kNoAllocStatusOffset = kNoAllocScratchBytes - 256;
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
char *g_noalloc_ptr[kNoAllocMaxDevices];
}  // namespace
}  // namespace swa

static __device__ __align__(256) unsigned char g_noalloc_scratch[swa::kNoAllocScratchBytes];

extern "C" swa_status swa_build_sat_noalloc(const void *d_image, int64_t rows, int64_t cols,
                                           int64_t pitch_bytes, swa_dtype dtype,
                                           uint32_t flags, uint64_t *d_S, uint64_t *d_Q,
                                           int64_t ld, uint32_t *d_status, swa_stream stream)
{
    using namespace swa;
    const int64_t pb = dtype == SWA_U16 ? 2 : 1;
    const bool wq = (flags & SWA_WITH_SQ) != 0;
    if (!d_image || !d_S || (wq && !d_Q) || rows <= 0 || cols <= 0 ||
        (dtype != SWA_U8 && dtype != SWA_U16) || (flags & ~(uint32_t)SWA_WITH_SQ) ||
        pitch_bytes < cols * pb || ld < cols || (ld % 16) || ((uintptr_t)d_S & 15) ||
        (wq && ((uintptr_t)d_Q & 15)) || ((uintptr_t)d_status & 3)) {
        set_error("bad arguments to swa_build_sat_noalloc");
        return SWA_EINVAL;
    }
    if (dtype == SWA_U16 && ((uintptr_t)d_image % 2 || pitch_bytes % 2)) {
        set_error("uint16 images need a 2-byte aligned base and an even pitch");
        return SWA_EINVAL;
    }
    {
        const unsigned __int128 n = (unsigned __int128)rows * (unsigned __int128)cols;
        const unsigned __int128 mx = dtype == SWA_U8 ? 255 : 65535;
        const unsigned __int128 lim = (unsigned __int128)1 << 64;
        if (n * mx >= lim || (wq && n * mx * mx >= lim)) {
            set_error("a table entry could exceed 2^64-1");
            return SWA_EOVERFLOW;
        }
    }
    BuildPlan p = make_plan(rows, cols, pitch_bytes, dtype, flags, d_image);
    p.ld = ld;
    if (p.scratch_bytes > kNoAllocStatusOffset) {
        set_error("swa_build_sat_noalloc: a %lldx%lld image needs %lld bytes of scratch; the "
                  "fixed array holds %lld (use swa_build_sat)",
                  (long long)rows, (long long)cols, (long long)p.scratch_bytes,
                  (long long)kNoAllocStatusOffset);
        return SWA_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("cudaGetDevice: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    char *scratch = nullptr;
    {
        // First call on this device: look up the array's device address
        // (host code cannot use the symbol itself as a pointer).
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                set_error("cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return SWA_ECUDA;
            }
            g_noalloc_ptr[dev] = static_cast<char *>(ptr);
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t *status = d_status ? d_status
                                : reinterpret_cast<uint32_t *>(scratch + kNoAllocStatusOffset);
    if ((e = cudaMemsetAsync(status, 0, sizeof(uint32_t), st)) != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    const char *img = static_cast<const char *>(d_image);
    if (dtype == SWA_U8) return dispatch_onepass<uint8_t>(p, img, d_S, d_Q, scratch, status, st);
    return dispatch_onepass<uint16_t>(p, img, d_S, d_Q, scratch, status, st);
}
