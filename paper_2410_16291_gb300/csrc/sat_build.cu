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
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "sat_tile.cuh"
#include "swa_internal.h"

namespace swa {
namespace {

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
__global__ void __launch_bounds__(kWarps * 32, 2)
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
    constexpr int PF = 8;                              // rows in flight per warp
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
        int64_t s = 0;
        for (; s + 8 <= nsx; s += 8) {
            uint64_t vs[8], vq[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                vs[k] = c.tt_s[b * nsx + s + k];
                if (WQ) vq[k] = c.tt_q[b * nsx + s + k];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                c.tk_s[(s + k) * nby + b] = run_s;
                run_s += vs[k];
                if (WQ) { c.tk_q[(s + k) * nby + b] = run_q; run_q += vq[k]; }
            }
        }
        for (; s < nsx; ++s) {
            const uint64_t vs = c.tt_s[b * nsx + s];
            c.tk_s[s * nby + b] = run_s;
            run_s += vs;
            if (WQ) {
                const uint64_t vq = c.tt_q[b * nsx + s];
                c.tk_q[s * nby + b] = run_q;
                run_q += vq;
            }
        }
    }
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

template <typename T, bool WQ, bool VEC, int TH, int W, bool THR, bool LAT>
__global__ void __launch_bounds__(W * 32, 1)
k_onepass(OnePass a, const __grid_constant__ CUtensorMap tmS,
          const __grid_constant__ CUtensorMap tmQ)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    WarpRes w = warp_res<T, TH, WQ>(smem_raw);
    TileCtx c;
    c.img = a.img;
    c.pitch = a.pitch;
    c.rows = a.rows;
    c.cols = a.cols;
    c.nby = a.nby;
    c.nsx = a.nsx;
    c.flag_v = a.flag_v;
    c.flag_h = a.flag_h;
    c.flag_c = a.flag_c;
    c.corner = a.corner;
    c.agg_v = a.agg_v;
    c.inc_v = a.inc_v;
    c.agg_h = a.agg_h;
    c.inc_h = a.inc_h;
    c.tmS = &tmS;
    c.tmQ = &tmQ;
    c.thr = a.thr;
    c.corner_mode = a.corner_mode != 0;
    c.lat_s = a.lat_s;
    c.lat_q = a.lat_q;
    c.lat_ld = a.lat_ld;
    c.lat_stride = a.lat_stride;
    const int64_t ntiles = a.nby * a.nsx;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(a.ticket, 1u);
        t = __shfl_sync(kFull, t, 0);
        if ((int64_t)t >= ntiles || *(volatile uint32_t *)a.err) break;
        if (t == 0 && a.stall_tile0) continue;
        const uint32_t tile = a.diag ? diag_tile(t, a.nby, a.nsx) : t;
        if (!onepass_tile<T, WQ, VEC, TH, THR, LAT>(c, tile, a.err, w)) break;
    }
    cp_async_wait_all();
    if (lane == 0) bulk_wait_all();
    __syncwarp();
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

// Rows per single-pass tile: 64 for both pixel types (uint16 tiles are staged
// in two 32-row parts, see onepass_tile).
template <typename T> constexpr int onepass_rows() { return 64; }

// Warps per block of the single-pass build: as many independent warps as
// the shared memory of one SM holds (227 KB per block, 1 KB for alignment),
// at most 14 (14 x 32 threads x 144 registers fill the SM's 65,536; the
// tile routine needs up to 140).  One block runs per SM.
constexpr int kSmemPerBlock = 227 * 1024;
constexpr int kOnePassMaxWarps = 14;
template <typename T, bool WQ> constexpr int onepass_warps()
{
    return (kSmemPerBlock - 1024) / onepass_warp_bytes<T, onepass_rows<T>(), WQ>() <
                   kOnePassMaxWarps
               ? (kSmemPerBlock - 1024) / onepass_warp_bytes<T, onepass_rows<T>(), WQ>()
               : kOnePassMaxWarps;
}

template <typename T, bool WQ, bool VEC, bool THR = false, bool LAT = false>
swa_status launch_onepass(const BuildPlan &p, const char *img, uint64_t *S, uint64_t *Q,
                          char *scratch, uint32_t *err, cudaStream_t st)
{
    constexpr int TH = onepass_rows<T>();
    constexpr int W = onepass_warps<T, WQ>();
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
    a.flag_c = a.flag_h + p.nby * p.nsx;
    a.agg_v = reinterpret_cast<uint64_t *>(scratch + p.off_cs);
    a.inc_v = a.agg_v + (size_t)p.nby * p.nsx * 512;
    a.agg_h = reinterpret_cast<uint64_t *>(scratch + p.off_rs);
    a.inc_h = a.agg_h + (size_t)p.nby * p.nsx * (2 * TH + 2);
    a.corner = reinterpret_cast<uint64_t *>(scratch + p.off_bt);
    a.stall_tile0 = (test_hooks() & SWA_HOOK_STALL_TILE0) ? 1u : 0u;
    a.diag = ticket_order_diag() ? 1u : 0u;
    a.thr = p.thr;
    a.corner_mode = p.corner ? 1u : 0u;
    a.lat_s = p.lat_S;
    a.lat_q = p.lat_Q;
    a.lat_ld = p.lat_ld;
    a.lat_stride = p.lat_s;
    CUtensorMap tmS, tmQ;
    if (!table_tensor_map(&tmS, S, p.rows, p.ld) ||
        !table_tensor_map(&tmQ, WQ ? Q : S, p.rows, p.ld)) {
        set_error("cuTensorMapEncodeTiled failed for a %lldx%lld table", (long long)p.rows,
                  (long long)p.ld);
        return SWA_ECUDA;
    }
    const size_t smem = 1024 + (size_t)W * onepass_warp_bytes<T, TH, WQ>();
    auto kern = k_onepass<T, WQ, VEC, TH, W, THR, LAT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return launch_error("cudaFuncSetAttribute", e);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = p.nby * p.nsx;
    int64_t blocks = (int64_t)sms * per_sm;
    const int64_t need = (tiles + W - 1) / W;
    if (blocks > need) blocks = need;
    if ((e = cudaMemsetAsync(scratch + p.off_ticket, 0, p.off_cs - p.off_ticket, st)) !=
        cudaSuccess)
        return launch_error("cudaMemsetAsync", e);
    {
        LaunchScope ls("sat_build", st);
        kern<<<(unsigned)blocks, W * 32, smem, st>>>(a, tmS, tmQ);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return launch_error("SAT build launch failed", e);
    return SWA_OK;
}

template <typename T>
swa_status dispatch_onepass(const BuildPlan &p, const char *img, uint64_t *S, uint64_t *Q,
                            char *scratch, uint32_t *err, cudaStream_t st)
{
    if (p.count)        // indicator table: S only
        return p.vec ? launch_onepass<T, false, true, true>(p, img, S, Q, scratch, err, st)
                     : launch_onepass<T, false, false, true>(p, img, S, Q, scratch, err, st);
    if (p.with_q && p.lat_s && p.lat_S)  // S, Q and their corner lattice
        return p.vec ? launch_onepass<T, true, true, false, true>(p, img, S, Q, scratch, err, st)
                     : launch_onepass<T, true, false, false, true>(p, img, S, Q, scratch, err,
                                                                   st);
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
    p.count = (flags & kCountPlan) != 0;
    // Corner lattice stride (flag bits 8..15; single pass with Q only).  The
    // caller supplies the lattice arrays (lat_S, lat_Q, lat_ld).
    p.lat_s = (!p.twopass && !p.count && p.with_q) ? (int)((flags >> SWA_LATTICE_SHIFT) & 0xffu)
                                                   : 0;
    if (rows >= (1ll << 31) || cols >= (1ll << 31)) p.lat_s = 0;   // 32-bit lattice indices
    p.lat_rows = p.lat_s ? rows / p.lat_s : 0;
    p.lat_cols = p.lat_s ? cols / p.lat_s : 0;
    if (!p.lat_rows || !p.lat_cols) p.lat_s = 0;
    p.lat_ld = p.lat_s ? (p.lat_cols + kLdAlign - 1) / kLdAlign * kLdAlign : 0;
    p.th = p.twopass ? kTH
                     : (dtype == SWA_U8 ? onepass_rows<uint8_t>() : onepass_rows<uint16_t>());
    p.nby = (rows + p.th - 1) / p.th;
    p.nsx = (cols + kSliceCols - 1) / kSliceCols;
    p.corner = corner_mode_for(p.nsx, dtype);
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
        // ticket, then the three flag arrays (zeroed per build), then records.
        const int64_t tiles = p.nby * p.nsx;
        p.off_err = 0;
        p.off_ticket = 0;
        p.off_stat = 256;
        off = align256(256 + 3 * tiles * 4);
        p.off_cs = off;                                   // vertical records
        off = align256(off + 2 * tiles * 512 * 8);
        p.off_rs = off;                                   // horizontal records
        off = align256(off + 2 * tiles * (2 * p.th + 2) * 8);
        p.off_bt = off;                                   // corner records
        off = align256(off + tiles * 2 * 8);
    }
    p.scratch_bytes = off;
    return p;
}

// Ticket order of the single-pass builds: anti-diagonals (diag_tile) unless
// the SWA_HOOK_ROW_ORDER test hook asks for row-major order.
bool ticket_order_diag() { return !(test_hooks() & SWA_HOOK_ROW_ORDER); }

// Corner or edge mode for an image of nsx column slices.  With diagonal
// tickets edge mode measured at least as fast at every width (uint8 and
// uint16, 64 to 512 slices), so it is the default; with row-major tickets
// corner mode wins from kCornerMinSlices{U8,U16} slices.  The
// SWA_HOOK_CORNER_MODE test hook forces corner mode at every width.
bool corner_mode_for(int64_t nsx, int dtype)
{
    if (test_hooks() & SWA_HOOK_CORNER_MODE) return true;
    if (ticket_order_diag()) return false;
    return nsx >= (dtype == SWA_U8 ? kCornerMinSlicesU8 : kCornerMinSlicesU16);
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
    if (e != cudaSuccess) {
        set_error("cudaGetDevice: %s", cudaGetErrorString(e));
        return SWA_ECUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device ordinal %d beyond the no-alloc table (%d devices)", dev,
                  kNoAllocMaxDevices);
        return SWA_EINVAL;
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
