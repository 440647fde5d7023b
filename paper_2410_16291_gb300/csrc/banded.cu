// Out-of-core analysis in row bands (swa_analyze_banded).
//
// The four-corner sum of Section II-B reads the table at rows y0-1 and y1 of
// a window spanning rows y0..y1.  A table built from image row L instead of
// row 0 differs from the full table by the same column sums in both rows, so
// the difference -- the window's sum -- is unchanged for every window with
// y0 >= L (for y0 == L the upper corners are the "row -1" zeros).  Band b
// therefore serves the windows whose bottom row lies in
// [b*B, min((b+1)*B, rows)): it builds the tables of image rows [L_b, hi_b),
// where L_b is the top row of the band's first window over all queries (at
// most max(wh)-1 rows above b*B), evaluates those windows with the table row
// offset row0 = i_begin*sy - L_b, and reuses the same table buffers for the
// next band.  Device memory is bounded by about B + max(wh) rows of image
// and tables, whatever the image height.
//
// Pipelining: image bands are uploaded on one stream and results downloaded
// on another, two buffers deep, so the copies of bands b+1 and b-1 overlap
// the build and queries of band b on the caller's stream.  A band's halo rows
// (the previous band's last rows) are copied from the previous band's
// buffer on the device, so every image byte crosses the host link once.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "swa_internal.h"

namespace swa {
namespace {

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Output rows [*ib, *ie) whose windows' bottom rows lie in [lo, hi).
void rows_ending_in(int64_t rows, int64_t wh, int64_t sy, int64_t lo, int64_t hi, int64_t *ib,
                    int64_t *ie)
{
    const int64_t R = (rows - wh) / sy + 1;
    auto first = [&](int64_t y) {      // smallest i with i*sy + wh - 1 >= y
        const int64_t num = y - wh + 1;
        return std::min(num <= 0 ? 0 : (num + sy - 1) / sy, R);
    };
    *ib = first(lo);
    *ie = first(hi);
}

bool on_device(const void *p, swa_status *st)
{
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "cudaPointerGetAttributes");
        return false;
    }
    *st = SWA_OK;
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copies `rows` rows of `pitch` bytes (a multiple of 16, 16-byte aligned
// buffers) from src to dst in 16-byte words: the halo rows that a band
// shares with the previous one.  (A pitched device-to-device cudaMemcpy2D of
// the same rows measured several times slower.)
__global__ void __launch_bounds__(256) k_copy_rows(uint4 *__restrict__ dst,
                                                   const uint4 *__restrict__ src, int64_t words)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __ldg(src + i);
}

struct BandQuery {
    int k;                 // query index
    int64_t ib, ie;        // output rows of this band
};

struct Band {
    int64_t L, hi;         // image rows [L, hi) whose tables the band builds
    std::vector<BandQuery> q;
};

// Device allocations of one call, released in stream order on exit.
struct Allocs {
    cudaStream_t s;
    std::vector<std::pair<void *, int64_t>> v;
    void *get(int64_t bytes, swa_status *st)
    {
        void *p = nullptr;
        if (dev_alloc(&p, bytes, s, st) != cudaSuccess) return nullptr;
        v.push_back({p, bytes});
        return p;
    }
    ~Allocs()
    {
        for (auto &a : v) dev_free(a.first, a.second, s);
    }
};

}  // namespace
}  // namespace swa

using namespace swa;

extern "C" {

swa_status swa_band_range(int64_t rows, int64_t wh, int64_t sy, int64_t band_rows, int64_t b,
                          int64_t *i_begin, int64_t *i_end)
{
    if (rows <= 0 || wh <= 0 || wh > rows || sy <= 0 || band_rows <= 0 || b < 0 || !i_begin ||
        !i_end) {
        set_error("bad band arguments");
        return SWA_EINVAL;
    }
    const int64_t lo = b >= (rows + band_rows - 1) / band_rows ? rows : b * band_rows;
    rows_ending_in(rows, wh, sy, lo, std::min(rows, lo + std::min(band_rows, rows)), i_begin,
                   i_end);
    return SWA_OK;
}

swa_status swa_analyze_banded(const void *image, int64_t rows, int64_t cols, int64_t pitch_bytes,
                              swa_dtype dtype, const swa_window *windows, int32_t n,
                              int64_t band_rows, swa_stream stream)
{
    if (!image || rows <= 0 || cols <= 0 || (dtype != SWA_U8 && dtype != SWA_U16) ||
        pitch_bytes < cols * pixel_bytes(dtype) || !windows || n <= 0 ||
        n > SWA_MAX_WINDOWS || band_rows < 0) {
        set_error("bad banded-analysis arguments");
        return SWA_EINVAL;
    }
    const int64_t pb = pixel_bytes(dtype);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    swa_status st = SWA_OK;

    // Queries.
    bool with_q = false;
    int64_t hmax = 1;
    std::vector<int64_t> R(n), C(n);
    std::vector<char> host_out(n, 0);
    for (int k = 0; k < n; ++k) {
        const swa_window &w = windows[k];
        if (w.wh <= 0 || w.ww <= 0 || w.sy <= 0 || w.sx <= 0 || w.wh > rows || w.ww > cols) {
            set_error("window %d (%lldx%lld stride %lldx%lld) does not fit a %lldx%lld image", k,
                      (long long)w.wh, (long long)w.ww, (long long)w.sy, (long long)w.sx,
                      (long long)rows, (long long)cols);
            return SWA_EINVAL;
        }
        const uint32_t o = w.outputs;
        if (o == 0 || (o & ~7u) || w.reserved || ((o & SWA_OUT_SUM) && !w.sum) ||
            ((o & SWA_OUT_MEAN) && !w.mean) || ((o & SWA_OUT_STD) && !w.std)) {
            set_error("window %d: bad output mask or a requested output pointer is NULL", k);
            return SWA_EINVAL;
        }
        R[k] = (rows - w.wh) / w.sy + 1;
        C[k] = (cols - w.ww) / w.sx + 1;
        if (w.out_ld < C[k]) {
            set_error("window %d: out_ld %lld < output columns %lld", k, (long long)w.out_ld,
                      (long long)C[k]);
            return SWA_EINVAL;
        }
        if (o & SWA_OUT_STD) with_q = true;
        hmax = std::max(hmax, w.wh);
        const void *outs[3] = {w.sum, w.mean, w.std};
        for (int j = 0; j < 3; ++j) {
            if (!(o & (1u << j))) continue;
            const bool dev = on_device(outs[j], &st);
            if (st != SWA_OK) return st;
            if (!dev) host_out[k] = 1;
        }
    }
    const bool host_in = !on_device(image, &st);
    if (st != SWA_OK) return st;
    if (!host_in && dtype == SWA_U16 && ((uintptr_t)image % 2 || pitch_bytes % 2)) {
        set_error("uint16 images need a 2-byte aligned base and an even pitch");
        return SWA_EINVAL;
    }

    // Band height: given, or tables of about 8 GiB; then as tall as the
    // overflow guard allows for B + max(wh) - 1 table rows.
    const int64_t halo = hmax - 1;
    const int64_t ld = round_up(cols, kLdAlign);
    const int64_t row_tab = ld * 8 * (with_q ? 2 : 1);
    int64_t B = band_rows ? band_rows : std::max<int64_t>(1, ((int64_t)8 << 30) / row_tab - halo);
    B = std::min(B, rows);
    if (!fits_u64(std::min(rows, B + halo), cols, dtype, with_q)) {
        if (band_rows) {
            set_error("bands of %lld rows (+%lld halo) x %lld columns could overflow a table "
                      "entry; use fewer rows per band",
                      (long long)B, (long long)halo, (long long)cols);
            return SWA_EOVERFLOW;
        }
        int64_t lo = 0, hi = B;                 // largest B' in [1, B] that fits
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo + 1) / 2;
            if (fits_u64(std::min(rows, mid + halo), cols, dtype, with_q)) lo = mid;
            else hi = mid - 1;
        }
        if (lo < 1) {
            set_error("even a one-row band (+%lld halo rows) could overflow a table entry",
                      (long long)halo);
            return SWA_EOVERFLOW;
        }
        B = lo;
    }

    // Band plan: only bands that end at least one window.
    std::vector<Band> bands;
    int64_t max_rows = 0;
    std::vector<int64_t> max_out(n, 0);
    for (int64_t lo = 0; lo < rows; lo += B) {
        const int64_t hi = std::min(rows, lo + B);
        Band bd;
        bd.L = hi;
        bd.hi = hi;
        for (int k = 0; k < n; ++k) {
            int64_t ib, ie;
            rows_ending_in(rows, windows[k].wh, windows[k].sy, lo, hi, &ib, &ie);
            if (ib >= ie) continue;
            bd.q.push_back({k, ib, ie});
            bd.L = std::min(bd.L, ib * windows[k].sy);
            max_out[k] = std::max(max_out[k], ie - ib);
        }
        if (bd.q.empty()) continue;
        max_rows = std::max(max_rows, bd.hi - bd.L);
        bands.push_back(std::move(bd));
    }

    // Device buffers.  Host image: the whole image when it takes at most a
    // quarter of the free device memory (bands are uploaded into place, so
    // a band's halo rows are already there), else two band buffers (a band's
    // halo rows are copied from the previous band's buffer on the device).
    // Then the tables and build scratch of the tallest band and two sets of
    // output staging (host outputs).
    Allocs mem{s, {}};
    int64_t dpitch = host_in ? round_up(cols * pb, 16) : pitch_bytes;
    char *img[2] = {nullptr, nullptr};
    bool whole = false;
    if (host_in) {
        size_t free_b = 0, total_b = 0;
        cudaError_t e0 = cudaMemGetInfo(&free_b, &total_b);
        if (e0 != cudaSuccess) return cuda_fail(e0, "cudaMemGetInfo");
        whole = rows * cols * pb <= (int64_t)(free_b / 4) &&
                !(test_hooks() & SWA_HOOK_BAND_BUFFERS);
        if (whole) {
            // Rows back to back, as on the host when its rows are contiguous:
            // then every band's upload is one linear copy (a pitched copy of
            // the same rows ran ~4% slower over the host link); the build
            // reads rows at any alignment.
            dpitch = cols * pb;
            if (!(img[0] = static_cast<char *>(mem.get(dpitch * rows, &st)))) return st;
            img[1] = img[0];
        } else {
            for (int j = 0; j < 2; ++j)
                if (!(img[j] = static_cast<char *>(mem.get(dpitch * max_rows, &st)))) return st;
        }
    }
    const uint32_t flags = with_q ? SWA_WITH_SQ : 0u;
    // The plan's scratch grows with the row count; the tallest band's plan
    // (vector loads assumed possible) bounds every band's.
    const BuildPlan pmax = make_plan(max_rows, cols, dpitch, dtype, flags, nullptr);
    uint64_t *S = static_cast<uint64_t *>(mem.get(ld * max_rows * 8, &st));
    if (!S) return st;
    uint64_t *Q = nullptr;
    if (with_q && !(Q = static_cast<uint64_t *>(mem.get(ld * max_rows * 8, &st)))) return st;
    char *scratch = static_cast<char *>(mem.get(pmax.scratch_bytes, &st));
    if (!scratch) return st;
    uint32_t *err = static_cast<uint32_t *>(mem.get(256, &st));
    if (!err) return st;
    cudaError_t e;
    if ((e = cudaMemsetAsync(err, 0, 256, s)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    // staging[j][k][o]: output o of query k for buffer j
    std::vector<void *> staging(2 * n * 3, nullptr);
    for (int j = 0; j < 2; ++j)
        for (int k = 0; k < n; ++k) {
            if (!host_out[k] || !max_out[k]) continue;
            for (int o = 0; o < 3; ++o) {
                if (!(windows[k].outputs & (1u << o))) continue;
                void *p = mem.get(max_out[k] * C[k] * 8, &st);
                if (!p) return st;
                staging[(j * n + k) * 3 + o] = p;
            }
        }

    // Copy stream and the events that order it against the compute stream:
    // up[j] (band buffer j uploaded), done[j] (band results in staging j),
    // freed[j] (band buffer j no longer read: two-buffer mode), drained[j]
    // (staging j copied to the host).
    cudaStream_t cs = nullptr, ds = nullptr;       // uploads, downloads
    cudaEvent_t up[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
    cudaEvent_t freed[2] = {nullptr, nullptr}, drained[2] = {nullptr, nullptr};
    bool freed_recorded[2] = {false, false}, drained_recorded[2] = {false, false};
    auto cleanup = [&]() {
        for (cudaStream_t x : {cs, ds}) {
            if (!x) continue;
            cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
        }
        for (int j = 0; j < 2; ++j) {
            if (up[j]) cudaEventDestroy(up[j]);
            if (done[j]) cudaEventDestroy(done[j]);
            if (freed[j]) cudaEventDestroy(freed[j]);
            if (drained[j]) cudaEventDestroy(drained[j]);
        }
    };
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&ds, cudaStreamNonBlocking)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "cudaStreamCreate");
    }
    for (int j = 0; j < 2; ++j)
        if ((e = cudaEventCreateWithFlags(&up[j], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&done[j], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&freed[j], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&drained[j], cudaEventDisableTiming)) != cudaSuccess) {
            cleanup();
            return cuda_fail(e, "cudaEventCreate");
        }
    // The copy streams start after the caller's earlier work (and the memsets).
    if ((e = cudaEventRecord(up[0], s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(cs, up[0], 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(ds, up[0], 0)) != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "ordering the copy stream");
    }

    // Rows [*k0, *k1) of band t that the previous band holds (two-buffer mode).
    auto overlap = [&](size_t t, int64_t *k0, int64_t *k1) {
        *k0 = *k1 = bands[t].L;
        if (t == 0) return;
        const Band &bd = bands[t], &pv = bands[t - 1];
        const int64_t a0 = std::max(bd.L, pv.L), a1 = std::min(bd.hi, pv.hi);
        if (a1 > a0) { *k0 = a0; *k1 = a1; }
    };
    int64_t uploaded = 0;                              // whole mode: rows [0, uploaded) are there
    // Upload band t's rows that are not on the device yet (copy stream).
    auto upload = [&](size_t t) -> swa_status {
        if (!host_in) return SWA_OK;
        const int j = (int)(t & 1);
        const Band &bd = bands[t];
        char *base = whole ? img[0] : img[j] - bd.L * dpitch;   // + y * dpitch = row y
        auto from_host = [&](int64_t y0, int64_t y1) -> cudaError_t {
            if (y1 <= y0) return cudaSuccess;
            if (pitch_bytes == cols * pb && dpitch == pitch_bytes)
                return cudaMemcpyAsync(base + y0 * dpitch,
                                       static_cast<const char *>(image) + y0 * pitch_bytes,
                                       (size_t)((y1 - y0) * dpitch), cudaMemcpyHostToDevice, cs);
            return cudaMemcpy2DAsync(base + y0 * dpitch, (size_t)dpitch,
                                     static_cast<const char *>(image) + y0 * pitch_bytes,
                                     (size_t)pitch_bytes, (size_t)(cols * pb), (size_t)(y1 - y0),
                                     cudaMemcpyHostToDevice, cs);
        };
        cudaError_t e2 = cudaSuccess;
        if (whole) {
            e2 = from_host(std::max(uploaded, bd.L), bd.hi);
            uploaded = std::max(uploaded, bd.hi);
        } else {
            if (freed_recorded[j]) e2 = cudaStreamWaitEvent(cs, freed[j], 0);
            int64_t k0, k1;
            overlap(t, &k0, &k1);
            if (e2 == cudaSuccess) e2 = from_host(bd.L, k0);
            if (e2 == cudaSuccess) e2 = from_host(std::max(k1, bd.L), bd.hi);
        }
        if (e2 == cudaSuccess) e2 = cudaEventRecord(up[j], cs);
        return e2 == cudaSuccess ? SWA_OK : cuda_fail(e2, "image band upload");
    };

    if (!bands.empty() && (st = upload(0)) != SWA_OK) {
        cleanup();
        return st;
    }
    for (size_t t = 0; t < bands.size() && st == SWA_OK; ++t) {
        const int j = (int)(t & 1);
        const Band &bd = bands[t];
        const char *src = !host_in ? static_cast<const char *>(image) + bd.L * pitch_bytes
                          : whole  ? img[0] + bd.L * dpitch
                                   : img[j];
        if (host_in) {
            if ((e = cudaStreamWaitEvent(s, up[j], 0)) != cudaSuccess) {
                st = cuda_fail(e, "waiting for an upload");
                break;
            }
            if (!whole) {
                // The halo rows from the previous band's buffer, on the compute
                // stream (the previous band's work is done, so the copy has the
                // GPU to itself); then that buffer is free for the next upload.
                int64_t k0, k1;
                overlap(t, &k0, &k1);
                if (k1 > k0) {
                    const int64_t words = (k1 - k0) * dpitch / 16;
                    const unsigned grid =
                        (unsigned)std::min<int64_t>((words + 255) / 256, 8192);
                    LaunchScope ls("band_halo", s);
                    k_copy_rows<<<grid, 256, 0, s>>>(
                        reinterpret_cast<uint4 *>(img[j] + (k0 - bd.L) * dpitch),
                        reinterpret_cast<const uint4 *>(img[1 - j] +
                                                        (k0 - bands[t - 1].L) * dpitch),
                        words);
                    if ((e = cudaGetLastError()) != cudaSuccess) {
                        st = cuda_fail(e, "image band halo copy");
                        break;
                    }
                }
                if ((e = cudaEventRecord(freed[1 - j], s)) != cudaSuccess) {
                    st = cuda_fail(e, "recording a free buffer");
                    break;
                }
                freed_recorded[1 - j] = true;
            }
        }
        // The next band's upload overlaps this band's work.
        if (t + 1 < bands.size() && (st = upload(t + 1)) != SWA_OK) break;
        // Staging set j held band t-2's results until their download ended.
        if (drained_recorded[j] && (e = cudaStreamWaitEvent(s, drained[j], 0)) != cudaSuccess) {
            st = cuda_fail(e, "waiting for a download");
            break;
        }
        const BuildPlan p = make_plan(bd.hi - bd.L, cols, dpitch, dtype, flags, src);
        if ((st = launch_build(p, src, S, Q, scratch, err, s)) != SWA_OK) break;
        WinDesc d[SWA_MAX_WINDOWS];
        int m = 0;
        for (const BandQuery &bq : bd.q) {
            const swa_window &w = windows[bq.k];
            WinDesc &x = d[m++];
            memset(&x, 0, sizeof(x));
            x.wh = w.wh;
            x.ww = w.ww;
            x.sy = w.sy;
            x.sx = w.sx;
            x.R = bq.ie - bq.ib;
            x.C = C[bq.k];
            x.row0 = bq.ib * w.sy - bd.L;
            x.outputs = w.outputs;
            x.vmax = dtype == SWA_U8 ? 255u : 65535u;
            if (host_out[bq.k]) {
                x.out_ld = C[bq.k];
                x.sum = static_cast<uint64_t *>(staging[(j * n + bq.k) * 3 + 0]);
                x.mean = static_cast<double *>(staging[(j * n + bq.k) * 3 + 1]);
                x.std = static_cast<double *>(staging[(j * n + bq.k) * 3 + 2]);
            } else {
                x.out_ld = w.out_ld;
                const int64_t off = bq.ib * w.out_ld;
                x.sum = w.sum ? w.sum + off : nullptr;
                x.mean = w.mean ? w.mean + off : nullptr;
                x.std = w.std ? w.std + off : nullptr;
            }
        }
        if ((st = launch_windows(S, Q, ld, d, m, s)) != SWA_OK) break;
        if ((e = cudaEventRecord(done[j], s)) != cudaSuccess) {
            st = cuda_fail(e, "recording a band");
            break;
        }
        // Results of host-destined queries go back on the download stream.
        bool waited = false;
        for (const BandQuery &bq : bd.q) {
            if (!host_out[bq.k]) continue;
            if (!waited && (e = cudaStreamWaitEvent(ds, done[j], 0)) != cudaSuccess) {
                st = cuda_fail(e, "ordering a download");
                break;
            }
            waited = true;
            const swa_window &w = windows[bq.k];
            void *hs[3] = {w.sum, w.mean, w.std};
            for (int o = 0; o < 3 && st == SWA_OK; ++o) {
                if (!(w.outputs & (1u << o))) continue;
                char *dst = static_cast<char *>(hs[o]) + bq.ib * w.out_ld * 8;
                if ((e = cudaMemcpy2DAsync(dst, (size_t)(w.out_ld * 8),
                                           staging[(j * n + bq.k) * 3 + o], (size_t)(C[bq.k] * 8),
                                           (size_t)(C[bq.k] * 8), (size_t)(bq.ie - bq.ib),
                                           cudaMemcpyDefault, ds)) != cudaSuccess)
                    st = cuda_fail(e, "result download");
            }
            if (st != SWA_OK) break;
        }
        if (st == SWA_OK && waited) {
            if ((e = cudaEventRecord(drained[j], ds)) != cudaSuccess) {
                st = cuda_fail(e, "recording a download");
                break;
            }
            drained_recorded[j] = true;
        }
    }
    // Join the copy streams back into the caller's stream, wait, and report a
    // device-side error of any band's build.
    for (cudaStream_t x : {cs, ds}) {
        cudaEvent_t fin = x == cs ? up[0] : up[1];
        if ((e = cudaEventRecord(fin, x)) == cudaSuccess) e = cudaStreamWaitEvent(s, fin, 0);
        if (st == SWA_OK && e != cudaSuccess) st = cuda_fail(e, "joining the copy streams");
    }
    uint32_t herr = 0;
    e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st == SWA_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    if (st == SWA_OK && (herr & kErrTimeout)) {
        set_error("a look-back wait exceeded its limit");
        st = SWA_ETIMEOUT;
    }
    cleanup();
    return st;
}

}  // extern "C"
