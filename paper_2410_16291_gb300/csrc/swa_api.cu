// C ABI of libswa.so: argument checks, memory, stream ordering and the
// launches of the SAT build and window kernels.  Declared in include/swa.h.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "swa_internal.h"

namespace swa {
namespace {

constexpr int kMaxDevices = 64;

std::mutex g_mu;
cudaMemPool_t g_pool[kMaxDevices];
bool g_pool_ready[kMaxDevices];
std::atomic<int64_t> g_in_use[kMaxDevices];
std::atomic<int64_t> g_limit{-1};
std::atomic<int64_t> g_launches{0};
std::atomic<uint32_t> g_hooks{0};
std::unordered_set<Handle *> g_live;
thread_local char t_err[512];

// The library's stream-ordered pool on the current device.  It keeps freed
// memory cached (release threshold = max) so a rebuild of the same size does
// not map new pages; swa_trim hands it back.
cudaError_t pool_for(int dev, cudaMemPool_t *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_pool_ready[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pool[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t thr = UINT64_MAX;
        e = cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr);
        if (e != cudaSuccess) return e;
        g_pool_ready[dev] = true;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

bool live(const swa_sat *h)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return h && g_live.count((Handle *)h) && ((const Handle *)h)->tag == kHandleTag;
}

swa_status check_window(const Handle *h, const swa_window &w, WinDesc *d)
{
    if (w.wh <= 0 || w.ww <= 0 || w.sy <= 0 || w.sx <= 0 || w.wh > h->rows ||
        w.ww > h->cols) {
        set_error("window %lldx%lld stride %lldx%lld does not fit a %lldx%lld image",
                  (long long)w.wh, (long long)w.ww, (long long)w.sy, (long long)w.sx,
                  (long long)h->rows, (long long)h->cols);
        return SWA_EINVAL;
    }
    const uint32_t o = w.outputs;
    if (o == 0 || (o & ~7u) || w.reserved) {
        set_error("bad output mask 0x%x", o);
        return SWA_EINVAL;
    }
    if (((o & SWA_OUT_SUM) && !w.sum) || ((o & SWA_OUT_MEAN) && !w.mean) ||
        ((o & SWA_OUT_STD) && !w.std)) {
        set_error("a requested output pointer is NULL");
        return SWA_EINVAL;
    }
    if ((o & SWA_OUT_STD) && !h->Q) {
        set_error("std needs a table built with SWA_WITH_SQ");
        return SWA_EINVAL;
    }
    d->wh = w.wh;
    d->ww = w.ww;
    d->sy = w.sy;
    d->sx = w.sx;
    d->R = (h->rows - w.wh) / w.sy + 1;
    d->C = (h->cols - w.ww) / w.sx + 1;
    if (w.out_ld < d->C) {
        set_error("out_ld %lld < output columns %lld", (long long)w.out_ld, (long long)d->C);
        return SWA_EINVAL;
    }
    d->out_ld = w.out_ld;
    d->row0 = 0;
    d->area = 0;
    d->outputs = o;
    d->vmax = (h->flags & SWA_COUNT) ? 1u : h->dtype == SWA_U8 ? 255u : 65535u;
    d->sum = w.sum;
    d->mean = w.mean;
    d->std = w.std;
    return SWA_OK;
}

// A query whose every corner lies on the handle's corner lattice (strides
// (s, s), sides multiples of s, windows from table row 0), rewritten as the
// stride-1 query of side wh/s x ww/s on the lattice with the true area: the
// corner rows s*i - 1 and s*i + wh - 1 are lattice rows i - 1 and
// i + wh/s - 1 (row -1 reading as 0, like the table's), and the lattice's
// output grid, lat_rows - wh/s + 1 rows, is the query's
// floor((rows - wh)/s) + 1 (likewise for columns).
bool on_lattice(const Handle *h, const WinDesc &d, WinDesc *out)
{
    const int64_t st = h->lat_s;
    if (!st || d.sy != st || d.sx != st || d.wh % st || d.ww % st || d.row0 != 0) return false;
    WinDesc x = d;
    x.wh = d.wh / st;
    x.ww = d.ww / st;
    x.sy = 1;
    x.sx = 1;
    x.area = (uint64_t)(d.wh * d.ww);
    if (h->lat_rows - x.wh + 1 != d.R || h->lat_cols - x.ww + 1 != d.C) return false;
    *out = x;
    return true;
}

// The lattice flag for a set of queries: SWA_LATTICE(s) for the stride s
// (8..255) at which the most queries have strides (s, s) and sides that are
// multiples of s, or 0 if none has.
uint32_t lattice_for(const swa_window *w, int n)
{
    int64_t best = 0;
    int best_n = 0;
    for (int k = 0; k < n; ++k) {
        const int64_t st = w[k].sy;
        if (st < 8 || st > 255 || w[k].sx != st || w[k].wh % st || w[k].ww % st) continue;
        int c = 0;
        for (int q = 0; q < n; ++q)
            c += w[q].sy == st && w[q].sx == st && w[q].wh % st == 0 && w[q].ww % st == 0;
        if (c > best_n) { best_n = c; best = st; }
    }
    return best ? SWA_LATTICE(best) : 0u;
}

// Order `s` after the build, run the windows, then join `s` back into the
// handle's home stream so that swa_free and swa_sync come after this call.
swa_status run_windows(const Handle *h, const WinDesc *d, int n, cudaStream_t s)
{
    cudaError_t e;
    Handle *hm = const_cast<Handle *>(h);
    if (s != h->stream) {
        if ((e = cudaEventRecord(hm->use_event, h->stream)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, hm->use_event, 0)) != cudaSuccess)
            return cuda_fail(e, "ordering after the build");
    }
    // Queries the corner lattice serves go in a launch of their own on it.
    WinDesc lat[SWA_MAX_WINDOWS], rest[SWA_MAX_WINDOWS];
    int nl = 0, nr = 0;
    for (int k = 0; k < n; ++k)
        if (!on_lattice(h, d[k], &lat[nl])) rest[nr++] = d[k];
        else ++nl;
    swa_status st = SWA_OK;
    if (nl) st = launch_windows(h->LS, h->LQ, h->lat_ld, lat, nl, s);
    if (st == SWA_OK && nr) st = launch_windows(h->S, h->Q, h->ld, rest, nr, s);
    if (st != SWA_OK) return st;
    if (s != h->stream) {
        if ((e = cudaEventRecord(hm->use_event, s)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(h->stream, hm->use_event, 0)) != cudaSuccess)
            return cuda_fail(e, "joining the home stream");
    }
    return SWA_OK;
}

}  // namespace

swa_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SWA_ENOMEM : SWA_ECUDA;
}

int64_t pixel_bytes(int dtype) { return dtype == SWA_U8 ? 1 : 2; }

bool fits_u64(int64_t rows, int64_t cols, int dtype, bool with_q)
{
    const unsigned __int128 n = (unsigned __int128)rows * (unsigned __int128)cols;
    const unsigned __int128 mx = dtype == SWA_U8 ? 255 : 65535;
    const unsigned __int128 lim = (unsigned __int128)1 << 64;
    if (n * mx >= lim) return false;
    if (with_q && n * mx * mx >= lim) return false;
    return true;
}

// Host images of at least this many bytes are analysed band by band.
constexpr int64_t kStreamedAnalyzeBytes = 256ll << 20;

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
}

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

uint32_t test_hooks() { return g_hooks.load(); }

namespace {
struct ProfRecord { const char *name; cudaEvent_t a, b; };
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
std::vector<ProfRecord> g_prof;            // records of the current session
std::vector<cudaEvent_t> g_prof_free;      // reusable events
cudaEvent_t prof_event()
{
    if (!g_prof_free.empty()) {
        cudaEvent_t e = g_prof_free.back();
        g_prof_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}
}  // namespace

LaunchScope::LaunchScope(const char *name, cudaStream_t s) : name_(name), s_(s), slot_(-1)
{
    count_launch();
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRecord r{name, prof_event(), prof_event()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    g_prof.push_back(r);
    slot_ = (int)g_prof.size() - 1;
}

LaunchScope::~LaunchScope()
{
    if (slot_ < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (slot_ < (int)g_prof.size()) cudaEventRecord(g_prof[slot_].b, s_);
}

cudaError_t dev_alloc(void **p, int64_t bytes, cudaStream_t s, swa_status *st)
{
    *p = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *st = cuda_fail(e, "cudaGetDevice"); return e; }
    const int64_t lim = g_limit.load();
    if (lim >= 0 && g_in_use[dev].load() + bytes > lim) {
        set_error("memory limit: %lld bytes in use + %lld requested > %lld",
                  (long long)g_in_use[dev].load(), (long long)bytes, (long long)lim);
        *st = SWA_ENOMEM;
        return cudaErrorMemoryAllocation;
    }
    cudaMemPool_t pool;
    if ((e = pool_for(dev, &pool)) != cudaSuccess) { *st = cuda_fail(e, "memory pool"); return e; }
    e = cudaMallocFromPoolAsync(p, (size_t)(bytes > 0 ? bytes : 1), pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        *st = cuda_fail(e, "device allocation");
        return e;
    }
    g_in_use[dev].fetch_add(bytes);
    *st = SWA_OK;
    return cudaSuccess;
}

void dev_free(void *p, int64_t bytes, cudaStream_t s)
{
    if (!p) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaFreeAsync(p, s);
    g_in_use[dev].fetch_sub(bytes);
}

}  // namespace swa

using namespace swa;

extern "C" {

const char *swa_status_str(swa_status s)
{
    switch (s) {
    case SWA_OK: return "ok";
    case SWA_EINVAL: return "invalid argument";
    case SWA_EOVERFLOW: return "a table entry could overflow uint64";
    case SWA_ENOMEM: return "out of device memory or over the memory limit";
    case SWA_ECUDA: return "CUDA error";
    case SWA_ETIMEOUT: return "a kernel waited too long for another block";
    }
    return "unknown status";
}

const char *swa_last_error(void) { return t_err; }

int64_t swa_launch_count(void) { return g_launches.load(); }

swa_status swa_profile_begin(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof) { g_prof_free.push_back(r.a); g_prof_free.push_back(r.b); }
    g_prof.clear();
    g_prof_on.store(true);
    return SWA_OK;
}

int32_t swa_profile_end(swa_kernel_time *out, int32_t max)
{
    g_prof_on.store(false);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::vector<swa_kernel_time> acc;
    int32_t rc = 0;
    for (auto &r : g_prof) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            rc = -1;
            continue;
        }
        size_t k = 0;
        while (k < acc.size() && strncmp(acc[k].name, r.name, sizeof(acc[k].name) - 1)) ++k;
        if (k == acc.size()) {
            swa_kernel_time t;
            memset(&t, 0, sizeof(t));
            strncpy(t.name, r.name, sizeof(t.name) - 1);
            acc.push_back(t);
        }
        acc[k].launches += 1;
        acc[k].total_ms += ms;
        if (ms > acc[k].max_ms) acc[k].max_ms = ms;
    }
    for (auto &r : g_prof) { g_prof_free.push_back(r.a); g_prof_free.push_back(r.b); }
    g_prof.clear();
    if (rc < 0) return -1;
    for (int32_t k = 0; k < (int32_t)acc.size() && k < max && out; ++k) out[k] = acc[k];
    return (int32_t)acc.size();
}

int32_t swa_version(void) { return 10000; }

swa_status swa_set_test_hooks(uint32_t hooks)
{
    if (hooks & ~(uint32_t)(SWA_HOOK_STALL_TILE0 | SWA_HOOK_BAND_BUFFERS | SWA_HOOK_CORNER_MODE |
                            SWA_HOOK_ROW_ORDER))
        return SWA_EINVAL;
    g_hooks.store(hooks);
    return SWA_OK;
}

swa_status swa_window_shape(int64_t rows, int64_t cols, int64_t wh, int64_t ww, int64_t sy,
                            int64_t sx, int64_t *out_r, int64_t *out_c)
{
    if (!out_r || !out_c || rows <= 0 || cols <= 0 || wh <= 0 || ww <= 0 || sy <= 0 ||
        sx <= 0 || wh > rows || ww > cols) {
        set_error("window %lldx%lld stride %lldx%lld does not fit a %lldx%lld image",
                  (long long)wh, (long long)ww, (long long)sy, (long long)sx, (long long)rows,
                  (long long)cols);
        return SWA_EINVAL;
    }
    *out_r = (rows - wh) / sy + 1;
    *out_c = (cols - ww) / sx + 1;
    return SWA_OK;
}

swa_status swa_sat_bytes(int64_t rows, int64_t cols, swa_dtype dtype, uint32_t flags,
                         int64_t *table_bytes, int64_t *scratch_bytes)
{
    if (rows <= 0 || cols <= 0 || (dtype != SWA_U8 && dtype != SWA_U16) ||
        (flags & ~(3u | SWA_LATTICE_MASK)))
        return SWA_EINVAL;
    BuildPlan p = make_plan(rows, cols, cols * pixel_bytes(dtype), dtype, flags, nullptr);
    if (table_bytes)
        *table_bytes = p.ld * rows * 8 * (p.with_q ? 2 : 1) + 2 * p.lat_rows * p.lat_ld * 8;
    if (scratch_bytes) *scratch_bytes = p.scratch_bytes;
    return SWA_OK;
}

swa_status swa_set_memory_limit(int64_t bytes)
{
    g_limit.store(bytes < 0 ? -1 : bytes);
    return SWA_OK;
}

int64_t swa_memory_in_use(void)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
    return g_in_use[dev].load();
}

swa_status swa_trim(int64_t keep_bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaMemPool_t pool;
    if ((e = pool_for(dev, &pool)) != cudaSuccess) return cuda_fail(e, "memory pool");
    if ((e = cudaMemPoolTrimTo(pool, (size_t)(keep_bytes > 0 ? keep_bytes : 0))) != cudaSuccess)
        return cuda_fail(e, "cudaMemPoolTrimTo");
    return SWA_OK;
}

}  // extern "C"

namespace {

// Builds a handle: the tables of the image (count == false; flags as given)
// or the table of its indicator "pixel > thr" (count == true; S only, also
// serving as Q since the indicator's squares are the indicator).
swa_status build_handle(const void *d_image, int64_t rows, int64_t cols, int64_t pitch_bytes,
                        swa_dtype dtype, uint32_t flags, bool count, uint32_t thr,
                        swa_stream stream, swa_sat **out)
{
    if (out) *out = nullptr;
    if (!d_image || !out || rows <= 0 || cols <= 0 || (dtype != SWA_U8 && dtype != SWA_U16) ||
        (flags & ~(3u | SWA_LATTICE_MASK)) || pitch_bytes < cols * pixel_bytes(dtype)) {
        set_error("bad build arguments");
        return SWA_EINVAL;
    }
    if (const uint32_t ls = (flags & SWA_LATTICE_MASK) >> SWA_LATTICE_SHIFT) {
        if (ls < 8 || !(flags & SWA_WITH_SQ) || (flags & SWA_TWOPASS) || count) {
            set_error("a corner lattice needs a stride of 8 to 255, SWA_WITH_SQ and the "
                      "single-pass build");
            return SWA_EINVAL;
        }
    }
    if (dtype == SWA_U16 && ((uintptr_t)d_image % 2 || pitch_bytes % 2)) {
        set_error("uint16 images need a 2-byte aligned base and an even pitch");
        return SWA_EINVAL;
    }
    // A count table has entries <= rows*cols; otherwise the a3 bound.
    const bool wq = !count && (flags & SWA_WITH_SQ);
    if (!count && !fits_u64(rows, cols, dtype, wq)) {
        set_error("%lldx%lld %s image: a table entry could exceed 2^64-1", (long long)rows,
                  (long long)cols, dtype == SWA_U8 ? "uint8" : "uint16");
        return SWA_EOVERFLOW;
    }
    BuildPlan p = make_plan(rows, cols, pitch_bytes, dtype, count ? kCountPlan : flags, d_image);
    p.thr = thr;
    const int64_t tbytes = p.ld * rows * 8;
    const int64_t lbytes = p.lat_rows * p.lat_ld * 8;     // one lattice array
    const int64_t lim = g_limit.load();
    if (lim == 0 || (lim > 0 && tbytes * (wq ? 2 : 1) + 2 * lbytes + p.scratch_bytes > lim)) {
        set_error("memory limit %lld bytes < %lld needed", (long long)lim,
                  (long long)(tbytes * (wq ? 2 : 1) + 2 * lbytes + p.scratch_bytes));
        return SWA_ENOMEM;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Handle *h = new (std::nothrow) Handle();
    if (!h) return SWA_ENOMEM;
    h->tag = kHandleTag;
    h->rows = rows;
    h->cols = cols;
    h->ld = p.ld;
    h->dtype = dtype;
    h->flags = count ? (SWA_WITH_SQ | SWA_COUNT) : flags;
    h->stream = s;
    h->table_bytes = tbytes * (wq ? 2 : 1) + 2 * lbytes;
    cudaError_t e = cudaGetDevice(&h->device);
    swa_status st = SWA_OK;
    void *mem = nullptr;
    char *scratch = nullptr;
    if (e != cudaSuccess) { st = cuda_fail(e, "cudaGetDevice"); goto fail; }
    if ((e = cudaEventCreateWithFlags(&h->use_event, cudaEventDisableTiming)) != cudaSuccess) {
        st = cuda_fail(e, "cudaEventCreate");
        goto fail;
    }
    if (dev_alloc(&mem, tbytes, s, &st) != cudaSuccess) goto fail;
    h->S = static_cast<uint64_t *>(mem);
    if (wq) {
        if (dev_alloc(&mem, tbytes, s, &st) != cudaSuccess) goto fail;
        h->Q = static_cast<uint64_t *>(mem);
    }
    if (count) h->Q = h->S;
    if (lbytes) {
        if (dev_alloc(&mem, lbytes, s, &st) != cudaSuccess) goto fail;
        h->LS = static_cast<uint64_t *>(mem);
        if (dev_alloc(&mem, lbytes, s, &st) != cudaSuccess) goto fail;
        h->LQ = static_cast<uint64_t *>(mem);
        h->lat_s = p.lat_s;
        h->lat_rows = p.lat_rows;
        h->lat_cols = p.lat_cols;
        h->lat_ld = p.lat_ld;
        p.lat_S = h->LS;
        p.lat_Q = h->LQ;
    }
    if (dev_alloc(&mem, 256, s, &st) != cudaSuccess) goto fail;
    h->d_err = static_cast<uint32_t *>(mem);
    if ((e = cudaMemsetAsync(h->d_err, 0, 256, s)) != cudaSuccess) {
        st = cuda_fail(e, "cudaMemsetAsync");
        goto fail;
    }
    if (dev_alloc(&mem, p.scratch_bytes, s, &st) != cudaSuccess) goto fail;
    scratch = static_cast<char *>(mem);
    st = launch_build(p, d_image, h->S, h->Q, scratch, h->d_err, s);
    dev_free(scratch, p.scratch_bytes, s);
    scratch = nullptr;
    if (st != SWA_OK) goto fail;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_live.insert(h);
    }
    *out = reinterpret_cast<swa_sat *>(h);
    return SWA_OK;
fail:
    if (scratch) dev_free(scratch, p.scratch_bytes, s);
    if (h->S) dev_free(h->S, tbytes, s);
    if (h->Q && h->Q != h->S) dev_free(h->Q, tbytes, s);
    if (h->LS) dev_free(h->LS, lbytes, s);
    if (h->LQ) dev_free(h->LQ, lbytes, s);
    if (h->d_err) dev_free(h->d_err, 256, s);
    if (h->use_event) cudaEventDestroy(h->use_event);
    h->tag = kFreedTag;
    delete h;
    return st;
}

}  // namespace

extern "C" {

swa_status swa_build_sat(const void *d_image, int64_t rows, int64_t cols, int64_t pitch_bytes,
                         swa_dtype dtype, uint32_t flags, swa_stream stream, swa_sat **out)
{
    return build_handle(d_image, rows, cols, pitch_bytes, dtype, flags, false, 0u, stream, out);
}

swa_status swa_build_count_sat(const void *d_image, int64_t rows, int64_t cols,
                               int64_t pitch_bytes, swa_dtype dtype, uint32_t threshold,
                               swa_stream stream, swa_sat **out)
{
    return build_handle(d_image, rows, cols, pitch_bytes, dtype, 0u, true, threshold, stream,
                        out);
}

swa_status swa_window_stats(const swa_sat *sat, int64_t wh, int64_t ww, int64_t sy, int64_t sx,
                            uint32_t outputs, uint64_t *d_sum, double *d_mean, double *d_std,
                            int64_t out_ld, swa_stream stream)
{
    swa_window w;
    memset(&w, 0, sizeof(w));
    w.wh = wh;
    w.ww = ww;
    w.sy = sy;
    w.sx = sx;
    w.outputs = outputs;
    w.sum = d_sum;
    w.mean = d_mean;
    w.std = d_std;
    w.out_ld = out_ld;
    return swa_window_stats_multi(sat, &w, 1, stream);
}

swa_status swa_window_stats_multi(const swa_sat *sat, const swa_window *windows, int32_t n,
                                  swa_stream stream)
{
    if (!live(sat)) { set_error("not a live handle"); return SWA_EINVAL; }
    if (!windows || n <= 0 || n > SWA_MAX_WINDOWS) { set_error("bad window list"); return SWA_EINVAL; }
    const Handle *h = reinterpret_cast<const Handle *>(sat);
    WinDesc d[SWA_MAX_WINDOWS];
    for (int k = 0; k < n; ++k) {
        swa_status st = check_window(h, windows[k], &d[k]);
        if (st != SWA_OK) return st;
    }
    return run_windows(h, d, n, static_cast<cudaStream_t>(stream));
}

swa_status swa_sat_data(const swa_sat *sat, const uint64_t **d_S, const uint64_t **d_Q,
                        int64_t *ld)
{
    if (!live(sat)) return SWA_EINVAL;
    const Handle *h = reinterpret_cast<const Handle *>(sat);
    if (d_S) *d_S = h->S;
    if (d_Q) *d_Q = h->Q;
    if (ld) *ld = h->ld;
    return SWA_OK;
}

swa_status swa_sat_lattice(const swa_sat *sat, const uint64_t **d_LS, const uint64_t **d_LQ,
                           int64_t *rows, int64_t *cols, int64_t *ld, int32_t *stride)
{
    if (!live(sat)) return SWA_EINVAL;
    const Handle *h = reinterpret_cast<const Handle *>(sat);
    if (d_LS) *d_LS = h->LS;
    if (d_LQ) *d_LQ = h->LQ;
    if (rows) *rows = h->lat_rows;
    if (cols) *cols = h->lat_cols;
    if (ld) *ld = h->lat_ld;
    if (stride) *stride = h->lat_s;
    return SWA_OK;
}

swa_status swa_sat_info(const swa_sat *sat, int64_t *rows, int64_t *cols, int32_t *dtype,
                        uint32_t *flags)
{
    if (!live(sat)) return SWA_EINVAL;
    const Handle *h = reinterpret_cast<const Handle *>(sat);
    if (rows) *rows = h->rows;
    if (cols) *cols = h->cols;
    if (dtype) *dtype = h->dtype;
    if (flags) *flags = h->flags;
    return SWA_OK;
}

swa_status swa_sync(const swa_sat *sat)
{
    if (!live(sat)) return SWA_EINVAL;
    const Handle *h = reinterpret_cast<const Handle *>(sat);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    uint32_t err = 0;
    if ((e = cudaMemcpy(&err, h->d_err, sizeof(err), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading the device error word");
    if (err & kErrTimeout) {
        set_error("a look-back wait exceeded its limit");
        return SWA_ETIMEOUT;
    }
    return SWA_OK;
}

swa_status swa_sat_status(const swa_sat *sat)
{
    if (!live(sat)) return SWA_EINVAL;
    const Handle *h = reinterpret_cast<const Handle *>(sat);
    // A private non-blocking stream per thread, so that the read neither
    // waits for nor joins any other stream's work (the legacy default stream
    // would wait for every blocking stream).
    static thread_local cudaStream_t qs[kMaxDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond the library's table of %d", dev, kMaxDevices);
        return SWA_EINVAL;
    }
    if (!qs[dev] && (e = cudaStreamCreateWithFlags(&qs[dev], cudaStreamNonBlocking)) !=
                        cudaSuccess)
        return cuda_fail(e, "cudaStreamCreateWithFlags");
    uint32_t err = 0;
    if ((e = cudaMemcpyAsync(&err, h->d_err, sizeof(err), cudaMemcpyDeviceToHost, qs[dev])) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(qs[dev])) != cudaSuccess)
        return cuda_fail(e, "reading the device error word");
    if (err & kErrTimeout) {
        set_error("a look-back wait exceeded its limit");
        return SWA_ETIMEOUT;
    }
    return SWA_OK;
}

void swa_free(swa_sat *sat)
{
    if (!sat) return;
    Handle *h = reinterpret_cast<Handle *>(sat);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_live.count(h) || h->tag != kHandleTag) return;
        g_live.erase(h);
    }
    const int64_t tb = h->ld * h->rows * 8;
    dev_free(h->S, tb, h->stream);
    if (h->Q && h->Q != h->S) dev_free(h->Q, tb, h->stream);
    if (h->LS) dev_free(h->LS, h->lat_rows * h->lat_ld * 8, h->stream);
    if (h->LQ) dev_free(h->LQ, h->lat_rows * h->lat_ld * 8, h->stream);
    dev_free(h->d_err, 256, h->stream);
    cudaEventDestroy(h->use_event);
    h->tag = kFreedTag;
    delete h;
}

swa_status swa_analyze(const void *image, int64_t rows, int64_t cols, int64_t pitch_bytes,
                       swa_dtype dtype, const swa_window *windows, int32_t n, swa_stream stream)
{
    if (!image || rows <= 0 || cols <= 0 || (dtype != SWA_U8 && dtype != SWA_U16) ||
        pitch_bytes < cols * pixel_bytes(dtype) || !windows || n <= 0 ||
        n > SWA_MAX_WINDOWS) {
        set_error("bad analyze arguments");
        return SWA_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t flags = 0;
    for (int k = 0; k < n; ++k)
        if (windows[k].outputs & SWA_OUT_STD) flags |= SWA_WITH_SQ;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, image);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
    const bool host_in = attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged;
    const int64_t pb = pixel_bytes(dtype);
    // A large host image goes through the banded path: its upload then
    // overlaps the builds and queries band by band (same results: the
    // window sums are exact on band tables, see swa_analyze_banded).
    if (host_in && rows * cols * pb >= kStreamedAnalyzeBytes)
        return swa_analyze_banded(image, rows, cols, pitch_bytes, dtype, windows, n, 0, stream);
    const void *d_img = image;
    void *stage = nullptr;
    int64_t stage_bytes = 0, dpitch = pitch_bytes;
    swa_status st = SWA_OK;
    swa_sat *sat = nullptr;
    struct Tmp { void *p; int64_t bytes; };
    std::vector<Tmp> tmps;
    std::vector<swa_window> dw(windows, windows + n);

    if (host_in) {
        dpitch = (cols * pb + 15) / 16 * 16;
        stage_bytes = dpitch * rows;
        if (dev_alloc(&stage, stage_bytes, s, &st) != cudaSuccess) return st;
        if ((e = cudaMemcpy2DAsync(stage, (size_t)dpitch, image, (size_t)pitch_bytes,
                                   (size_t)(cols * pb), (size_t)rows, cudaMemcpyHostToDevice,
                                   s)) != cudaSuccess) {
            st = cuda_fail(e, "image upload");
            goto done;
        }
        d_img = stage;
    }
    // A window with any output in host memory gets device buffers for all of
    // its outputs (leading dimension C); results are copied back at the end.
    for (int k = 0; k < n; ++k) {
        int64_t R, C;
        if (swa_window_shape(rows, cols, dw[k].wh, dw[k].ww, dw[k].sy, dw[k].sx, &R, &C) !=
            SWA_OK) {
            st = SWA_EINVAL;
            set_error("window %d does not fit", k);
            goto done;
        }
        void **slots[3] = {(void **)&dw[k].sum, (void **)&dw[k].mean, (void **)&dw[k].std};
        bool any_host = false;
        for (int o = 0; o < 3; ++o) {
            if (!(dw[k].outputs & (1u << o)) || !*slots[o]) continue;
            cudaPointerAttributes a2;
            if ((e = cudaPointerGetAttributes(&a2, *slots[o])) != cudaSuccess) {
                st = cuda_fail(e, "cudaPointerGetAttributes");
                goto done;
            }
            if (a2.type != cudaMemoryTypeDevice && a2.type != cudaMemoryTypeManaged)
                any_host = true;
        }
        if (!any_host) continue;
        for (int o = 0; o < 3; ++o) {
            if (!(dw[k].outputs & (1u << o)) || !*slots[o]) continue;
            void *p = nullptr;
            if (dev_alloc(&p, R * C * 8, s, &st) != cudaSuccess) goto done;
            tmps.push_back({p, R * C * 8});
            *slots[o] = p;
        }
        dw[k].out_ld = C;
    }
    // Queries that all their corners' lattice serves read it instead of the
    // tables (the lattice needs Q, which std already asks for).
    if (flags & SWA_WITH_SQ) flags |= lattice_for(windows, n);
    if ((st = swa_build_sat(d_img, rows, cols, dpitch, dtype, flags, stream, &sat)) != SWA_OK)
        goto done;
    if ((st = swa_window_stats_multi(sat, dw.data(), n, stream)) != SWA_OK) goto done;
    // Copy host-destined outputs back.
    for (int k = 0; k < n; ++k) {
        int64_t R, C;
        swa_window_shape(rows, cols, dw[k].wh, dw[k].ww, dw[k].sy, dw[k].sx, &R, &C);
        void *hs[3] = {windows[k].sum, windows[k].mean, windows[k].std};
        void *ds[3] = {dw[k].sum, dw[k].mean, dw[k].std};
        for (int o = 0; o < 3; ++o) {
            if (!(dw[k].outputs & (1u << o)) || hs[o] == ds[o]) continue;
            if ((e = cudaMemcpy2DAsync(hs[o], (size_t)(windows[k].out_ld * 8), ds[o],
                                       (size_t)(C * 8), (size_t)(C * 8), (size_t)R,
                                       cudaMemcpyDefault, s)) != cudaSuccess) {
                st = cuda_fail(e, "result download");
                goto done;
            }
        }
    }
done:
    if (sat) {
        swa_status s2 = swa_sync(sat);
        if (st == SWA_OK) st = s2;
        swa_free(sat);
    }
    for (auto &t : tmps) dev_free(t.p, t.bytes, s);
    if (stage) dev_free(stage, stage_bytes, s);
    e = cudaStreamSynchronize(s);
    if (st == SWA_OK && e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    return st;
}

}  // extern "C"
