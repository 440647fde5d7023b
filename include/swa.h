/*
 * swa.h -- C ABI of the GB300 sliding-window-analysis library (libswa.so).
 *
 * The library computes, on one CUDA device, the method of "Accelerating
 * Biological Spatial Cluster Analysis with the Parallel Integral Image
 * Technique" (arXiv 2410.16291):
 *
 *   1. the summed-area table (integral image) S of an image and the table Q of
 *      its squared pixels, as exact uint64 inclusive 2-D prefix sums
 *      (Section II-B: each entry is the sum of all pixels above and to the
 *      left of its position, the position included);
 *   2. for every valid window position, the window's sum, mean and population
 *      standard deviation, by four lookups at the window's corners
 *      (Section II-B; the 4(r*c) lookup term of Section III-B), for any
 *      number of window sizes and strides on one resident table pair
 *      (Section V names this reuse as the paper's future work).
 *
 * Conventions shared by every call:
 *  - Pointers documented as "device" must be CUDA device (or managed) memory
 *    of the current device.  swa_analyze alone also accepts host memory.
 *  - swa_stream is a cudaStream_t passed as void*; NULL is the legacy default
 *    stream.  Calls enqueue work and return without waiting unless stated.
 *  - Images are row-major, rows x cols pixels of uint8 or uint16, with a row
 *    pitch in bytes >= cols * pixel size.
 *  - Tables are row-major uint64, rows x cols, with a leading dimension
 *    (elements) reported by swa_sat_data; entries past column cols-1 in a row
 *    are padding with unspecified contents.
 *  - Window outputs are row-major R x C arrays with a caller-chosen leading
 *    dimension out_ld >= C, where R = floor((rows - wh)/sy) + 1 and
 *    C = floor((cols - ww)/sx) + 1; output (i, j) is the window whose top-left
 *    pixel is (i*sy, j*sx) (valid windows only, Section III-A's
 *    (r - w + 1)(c - w + 1) positions at stride 1).
 *  - mean = Sw / n and std = sqrt(n*Qw - Sw^2) / n, n = wh*ww, where Sw and
 *    Qw are the window's exact sums of pixels and squared pixels and the
 *    difference n*Qw - Sw^2 is exact (128-bit).  Sums are exact.
 *  - Every call returns a swa_status and never aborts.  Errors detected on
 *    the device (a look-back that waited too long) are reported by swa_sync
 *    and by later calls on the same handle.
 *  - Distinct handles may be used from different host threads; one handle
 *    must not be freed while a call on it is in flight on another thread.
 */
#ifndef SWA_H
#define SWA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct swa_sat swa_sat;     /* opaque: owns the device tables S and Q */
typedef void *swa_stream;           /* a cudaStream_t */

typedef enum { SWA_U8 = 1, SWA_U16 = 2 } swa_dtype;

typedef enum {
    SWA_OK = 0,
    SWA_EINVAL = 1,     /* bad argument: null pointer, size <= 0, window larger
                           than the image, std asked of a table built without Q */
    SWA_EOVERFLOW = 2,  /* a table entry could exceed 2^64 - 1 (see swa_build_sat) */
    SWA_ENOMEM = 3,     /* device allocation failed or the memory limit is reached */
    SWA_ECUDA = 4,      /* a CUDA runtime call or launch failed */
    SWA_ETIMEOUT = 5    /* a kernel waited too long for another block's result */
} swa_status;

/* Build flags. */
enum {
    SWA_WITH_SQ = 1u,   /* also build Q, the table of squared pixels (needed for std) */
    SWA_TWOPASS = 2u,   /* read the image twice (reduce, then scan) instead of the
                           single pass with decoupled look-back */
    SWA_COUNT = 4u,     /* reported by swa_sat_info for count tables
                           (swa_build_count_sat); not a build flag */
    SWA_LATTICE_SHIFT = 8,      /* flag bits 8..15: corner lattice stride */
    SWA_LATTICE_MASK = 0xff00u
};
/* Build flag: also keep the corner lattice of stride s (8 <= s <= 255): the
 * entries of S and Q at rows y and columns x where y + 1 and x + 1 are
 * multiples of s, packed in their own small arrays (1/s^2 of the tables).
 * Every corner of a window at strides (s, s) whose sides are multiples of s
 * lies on that lattice (top-left pixel (s*i, s*j): corner rows s*i - 1 and
 * s*i + wh - 1), so swa_window_stats* evaluates such queries from the
 * lattice, reading dense rows instead of one scattered entry per 64-byte
 * line; results are the same.  Needs SWA_WITH_SQ, not SWA_TWOPASS.  Images
 * of 2^31 rows or columns or more, or smaller than s in either direction,
 * get no lattice (swa_sat_lattice reports stride 0).  The paper's corner
 * lookup (Section II-B) on a subsampled table. */
#define SWA_LATTICE(s) ((uint32_t)(s) << SWA_LATTICE_SHIFT)

/* Window output selection. */
enum { SWA_OUT_SUM = 1u, SWA_OUT_MEAN = 2u, SWA_OUT_STD = 4u };

/* One window query: size wh x ww, strides sy, sx, the outputs wanted and
 * where they go (device pointers; those not selected may be NULL). */
typedef struct {
    int64_t wh, ww, sy, sx;
    uint32_t outputs;           /* SWA_OUT_* bits */
    uint32_t reserved;          /* must be 0 */
    uint64_t *sum;              /* R x C, leading dimension out_ld */
    double *mean;
    double *std;
    int64_t out_ld;
} swa_window;

/*
 * Build S (and Q with SWA_WITH_SQ) of a device image.  Section II-B defines
 * the table; Section III-B its O(r*c) cost, here split over the whole GPU.
 *   d_image      device pointer to rows x cols pixels of dtype, read only, in
 *                stream order; the caller may free it once the stream has
 *                passed this call.
 *   pitch_bytes  distance between rows, >= cols * pixel size; for uint16 the
 *                base address and the pitch must be even (SWA_EINVAL otherwise).
 *   flags        SWA_WITH_SQ, SWA_TWOPASS, SWA_LATTICE(s).
 *   stream       the build runs on it; the handle keeps it as its home stream.
 *   out          receives a new handle that owns S and Q (stream-ordered
 *                allocations on `stream`); set to NULL on error.
 * Returns SWA_EOVERFLOW when rows*cols*max_pixel (or rows*cols*max_pixel^2
 * with SWA_WITH_SQ) is >= 2^64, so that no entry can wrap: for uint8 this
 * never happens below 2.8e14 px; a uint16 image with Q must have fewer than
 * 4,295,098,372 px.
 */
swa_status swa_build_sat(const void *d_image, int64_t rows, int64_t cols,
                         int64_t pitch_bytes, swa_dtype dtype, uint32_t flags,
                         swa_stream stream, swa_sat **out);

/*
 * Threshold count table: the summed-area table (Section II-B) of the 0/1
 * indicator image "pixel > threshold", built in the same single pass
 * without materialising the indicator.  Window statistics on the handle
 * (swa_window_stats*) then give, per window, the number of pixels above the
 * threshold (sum), their fraction (mean) and the indicator's population std
 * (std = sqrt(p(1-p)) for fraction p) -- a count-of-positives map of the
 * kind the paper's Section V names among additional sliding window
 * analyses for cluster calling.  The indicator's squares equal its values,
 * so the handle holds one uint64 table that serves as both S and Q
 * (swa_sat_data returns the same pointer twice; swa_sat_info reports
 * SWA_WITH_SQ | SWA_COUNT).  Entries are at most rows*cols, so there is no
 * overflow bound.  Arguments and errors as swa_build_sat (no flags).
 */
swa_status swa_build_count_sat(const void *d_image, int64_t rows, int64_t cols,
                               int64_t pitch_bytes, swa_dtype dtype, uint32_t threshold,
                               swa_stream stream, swa_sat **out);

/*
 * The single-pass build of S (and Q) without any device allocation, for
 * callers that cannot allocate device memory: applications whose own memory
 * manager reserves the device's memory up front and hands out every buffer,
 * and code in callbacks or latency-bound loops where an allocation (which may
 * synchronize the device or fail) is not acceptable.  The paper has no
 * counterpart; it is an interface variant of swa_build_sat.
 *   d_image, rows, cols, pitch_bytes, dtype: as swa_build_sat.
 *   flags        0 or SWA_WITH_SQ (SWA_TWOPASS is not accepted).
 *   d_S, d_Q     caller-owned device tables of rows x ld uint64 (d_Q only with
 *                SWA_WITH_SQ), 16-byte aligned; ld >= cols and a multiple of
 *                16.  Columns cols..ld-1 of each row are scratch that the
 *                build may overwrite.
 *   d_status     optional caller-owned device word: set to 0 by the call, and
 *                bit 0 set by the kernel if a look-back wait expired (the
 *                tables are then incomplete).  May be NULL, but then such a
 *                timeout cannot be observed: the bit goes to a word inside
 *                the fixed scratch array, which the next call clears.
 * Scratch lives in one fixed 64 MiB device array inside the library, which
 * every device that loads the library holds until the process exits.  An
 * image needing more (about 100 million pixels of either type) is rejected with SWA_EINVAL and a message; use swa_build_sat.  All
 * calls share the array: calls whose builds overlap on the GPU (concurrent
 * streams, or several host threads) race and must be serialized by the
 * caller.  The first call on each device looks up the array's address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Enqueues work on `stream` and returns.
 */
swa_status swa_build_sat_noalloc(const void *d_image, int64_t rows, int64_t cols,
                                 int64_t pitch_bytes, swa_dtype dtype, uint32_t flags,
                                 uint64_t *d_S, uint64_t *d_Q, int64_t ld,
                                 uint32_t *d_status, swa_stream stream);

/* Output grid of valid windows (host only, no device work).  SWA_EINVAL when
 * a size or stride is <= 0 or the window is larger than the image. */
swa_status swa_window_shape(int64_t rows, int64_t cols, int64_t wh, int64_t ww,
                            int64_t sy, int64_t sx, int64_t *out_r, int64_t *out_c);

/*
 * Sum, mean and std of every valid window (wh x ww, strides sy, sx) by four
 * corner lookups in S (and Q for std): Section II-B's rectangle sum, the
 * paper's window sum analysis of Section II-A and the integral-image average
 * and standard deviation it mentions there.  Outputs are device arrays of
 * R x C with leading dimension out_ld (see the conventions above); SWA_OUT_STD
 * needs a handle built with SWA_WITH_SQ.  Runs on `stream` after the build.
 */
swa_status swa_window_stats(const swa_sat *sat, int64_t wh, int64_t ww,
                            int64_t sy, int64_t sx, uint32_t outputs,
                            uint64_t *d_sum, double *d_mean, double *d_std,
                            int64_t out_ld, swa_stream stream);

/*
 * Several window queries on one resident table pair in one launch (the
 * reuse of one integral image across window sizes that Section V names as
 * future work).  Same semantics as n calls of swa_window_stats; at most
 * SWA_MAX_WINDOWS per call.
 */
#define SWA_MAX_WINDOWS 64
swa_status swa_window_stats_multi(const swa_sat *sat, const swa_window *windows,
                                  int32_t n, swa_stream stream);

/* Borrowed device views of S and Q (Q is NULL without SWA_WITH_SQ) and their
 * leading dimension in elements.  Valid until swa_free; read them only in
 * stream order after the build. */
swa_status swa_sat_data(const swa_sat *sat, const uint64_t **d_S,
                        const uint64_t **d_Q, int64_t *ld);

/*
 * Check tables against their image on the device, by the recurrence that
 * defines the summed-area table (Section II-B):
 *   S[y][x] - S[y][x-1] - S[y-1][x] + S[y-1][x-1] == I[y][x]  (mod 2^64),
 * index -1 reading as 0, and Q likewise with I[y][x]^2.  Tables that pass
 * everywhere are exactly the image's tables (induction over rows, then
 * columns; no entry reaches 2^64 under the overflow bound), so this checks
 * a whole build in place, without copying tables to the host.
 *   d_image, rows, cols, pitch_bytes, dtype: the image, as for swa_build_sat.
 *   d_S, d_Q     the tables (device, leading dimension ld >= cols); d_Q may
 *                be NULL (S only).  Any table will do: a handle's
 *                (swa_sat_data), a batch's (swa_batch_tables), a caller's.
 *   d_counts     caller device array of 3 uint64, written on `stream`: [0]
 *                S entries failing, [1] Q entries failing, [2] the smallest
 *                y * cols + x of a failing entry (UINT64_MAX if none).
 * Enqueues one kernel on `stream` (after two memsets) and returns; SWA_EINVAL
 * for bad arguments.  No paper counterpart beyond the definition: a
 * self-check for tests and for users who want to validate a build.
 */
swa_status swa_verify_tables(const void *d_image, int64_t rows, int64_t cols,
                             int64_t pitch_bytes, swa_dtype dtype, const uint64_t *d_S,
                             const uint64_t *d_Q, int64_t ld, uint64_t *d_counts,
                             swa_stream stream);

/* Borrowed device views of the corner lattice (see SWA_LATTICE): lattice
 * entry (a, b) of S is S[s*(a+1) - 1][s*(b+1) - 1], for a < rows / s and
 * b < cols / s, at d_LS[a * ld + b] (d_LQ likewise for Q).  A handle built
 * without a lattice (or too small to hold one) reports stride 0 and NULL
 * views.  Any output pointer may be NULL.  Valid until swa_free. */
swa_status swa_sat_lattice(const swa_sat *sat, const uint64_t **d_LS, const uint64_t **d_LQ,
                           int64_t *rows, int64_t *cols, int64_t *ld, int32_t *stride);

/* Shape, dtype and flags of a handle. */
swa_status swa_sat_info(const swa_sat *sat, int64_t *rows, int64_t *cols,
                        int32_t *dtype, uint32_t *flags);

/* Device bytes a build of this shape holds while the handle lives (tables)
 * and transiently during the build (scratch).  Host only. */
swa_status swa_sat_bytes(int64_t rows, int64_t cols, swa_dtype dtype, uint32_t flags,
                         int64_t *table_bytes, int64_t *scratch_bytes);

/* Wait for the handle's work on its home stream and on every stream a later
 * call used, then report any error the device recorded (SWA_ETIMEOUT). */
swa_status swa_sync(const swa_sat *sat);

/* The device error word of the handle's build, read without waiting for any
 * stream (a 4-byte copy on a private non-blocking stream): SWA_ETIMEOUT if a
 * look-back wait of the build expired (the tables are then incomplete), else
 * SWA_OK.  The caller must already know that the build has finished, e.g.
 * from an event recorded after it (or after a later call on the handle's
 * stream) that has completed; before that the answer may be stale.  For
 * request loops that cannot drain a busy stream with swa_sync.  No paper
 * counterpart (error reporting of the bounded waits). */
swa_status swa_sat_status(const swa_sat *sat);

/* Release S and Q, stream-ordered on the handle's home stream after every
 * call made on the handle.  NULL is a no-op; a handle that was already freed
 * is detected by its tag and ignored. */
void swa_free(swa_sat *sat);

/*
 * One request end to end (the plain per-request path): build the tables of
 * one image, evaluate n window queries, release the tables, and wait.
 * `image` and every output pointer may be host or device memory; host data
 * is staged through device memory on `stream`.  Pinned host memory gives
 * asynchronous copies.  A host image of 256 MiB or more is analysed as by
 * swa_analyze_banded with automatic bands, so that its upload overlaps the
 * work (the results are the same).  Returns after all results are in place.
 */
swa_status swa_analyze(const void *image, int64_t rows, int64_t cols,
                       int64_t pitch_bytes, swa_dtype dtype,
                       const swa_window *windows, int32_t n, swa_stream stream);

/*
 * Out-of-core analysis in row bands: the results of swa_analyze for images
 * whose tables do not fit in device memory, or whose squared-pixel table
 * would overflow uint64 as a whole (a uint16 image of more than
 * 4,295,098,370 pixels).  It rests on the corner lookup of Section II-B: a
 * window's sum is the difference of table rows y0-1 and y1, and a table
 * built from image row L instead of row 0 changes both rows by the same
 * column sums, so every window whose top row is at or below L still comes
 * out exact.  The call walks the image in bands of `band_rows` rows: band b
 * serves the windows whose BOTTOM row lies in [b*band_rows,
 * min((b+1)*band_rows, rows)) (swa_band_range), builds the tables of image
 * rows [L_b, min((b+1)*band_rows, rows)), L_b being the top row of the
 * band's first window over all queries (at most max(wh)-1 rows above the
 * band), evaluates the band's output rows into place, and reuses the table
 * buffers for the next band.  Device memory is about (band_rows + max wh)
 * rows of image and tables plus two bands of outputs, independent of `rows`.
 * Tables are not returned.  Image bands are uploaded and results downloaded
 * on an internal second stream, overlapping the work of the neighbouring
 * band; the call returns after every result is in place.
 *
 * image, pitch_bytes, dtype, windows, n, stream: as swa_analyze (the image
 * and every output may be host or device memory; pinned host memory gives
 * full-speed copies).  band_rows: rows per band, >= 1; 0 picks it so one
 * band's tables take about 8 GiB (lowered if needed to satisfy the bound
 * below).  The overflow bound applies per band, to (band_rows + max wh - 1)
 * rows; a window's sum is exact whenever it is below 2^64 itself.
 * Errors: as swa_analyze; SWA_EOVERFLOW if the given band_rows (or, with 0,
 * even one row plus the halo) could overflow a table entry.
 * No counterpart in the paper, which keeps whole tables in memory.
 */
swa_status swa_analyze_banded(const void *image, int64_t rows, int64_t cols,
                              int64_t pitch_bytes, swa_dtype dtype,
                              const swa_window *windows, int32_t n,
                              int64_t band_rows, swa_stream stream);

/* The band partition of swa_analyze_banded for one query (host only): output
 * rows [*i_begin, *i_end) are the windows whose bottom row i*sy + wh - 1
 * lies in [b*band_rows, min((b+1)*band_rows, rows)); empty (both = R) for b
 * past the last band.  SWA_EINVAL for non-positive sizes, wh > rows or
 * b < 0. */
swa_status swa_band_range(int64_t rows, int64_t wh, int64_t sy, int64_t band_rows,
                          int64_t b, int64_t *i_begin, int64_t *i_end);

/*
 * Batched engine: many images of uneven sizes and dtypes, each with its own
 * window queries.  A run is one persistent launch that builds the tables of
 * every image (the single-pass build, all images' tiles in one work queue),
 * followed by one launch that evaluates every query of every image.  A plan
 * owns the tables of all images (and the scratch) until swa_batch_free;
 * swa_batch_run only zeroes its counters and enqueues the two kernels, so it
 * allocates nothing and can be replayed from a CUDA graph.  Both tables are
 * built for every image.
 */
typedef struct {
    const void *image;          /* device pointer, as for swa_build_sat */
    int64_t rows, cols, pitch_bytes;
    swa_dtype dtype;
    int32_t n_windows;
    const swa_window *windows;  /* host array; the output pointers are device memory */
} swa_batch_item;

typedef struct {
    int32_t u8_tile_rows;       /* rows per uint8 tile: 32 or 64 (0: 64) */
    int32_t order;              /* 0: images in the given order; 1: largest first */
    int32_t ticket_order;       /* each image's tiles: 0 along anti-diagonals; 1 row by row */
    int32_t lookback;           /* 0: edge records (the default); 1: corner records */
    int32_t warps;              /* warps per build block: 9 or 8 (0: 9) */
    int32_t interleave;         /* images whose tiles share the build's work queue at
                                 * a time, their tickets merged by each image's
                                 * progress (every image keeps its own tile order):
                                 * 1 image after image; n > 1 groups of up to n
                                 * images that run the same tile routine (pixel
                                 * type, aligned rows or not), the images ordered
                                 * by that kind first (0: 8) */
    int32_t reserved[2];        /* must be 0 */
} swa_batch_config;

typedef struct swa_batch swa_batch;

/* Validate the items, allocate tables and scratch for all of them, upload
 * the work descriptors (waits for that upload on `stream`).  cfg may be
 * NULL (all defaults); its fields change speed only, never results: they
 * are the autotuner's search space.  Out-of-range fields or non-zero
 * reserved ones give SWA_EINVAL.  SWA_EINVAL / SWA_EOVERFLOW as for swa_build_sat and
 * swa_window_stats; SWA_ENOMEM if the plan does not fit. */
swa_status swa_batch_create(const swa_batch_item *items, int32_t n,
                            const swa_batch_config *cfg, swa_stream stream,
                            swa_batch **out);

/* Enqueue one pass over the whole batch on `stream`: every table and every
 * window output is (re)written. */
swa_status swa_batch_run(swa_batch *b, swa_stream stream);

/* Wait for the plan's stream and report a device-side wait that gave up
 * (SWA_ETIMEOUT). */
swa_status swa_batch_sync(swa_batch *b);

/* Device views of item `item`'s tables (as for swa_sat_data). */
swa_status swa_batch_tables(const swa_batch *b, int32_t item, const uint64_t **d_S,
                            const uint64_t **d_Q, int64_t *ld);

/* Device bytes the plan holds (-1 for a bad plan). */
int64_t swa_batch_bytes(const swa_batch *b);

/* Release the plan (stream-ordered on the stream it was created on). */
void swa_batch_free(swa_batch *b);

/* Process-wide cap on the device bytes this library holds (tables, scratch
 * and staging) on each device; a request beyond it fails with SWA_ENOMEM.
 * A negative value removes the cap (the default). */
swa_status swa_set_memory_limit(int64_t bytes);

/* Bytes this library currently holds on the current device. */
int64_t swa_memory_in_use(void);

/* Return cached device memory above `keep_bytes` to the system. */
swa_status swa_trim(int64_t keep_bytes);

/* Static description of a status code. */
const char *swa_status_str(swa_status s);

/* Description of the last error on the calling host thread ("" if none). */
const char *swa_last_error(void);

/* Kernels this library launched in the process so far (all devices). */
int64_t swa_launch_count(void);

/* Per-kernel device time, for measurement.  Between swa_profile_begin and
 * swa_profile_end every kernel the library launches is bracketed by two CUDA
 * events on its own stream.  swa_profile_end waits for those events, writes
 * at most `max` entries (one per kernel name: launches, summed and largest
 * duration) and returns the number of distinct kernels, or -1 on a CUDA
 * error.  Profiling is process-wide; do not nest it. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
    double max_ms;
} swa_kernel_time;
swa_status swa_profile_begin(void);
int32_t swa_profile_end(swa_kernel_time *out, int32_t max);

/* Test hooks (process-wide bit set, 0 = none).  SWA_HOOK_STALL_TILE0: in the
 * single-pass build the tile taken first never publishes its carries, so
 * every other tile's bounded wait expires (after about 2 s) and swa_sync
 * returns SWA_ETIMEOUT; the kernel still exits.  For failure-path tests.
 * SWA_HOOK_BAND_BUFFERS: swa_analyze_banded stages a host image in two band
 * buffers (halo rows copied on the device) even when the whole image would
 * fit, so the mode used for images larger than a quarter of the free device
 * memory can be tested on small ones.  SWA_HOOK_CORNER_MODE: single-pass
 * builds take the corner term from the tile above-left (corner mode) instead
 * of the horizontal records (edge mode, the default).  SWA_HOOK_ROW_ORDER:
 * single-pass builds hand out tiles in row-major order instead of along
 * anti-diagonals.  The last two keep the alternative paths tested; results
 * are the same either way. */
enum { SWA_HOOK_STALL_TILE0 = 1u, SWA_HOOK_BAND_BUFFERS = 2u, SWA_HOOK_CORNER_MODE = 4u,
       SWA_HOOK_ROW_ORDER = 8u };
swa_status swa_set_test_hooks(uint32_t hooks);

/* ABI version: major * 10000 + minor * 100 + patch. */
int32_t swa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SWA_H */
