/*
 * CPU oracle for parallel-integral-image sliding window analysis
 * (arXiv 2410.16291).  TEST INFRASTRUCTURE ONLY: the tests, the smoke check
 * and the benchmark's CPU-baseline leg may call this code; the library's
 * compute path never does.  It shares no source with the CUDA kernels.
 *
 * Plain, serial, unblocked C.  Every result is an exact integer except the
 * final mean and standard deviation, which are formed from exact integer
 * moments and rounded by IEEE double operations.
 *
 * Definitions followed (paper sections):
 *  - Sliding window analysis (Section II-A): a fixed-size window is moved over
 *    the image; at each position an analysis (sum; also average and standard
 *    deviation) is applied to the window and stored in a new array.
 *  - Valid windows only, anchored at the top-left corner: the naive cost
 *    O((r - w + 1)(c - w + 1) w^2) of Section III-A counts exactly the window
 *    positions that fit inside the image at stride 1.  With strides (sy, sx),
 *    output (i, j) is the window whose top-left pixel is (i*sy, j*sx), and the
 *    grid has floor((r - wh)/sy) + 1 rows and floor((c - ww)/sx) + 1 columns.
 *  - Integral image (Section II-B): each table entry is the sum of all pixels
 *    above and to the left of its position, read inclusively:
 *    S[y][x] = sum_{i <= y, j <= x} I[i][j]; Q is the same table of I^2.
 *    A rectangle's sum is the four-corner combination (Section II-B, and the
 *    4(r*c) lookup term of Section III-B), an index of -1 reading as 0.
 *  - DP-naive-SWA (Section IV-A) is only described as reducing additions by
 *    dynamic programming; it is read here as separable moving sums.
 *  - mean = (double)Sw / (double)n, and the population standard deviation
 *    std = sqrt((double)D) / (double)n with D = n*Qw - Sw^2 computed exactly
 *    in 128-bit integers, n = wh*ww.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

#define DT_U8 1
#define DT_U16 2

/* Return codes. */
#define OK 0
#define E_ARG -1
#define E_MEM -2
#define E_OVERFLOW -3

static inline uint64_t pix(const void *img, int64_t pitch, int dtype,
                           int64_t y, int64_t x)
{
    const uint8_t *row = (const uint8_t *)img + y * pitch;
    if (dtype == DT_U8) return row[x];
    uint16_t v;
    memcpy(&v, row + 2 * x, 2);
    return v;
}

static int args_ok(const void *img, int64_t rows, int64_t cols,
                   int64_t pitch, int dtype)
{
    if (!img || rows <= 0 || cols <= 0) return 0;
    if (dtype != DT_U8 && dtype != DT_U16) return 0;
    if (pitch < cols * (dtype == DT_U8 ? 1 : 2)) return 0;
    return 1;
}

/* Whether every entry of S (and of Q when with_sq) fits in uint64: the
 * largest entry is the total, at most rows*cols*max and rows*cols*max^2. */
int oracle_fits_u64(int64_t rows, int64_t cols, int dtype, int with_sq)
{
    if (rows <= 0 || cols <= 0) return 0;
    u128 maxv = dtype == DT_U8 ? 255 : 65535;
    u128 n = (u128)rows * (u128)cols;
    u128 lim = (u128)1 << 64;
    if (n * maxv >= lim) return 0;
    if (with_sq && n * maxv * maxv >= lim) return 0;
    return 1;
}

/* Output grid of valid windows; 0 when the window does not fit. */
int oracle_window_shape(int64_t rows, int64_t cols, int64_t wh, int64_t ww,
                        int64_t sy, int64_t sx, int64_t *R, int64_t *C)
{
    if (rows <= 0 || cols <= 0 || wh <= 0 || ww <= 0 || sy <= 0 || sx <= 0)
        return E_ARG;
    if (wh > rows || ww > cols) return E_ARG;
    *R = (rows - wh) / sy + 1;
    *C = (cols - ww) / sx + 1;
    return OK;
}

/* Round-to-nearest-even conversion of an exact 128-bit integer, done by the
 * host compiler's own integer-to-double conversion. */
double oracle_u128_to_double(uint64_t hi, uint64_t lo)
{
    u128 v = ((u128)hi << 64) | lo;
    return (double)v;
}

/* mean = Sw / n and population std = sqrt(n*Qw - Sw^2) / n. */
void oracle_stats_from_moments(uint64_t n, uint64_t Sw, uint64_t Qw,
                               double *mean, double *std)
{
    if (mean) *mean = (double)Sw / (double)n;
    if (std) {
        u128 D = (u128)n * (u128)Qw - (u128)Sw * (u128)Sw;
        *std = sqrt((double)D) / (double)n;
    }
}

/*
 * Summed-area tables, by the definition's recurrence taken row by row:
 * a running sum along the row plus the previous row of the table.
 * S and Q are rows x cols, row-major with leading dimension ld_out.
 * Q may be NULL.
 */
int oracle_sat(const void *img, int64_t rows, int64_t cols, int64_t pitch,
               int dtype, uint64_t *S, uint64_t *Q, int64_t ld_out)
{
    if (!args_ok(img, rows, cols, pitch, dtype) || !S || ld_out < cols) return E_ARG;
    if (!oracle_fits_u64(rows, cols, dtype, Q != NULL)) return E_OVERFLOW;
    for (int64_t y = 0; y < rows; ++y) {
        uint64_t rs = 0, rq = 0;
        for (int64_t x = 0; x < cols; ++x) {
            uint64_t v = pix(img, pitch, dtype, y, x);
            rs += v;
            rq += v * v;
            S[y * ld_out + x] = rs + (y ? S[(y - 1) * ld_out + x] : 0);
            if (Q) Q[y * ld_out + x] = rq + (y ? Q[(y - 1) * ld_out + x] : 0);
        }
    }
    return OK;
}

/*
 * Selected rows of S and Q without holding the whole tables: streams the
 * image once, keeping only the current table row.  req[] must be strictly
 * increasing row indices; row k of the outputs (ld cols) receives table row
 * req[k].  Q_out may be NULL.
 */
int oracle_sat_rows(const void *img, int64_t rows, int64_t cols, int64_t pitch,
                    int dtype, const int64_t *req, int64_t nreq,
                    uint64_t *S_out, uint64_t *Q_out)
{
    if (!args_ok(img, rows, cols, pitch, dtype) || !req || nreq < 0 || !S_out)
        return E_ARG;
    for (int64_t k = 0; k < nreq; ++k)
        if (req[k] < 0 || req[k] >= rows || (k && req[k] <= req[k - 1])) return E_ARG;
    if (!oracle_fits_u64(rows, cols, dtype, Q_out != NULL)) return E_OVERFLOW;
    uint64_t *s = (uint64_t *)calloc((size_t)cols, sizeof(uint64_t));
    uint64_t *q = (uint64_t *)calloc((size_t)cols, sizeof(uint64_t));
    if (!s || !q) { free(s); free(q); return E_MEM; }
    int64_t k = 0;
    for (int64_t y = 0; y < rows && k < nreq; ++y) {
        uint64_t rs = 0, rq = 0;
        for (int64_t x = 0; x < cols; ++x) {
            uint64_t v = pix(img, pitch, dtype, y, x);
            rs += v;
            rq += v * v;
            s[x] += rs;
            q[x] += rq;
        }
        if (y == req[k]) {
            memcpy(S_out + k * cols, s, sizeof(uint64_t) * (size_t)cols);
            if (Q_out) memcpy(Q_out + k * cols, q, sizeof(uint64_t) * (size_t)cols);
            ++k;
        }
    }
    free(s);
    free(q);
    return OK;
}

/* One window by the definition: sum the n pixels (and their squares). */
int oracle_window_one(const void *img, int64_t rows, int64_t cols, int64_t pitch,
                      int dtype, int64_t y0, int64_t x0, int64_t wh, int64_t ww,
                      uint64_t *sum, uint64_t *sumsq, double *mean, double *std)
{
    if (!args_ok(img, rows, cols, pitch, dtype)) return E_ARG;
    if (wh <= 0 || ww <= 0 || y0 < 0 || x0 < 0 || y0 + wh > rows || x0 + ww > cols)
        return E_ARG;
    uint64_t s = 0, q = 0;
    for (int64_t y = y0; y < y0 + wh; ++y)
        for (int64_t x = x0; x < x0 + ww; ++x) {
            uint64_t v = pix(img, pitch, dtype, y, x);
            s += v;
            q += v * v;
        }
    if (sum) *sum = s;
    if (sumsq) *sumsq = q;
    oracle_stats_from_moments((uint64_t)(wh * ww), s, q, mean, std);
    return OK;
}

/*
 * Naive SWA (Section III-A): every valid window summed pixel by pixel.
 * Outputs are R x C with leading dimension ld; any output pointer may be NULL.
 */
int oracle_window_brute(const void *img, int64_t rows, int64_t cols, int64_t pitch,
                        int dtype, int64_t wh, int64_t ww, int64_t sy, int64_t sx,
                        uint64_t *sum, double *mean, double *std, int64_t ld)
{
    int64_t R, C;
    if (!args_ok(img, rows, cols, pitch, dtype)) return E_ARG;
    if (oracle_window_shape(rows, cols, wh, ww, sy, sx, &R, &C) != OK) return E_ARG;
    if (ld < C) return E_ARG;
    for (int64_t i = 0; i < R; ++i)
        for (int64_t j = 0; j < C; ++j) {
            uint64_t s, q;
            double m, d;
            oracle_window_one(img, rows, cols, pitch, dtype, i * sy, j * sx, wh, ww,
                              &s, &q, &m, &d);
            if (sum) sum[i * ld + j] = s;
            if (mean) mean[i * ld + j] = m;
            if (std) std[i * ld + j] = d;
        }
    return OK;
}

/* Table entry with index -1 reading as 0. */
static inline uint64_t at(const uint64_t *T, int64_t ld, int64_t y, int64_t x)
{
    return (y < 0 || x < 0) ? 0 : T[y * ld + x];
}

/*
 * Integral image SWA (Section II-B, III-B): four lookups per window on
 * tables built by oracle_sat.  Q may be NULL when std is not requested.
 */
int oracle_window_sat(const uint64_t *S, const uint64_t *Q, int64_t ld_sat,
                      int64_t rows, int64_t cols, int64_t wh, int64_t ww,
                      int64_t sy, int64_t sx, uint64_t *sum, double *mean,
                      double *std, int64_t ld)
{
    int64_t R, C;
    if (!S || (std && !Q)) return E_ARG;
    if (oracle_window_shape(rows, cols, wh, ww, sy, sx, &R, &C) != OK) return E_ARG;
    if (ld < C || ld_sat < cols) return E_ARG;
    uint64_t n = (uint64_t)(wh * ww);
    for (int64_t i = 0; i < R; ++i)
        for (int64_t j = 0; j < C; ++j) {
            int64_t y0 = i * sy, x0 = j * sx, y1 = y0 + wh - 1, x1 = x0 + ww - 1;
            uint64_t s = at(S, ld_sat, y1, x1) - at(S, ld_sat, y0 - 1, x1)
                       - at(S, ld_sat, y1, x0 - 1) + at(S, ld_sat, y0 - 1, x0 - 1);
            uint64_t q = 0;
            if (Q)
                q = at(Q, ld_sat, y1, x1) - at(Q, ld_sat, y0 - 1, x1)
                  - at(Q, ld_sat, y1, x0 - 1) + at(Q, ld_sat, y0 - 1, x0 - 1);
            if (sum) sum[i * ld + j] = s;
            oracle_stats_from_moments(n, s, q, mean ? &mean[i * ld + j] : NULL,
                                      std ? &std[i * ld + j] : NULL);
        }
    return OK;
}

/*
 * DP-naive-SWA, read as separable moving sums (Section IV-A): for every row a
 * running horizontal sum of width ww (add the entering pixel, drop the
 * leaving one), then a running vertical sum of height wh over those.  It
 * never forms a summed-area table.
 */
int oracle_window_sliding(const void *img, int64_t rows, int64_t cols, int64_t pitch,
                          int dtype, int64_t wh, int64_t ww, int64_t sy, int64_t sx,
                          uint64_t *sum, double *mean, double *std, int64_t ld)
{
    int64_t R, C;
    if (!args_ok(img, rows, cols, pitch, dtype)) return E_ARG;
    if (oracle_window_shape(rows, cols, wh, ww, sy, sx, &R, &C) != OK) return E_ARG;
    if (ld < C) return E_ARG;
    int64_t H = cols - ww + 1;               /* horizontal positions, stride 1 */
    /* ring of the last wh rows of horizontal sums */
    uint64_t *hs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(wh * H));
    uint64_t *hq = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(wh * H));
    uint64_t *vs = (uint64_t *)calloc((size_t)H, sizeof(uint64_t));
    uint64_t *vq = (uint64_t *)calloc((size_t)H, sizeof(uint64_t));
    if (!hs || !hq || !vs || !vq) { free(hs); free(hq); free(vs); free(vq); return E_MEM; }
    uint64_t n = (uint64_t)(wh * ww);
    for (int64_t y = 0; y < rows; ++y) {
        uint64_t *rs = hs + (y % wh) * H, *rq = hq + (y % wh) * H;
        if (y >= wh)                           /* the row leaving the window */
            for (int64_t x = 0; x < H; ++x) { vs[x] -= rs[x]; vq[x] -= rq[x]; }
        uint64_t a = 0, b = 0;
        for (int64_t x = 0; x < ww; ++x) {
            uint64_t v = pix(img, pitch, dtype, y, x);
            a += v;
            b += v * v;
        }
        rs[0] = a;
        rq[0] = b;
        for (int64_t x = 1; x < H; ++x) {
            uint64_t vin = pix(img, pitch, dtype, y, x + ww - 1);
            uint64_t vout = pix(img, pitch, dtype, y, x - 1);
            a = a + vin - vout;
            b = b + vin * vin - vout * vout;
            rs[x] = a;
            rq[x] = b;
        }
        for (int64_t x = 0; x < H; ++x) { vs[x] += rs[x]; vq[x] += rq[x]; }
        int64_t top = y - wh + 1;              /* window rows top..y are summed */
        if (top >= 0 && top % sy == 0) {
            int64_t i = top / sy;
            for (int64_t j = 0; j < C; ++j) {
                uint64_t s = vs[j * sx], q = vq[j * sx];
                if (sum) sum[i * ld + j] = s;
                oracle_stats_from_moments(n, s, q, mean ? &mean[i * ld + j] : NULL,
                                          std ? &std[i * ld + j] : NULL);
            }
        }
    }
    free(hs); free(hq); free(vs); free(vq);
    return OK;
}

/* Plain total of all pixels (and of their squares), by a flat loop. */
int oracle_total(const void *img, int64_t rows, int64_t cols, int64_t pitch,
                 int dtype, uint64_t *sum, uint64_t *sumsq)
{
    if (!args_ok(img, rows, cols, pitch, dtype)) return E_ARG;
    uint64_t s = 0, q = 0;
    for (int64_t y = 0; y < rows; ++y)
        for (int64_t x = 0; x < cols; ++x) {
            uint64_t v = pix(img, pitch, dtype, y, x);
            s += v;
            q += v * v;
        }
    if (sum) *sum = s;
    if (sumsq) *sumsq = q;
    return OK;
}

/*
 * Integral-image SWA for selected output rows only (sampled full-size
 * checks): row k of the outputs (ld entries apart) receives output row
 * out_rows[k].  Same lookups as oracle_window_sat.
 */
int oracle_window_sat_rows(const uint64_t *S, const uint64_t *Q, int64_t ld_sat,
                           int64_t rows, int64_t cols, int64_t wh, int64_t ww,
                           int64_t sy, int64_t sx, const int64_t *out_rows,
                           int64_t nrows, uint64_t *sum, double *mean, double *std,
                           int64_t ld)
{
    int64_t R, C;
    if (!S || (std && !Q) || !out_rows) return E_ARG;
    if (oracle_window_shape(rows, cols, wh, ww, sy, sx, &R, &C) != OK) return E_ARG;
    if (ld < C || ld_sat < cols) return E_ARG;
    uint64_t n = (uint64_t)(wh * ww);
    for (int64_t k = 0; k < nrows; ++k) {
        int64_t i = out_rows[k];
        if (i < 0 || i >= R) return E_ARG;
        for (int64_t j = 0; j < C; ++j) {
            int64_t y0 = i * sy, x0 = j * sx, y1 = y0 + wh - 1, x1 = x0 + ww - 1;
            uint64_t s = at(S, ld_sat, y1, x1) - at(S, ld_sat, y0 - 1, x1)
                       - at(S, ld_sat, y1, x0 - 1) + at(S, ld_sat, y0 - 1, x0 - 1);
            uint64_t q = 0;
            if (Q)
                q = at(Q, ld_sat, y1, x1) - at(Q, ld_sat, y0 - 1, x1)
                  - at(Q, ld_sat, y1, x0 - 1) + at(Q, ld_sat, y0 - 1, x0 - 1);
            if (sum) sum[k * ld + j] = s;
            oracle_stats_from_moments(n, s, q, mean ? &mean[k * ld + j] : NULL,
                                      std ? &std[k * ld + j] : NULL);
        }
    }
    return OK;
}

/* oracle_stats_from_moments over arrays (a plain loop; for bulk tests). */
void oracle_stats_bulk(const uint64_t *n, const uint64_t *sw, const uint64_t *qw,
                       int64_t count, double *mean, double *std)
{
    for (int64_t i = 0; i < count; ++i)
        oracle_stats_from_moments(n[i], sw[i], qw[i], &mean[i], &std[i]);
}

/*
 * Threshold count map (the "additional SWA algorithms" of Section V, for
 * cluster calling): for every valid window, the number of pixels strictly
 * greater than `thr`, by the definition (a double loop over the window).
 * frac = (double)count / (double)n is the fraction of such pixels and std the
 * population standard deviation of the window's 0/1 indicator values (its
 * squared values equal the values, so Qw = Sw = count).  Outputs are R x C
 * with leading dimension ld; any output pointer may be NULL.
 */
int oracle_count_brute(const void *img, int64_t rows, int64_t cols, int64_t pitch,
                       int dtype, uint64_t thr, int64_t wh, int64_t ww, int64_t sy,
                       int64_t sx, uint64_t *count, double *frac, double *std, int64_t ld)
{
    int64_t R, C;
    if (!args_ok(img, rows, cols, pitch, dtype)) return E_ARG;
    if (oracle_window_shape(rows, cols, wh, ww, sy, sx, &R, &C) != OK) return E_ARG;
    if (ld < C) return E_ARG;
    const uint64_t n = (uint64_t)wh * (uint64_t)ww;
    for (int64_t i = 0; i < R; ++i)
        for (int64_t j = 0; j < C; ++j) {
            uint64_t c = 0;
            for (int64_t y = i * sy; y < i * sy + wh; ++y)
                for (int64_t x = j * sx; x < j * sx + ww; ++x)
                    c += pix(img, pitch, dtype, y, x) > thr ? 1u : 0u;
            double m, d;
            oracle_stats_from_moments(n, c, c, &m, &d);
            if (count) count[i * ld + j] = c;
            if (frac) frac[i * ld + j] = m;
            if (std) std[i * ld + j] = d;
        }
    return OK;
}

/*
 * Integral-image SWA for selected output rows of an image whose tables need
 * not fit in host memory (the row-streaming reading of Section II-B): the
 * image is read once from the top while the running table rows of S and Q
 * (column sums of the row prefix sums) are kept; as the stream passes a table
 * row that a requested window's corners lie on -- row y0 - 1 or row
 * y0 + wh - 1 of a requested output row -- that row is copied out.  The four
 * lookups of oracle_window_sat are then made on the copied rows (index -1
 * reading as 0).  out_rows must be strictly increasing; row k of the outputs
 * (ld entries apart) receives output row out_rows[k].  Q is formed only when
 * std is requested.
 */
static int64_t find_row(const int64_t *need, int64_t nn, int64_t y)
{
    int64_t lo = 0, hi = nn - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (need[mid] < y) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

int oracle_window_rows_stream(const void *img, int64_t rows, int64_t cols, int64_t pitch,
                              int dtype, int64_t wh, int64_t ww, int64_t sy, int64_t sx,
                              const int64_t *out_rows, int64_t nrows, uint64_t *sum,
                              double *mean, double *std, int64_t ld)
{
    int64_t R, C;
    if (!args_ok(img, rows, cols, pitch, dtype) || !out_rows || nrows < 0) return E_ARG;
    if (oracle_window_shape(rows, cols, wh, ww, sy, sx, &R, &C) != OK) return E_ARG;
    if (ld < C) return E_ARG;
    for (int64_t k = 0; k < nrows; ++k)
        if (out_rows[k] < 0 || out_rows[k] >= R || (k && out_rows[k] <= out_rows[k - 1]))
            return E_ARG;
    if (nrows == 0) return OK;
    const int with_q = std != NULL;
    if (!oracle_fits_u64(rows, cols, dtype, with_q)) return E_OVERFLOW;
    /* The table rows the corners lie on, increasing and distinct: a merge of
     * the top rows (y0 - 1, when y0 > 0) and the bottom rows (y0 + wh - 1). */
    int64_t *need = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * nrows));
    if (!need) return E_MEM;
    int64_t nn = 0, a = 0, b = 0;
    while (a < nrows || b < nrows) {
        int64_t top = a < nrows ? out_rows[a] * sy - 1 : INT64_MAX;
        int64_t bot = b < nrows ? out_rows[b] * sy + wh - 1 : INT64_MAX;
        if (top < 0) { ++a; continue; }
        int64_t y = top < bot ? top : bot;
        if (top == y) ++a;
        if (bot == y) ++b;
        if (!nn || need[nn - 1] != y) need[nn++] = y;
    }
    uint64_t *s = (uint64_t *)calloc((size_t)cols, sizeof(uint64_t));
    uint64_t *q = (uint64_t *)calloc((size_t)cols, sizeof(uint64_t));
    uint64_t *Ss = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nn * cols));
    uint64_t *Qs = with_q ? (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nn * cols)) : NULL;
    if (!s || !q || !Ss || (with_q && !Qs)) {
        free(need); free(s); free(q); free(Ss); free(Qs);
        return E_MEM;
    }
    int64_t k = 0;
    for (int64_t y = 0; y <= need[nn - 1]; ++y) {
        uint64_t rs = 0, rq = 0;
        for (int64_t x = 0; x < cols; ++x) {
            uint64_t v = pix(img, pitch, dtype, y, x);
            rs += v;
            s[x] += rs;
            if (with_q) {
                rq += v * v;
                q[x] += rq;
            }
        }
        if (y == need[k]) {
            memcpy(Ss + k * cols, s, sizeof(uint64_t) * (size_t)cols);
            if (with_q) memcpy(Qs + k * cols, q, sizeof(uint64_t) * (size_t)cols);
            ++k;
        }
    }
    const uint64_t n = (uint64_t)(wh * ww);
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = out_rows[r], y0 = i * sy, y1 = y0 + wh - 1;
        /* saved row of table row y1, and of y0 - 1 (-1 when y0 == 0) */
        const int64_t kb = find_row(need, nn, y1);
        const int64_t kt = y0 > 0 ? find_row(need, nn, y0 - 1) : -1;
        for (int64_t j = 0; j < C; ++j) {
            const int64_t x0 = j * sx, x1 = x0 + ww - 1;
            uint64_t sw = at(Ss, cols, kb, x1) - at(Ss, cols, kt, x1)
                        - at(Ss, cols, kb, x0 - 1) + at(Ss, cols, kt, x0 - 1);
            uint64_t qw = 0;
            if (with_q)
                qw = at(Qs, cols, kb, x1) - at(Qs, cols, kt, x1)
                   - at(Qs, cols, kb, x0 - 1) + at(Qs, cols, kt, x0 - 1);
            if (sum) sum[r * ld + j] = sw;
            oracle_stats_from_moments(n, sw, qw, mean ? &mean[r * ld + j] : NULL,
                                      std ? &std[r * ld + j] : NULL);
        }
    }
    free(need); free(s); free(q); free(Ss); free(Qs);
    return OK;
}
