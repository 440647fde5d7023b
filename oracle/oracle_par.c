/*
 * Row-parallel variants of the CPU oracle, for timing the CPU baseline on all
 * host cores.  TEST INFRASTRUCTURE ONLY (the benchmark's CPU legs and the
 * tests that pin these functions equal to the serial ones in oracle.c).
 *
 * The parallel integral image of Section III-B on a multi-core CPU, in its
 * plain row-band form:
 *   1. every thread sums the columns of its band of rows (per-band column
 *      totals of I and of I^2);
 *   2. one thread turns them into the table row just above each band,
 *      S[y_b - 1][x] = sum_{j <= x} sum_{i < y_b} I[i][j] (a running sum
 *      over the bands above, then over x);
 *   3. every thread builds its band's rows from that carry row with the
 *      serial recurrence S[y][x] = S[y - 1][x] + sum_{j <= x} I[y][j].
 * Window statistics are independent per output row: threads take output
 * rows and make the four lookups of oracle_window_sat.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define DT_U8 1
#define DT_U16 2
#define OK 0
#define E_ARG -1
#define E_MEM -2
#define E_OVERFLOW -3

int oracle_fits_u64(int64_t rows, int64_t cols, int dtype, int with_sq);
int oracle_window_shape(int64_t rows, int64_t cols, int64_t wh, int64_t ww, int64_t sy,
                        int64_t sx, int64_t *out_r, int64_t *out_c);
void oracle_stats_from_moments(uint64_t n, uint64_t sw, uint64_t qw, double *mean,
                               double *std);

static inline uint64_t pix(const void *img, int64_t pitch, int dtype, int64_t y, int64_t x)
{
    const uint8_t *row = (const uint8_t *)img + y * pitch;
    if (dtype == DT_U8) return row[x];
    uint16_t v;
    memcpy(&v, row + 2 * x, 2);
    return v;
}

/* Threads used by the parallel functions (0: OpenMP's default). */
int oracle_par_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

int oracle_sat_par(const void *img, int64_t rows, int64_t cols, int64_t pitch, int dtype,
                   uint64_t *S, uint64_t *Q, int64_t ld_out)
{
    if (!img || rows <= 0 || cols <= 0 || !S || ld_out < cols) return E_ARG;
    if (dtype != DT_U8 && dtype != DT_U16) return E_ARG;
    if (pitch < cols * (dtype == DT_U8 ? 1 : 2)) return E_ARG;
    if (!oracle_fits_u64(rows, cols, dtype, Q != NULL)) return E_OVERFLOW;
    const int nb = omp_get_max_threads();
    const int64_t band = (rows + nb - 1) / nb;
    /* per band: column totals (phase 1), then the carry row (phase 2) */
    uint64_t *cs = (uint64_t *)calloc((size_t)(nb * cols), sizeof(uint64_t));
    uint64_t *cq = (uint64_t *)calloc((size_t)(nb * cols), sizeof(uint64_t));
    if (!cs || !cq) { free(cs); free(cq); return E_MEM; }
#pragma omp parallel for schedule(static, 1)
    for (int b = 0; b < nb; ++b) {
        const int64_t y0 = b * band, y1 = y0 + band < rows ? y0 + band : rows;
        uint64_t *ts = cs + b * cols, *tq = cq + b * cols;
        for (int64_t y = y0; y < y1; ++y)
            for (int64_t x = 0; x < cols; ++x) {
                const uint64_t v = pix(img, pitch, dtype, y, x);
                ts[x] += v;
                tq[x] += v * v;
            }
    }
    /* carry of band b = table row above it: column totals of bands < b,
     * accumulated down the bands, then prefix-summed along the row */
    {
        uint64_t *acc_s = (uint64_t *)calloc((size_t)cols, sizeof(uint64_t));
        uint64_t *acc_q = (uint64_t *)calloc((size_t)cols, sizeof(uint64_t));
        if (!acc_s || !acc_q) { free(acc_s); free(acc_q); free(cs); free(cq); return E_MEM; }
        for (int b = 0; b < nb; ++b) {
            uint64_t *ts = cs + b * cols, *tq = cq + b * cols;
            uint64_t ps = 0, pq = 0;
            for (int64_t x = 0; x < cols; ++x) {
                const uint64_t bs = ts[x], bq = tq[x];
                ps += acc_s[x];
                pq += acc_q[x];
                ts[x] = ps;                    /* S[y_b - 1][x] */
                tq[x] = pq;
                acc_s[x] += bs;
                acc_q[x] += bq;
            }
        }
        free(acc_s);
        free(acc_q);
    }
#pragma omp parallel for schedule(static, 1)
    for (int b = 0; b < nb; ++b) {
        const int64_t y0 = b * band, y1 = y0 + band < rows ? y0 + band : rows;
        const uint64_t *ps = cs + b * cols, *pq = cq + b * cols;
        for (int64_t y = y0; y < y1; ++y) {
            uint64_t rs = 0, rq = 0;
            for (int64_t x = 0; x < cols; ++x) {
                const uint64_t v = pix(img, pitch, dtype, y, x);
                rs += v;
                rq += v * v;
                S[y * ld_out + x] = rs + (y > y0 ? S[(y - 1) * ld_out + x] : ps[x]);
                if (Q) Q[y * ld_out + x] = rq + (y > y0 ? Q[(y - 1) * ld_out + x] : pq[x]);
            }
        }
    }
    free(cs);
    free(cq);
    return OK;
}

static inline uint64_t at(const uint64_t *T, int64_t ld, int64_t y, int64_t x)
{
    return (y < 0 || x < 0) ? 0 : T[y * ld + x];
}

int oracle_window_sat_par(const uint64_t *S, const uint64_t *Q, int64_t ld_sat, int64_t rows,
                          int64_t cols, int64_t wh, int64_t ww, int64_t sy, int64_t sx,
                          uint64_t *sum, double *mean, double *std, int64_t ld)
{
    int64_t R, C;
    if (!S || (std && !Q)) return E_ARG;
    if (oracle_window_shape(rows, cols, wh, ww, sy, sx, &R, &C) != OK) return E_ARG;
    if (ld < C || ld_sat < cols) return E_ARG;
    const uint64_t n = (uint64_t)(wh * ww);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < R; ++i)
        for (int64_t j = 0; j < C; ++j) {
            const int64_t y0 = i * sy, x0 = j * sx, y1 = y0 + wh - 1, x1 = x0 + ww - 1;
            const uint64_t s = at(S, ld_sat, y1, x1) - at(S, ld_sat, y0 - 1, x1)
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
