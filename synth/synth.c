/*
 * Seeded synthetic images shaped like the paper's immunofluorescence whole
 * tumour sections (Section IV-A: pancreatic ductal adenocarcinoma images of
 * 30k x 30k up to 70k x 85k pixels, which are not available here).
 *
 * This module holds input generation only: no summed-area table, window sum,
 * mean or standard deviation is computed here.  It is shared by the CPU
 * oracle's tests, the CUDA path's tests and the benchmark, and by nothing
 * else.
 *
 * Determinism: every random number is a counter-based draw (SplitMix64's
 * output function, Steele, Lea and Flood, OOPSLA 2014, applied to a key plus
 * a counter), so an image depends on (seed, shape, parameters) only, never on
 * the thread count.  The transcendental functions used (exp, log) are written
 * here from their series with IEEE basic operations only and the file is
 * compiled with -ffp-contract=off, so x86-64 and aarch64 hosts produce the
 * same bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG --- */

static inline uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Key of one named stream of draws under one seed. */
static inline uint64_t sm_key(uint64_t seed, uint64_t stream)
{
    return sm_mix(seed * 0x9E3779B97F4A7C15ULL + sm_mix(stream + 0x632BE59BD9B4E019ULL));
}

/* The ctr-th 64-bit draw of a stream. */
static inline uint64_t sm_draw(uint64_t key, uint64_t ctr)
{
    return sm_mix(key + (ctr + 1) * 0x9E3779B97F4A7C15ULL);
}

/* Uniform in the open interval (0, 1): 53 random bits, centred in their cell. */
static inline double sm_unif(uint64_t key, uint64_t ctr)
{
    return ((double)(sm_draw(key, ctr) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* Stream identifiers. */
enum { ST_PARENT = 1, ST_NCHILD, ST_CHILD, ST_BG, ST_CLUSTER, ST_BATCH, ST_REQ };

/* ------------------------------------------------ portable exp and log --- */

/* ln 2 split so that k * LN2_HI is exact for |k| < 2^20 (Cody and Waite's
 * argument reduction). */
static const double LN2_HI = 6.93147180369123816490e-01;
static const double LN2_LO = 1.90821492927058770002e-10;
static const double INV_LN2 = 1.44269504088896338700e+00;

/* e^x from the Taylor series of e^r on |r| <= ln2/2 (degree 14, relative
 * truncation error below 1e-17), scaled by 2^k with ldexp (exact). */
static double px_exp(double x)
{
    if (x < -700.0) return 0.0;
    if (x > 700.0) return HUGE_VAL;
    double k = floor(x * INV_LN2 + 0.5);
    double r = (x - k * LN2_HI) - k * LN2_LO;
    double p = 1.0 / 87178291200.0;                 /* 1/14! */
    static const double inv_fact[14] = {
        1.0 / 6227020800.0, 1.0 / 479001600.0, 1.0 / 39916800.0,
        1.0 / 3628800.0, 1.0 / 362880.0, 1.0 / 40320.0, 1.0 / 5040.0,
        1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0, 1.0 };
    for (int i = 0; i < 14; ++i) p = p * r + inv_fact[i];
    return ldexp(p, (int)k);
}

/* ln(u) for u > 0: u = m 2^e with m in [sqrt(1/2), sqrt(2)), then
 * ln m = 2 atanh(t), t = (m-1)/(m+1), |t| < 0.172, series to t^23. */
static double px_log(double u)
{
    int e;
    double m = frexp(u, &e);                        /* m in [0.5, 1) */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double t = (m - 1.0) / (m + 1.0);
    double t2 = t * t;
    double s = 1.0 / 23.0;
    for (int k = 21; k >= 1; k -= 2) s = s * t2 + 1.0 / (double)k;
    return (double)e * LN2_HI + ((double)e * LN2_LO + 2.0 * t * s);
}

/* Standard normal by Marsaglia's polar method; draws (ctr*128 + 2a, +1) for
 * attempt a, so the result is a function of ctr alone. */
static double px_normal(uint64_t key, uint64_t ctr)
{
    for (uint64_t a = 0; a < 64; ++a) {
        double v1 = 2.0 * sm_unif(key, ctr * 128 + 2 * a) - 1.0;
        double v2 = 2.0 * sm_unif(key, ctr * 128 + 2 * a + 1) - 1.0;
        double s = v1 * v1 + v2 * v2;
        if (s > 0.0 && s < 1.0) return v1 * sqrt(-2.0 * px_log(s) / s);
    }
    return 0.0;   /* probability (1 - pi/4)^64 < 1e-42 */
}

/* Poisson(lambda) by multiplying uniforms (Knuth, TAOCP vol. 2, 3.4.1). */
static int px_poisson(double lambda, uint64_t key, uint64_t ctr)
{
    double L = px_exp(-lambda), p = 1.0;
    int k = 0;
    do {
        p *= sm_unif(key, ctr * 1024 + (uint64_t)k);
        ++k;
    } while (p > L && k < 1000);
    return k - 1;
}

/* ------------------------------------------ cell-centroid binary mask --- */

/*
 * Thomas (Neyman-Scott) cluster process: parent centres uniform over the
 * image, Poisson(mean_children) children per parent, child offsets normal
 * with standard deviation sigma per axis, rounded and clipped to the image.
 * Pixels are set to 1 until exactly n_ones distinct pixels are set.
 * Returns the number of ones written (n_ones unless it exceeds rows*cols).
 */
int64_t synth_mask_u8(uint8_t *img, int64_t rows, int64_t cols, int64_t pitch,
                      uint64_t seed, int64_t n_ones, double sigma,
                      double mean_children)
{
    if (!img || rows <= 0 || cols <= 0 || pitch < cols) return -1;
    for (int64_t y = 0; y < rows; ++y) memset(img + y * pitch, 0, (size_t)cols);
    if (n_ones > rows * cols) n_ones = rows * cols;
    uint64_t kp = sm_key(seed, ST_PARENT), kn = sm_key(seed, ST_NCHILD),
             kc = sm_key(seed, ST_CHILD);
    int64_t set = 0;
    for (uint64_t p = 0; set < n_ones && p < (1ULL << 40); ++p) {
        double py = sm_unif(kp, 2 * p) * (double)rows;
        double px = sm_unif(kp, 2 * p + 1) * (double)cols;
        int nc = px_poisson(mean_children, kn, p);
        for (int c = 0; c < nc && set < n_ones; ++c) {
            uint64_t ctr = (p << 12) + (uint64_t)c;
            double dy = sigma * px_normal(kc, 2 * ctr);
            double dx = sigma * px_normal(kc, 2 * ctr + 1);
            double fy = floor(py + dy + 0.5), fx = floor(px + dx + 0.5);
            int64_t y = fy < 0 ? 0 : (fy > (double)(rows - 1) ? rows - 1 : (int64_t)fy);
            int64_t x = fx < 0 ? 0 : (fx > (double)(cols - 1) ? cols - 1 : (int64_t)fx);
            uint8_t *q = img + y * pitch + x;
            if (!*q) { *q = 1; ++set; }
        }
    }
    return set;
}

/* ------------------------------------------------ intensity images ------ */

typedef struct { double cy, cx, sigma, amp; } blob_t;

/* Cluster parameters: centre uniform over the image, sigma ~ U[smin, smax],
 * amplitude ~ U[amin, amax]. */
static void make_blobs(blob_t *b, int64_t n, int64_t rows, int64_t cols,
                       uint64_t seed, double smin, double smax,
                       double amin, double amax)
{
    uint64_t k = sm_key(seed, ST_CLUSTER);
    for (int64_t i = 0; i < n; ++i) {
        b[i].cy = sm_unif(k, 4 * (uint64_t)i) * (double)rows;
        b[i].cx = sm_unif(k, 4 * (uint64_t)i + 1) * (double)cols;
        b[i].sigma = smin + (smax - smin) * sm_unif(k, 4 * (uint64_t)i + 2);
        b[i].amp = amin + (amax - amin) * sm_unif(k, 4 * (uint64_t)i + 3);
    }
}

#define BAND 32

/*
 * Shared body of the u8 and u16 intensity generators.  value(y, x) =
 * min(vmax, floor(bg(y, x) + sum_k blob_k(y, x) + 0.5)) where
 *   blob_k(y, x) = amp_k * g(y - cy_k) * g(x - cx_k), g(d) = exp(-d^2 / (2 s^2)),
 * truncated to (y - cy)^2 + (x - cx)^2 <= 16 s^2, and the blobs are added in
 * index order into a double accumulator per pixel (so the sum does not
 * depend on the thread count).
 *   bg_kind 0: Gamma(shape 2, scale bg_a) = -bg_a ln(u1 u2)
 *   bg_kind 1: log-normal exp(bg_a + bg_b N(0,1))
 */
static int intensity_impl(void *img, int bytes_pp, int64_t rows, int64_t cols,
                          int64_t pitch, uint64_t seed, int64_t n_clusters,
                          double smin, double smax, double amin, double amax,
                          int bg_kind, double bg_a, double bg_b, double vmax)
{
    if (!img || rows <= 0 || cols <= 0 || pitch < cols * bytes_pp || n_clusters < 0)
        return -1;
    blob_t *bl = (blob_t *)malloc(sizeof(blob_t) * (size_t)(n_clusters ? n_clusters : 1));
    if (!bl) return -2;
    make_blobs(bl, n_clusters, rows, cols, seed, smin, smax, amin, amax);

    /* Bucket blobs by BAND-row band, in index order. */
    int64_t nbands = (rows + BAND - 1) / BAND;
    int64_t *cnt = (int64_t *)calloc((size_t)nbands + 1, sizeof(int64_t));
    if (!cnt) { free(bl); return -2; }
    for (int64_t i = 0; i < n_clusters; ++i) {
        double r = 4.0 * bl[i].sigma;
        int64_t y0 = (int64_t)floor(bl[i].cy - r), y1 = (int64_t)ceil(bl[i].cy + r);
        if (y0 < 0) y0 = 0;
        if (y1 > rows - 1) y1 = rows - 1;
        if (y1 < y0) continue;
        for (int64_t b = y0 / BAND; b <= y1 / BAND; ++b) cnt[b + 1]++;
    }
    for (int64_t b = 0; b < nbands; ++b) cnt[b + 1] += cnt[b];
    int64_t *lst = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cnt[nbands] ? cnt[nbands] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nbands);
    if (!lst || !fill) { free(bl); free(cnt); free(lst); free(fill); return -2; }
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)nbands);
    for (int64_t i = 0; i < n_clusters; ++i) {
        double r = 4.0 * bl[i].sigma;
        int64_t y0 = (int64_t)floor(bl[i].cy - r), y1 = (int64_t)ceil(bl[i].cy + r);
        if (y0 < 0) y0 = 0;
        if (y1 > rows - 1) y1 = rows - 1;
        if (y1 < y0) continue;
        for (int64_t b = y0 / BAND; b <= y1 / BAND; ++b) lst[fill[b]++] = i;
    }
    free(fill);

    uint64_t kb = sm_key(seed, ST_BG);
    int err = 0;
#pragma omp parallel
    {
        double *acc = (double *)malloc(sizeof(double) * (size_t)(BAND * cols));
        int64_t gmax = 1 + 2 * (int64_t)ceil(4.0 * smax) + 2;
        double *gx = (double *)malloc(sizeof(double) * (size_t)gmax);
        if (!acc || !gx) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t b = 0; b < nbands; ++b) {
            if (!acc || !gx) continue;
            int64_t ya = b * BAND, yb = ya + BAND < rows ? ya + BAND : rows;
            memset(acc, 0, sizeof(double) * (size_t)((yb - ya) * cols));
            for (int64_t li = cnt[b]; li < cnt[b + 1]; ++li) {
                const blob_t *B = &bl[lst[li]];
                double s = B->sigma, r = 4.0 * s, r2 = 16.0 * s * s;
                double inv2s2 = 1.0 / (2.0 * s * s);
                int64_t x0 = (int64_t)floor(B->cx - r), x1 = (int64_t)ceil(B->cx + r);
                if (x0 < 0) x0 = 0;
                if (x1 > cols - 1) x1 = cols - 1;
                for (int64_t x = x0; x <= x1; ++x) {
                    double d = (double)x - B->cx;
                    gx[x - x0] = px_exp(-d * d * inv2s2);
                }
                int64_t y0 = (int64_t)floor(B->cy - r), y1 = (int64_t)ceil(B->cy + r);
                if (y0 < ya) y0 = ya;
                if (y1 > yb - 1) y1 = yb - 1;
                for (int64_t y = y0; y <= y1; ++y) {
                    double dy = (double)y - B->cy;
                    double gy = B->amp * px_exp(-dy * dy * inv2s2);
                    double *row = acc + (y - ya) * cols;
                    for (int64_t x = x0; x <= x1; ++x) {
                        double dx = (double)x - B->cx;
                        if (dx * dx + dy * dy <= r2) row[x] += gy * gx[x - x0];
                    }
                }
            }
            for (int64_t y = ya; y < yb; ++y) {
                const double *row = acc + (y - ya) * cols;
                for (int64_t x = 0; x < cols; ++x) {
                    uint64_t idx = (uint64_t)y * (uint64_t)cols + (uint64_t)x;
                    double bg;
                    if (bg_kind == 0)
                        bg = -bg_a * px_log(sm_unif(kb, 2 * idx) * sm_unif(kb, 2 * idx + 1));
                    else
                        bg = px_exp(bg_a + bg_b * px_normal(kb, idx));
                    double v = floor(bg + row[x] + 0.5);
                    if (v > vmax) v = vmax;
                    if (v < 0.0) v = 0.0;
                    if (bytes_pp == 1)
                        ((uint8_t *)img)[y * pitch + x] = (uint8_t)v;
                    else
                        *(uint16_t *)((uint8_t *)img + y * pitch + 2 * x) = (uint16_t)v;
                }
            }
        }
        free(acc);
        free(gx);
    }
    free(bl); free(cnt); free(lst);
    return err ? -2 : 0;
}

/* uint8 intensity image: Gamma(2, 20) background, n_clusters Gaussian
 * clusters with sigma ~ U[10, 60] px and amplitude ~ U[60, 200], clipped to
 * 255. */
int synth_intensity_u8(uint8_t *img, int64_t rows, int64_t cols, int64_t pitch,
                       uint64_t seed, int64_t n_clusters)
{
    return intensity_impl(img, 1, rows, cols, pitch, seed, n_clusters,
                          10.0, 60.0, 60.0, 200.0, 0, 20.0, 0.0, 255.0);
}

/* uint16 intensity image: log-normal(mu 6, sigma 1.5) background, clusters as
 * for uint8 with amplitudes scaled by 256, clipped to 65535. */
int synth_intensity_u16(uint16_t *img, int64_t rows, int64_t cols,
                        int64_t pitch_bytes, uint64_t seed, int64_t n_clusters)
{
    return intensity_impl(img, 2, rows, cols, pitch_bytes, seed, n_clusters,
                          10.0, 60.0, 60.0 * 256.0, 200.0 * 256.0, 1, 6.0, 1.5,
                          65535.0);
}

/* Uniform 64-bit draws of a named stream (for host-side recipes such as the
 * batched and served workloads): out[i] = draw(seed, stream, first + i). */
void synth_draws(uint64_t seed, uint64_t stream, uint64_t first, int64_t n,
                 uint64_t *out)
{
    uint64_t k = sm_key(seed, ST_BATCH + stream);
    for (int64_t i = 0; i < n; ++i) out[i] = sm_draw(k, first + (uint64_t)i);
}

/* The portable exp and log, exported so tests can check their accuracy. */
double synth_exp(double x) { return px_exp(x); }
double synth_log(double x) { return px_log(x); }

int synth_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
