/*
 * hd_oracle.c -- plain, slow CPU oracle of the hybrid multi-noise denoiser.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The product path (the
 * CUDA library) never calls it, and the two share no code.
 *
 * What it computes (Youssef, Mahmoud, El-Horbaty, "A Parallel Hybrid
 * Technique for Multi-Noise Removal from Grayscale Medical Images"):
 *
 *   hybrid = Wiener( AdaptiveMedian( g ) )            (Algorithm 1, step 4)
 *
 * Adaptive median (Algorithm 1, step 6; Section IV): for window sizes
 * k = 3, 5, ..., Smax, over the k x k neighbourhood of the NOISY image g:
 *   level A:  zmin < zmed < zmax            -> the pixel is processed at k
 *   level B:  zmin < zxy  < zmax  ? zxy : zmed
 * A pixel processed at some k is never touched again.  A pixel that fails
 * level A for every k up to Smax is given zmed of the Smax window (textbook
 * reading of the unresolved case) or keeps zxy (literal reading of the
 * listing, where the working copy starts as the input).
 *
 * Wiener (Algorithm 1, step 4d; spatial local-statistics form): over a
 * wh x ww window of the adaptive-median output f (wh rows, ww columns, both
 * odd; the paper gives no window, square ones are wh = ww = w), n = wh*ww,
 *   S1 = sum f, S2 = sum f^2 (exact integers), D = n*S2 - S1^2,
 *   mu = S1/n, sigma2 = D/n^2,
 *   nu2 = mean over all pixels of sigma2 (unless the caller supplies it)
 *       = fl( fl(sum D) / (n^2 * H * W) ),
 *   y = mu + max(sigma2 - nu2, 0) / max(sigma2, nu2) * (f - mu)
 *     (y = mu where sigma2 = nu2 = 0),
 *   out = min(maxv, floor(y + 0.5)).
 * y is evaluated in binary64 (the paper's precision, im2double in step 2).
 * A binary32 twin follows the fixed evaluation order that the GPU kernel
 * uses for its FP32 gain, so that the integer rounding decision can be
 * compared in the same precision on both sides.
 *
 * Contrast stretch (Algorithm 1, step 4e; a separate post-step, see
 * oracle_contrast): linear between histogram saturation limits.
 *
 * Borders: out-of-range indices map by half-sample symmetric reflection with
 * period 2N (the paper states no border rule), or, for the Wiener stage only,
 * read as zero while still counting in n.
 *
 * Build: cc -O2 -ffp-contract=off -fPIC -shared -o liboracle.so hd_oracle.c
 * (-ffp-contract=off keeps a*b+c as two rounded operations on every host.)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_SMAX 2
#define ORACLE_ERR_WINDOW 3
#define ORACLE_ERR_OOM 5

/* Half-sample symmetric extension: ... 2 1 0 | 0 1 2 ... N-1 | N-1 N-2 ... */
static long reflect_index(long i, long n)
{
    long p = 2 * n;
    long m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

static int cmp_u16(const void *a, const void *b)
{
    uint16_t x = *(const uint16_t *)a, y = *(const uint16_t *)b;
    return (x > y) - (x < y);
}

/* Algorithm 1, step 6a: Smax must be an odd integer greater than one. */
int oracle_check_smax(int Smax)
{
    if (Smax <= 1 || Smax % 2 == 0) return ORACLE_ERR_SMAX;
    return ORACLE_OK;
}

/*
 * Adaptive median filter, Algorithm 1 step 6, whole image (one partition).
 *   g      : H x W input, row-major, values as uint16 (8-bit images widened)
 *   f      : H x W output
 *   Smax   : largest window, odd > 1
 *   keep_unresolved : 0 -> unresolved pixels get zmed(Smax); 1 -> keep zxy
 *   k_out  : optional H x W; the window size at which each pixel passed
 *            level A, or 0 if it never did (diagnostics for the tests)
 * Window size k is the outer loop (Section IV: the window grows from 3x3 to
 * Smax); for each k every pixel that no smaller window has resolved is
 * tested again (resolved[] marks the others).
 */
int oracle_amf(const uint16_t *g, uint16_t *f, long H, long W, int Smax,
               int keep_unresolved, uint8_t *k_out)
{
    if (!g || !f || H < 1 || W < 1) return ORACLE_ERR_ARG;
    if (oracle_check_smax(Smax) != ORACLE_OK) return ORACLE_ERR_SMAX;

    long npx = H * W;
    uint8_t *resolved = (uint8_t *)calloc((size_t)npx, 1);     /* pixel passed level A at some k */
    uint16_t *win = (uint16_t *)malloc((size_t)Smax * Smax * sizeof(uint16_t));
    if (!resolved || !win) { free(resolved); free(win); return ORACLE_ERR_OOM; }

    memcpy(f, g, (size_t)npx * sizeof(uint16_t));              /* f = g */
    if (k_out) memset(k_out, 0, (size_t)npx);

    for (int k = 3; k <= Smax; k += 2) {
        int r = k / 2;
        int cnt = k * k;
        for (long y = 0; y < H; ++y) {
            for (long x = 0; x < W; ++x) {
                long p = y * W + x;
                if (resolved[p]) continue;
                /* k x k neighbourhood of the noisy image g */
                int m = 0;
                for (int dy = -r; dy <= r; ++dy) {
                    long yy = reflect_index(y + dy, H);
                    for (int dx = -r; dx <= r; ++dx) {
                        long xx = reflect_index(x + dx, W);
                        win[m++] = g[yy * W + xx];
                    }
                }
                qsort(win, (size_t)cnt, sizeof(uint16_t), cmp_u16);
                uint16_t zmin = win[0];
                uint16_t zmax = win[cnt - 1];
                uint16_t zmed = win[(cnt - 1) / 2];
                uint16_t zxy = g[p];
                int level_a = (zmed > zmin) && (zmax > zmed);             /* zmed is not an impulse */
                if (level_a) {
                    int level_b = (zxy > zmin) && (zmax > zxy);           /* zxy is not an impulse */
                    f[p] = level_b ? zxy : zmed;
                    resolved[p] = 1;
                    if (k_out) k_out[p] = (uint8_t)k;
                } else if (k == Smax && !keep_unresolved) {
                    f[p] = zmed;                                           /* unresolved */
                }
            }
        }
    }
    free(resolved);
    free(win);
    return ORACLE_OK;
}

/*
 * Wiener local statistics over a wh x ww window (wh rows, ww columns, both
 * odd; the square window is wh = ww = w): S1 and D = n*S2 - S1^2 for every
 * pixel, n = wh*ww.
 * border_zero = 0: symmetric reflection; 1: zero outside, still counted in n.
 */
static void wiener_stats(const uint16_t *f, long H, long W, int wh, int ww, int border_zero,
                         uint64_t *S1_out, uint64_t *D_out)
{
    int ry = wh / 2, rx = ww / 2;
    uint64_t n = (uint64_t)wh * (uint64_t)ww;
    for (long y = 0; y < H; ++y) {
        for (long x = 0; x < W; ++x) {
            uint64_t S1 = 0, S2 = 0;
            for (int dy = -ry; dy <= ry; ++dy) {
                for (int dx = -rx; dx <= rx; ++dx) {
                    long yy = y + dy, xx = x + dx;
                    uint64_t v;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) {
                        if (border_zero) v = 0;
                        else v = f[reflect_index(yy, H) * W + reflect_index(xx, W)];
                    } else {
                        v = f[yy * W + xx];
                    }
                    S1 += v;
                    S2 += v * v;
                }
            }
            S1_out[y * W + x] = S1;
            D_out[y * W + x] = n * S2 - S1 * S1;
        }
    }
}

/*
 * Wiener filter of an integer image f over a wh x ww window.
 *   noise_var_in < 0 : estimate nu2 as the mean local variance of f
 *   maxv             : largest representable output value (2^bits - 1)
 * Outputs (each optional):
 *   out64 / y64 : binary64 evaluation and its rounded integer
 *   out32 / y32 : binary32 twin (kernel evaluation order) and its integer
 *   nu2_out     : the noise variance used
 *   sumD_out    : sum of D over all pixels as two 64-bit words {lo, hi}
 */
int oracle_wiener_rect(const uint16_t *f, long H, long W, int wh, int ww, int border_zero,
                       double noise_var_in, int maxv,
                       uint16_t *out64, double *y64, uint16_t *out32, float *y32,
                       double *nu2_out, uint64_t *sumD_out)
{
    if (!f || H < 1 || W < 1 || maxv < 1) return ORACLE_ERR_ARG;
    if (wh < 1 || wh % 2 == 0 || ww < 1 || ww % 2 == 0) return ORACLE_ERR_WINDOW;

    long npx = H * W;
    uint64_t *S1 = (uint64_t *)malloc((size_t)npx * sizeof(uint64_t));
    uint64_t *D = (uint64_t *)malloc((size_t)npx * sizeof(uint64_t));
    if (!S1 || !D) { free(S1); free(D); return ORACLE_ERR_OOM; }
    wiener_stats(f, H, W, wh, ww, border_zero, S1, D);

    uint64_t n = (uint64_t)wh * (uint64_t)ww;

    /* global noise variance: exact integer sum, then binary64 */
    unsigned __int128 sumD = 0;
    for (long p = 0; p < npx; ++p) sumD += D[p];
    if (sumD_out) {
        sumD_out[0] = (uint64_t)sumD;
        sumD_out[1] = (uint64_t)(sumD >> 64);
    }
    double nu2;
    if (noise_var_in < 0.0) {
        double denom = (double)n * (double)n * (double)H * (double)W;
        nu2 = (double)sumD / denom;
    } else {
        nu2 = noise_var_in;
    }
    if (nu2_out) *nu2_out = nu2;

    /* binary32 twin constants (kernel evaluation order) */
    float inv_n32 = 1.0f / (float)n;
    float inv_n2_32 = 1.0f / (float)(n * n);
    float nu2_32 = (float)nu2;

    for (long p = 0; p < npx; ++p) {
        /* binary64: the definition */
        double mu = (double)S1[p] / (double)n;
        double sigma2 = (double)D[p] / ((double)n * (double)n);
        double num = sigma2 - nu2 > 0.0 ? sigma2 - nu2 : 0.0;
        double den = sigma2 > nu2 ? sigma2 : nu2;
        double y;
        if (den > 0.0) y = mu + (num / den) * ((double)f[p] - mu);
        else y = mu;
        if (y64) y64[p] = y;
        if (out64) {
            double q = floor(y + 0.5);
            if (q < 0.0) q = 0.0;
            if (q > (double)maxv) q = (double)maxv;
            out64[p] = (uint16_t)q;
        }

        /* binary32 twin: every operation rounded to nearest, no fused ops */
        if (y32 || out32) {
            float mu32 = (float)S1[p] * inv_n32;
            float s2_32 = (float)D[p] * inv_n2_32;
            float den32 = s2_32 > nu2_32 ? s2_32 : nu2_32;
            float num32 = s2_32 - nu2_32;
            if (!(num32 > 0.0f)) num32 = 0.0f;
            float yf;
            if (den32 > 0.0f) {
                float gain = num32 / den32;
                float dev = (float)f[p] - mu32;
                float prod = gain * dev;
                yf = mu32 + prod;
            } else {
                yf = mu32;
            }
            if (y32) y32[p] = yf;
            if (out32) {
                float q = floorf(yf + 0.5f);
                if (q < 0.0f) q = 0.0f;
                if (q > (float)maxv) q = (float)maxv;
                out32[p] = (uint16_t)q;
            }
        }
    }
    free(S1);
    free(D);
    return ORACLE_OK;
}

/* The square window w x w. */
int oracle_wiener(const uint16_t *f, long H, long W, int w, int border_zero,
                  double noise_var_in, int maxv,
                  uint16_t *out64, double *y64, uint16_t *out32, float *y32,
                  double *nu2_out, uint64_t *sumD_out)
{
    return oracle_wiener_rect(f, H, W, w, w, border_zero, noise_var_in, maxv, out64, y64, out32, y32,
                              nu2_out, sumD_out);
}

/* Per-pixel local statistics over a wh x ww window, exposed for the
 * closed-form tests. */
int oracle_wiener_stats(const uint16_t *f, long H, long W, int wh, int ww, int border_zero,
                        uint64_t *S1_out, uint64_t *D_out)
{
    if (!f || !S1_out || !D_out || H < 1 || W < 1) return ORACLE_ERR_ARG;
    if (wh < 1 || wh % 2 == 0 || ww < 1 || ww % 2 == 0) return ORACLE_ERR_WINDOW;
    wiener_stats(f, H, W, wh, ww, border_zero, S1_out, D_out);
    return ORACLE_OK;
}

/*
 * Adaptive median for a single pixel (used to check sampled outputs of very
 * large images one by one).  Returns the filtered value, or -1 on bad input.
 */
int oracle_amf_pixel(const uint16_t *g, long H, long W, int Smax, int keep_unresolved,
                     long y, long x)
{
    if (!g || H < 1 || W < 1 || y < 0 || y >= H || x < 0 || x >= W) return -1;
    if (oracle_check_smax(Smax) != ORACLE_OK) return -1;
    uint16_t *win = (uint16_t *)malloc((size_t)Smax * Smax * sizeof(uint16_t));
    if (!win) return -1;
    uint16_t zxy = g[y * W + x];
    int result = -1;
    for (int k = 3; k <= Smax; k += 2) {
        int r = k / 2, cnt = k * k, m = 0;
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                win[m++] = g[reflect_index(y + dy, H) * W + reflect_index(x + dx, W)];
        qsort(win, (size_t)cnt, sizeof(uint16_t), cmp_u16);
        uint16_t zmin = win[0], zmax = win[cnt - 1], zmed = win[(cnt - 1) / 2];
        if (zmed > zmin && zmax > zmed) {
            result = (zxy > zmin && zmax > zxy) ? zxy : zmed;
            break;
        }
        if (k == Smax) result = keep_unresolved ? zxy : zmed;
    }
    free(win);
    return result;
}

/*
 * Contrast stretch (Algorithm 1, step 4e; the post-processing box of the
 * hybrid's architecture figure).  The paper names the step and gives no rule.
 * Reading: a linear stretch between two saturation limits taken from the
 * image's histogram, so that at most k pixels saturate at each end,
 *   k  = floor(fl64(tol * N)),  0 <= tol < 1/2,  N = number of pixels,
 *   lo = the smallest v with #{x <= v} >= k + 1   (the k-th smallest value, from 0),
 *   hi = the smallest v with #{x <= v} >= N - k   (the k-th largest value),
 *   lo == hi:  out = x                            (nothing to stretch),
 *   otherwise  out = floor((clamp(x, lo, hi) - lo) * maxv / (hi - lo) + 1/2)
 * with exact integers (round half up).  tol = 0 is the min-max stretch.
 * lohi (optional) receives lo and hi.
 */
int oracle_contrast(const uint16_t *x, long N, int bits, double tol, uint16_t *out, long *lohi)
{
    if (!x || !out || N < 1 || bits < 1 || bits > 16) return ORACLE_ERR_ARG;
    if (!(tol >= 0.0 && tol < 0.5)) return ORACLE_ERR_ARG;
    const long maxv = (1L << bits) - 1;
    uint64_t *hist = (uint64_t *)calloc((size_t)maxv + 1, sizeof(uint64_t));
    if (!hist) return ORACLE_ERR_OOM;
    for (long i = 0; i < N; ++i) {
        if (x[i] > maxv) {
            free(hist);
            return ORACLE_ERR_ARG;
        }
        hist[x[i]] += 1;
    }
    const uint64_t k = (uint64_t)floor(tol * (double)N);
    const uint64_t t_lo = k + 1, t_hi = (uint64_t)N - k;
    long lo = -1, hi = -1;
    uint64_t cum = 0;
    for (long v = 0; v <= maxv; ++v) {
        cum += hist[v];
        if (lo < 0 && cum >= t_lo) lo = v;
        if (hi < 0 && cum >= t_hi) hi = v;
    }
    free(hist);
    for (long i = 0; i < N; ++i) {
        if (lo == hi) {
            out[i] = x[i];
            continue;
        }
        long c = x[i] < lo ? lo : (x[i] > hi ? hi : x[i]);
        /* floor(p/q + 1/2) = floor((2p + q) / (2q)) for p = (c - lo) * maxv, q = hi - lo */
        const uint64_t p = (uint64_t)(c - lo) * (uint64_t)maxv, q = (uint64_t)(hi - lo);
        out[i] = (uint16_t)((2 * p + q) / (2 * q));
    }
    if (lohi) {
        lohi[0] = lo;
        lohi[1] = hi;
    }
    return ORACLE_OK;
}

/*
 * Noise variance from a clean reference (Algorithm 1, step 4d passes the
 * original image to the Wiener stage; the reading is that it supplies the
 * noise variance): nu2 = mean over pixels of (f - ref)^2, the sum an exact
 * integer, then fl64(fl64(sum) / N).  sum_out (optional) receives the sum.
 */
int oracle_reference_noise_var(const uint16_t *f, const uint16_t *ref, long N, double *nu2, uint64_t *sum_out)
{
    if (!f || !ref || !nu2 || N < 1) return ORACLE_ERR_ARG;
    uint64_t s = 0;
    for (long i = 0; i < N; ++i) {
        const int64_t d = (int64_t)f[i] - (int64_t)ref[i];
        s += (uint64_t)(d * d);
    }
    *nu2 = (double)s / (double)N;
    if (sum_out) *sum_out = s;
    return ORACLE_OK;
}
