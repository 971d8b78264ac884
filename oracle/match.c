/*
 * CPU oracle: exact best-match search of classified range-domain matching.
 *
 * TEST INFRASTRUCTURE ONLY. Called from the oracle's Python side (oracle/match.py), which the
 * tests, __graft_entry__.smoke() and bench.py's CPU baseline use. It shares no code with the
 * CUDA library.
 *
 * What it computes (Revathy & Jayamohan, Section 1 and Section 3):
 *   for every listed range r and every domain d of its pool (given explicitly, ascending) and
 *   every square isometry t (0..7), fit r ~ s * T_t(S_d / 4) + o by least squares with
 *   |s| <= 1, and keep the candidate of least collage error SSE. Ties go to the smaller domain
 *   index, then the smaller isometry index (the scan order is ascending d, then t, and only a
 *   strictly smaller SSE replaces the incumbent).
 *
 * With n = B*B, A = sum r, Bs = sum r^2, C = sum S, E = sum S^2, X = sum r * T_t(S),
 * P = n X - A C and Q = n E - C^2, the least-squares contrast is s = 4P/Q and
 *   16 n SSE = 16 (n Bs - A^2) - gain,
 *   gain = 16 P^2 / Q          if Q > 0 and 4|P| <= Q   (unclamped),
 *   gain = 8 |P| - Q           if 4|P| > Q              (s clamped to sign(P)),
 *   gain = 0                   if Q == 0                (flat domain: s = 0).
 * Least SSE is greatest gain; gains are compared exactly as fractions with 128-bit integers.
 * Outputs are converted to binary64 only at the end.
 *
 * Domain d has its top-left pixel at ((d / nDx) * sigma, (d % nDx) * sigma) and is contracted
 * by 2x2 sums; ranges are row-major B x B tiles. Isometries as in oracle/geometry.py.
 */
#include <stdint.h>
#include <stdlib.h>

typedef __int128 i128;

typedef struct {
    i128 num; /* gain = num / den, den > 0 */
    i128 den;
} gain_t;

static int gain_greater(gain_t a, gain_t b) { return a.num * b.den > b.num * a.den; }

static void iso_source(int B, int t, int y, int x, int *sy, int *sx) {
    int N = B - 1;
    switch (t) {
    case 0: *sy = y;     *sx = x;     break;
    case 1: *sy = N - x; *sx = y;     break;
    case 2: *sy = N - y; *sx = N - x; break;
    case 3: *sy = x;     *sx = N - y; break;
    case 4: *sy = y;     *sx = N - x; break;
    case 5: *sy = N - y; *sx = x;     break;
    case 6: *sy = x;     *sx = y;     break;
    default:*sy = N - x; *sx = N - y; break;
    }
}

/* Returns 0 on success, -1 on an argument error. */
int oracle_match(const uint8_t *img, int64_t pitch, int H, int W, int B, int sigma,
                 int64_t n_list, const int64_t *range_ids,
                 const int64_t *pool_ptr, const int32_t *pool_dom,
                 int32_t *out_dom, int32_t *out_iso, double *out_s, double *out_o,
                 double *out_sse, int n_threads) {
    if (B != 8 && B != 16) return -1;
    if (sigma < 1 || H < 2 * B || W < 2 * B || H % B || W % B || pitch < W) return -1;
    const int nDy = (H - 2 * B) / sigma + 1, nDx = (W - 2 * B) / sigma + 1;
    const int64_t Dn = (int64_t)nDy * nDx;
    const int64_t R = (int64_t)(H / B) * (W / B);
    const int n = B * B;
    for (int64_t i = 0; i < n_list; ++i) {
        if (range_ids[i] < 0 || range_ids[i] >= R) return -1;
        if (pool_ptr[i + 1] < pool_ptr[i]) return -1;
        for (int64_t k = pool_ptr[i]; k < pool_ptr[i + 1]; ++k)
            if (pool_dom[k] < 0 || pool_dom[k] >= Dn) return -1;
    }
    (void)n_threads;

#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
    for (int64_t i = 0; i < n_list; ++i) {
        const int64_t r = range_ids[i];
        const int ry = (int)(r / (W / B)) * B, rx = (int)(r % (W / B)) * B;
        int64_t rb[16][16], S[16][16];
        int64_t A = 0, Bs = 0;
        for (int y = 0; y < B; ++y)
            for (int x = 0; x < B; ++x) {
                rb[y][x] = img[(int64_t)(ry + y) * pitch + rx + x];
                A += rb[y][x];
                Bs += rb[y][x] * rb[y][x];
            }
        int have = 0;
        gain_t best = {0, 1};
        int32_t best_d = -1, best_t = 0;
        int64_t best_P = 0, best_Q = 0, best_C = 0;
        for (int64_t k = pool_ptr[i]; k < pool_ptr[i + 1]; ++k) {
            const int32_t d = pool_dom[k];
            const int dy = (d / nDx) * sigma, dx = (d % nDx) * sigma;
            int64_t C = 0, E = 0;
            for (int y = 0; y < B; ++y)
                for (int x = 0; x < B; ++x) {
                    const uint8_t *p = img + (int64_t)(dy + 2 * y) * pitch + dx + 2 * x;
                    S[y][x] = (int64_t)p[0] + p[1] + p[pitch] + p[pitch + 1];
                    C += S[y][x];
                    E += S[y][x] * S[y][x];
                }
            const int64_t Q = (int64_t)n * E - C * C;
            for (int t = 0; t < 8; ++t) {
                int64_t X = 0;
                for (int y = 0; y < B; ++y)
                    for (int x = 0; x < B; ++x) {
                        int sy, sx;
                        iso_source(B, t, y, x, &sy, &sx);
                        X += rb[y][x] * S[sy][sx];
                    }
                const int64_t P = (int64_t)n * X - A * C;
                const int64_t absP = P < 0 ? -P : P;
                gain_t g;
                if (Q == 0) {
                    g.num = 0;
                    g.den = 1;
                } else if (4 * absP <= Q) {
                    g.num = (i128)16 * (i128)P * (i128)P;
                    g.den = Q;
                } else {
                    g.num = (i128)8 * absP - Q;
                    g.den = 1;
                }
                if (!have || gain_greater(g, best)) {
                    have = 1;
                    best = g;
                    best_d = d;
                    best_t = t;
                    best_P = P;
                    best_Q = Q;
                    best_C = C;
                }
            }
        }
        double s = 0.0, o = 0.0, sse = 0.0;
        if (have) {
            if (best_Q == 0) {
                s = 0.0;
            } else if (4 * (best_P < 0 ? -best_P : best_P) <= best_Q) {
                s = (4.0 * (double)best_P) / (double)best_Q;
            } else {
                s = best_P > 0 ? 1.0 : -1.0;
            }
            o = ((double)A - s * ((double)best_C / 4.0)) / (double)n;
            /* SSE = (16 (n Bs - A^2) den - num) / (16 n den) */
            const i128 base = (i128)16 * ((i128)n * Bs - (i128)A * A);
            const i128 num = base * best.den - best.num;
            sse = (double)num / ((double)16.0 * (double)n * (double)best.den);
        }
        out_dom[i] = best_d;
        out_iso[i] = best_t;
        out_s[i] = s;
        out_o[i] = o;
        out_sse[i] = sse;
    }
    return 0;
}
