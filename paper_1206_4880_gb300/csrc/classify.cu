// Classification kernels: block moments, differential box counting (DBC) local fractal
// dimension and LFD classes (Revathy & Jayamohan, Section 3.1, Eq. 2-3).
//
// DBC reading used throughout the library (the paper cites Sarkar & Chaudhuri without
// restating the estimator): an M x M block with G grey levels is covered by s x s cells,
// s = 2, 4, ..., M/2; a cell contributes floor(max/h) - floor(min/h) + 1 boxes of height
// h = s*G/M; N_s sums the cells; FD is the least-squares slope of log2 N_s against log2(M/s).
// M = 8: s in {2, 4}, FD = log2 N_2 - log2 N_4. Ranges use their pixels (G = 256, h = 64, 128:
// shifts 6 and 7); domains use their contracted block of integer 2x2 sums (G = 1024, shifts 8
// and 9, identical to the 2x2 average with G = 256).
// M = 16: s in {2, 4, 8} at equally spaced abscissae, where the middle point has zero weight and
// FD = (log2 N_2 - log2 N_8) / 2; pixel box heights 32, 64, 128 (shifts 5, 6, 7), sums 128, 256,
// 512 (shifts 7, 8, 9). Counts are stored per block as n_scales(B) consecutive int32.
#include <climits>
#include <cmath>
#include <mutex>

#include "fic_internal.cuh"

namespace fic {

// ------------------------------------------------------------------------------------------
// Host: correctly rounded log2 of small integers in double-double arithmetic (error-free
// transformations of Knuth/Dekker, double-double division as in Hida, Li & Bailey's QD
// library), then rounded to binary64. ln m = 2 atanh((m-1)/(m+1)) for m in [1, 2).
namespace {
struct dd {
    double hi, lo;
};
dd two_sum(double a, double b) {
    double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
dd quick_two_sum(double a, double b) {
    double s = a + b;
    return {s, b - (s - a)};
}
dd two_prod(double a, double b) {
    double p = a * b;
    return {p, std::fma(a, b, -p)};
}
dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}
dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_add(a, dd_neg(dd_mul(b, {q1, 0.0})));
    double q2 = r.hi / b.hi;
    r = dd_add(r, dd_neg(dd_mul(b, {q2, 0.0})));
    double q3 = r.hi / b.hi;
    return dd_add(quick_two_sum(q1, q2), {q3, 0.0});
}
dd dd_ln_mantissa(double m) {  // ln m, m in [1, 2]
    dd z = dd_div({m - 1.0, 0.0}, {m + 1.0, 0.0});
    dd z2 = dd_mul(z, z), term = z, sum = z;
    for (int k = 1; k < 60; ++k) {
        term = dd_mul(term, z2);
        sum = dd_add(sum, dd_div(term, {2.0 * k + 1.0, 0.0}));
    }
    return dd_add(sum, sum);
}
}  // namespace

double log2_correctly_rounded(int n) {
    if (n <= 0) return 0.0;
    int e = 0;
    while ((1 << (e + 1)) <= n) ++e;
    const double m = (double)n / (double)(1 << e);
    static const dd ln2 = dd_ln_mantissa(2.0);
    dd r = dd_add({(double)e, 0.0}, dd_div(dd_ln_mantissa(m), ln2));
    return r.hi;
}

const Log2Tab &log2_table() {
    static Log2Tab tab;
    static std::once_flag once;
    std::call_once(once, [] {
        tab.v[0] = 0.0;
        for (int i = 1; i <= 512; ++i) tab.v[i] = log2_correctly_rounded(i);
    });
    return tab;
}

// ------------------------------------------------------------------------------------------
// Device.
__device__ __forceinline__ double fd_of(const Log2Tab &L, int n2, int n4) {
    return __dsub_rn(L.v[n2], L.v[n4]);
}

// Rows read as 32-bit words when the image base, its pitch and the block's first column are all
// multiples of 4 (strides 4, 8, ... on an aligned image); otherwise byte by byte.
__device__ __forceinline__ bool word_rows(const uint8_t *img, int pitch, int x0) {
    return ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch | (uintptr_t)x0) & 3u) == 0;
}
// Two 2x2 sums from one word of each of two rows (pixels 4k .. 4k + 3), packed as
// (p0 + p1 + q0 + q1) | (p2 + p3 + q2 + q3) << 16; each sum is at most 1020, so no half carries.
__device__ __forceinline__ uint32_t pair_sums(uint32_t a, uint32_t b) {
    return (a & 0x00FF00FFu) + ((a >> 8) & 0x00FF00FFu) + (b & 0x00FF00FFu) + ((b >> 8) & 0x00FF00FFu);
}
// The same two sums from bytes.
__device__ __forceinline__ uint32_t pair_sums_bytes(const uint8_t *r0, const uint8_t *r1) {
    const uint32_t s0 = (uint32_t)__ldg(r0) + __ldg(r0 + 1) + __ldg(r1) + __ldg(r1 + 1);
    const uint32_t s1 = (uint32_t)__ldg(r0 + 2) + __ldg(r0 + 3) + __ldg(r1 + 2) + __ldg(r1 + 3);
    return s0 | (s1 << 16);
}
// n consecutive pixels of one row into v[0 .. n), n a multiple of 4.
template <int N>
__device__ __forceinline__ void load_row(const uint8_t *row, bool words, int *v) {
    if (words) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(row);
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const uint32_t x = __ldg(w + k);
#pragma unroll
            for (int i = 0; i < 4; ++i) v[4 * k + i] = (int)((x >> (8 * i)) & 0xFFu);
        }
    } else {
#pragma unroll
        for (int x = 0; x < N; ++x) v[x] = __ldg(row + x);
    }
}
// The 2x2 sums of rows r0, r1 over 4 M pixels, as M packed pairs.
template <int M>
__device__ __forceinline__ void load_pair_sums(const uint8_t *r0, const uint8_t *r1, bool words, uint32_t *pk) {
    if (words) {
        const uint32_t *w0 = reinterpret_cast<const uint32_t *>(r0), *w1 = reinterpret_cast<const uint32_t *>(r1);
#pragma unroll
        for (int k = 0; k < M; ++k) pk[k] = pair_sums(__ldg(w0 + k), __ldg(w1 + k));
    } else {
#pragma unroll
        for (int k = 0; k < M; ++k) pk[k] = pair_sums_bytes(r0 + 4 * k, r1 + 4 * k);
    }
}

// One thread per range: moments, N_2, N_4 and FD of the 8x8 pixel block.
__device__ __forceinline__ void range_stats(int r, const uint8_t *__restrict__ img, const Geo &g, const Log2Tab &L,
                                            int32_t *__restrict__ rsum, int32_t *__restrict__ rsumsq,
                                            int32_t *__restrict__ rcounts, double *__restrict__ rfd) {
    if (r >= g.R) return;
    const int rq = fdiv(r, g.fRx);
    const int y0 = rq * 8, x0 = (r - rq * g.nRx) * 8;
    const bool words = word_rows(img, g.pitch, x0);
    int v[8][8];
#pragma unroll
    for (int y = 0; y < 8; ++y) load_row<8>(img + (size_t)(y0 + y) * g.pitch + x0, words, v[y]);
    int A = 0, Bs = 0, n2 = 0, n4 = 0;
#pragma unroll
    for (int y = 0; y < 8; ++y)
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            A += v[y][x];
            Bs += v[y][x] * v[y][x];
        }
#pragma unroll
    for (int cy = 0; cy < 8; cy += 2)
#pragma unroll
        for (int cx = 0; cx < 8; cx += 2) {
            int mx = max(max(v[cy][cx], v[cy][cx + 1]), max(v[cy + 1][cx], v[cy + 1][cx + 1]));
            int mn = min(min(v[cy][cx], v[cy][cx + 1]), min(v[cy + 1][cx], v[cy + 1][cx + 1]));
            n2 += (mx >> 6) - (mn >> 6) + 1;
        }
#pragma unroll
    for (int cy = 0; cy < 8; cy += 4)
#pragma unroll
        for (int cx = 0; cx < 8; cx += 4) {
            int mx = 0, mn = 255;
#pragma unroll
            for (int y = 0; y < 4; ++y)
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    mx = max(mx, v[cy + y][cx + x]);
                    mn = min(mn, v[cy + y][cx + x]);
                }
            n4 += (mx >> 7) - (mn >> 7) + 1;
        }
    rsum[r] = A;
    rsumsq[r] = Bs;
    rcounts[2 * r] = n2;
    rcounts[2 * r + 1] = n4;
    rfd[r] = fd_of(L, n2, n4);
}

// One thread per domain: contracted block of 2x2 sums S (kept for packing and exact search),
// C = sum S, E = sum S^2, N_2, N_4, FD; the block's largest FD and the complement of its least
// FD go to extent_bits by atomicMax on the bit patterns (FD > 0, so they order like the values;
// both words start at zero).
__device__ __forceinline__ void dom_stats(int d, const uint8_t *__restrict__ img, const Geo &g, const Log2Tab &L,
                                          uint16_t *__restrict__ domS, int32_t *__restrict__ dsum,
                                          int32_t *__restrict__ dsumsq, int32_t *__restrict__ dcounts,
                                          double *__restrict__ dfd, unsigned long long *extent_bits) {
    unsigned long long fbits_min = ~0ull, fbits_max = 0ull;
    if (d < g.Dn) {
        const int dq = fdiv(d, g.fDx);
        const int y0 = dq * g.sigma, x0 = (d - dq * g.nDx) * g.sigma;
        const bool words = word_rows(img, g.pitch, x0);
        int S[8][8];
        int C = 0, E = 0, n2 = 0, n4 = 0;
        uint4 *dst = reinterpret_cast<uint4 *>(domS + (size_t)d * 64);
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const uint8_t *r0 = img + (size_t)(y0 + 2 * y) * g.pitch + x0;
            uint32_t pk[4];
            load_pair_sums<4>(r0, r0 + g.pitch, words, pk);
            dst[y] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                S[y][2 * k] = (int)(pk[k] & 0xFFFFu);
                S[y][2 * k + 1] = (int)(pk[k] >> 16);
            }
#pragma unroll
            for (int x = 0; x < 8; ++x) {
                C += S[y][x];
                E += S[y][x] * S[y][x];
            }
        }
#pragma unroll
        for (int cy = 0; cy < 8; cy += 2)
#pragma unroll
            for (int cx = 0; cx < 8; cx += 2) {
                int mx = max(max(S[cy][cx], S[cy][cx + 1]), max(S[cy + 1][cx], S[cy + 1][cx + 1]));
                int mn = min(min(S[cy][cx], S[cy][cx + 1]), min(S[cy + 1][cx], S[cy + 1][cx + 1]));
                n2 += (mx >> 8) - (mn >> 8) + 1;
            }
#pragma unroll
        for (int cy = 0; cy < 8; cy += 4)
#pragma unroll
            for (int cx = 0; cx < 8; cx += 4) {
                int mx = 0, mn = 1 << 20;
#pragma unroll
                for (int y = 0; y < 4; ++y)
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        mx = max(mx, S[cy + y][cx + x]);
                        mn = min(mn, S[cy + y][cx + x]);
                    }
                n4 += (mx >> 9) - (mn >> 9) + 1;
            }
        const double f = fd_of(L, n2, n4);
        dsum[d] = C;
        dsumsq[d] = E;
        dcounts[2 * d] = n2;
        dcounts[2 * d + 1] = n4;
        dfd[d] = f;
        fbits_min = fbits_max = (unsigned long long)__double_as_longlong(f);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        fbits_min = min(fbits_min, __shfl_xor_sync(0xffffffffu, fbits_min, off));
        fbits_max = max(fbits_max, __shfl_xor_sync(0xffffffffu, fbits_max, off));
    }
    if ((threadIdx.x & 31) == 0 && fbits_max != 0ull) {
        atomicMax(&extent_bits[0], ~fbits_min);  // the least FD as the largest complement
        atomicMax(&extent_bits[1], fbits_max);
    }
}

// Classes of ranges (i < R) and domains (i >= R): Eq. 2-3 in K equal FD classes.
__global__ void k_bins(Geo g, const double *__restrict__ rfd, const double *__restrict__ dfd,
                       const unsigned long long *__restrict__ extent_bits, double *fd_extent,
                       uint8_t *__restrict__ rbin, uint8_t *__restrict__ dbin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double Fl = __longlong_as_double((long long)~extent_bits[0]);
    const double Fm = __longlong_as_double((long long)extent_bits[1]);
    if (i == 0) {
        fd_extent[0] = Fl;
        fd_extent[1] = Fm;
    }
    if (i >= g.R + g.Dn) return;
    const double f = i < g.R ? rfd[i] : dfd[i - g.R];
    int b = 0;
    if (Fm != Fl) {
        const double t = __dsub_rn(f, Fl);
        const double u = __dsub_rn(Fm, Fl);
        const double v = __ddiv_rn(t, u);
        const double q = floor(__dmul_rn(v, (double)g.K));
        b = q < 0.0 ? 0 : (q > (double)(g.K - 1) ? g.K - 1 : (int)q);
    }
    if (i < g.R)
        rbin[i] = (uint8_t)b;
    else
        dbin[i - g.R] = (uint8_t)b;
}

// ---- B = 16 -----------------------------------------------------------------------------------
__device__ __forceinline__ double fd16_of(const Log2Tab &L, int n2, int n8) {
    return __dmul_rn(__dsub_rn(L.v[n2], L.v[n8]), 0.5);
}

// Box counts of a 16x16 block streamed two rows at a time: the 2x2 cells of each row pair
// complete at once; 4x4 and 8x8 cells gather their 2x2 cells' extremes until they close.
// SH is the box-height shift of s = 2 (5 for pixels, 7 for sums); s = 4, 8 use SH + 1, SH + 2.
template <int SH>
struct Dbc16 {
    int n2 = 0, n4 = 0, n8 = 0;
    int mx4[4], mn4[4], mx8[2], mn8[2];
    __device__ __forceinline__ void reset4() {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            mx4[k] = INT_MIN;
            mn4[k] = INT_MAX;
        }
    }
    __device__ __forceinline__ void reset8() {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            mx8[k] = INT_MIN;
            mn8[k] = INT_MAX;
        }
    }
    // rows a[16], b[16] of row pair p (0..7)
    __device__ __forceinline__ void row_pair(int p, const int *a, const int *b) {
        if ((p & 1) == 0) reset4();
        if ((p & 3) == 0) reset8();
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int mx = max(max(a[2 * c], a[2 * c + 1]), max(b[2 * c], b[2 * c + 1]));
            const int mn = min(min(a[2 * c], a[2 * c + 1]), min(b[2 * c], b[2 * c + 1]));
            n2 += (mx >> SH) - (mn >> SH) + 1;
            mx4[c >> 1] = max(mx4[c >> 1], mx);
            mn4[c >> 1] = min(mn4[c >> 1], mn);
            mx8[c >> 2] = max(mx8[c >> 2], mx);
            mn8[c >> 2] = min(mn8[c >> 2], mn);
        }
        if (p & 1)
#pragma unroll
            for (int k = 0; k < 4; ++k) n4 += (mx4[k] >> (SH + 1)) - (mn4[k] >> (SH + 1)) + 1;
        if ((p & 3) == 3)
#pragma unroll
            for (int k = 0; k < 2; ++k) n8 += (mx8[k] >> (SH + 2)) - (mn8[k] >> (SH + 2)) + 1;
    }
};

// One thread per 16x16 range.
__device__ __forceinline__ void range_stats16(int r, const uint8_t *__restrict__ img, const Geo &g,
                                              const Log2Tab &L, int32_t *__restrict__ rsum,
                                              int32_t *__restrict__ rsumsq, int32_t *__restrict__ rcounts,
                                              double *__restrict__ rfd) {
    if (r >= g.R) return;
    const int rq = fdiv(r, g.fRx);
    const int y0 = rq * 16, x0 = (r - rq * g.nRx) * 16;
    const bool words = word_rows(img, g.pitch, x0);
    Dbc16<5> dbc;
    int A = 0, Bs = 0;
    for (int p = 0; p < 8; ++p) {
        int a[16], b[16];
        const uint8_t *r0 = img + (size_t)(y0 + 2 * p) * g.pitch + x0;
        load_row<16>(r0, words, a);
        load_row<16>(r0 + g.pitch, words, b);
#pragma unroll
        for (int x = 0; x < 16; ++x) {
            A += a[x] + b[x];
            Bs += a[x] * a[x] + b[x] * b[x];
        }
        dbc.row_pair(p, a, b);
    }
    rsum[r] = A;
    rsumsq[r] = Bs;
    rcounts[3 * r] = dbc.n2;
    rcounts[3 * r + 1] = dbc.n4;
    rcounts[3 * r + 2] = dbc.n8;
    rfd[r] = fd16_of(L, dbc.n2, dbc.n8);
}

// One thread per 32x32 domain: its 16x16 block of 2x2 sums S (stored), C, E, counts and FD; the
// FD extent as in dom_stats.
__device__ __forceinline__ void dom_stats16(int d, const uint8_t *__restrict__ img, const Geo &g,
                                            const Log2Tab &L, uint16_t *__restrict__ domS,
                                            int32_t *__restrict__ dsum, int32_t *__restrict__ dsumsq,
                                            int32_t *__restrict__ dcounts, double *__restrict__ dfd,
                                            unsigned long long *extent_bits) {
    unsigned long long fbits_min = ~0ull, fbits_max = 0ull;
    if (d < g.Dn) {
        const int dq = fdiv(d, g.fDx);
        const int y0 = dq * g.sigma, x0 = (d - dq * g.nDx) * g.sigma;
        const bool words = word_rows(img, g.pitch, x0);
        Dbc16<7> dbc;
        int C = 0, E = 0;
        uint4 *dst = reinterpret_cast<uint4 *>(domS + (size_t)d * 256);
        for (int p = 0; p < 8; ++p) {
            int a[16], b[16];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int *S = h ? b : a;
                const uint8_t *q0 = img + (size_t)(y0 + 4 * p + 2 * h) * g.pitch + x0;
                uint32_t pk[8];
                load_pair_sums<8>(q0, q0 + g.pitch, words, pk);
                dst[(2 * p + h) * 2] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                dst[(2 * p + h) * 2 + 1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    S[2 * k] = (int)(pk[k] & 0xFFFFu);
                    S[2 * k + 1] = (int)(pk[k] >> 16);
                }
#pragma unroll
                for (int x = 0; x < 16; ++x) {
                    C += S[x];
                    E += S[x] * S[x];
                }
            }
            dbc.row_pair(p, a, b);
        }
        const double f = fd16_of(L, dbc.n2, dbc.n8);
        dsum[d] = C;
        dsumsq[d] = E;
        dcounts[3 * d] = dbc.n2;
        dcounts[3 * d + 1] = dbc.n4;
        dcounts[3 * d + 2] = dbc.n8;
        dfd[d] = f;
        fbits_min = fbits_max = (unsigned long long)__double_as_longlong(f);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        fbits_min = min(fbits_min, __shfl_xor_sync(0xffffffffu, fbits_min, off));
        fbits_max = max(fbits_max, __shfl_xor_sync(0xffffffffu, fbits_max, off));
    }
    if ((threadIdx.x & 31) == 0 && fbits_max != 0ull) {
        atomicMax(&extent_bits[0], ~fbits_min);  // the least FD as the largest complement
        atomicMax(&extent_bits[1], fbits_max);
    }
}

// Range and domain statistics in one launch: blocks [0, nbr) take 128 ranges each, the rest 128
// domains each (whole blocks, so the domain blocks' warp reductions see full warps).
template <int B>
__global__ void __launch_bounds__(128) k_block_stats(const uint8_t *__restrict__ img, Geo g, Log2Tab L, int nbr,
                                                     int32_t *__restrict__ rsum, int32_t *__restrict__ rsumsq,
                                                     int32_t *__restrict__ rcounts, double *__restrict__ rfd,
                                                     uint16_t *__restrict__ domS, int32_t *__restrict__ dsum,
                                                     int32_t *__restrict__ dsumsq, int32_t *__restrict__ dcounts,
                                                     double *__restrict__ dfd, unsigned long long *extent_bits) {
    if ((int)blockIdx.x < nbr) {
        const int r = blockIdx.x * 128 + threadIdx.x;
        if (B == 16)
            range_stats16(r, img, g, L, rsum, rsumsq, rcounts, rfd);
        else
            range_stats(r, img, g, L, rsum, rsumsq, rcounts, rfd);
    } else {
        const int d = (blockIdx.x - nbr) * 128 + threadIdx.x;
        if (B == 16)
            dom_stats16(d, img, g, L, domS, dsum, dsumsq, dcounts, dfd, extent_bits);
        else
            dom_stats(d, img, g, L, domS, dsum, dsumsq, dcounts, dfd, extent_bits);
    }
}

cudaError_t launch_classify(const uint8_t *img, const Geo &g, const EncodeBufs &b,
                            cudaStream_t st) {
    const Log2Tab &L = log2_table();
    // extent_bits = {complement of the least FD's bits, the largest FD's bits}, both reduced by
    // atomicMax from zero: the caller zeroes them with the image's counters
    const int nbr = (g.R + 127) / 128, nbd = (g.Dn + 127) / 128;
    if (g.B == 16)
        k_block_stats<16><<<nbr + nbd, 128, 0, st>>>(img, g, L, nbr, b.range_sum, b.range_sumsq, b.range_counts,
                                                     b.range_fd, b.dom_S, b.dom_sum, b.dom_sumsq, b.dom_counts,
                                                     b.dom_fd, b.extent_bits);
    else
        k_block_stats<8><<<nbr + nbd, 128, 0, st>>>(img, g, L, nbr, b.range_sum, b.range_sumsq, b.range_counts,
                                                    b.range_fd, b.dom_S, b.dom_sum, b.dom_sumsq, b.dom_counts,
                                                    b.dom_fd, b.extent_bits);
    ++g_launches;
    const int n = g.R + g.Dn;
    k_bins<<<(n + 255) / 256, 256, 0, st>>>(g, b.range_fd, b.dom_fd, b.extent_bits, b.fd_extent,
                                            b.range_bin, b.dom_bin);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
