// Classification kernels: block moments, differential box counting (DBC) local fractal
// dimension and LFD classes (Revathy & Jayamohan, Section 3.1, Eq. 2-3).
//
// DBC reading used throughout the library (the paper cites Sarkar & Chaudhuri without
// restating the estimator): an 8x8 block with G grey levels is covered by s x s cells,
// s in {2, 4}; a cell contributes floor(max/h) - floor(min/h) + 1 boxes of height
// h = s*G/8; N_s sums the cells; FD = log2 N_2 - log2 N_4 (the least-squares slope of
// log N_s against log(8/s) through two points). Ranges use their pixels (G = 256, h = 64, 128:
// shifts 6 and 7); domains use their contracted block of integer 2x2 sums (G = 1024, shifts 8
// and 9, identical to the 2x2 average with G = 256).
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
        for (int i = 1; i <= 64; ++i) tab.v[i] = log2_correctly_rounded(i);
    });
    return tab;
}

// ------------------------------------------------------------------------------------------
// Device.
__device__ __forceinline__ double fd_of(const Log2Tab &L, int n2, int n4) {
    return __dsub_rn(L.v[n2], L.v[n4]);
}

// One thread per range: moments, N_2, N_4 and FD of the 8x8 pixel block.
__global__ void k_range_stats(const uint8_t *__restrict__ img, Geo g, Log2Tab L,
                              int32_t *__restrict__ rsum, int32_t *__restrict__ rsumsq,
                              int32_t *__restrict__ rcounts, double *__restrict__ rfd) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.R) return;
    const int y0 = (r / g.nRx) * 8, x0 = (r % g.nRx) * 8;
    int v[8][8];
#pragma unroll
    for (int y = 0; y < 8; ++y) {
        const uint8_t *row = img + (size_t)(y0 + y) * g.pitch + x0;
#pragma unroll
        for (int x = 0; x < 8; ++x) v[y][x] = __ldg(row + x);
    }
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
// C = sum S, E = sum S^2, N_2, N_4, FD; the block's least/largest FD go to extent_bits by
// atomic min/max on the bit patterns (FD > 0, so they order like the values).
__global__ void k_dom_stats(const uint8_t *__restrict__ img, Geo g, Log2Tab L,
                            uint16_t *__restrict__ domS, int32_t *__restrict__ dsum,
                            int32_t *__restrict__ dsumsq, int32_t *__restrict__ dcounts,
                            double *__restrict__ dfd, unsigned long long *extent_bits) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long fbits_min = ~0ull, fbits_max = 0ull;
    if (d < g.Dn) {
        const int y0 = (d / g.nDx) * g.sigma, x0 = (d % g.nDx) * g.sigma;
        int S[8][8];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const uint8_t *r0 = img + (size_t)(y0 + 2 * y) * g.pitch + x0;
            const uint8_t *r1 = r0 + g.pitch;
#pragma unroll
            for (int x = 0; x < 8; ++x)
                S[y][x] = (int)__ldg(r0 + 2 * x) + __ldg(r0 + 2 * x + 1) + __ldg(r1 + 2 * x) +
                          __ldg(r1 + 2 * x + 1);
        }
        int C = 0, E = 0, n2 = 0, n4 = 0;
        uint4 *dst = reinterpret_cast<uint4 *>(domS + (size_t)d * 64);
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            uint4 pk;
            pk.x = (uint32_t)S[y][0] | ((uint32_t)S[y][1] << 16);
            pk.y = (uint32_t)S[y][2] | ((uint32_t)S[y][3] << 16);
            pk.z = (uint32_t)S[y][4] | ((uint32_t)S[y][5] << 16);
            pk.w = (uint32_t)S[y][6] | ((uint32_t)S[y][7] << 16);
            dst[y] = pk;
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
        atomicMin(&extent_bits[0], fbits_min);
        atomicMax(&extent_bits[1], fbits_max);
    }
}

// Classes of ranges (i < R) and domains (i >= R): Eq. 2-3 in K equal FD classes.
__global__ void k_bins(Geo g, const double *__restrict__ rfd, const double *__restrict__ dfd,
                       const unsigned long long *__restrict__ extent_bits, double *fd_extent,
                       uint8_t *__restrict__ rbin, uint8_t *__restrict__ dbin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double Fl = __longlong_as_double((long long)extent_bits[0]);
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

cudaError_t launch_classify(const uint8_t *img, const Geo &g, const EncodeBufs &b,
                            cudaStream_t st) {
    const Log2Tab &L = log2_table();
    cudaError_t e;
    // extent_bits[0] = all ones (min identity), extent_bits[1] = 0 (max identity)
    if ((e = cudaMemsetAsync(b.extent_bits, 0xff, sizeof(unsigned long long), st))) return e;
    if ((e = cudaMemsetAsync(b.extent_bits + 1, 0, sizeof(unsigned long long), st))) return e;
    k_range_stats<<<(g.R + 127) / 128, 128, 0, st>>>(img, g, L, b.range_sum, b.range_sumsq,
                                                     b.range_counts, b.range_fd);
    ++g_launches;
    k_dom_stats<<<(g.Dn + 127) / 128, 128, 0, st>>>(img, g, L, b.dom_S, b.dom_sum, b.dom_sumsq,
                                                    b.dom_counts, b.dom_fd, b.extent_bits);
    ++g_launches;
    const int n = g.R + g.Dn;
    k_bins<<<(n + 255) / 256, 256, 0, st>>>(g, b.range_fd, b.dom_fd, b.extent_bits, b.fd_extent,
                                            b.range_bin, b.dom_bin);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
