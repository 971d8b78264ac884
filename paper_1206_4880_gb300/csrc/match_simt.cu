// Exact range-domain matching on CUDA cores: the plain GPU search (every domain of every pool),
// and the exact re-search of the few ranges the tensor engine's ranking could not certify
// (restricted to the domain chunks that could still hold the winner).
//
// For a range r, a domain d of its pool (Section 3.1 Eq. 3) and an isometry t, the correlation
// X_t = sum_p r[p] * (T_t S_d)[p] is formed exactly in 32-bit integers (packed byte x halfword
// dot products), then P = n X - A C and Q = n E - C^2 give the exact least-squares gain
// (Section 1's intensity map with |s| <= 1); the best (gain, -d, -t) wins.
//
// One CTA per range: the range's 8 inverse-permuted copies sit in shared memory, each thread
// walks every 256th domain, and a shared-memory tree picks the block's best.
#include <climits>

#include "fic_internal.cuh"

namespace fic {

namespace {

constexpr int kSimtThreads = 256;

template <int B>
struct ScanShared {
    using G = typename FitOf<B>::G;
    // rp[t][q] = r[p] with src_t(p) = q, so that X_t = sum_q S[q] * rp[t][q]; bytes, 16-aligned
    alignas(16) uint8_t rp[8][B * B];
    // per warp: its best candidate (the block reduction's second level)
    G g[kSimtThreads / 32];
    long long P[kSimtThreads / 32], Q[kSimtThreads / 32];
    int d[kSimtThreads / 32], t[kSimtThreads / 32], C[kSimtThreads / 32];
    int flagged[kSimtThreads];
    int single[2 * kSimtThreads];  // first positions of flagged 16-domain groups
    int n_flagged, n_single;
    float thr;
};

template <int B>
struct Best {
    typename FitOf<B>::G g;
    int d, t, C;
    long long P, Q;
};

template <int B>
__device__ __forceinline__ void load_range(ScanShared<B> &sh, const Geo &g, const uint8_t *img, int r) {
    for (int p = threadIdx.x; p < B * B; p += kSimtThreads) {
        const int y = p / B, x = p % B;
        const int ry = (r / g.nRx) * B, rx = (r % g.nRx) * B;
        const uint8_t v = img[(size_t)(ry + y) * g.pitch + rx + x];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int sy, sx;
            iso_src(B, t, y, x, sy, sx);
            sh.rp[t][sy * B + sx] = v;
        }
    }
}

// Exact evaluation of domain d under all 8 isometries against the range in sh.rp (corr8), kept
// in b if it is better (gain, then smaller domain id, then smaller isometry).
template <int B>
__device__ __forceinline__ void scan_domain(const ScanShared<B> &sh, int d, long long A,
                                            const uint16_t *__restrict__ domS,
                                            const int32_t *__restrict__ dsum,
                                            const int32_t *__restrict__ dsumsq, Best<B> &b) {
    constexpr int n = B * B;
    unsigned X[8];
    corr8<B>(sh.rp, domS + (size_t)d * n, X);
    const long long C = dsum[d];
    const long long Q = (long long)n * dsumsq[d] - C * C;
    // with the domain fixed the clamped gain grows with |P|: its best isometry is the largest
    // |P|, ties to the smaller t; one exact gain and one comparison per domain
    long long P = (long long)n * (long long)X[0] - A * C, aP = P < 0 ? -P : P;
    int bt = 0;
#pragma unroll
    for (int t = 1; t < 8; ++t) {
        const long long Pt = (long long)n * (long long)X[t] - A * C;
        const long long at = Pt < 0 ? -Pt : Pt;
        if (at > aP) {
            aP = at;
            bt = t;
            P = Pt;
        }
    }
    const auto gg = FitOf<B>::gain(P, Q);
    if (cand_better(gg, d, bt, b.g, b.d, b.t)) {
        b.g = gg;
        b.d = d;
        b.t = bt;
        b.P = P;
        b.Q = Q;
        b.C = (int)C;
    }
}

// A warp's lane-wise best values exchanged over xor lane offsets.
__device__ __forceinline__ Gain shfl_xor_gain(const Gain &g, int off) {
    return Gain{__shfl_xor_sync(0xffffffffu, g.num, off), __shfl_xor_sync(0xffffffffu, g.den, off)};
}
__device__ __forceinline__ GainW shfl_xor_gain(const GainW &g, int off) {
    GainW o;
    const unsigned long long lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)g.num, off);
    const long long hi = __shfl_xor_sync(0xffffffffu, (long long)(g.num >> 64), off);
    o.num = (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | (unsigned __int128)lo);
    o.den = __shfl_xor_sync(0xffffffffu, g.den, off);
    return o;
}
// The best of a warp's 32 candidates (gain, then smaller domain id, then smaller isometry), in
// every lane.
template <int B>
__device__ __forceinline__ void warp_best(Best<B> &b) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        Best<B> o;
        o.g = shfl_xor_gain(b.g, off);
        o.d = __shfl_xor_sync(0xffffffffu, b.d, off);
        o.t = __shfl_xor_sync(0xffffffffu, b.t, off);
        o.C = __shfl_xor_sync(0xffffffffu, b.C, off);
        o.P = __shfl_xor_sync(0xffffffffu, b.P, off);
        o.Q = __shfl_xor_sync(0xffffffffu, b.Q, off);
        if (cand_better(o.g, o.d, o.t, b.g, b.d, b.t)) b = o;
    }
}

// Block-wide best and the code of range r (thread 0 writes it): each warp's best by shuffles,
// then the warps' bests by the first warp.
template <int B>
__device__ __forceinline__ void reduce_and_write(ScanShared<B> &sh, const Best<B> &b, int r, long long A,
                                                 long long Bs, const fic_codes &out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Best<B> m = b;
    warp_best<B>(m);
    if (lane == 0) {
        sh.g[warp] = m.g;
        sh.d[warp] = m.d;
        sh.t[warp] = m.t;
        sh.P[warp] = m.P;
        sh.Q[warp] = m.Q;
        sh.C[warp] = m.C;
    }
    __syncthreads();
    if (warp == 0) {
        Best<B> x = m;
        if (lane < kSimtThreads / 32) {
            x = Best<B>{sh.g[lane], sh.d[lane], sh.t[lane], sh.C[lane], sh.P[lane], sh.Q[lane]};
        } else {
            x.g.num = -1;  // no candidate
            x.g.den = 1;
            x.d = INT_MAX;
            x.t = 0;
        }
        warp_best<B>(x);
        if (lane == 0) {
            double s, o, sse;
            finalize_code(B * B, A, Bs, x.C, x.P, x.Q, x.g, s, o, sse);
            out.dom[r] = x.d;
            out.iso[r] = x.t;
            out.s[r] = s;
            out.o[r] = o;
            out.sse[r] = sse;
        }
    }
    __syncthreads();
}

// A chunk key's bound reaches the re-search threshold: score * (1 + 2^-13) + 2^-16 >= thr,
// evaluated rounded up (thr itself is rounded down), so no chunk that exact arithmetic would flag
// is missed.
__device__ __forceinline__ bool reaches(uint32_t score_bits, float thr) {
    return __fmaf_ru(__uint_as_float(score_bits), 1.0f + 1.0f / 8192.0f, 1.0f / 65536.0f) >= thr;
}

template <class G>
__device__ __forceinline__ G no_gain() {
    G g;
    g.num = -1;
    g.den = 1;
    return g;
}

}  // namespace

// Plain search: CTA r scans the whole pool of range r.
template <int B>
__global__ void __launch_bounds__(kSimtThreads)
    k_match_simt(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
                 const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
                 const int32_t *__restrict__ rsum, const int32_t *__restrict__ rsumsq,
                 const int32_t *__restrict__ dom_order, const int32_t *__restrict__ win_lo,
                 const int32_t *__restrict__ win_hi, fic_codes out) {
    __shared__ __align__(16) ScanShared<B> sh;
    const int r = blockIdx.x;
    load_range<B>(sh, g, img, r);
    __syncthreads();
    const long long A = rsum[r], Bs = rsumsq[r];
    Best<B> b{no_gain<typename FitOf<B>::G>(), INT_MAX, 0, 0, 0, 0};
    for (int j = win_lo[r] + threadIdx.x; j < win_hi[r]; j += kSimtThreads)
        scan_domain<B>(sh, dom_order[j], A, domS, dsum, dsumsq, b);
    reduce_and_write<B>(sh, b, r, A, Bs, out);
}

// Re-search of uncertified ranges of one image. Slot k holds class-sorted position fb_pos[k] and
// the exact best of its evaluated candidates; the 512-domain chunks of the range's tile whose best
// FP32 score could still reach that best (score * (1 + 2^-13) + 2^-16 >= best gain / (8 n), less
// 2^-16 sqrt(64 sum r^2 - A^2) for 8x8 ranges: the bound the re-evaluation certifies with) are
// scanned exactly. TM ranges per tile, H key columns
// per row (chunk_max layout [chunk][TM][H] of (best key, runner-up score bits)).
template <int B, int TM, int H>
__global__ void __launch_bounds__(kSimtThreads, 2)
    k_rescan(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
             const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
             const int32_t *__restrict__ rsumsq, const int32_t *__restrict__ dom_order,
             const int4 *__restrict__ rng_info, int rng_off, int dom_off, const int4 *__restrict__ tile_win,
             const int4 *__restrict__ tile_items, const uint32_t *__restrict__ chunk_max,
             const int32_t *__restrict__ fb_pos, const FallbackBest *__restrict__ fb_best,
             const int32_t *__restrict__ counters, fic_codes out) {
    __shared__ __align__(16) ScanShared<B> sh;
    using G = typename FitOf<B>::G;
    const int n = min(counters[0], g.R);
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int i = fb_pos[k];
        const int4 ri = rng_info[i];
        const int r = ri.w;
        load_range<B>(sh, g, img, r);
        __syncthreads();
        const FallbackBest fb = fb_best[k];
        G g0;
        g0.num = fb.num;
        g0.den = fb.den;
        Best<B> b{g0, fb.d, fb.t, fb.C, fb.P, fb.Q};
        // chunks are flagged when score * (1 + 2^-13) + 2^-16 >= best gain / (8 n), evaluated in
        // FP32 with the left side rounded up and the threshold rounded down (so a superset of the
        // exactly flagged chunks; the FP64 threshold's own rounding, 2^-52 relatively, lies well
        // inside the margin's slack). One thread forms the threshold: FP64 throughput is low.
        const long long A = ri.x, Bs = rsumsq[r];
        // with 8x8 ranges the score's own rounding adds 2^-16 sqrt(64 Bs - A^2) to the bound
        // (k_match_tc); moving it to the threshold's side keeps the flag test one FMA
        if (threadIdx.x == 0) {
            double thr = __ddiv_rn(i128_to_double_rn(fb.num), 8.0 * B * B * (double)fb.den);
            if (B == 8) thr -= (double)__fsqrt_ru(__ll2float_ru(64LL * Bs - A * A)) * (1.0 / 65536.0);
            sh.thr = fb.num < 0 ? -1.0f : __double2float_rd(thr);
        }
        const int ig = rng_off + i, row = ig % TM;
        const int4 tw = tile_win[ig / TM];
        const int4 ti = tile_items[ig / TM];
        const int nch = ti.w;
        const int c_lo = tw.x / kChunkDom;  // the tile's first chunk of the absolute grid
        // the chunks, 256 at a time in parallel: a key column whose runner-up group score reaches
        // the threshold has its whole chunk scanned; one whose best group score alone reaches it
        // contributes only that 16-domain group (every domain outside it scores at most the
        // runner-up); then all threads scan the flagged chunks' and groups' domains
        for (int base = 0; base < nch; base += kSimtThreads) {
            if (threadIdx.x == 0) sh.n_flagged = sh.n_single = 0;
            __syncthreads();
            const float thr = sh.thr;
            const int c = base + threadIdx.x;
            if (c < nch) {
                const uint2 *e = reinterpret_cast<const uint2 *>(chunk_max) + ((size_t)(ti.z + c) * TM + row) * H;
                uint2 k[H];  // (best key, runner-up score bits) per half
                bool full = false;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    k[h] = e[h];
                    full = full || (k[h].y != 0 && reaches(k[h].y, thr));
                }
                if (full) {
                    sh.flagged[atomicAdd(&sh.n_flagged, 1)] = c;
                } else {
#pragma unroll
                    for (int h = 0; h < H; ++h)
                        if (k[h].x != 0 && reaches(k[h].x & 0xFFFFFE00u, thr))
                            sh.single[atomicAdd(&sh.n_single, 1)] =
                                ((c + c_lo) * kChunkDom + 511 - (int)(k[h].x & 511u)) & ~15;
                }
            }
            __syncthreads();
            const int nf = sh.n_flagged, nsg = sh.n_single;
            // every position of the flagged chunks, then of the flagged groups, as one sequence that
            // each thread walks with stride kSimtThreads; the next domain's id is loaded while the
            // current domain is scanned, so a domain costs one dependent load round instead of two
            auto pos_at = [&](int u) -> int {  // u-th position of the sequence, or -1 (outside the pool)
                if (u < nf * kChunkDom) {
                    const int j = (sh.flagged[u / kChunkDom] + c_lo) * kChunkDom + u % kChunkDom;
                    return (j >= ri.y && j < ri.z) ? j : -1;
                }
                u -= nf * kChunkDom;
                const int j = sh.single[u >> 4] + (u & 15);
                return (j >= ri.y && j < ri.z) ? j : -1;
            };
            const int total = nf * kChunkDom + 16 * nsg;
            int u = threadIdx.x, j = u < total ? pos_at(u) : -1;
            int d = j >= 0 ? dom_order[j - dom_off] : -1;
            while (u < total) {
                const int un = u + kSimtThreads;
                const int jn = un < total ? pos_at(un) : -1;
                const int dn = jn >= 0 ? dom_order[jn - dom_off] : -1;
                if (d >= 0) scan_domain<B>(sh, d, A, domS, dsum, dsumsq, b);
                u = un;
                d = dn;
            }
            __syncthreads();
        }
        reduce_and_write<B>(sh, b, r, A, Bs, out);
    }
}

cudaError_t launch_match_simt(const uint8_t *img, const Geo &g, const EncodeBufs &b,
                              const fic_codes &out, cudaStream_t st) {
    if (g.B == 16)
        k_match_simt<16><<<g.R, kSimtThreads, 0, st>>>(g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sum,
                                                       b.range_sumsq, b.dom_order, b.win_lo, b.win_hi, out);
    else
        k_match_simt<8><<<g.R, kSimtThreads, 0, st>>>(g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sum,
                                                      b.range_sumsq, b.dom_order, b.win_lo, b.win_hi, out);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_rescan(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                          const fic_codes &out, int num_sms, cudaStream_t st) {
    if (g.B == 16)
        k_rescan<16, 2 * kTileM, 1><<<8 * num_sms, kSimtThreads, 0, st>>>(
            g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sumsq, b.dom_order, b.rng_info, b.rng_off, b.dom_off,
            tb.tile_win, tb.tile_items, tb.chunk_max, b.fallback, b.fb_best, b.counters, out);
    else
        k_rescan<8, kTileM, 2><<<8 * num_sms, kSimtThreads, 0, st>>>(
            g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sumsq, b.dom_order, b.rng_info, b.rng_off, b.dom_off,
            tb.tile_win, tb.tile_items, tb.chunk_max, b.fallback, b.fb_best, b.counters, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
