// Exact range-domain matching on CUDA cores: the plain GPU search (every domain of every pool),
// and the exact re-search of the few ranges the tensor engine's ranking could not certify
// (restricted to the domain chunks that could still hold the winner).
//
// For a range r, a domain d of its pool (Section 3.1 Eq. 3) and an isometry t, the correlation
// X_t = sum_p r[p] * (T_t S_d)[p] is formed exactly (integer products <= 255*1020 and sums
// < 2^24 are exact in FP32 FMA), then P = 64 X - A C and Q = 64 E - C^2 give the exact
// least-squares gain (Section 1's intensity map with |s| <= 1); the best (gain, -d, -t) wins.
//
// One CTA per range: the range's 8 inverse-permuted copies sit in shared memory, each thread
// walks every 256th domain, and a shared-memory tree picks the block's best.
#include <climits>

#include "fic_internal.cuh"

namespace fic {

namespace {

constexpr int kSimtThreads = 256;

struct ScanShared {
    // rp[t][q] = r[p] with src_t(p) = q, so that X_t = sum_q S[q] * rp[t][q]
    float rp[8][64];
    long long num[kSimtThreads], den[kSimtThreads], P[kSimtThreads], Q[kSimtThreads];
    int d[kSimtThreads], t[kSimtThreads], C[kSimtThreads];
    int flagged[kSimtThreads];
    int n_flagged;
};

struct Best {
    Gain g;
    int d, t, C;
    long long P, Q;
};

__device__ __forceinline__ void load_range(ScanShared &sh, const Geo &g, const uint8_t *img, int r) {
    const int tid = threadIdx.x;
    if (tid < 64) {
        const int y = tid >> 3, x = tid & 7;
        const int ry = (r / g.nRx) * 8, rx = (r % g.nRx) * 8;
        const float v = (float)img[(size_t)(ry + y) * g.pitch + rx + x];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int sy, sx;
            iso_src(8, t, y, x, sy, sx);
            sh.rp[t][sy * 8 + sx] = v;
        }
    }
}

// Exact evaluation of domain d under all 8 isometries against the range in sh.rp.
__device__ __forceinline__ void scan_domain(const ScanShared &sh, int d, long long A,
                                            const uint16_t *__restrict__ domS,
                                            const int32_t *__restrict__ dsum,
                                            const int32_t *__restrict__ dsumsq, Best &b) {
    float S[64];
    const uint4 *src = reinterpret_cast<const uint4 *>(domS + (size_t)d * 64);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint4 u = __ldg(src + k);
        const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            S[8 * k + 2 * h] = (float)(w4[h] & 0xffffu);
            S[8 * k + 2 * h + 1] = (float)(w4[h] >> 16);
        }
    }
    float acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = 0.f;
#pragma unroll
    for (int q = 0; q < 64; q += 4) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float4 rv = *reinterpret_cast<const float4 *>(&sh.rp[t][q]);
            acc[t] = fmaf(S[q], rv.x, acc[t]);
            acc[t] = fmaf(S[q + 1], rv.y, acc[t]);
            acc[t] = fmaf(S[q + 2], rv.z, acc[t]);
            acc[t] = fmaf(S[q + 3], rv.w, acc[t]);
        }
    }
    const long long C = dsum[d];
    const long long Q = 64LL * dsumsq[d] - C * C;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const long long X = (long long)acc[t];
        const long long P = 64LL * X - A * C;
        const Gain gg = exact_gain(P, Q);
        if (cand_better(gg, d, t, b.g, b.d, b.t)) {
            b.g = gg;
            b.d = d;
            b.t = t;
            b.P = P;
            b.Q = Q;
            b.C = (int)C;
        }
    }
}

// Block-wide best and the code of range r (thread 0 writes it).
__device__ __forceinline__ void reduce_and_write(ScanShared &sh, const Best &b, int r, long long A,
                                                 long long Bs, const fic_codes &out) {
    const int tid = threadIdx.x;
    sh.num[tid] = b.g.num;
    sh.den[tid] = b.g.den;
    sh.d[tid] = b.d;
    sh.t[tid] = b.t;
    sh.P[tid] = b.P;
    sh.Q[tid] = b.Q;
    sh.C[tid] = b.C;
    __syncthreads();
    for (int s = kSimtThreads / 2; s > 0; s >>= 1) {
        if (tid < s) {
            const Gain ga{sh.num[tid], sh.den[tid]}, gb{sh.num[tid + s], sh.den[tid + s]};
            if (cand_better(gb, sh.d[tid + s], sh.t[tid + s], ga, sh.d[tid], sh.t[tid])) {
                sh.num[tid] = gb.num;
                sh.den[tid] = gb.den;
                sh.d[tid] = sh.d[tid + s];
                sh.t[tid] = sh.t[tid + s];
                sh.P[tid] = sh.P[tid + s];
                sh.Q[tid] = sh.Q[tid + s];
                sh.C[tid] = sh.C[tid + s];
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        double s, o, sse;
        finalize_code(64, A, Bs, sh.C[0], sh.P[0], sh.Q[0], Gain{sh.num[0], sh.den[0]}, s, o, sse);
        out.dom[r] = sh.d[0];
        out.iso[r] = sh.t[0];
        out.s[r] = s;
        out.o[r] = o;
        out.sse[r] = sse;
    }
    __syncthreads();
}

}  // namespace

// Plain search: CTA r scans the whole pool of range r.
__global__ void __launch_bounds__(kSimtThreads)
    k_match_simt(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
                 const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
                 const int32_t *__restrict__ rsum, const int32_t *__restrict__ rsumsq,
                 const int32_t *__restrict__ dom_order, const int32_t *__restrict__ win_lo,
                 const int32_t *__restrict__ win_hi, fic_codes out) {
    __shared__ __align__(16) ScanShared sh;
    const int r = blockIdx.x;
    load_range(sh, g, img, r);
    __syncthreads();
    const long long A = rsum[r], Bs = rsumsq[r];
    Best b{{-1, 1}, INT_MAX, 0, 0, 0, 0};
    for (int j = win_lo[r] + threadIdx.x; j < win_hi[r]; j += kSimtThreads)
        scan_domain(sh, dom_order[j], A, domS, dsum, dsumsq, b);
    reduce_and_write(sh, b, r, A, Bs, out);
}

// Re-search of uncertified ranges of one image. Slot k holds class-sorted position fb_pos[k] and
// the exact best of its evaluated candidates; the 512-domain chunks of the range's tile whose best
// FP32 score could still reach that best (score * (1 + 2^-16) + 2^-8 >= best gain / 512, the
// bound k_reeval certifies with) are scanned exactly.
__global__ void __launch_bounds__(kSimtThreads)
    k_rescan(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
             const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
             const int32_t *__restrict__ rsumsq, const int32_t *__restrict__ dom_order,
             const int4 *__restrict__ rng_info, int rng_off, int dom_off, const int4 *__restrict__ tile_win,
             const int4 *__restrict__ tile_items, const uint32_t *__restrict__ chunk_max,
             const int32_t *__restrict__ fb_pos, const FallbackBest *__restrict__ fb_best,
             const int32_t *__restrict__ counters, fic_codes out) {
    __shared__ __align__(16) ScanShared sh;
    const int n = min(counters[0], g.R);
    for (int k = blockIdx.x; k < n; k += gridDim.x) {
        const int i = fb_pos[k];
        const int4 ri = rng_info[i];
        const int r = ri.w;
        load_range(sh, g, img, r);
        __syncthreads();
        const FallbackBest fb = fb_best[k];
        Best b{{fb.num, fb.den}, fb.d, fb.t, fb.C, fb.P, fb.Q};
        const double thr = fb.num < 0 ? -1.0 : (double)fb.num / (512.0 * (double)fb.den);
        const long long A = ri.x, Bs = rsumsq[r];
        const int ig = rng_off + i, row = ig % kTileM;
        const int4 tw = tile_win[ig / kTileM];
        const int4 ti = tile_items[ig / kTileM];
        const int nch = ti.w;
        // flag the chunks whose best score reaches the threshold (256 chunks at a time, in
        // parallel), then scan the flagged chunks' domains with all threads
        for (int base = 0; base < nch; base += kSimtThreads) {
            if (threadIdx.x == 0) sh.n_flagged = 0;
            __syncthreads();
            const int c = base + threadIdx.x;
            if (c < nch) {
                const size_t e = ((size_t)(ti.z + c) * kTileM + row) * 2;
                const uint32_t key = max(chunk_max[e], chunk_max[e + 1]);
                const double s1 = (double)__uint_as_float(key);
                if (key != 0 && s1 * (1.0 + 1.0 / 65536.0) + 1.0 / 256.0 >= thr)
                    sh.flagged[atomicAdd(&sh.n_flagged, 1)] = c;
            }
            __syncthreads();
            const int nf = sh.n_flagged;
            for (int f = 0; f < nf; ++f) {
                const int cc = sh.flagged[f];
                const int j0 = max(ri.y, tw.x + cc * kChunkDom);
                const int j1 = min(ri.z, min(tw.x + (cc + 1) * kChunkDom, tw.y));
                for (int j = j0 + threadIdx.x; j < j1; j += kSimtThreads)
                    scan_domain(sh, dom_order[j - dom_off], A, domS, dsum, dsumsq, b);
            }
            __syncthreads();
        }
        reduce_and_write(sh, b, r, A, Bs, out);
    }
}

cudaError_t launch_match_simt(const uint8_t *img, const Geo &g, const EncodeBufs &b,
                              const fic_codes &out, cudaStream_t st) {
    k_match_simt<<<g.R, kSimtThreads, 0, st>>>(g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sum,
                                               b.range_sumsq, b.dom_order, b.win_lo, b.win_hi, out);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_rescan(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                          const fic_codes &out, int num_sms, cudaStream_t st) {
    k_rescan<<<4 * num_sms, kSimtThreads, 0, st>>>(g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sumsq,
                                                   b.dom_order, b.rng_info, b.rng_off, b.dom_off, tb.tile_win,
                                                   tb.tile_items, tb.chunk_max, b.fallback, b.fb_best, b.counters,
                                                   out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
