// Exact range-domain matching on CUDA cores: the plain GPU search, and the exact re-search of
// ranges the tensor engine's ranking could not certify.
//
// For a range r and every domain d of its pool (Section 3.1 Eq. 3) and isometry t, the
// correlation X_t = sum_p r[p] * (T_t S_d)[p] is formed exactly (integer products <= 255*1020
// and sums < 2^24 are exact in FP32 FMA), then P = 64 X - A C and Q = 64 E - C^2 give the exact
// least-squares gain (Section 1's intensity map with |s| <= 1); the best (gain, -d, -t) wins.
//
// One CTA per range: the range's 8 inverse-permuted copies sit in shared memory, each thread
// walks every 256th domain of the pool, and a shared-memory tree picks the block's best.
#include <climits>

#include "fic_internal.cuh"

namespace fic {

constexpr int kSimtThreads = 256;

__global__ void __launch_bounds__(kSimtThreads)
    k_match_simt(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
                 const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
                 const int32_t *__restrict__ rsum, const int32_t *__restrict__ rsumsq,
                 const int32_t *__restrict__ dom_order, const int32_t *__restrict__ win_lo,
                 const int32_t *__restrict__ win_hi, const int32_t *__restrict__ list,
                 const int32_t *__restrict__ list_count, int n_list_max, fic_codes out) {
    // rp[t][q] = r[p] with src_t(p) = q, so that X_t = sum_q S[q] * rp[t][q]
    __shared__ __align__(16) float rp[8][64];
    __shared__ long long red_num[kSimtThreads], red_den[kSimtThreads], red_P[kSimtThreads],
        red_Q[kSimtThreads];
    __shared__ int red_d[kSimtThreads], red_t[kSimtThreads], red_C[kSimtThreads];

    const int tid = threadIdx.x;
    int n_items = g.R;
    if (list) n_items = min(*list_count, n_list_max);
    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int r = list ? list[item] : item;
        if (tid < 64) {
            const int y = tid >> 3, x = tid & 7;
            const int ry = (r / g.nRx) * 8, rx = (r % g.nRx) * 8;
            const float v = (float)img[(size_t)(ry + y) * g.pitch + rx + x];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                int sy, sx;
                iso_src(8, t, y, x, sy, sx);
                rp[t][sy * 8 + sx] = v;
            }
        }
        __syncthreads();
        const long long A = rsum[r], Bs = rsumsq[r];
        const int lo = win_lo[r], hi = win_hi[r];
        Gain best{-1, 1};
        int bd = INT_MAX, bt = 0, bC = 0;
        long long bP = 0, bQ = 0;
        for (int j = lo + tid; j < hi; j += kSimtThreads) {
            const int d = dom_order[j];
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
                    const float4 rv = *reinterpret_cast<const float4 *>(&rp[t][q]);
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
                if (cand_better(gg, d, t, best, bd, bt)) {
                    best = gg;
                    bd = d;
                    bt = t;
                    bP = P;
                    bQ = Q;
                    bC = (int)C;
                }
            }
        }
        red_num[tid] = best.num;
        red_den[tid] = best.den;
        red_d[tid] = bd;
        red_t[tid] = bt;
        red_P[tid] = bP;
        red_Q[tid] = bQ;
        red_C[tid] = bC;
        __syncthreads();
        for (int s = kSimtThreads / 2; s > 0; s >>= 1) {
            if (tid < s) {
                const Gain ga{red_num[tid], red_den[tid]}, gb{red_num[tid + s], red_den[tid + s]};
                if (cand_better(gb, red_d[tid + s], red_t[tid + s], ga, red_d[tid], red_t[tid])) {
                    red_num[tid] = gb.num;
                    red_den[tid] = gb.den;
                    red_d[tid] = red_d[tid + s];
                    red_t[tid] = red_t[tid + s];
                    red_P[tid] = red_P[tid + s];
                    red_Q[tid] = red_Q[tid + s];
                    red_C[tid] = red_C[tid + s];
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            double s, o, sse;
            finalize_code(64, A, Bs, red_C[0], red_P[0], red_Q[0], Gain{red_num[0], red_den[0]},
                          s, o, sse);
            out.dom[r] = red_d[0];
            out.iso[r] = red_t[0];
            out.s[r] = s;
            out.o[r] = o;
            out.sse[r] = sse;
        }
        __syncthreads();
    }
}

cudaError_t launch_match_simt(const uint8_t *img, const Geo &g, const EncodeBufs &b,
                              const int32_t *list, const int32_t *list_count, int n_list_max,
                              const fic_codes &out, cudaStream_t st) {
    // all ranges: one CTA each; a device-side list: a fixed grid strides over it
    const int grid = list ? 4 * 152 : g.R;
    if (grid <= 0) return cudaSuccess;
    k_match_simt<<<grid, kSimtThreads, 0, st>>>(g, img, b.dom_S, b.dom_sum, b.dom_sumsq,
                                                b.range_sum, b.range_sumsq, b.dom_order,
                                                b.win_lo, b.win_hi, list, list_count,
                                                n_list_max, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
