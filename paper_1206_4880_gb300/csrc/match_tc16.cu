// Tensor-core engine for 16x16 ranges and 32x32 domains (sm_103a: TMA, tcgen05, TMEM).
//
// The same contraction as the B = 8 engine with n = 256 pixels per block:
//
//   A_mat[i][p]       = r_i[p] - a_i             (class-sorted range i, fp16, |.| <= 255)
//   B_mat[8 j + t][p] = T_t(S_{d_j})[p] - c_j    (class-sorted domain j, isometry t, |.| <= 1020)
//   D[i][8 j + t] = Y = sum_p A_mat[i][p] * B_mat[8 j + t][p]
//
// with a = round(A / 256), c = round(C / 256). The products are integers, so exactness needs every
// partial sum below 2^24. By Cauchy-Schwarz any partial sum is at most
// sqrt(sum (r - a)^2) sqrt(sum (S - c)^2); with the variance bound (max - min)^2 / 4 and the mean
// rounding (|A/256 - a| <= 1/2), sum (r - a)^2 <= 256 (127.5^2 + 1/4) = 4,161,664 and
// sum (S - c)^2 <= 256 (510^2 + 1/4) = 66,585,664, so |partial| <= 2040.02 * 8160.01
// < 16,646,600 < 2^24 = 16,777,216: the FP32 accumulator holds Y exactly whatever the order of
// additions. With alpha = A - 256 a and gamma = C - 256 c (both in [-128, 128]),
// P = 256 X - A C = 256 Y - alpha gamma, and the epilogue forms P / 256 = fma(alpha, -gamma/256, Y)
// with one rounding (the product is exact in FP32), so no correction slice is needed.
//
// Scores: with p = |P| / 256, the clamped least-squares gain / 2048 (Section 1's intensity map,
// |s| <= 1) is 512 p^2 / Q for p <= Q / 1024 and p - Q / 2048 beyond; s = fma(m, m (512/Q), p - m)
// with m = min(p, Q / 1024) covers both. Keys and certification as in the B = 8 engine, with
// gain / 2048 in place of gain / 512.
//
// Kernel shape: persistent, one CTA per SM, 10 warps. A range tile is 256 class-sorted ranges,
// two M = 128 MMA operands resident in shared memory (4 K-quarters of 64 columns each, 128-byte
// swizzle); every B stage (one K-quarter of 16 domains x 8 isometries = 128 rows) feeds both, so a
// streamed byte of B serves 256 ranges. TMEM holds four 128 x 128 FP32 accumulators (two range
// tiles x double buffering). Warp 0 issues TMA loads, warp 1 the MMAs (M = 128, N = 128, K = 16,
// 16 per accumulator), warps 2-9 drain: warp w reads TMEM lane group w & 3 of range tile
// (w - 2) >> 2. Every wait is bounded as in the B = 8 engine.
#include <cuda.h>

#include <climits>
#include <mutex>

#include "fic_internal.cuh"
#include "tc_ptx.cuh"

namespace fic {

namespace {

constexpr int kTm16 = 2 * kTileM;                   // 256 ranges per range tile
constexpr int kDom16 = 16;                          // domains per accumulator tile
constexpr int kN16 = 8 * kDom16;                    // 128 accumulator columns
// B-operand ring stages (4 or 5: fic_params.pipeline_stages). The default 4: measured 0.8% faster at
// 2048x2048 stride 4 (matcher 10.02 against 10.10 ms) and 0.8% at 4096x4096 stride 8
constexpr int kStages16Default = 4;
constexpr int kQA = kTileM * 128;                   // one K-quarter of one MMA row tile: 16 KB
constexpr int kQB = kN16 * 128;                     // one K-quarter of one domain tile: 16 KB
constexpr int kEpi16 = 8;
constexpr int kTc16Threads = 32 * (2 + kEpi16);
constexpr int kTmem16 = 4 * kN16;                   // 512 columns
constexpr uint32_t kIdesc16 = (1u << 4) | ((uint32_t)(kN16 >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);

template <int S>
struct Tc16Shared {
    uint8_t A[2][4][kQA];          // [MMA row tile][K-quarter]
    uint8_t B[S][kQB];             // ring of K-quarters
    float4 aux[2][kChunkDom];      // per-domain constants of the current and next chunk
    unsigned long long full_a, empty_a, full_b[S], empty_b[S], tfull[2], tempty[2], aux_ready[2],
        drain, item_full[kItemRing], item_empty[kItemRing],
        never;  // completed by nothing: the forced wait of the testing hook (fic_debug_stall_matcher)
    int item_id[kItemRing];  // work items fetched by the producer, in this CTA's order (-1: none left)
    uint32_t tmem_base;
    int abort_flag;
};
template <int S>
constexpr size_t tc16_smem() { return sizeof(Tc16Shared<S>) + 1024; }
static_assert(sizeof(Tc16Shared<5>) + 1024 <= 232448, "shared memory per CTA");

// Scores of one accumulator tile for this thread's range row: 16 domains x 8 isometries. The 16
// domains (positions jh .. jh + 15, jh a multiple of 16) form one group, whose largest score goes
// on as one key into t1, t2 (the two largest group keys of the chunk), as in the B = 8 kernel.
template <bool MASK>
__device__ __forceinline__ void epi16(uint32_t taddr, const float4 *auxp, float alpha, int jh, int jrel, int lo_r,
                                      int hi_r, uint32_t &t1, uint32_t &t2) {
    float gmax = MASK ? -1.f : 0.f;  // the group's largest score
    uint32_t va[32], vb[32];
    tmem_ld32(taddr, va);
    tmem_ld_wait(va);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c < 3) {
            if (c & 1)
                tmem_ld32(taddr + (c + 1) * 32, va);
            else
                tmem_ld32(taddr + (c + 1) * 32, vb);
        }
        const uint32_t *cur = (c & 1) ? vb : va;
        float sv[4];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = 2 * q2 + h, l = 4 * c + q;
                const float4 a = auxp[l];
                float y[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) y[t] = fmaf(alpha, a.x, __uint_as_float(cur[8 * q + t]));
                const float p = max3f(max3_abs(y[0], y[1], y[2]), max3_abs(y[3], y[4], y[5]),
                                      fmaxf(fabsf(y[6]), fabsf(y[7])));
                const float mm = fminf(p, a.y);
                float sc = fmaf(mm, mm * a.z, p - mm);
                if (MASK) {
                    const int j = jh + l;
                    sc = (j >= lo_r && j < hi_r) ? sc : -1.f;
                }
                sv[2 * q2 + h] = sc;
            }
        }
        gmax = max3f(gmax, max3f(sv[0], sv[1], sv[2]), sv[3]);
        if (c < 3) {
            if (c & 1)
                tmem_ld_wait(va);
            else
                tmem_ld_wait(vb);
        }
    }
    // the group's key: its largest score's bits with the low 9 replaced by 511 - its offset in
    // the chunk (key 0 when no domain of the group is in the window)
    uint32_t key = (__float_as_uint(gmax) & 0xFFFFFE00u) | (uint32_t)(511 - jrel);
    if (MASK && gmax < 0.f) key = 0u;
    top2u(t1, t2, key);
}

}  // namespace

// ---- operand packing ------------------------------------------------------------------------
// One thread per (sorted range i, pixel row y): A_mat row i = pixels - round(A / 256);
// rng_info[i] = (A, pool start, pool end, range id), pools in batch-wide domain positions. Rows
// i >= R are zero with an empty window and range id -1.
__global__ void k_pack_ranges16(Geo g, const uint8_t *__restrict__ img, const int32_t *__restrict__ range_order,
                                const int32_t *__restrict__ rsum, const int32_t *__restrict__ win_lo,
                                const int32_t *__restrict__ win_hi, int R_pad, int dom_off,
                                __half *__restrict__ A_mat, int4 *__restrict__ rng_info) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gid >> 4, y = gid & 15;
    if (i >= R_pad) return;
    uint4 pk[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    if (i < g.R) {
        const int r = range_order[i];
        const uint8_t *row = img + (size_t)((r / g.nRx) * 16 + y) * g.pitch + (r % g.nRx) * 16;
        const int abar = (rsum[r] + 128) >> 8;  // round(A / 256)
        uint32_t w[8];
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const __half a = __int2half_rn((int)row[2 * h] - abar);
            const __half b = __int2half_rn((int)row[2 * h + 1] - abar);
            w[h] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
        }
        pk[0] = make_uint4(w[0], w[1], w[2], w[3]);
        pk[1] = make_uint4(w[4], w[5], w[6], w[7]);
        if (y == 0) rng_info[i] = make_int4(rsum[r], win_lo[r] + dom_off, win_hi[r] + dom_off, r);
    } else if (y == 0) {
        rng_info[i] = make_int4(0, 0, 0, -1);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(A_mat + (size_t)i * 256 + y * 16);
    dst[0] = pk[0];
    dst[1] = pk[1];
}

// One thread per (sorted domain j, isometry t, row y), two domains per 256-thread block: B_mat
// row 8j+t = T_t(S_{dom_order[j]}) - round(C / 256), each output row one 32-byte row of a staged
// layout converted pairwise to FP16; dom_aux[j] = (-gamma / 256, Q / 1024, 512 / Q or 0, 0) with
// gamma = C - 256 round(C / 256). Entries j >= Dn are zero.
__global__ void __launch_bounds__(256) k_pack_domains16(Geo g, const uint16_t *__restrict__ domS,
                                                        const int32_t *__restrict__ dom_order,
                                                        const int32_t *__restrict__ dsum,
                                                        const int32_t *__restrict__ dsumsq, int n_pad,
                                                        __half *__restrict__ B_mat, float4 *__restrict__ dom_aux) {
    __shared__ __align__(16) uint16_t L[2][4][256];
    const int jl = threadIdx.x >> 7, e = threadIdx.x & 127;
    const int j = blockIdx.x * 2 + jl, t = e >> 4, y = e & 15;
    const bool live = j < g.Dn;
    int d = 0, cbar = 0;
    if (live) {
        d = dom_order[j];
        cbar = (dsum[d] + 128) >> 8;  // round(C / 256)
        stage_layouts<16>(L[jl], e, domS[(size_t)d * 256 + e]);
        stage_layouts<16>(L[jl], e + 128, domS[(size_t)d * 256 + e + 128]);
    }
    __syncthreads();
    if (j >= n_pad) return;
    uint4 pk[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    if (live) {
        const uint4 *m = reinterpret_cast<const uint4 *>(iso_row<16>(L[jl], t, y));
        const uint32_t c2 = (0x6400u + (uint32_t)cbar) * 0x10001u;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint4 v = m[k];
            pk[k] = make_uint4(centred_h2(v.x, c2), centred_h2(v.y, c2), centred_h2(v.z, c2), centred_h2(v.w, c2));
        }
        if (t == 0 && y == 0) {
            const long long C = dsum[d];
            const long long Q = 256LL * dsumsq[d] - C * C;
            const int gamma = (int)C - 256 * cbar;
            dom_aux[j] = make_float4(-(float)gamma * (1.0f / 256.0f), (float)Q * (1.0f / 1024.0f),
                                     Q > 0 ? 512.0f / (float)Q : 0.f, 0.f);
        }
    } else if (t == 0 && y == 0) {
        dom_aux[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(B_mat + ((size_t)j * 8 + t) * 256 + y * 16);
    dst[0] = pk[0];
    dst[1] = pk[1];
}

// ---- the matching kernel ----------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(kTc16Threads, 1)
    k_match_tc16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const int4 *__restrict__ work, const int32_t *__restrict__ work_slot,
                 const int4 *__restrict__ tile_items,
                 const int32_t *__restrict__ counters_in, const int4 *__restrict__ tile_win,
                 const int4 *__restrict__ rng_info, const float4 *__restrict__ dom_aux,
                 unsigned long long *__restrict__ cand, uint32_t *__restrict__ chunk_max, int32_t *next_item,
                 int32_t *err, int32_t *lib_err, unsigned long long stall_ns) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (su32(smem_raw) & 1023u)) & 1023u;
    Tc16Shared<S> &sh = *reinterpret_cast<Tc16Shared<S> *>(smem_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = counters_in[1];
    volatile int *abort_flag = &sh.abort_flag;

    if (threadIdx.x == 0) {
        mbar_init(&sh.full_a, 1);
        mbar_init(&sh.empty_a, 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sh.tfull[s], 1);
            mbar_init(&sh.tempty[s], kEpi16);
            mbar_init(&sh.aux_ready[s], 32 * kEpi16);
        }
        for (int s = 0; s < S; ++s) {
            mbar_init(&sh.full_b[s], 1);
            mbar_init(&sh.empty_b[s], 1);
        }
        for (int s = 0; s < kItemRing; ++s) {
            mbar_init(&sh.item_full[s], 1);
            mbar_init(&sh.item_empty[s], 1 + kEpi16);
        }
        mbar_init(&sh.drain, 1);
        mbar_init(&sh.never, 1);
        sh.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(&sh.tmem_base, kTmem16);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
            uint32_t gs = 0;
            bool ok = true;
            // testing hook: a wait that nothing completes, before any copy or MMA is issued, so the
            // bounded-wait error path runs with nothing in flight
            if (stall_ns && !mbar_wait_for(&sh.never, 0, abort_flag, stall_ns)) ok = false;
            for (uint32_t li = 0; ok; ++li) {
                // the next item of the whole grid, handed to the MMA and epilogue warps
                const int s = li % kItemRing;
                ok = mbar_wait(&sh.item_empty[s], ((li / kItemRing) & 1) ^ 1, abort_flag);
                if (!ok) break;
                int it = atomicAdd(next_item, 1);
                if (it >= n_items) it = -1;
                sh.item_id[s] = it;
                mbar_arrive(&sh.item_full[s]);
                if (it < 0) break;
                const int4 w = work[it];
                ok = mbar_wait(&sh.empty_a, (li & 1) ^ 1, abort_flag);
                if (!ok) break;
                mbar_expect_tx(&sh.full_a, 8 * kQA);
#pragma unroll
                for (int m = 0; m < 2; ++m)
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        tma_load_2d(sh.A[m][q], &tmA, &sh.full_a, 64 * q, w.x * kTm16 + m * kTileM);
                const int nt = (w.z - w.y + kDom16 - 1) / kDom16;
                for (int k = 0; k < nt && ok; ++k) {
                    for (int q = 0; q < 4; ++q, ++gs) {
                        const int s = gs % S;
                        ok = mbar_wait(&sh.empty_b[s], ((gs / S) & 1) ^ 1, abort_flag);
                        if (!ok) break;
                        mbar_expect_tx(&sh.full_b[s], kQB);
                        tma_load_2d(sh.B[s], &tmB, &sh.full_b[s], 64 * q, 8 * (w.y + k * kDom16));
                    }
                }
            }
            if (!ok) {
                report_timeout(err, lib_err, abort_flag);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            uint32_t gs = 0, gt = 0;
            bool ok = true;
            for (uint32_t li = 0; ok; ++li) {
                const int s = li % kItemRing;
                ok = mbar_wait(&sh.item_full[s], (li / kItemRing) & 1, abort_flag);
                if (!ok) break;
                const int it = sh.item_id[s];
                mbar_arrive(&sh.item_empty[s]);
                if (it < 0) break;
                const int4 w = work[it];
                ok = mbar_wait(&sh.full_a, li & 1, abort_flag);
                if (!ok) break;
                tc_fence_after();
                const int nt = (w.z - w.y + kDom16 - 1) / kDom16;
                for (int k = 0; k < nt && ok; ++k, ++gt) {
                    const int acc = gt & 1;
                    ok = mbar_wait(&sh.tempty[acc], ((gt >> 1) & 1) ^ 1, abort_flag);
                    if (!ok) break;
                    tc_fence_after();
                    for (int q = 0; q < 4; ++q, ++gs) {
                        const int s = gs % S;
                        ok = mbar_wait(&sh.full_b[s], (gs / S) & 1, abort_flag);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t b0 = su32(sh.B[s]);
#pragma unroll
                        for (int m = 0; m < 2; ++m) {
                            const uint32_t a0 = su32(sh.A[m][q]);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                umma_f16(tmem + (uint32_t)((2 * acc + m) * kN16), sw128_desc(a0 + kk * 32),
                                         sw128_desc(b0 + kk * 32), kIdesc16, (q | kk) ? 1u : 0u);
                        }
                        umma_commit(&sh.empty_b[s]);
                    }
                    if (!ok) break;
                    umma_commit(&sh.tfull[acc]);
                }
                if (!ok) break;
                umma_commit(&sh.empty_a);
            }
            // all MMAs issued by this thread complete before TMEM is released
            umma_commit(&sh.drain);
            if (!mbar_wait(&sh.drain, 0, abort_flag) && !*abort_flag) ok = false;
            if (!ok) {
                report_timeout(err, lib_err, abort_flag);
            }
        }
    } else {
        // ---- epilogue: warps 2..9; warp w reads TMEM lane group (w & 3) of MMA row tile
        // (w - 2) >> 2, i.e. range rows m * 128 + lane group * 32 + lane of the range tile
        const int ew = warp - 2;
        const int lg = warp & 3;
        const int m = ew >> 2;
        const int row = m * kTileM + lg * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(m * kN16);
        uint32_t gt = 0, lc = 0;
        bool ok = true;
        for (uint32_t li = 0; ok; ++li) {
            const int s = li % kItemRing;
            ok = __all_sync(0xffffffffu, mbar_wait(&sh.item_full[s], (li / kItemRing) & 1, abort_flag));
            if (!ok) break;
            const int it = sh.item_id[s];
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.item_empty[s]);
            if (it < 0) break;
            const int4 w = work[it];
            const int nt = (w.z - w.y + kDom16 - 1) / kDom16;
            const int i = w.x * kTm16 + row;
            const int4 ri = rng_info[i];
            const bool valid = ri.w >= 0;
            const float alpha = (float)(ri.x - 256 * ((ri.x + 128) >> 8));
            const int lo_r = ri.y, hi_r = min(ri.z, w.z);
            const int4 tw = tile_win[w.x];
            const int f_lo = max(tw.z, w.y), f_hi = min(tw.w, w.z);  // columns valid for every row
            unsigned long long b1 = 0, b2 = 0;
            for (int k0 = 0, ntc = 0; k0 < nt && ok; k0 += ntc, ++lc) {
                const int jc = w.y + k0 * kDom16;
                const int cabs = jc / kChunkDom;
                ntc = min(nt - k0, ((cabs + 1) * kChunkDom - jc) / kDom16);
                const int ab = lc & 1;
                for (int k = ew * 32 + lane; k < ntc * kDom16; k += 32 * kEpi16) sh.aux[ab][k] = __ldg(&dom_aux[jc + k]);
                mbar_arrive(&sh.aux_ready[ab]);
                ok = __all_sync(0xffffffffu, mbar_wait(&sh.aux_ready[ab], (lc >> 1) & 1, abort_flag));
                if (!ok) break;
                uint32_t t1 = 0, t2 = 0;
                const int jrel0 = jc - cabs * kChunkDom;
                for (int k = 0; k < ntc; ++k, ++gt) {
                    const int acc = gt & 1;
                    ok = __all_sync(0xffffffffu, mbar_wait(&sh.tfull[acc], (gt >> 1) & 1, abort_flag));
                    if (!ok) break;
                    tc_fence_after();
                    const int jh = jc + k * kDom16;
                    const float4 *auxp = &sh.aux[ab][k * kDom16];
                    const uint32_t taddr = tbase + (uint32_t)(acc * 2 * kN16);
                    const int jrel = jrel0 + k * kDom16;
                    if (jh >= f_lo && jh + kDom16 <= f_hi)
                        epi16<false>(taddr, auxp, alpha, jh, jrel, lo_r, hi_r, t1, t2);
                    else
                        epi16<true>(taddr, auxp, alpha, jh, jrel, lo_r, hi_r, t1, t2);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh.tempty[acc]);
                }
                merge_chunk_key(b1, b2, t1, cabs * kChunkDom);
                merge_chunk_key(b1, b2, t2, cabs * kChunkDom);
                if (ok && valid)
                    reinterpret_cast<uint2 *>(chunk_max)[(size_t)(w.w + cabs - w.y / kChunkDom) * kTm16 + row] =
                        make_uint2(t1, t2 & 0xFFFFFE00u);
            }
            if (ok && valid) {
                // the tile's keys are row-major (row, item, 2): a range reads its keys at once
                const int4 ti = tile_items[w.x];
                unsigned long long *dst =
                    cand + (size_t)ti.x * kTm16 * 2 + ((size_t)row * ti.y + (work_slot[it] - ti.x)) * 2;
                dst[0] = b1;
                dst[1] = b2;
            }
        }
        if (!ok) {
            report_timeout(err, lib_err, abort_flag);
        }
    }

    // ---- teardown: copies in flight complete (bounded), then TMEM is freed
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        const unsigned long long t0 = gtimer();
        while (gtimer() - t0 < 5000000ull) {
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmem16);
    }
}

// ---- exact re-evaluation and certification ----------------------------------------------------
// One half-warp per class-sorted range position i of one image, as the B = 8 re-evaluation: the
// best group key's 16 domains are evaluated exactly under all 8 isometries (one lane per domain),
// the best is certified if the runner-up's
// score * (1 + 2^-13) + 2^-16 < exact best gain / 2048 (the key truncation errs by less than
// 2^-14 relatively, the score formula and the epilogue's single rounding of the exact Y by less
// than 2^-18 relatively; the absolute term only guards the degenerate scores near zero), else the
// range is queued for the exact re-search.
constexpr int kReeval16Threads = 256;
struct __align__(16) Reeval16Stage {
    uint8_t rp[8][256];  // the range's inverse-permuted copies rp[t][src_t(p)] = r[p]
};

// One half-warp's exact best, left for the block's finishing lanes (kinds as in the B = 8 kernel).
struct Reeval16Res {
    __int128 num;
    long long den, P, Q, A, Bs;
    int C, d, t, r, i;
    uint32_t u2;
    int kind, has1, has2;
};

// Exact evaluation of class-sorted range position i by one half-warp (lanes hmask, hl = lane
// mod 16; see k_reeval16).
__device__ __forceinline__ void reeval16_rank(const Geo &g, const uint8_t *__restrict__ img,
                                              const uint16_t *__restrict__ domS, const int32_t *__restrict__ dsum,
                                              const int32_t *__restrict__ dsumsq, const int32_t *__restrict__ rsumsq,
                                              const int32_t *__restrict__ dom_order, const int32_t *__restrict__ bin_off,
                                              int nbuckets, const int4 *__restrict__ rng_info, int rng_off, int dom_off,
                                              const int4 *__restrict__ tile_items,
                                              const unsigned long long *__restrict__ cand, int i, int hl, unsigned hmask,
                                              Reeval16Stage &sg16, Reeval16Res &res) {
    const int4 ri = rng_info[i];
    const int r = ri.w;
    const long long A = ri.x, Bs = rsumsq[r];
    const int ry = (r / g.nRx) * 16, rx = (r % g.nRx) * 16;
    // the range's 8 inverse-permuted copies, staged before the key merge so that the pixel loads
    // overlap the key loads (a flat range does not use them)
    Reeval16Stage &sg = sg16;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int px = 16 * hl + k, y = px >> 4, x = px & 15;
        const uint8_t v = img[(size_t)(ry + y) * g.pitch + rx + x];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int sy, sx;
            iso_src(16, t, y, x, sy, sx);
            sg.rp[t][sy * 16 + sx] = v;
        }
    }

    if (256LL * Bs - A * A == 0) {  // flat range: every candidate has P = 0
        int dmin = INT_MAX;
        const int wlo = ri.y - dom_off, whi = ri.z - dom_off;
        for (int bb = hl; bb < nbuckets; bb += 16)
            if (bin_off[bb] < bin_off[bb + 1] && bin_off[bb] >= wlo && bin_off[bb] < whi)
                dmin = min(dmin, dom_order[bin_off[bb]]);
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) dmin = min(dmin, __shfl_xor_sync(hmask, dmin, off));
        if (hl == 0) {
            const long long C = dsum[dmin];
            const long long Q = 256LL * dsumsq[dmin] - C * C;
            const GainW g0 = exact_gain_w(0, Q);
            res = Reeval16Res{g0.num, g0.den, 0, Q, A, Bs, (int)C, dmin, 0, r, i, 0u, 1, 1, 0};
        }
        return;
    }

    const int ig = rng_off + i;
    const int row = ig % kTm16;
    const int4 ti = tile_items[ig / kTm16];
    unsigned long long b1 = 0, b2 = 0;
    const unsigned long long *ck = cand + (size_t)ti.x * kTm16 * 2 + (size_t)row * ti.y * 2;
    for (int e = hl; e < 2 * ti.y; e += 16) top2(b1, b2, ck[e]);
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(hmask, b1, off);
        const unsigned long long o2 = __shfl_xor_sync(hmask, b2, off);
        top2(b1, b2, o1);
        top2(b1, b2, o2);
    }
    // exact evaluation of the best key's 16-domain group inside the pool window, as in the 8x8
    // re-evaluation (lane hl: the group's domain hl, all 8 isometries)
    __syncwarp(hmask);
    const int p1 = (int)(~(uint32_t)(b1 & 0xffffffffu));  // batch-wide positions
    int pos = b1 != 0 ? (p1 & ~15) + hl : -1;
    if (pos < ri.y || pos >= ri.z) pos = -1;
    GainW gg;
    gg.num = -1;
    gg.den = 1;
    int d = INT_MAX, bt = 0;
    long long P = 0, Q = 0, C = 0;
    if (pos >= 0) {
        d = dom_order[pos - dom_off];
        unsigned X[8];
        corr8<16>(sg.rp, domS + (size_t)d * 256, X);
        C = dsum[d];
        Q = 256LL * dsumsq[d] - C * C;
        // with the domain (so Q and C) fixed the clamped gain grows with |P|: the best isometry
        // is the largest |P|, ties to the smaller t (a flat domain has P = 0 for every t)
        P = 256LL * (long long)X[0] - A * C;
        long long aP = P < 0 ? -P : P;
#pragma unroll
        for (int t = 1; t < 8; ++t) {
            const long long Pt = 256LL * (long long)X[t] - A * C;
            const long long at = Pt < 0 ? -Pt : Pt;
            if (at > aP) {
                aP = at;
                bt = t;
                P = Pt;
            }
        }
        gg = exact_gain_w(P, Q);
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
        GainW og;
        const unsigned long long lo = __shfl_xor_sync(hmask, (unsigned long long)gg.num, off);
        const long long hi = __shfl_xor_sync(hmask, (long long)(gg.num >> 64), off);
        og.num = (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | (unsigned __int128)lo);
        og.den = __shfl_xor_sync(hmask, gg.den, off);
        const int od = __shfl_xor_sync(hmask, d, off), ot = __shfl_xor_sync(hmask, bt, off);
        const long long oP = __shfl_xor_sync(hmask, P, off), oQ = __shfl_xor_sync(hmask, Q, off);
        const long long oC = __shfl_xor_sync(hmask, C, off);
        if (cand_better(og, od, ot, gg, d, bt)) {
            gg = og;
            d = od;
            bt = ot;
            P = oP;
            Q = oQ;
            C = oC;
        }
    }
    if (hl == 0)
        res = Reeval16Res{gg.num, gg.den, P, Q, A, Bs, (int)C, d, bt, r, i, (uint32_t)(b2 >> 32), 2, b1 != 0, b2 != 0};
}

// Certification, code or queueing of one evaluated range, one lane per range (the FP64 steps
// serve all the block's ranges with one warp's instructions, as in the B = 8 kernel).
__device__ __forceinline__ void reeval16_finish(const Reeval16Res &e, int32_t *__restrict__ fallback,
                                                FallbackBest *__restrict__ fb_best, int32_t *counters,
                                                const fic_codes &out) {
    if (e.kind == 0) return;
    GainW gg;
    gg.num = e.num;
    gg.den = e.den;
    bool certified = e.kind == 1 || (e.has1 && gg.num >= 0);
    if (e.kind == 2 && certified && e.has2) {
        const double u2 = (double)__uint_as_float(e.u2);
        certified = (u2 * (1.0 + 1.0 / 8192.0) + 1.0 / 65536.0) * (2048.0 * (double)gg.den) < i128_to_double_rn(gg.num);
    }
    if (!certified) {
        const int slot = atomicAdd(&counters[0], 1);
        fallback[slot] = e.i;
        FallbackBest fb;
        fb.num = gg.num;
        fb.den = gg.den;
        fb.P = e.P;
        fb.Q = e.Q;
        fb.d = e.d;
        fb.t = e.t;
        fb.C = e.C;
        fb.pad = 0;
        fb_best[slot] = fb;
        return;
    }
    double s, o, sse;
    finalize_code(256, e.A, e.Bs, e.C, e.P, e.Q, gg, s, o, sse);
    out.dom[e.r] = e.d;
    out.iso[e.r] = e.t;
    out.s[e.r] = s;
    out.o[e.r] = o;
    out.sse[e.r] = sse;
}

__global__ void __launch_bounds__(kReeval16Threads) k_reeval16(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
                           const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
                           const int32_t *__restrict__ rsumsq, const int32_t *__restrict__ dom_order,
                           const int32_t *__restrict__ bin_off, int nbuckets, const int4 *__restrict__ rng_info,
                           int rng_off, int dom_off, const int4 *__restrict__ tile_items,
                           const unsigned long long *__restrict__ cand, const int32_t *__restrict__ gcounters,
                           int32_t *__restrict__ fallback, FallbackBest *__restrict__ fb_best, int32_t *counters,
                           fic_codes out) {
    __shared__ Reeval16Stage stage16[kReeval16Threads / 16];
    __shared__ Reeval16Res res[kReeval16Threads / 16];
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;
    const int hl = threadIdx.x & 15, slot = threadIdx.x >> 4;
    const unsigned hmask = 0xFFFFu << (threadIdx.x & 16);  // this half-warp
    if (gcounters[2] != 0) {
        // the matching kernel gave up: its keys are not trusted, so every code is marked invalid
        if (hl == 0 && i < g.R) poison_code(out, i);
        return;
    }
    if (i < g.R)
        reeval16_rank(g, img, domS, dsum, dsumsq, rsumsq, dom_order, bin_off, nbuckets, rng_info, rng_off, dom_off,
                      tile_items, cand, i, hl, hmask, stage16[slot], res[slot]);
    else if (hl == 0)
        res[slot].kind = 0;
    __syncthreads();
    if (threadIdx.x < kReeval16Threads / 16)
        reeval16_finish(res[threadIdx.x], fallback, fb_best, counters, out);
}

// ---- host side -------------------------------------------------------------------------------
cudaError_t launch_pack16(const uint8_t *img, const Geo &g, const EncodeBufs &b, cudaStream_t st, int part) {
    if (part != 2) {
        const long long n = (long long)b.R_pad * 16;
        k_pack_ranges16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, img, b.range_order, b.range_sum, b.win_lo,
                                                                    b.win_hi, b.R_pad, b.dom_off, b.A_mat,
                                                                    b.rng_info);
        ++g_launches;
    }
    if (part != 1) {
        const long long n = (long long)b.Dn_aux * 128;
        k_pack_domains16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, b.dom_S, b.dom_order, b.dom_sum,
                                                                     b.dom_sumsq, b.Dn_aux, b.B_mat, b.dom_aux);
        ++g_launches;
    }
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_tc16_variant(const CUtensorMap &tmA, const CUtensorMap &tmB, const TcBatch &tb, int grid,
                                cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err =
            cudaFuncSetAttribute(k_match_tc16<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc16_smem<S>());
    });
    if (attr_err) return attr_err;
    k_match_tc16<S><<<grid, kTc16Threads, tc16_smem<S>(), st>>>(tmA, tmB, tb.work, tb.work_slot, tb.tile_items,
                                                               tb.gcounters, tb.tile_win, tb.rng_info, tb.dom_aux,
                                                               tb.cand, tb.chunk_max, tb.gcounters + 5,
                                                               tb.gcounters + 2, tb.lib_error, tb.stall_ns);
    return cudaGetLastError();
}

cudaError_t launch_match_tc16(const TcBatch &tb, int num_sms, cudaStream_t st) {
    CUtensorMap tmA, tmB;
    cudaError_t e;
    if ((e = make_map_f16(&tmA, tb.A_mat, (unsigned long long)tb.R_pad, 256, kTileM, 64))) return e;
    if ((e = make_map_f16(&tmB, tb.B_mat, (unsigned long long)tb.Dn_aux * 8, 256, kN16, 64))) return e;
    const int grid = num_sms < tb.max_items ? num_sms : tb.max_items;
    if (grid <= 0) return cudaSuccess;
    if (tb.stages == 5)
        e = launch_tc16_variant<5>(tmA, tmB, tb, grid, st);
    else
        e = launch_tc16_variant<4>(tmA, tmB, tb, grid, st);
    if (e) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_reeval16(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                            const fic_codes &out, cudaStream_t st) {
    const long long threads = (long long)g.R * 16;
    k_reeval16<<<(unsigned)((threads + kReeval16Threads - 1) / kReeval16Threads), kReeval16Threads, 0, st>>>(
        g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sumsq, b.dom_order, b.bin_off, sort_buckets(g), b.rng_info,
        b.rng_off, b.dom_off, tb.tile_items, tb.cand, tb.gcounters, b.fallback, b.fb_best, b.counters, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
