// Tensor-core engine for classified range-domain matching (sm_103a: TMA, tcgen05, TMEM).
//
// The paper (Sections 1-3) compares every range with every domain of its dynamic pool; the
// comparison is a least-squares fit whose only range x domain term is the correlation
// X = sum_p r[p] * T_t(S_d)[p]. Here that term is one dense contraction per tile:
//
//   A_mat[i][p]          = r_i[p] - a_i            (class-sorted range i, fp16, |.| <= 255)
//   B_mat[8 j + t][p]    = T_t(S_{d_j})[p] - c_j   (class-sorted domain j, isometry t, fp16,
//                                                   |.| <= 1020)
//   D[i][8 j + t] = Y    = sum_p A_mat[i][p] * B_mat[8 j + t][p]
//
// with a = round(A / 64) and c = round(C / 64) the integer means (A = sum r, C = sum S). Every
// product and partial sum is an integer of magnitude < 64 * 255 * 1020 < 2^24, so the FP32
// accumulator holds Y exactly, and with alpha = A - 64 a and gamma = C - 64 c (both in
// [-32, 32]) the least-squares numerator is P = 64 X - A C = 64 Y - alpha gamma. A fifth K = 16
// step adds alpha_i * (-gamma_j / 64) (both exact in FP16; only column 64 of the slice is
// non-zero), so the accumulator ends as P / 64 with a relative error of a few 2^-24. The fused
// epilogue takes max_t |P_t| / 64 over the 8 isometry columns, inflates it to cover that error,
// forms the clamped least-squares gain (Section 1's intensity map with |s| <= 1) of it, an upper
// bound of the exact best gain of the pair, and keeps the two best (bound, j) keys per range;
// `k_reeval` evaluates those exactly in integers and certifies that no other domain can be better
// (else the range is re-searched exactly on CUDA cores).
//
// Kernel shape: persistent, one CTA per SM, 10 warps: warp 0 issues TMA loads (A tile 128 x 64,
// B tiles 256 x 64, 128-byte swizzle, a 3-stage ring by default), warp 1 owns TMEM (two 128 x 256 FP32
// accumulators) and issues tcgen05.mma (M = 128, N = 256, K = 16, four per tile), warps 2-9
// (one thread per TMEM lane = range row, two warps per row group, one per accumulator) drain the
// accumulators with tcgen05.ld. Every wait is
// bounded by a wall-clock limit; a timeout sets an error word, lets in-flight copies and MMAs
// finish (bounded), frees TMEM and returns.
#include <cuda.h>

#include <climits>
#include <cstring>
#include <mutex>

#include "fic_internal.cuh"
#include "tc_ptx.cuh"

namespace fic {

bool tensor_engine_available(int device) {
    int major = 0, minor = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return major == 10 && minor == 3;
}

namespace {

// B-operand ring stages (3 or 4: fic_params.pipeline_stages). The default 3: measured 0.1% faster at
// 1024x1024 (matcher 0.885 against 0.887 ms), 0.5% at 4096x4096 and 0.4% on the 64-image batch
constexpr int kStagesDefault = 3;
constexpr int kTileN = 8 * kTileDom;     // 256 accumulator columns
constexpr int kABytes = kTileM * 128;    // 128 rows x 64 fp16
constexpr int kBBytes = kTileN * 128;    // 256 rows x 64 fp16
constexpr int kA1Bytes = kTileM * 32;    // 128 rows x 16 fp16 (correction slice)
constexpr int kB1Bytes = kTileN * 32;    // 256 rows x 16 fp16
constexpr int kEpiWarps = 8;             // two per TMEM lane group, one per accumulator
constexpr int kTcThreads = 32 * (2 + kEpiWarps);
constexpr int kTmemCols = 2 * kTileN;    // two accumulators
// instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = F16 (0), both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);

template <int S>
struct TcShared {
    uint8_t A[2][kABytes];
    uint8_t B[S][kBBytes];
    uint8_t A1[2][kA1Bytes];
    uint8_t B1[S][kB1Bytes];
    // (Q / 256, 128 / Q) of two domains per entry, per epilogue warp set: current, next chunk
    float4 aux[2][2][kChunkDom / 2];
    unsigned long long full_a[2], empty_a[2], full_b[S], empty_b[S], tfull[2],
        tempty[2], aux_ready[2][2], drain, item_full[kItemRing], item_empty[kItemRing],
        never;  // completed by nothing: the forced wait of the testing hook (fic_debug_stall_matcher)
    int item_id[kItemRing];  // work items fetched by the producer, in this CTA's order (-1: none left)
    uint32_t tmem_base;
    int abort_flag;
};
template <int S>
constexpr size_t tc_smem() { return sizeof(TcShared<S>) + 1024; }
static_assert(sizeof(TcShared<4>) + 1024 <= 232448, "shared memory per CTA");

// Scores of one accumulator tile: 32 domains x 8 isometries for this thread's range row. Per
// domain: p = max_t |P_t| / 64, the clamped least-squares gain / 512 of p:
// s = 128 m^2 / Q + (p - m), m = min(p, Q / 256) (the exact gain / 512 up to the accumulator's
// and this formula's rounding), formed as m (m 128 / Q - 1) + p with two FMAs. The inner FMA's
// result lies in [-1, -1/2], so its rounding errs by at most 2^-25 absolutely and the score by
// at most m 2^-25 <= p 2^-25 beyond its relative errors; with |P| <= sqrt(Q_r Q) (Cauchy-Schwarz,
// Q_r = 64 sum r^2 - A^2) and Q <= 64^2 510^2 that is below 2^-16 sqrt(Q_r), a per-range term
// the certification adds to its margin. Each 16 domains of the tile form one ranking group
// (positions jt .. jt + 15 and jt + 16 .. jt + 31, jt a multiple of 32): only the group's largest
// score goes on, as one 32-bit key (its bits with the low 9 replaced by 511 - the group's offset
// in its 512-domain chunk; jrel is the tile's), into t1, t2, the two largest group keys of the
// chunk; the exact re-evaluation evaluates the best group whole, so no domain position within a
// group is kept. MASK: domains outside this row's pool window [lo_r, hi_r) score -1, and a group
// with none inside gives key 0.
__device__ __forceinline__ float absmax8(const uint32_t *v) {
    // a tree of depth two: three independent maxima of magnitudes, then their maximum
    const float a = max3_abs(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]));
    const float b = max3_abs(__uint_as_float(v[3]), __uint_as_float(v[4]), __uint_as_float(v[5]));
    const float c = fmaxf(fabsf(__uint_as_float(v[6])), fabsf(__uint_as_float(v[7])));
    return max3f(a, b, c);
}

// Key of a group whose first domain sits at offset jrel of its chunk: the score's bits with the
// low 9 replaced by base = 511 - jrel (nothing above bit 8), one lop3 of (bits, base, 0xFFFFFE00)
// with the truth table (a & c & ~b) | (b & ~c) = 0x64.
__device__ __forceinline__ uint32_t chunk_key(float sc, uint32_t base) {
    uint32_t key;
    asm("lop3.b32 %0, %1, %2, %3, 0x64;" : "=r"(key) : "r"(__float_as_uint(sc)), "r"(base), "n"(0xFFFFFE00u));
    return key;
}

template <bool MASK>
__device__ __forceinline__ void epi_tile(uint32_t taddr, const float4 *auxp, int jt, int jrel, int lo_r, int hi_r,
                                         uint32_t &t1, uint32_t &t2) {
    float gmax = MASK ? -1.f : 0.f;  // the current group's largest score
    uint32_t va[32], vb[32];
    tmem_ld32(taddr, va);
    tmem_ld_wait(va);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        // columns 32 c .. 32 c + 31 = domains 4 c .. 4 c + 3; the next 32 columns load meanwhile
        if (c < 7) {
            if (c & 1)
                tmem_ld32(taddr + (c + 1) * 32, va);
            else
                tmem_ld32(taddr + (c + 1) * 32, vb);
        }
        const uint32_t *cur = (c & 1) ? vb : va;
        float sv[4];
#pragma unroll
        for (int q2 = 0; q2 < 2; ++q2) {
            // two domains' (Q / 256, 128 / Q) per 16-byte shared load
            const float4 a2 = auxp[2 * c + q2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = 2 * q2 + h, l = 4 * c + q;
                const float qy = h ? a2.z : a2.x, qz = h ? a2.w : a2.y;
                // accumulator = P / 64 up to the FP32 accumulation error, which k_reeval's
                // certification margin covers
                const float p = absmax8(cur + 8 * q);
                const float mm = fminf(p, qy);
                float sc = fmaf(mm, fmaf(mm, qz, -1.f), p);
                if (MASK) {
                    const int j = jt + l;
                    sc = (j >= lo_r && j < hi_r) ? sc : -1.f;
                }
                sv[q] = sc;
            }
        }
        // one link of the running group maximum per 4 domains
        gmax = max3f(gmax, max3f(sv[0], sv[1], sv[2]), sv[3]);
        if ((c & 3) == 3) {
            // the group of domains 16 (c >> 2) .. + 15 is complete
            uint32_t key = chunk_key(gmax, 511u - (uint32_t)(jrel + 16 * (c >> 2)));
            if (MASK && gmax < 0.f) key = 0u;  // no domain of the group in the window
            top2u(t1, t2, key);
            gmax = MASK ? -1.f : 0.f;
        }
        if (c < 7) {
            if (c & 1)
                tmem_ld_wait(va);
            else
                tmem_ld_wait(vb);
        }
    }
}

}  // namespace

// ---- operand packing ------------------------------------------------------------------------
// One thread per (sorted range i, pixel row y): A_mat row i = pixels - round(A / 64), A1 row i =
// (A - 64 round(A / 64), 0, ...); rng_info[i] = (A, pool start, pool end, range id) with the pool
// in batch-wide domain positions (dom_off + position in this image's dom_order). Rows i >= R are
// zero with an empty window and range id -1.
__global__ void k_pack_ranges(Geo g, const uint8_t *__restrict__ img, const int32_t *__restrict__ range_order,
                              const int32_t *__restrict__ rsum, const int32_t *__restrict__ win_lo,
                              const int32_t *__restrict__ win_hi, int R_pad, int dom_off,
                              __half *__restrict__ A_mat, uint4 *__restrict__ A1, int4 *__restrict__ rng_info) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gid >> 3, y = gid & 7;
    if (i >= R_pad) return;
    uint4 pk = make_uint4(0, 0, 0, 0);
    if (i < g.R) {
        const int r = range_order[i];
        const uint8_t *row = img + (size_t)((r / g.nRx) * 8 + y) * g.pitch + (r % g.nRx) * 8;
        const int abar = (rsum[r] + 32) >> 6;  // round(A / 64)
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __half a = __int2half_rn((int)row[2 * h] - abar);
            const __half b = __int2half_rn((int)row[2 * h + 1] - abar);
            w[h] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
        }
        pk = make_uint4(w[0], w[1], w[2], w[3]);
        if (y == 0) {
            rng_info[i] = make_int4(rsum[r], win_lo[r] + dom_off, win_hi[r] + dom_off, r);
            const int alpha = rsum[r] - 64 * abar;
            A1[2 * i] = make_uint4((uint32_t)__half_as_ushort(__int2half_rn(alpha)), 0, 0, 0);
            A1[2 * i + 1] = make_uint4(0, 0, 0, 0);
        }
    } else if (y == 0) {
        rng_info[i] = make_int4(0, 0, 0, -1);
        A1[2 * i] = make_uint4(0, 0, 0, 0);
        A1[2 * i + 1] = make_uint4(0, 0, 0, 0);
    }
    reinterpret_cast<uint4 *>(A_mat + (size_t)i * 64)[y] = pk;
}

// k_pack_ranges for one range tile per 1024-thread block, in class mode, with the work the
// separate window kernels would do: each range's pool window is read off the class offsets
// (classes within w of its own; every domain if that is empty), the image's match count gains
// 8 |window| per range, and the tile's union and intersection of windows and its chunk count
// (as k_tile_windows) are formed by a block reduction. m0: the image's first tile in the batch.
__global__ void __launch_bounds__(1024) k_pack_ranges_tile(Geo g, const uint8_t *__restrict__ img,
                                                           const int32_t *__restrict__ range_order,
                                                           const int32_t *__restrict__ rsum,
                                                           const uint8_t *__restrict__ rbin,
                                                           const int32_t *__restrict__ bin_off, int dom_off, int m0,
                                                           __half *__restrict__ A_mat, uint4 *__restrict__ A1,
                                                           int4 *__restrict__ rng_info, int4 *__restrict__ tile_win,
                                                           int32_t *__restrict__ n_chunks, long long *matches) {
    __shared__ int4 wred[32];
    __shared__ long long mred[32];
    const int i = blockIdx.x * kTileM + (threadIdx.x >> 3), y = threadIdx.x & 7;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 pk = make_uint4(0, 0, 0, 0);
    int lo = 0, hi = 0;
    const bool valid = i < g.R;
    if (valid) {
        const int r = range_order[i];
        const int b = rbin[r];
        lo = bin_off[max(0, b - g.w)];
        hi = bin_off[min(g.K - 1, b + g.w) + 1];
        if (lo == hi) {  // no domain in the window: search every domain
            lo = 0;
            hi = g.Dn;
        }
        const uint8_t *row = img + (size_t)((r / g.nRx) * 8 + y) * g.pitch + (r % g.nRx) * 8;
        const int abar = (rsum[r] + 32) >> 6;  // round(A / 64)
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __half a = __int2half_rn((int)row[2 * h] - abar);
            const __half bb = __int2half_rn((int)row[2 * h + 1] - abar);
            w[h] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(bb) << 16);
        }
        pk = make_uint4(w[0], w[1], w[2], w[3]);
        if (y == 0) {
            rng_info[i] = make_int4(rsum[r], lo + dom_off, hi + dom_off, r);
            const int alpha = rsum[r] - 64 * abar;
            A1[2 * i] = make_uint4((uint32_t)__half_as_ushort(__int2half_rn(alpha)), 0, 0, 0);
            A1[2 * i + 1] = make_uint4(0, 0, 0, 0);
        }
    } else if (y == 0) {
        rng_info[i] = make_int4(0, 0, 0, -1);
        A1[2 * i] = make_uint4(0, 0, 0, 0);
        A1[2 * i + 1] = make_uint4(0, 0, 0, 0);
    }
    reinterpret_cast<uint4 *>(A_mat + (size_t)i * 64)[y] = pk;
    // tile windows (batch-wide positions) and the match count
    int lo_u = valid ? lo + dom_off : INT_MAX, hi_u = valid ? hi + dom_off : INT_MIN;
    int lo_i = valid ? lo + dom_off : INT_MIN, hi_i = valid ? hi + dom_off : INT_MAX;
    long long mc = (valid && y == 0) ? 8LL * (hi - lo) : 0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo_u = min(lo_u, __shfl_xor_sync(0xffffffffu, lo_u, off));
        hi_u = max(hi_u, __shfl_xor_sync(0xffffffffu, hi_u, off));
        lo_i = max(lo_i, __shfl_xor_sync(0xffffffffu, lo_i, off));
        hi_i = min(hi_i, __shfl_xor_sync(0xffffffffu, hi_i, off));
        mc += __shfl_xor_sync(0xffffffffu, mc, off);
    }
    if (lane == 0) {
        wred[warp] = make_int4(lo_u, hi_u, lo_i, hi_i);
        mred[warp] = mc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int4 t = wred[0];
        long long m = mred[0];
        for (int k = 1; k < 32; ++k) {
            t.x = min(t.x, wred[k].x);
            t.y = max(t.y, wred[k].y);
            t.z = max(t.z, wred[k].z);
            t.w = min(t.w, wred[k].w);
            m += mred[k];
        }
        tile_win[m0 + blockIdx.x] = t;
        n_chunks[m0 + blockIdx.x] = t.y > t.x ? (t.y - 1) / kChunkDom - t.x / kChunkDom + 1 : 0;
        if (m) atomicAdd(reinterpret_cast<unsigned long long *>(matches), (unsigned long long)m);
    }
}

// Sixteen domains per 256-thread block: B_mat row 8j+t = T_t(S_{dom_order[j]}) - round(C / 64).
// Sixteen threads per sorted domain j stage its block (one 8-byte load of four elements each) into
// four layouts in shared memory; then each warp writes the rows of two domains, 2 x 8 rows x 128 B,
// lane l of store k taking 16-byte piece 32 k + l (one row y of one isometry t, from one layout row,
// converted pairwise to FP16), so that every store instruction covers 512 contiguous bytes. B1 rows
// are (-gamma / 64, 0, ...) and dom_aux2[j] = (Q / 256, 128 / Q or 0), the constants of the
// epilogue's clamped gain. Entries Dn <= j < n_pad are zero.
__global__ void __launch_bounds__(256) k_pack_domains(Geo g, const uint16_t *__restrict__ domS,
                                                      const int32_t *__restrict__ dom_order,
                                                      const int32_t *__restrict__ dsum,
                                                      const int32_t *__restrict__ dsumsq, int n_pad,
                                                      __half *__restrict__ B_mat, uint4 *__restrict__ B1,
                                                      float2 *__restrict__ dom_aux2) {
    __shared__ __align__(16) uint16_t L[16][4][64];
    __shared__ uint32_t c2s[16], cgs[16];  // per domain: centring pair, -gamma / 64 as FP16 bits
    const int jl = threadIdx.x >> 4, e = threadIdx.x & 15;
    const int j0 = blockIdx.x * 16;
    const int j = j0 + jl;
    if (j < g.Dn) {
        const int d = dom_order[j];
        const int C = dsum[d];
        const int cbar = (C + 32) >> 6;  // round(C / 64)
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(domS + (size_t)d * 64) + e);  // elements 4e .. 4e + 3
        stage_layouts<8>(L[jl], 4 * e, (uint16_t)(v.x & 0xFFFFu));
        stage_layouts<8>(L[jl], 4 * e + 1, (uint16_t)(v.x >> 16));
        stage_layouts<8>(L[jl], 4 * e + 2, (uint16_t)(v.y & 0xFFFFu));
        stage_layouts<8>(L[jl], 4 * e + 3, (uint16_t)(v.y >> 16));
        if (e == 0) {
            c2s[jl] = (0x6400u + (uint32_t)cbar) * 0x10001u;
            const int gamma = C - 64 * cbar;
            cgs[jl] = __half_as_ushort(__float2half_rn(-(float)gamma * (1.0f / 64.0f)));  // exact: |gamma| <= 32
            const long long Q = 64LL * dsumsq[d] - (long long)C * C;
            dom_aux2[j] = make_float2((float)Q * (1.0f / 256.0f), Q > 0 ? 128.0f / (float)Q : 0.f);
        }
    } else if (j < n_pad && e == 0) {
        dom_aux2[j] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int u = 32 * k + lane;  // 16-byte piece of the warp's two domains
        const int dl = 2 * warp + (u >> 6), t = (u >> 3) & 7, y = u & 7;
        const int jj = j0 + dl;
        if (jj >= n_pad) continue;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (jj < g.Dn) {
            const uint4 m = *reinterpret_cast<const uint4 *>(iso_row<8>(L[dl], t, y));
            const uint32_t c2 = c2s[dl];
            val = make_uint4(centred_h2(m.x, c2), centred_h2(m.y, c2), centred_h2(m.z, c2), centred_h2(m.w, c2));
        }
        reinterpret_cast<uint4 *>(B_mat)[(size_t)jj * 64 + (u & 63)] = val;
    }
    {
        // B1: 8 rows x 32 bytes per domain, 16-byte piece lane of the warp's two domains
        const int dl = 2 * warp + (lane >> 4);
        const int jj = j0 + dl;
        if (jj < n_pad) {
            const bool lead = (lane & 1) == 0 && jj < g.Dn;  // first 16 bytes of a row hold the value
            B1[(size_t)jj * 16 + (lane & 15)] = make_uint4(lead ? cgs[dl] : 0u, 0, 0, 0);
        }
    }
}

// One block (TM threads) per range tile of the batch: the union [lo_u, hi_u) of its rows' pool
// windows and the intersection [lo_i, hi_i) over its valid rows; tile_win[m] = (lo_u, hi_u, lo_i,
// hi_i); n_chunks[m] = number of chunks of the absolute grid (batch-wide domain positions
// [512 c, 512 (c + 1))) the union meets.
template <int TM>
__global__ void k_tile_windows(const int4 *__restrict__ rng_info, int4 *__restrict__ tile_win,
                               int32_t *__restrict__ n_chunks) {
    const int m = blockIdx.x, i = m * TM + threadIdx.x;
    const int4 ri = rng_info[i];
    const bool valid = ri.w >= 0;
    int lo_u = valid ? ri.y : INT_MAX, hi_u = valid ? ri.z : INT_MIN;
    int lo_i = valid ? ri.y : INT_MIN, hi_i = valid ? ri.z : INT_MAX;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo_u = min(lo_u, __shfl_xor_sync(0xffffffffu, lo_u, off));
        hi_u = max(hi_u, __shfl_xor_sync(0xffffffffu, hi_u, off));
        lo_i = max(lo_i, __shfl_xor_sync(0xffffffffu, lo_i, off));
        hi_i = min(hi_i, __shfl_xor_sync(0xffffffffu, hi_i, off));
    }
    __shared__ int4 w[TM / 32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = make_int4(lo_u, hi_u, lo_i, hi_i);
    __syncthreads();
    if (threadIdx.x == 0) {
        int4 t = w[0];
        for (int k = 1; k < TM / 32; ++k) {
            t.x = min(t.x, w[k].x);
            t.y = max(t.y, w[k].y);
            t.z = max(t.z, w[k].z);
            t.w = min(t.w, w[k].w);
        }
        tile_win[m] = t;
        n_chunks[m] = t.y > t.x ? (t.y - 1) / kChunkDom - t.x / kChunkDom + 1 : 0;
    }
}

// Block-wide exclusive scan of one int per thread (blockDim.x == 1024); returns the thread's
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ int block_scan_1024(int v, int *sc, int *total) {
    sc[threadIdx.x] = v;
    __syncthreads();
    for (int s = 1; s < 1024; s <<= 1) {
        const int a = threadIdx.x >= (unsigned)s ? sc[threadIdx.x - s] : 0;
        __syncthreads();
        sc[threadIdx.x] += a;
        __syncthreads();
    }
    const int incl = sc[threadIdx.x];
    *total = sc[1023];
    __syncthreads();
    return incl - v;
}

// One block of 1024 threads: the work list and its schedule. Chunks of the absolute grid are
// grouped cpi at a time (domain group G = positions [512 cpi G, 512 cpi (G + 1))), cpi chosen so
// the batch has about `target` items but at most cpi_cap (so one group's B rows stay L2-resident
// while every range tile meeting the group streams them); the last two groups are cut in up to
// four. A work item is (range tile m, group G):
// the part of m's union window inside G, its first domain rounded down to the accumulator tile
// width td (the extra columns lie below every row's window and are masked). tile_items[m] =
// (first key slot, items, first chunk id, chunks): m's items own consecutive key slots in group
// order and its chunks consecutive chunk ids. The schedule (work, work_slot) is group-major, so
// the SMs working at the same time read the same B rows; within a group the order is that of
// the atomic cursor (results do not depend on it: every item writes its own key slot and chunk
// entries). gcounters[1] = items, [3] = chunks, [4] = cpi.
__device__ __forceinline__ int tile_chunk_lo(int4 t) { return t.x / kChunkDom; }
__device__ __forceinline__ int tile_chunk_hi(int4 t) { return (t.y - 1) / kChunkDom + 1; }  // exclusive

__global__ void k_work_list(int n_mtiles, int target, int cpi_cap, int td, int ng_max, int nc,
                            const int4 *__restrict__ tile_win, const int32_t *__restrict__ n_chunks,
                            int4 *__restrict__ work, int32_t *__restrict__ work_slot,
                            int4 *__restrict__ tile_items, int32_t *__restrict__ grp, int32_t *gcounters) {
    __shared__ int sc[1024];
    __shared__ int total_chunks_s;
    // group counters and cursors: in shared memory when they fit (the atomics below are then
    // cheap), else in the global array
    constexpr int kSmemGroups = 8192;
    __shared__ int sgrp[kSmemGroups];
    int *grp_c = ng_max <= kSmemGroups ? sgrp : grp;
    int tot = 0;
    for (int m = threadIdx.x; m < n_mtiles; m += 1024) tot += n_chunks[m];
    int all = 0;
    block_scan_1024(tot, sc, &all);
    if (threadIdx.x == 0) total_chunks_s = all;
    __syncthreads();
    const int total = total_chunks_s;
    const int cpi = max(1, min(cpi_cap, (total + target - 1) / max(1, target)));
    // the last two groups of the grid (nc chunks) are cut into groups of sub = ceil(cpi / 4)
    // chunks: the items taken last are then short, and the persistent CTAs finish closer together
    const int sub = (cpi + 3) / 4;
    const int g1 = sub < cpi ? max(0, (nc + cpi - 1) / cpi - 2) : ng_max;  // full groups before the tail
    const int c1 = g1 * cpi;                                                 // first chunk of the tail
    auto group_of = [=](int ch) { return ch < c1 ? ch / cpi : g1 + (ch - c1) / sub; };
    auto group_lo = [=](int G) { return G < g1 ? G * cpi : c1 + (G - g1) * sub; };  // first chunk
    for (int G = threadIdx.x; G < ng_max; G += 1024) grp_c[G] = 0;
    __syncthreads();
    // key slots and chunk ids per tile (tile-major); group counts
    int item_base = 0, chunk_base = 0;
    for (int m0 = 0; m0 < n_mtiles; m0 += 1024) {
        const int m = m0 + threadIdx.x;
        const int c = m < n_mtiles ? n_chunks[m] : 0;
        int q = 0, glo = 0;
        if (c > 0) {
            const int4 t = tile_win[m];
            glo = group_of(tile_chunk_lo(t));
            q = group_of(tile_chunk_hi(t) - 1) - glo + 1;
        }
        int q_all = 0, c_all = 0;
        const int q_off = item_base + block_scan_1024(q, sc, &q_all);
        const int c_off = chunk_base + block_scan_1024(c, sc, &c_all);
        if (m < n_mtiles) {
            tile_items[m] = make_int4(q_off, q, c_off, c);
            for (int k = 0; k < q; ++k) atomicAdd(&grp_c[glo + k], 1);
        }
        item_base += q_all;
        chunk_base += c_all;
    }
    __syncthreads();
    // exclusive scan of the group counts: grp[G] becomes group G's schedule cursor
    int carry = 0;
    for (int g0 = 0; g0 < ng_max; g0 += 1024) {
        const int G = g0 + threadIdx.x;
        const int v = G < ng_max ? grp_c[G] : 0;
        int g_all = 0;
        const int off = carry + block_scan_1024(v, sc, &g_all);
        if (G < ng_max) grp_c[G] = off;
        carry += g_all;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < n_mtiles; m += 1024) {
        const int4 ti = tile_items[m];
        if (ti.y == 0) continue;
        const int4 t = tile_win[m];
        const int c_lo = tile_chunk_lo(t), glo = group_of(c_lo);
        for (int k = 0; k < ti.y; ++k) {
            const int G = glo + k;
            const int d0 = max(t.x, group_lo(G) * kChunkDom) / td * td;
            const int d1 = min(t.y, group_lo(G + 1) * kChunkDom);
            const int pos = atomicAdd(&grp_c[G], 1);
            work[pos] = make_int4(m, d0, d1, ti.z + d0 / kChunkDom - c_lo);
            work_slot[pos] = ti.x + k;
        }
    }
    if (threadIdx.x == 0) {
        gcounters[1] = item_base;
        gcounters[3] = chunk_base;
        gcounters[4] = cpi;
    }
}

// ---- the matching kernel ----------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_match_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmA1, const __grid_constant__ CUtensorMap tmB1,
               const int4 *__restrict__ work, const int32_t *__restrict__ work_slot,
               const int4 *__restrict__ tile_items,
               const int32_t *__restrict__ counters_in, const int4 *__restrict__ tile_win,
               const int4 *__restrict__ rng_info, const float4 *__restrict__ dom_aux,
               unsigned long long *__restrict__ cand, uint32_t *__restrict__ chunk_max, int32_t *next_item,
               int32_t *err, int32_t *lib_err, unsigned long long stall_ns) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (su32(smem_raw) & 1023u)) & 1023u;
    TcShared<S> &sh = *reinterpret_cast<TcShared<S> *>(smem_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = counters_in[1];
    volatile int *abort_flag = &sh.abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sh.full_a[s], 1);
            mbar_init(&sh.empty_a[s], 1);
            mbar_init(&sh.tfull[s], 1);
            mbar_init(&sh.tempty[s], kEpiWarps / 2);  // the accumulator's four warps
            mbar_init(&sh.aux_ready[0][s], 32 * kEpiWarps / 2);  // one warp set each
            mbar_init(&sh.aux_ready[1][s], 32 * kEpiWarps / 2);
        }
        for (int s = 0; s < S; ++s) {
            mbar_init(&sh.full_b[s], 1);
            mbar_init(&sh.empty_b[s], 1);
        }
        for (int s = 0; s < kItemRing; ++s) {
            mbar_init(&sh.item_full[s], 1);
            mbar_init(&sh.item_empty[s], 1 + kEpiWarps);
        }
        mbar_init(&sh.drain, 1);
        mbar_init(&sh.never, 1);
        sh.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(&sh.tmem_base, kTmemCols);
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
            uint32_t gt = 0;
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
                const int ab = li & 1;
                ok = mbar_wait(&sh.empty_a[ab], ((li >> 1) & 1) ^ 1, abort_flag);
                if (!ok) break;
                mbar_expect_tx(&sh.full_a[ab], kABytes + kA1Bytes);
                tma_load_2d(sh.A[ab], &tmA, &sh.full_a[ab], 0, w.x * kTileM);
                tma_load_2d(sh.A1[ab], &tmA1, &sh.full_a[ab], 0, w.x * kTileM);
                const int nt = (w.z - w.y + kTileDom - 1) / kTileDom;
                for (int k = 0; k < nt; ++k, ++gt) {
                    const int s = gt % S;
                    ok = mbar_wait(&sh.empty_b[s], ((gt / S) & 1) ^ 1, abort_flag);
                    if (!ok) break;
                    mbar_expect_tx(&sh.full_b[s], kBBytes + kB1Bytes);
                    tma_load_2d(sh.B[s], &tmB, &sh.full_b[s], 0, 8 * (w.y + k * kTileDom));
                    tma_load_2d(sh.B1[s], &tmB1, &sh.full_b[s], 0, 8 * (w.y + k * kTileDom));
                }
            }
            if (!ok) {
                report_timeout(err, lib_err, abort_flag);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            uint32_t gt = 0;
            bool ok = true;
            for (uint32_t li = 0; ok; ++li) {
                const int s = li % kItemRing;
                ok = mbar_wait(&sh.item_full[s], (li / kItemRing) & 1, abort_flag);
                if (!ok) break;
                const int it = sh.item_id[s];
                mbar_arrive(&sh.item_empty[s]);
                if (it < 0) break;
                const int4 w = work[it];
                const int ab = li & 1;
                ok = mbar_wait(&sh.full_a[ab], (li >> 1) & 1, abort_flag);
                if (!ok) break;
                tc_fence_after();
                const uint32_t a0 = su32(sh.A[ab]);
                const int nt = (w.z - w.y + kTileDom - 1) / kTileDom;
                for (int k = 0; k < nt; ++k, ++gt) {
                    const int s = gt % S, acc = gt & 1;
                    ok = mbar_wait(&sh.tempty[acc], ((gt >> 1) & 1) ^ 1, abort_flag);
                    if (!ok) break;
                    ok = mbar_wait(&sh.full_b[s], (gt / S) & 1, abort_flag);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t b0 = su32(sh.B[s]);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_f16(tmem + acc * kTileN, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), kIdesc,
                                 kk > 0 ? 1u : 0u);
                    // K = 64..79: alpha_i * (-gamma_j / 64), turning Y into P / 64
                    umma_f16(tmem + acc * kTileN, sw32_desc(su32(sh.A1[ab])), sw32_desc(su32(sh.B1[s])), kIdesc, 1u);
                    umma_commit(&sh.empty_b[s]);
                    umma_commit(&sh.tfull[acc]);
                }
                if (!ok) break;
                umma_commit(&sh.empty_a[ab]);
            }
            // all MMAs issued by this thread complete before TMEM is released
            umma_commit(&sh.drain);
            if (!mbar_wait(&sh.drain, 0, abort_flag) && !*abort_flag) ok = false;
            if (!ok) {
                report_timeout(err, lib_err, abort_flag);
            }
        }
    } else {
        // ---- epilogue: warps 2..9. Warp w reads TMEM lane group (w & 3) (range rows) of every
        // tile of accumulator (w - 2) >> 2 (whole tiles: 32 domains x 8 isometries), so the tiles
        // alternate between the two warp sets and each warp's fixed cost per tile serves 32 domains.
        // The set is the "half" of the chunk and item keys: each set ranks the groups of its tiles.
        const int ew = warp - 2;
        const int lg = warp & 3;
        const int half = ew >> 2;
        const int row = lg * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
        uint32_t gt = 0, lc = 0;  // accumulator tiles and chunks this CTA has processed
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
            const int nt = (w.z - w.y + kTileDom - 1) / kTileDom;
            const int i = w.x * kTileM + row;
            const int4 ri = rng_info[i];
            const bool valid = ri.w >= 0;
            const int lo_r = ri.y, hi_r = min(ri.z, w.z);
            const int4 tw = tile_win[w.x];
            const int f_lo = max(tw.z, w.y), f_hi = min(tw.w, w.z);  // columns valid for every row
            unsigned long long b1 = 0, b2 = 0;
            // accumulator tiles grouped by chunk of the absolute grid (the first chunk of an item
            // may be partial: items start where the tile's window or the domain group starts)
            for (int k0 = 0, ntc = 0; k0 < nt && ok; k0 += ntc, ++lc) {
                const int jc = w.y + k0 * kTileDom;
                const int cabs = jc / kChunkDom;
                ntc = min(nt - k0, ((cabs + 1) * kChunkDom - jc) / kTileDom);
                // per-domain constants of this chunk into the set's shared buffer (double-buffered
                // by chunk parity; a thread reaches chunk lc + 2 only after every thread of its set
                // has left chunk lc). Each set keeps its own copy, so the sets, which drain
                // alternate tiles, do not wait for each other at chunk boundaries.
                const int ab = lc & 1;
                for (int k = (ew & 3) * 32 + lane; k < ntc * kTileDom / 2; k += 32 * (kEpiWarps / 2))
                    sh.aux[half][ab][k] = __ldg(&dom_aux[jc / 2 + k]);  // dom_aux holds float2 pairs here
                mbar_arrive(&sh.aux_ready[half][ab]);
                ok = __all_sync(0xffffffffu, mbar_wait(&sh.aux_ready[half][ab], (lc >> 1) & 1, abort_flag));
                if (!ok) break;
                // the chunk's two best 32-bit keys, folded into the 64-bit keys once per chunk
                uint32_t t1 = 0, t2 = 0;
                const int jrel0 = jc - cabs * kChunkDom;
                for (int k = 0; k < ntc; ++k, ++gt) {
                    const int acc = gt & 1;
                    if (acc != half) continue;  // the other set's tile
                    ok = __all_sync(0xffffffffu, mbar_wait(&sh.tfull[acc], (gt >> 1) & 1, abort_flag));
                    if (!ok) break;
                    tc_fence_after();
                    const int jt = jc + k * kTileDom;
                    const float4 *auxp = &sh.aux[half][ab][(k * kTileDom) / 2];
                    const uint32_t taddr = tbase + acc * kTileN;
                    const int jrel = jrel0 + k * kTileDom;
                    if (jt >= f_lo && jt + kTileDom <= f_hi)
                        epi_tile<false>(taddr, auxp, jt, jrel, lo_r, hi_r, t1, t2);
                    else
                        epi_tile<true>(taddr, auxp, jt, jrel, lo_r, hi_r, t1, t2);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh.tempty[acc]);
                }
                merge_chunk_key(b1, b2, t1, cabs * kChunkDom);
                merge_chunk_key(b1, b2, t2, cabs * kChunkDom);
                if (ok && valid)
                    reinterpret_cast<uint2 *>(chunk_max)[((size_t)(w.w + cabs - w.y / kChunkDom) * kTileM + row) * 2 + half] =
                        make_uint2(t1, t2 & 0xFFFFFE00u);
            }
            if (ok && valid) {
                // the tile's keys are row-major (row, item, half, 2): a range reads its keys at once
                const int4 ti = tile_items[w.x];
                unsigned long long *dst =
                    cand + (size_t)ti.x * kTileM * 4 + (((size_t)row * ti.y + (work_slot[it] - ti.x)) * 2 + half) * 2;
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
        // give TMA loads already issued time to land before shared memory is released
        const unsigned long long t0 = gtimer();
        while (gtimer() - t0 < 5000000ull) {
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ---- exact re-evaluation and certification ----------------------------------------------------
constexpr int kReevalThreads = 256;
// Per-warp staging of one range: its 8 inverse-permuted copies rp[t][src_t(p)] = r[p].
struct __align__(16) ReevalStage {
    uint8_t rp[8][64];
};

// One half-warp's exact best, left for the block's finishing lanes. kind 0: no range; 1: flat range
// (its code as is); 2: ranked range (certify, then code or queue). u2: the runner-up key's score
// bits.
struct ReevalRes {
    long long num, den, P, Q, A, Bs;
    int C, d, t, r, i;
    uint32_t u2;
    int kind, has1, has2;
};

// Exact evaluation of class-sorted range position i by one half-warp (lanes hmask, hl = lane
// mod 16; see k_reeval).
__device__ __forceinline__ void reeval_rank(const Geo &g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
                                            const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
                                            const int32_t *__restrict__ rsumsq, const int32_t *__restrict__ dom_order,
                                            const int32_t *__restrict__ bin_off, int nbuckets,
                                            const int4 *__restrict__ rng_info, int rng_off, int dom_off,
                                            const int4 *__restrict__ tile_items,
                                            const unsigned long long *__restrict__ cand, int i, int hl, unsigned hmask,
                                            ReevalStage &sg, ReevalRes &res) {
    const int4 ri = rng_info[i];
    const int r = ri.w;
    const long long A = ri.x, Bs = rsumsq[r];
    const int ry = (r / g.nRx) * 8, rx = (r % g.nRx) * 8;
    // the range's 8 inverse-permuted copies, staged before the key merge so that the pixel loads
    // overlap the key loads (a flat range does not use them)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int px = 4 * hl + k, y = px >> 3, x = px & 7;
        const uint8_t v = img[(size_t)(ry + y) * g.pitch + rx + x];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int sy, sx;
            iso_src(8, t, y, x, sy, sx);
            sg.rp[t][sy * 8 + sx] = v;
        }
    }

    if (64LL * Bs - A * A == 0) {  // flat range
        // the pool is a union of whole sort buckets, each holding ascending domain ids: the
        // smallest id of the pool is the smallest first entry of a bucket inside the window
        int dmin = INT_MAX;
        const int wlo = ri.y - dom_off, whi = ri.z - dom_off;
        for (int bb = hl; bb < nbuckets; bb += 16)
            if (bin_off[bb] < bin_off[bb + 1] && bin_off[bb] >= wlo && bin_off[bb] < whi)
                dmin = min(dmin, dom_order[bin_off[bb]]);
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) dmin = min(dmin, __shfl_xor_sync(hmask, dmin, off));
        if (hl == 0) {
            const long long C = dsum[dmin];
            const long long Q = 64LL * dsumsq[dmin] - C * C;
            // X = (A / 64) C exactly for a constant block, so P = 64 X - A C = 0
            const Gain g0 = exact_gain(0, Q);
            res = ReevalRes{g0.num, g0.den, 0, Q, A, Bs, (int)C, dmin, 0, r, i, 0u, 1, 1, 0};
        }
        return;
    }

    // merge the top-2 keys of all work items of this range's tile
    const int ig = rng_off + i;
    const int row = ig % kTileM;
    const int4 ti = tile_items[ig / kTileM];
    unsigned long long b1 = 0, b2 = 0;
    const unsigned long long *ck = cand + (size_t)ti.x * kTileM * 4 + (size_t)row * ti.y * 4;
    for (int e = hl; e < 4 * ti.y; e += 16) top2(b1, b2, ck[e]);
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(hmask, b1, off);
        const unsigned long long o2 = __shfl_xor_sync(hmask, b2, off);
        top2(b1, b2, o1);
        top2(b1, b2, o2);
    }
    // exact evaluation of the best key's group: the epilogue ranks 16-domain groups by their best
    // key, so every domain outside that group scores at most the runner-up key, and only the
    // group's domains inside the pool window can be certified (the runner-up's own domain is
    // bounded by its key, so it can never pass the test below). With the range's inverse-permuted
    // copies staged above, lane hl forms X_t of the group's domain hl for all 8 isometries
    // exactly (corr8) and keeps its best (gain, then smaller t); a half-warp reduction keeps the
    // best (gain, then smaller domain id, then smaller t).
    __syncwarp(hmask);
    const int p1 = (int)(~(uint32_t)(b1 & 0xffffffffu));  // batch-wide positions
    int pos = b1 != 0 ? (p1 & ~15) + hl : -1;
    if (pos < ri.y || pos >= ri.z) pos = -1;
    Gain gg{-1, 1};
    int d = INT_MAX, bt = 0;
    long long P = 0, Q = 0, C = 0;
    if (pos >= 0) {
        d = dom_order[pos - dom_off];
        unsigned X[8];
        corr8<8>(sg.rp, domS + (size_t)d * 64, X);
        C = dsum[d];
        Q = 64LL * dsumsq[d] - C * C;
        // with the domain (so Q and C) fixed the clamped gain grows with |P|: the best isometry
        // is the largest |P|, ties to the smaller t (a flat domain has P = 0 for every t)
        P = 64LL * (long long)X[0] - A * C;
        long long aP = P < 0 ? -P : P;
#pragma unroll
        for (int t = 1; t < 8; ++t) {
            const long long Pt = 64LL * (long long)X[t] - A * C;
            const long long at = Pt < 0 ? -Pt : Pt;
            if (at > aP) {
                aP = at;
                bt = t;
                P = Pt;
            }
        }
        gg = exact_gain(P, Q);
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
        const Gain og{__shfl_xor_sync(hmask, gg.num, off), __shfl_xor_sync(hmask, gg.den, off)};
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
        res = ReevalRes{gg.num, gg.den, P, Q, A, Bs, (int)C, d, bt, r, i, (uint32_t)(b2 >> 32), 2, b1 != 0, b2 != 0};
}

// Certification, code or queueing of one evaluated range (one thread). The FP64 steps run here,
// one lane per range, so that one warp's FP64 instructions serve all the block's ranges: FP64
// throughput on sm_103 is a small fraction of FP32, and with each warp finishing its own range on
// one lane the FP64 pipe was this kernel's limit.
__device__ __forceinline__ void reeval_finish(const ReevalRes &e, int32_t *__restrict__ fallback,
                                              FallbackBest *__restrict__ fb_best, int32_t *counters,
                                              const fic_codes &out) {
    if (e.kind == 0) return;
    const Gain gg{e.num, e.den};
    bool certified = e.kind == 1 || (e.has1 && gg.num >= 0);
    if (e.kind == 2 && certified && e.has2) {
        // runner-up score (truncated key) * (1 + 2^-13) + 2^-16 bounds every other domain's exact
        // gain / 512: the key drops < 2^-14 relatively (9 low bits hold the chunk offset), the
        // FP32 score formula errs < 20 * 2^-24 relatively, and the accumulator's P / 64 (an exact
        // integer Y plus one rounded correction of magnitude <= 16) errs < 2^-22 (|P / 64| + 16);
        // the score's slope in p is at most 1, so that moves it by < 2^-21 relatively plus
        // < 2^-18 absolutely; the score's inner FMA adds < 2^-16 sqrt(Q_r) absolutely (epi_tile)
        const double u2 = (double)__uint_as_float(e.u2);
        const double sq = (double)__fsqrt_ru(__ll2float_ru(64LL * e.Bs - e.A * e.A));
        // bound < exact gain / 512, compared as bound * 512 den < gain numerator (no division)
        certified = (u2 * (1.0 + 1.0 / 8192.0) + (1.0 + sq) / 65536.0) * (512.0 * (double)gg.den) < (double)gg.num;
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
    finalize_code(64, e.A, e.Bs, e.C, e.P, e.Q, gg, s, o, sse);
    out.dom[e.r] = e.d;
    out.iso[e.r] = e.t;
    out.s[e.r] = s;
    out.o[e.r] = o;
    out.sse[e.r] = sse;
}

// One half-warp per class-sorted range position i of one image. Merges the range's top-2 group
// keys over its tile's work items, evaluates the best key's 16-domain group under all 8
// isometries exactly, keeps the best (gain, then smaller domain id, then smaller isometry) and
// certifies it: every domain outside the evaluated group has an FP32 score at most the runner-up
// key's, and an FP32 score is an upper bound of that domain's exact gain / 512 up to a relative
// 20 * 2^-24 (it is formed from exact integers and 24-bit constants by a handful of
// single-rounding operations) and an absolute 2^-16 sqrt(Q_r) (Q_r = 64 sum r^2 - A^2), so if
// runner-up * (1 + 2^-13) + 2^-16 (1 + sqrt(Q_r)) < exact best, no other domain can win or tie. Otherwise the range is queued with its exact best for k_rescan. Flat ranges
// (n Bs = A^2) have zero error for every candidate; their code is the smallest domain id of the
// pool with t = 0.
__global__ void k_reeval(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
                         const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
                         const int32_t *__restrict__ rsumsq, const int32_t *__restrict__ dom_order,
                         const int32_t *__restrict__ bin_off, int nbuckets,
                         const int4 *__restrict__ rng_info, int rng_off, int dom_off,
                         const int4 *__restrict__ tile_items, const unsigned long long *__restrict__ cand,
                         const int32_t *__restrict__ gcounters, int32_t *__restrict__ fallback,
                         FallbackBest *__restrict__ fb_best, int32_t *counters, fic_codes out) {
    __shared__ ReevalStage stage[kReevalThreads / 16];
    __shared__ ReevalRes res[kReevalThreads / 16];
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 4;  // sorted position in this image
    const int hl = threadIdx.x & 15, slot = threadIdx.x >> 4;
    const unsigned hmask = 0xFFFFu << (threadIdx.x & 16);  // this half-warp
    if (gcounters[2] != 0) {
        // the matching kernel gave up: its keys are not trusted, so every code is marked invalid
        if (hl == 0 && i < g.R) poison_code(out, i);
        return;
    }
    if (i < g.R)
        reeval_rank(g, img, domS, dsum, dsumsq, rsumsq, dom_order, bin_off, nbuckets, rng_info, rng_off, dom_off,
                    tile_items, cand, i, hl, hmask, stage[slot], res[slot]);
    else if (hl == 0)
        res[slot].kind = 0;
    __syncthreads();
    if (threadIdx.x < kReevalThreads / 16) reeval_finish(res[threadIdx.x], fallback, fb_best, counters, out);
}

// ---- host side -------------------------------------------------------------------------------
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    return fn;
}

}  // namespace

cudaError_t make_map_f16(CUtensorMap *map, void *base, unsigned long long rows, unsigned cols, unsigned box_rows,
                         unsigned box_cols) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE,
                    box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {
}  // namespace

cudaError_t launch_pack(const uint8_t *img, const Geo &g, const EncodeBufs &b, cudaStream_t st, int part) {
    if (part != 2) {
        const long long n = (long long)b.R_pad * 8;
        k_pack_ranges<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, img, b.range_order, b.range_sum, b.win_lo,
                                                                  b.win_hi, b.R_pad, b.dom_off, b.A_mat,
                                                                  (uint4 *)b.A1_mat, b.rng_info);
        ++g_launches;
    }
    if (part != 1) {
        const long long n = (long long)b.Dn_aux * 16;
        k_pack_domains<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, b.dom_S, b.dom_order, b.dom_sum,
                                                                   b.dom_sumsq, b.Dn_aux, b.B_mat, (uint4 *)b.B1_mat,
                                                                   // float2 pairs indexed by batch-wide domain position
                                                                   reinterpret_cast<float2 *>(b.dom_aux - b.dom_off) +
                                                                       b.dom_off);
        ++g_launches;
    }
    return cudaGetLastError();
}

cudaError_t launch_pack_ranges_tiles(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                                     cudaStream_t st) {
    k_pack_ranges_tile<<<b.R_pad / kTileM, 1024, 0, st>>>(g, img, b.range_order, b.range_sum, b.range_bin, b.bin_off,
                                                         b.dom_off, b.mt_off, b.A_mat, (uint4 *)b.A1_mat,
                                                         b.rng_info, tb.tile_win, tb.n_chunks, b.matches);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_work_list(const TcBatch &tb, int target_items, cudaStream_t st, bool tiles_done) {
    if (!tiles_done) {
        if (tb.tm == 2 * kTileM)
            k_tile_windows<2 * kTileM><<<tb.n_mtiles, 2 * kTileM, 0, st>>>(tb.rng_info, tb.tile_win, tb.n_chunks);
        else
            k_tile_windows<kTileM><<<tb.n_mtiles, kTileM, 0, st>>>(tb.rng_info, tb.tile_win, tb.n_chunks);
        ++g_launches;
    }
    const int target = max(1, min(target_items, kMaxItemTarget));
    k_work_list<<<1, 1024, 0, st>>>(tb.n_mtiles, target, tb.cpi_cap, tb.B == 16 ? 16 : kTileDom, tb.ng_max,
                                    (tb.Dn_aux + kChunkDom - 1) / kChunkDom, tb.tile_win, tb.n_chunks, tb.work, tb.work_slot, tb.tile_items, tb.grp,
                                    tb.gcounters);
    ++g_launches;
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_tc_variant(const CUtensorMap &tmA, const CUtensorMap &tmB, const CUtensorMap &tmA1,
                              const CUtensorMap &tmB1, const TcBatch &tb, int grid, cudaStream_t st) {
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(k_match_tc<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<S>());
    });
    if (attr_err) return attr_err;
    k_match_tc<S><<<grid, kTcThreads, tc_smem<S>(), st>>>(tmA, tmB, tmA1, tmB1, tb.work, tb.work_slot, tb.tile_items,
                                                         tb.gcounters, tb.tile_win, tb.rng_info, tb.dom_aux, tb.cand,
                                                         tb.chunk_max, tb.gcounters + 5, tb.gcounters + 2,
                                                         tb.lib_error, tb.stall_ns);
    return cudaGetLastError();
}

cudaError_t launch_match_tc(const TcBatch &tb, int num_sms, cudaStream_t st) {
    CUtensorMap tmA, tmB, tmA1, tmB1;
    cudaError_t e;
    if ((e = make_map_f16(&tmA, tb.A_mat, (unsigned long long)tb.R_pad, 64, kTileM, 64))) return e;
    if ((e = make_map_f16(&tmB, tb.B_mat, (unsigned long long)tb.Dn_aux * 8, 64, kTileN, 64))) return e;
    if ((e = make_map_f16(&tmA1, tb.A1_mat, (unsigned long long)tb.R_pad, 16, kTileM, 16))) return e;
    if ((e = make_map_f16(&tmB1, tb.B1_mat, (unsigned long long)tb.Dn_aux * 8, 16, kTileN, 16))) return e;
    const int grid = num_sms < tb.max_items ? num_sms : tb.max_items;
    if (grid <= 0) return cudaSuccess;
    if (tb.stages == 4)
        e = launch_tc_variant<4>(tmA, tmB, tmA1, tmB1, tb, grid, st);
    else
        e = launch_tc_variant<3>(tmA, tmB, tmA1, tmB1, tb, grid, st);
    if (e) return e;
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_reeval(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                          const fic_codes &out, cudaStream_t st) {
    const long long threads = (long long)g.R * 16;
    k_reeval<<<(unsigned)((threads + kReevalThreads - 1) / kReevalThreads), kReevalThreads, 0, st>>>(
        g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sumsq, b.dom_order, b.bin_off, sort_buckets(g), b.rng_info,
        b.rng_off, b.dom_off, tb.tile_items, tb.cand, tb.gcounters, b.fallback, b.fb_best, b.counters, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
