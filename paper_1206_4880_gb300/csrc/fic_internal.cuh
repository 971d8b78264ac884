// Internal declarations of the fic CUDA library (sm_103a). Not part of the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/fic.h"

namespace fic {

constexpr int kMaxClasses = 255;

// An NVTX range named after the entry point for the duration of a host call (what a profiler's
// timeline shows as the call's enqueue time; nothing is recorded unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Kernels launched by the current fic_* call on this thread (reset at each entry point).
extern thread_local int g_launches;

// Division by an invariant divisor 1 <= d < 2^31 of dividends 0 <= x < 2^31 with one multiply-high,
// one add and one shift (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994): s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1, q = (mulhi(x, m) + x) >> s.
// The kernels index ranges and domains by row-major ids, and a division by a value known only at
// run time costs tens of instructions.
struct FastDiv {
    uint32_t d = 1, m = 1, s = 0;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    f.d = d;
    while ((1u << f.s) < d) ++f.s;
    f.m = (uint32_t)((((unsigned long long)1 << 32) * (((unsigned long long)1 << f.s) - d)) / d + 1);
    return f;
}
__device__ __forceinline__ int fdiv(int x, const FastDiv &f) {
    return (int)((__umulhi((uint32_t)x, f.m) + (uint32_t)x) >> f.s);
}

// Derived geometry of one image (Section 1 range partition, Section 2 domain grid).
struct Geo {
    int H, W, pitch;
    int B, n, sigma;     // range side, pixels per range, domain stride
    int nRy, nRx, R;     // range grid
    int nDy, nDx, Dn;    // domain grid
    int K, w;            // classes and pool half-width (Section 3.1 Eq. 2-3)
    int literal;         // 1: Eq. 3 window on FD values (FIC_FLAG_LITERAL_WINDOW)
    FastDiv fRx, fDx, fS;  // division by nRx, by nDx and by sigma
    int group_chunks;    // tensor engine: chunk cap of a domain group
    int stages;          // tensor engine: B-operand ring stages (0: the kernel's default)
};

// Correctly rounded log2(n) for n = 0..512 (entry 0 unused; box counts of 16x16 blocks reach
// 512); passed to kernels by value.
struct Log2Tab {
    double v[513];
};
const Log2Tab &log2_table();
double log2_correctly_rounded(int n);

// ----------------------------------------------------------------------------------------
// Square isometries: (T_t X)[y][x] = X[sy][sx], N = B - 1:
//   t: 0 (y, x)  1 (N-x, y)  2 (N-y, N-x)  3 (x, N-y)  4 (y, N-x)  5 (N-y, x)  6 (x, y)  7 (N-x, N-y).
// Written without branches (threads of a warp often hold different t): (u, v) = (y, x), swapped
// for t in {1, 3, 6, 7}; sy = u mirrored for t in {1, 2, 5, 7}; sx = v mirrored for t in {2, 3, 4, 7}.
__host__ __device__ __forceinline__ void iso_src(int B, int t, int y, int x, int &sy, int &sx) {
    const int N = B - 1;
    const bool swap = (0xCA >> t) & 1, fy = (0xA6 >> t) & 1, fx = (0x9C >> t) & 1;
    const int u = swap ? x : y, v = swap ? y : x;
    sy = fy ? N - u : u;
    sx = fx ? N - v : v;
}

// Whether a code's domain and isometry can be used to index the image: decoding kernels skip
// invalid codes (such as those an encode writes when its matcher gave up) instead of reading
// outside the image.
__host__ __device__ __forceinline__ bool valid_code(const Geo &g, int d, int t) {
    return (unsigned)d < (unsigned)g.Dn && (unsigned)t < 8u;
}

// Exact correlations of one domain block with a range under all 8 isometries: X_t = sum_q S[q]
// rp[t][q], where rp[t][q] = r[p] with iso_src(t, p) = q (the range's 8 inverse-permuted byte
// copies, 16-byte aligned rows) and S is the domain's block of B*B 16-bit 2x2 sums (16-byte
// aligned). Two products per __dp2a (a pair of sums against two bytes), 16 source indices per
// step, unsigned: X < B^2 * 255 * 1020 < 2^31.
// corr<B, NT>(rp, S, X) forms X_t of isometries t = 0 .. NT - 1 of the rows it is given (rp + t0
// for isometries t0 .. t0 + NT - 1); corr8 is all eight.
template <int B, int NT>
__device__ __forceinline__ void corr(const uint8_t (*rp)[B * B], const uint16_t *__restrict__ S, unsigned (&X)[NT]) {
    constexpr int n = B * B;
    const uint4 *Sd = reinterpret_cast<const uint4 *>(S);
#pragma unroll
    for (int t = 0; t < NT; ++t) X[t] = 0;
#pragma unroll(B == 8 ? 4 : 2)
    for (int q0 = 0; q0 < n; q0 += 16) {
        const uint4 sa = __ldg(Sd + q0 / 8), sb = __ldg(Sd + q0 / 8 + 1);  // S[q0 .. q0 + 15]
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const uint4 r = *reinterpret_cast<const uint4 *>(&rp[t][q0]);  // rp[t][q0 .. q0 + 15]
            unsigned acc = X[t];
            acc = __dp2a_lo(sa.x, r.x, acc);
            acc = __dp2a_hi(sa.y, r.x, acc);
            acc = __dp2a_lo(sa.z, r.y, acc);
            acc = __dp2a_hi(sa.w, r.y, acc);
            acc = __dp2a_lo(sb.x, r.z, acc);
            acc = __dp2a_hi(sb.y, r.z, acc);
            acc = __dp2a_lo(sb.z, r.w, acc);
            acc = __dp2a_hi(sb.w, r.w, acc);
            X[t] = acc;
        }
    }
}
template <int B>
__device__ __forceinline__ void corr8(const uint8_t (*rp)[B * B], const uint16_t *__restrict__ S, unsigned (&X)[8]) {
    corr<B, 8>(rp, S, X);
}

// Four layouts of a block S (side B, N = B - 1) in shared memory: L0 as stored, L1 transposed,
// L2 with each row reversed, L3[a][b] = S[N - b][a]. Row y of the isometry T_t(S) of iso_src is
// then one contiguous row: row (swap ? fx : fy) ? N - y : y of layout swap + 2 (swap ? fy : fx).
// stage_layouts places element e = B a + b of S in all four.
template <int B>
__device__ __forceinline__ void stage_layouts(uint16_t (*L)[B * B], int e, uint16_t v) {
    const int a = e / B, b = e % B, N = B - 1;
    L[0][a * B + b] = v;
    L[1][b * B + a] = v;
    L[2][a * B + N - b] = v;
    L[3][b * B + N - a] = v;
}
template <int B>
__device__ __forceinline__ const uint16_t *iso_row(const uint16_t (*L)[B * B], int t, int y) {
    const int swap = (0xCA >> t) & 1, fy = (0xA6 >> t) & 1, fx = (0x9C >> t) & 1;
    const int row = (swap ? fx : fy) ? B - 1 - y : y;
    return L[swap + 2 * (swap ? fy : fx)] + row * B;
}

// FP16 pair (v0 - c, v1 - c) from packed 16-bit integers v0, v1 in [0, 1023] (pair = v0 | v1 << 16)
// and cpair = (0x6400 + c) * 0x10001, c in [0, 1023]: 0x6400 + v is the FP16 pattern of 1024 + v,
// and the difference of two such values is an integer of magnitude < 1024, exact in FP16.
__device__ __forceinline__ uint32_t centred_h2(uint32_t pair, uint32_t cpair) {
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(pair + 0x64006400u), "r"(cpair));
    return r;
}

// ----------------------------------------------------------------------------------------
// Exact least-squares gain of one candidate (B = 8, n = 64).
// With P = n X - A C and Q = n E - C^2, 16 n SSE = 16 (n Bs - A^2) - gain where
//   gain = 16 P^2 / Q   (Q > 0, 4|P| <= Q; contrast s = 4P/Q not clamped)
//   gain = 8 |P| - Q    (4|P| > Q; s clamped to sign(P))
//   gain = 0            (Q = 0; flat domain, s = 0).
// For n = 64: |P| < 2^28, 16 P^2 < 2^61, Q < 2^31, so num/den fit in int64 and cross products
// in 128 bits.
struct Gain {
    long long num, den;  // gain = num / den, den > 0
};

__device__ __forceinline__ Gain exact_gain(long long P, long long Q) {
    Gain g;
    const long long aP = P < 0 ? -P : P;
    if (Q == 0) {
        g.num = 0;
        g.den = 1;
    } else if (4 * aP <= Q) {
        g.num = 16 * P * P;
        g.den = Q;
    } else {
        g.num = 8 * aP - Q;
        g.den = 1;
    }
    return g;
}

__device__ __forceinline__ int gain_cmp(Gain a, Gain b) {
    const __int128 l = (__int128)a.num * b.den, r = (__int128)b.num * a.den;
    return l > r ? 1 : (l < r ? -1 : 0);
}

// Candidate order: larger gain, then smaller domain id, then smaller isometry.
__device__ __forceinline__ bool cand_better(Gain ga, int da, int ta, Gain gb, int db, int tb) {
    const int c = gain_cmp(ga, gb);
    if (c != 0) return c > 0;
    if (da != db) return da < db;
    return ta < tb;
}

// Contrast, brightness and collage error of the chosen candidate in binary64, from exact
// integers, with explicit rounding (no contraction).
__device__ __forceinline__ void finalize_code(int n, long long A, long long Bs, long long C,
                                              long long P, long long Q, Gain g, double &s,
                                              double &o, double &sse) {
    const long long aP = P < 0 ? -P : P;
    if (Q == 0)
        s = 0.0;
    else if (4 * aP <= Q)
        s = __ddiv_rn(__dmul_rn(4.0, (double)P), (double)Q);
    else
        s = P > 0 ? 1.0 : -1.0;
    // C / 4 and the division by n (a power of two) are exact scalings: multiplications by the
    // exact reciprocals give the same doubles as the divisions, without the FP64 divide sequence
    o = __dmul_rn(__dsub_rn((double)A, __dmul_rn(s, __dmul_rn((double)C, 0.25))), 1.0 / (double)n);
    const long long base = 16 * ((long long)n * Bs - A * A);
    const long long num = base * g.den - g.num;  // < 2^62 for n = 64
    sse = __ddiv_rn((double)num, __dmul_rn(__dmul_rn(16.0, (double)n), (double)g.den));
}

// ----------------------------------------------------------------------------------------
// The same for B = 16 (n = 256): |P| < 2^35 and Q < 2^37, so 16 P^2 needs 128 bits.
struct GainW {
    __int128 num;
    long long den;
};

__device__ __forceinline__ GainW exact_gain_w(long long P, long long Q) {
    GainW g;
    const long long aP = P < 0 ? -P : P;
    if (Q == 0) {
        g.num = 0;
        g.den = 1;
    } else if (4 * aP <= Q) {
        g.num = (__int128)16 * ((__int128)P * (__int128)P);
        g.den = Q;
    } else {
        g.num = (__int128)(8 * aP - Q);
        g.den = 1;
    }
    return g;
}

__device__ __forceinline__ int gain_cmp(GainW a, GainW b) {
    const __int128 l = a.num * (__int128)b.den, r = b.num * (__int128)a.den;  // < 2^113
    return l > r ? 1 : (l < r ? -1 : 0);
}

__device__ __forceinline__ bool cand_better(GainW ga, int da, int ta, GainW gb, int db, int tb) {
    const int c = gain_cmp(ga, gb);
    if (c != 0) return c > 0;
    if (da != db) return da < db;
    return ta < tb;
}

// Round-to-nearest-even conversion of a 128-bit integer: the top 64 significant bits with the
// dropped bits folded into bit 0 (a sticky bit well below the rounding position) convert to the
// same double as the whole value; the power-of-two scaling is exact.
__device__ __forceinline__ double i128_to_double_rn(__int128 v) {
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    double r;
    if (hi == 0) {
        r = __ull2double_rn(lo);
    } else {
        const int sh = 64 - __clzll((long long)hi);  // 1..64 bits above the low word
        unsigned long long top = (unsigned long long)(u >> sh);
        const unsigned long long dropped = sh == 64 ? lo : (lo & ((1ull << sh) - 1ull));
        top |= dropped != 0ull ? 1ull : 0ull;
        r = __dmul_rn(__ull2double_rn(top), __longlong_as_double((long long)(1023 + sh) << 52));
    }
    return neg ? -r : r;
}

__device__ __forceinline__ void finalize_code(int n, long long A, long long Bs, long long C,
                                              long long P, long long Q, GainW g, double &s,
                                              double &o, double &sse) {
    const long long aP = P < 0 ? -P : P;
    if (Q == 0)
        s = 0.0;
    else if (4 * aP <= Q)
        s = __ddiv_rn(__dmul_rn(4.0, (double)P), (double)Q);
    else
        s = P > 0 ? 1.0 : -1.0;
    // C / 4 and the division by n (a power of two) are exact scalings: multiplications by the
    // exact reciprocals give the same doubles as the divisions, without the FP64 divide sequence
    o = __dmul_rn(__dsub_rn((double)A, __dmul_rn(s, __dmul_rn((double)C, 0.25))), 1.0 / (double)n);
    const long long base = 16 * ((long long)n * Bs - A * A);  // < 2^37
    const __int128 num = (__int128)base * (__int128)g.den - g.num;
    sse = __ddiv_rn(i128_to_double_rn(num), __dmul_rn(__dmul_rn(16.0, (double)n), (double)g.den));
}

// Gain type and exact gain of a B x B block.
template <int B>
struct FitOf;
template <>
struct FitOf<8> {
    using G = Gain;
    __device__ static __forceinline__ G gain(long long P, long long Q) { return exact_gain(P, Q); }
};
template <>
struct FitOf<16> {
    using G = GainW;
    __device__ static __forceinline__ G gain(long long P, long long Q) { return exact_gain_w(P, Q); }
};

// Exact best of the evaluated candidates of a range the ranking could not certify (num < 0:
// none).
struct __align__(16) FallbackBest {
    __int128 num;
    long long den, P, Q;
    int d, t, C, pad;
};

// ----------------------------------------------------------------------------------------
// Workspace carving.
struct Carver {
    char *base;
    size_t off, cap;
    bool ok;
    explicit Carver(void *b, size_t c) : base((char *)b), off(0), cap(c), ok(true) {}
    template <class T>
    T *take(size_t count, size_t align = 256) {
        off = (off + align - 1) / align * align;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        if (off > cap) ok = false;
        return p;
    }
};

// Encode-side internal buffers (all device, carved from the caller's workspace).
struct EncodeBufs {
    // classification
    int32_t *range_sum, *range_sumsq, *range_counts;
    double *range_fd;
    uint8_t *range_bin;
    int32_t *dom_sum, *dom_sumsq, *dom_counts;
    double *dom_fd;
    uint8_t *dom_bin;
    double *fd_extent;
    unsigned long long *extent_bits;  // [2] min/max FD bit patterns during the reduction
    uint16_t *dom_S;                  // [Dn][n] integer 2x2 sums of every domain (n = B^2)
    // pools
    int32_t *dom_order, *bin_off, *range_order, *rbin_off, *win_lo, *win_hi;
    uint8_t *dom_key, *range_key;  // [Dn], [R] sort keys (class, or FD rank in literal mode)
    int nbuckets;          // sort buckets: K, or the number of distinct FD values
    int32_t *sort_counts;  // [256][nblk rounded up to 4] per-block class histograms of the domain sort
    int32_t *sort_offs;    // the same for the range sort
    // literal window with 16x16 ranges: FD-rank keys (up to 12 bits) radix-sorted
    int32_t *lit_key, *lit_t1, *lit_t2, *lit_counts;  // [max(R, Dn)] keys and sort buffers, histograms
    int32_t *lit_rank;     // [kFdPairs16] key of every (N_2, N_8) pair
    uint8_t *lit_digit;    // [max(R, Dn)] radix digits
    double *lit_sfd;       // [Dn] FDs of the FD-sorted domains
    // tensor engine: this image's slice of the batch-wide arrays (TcBatch)
    __half *A_mat;         // [R_pad][n]   range pixels - a, class-sorted ranges
    __half *B_mat;         // [8 Dn_aux][n] T_t(S_d) - c, class-sorted domains x isometries
    __half *A1_mat;        // [R_pad][16] (alpha, 0, ...): correction slice of the A operand (B = 8)
    __half *B1_mat;        // [8 Dn_aux][16] (-gamma / 64, 0, ...): correction slice of B (B = 8)
    float4 *dom_aux;       // [Dn_aux] per sorted domain: B = 8: (0, Q / 256, 128 / Q, 0);
                           // B = 16: (-gamma / 256, Q / 1024, 512 / Q, 0) (1/Q terms 0 if Q = 0)
    int4 *rng_info;        // [R_pad] per sorted range: A, pool start, pool end (batch-wide
                           // domain positions), range id (-1 for padding rows)
    int rng_off, dom_off, mt_off;  // first batch-wide sorted range, sorted domain, range tile
    // exact re-search queue of this image
    int32_t *fallback;     // [R] class-sorted positions of ranges to re-search exactly
    FallbackBest *fb_best; // [R] their exact best evaluated candidate
    int32_t *counters;     // [8] this image: [0] re-search count
    long long *matches;    // [1] sum of this image's pool sizes x 8
    int R_pad, Dn_pad, Dn_aux, n_mtiles, max_chunks, sort_blocks_dom, sort_blocks_rng;
};

// Tensor-engine arrays shared by every image of a batch: class-sorted ranges and domains of all
// images concatenated, so one persistent kernel launch serves the whole batch.
struct TcBatch {
    int B;                 // range side: 8 or 16
    int tm;                // ranges per range tile: 128 (B = 8) or 256 (B = 16, two MMA row tiles)
    int halves;            // key columns per row: 2 (B = 8: two column halves), 1 (B = 16)
    __half *A_mat, *B_mat, *A1_mat, *B1_mat;
    float4 *dom_aux;
    int4 *rng_info;
    int4 *tile_win;        // [n_mtiles] union (x, y) and intersection (z, w) of row windows
    int32_t *n_chunks;     // [n_mtiles] 512-domain chunks (absolute grid) the union window meets
    int4 *tile_items;      // [n_mtiles] first key slot, items, first chunk, chunks
    int4 *work;            // [max_items] (range tile, first domain, end domain, first chunk),
                           // in schedule order (by domain group)
    int32_t *work_slot;    // [max_items] key slot of each scheduled item
    int32_t *grp;          // [ng_max] per domain group: item count, then schedule cursor
    unsigned long long *cand;  // top-2 keys: range tile m owns [first slot, + items) x tm x halves x 2
                               // entries, ordered (row, item, half, key)
    uint32_t *chunk_max;   // [max_chunks][tm rows][halves][2] best key, runner-up score per chunk
    int32_t *gcounters;    // [8]: [1] work items, [2] device error, [3] chunks, [4] chunks per group,
                           // [5] next work item to hand out (zero before the matcher)
    int32_t *lib_error = nullptr;  // the library's per-device error word (fic_check), or nullptr
    unsigned long long stall_ns = 0;  // testing hook (fic_debug_stall_matcher): > 0 makes every
                                      // matcher CTA wait this long on a barrier nothing completes
    int R_pad, Dn_aux, n_mtiles, max_items, max_chunks, ng_max, cpi_cap;
    int stages = 0;        // matcher B-operand ring stages (0: the kernel's default)
};

// Marks the code of range r invalid (dom = iso = -1, s = o = sse = NaN): written when the matching
// kernel gave up, so that stale or uninitialised codes are never mistaken for results.
__device__ __forceinline__ void poison_code(const fic_codes &out, int r) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    out.dom[r] = -1;
    out.iso[r] = -1;
    out.s[r] = nan;
    out.o[r] = nan;
    out.sse[r] = nan;
}

// 16x16 blocks: FD = (log2 N_2 - log2 N_8) / 2 with 64 <= N_2 <= 512 and 4 <= N_8 <= 8 (box counts
// at s = 2 and s = 8); the literal window sorts blocks by the rank of their FD among these pairs
constexpr int kFdN2Lo16 = 64, kFdN2Hi16 = 512, kFdN8Lo16 = 4, kFdN8Hi16 = 8;
constexpr int kFdPairs16 = (kFdN2Hi16 - kFdN2Lo16 + 1) * (kFdN8Hi16 - kFdN8Lo16 + 1);  // 2245
constexpr int kSortChunk = 1024;  // elements per counting-sort block (4 per histogram thread)
// ints of a counting sort's block histograms for n keys: 256 classes x the block count rounded up
// to a multiple of 4
inline size_t sort_counts_ints(int n) { return (size_t)(((n + kSortChunk - 1) / kSortChunk + 3) & ~3) * 256; }
constexpr int kTileM = 128;       // rows of one MMA (ranges per B = 8 range tile)
constexpr int kTileDom = 32;      // domains per accumulator tile (8 isometries -> N = 256)
constexpr int kChunkTiles = 16;   // accumulator tiles per chunk (the re-search granule)
constexpr int kChunkDom = kTileDom * kChunkTiles;
// default work items per SM the work list aims for: smaller items shorten the tail of the
// persistent CTAs until per-item costs (A tile loads, key slots) dominate; the work list also cuts
// the last two domain groups in four, so the items taken last are short whatever this is. Matcher
// on GB300, 1024x1024 stride 4: 8 -> 0.884 ms, 16 -> 0.881, 24 -> 0.881, 32 -> 0.887, 48 -> 0.901,
// 64 -> 0.909 (4096x4096 within 0.2% from 8 to 64)
constexpr int kItemsPerSm = 24;
// the same for 16x16 ranges (256-range tiles, 16-chunk groups), 4096x4096 stride 8: 8 -> 46.05 ms,
// 16 -> 46.02, 24 -> 46.02, 32 -> 46.04, 48 -> 46.07, 64 -> 46.07; at 2048x2048 stride 4, 16 items
// per SM made the groups large enough that their B rows were re-read from DRAM (3.45 GB a launch
// against 1.15 GB at 48-64)
constexpr int kItemsPerSm16 = 48;
constexpr int kMaxItemTarget = 64 * 256;  // items_per_sm <= 64, SMs <= 256
// The persistent matchers take work items in list order from a global counter (gcounters[5]): the
// producer thread of a CTA fetches one and hands it to the MMA and epilogue warps through a ring
// of this many shared-memory slots, so a CTA that finishes early takes the next item.
constexpr int kItemRing = 4;

// Ranges per range tile of the tensor engine and box-count scales of a B x B block.
__host__ __device__ constexpr int tile_rows(int B) { return B == 16 ? 2 * kTileM : kTileM; }
__host__ __device__ constexpr int n_scales(int B) { return B == 16 ? 3 : 2; }

// Carves the workspace for n images: per-image buffers, then the batch-wide arrays. Returns the
// bytes needed (with base == nullptr, only the size).
size_t encode_workspace(const Geo *g, int n, EncodeBufs *b, TcBatch *tb, void *ws, size_t cap, bool *ok);

// Launchers (each returns cudaGetLastError()).
cudaError_t launch_classify(const uint8_t *img, const Geo &g, const EncodeBufs &b,
                            cudaStream_t st);
cudaError_t launch_pools(const Geo &g, const EncodeBufs &b, cudaStream_t st);
int sort_buckets(const Geo &g);  // buckets of the pool sort: K, or distinct FD values
// class-mode pools split for concurrent streams (see pools.cu); sort scratch sized by
// sort_scratch_ints
cudaError_t launch_pools_domains(const Geo &g, const EncodeBufs &b, cudaStream_t st);
cudaError_t launch_pools_ranges_sort(const Geo &g, const EncodeBufs &b, cudaStream_t st);
cudaError_t launch_pools_windows(const Geo &g, const EncodeBufs &b, cudaStream_t st);
cudaError_t launch_match_simt(const uint8_t *img, const Geo &g, const EncodeBufs &b,
                              const fic_codes &out, cudaStream_t st);
cudaError_t launch_rescan(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                          const fic_codes &out, int num_sms, cudaStream_t st);
// operand packing: part 0 both, 1 ranges only, 2 domains only
cudaError_t launch_pack(const uint8_t *img, const Geo &g, const EncodeBufs &b, cudaStream_t st, int part = 0);
// range packing, pool windows, match count and tile windows of one image in one launch (8x8
// ranges, class mode)
cudaError_t launch_pack_ranges_tiles(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                                     cudaStream_t st);
// tiles_done: the tile windows are already formed (launch_pack_ranges_tiles)
cudaError_t launch_work_list(const TcBatch &tb, int target_items, cudaStream_t st, bool tiles_done = false);
cudaError_t launch_match_tc(const TcBatch &tb, int num_sms, cudaStream_t st);
cudaError_t launch_reeval(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                          const fic_codes &out, cudaStream_t st);
// B = 16 tensor engine (match_tc16.cu)
cudaError_t launch_pack16(const uint8_t *img, const Geo &g, const EncodeBufs &b, cudaStream_t st, int part = 0);
cudaError_t launch_match_tc16(const TcBatch &tb, int num_sms, cudaStream_t st);
cudaError_t launch_reeval16(const uint8_t *img, const Geo &g, const EncodeBufs &b, const TcBatch &tb,
                            const fic_codes &out, cudaStream_t st);
cudaError_t launch_info(const EncodeBufs *b, int n, const TcBatch &tb, fic_encode_info *info, cudaStream_t st);

// decode
cudaError_t launch_decode_step(const fic_codes &c, const Geo &g, const float *x, float *y,
                               cudaStream_t st);
// x_iters of the Jacobi iteration from x0 (NULL: 128 everywhere) into out, iters >= 1; tmp holds
// H * W floats of scratch. Even strides iterate on the plane of 2x2 averages and write x only at
// the last step; odd strides take full-resolution steps.
cudaError_t launch_decode_iterate(const fic_codes &c, const Geo &g, int iters, const float *x0, float *out,
                                  float *tmp, cudaStream_t st);
cudaError_t launch_fill(float *x, size_t n, float v, cudaStream_t st);
// Domain -> ranges index of the adjoint (decode.cu): key[R], list[R] (range ids sorted by domain),
// t1[R], t2[R] sort buffers, off[Dn + 1] segment starts, digit[R] bytes, counts (radix
// histograms), acc[R * B * B] per-domain accumulated cells (at each domain's segment start).
struct AdjointCsr {
    int32_t *key, *list, *t1, *t2, *off, *counts;
    uint8_t *digit;
    int4 *ent;   // [R] per list position: (range id, isometry, s / 4 as float bits, 0)
    float *acc;
};
// The adjoint of `iters` decoding steps for an even stride, on the plane of 2x2 averages:
// checkpoints every ck steps (ckpt: nseg planes, seg: ck planes, nu: 2 planes, pk: R records;
// planes are H * W / 4 floats), the gradient terms accumulated into gs, go (float-float per range).
// The domain -> ranges index `a` must be built first.
cudaError_t launch_backward_plane(const fic_codes &c, const Geo &g, const AdjointCsr &a, int iters, int ck,
                                  const float *x0, const float *grad_out, float *ckpt, float *seg, float *nu,
                                  int4 *pk, float2 *gs, float2 *go, cudaStream_t st);
bool decode_on_plane(const Geo &g);
// Stable sort of 0 .. n-1 by key (pools.cu); scratch sizes: see launch_radix_sort.
size_t radix_counts_ints(int n);
cudaError_t launch_radix_sort(const int32_t *key, int n, uint32_t key_max, int32_t *perm, int32_t *t1, int32_t *t2,
                              uint8_t *digit, int32_t *counts, cudaStream_t st);
// Validates the geometry and parameters of one image and derives its grids (the checks every entry
// point applies); sets the thread's error message on failure.
fic_status make_geometry(const fic_geom *gm, const fic_params *p, Geo *g);
// Sets the message fic_last_error() returns on this thread.
void set_error(const char *msg);
// The calling thread's current CUDA context (a CUcontext, nullptr if none); false if the driver
// cannot be asked.
bool current_context(void **ctx);

}  // namespace fic
