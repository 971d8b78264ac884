// Tensor-core engine for classified range-domain matching (sm_103a: TMA, tcgen05, TMEM).
//
// The paper (Sections 1-3) compares every range with every domain of its dynamic pool; the
// comparison is a least-squares fit whose only range x domain term is the correlation
// X = sum_p r[p] * T_t(S_d)[p]. Here that term is one dense contraction per tile:
//
//   A_mat[i][p]          = 64 * r_i[p]             (class-sorted range i, fp16, exact <= 16320)
//   B_mat[8 j + t][p]    = T_t(S_{d_j})[p]         (class-sorted domain j, isometry t, fp16,
//                                                   exact <= 1020)
//   D[i][8 j + t]        = sum_p A_mat[i][p] * B_mat[8 j + t][p] = 64 X
//
// 64 X < 2^30 is a multiple of 64 and every partial sum is a non-negative integer multiple of
// 64 below 2^30, so FP32 accumulation is exact. The fused epilogue turns each row's 8 isometry
// columns of domain j into an FP32 estimate of the best least-squares gain (Section 1's intensity
// map with |s| <= 1) and keeps the two best (gain, j) keys per range; `k_reeval` evaluates those
// exactly in integers and certifies that no other domain can be better (else the range is
// re-searched exactly on CUDA cores).
//
// Kernel shape: persistent, one CTA per SM, 10 warps: warp 0 issues TMA loads (A tile 128 x 64,
// B tiles 256 x 64, 128-byte swizzle, 4-stage ring), warp 1 owns TMEM (two 128 x 256 FP32
// accumulators) and issues tcgen05.mma (M = 128, N = 256, K = 16, four per tile), warps 2-9
// (one thread per TMEM lane = range row, two warps per row group, one per column half) drain the
// accumulators with tcgen05.ld. Every wait is
// bounded by a wall-clock limit; a timeout sets an error word, lets in-flight copies and MMAs
// finish (bounded), frees TMEM and returns.
#include <cuda.h>

#include <climits>
#include <cstring>
#include <mutex>

#include "fic_internal.cuh"

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

constexpr int kStages = 4;
constexpr int kTileN = 8 * kTileDom;     // 256 accumulator columns
constexpr int kABytes = kTileM * 128;    // 128 rows x 64 fp16
constexpr int kBBytes = kTileN * 128;    // 256 rows x 64 fp16
constexpr int kEpiWarps = 8;             // two per TMEM lane group, one per column half
constexpr int kTcThreads = 32 * (2 + kEpiWarps);
constexpr int kChunkDom = kTileDom * kChunkTiles;
constexpr int kTmemCols = 2 * kTileN;    // two accumulators
constexpr unsigned long long kTimeoutNs = 2000000000ull;  // 2 s per wait
// instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = F16 (0), both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);

struct TcShared {
    uint8_t A[2][kABytes];
    uint8_t B[kStages][kBBytes];
    float4 aux[2][kChunkDom];  // per-domain constants of the current and next work item
    unsigned long long full_a[2], empty_a[2], full_b[kStages], empty_b[kStages], tfull[2],
        tempty[2], aux_ready[2], drain;
    uint32_t tmem_base;
    int abort_flag;
};
constexpr size_t kTcSmem = sizeof(TcShared) + 1024;

// ---- PTX wrappers ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of parity `parity`; false on timeout or when another role gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity, volatile int *abort_flag) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_test(b, parity)) return true;
        if ((i & 63) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > kTimeoutNs) return false;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, unsigned long long *bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            su32(dst)),
        "l"((unsigned long long)map), "r"(su32(bar)), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, unsigned long long adesc, unsigned long long bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
// K-major operand tile in shared memory, rows of 128 bytes, 128-byte swizzle, 8-row groups
// 1024 bytes apart; bits: start >> 4 [0,14), leading offset >> 4 [16,30) (unused for this
// layout), stride offset >> 4 [32,46), descriptor version 1 [46,48), swizzle mode 2 [61,64).
__device__ __forceinline__ unsigned long long sw128_desc(uint32_t saddr) {
    return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((unsigned long long)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
          "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
          "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
// Waits for this thread's tcgen05.ld results; naming the destination registers as operands keeps
// the compiler from reading them before the wait.
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&v)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
                   "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]),
                   "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]),
                   "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}
__device__ __forceinline__ float fmax3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmin3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ float max8(const uint32_t *v) {
    const float a = fmax3f(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]));
    const float b = fmax3f(__uint_as_float(v[3]), __uint_as_float(v[4]), __uint_as_float(v[5]));
    return fmax3f(a, b, fmaxf(__uint_as_float(v[6]), __uint_as_float(v[7])));
}
__device__ __forceinline__ float min8(const uint32_t *v) {
    const float a = fmin3f(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]));
    const float b = fmin3f(__uint_as_float(v[3]), __uint_as_float(v[4]), __uint_as_float(v[5]));
    return fmin3f(a, b, fminf(__uint_as_float(v[6]), __uint_as_float(v[7])));
}

__device__ __forceinline__ void top2(unsigned long long &b1, unsigned long long &b2, unsigned long long k) {
    const unsigned long long lo = k < b1 ? k : b1;
    b1 = k > b1 ? k : b1;
    b2 = lo > b2 ? lo : b2;
}
__device__ __forceinline__ void top2u(uint32_t &b1, uint32_t &b2, uint32_t k) {
    const uint32_t lo = min(k, b1);
    b1 = max(k, b1);
    b2 = max(b2, lo);
}

// Scores of one column half of an accumulator tile: 16 domains x 8 isometries for this thread's
// range row. Per domain: p = max_t |P_t| from the max and min correlation, the clamped
// least-squares gain / 8 estimate g8 = 2 m^2 / Q + (p - m), m = min(p, Q/4), and a 32-bit key
// (g8's bits with the low 4 replaced by 15 - local index); t1, t2 keep the two largest keys.
// MASK: keys of domains outside this row's pool window [lo_r, hi_r) are 0.
template <bool MASK>
__device__ __forceinline__ void epi_half(uint32_t taddr, const float4 *auxp, float A, int jh, int lo_r,
                                         int hi_r, uint32_t &t1, uint32_t &t2) {
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
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = 4 * c + q;
            const float4 a = auxp[l];
            const float xmax = max8(cur + 8 * q), xmin = min8(cur + 8 * q);
            const float p = fmaxf(fmaf(-A, a.x, xmax), fmaf(A, a.x, -xmin));
            const float mm = fminf(p, a.y);
            const float g8 = fmaf(mm, mm * a.z, p - mm);
            uint32_t key = (__float_as_uint(g8) & 0xFFFFFFF0u) | (uint32_t)(15 - l);
            if (MASK) {
                const int j = jh + l;
                key = (j >= lo_r && j < hi_r) ? key : 0u;
            }
            top2u(t1, t2, key);
        }
        if (c < 3) {
            if (c & 1)
                tmem_ld_wait(va);
            else
                tmem_ld_wait(vb);
        }
    }
}

// Folds a half-tile key (local index in the low 4 bits) into the running 64-bit keys
// (score bits << 32 | ~domain position).
__device__ __forceinline__ void merge_half_key(unsigned long long &b1, unsigned long long &b2, uint32_t t, int jh) {
    const int j = jh + 15 - (int)(t & 15u);
    const unsigned long long k =
        t ? (((unsigned long long)(t & 0xFFFFFFF0u) << 32) | (unsigned long long)(uint32_t)(~j)) : 0ull;
    top2(b1, b2, k);
}

}  // namespace

// ---- operand packing ------------------------------------------------------------------------
// One thread per (sorted range i, pixel row y): A_mat row i = 64 * pixels; rng_info[i] =
// (A, pool start, pool end, range id). Rows i >= R are zero with an empty window.
__global__ void k_pack_ranges(Geo g, const uint8_t *__restrict__ img, const int32_t *__restrict__ range_order,
                              const int32_t *__restrict__ rsum, const int32_t *__restrict__ win_lo,
                              const int32_t *__restrict__ win_hi, int R_pad, __half *__restrict__ A_mat,
                              int4 *__restrict__ rng_info) {
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gid >> 3, y = gid & 7;
    if (i >= R_pad) return;
    uint4 pk = make_uint4(0, 0, 0, 0);
    if (i < g.R) {
        const int r = range_order[i];
        const uint8_t *row = img + (size_t)((r / g.nRx) * 8 + y) * g.pitch + (r % g.nRx) * 8;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __half a = __float2half_rn(64.f * (float)row[2 * h]);
            const __half b = __float2half_rn(64.f * (float)row[2 * h + 1]);
            w[h] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
        }
        pk = make_uint4(w[0], w[1], w[2], w[3]);
        if (y == 0) rng_info[i] = make_int4(rsum[r], win_lo[r], win_hi[r], r);
    } else if (y == 0) {
        rng_info[i] = make_int4(0, 0, 0, -1);
    }
    reinterpret_cast<uint4 *>(A_mat + (size_t)i * 64)[y] = pk;
}

// One thread per (sorted domain j, isometry t, row y): B_mat row 8j+t = T_t(S_{dom_order[j]});
// dom_aux[j] = (C, Q/4, 2/Q or 0, 0). Entries j >= Dn are zero.
__global__ void k_pack_domains(Geo g, const uint16_t *__restrict__ domS, const int32_t *__restrict__ dom_order,
                               const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq, int n_pad,
                               __half *__restrict__ B_mat, float4 *__restrict__ dom_aux) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = (int)(gid >> 6), t = (int)(gid >> 3) & 7, y = (int)gid & 7;
    if (j >= n_pad) return;
    uint4 pk = make_uint4(0, 0, 0, 0);
    if (j < g.Dn) {
        const int d = dom_order[j];
        const uint16_t *S = domS + (size_t)d * 64;
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            int sy, sx;
            iso_src(8, t, y, 2 * h, sy, sx);
            const __half a = __float2half_rn((float)S[sy * 8 + sx]);
            iso_src(8, t, y, 2 * h + 1, sy, sx);
            const __half b = __float2half_rn((float)S[sy * 8 + sx]);
            w[h] = (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
        }
        pk = make_uint4(w[0], w[1], w[2], w[3]);
        if (t == 0 && y == 0) {
            const long long C = dsum[d];
            const long long Q = 64LL * dsumsq[d] - C * C;
            dom_aux[j] = make_float4((float)C, (float)Q * 0.25f, Q > 0 ? 2.0f / (float)Q : 0.f, 0.f);
        }
    } else if (t == 0 && y == 0) {
        dom_aux[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    reinterpret_cast<uint4 *>(B_mat + ((size_t)j * 8 + t) * 64)[y] = pk;
}

// One block (128 threads) per range tile: the union [lo_u, hi_u) of its rows' pool windows and
// the intersection [lo_i, hi_i) over its valid rows; tile_win[m] = (lo_u, hi_u, lo_i, hi_i).
__global__ void k_tile_windows(int R, const int4 *__restrict__ rng_info, int4 *__restrict__ tile_win,
                               int32_t *__restrict__ n_chunks) {
    const int m = blockIdx.x, i = m * kTileM + threadIdx.x;
    const bool valid = i < R;
    const int4 ri = rng_info[i];
    int lo_u = valid ? ri.y : INT_MAX, hi_u = valid ? ri.z : INT_MIN;
    int lo_i = valid ? ri.y : INT_MIN, hi_i = valid ? ri.z : INT_MAX;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lo_u = min(lo_u, __shfl_xor_sync(0xffffffffu, lo_u, off));
        hi_u = max(hi_u, __shfl_xor_sync(0xffffffffu, hi_u, off));
        lo_i = max(lo_i, __shfl_xor_sync(0xffffffffu, lo_i, off));
        hi_i = min(hi_i, __shfl_xor_sync(0xffffffffu, hi_i, off));
    }
    __shared__ int4 w[4];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = make_int4(lo_u, hi_u, lo_i, hi_i);
    __syncthreads();
    if (threadIdx.x == 0) {
        int4 t = w[0];
        for (int k = 1; k < 4; ++k) {
            t.x = min(t.x, w[k].x);
            t.y = max(t.y, w[k].y);
            t.z = max(t.z, w[k].z);
            t.w = min(t.w, w[k].w);
        }
        tile_win[m] = t;
        const int chunk = kTileDom * kChunkTiles;
        n_chunks[m] = t.y > t.x ? (t.y - t.x + chunk - 1) / chunk : 0;
    }
}

// One block: work items (m, j0, j1, chunk) for every tile's chunks, tile-major; the count goes
// to counters[1].
__global__ void k_work_list(int n_mtiles, const int4 *__restrict__ tile_win, const int32_t *__restrict__ n_chunks,
                            int4 *__restrict__ work, int32_t *counters) {
    __shared__ int base_s;
    if (threadIdx.x == 0) base_s = 0;
    __syncthreads();
    const int chunk = kTileDom * kChunkTiles;
    for (int m0 = 0; m0 < n_mtiles; m0 += blockDim.x) {
        const int m = m0 + threadIdx.x;
        const int c = m < n_mtiles ? n_chunks[m] : 0;
        // inclusive scan over the block (Hillis-Steele in shared memory)
        __shared__ int sc[1024];
        sc[threadIdx.x] = c;
        __syncthreads();
        for (int s = 1; s < (int)blockDim.x; s <<= 1) {
            const int a = threadIdx.x >= (unsigned)s ? sc[threadIdx.x - s] : 0;
            __syncthreads();
            sc[threadIdx.x] += a;
            __syncthreads();
        }
        const int start = base_s + sc[threadIdx.x] - c;
        if (m < n_mtiles) {
            const int4 t = tile_win[m];
            for (int k = 0; k < c; ++k) {
                const int j0 = t.x + k * chunk;
                work[start + k] = make_int4(m, j0, min(j0 + chunk, t.y), k);
            }
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base_s += sc[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) counters[1] = base_s;
}

// ---- the matching kernel ----------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1)
    k_match_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int R,
               const int4 *__restrict__ work, const int32_t *__restrict__ counters_in,
               const int4 *__restrict__ tile_win, const int4 *__restrict__ rng_info,
               const float4 *__restrict__ dom_aux, int max_chunks, unsigned long long *__restrict__ cand,
               int32_t *err) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t pad = (1024u - (su32(smem_raw) & 1023u)) & 1023u;
    TcShared &sh = *reinterpret_cast<TcShared *>(smem_raw + pad);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_items = counters_in[1];
    volatile int *abort_flag = &sh.abort_flag;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sh.full_a[s], 1);
            mbar_init(&sh.empty_a[s], 1);
            mbar_init(&sh.tfull[s], 1);
            mbar_init(&sh.tempty[s], kEpiWarps);
            mbar_init(&sh.aux_ready[s], 32 * kEpiWarps);
        }
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&sh.full_b[s], 1);
            mbar_init(&sh.empty_b[s], 1);
        }
        mbar_init(&sh.drain, 1);
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
            uint32_t gt = 0, li = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++li) {
                const int4 w = work[it];
                const int ab = li & 1;
                ok = mbar_wait(&sh.empty_a[ab], ((li >> 1) & 1) ^ 1, abort_flag);
                if (!ok) break;
                mbar_expect_tx(&sh.full_a[ab], kABytes);
                tma_load_2d(sh.A[ab], &tmA, &sh.full_a[ab], 0, w.x * kTileM);
                const int nt = (w.z - w.y + kTileDom - 1) / kTileDom;
                for (int k = 0; k < nt; ++k, ++gt) {
                    const int s = gt % kStages;
                    ok = mbar_wait(&sh.empty_b[s], ((gt / kStages) & 1) ^ 1, abort_flag);
                    if (!ok) break;
                    mbar_expect_tx(&sh.full_b[s], kBBytes);
                    tma_load_2d(sh.B[s], &tmB, &sh.full_b[s], 0, 8 * (w.y + k * kTileDom));
                }
            }
            if (!ok) {
                atomicExch(err, (int)FIC_ERR_DEVICE_TIMEOUT);
                *abort_flag = 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            uint32_t gt = 0, li = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++li) {
                const int4 w = work[it];
                const int ab = li & 1;
                ok = mbar_wait(&sh.full_a[ab], (li >> 1) & 1, abort_flag);
                if (!ok) break;
                tc_fence_after();
                const uint32_t a0 = su32(sh.A[ab]);
                const int nt = (w.z - w.y + kTileDom - 1) / kTileDom;
                for (int k = 0; k < nt; ++k, ++gt) {
                    const int s = gt % kStages, acc = gt & 1;
                    ok = mbar_wait(&sh.tempty[acc], ((gt >> 1) & 1) ^ 1, abort_flag);
                    if (!ok) break;
                    ok = mbar_wait(&sh.full_b[s], (gt / kStages) & 1, abort_flag);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t b0 = su32(sh.B[s]);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        umma_f16(tmem + acc * kTileN, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), kIdesc,
                                 kk > 0 ? 1u : 0u);
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
                atomicExch(err, (int)FIC_ERR_DEVICE_TIMEOUT);
                *abort_flag = 1;
            }
        }
    } else {
        // ---- epilogue: warps 2..9. Warp w reads TMEM lane group (w & 3) (range rows) and column
        // half (w - 2) >> 2 of every accumulator tile (16 domains x 8 isometries).
        const int ew = warp - 2;
        const int lg = warp & 3;
        const int half = ew >> 2;
        const int row = lg * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(half * (kTileN / 2));
        uint32_t gt = 0, li = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++li) {
            const int4 w = work[it];
            const int nt = (w.z - w.y + kTileDom - 1) / kTileDom;
            // per-domain constants of this item into shared memory (double-buffered by item parity;
            // a thread reaches item li + 2 only after every thread has left item li)
            const int ab = li & 1;
            for (int k = ew * 32 + lane; k < nt * kTileDom; k += 32 * kEpiWarps)
                sh.aux[ab][k] = __ldg(&dom_aux[w.y + k]);
            mbar_arrive(&sh.aux_ready[ab]);
            ok = __all_sync(0xffffffffu, mbar_wait(&sh.aux_ready[ab], (li >> 1) & 1, abort_flag));
            if (!ok) break;
            const int i = w.x * kTileM + row;
            const int4 ri = rng_info[i];
            const bool valid = i < R;
            const float A = (float)ri.x;
            const int lo_r = ri.y, hi_r = min(ri.z, w.z);
            const int4 tw = tile_win[w.x];
            const int f_lo = max(tw.z, w.y), f_hi = min(tw.w, w.z);  // columns valid for every row
            unsigned long long b1 = 0, b2 = 0;
            for (int k = 0; k < nt; ++k, ++gt) {
                const int acc = gt & 1;
                ok = __all_sync(0xffffffffu, mbar_wait(&sh.tfull[acc], (gt >> 1) & 1, abort_flag));
                if (!ok) break;
                tc_fence_after();
                const int jh = w.y + k * kTileDom + half * (kTileDom / 2);
                const float4 *auxp = &sh.aux[ab][k * kTileDom + half * (kTileDom / 2)];
                const uint32_t taddr = tbase + acc * kTileN;
                uint32_t t1 = 0, t2 = 0;
                if (jh >= f_lo && jh + kTileDom / 2 <= f_hi)
                    epi_half<false>(taddr, auxp, A, jh, lo_r, hi_r, t1, t2);
                else
                    epi_half<true>(taddr, auxp, A, jh, lo_r, hi_r, t1, t2);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.tempty[acc]);
                merge_half_key(b1, b2, t1, jh);
                merge_half_key(b1, b2, t2, jh);
            }
            if (ok && valid) {
                unsigned long long *dst = cand + (((size_t)i * max_chunks + w.w) * 2 + half) * 2;
                dst[0] = b1;
                dst[1] = b2;
            }
        }
        if (!ok) {
            atomicExch(err, (int)FIC_ERR_DEVICE_TIMEOUT);
            *abort_flag = 1;
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
// One warp per class-sorted range position i. Merges the range's top-2 keys over its tile's
// chunks, evaluates both candidates under all 8 isometries exactly, keeps the best (gain, then
// smaller domain id, then smaller isometry) and certifies it: every other domain's FP32 score is
// at most the runner-up's, and an FP32 score differs from that domain's exact gain / 8 by less
// than a relative 20 * 2^-24 (it is formed from exact integers and 24-bit constants by a handful
// of single-rounding operations), so if runner-up * (1 + 2^-16) < exact best, no other domain
// can win or tie. Otherwise the range is queued with its exact best for k_rescan.
// Otherwise the range goes to the exact re-search list. Flat ranges (n Bs = A^2) have zero error
// for every candidate; their code is the smallest domain id of the pool with t = 0.
__global__ void k_reeval(Geo g, const uint8_t *__restrict__ img, const uint16_t *__restrict__ domS,
                         const int32_t *__restrict__ dsum, const int32_t *__restrict__ dsumsq,
                         const int32_t *__restrict__ rsumsq, const int32_t *__restrict__ dom_order,
                         const int32_t *__restrict__ bin_off, const uint8_t *__restrict__ rbin,
                         const int4 *__restrict__ rng_info, const int4 *__restrict__ tile_win,
                         const unsigned long long *__restrict__ cand, int max_chunks, int32_t *__restrict__ fallback,
                         FallbackBest *__restrict__ fb_best, int32_t *counters, fic_codes out) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= g.R) return;
    if (counters[2] != 0) return;  // the matching kernel gave up: its keys are not trusted
    const int4 ri = rng_info[i];
    const int r = ri.w;
    const long long A = ri.x, Bs = rsumsq[r];
    const int ry = (r / g.nRx) * 8, rx = (r % g.nRx) * 8;

    if (64LL * Bs - A * A == 0) {  // flat range
        int dmin = INT_MAX;
        const int b = rbin[r];
        const int blo = max(0, b - g.w), bhi = min(g.K - 1, b + g.w);
        if (bin_off[blo] == bin_off[bhi + 1]) {
            dmin = 0;  // empty class window: the pool is every domain
        } else {
            for (int bb = blo + lane; bb <= bhi; bb += 32)
                if (bin_off[bb] < bin_off[bb + 1]) dmin = min(dmin, dom_order[bin_off[bb]]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) dmin = min(dmin, __shfl_xor_sync(0xffffffffu, dmin, off));
        }
        if (lane == 0) {
            const long long C = dsum[dmin];
            const long long Q = 64LL * dsumsq[dmin] - C * C;
            // X = (A / 64) C exactly for a constant block, so P = 64 X - A C = 0
            double s, o, sse;
            finalize_code(64, A, Bs, C, 0, Q, exact_gain(0, Q), s, o, sse);
            out.dom[r] = dmin;
            out.iso[r] = 0;
            out.s[r] = s;
            out.o[r] = o;
            out.sse[r] = sse;
        }
        return;
    }

    // merge the top-2 keys of all chunks
    const int m = i / kTileM;
    const int4 tw = tile_win[m];
    const int chunk = kTileDom * kChunkTiles;
    const int nch = tw.y > tw.x ? (tw.y - tw.x + chunk - 1) / chunk : 0;
    unsigned long long b1 = 0, b2 = 0;
    for (int e = lane; e < 4 * nch; e += 32) top2(b1, b2, cand[(size_t)i * max_chunks * 4 + e]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o1 = __shfl_xor_sync(0xffffffffu, b1, off);
        const unsigned long long o2 = __shfl_xor_sync(0xffffffffu, b2, off);
        top2(b1, b2, o1);
        top2(b1, b2, o2);
    }
    // exact evaluation: lane = 8 * candidate + t for lanes 0..15
    const int cidx = lane >> 3, t = lane & 7;
    const unsigned long long key = cidx == 0 ? b1 : b2;
    const bool has = lane < 16 && key != 0 && (int)(~(uint32_t)(key & 0xffffffffu)) < g.Dn;
    Gain gg{-1, 1};
    int d = INT_MAX;
    long long P = 0, Q = 0, C = 0;
    if (has) {
        const int j = (int)(~(uint32_t)(key & 0xffffffffu));
        d = dom_order[j];
        const uint16_t *S = domS + (size_t)d * 64;
        long long X = 0;
        for (int y = 0; y < 8; ++y) {
            const uint8_t *row = img + (size_t)(ry + y) * g.pitch + rx;
            for (int x = 0; x < 8; ++x) {
                int sy, sx;
                iso_src(8, t, y, x, sy, sx);
                X += (long long)row[x] * S[sy * 8 + sx];
            }
        }
        C = dsum[d];
        Q = 64LL * dsumsq[d] - C * C;
        P = 64LL * X - A * C;
        gg = exact_gain(P, Q);
    }
    int bt = t;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Gain og{__shfl_xor_sync(0xffffffffu, gg.num, off), __shfl_xor_sync(0xffffffffu, gg.den, off)};
        const int od = __shfl_xor_sync(0xffffffffu, d, off), ot = __shfl_xor_sync(0xffffffffu, bt, off);
        const long long oP = __shfl_xor_sync(0xffffffffu, P, off), oQ = __shfl_xor_sync(0xffffffffu, Q, off);
        const long long oC = __shfl_xor_sync(0xffffffffu, C, off);
        if (cand_better(og, od, ot, gg, d, bt)) {
            gg = og;
            d = od;
            bt = ot;
            P = oP;
            Q = oQ;
            C = oC;
        }
    }
    if (lane != 0) return;
    bool certified = b1 != 0 && gg.num >= 0;
    if (certified && b2 != 0) {
        const double u2 = (double)__uint_as_float((uint32_t)(b2 >> 32));
        const double g8 = (double)gg.num / (8.0 * (double)gg.den);
        certified = u2 * (1.0 + 1.0 / 65536.0) < g8;
    }
    if (!certified) {
        const int slot = atomicAdd(&counters[0], 1);
        fallback[slot] = i;
        FallbackBest fb;
        fb.num = gg.num;
        fb.den = gg.den;
        fb.P = P;
        fb.Q = Q;
        fb.d = d;
        fb.t = bt;
        fb.C = (int)C;
        fb.pad = 0;
        fb_best[slot] = fb;
        return;
    }
    double s, o, sse;
    finalize_code(64, A, Bs, C, P, Q, gg, s, o, sse);
    out.dom[r] = d;
    out.iso[r] = bt;
    out.s[r] = s;
    out.o[r] = o;
    out.sse[r] = sse;
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

// rows x 64 fp16, row-major (128-byte rows); box = box_rows x 64; 128-byte swizzle.
cudaError_t make_map(CUtensorMap *map, void *base, unsigned long long rows, unsigned box_rows) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {64, rows};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {64, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_pack(const uint8_t *img, const Geo &g, const EncodeBufs &b, cudaStream_t st) {
    {
        const long long n = (long long)b.R_pad * 8;
        k_pack_ranges<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, img, b.range_order, b.range_sum, b.win_lo,
                                                                  b.win_hi, b.R_pad, b.A_mat, b.rng_info);
        ++g_launches;
    }
    {
        const long long n = (long long)b.Dn_aux * 64;
        k_pack_domains<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, b.dom_S, b.dom_order, b.dom_sum,
                                                                   b.dom_sumsq, b.Dn_aux, b.B_mat, b.dom_aux);
        ++g_launches;
    }
    k_tile_windows<<<b.n_mtiles, kTileM, 0, st>>>(g.R, b.rng_info, b.tile_win, b.n_chunks);
    ++g_launches;
    k_work_list<<<1, 1024, 0, st>>>(b.n_mtiles, b.tile_win, b.n_chunks, b.work, b.counters);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_match_tc(const Geo &g, const EncodeBufs &b, int num_sms, cudaStream_t st) {
    CUtensorMap tmA, tmB;
    cudaError_t e;
    if ((e = make_map(&tmA, b.A_mat, (unsigned long long)b.R_pad, kTileM))) return e;
    if ((e = make_map(&tmB, b.B_mat, (unsigned long long)b.Dn_aux * 8, kTileN))) return e;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(k_match_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
    });
    if (attr_err) return attr_err;
    const int grid = num_sms < b.max_items ? num_sms : b.max_items;
    if (grid <= 0) return cudaSuccess;
    k_match_tc<<<grid, kTcThreads, kTcSmem, st>>>(tmA, tmB, g.R, b.work, b.counters, b.tile_win, b.rng_info,
                                                   b.dom_aux, b.max_chunks, b.cand, b.counters + 2);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_reeval(const uint8_t *img, const Geo &g, const EncodeBufs &b, const fic_codes &out,
                          cudaStream_t st) {
    const long long threads = (long long)g.R * 32;
    k_reeval<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        g, img, b.dom_S, b.dom_sum, b.dom_sumsq, b.range_sumsq, b.dom_order, b.bin_off, b.range_bin, b.rng_info,
        b.tile_win, b.cand, b.max_chunks, b.fallback, b.fb_best, b.counters, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
