// Dynamic domain pools (Revathy & Jayamohan, Section 3.1 Eq. 3; Section 3.2).
//
// The paper stores the domain FDs in a height-balanced (AVL) tree and answers each range's
// query d_r - D_f <= d_d <= d_r + D_f by a tree search. The in-order traversal of such a tree
// is the sorted sequence of its keys, and a range query returns a contiguous run of it. Here
// the "tree" is that sorted sequence itself: a stable counting sort of the domains by LFD class
// (`dom_order`, `bin_off`), built in O(Dn), and each range's pool is the contiguous slice of the
// classes within w of its own. Ranges are sorted the same way so that ranges sharing a pool are
// adjacent (the tensor engine tiles them together).
#include "fic_internal.cuh"

namespace fic {

// Per-block class histograms: counts[blk * 256 + k].
__global__ void k_sort_hist(const uint8_t *__restrict__ keys, int n, int32_t *__restrict__ counts) {
    __shared__ int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortChunk;
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x)
        if (base + i < n) atomicAdd(&h[keys[base + i]], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x) counts[blockIdx.x * 256 + k] = h[k];
}

// One block of 256 threads: class totals, class starts (bin_off) and per-block scatter bases.
__global__ void k_sort_scan(const int32_t *__restrict__ counts, int nblk, int K,
                            int32_t *__restrict__ offs, int32_t *__restrict__ bin_off) {
    __shared__ int tot[256];
    const int k = threadIdx.x;
    int t = 0;
    for (int b = 0; b < nblk; ++b) t += counts[b * 256 + k];
    tot[k] = t;
    __syncthreads();
    if (k == 0) {
        int run = 0;
        for (int i = 0; i < 256; ++i) {
            const int c = tot[i];
            tot[i] = run;
            run += c;
        }
        bin_off[K] = run;
    }
    __syncthreads();
    int run = tot[k];
    if (k < K) bin_off[k] = run;
    for (int b = 0; b < nblk; ++b) {
        offs[b * 256 + k] = run;
        run += counts[b * 256 + k];
    }
}

// Stable scatter: block b places its kSortChunk keys, in index order, after the elements of
// the same class from blocks < b. Within a 256-element step, a thread's rank among equal keys
// is (earlier warps' counts) + (earlier lanes with the same key).
__global__ void __launch_bounds__(256) k_sort_scatter(const uint8_t *__restrict__ keys, int n,
                                                      const int32_t *__restrict__ offs,
                                                      int32_t *__restrict__ order) {
    __shared__ int run[256];
    __shared__ int wc[8][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    run[tid] = offs[blockIdx.x * 256 + tid];
    const int base = blockIdx.x * kSortChunk;
    const unsigned lt = (1u << lane) - 1u;
    for (int sub = 0; sub < kSortChunk; sub += 256) {
#pragma unroll
        for (int w = 0; w < 8; ++w) wc[w][tid] = 0;
        __syncthreads();
        const int i = base + sub + tid;
        const bool valid = i < n;
        const int key = valid ? (int)keys[i] : 256 + lane;  // invalid lanes never match others
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wc[warp][key] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = run[key] + rank;
            for (int w = 0; w < warp; ++w) pos += wc[w][key];
            order[pos] = i;
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) add += wc[w][tid];
        run[tid] += add;
        __syncthreads();
    }
}

// Pool window of every range and the algorithmic match count sum_r |Pool(r)| * 8.
__global__ void k_windows(Geo g, const uint8_t *__restrict__ rbin, const int32_t *__restrict__ bin_off,
                          int32_t *__restrict__ win_lo, int32_t *__restrict__ win_hi,
                          long long *matches) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    long long m = 0;
    if (r < g.R) {
        const int b = rbin[r];
        const int blo = max(0, b - g.w), bhi = min(g.K - 1, b + g.w);
        int lo = bin_off[blo], hi = bin_off[bhi + 1];
        if (lo == hi) {  // no domain in the window: search every domain
            lo = 0;
            hi = g.Dn;
        }
        win_lo[r] = lo;
        win_hi[r] = hi;
        m = (long long)(hi - lo) * 8;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd((unsigned long long *)matches, (unsigned long long)m);
}

static cudaError_t counting_sort(const uint8_t *keys, int n, int K, int32_t *counts, int32_t *offs,
                                 int32_t *order, int32_t *bin_off, cudaStream_t st) {
    const int nblk = (n + kSortChunk - 1) / kSortChunk;
    k_sort_hist<<<nblk, 256, 0, st>>>(keys, n, counts);
    ++g_launches;
    k_sort_scan<<<1, 256, 0, st>>>(counts, nblk, K, offs, bin_off);
    ++g_launches;
    k_sort_scatter<<<nblk, 256, 0, st>>>(keys, n, offs, order);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_pools(const Geo &g, const EncodeBufs &b, cudaStream_t st) {
    cudaError_t e;
    if ((e = counting_sort(b.dom_bin, g.Dn, g.K, b.sort_counts, b.sort_offs, b.dom_order,
                           b.bin_off, st)))
        return e;
    if ((e = counting_sort(b.range_bin, g.R, g.K, b.sort_counts, b.sort_offs, b.range_order,
                           b.rbin_off, st)))
        return e;
    if ((e = cudaMemsetAsync(b.matches, 0, sizeof(long long), st))) return e;
    k_windows<<<(g.R + 255) / 256, 256, 0, st>>>(g, b.range_bin, b.bin_off, b.win_lo, b.win_hi,
                                                 b.matches);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
