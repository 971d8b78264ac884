// Dynamic domain pools (Revathy & Jayamohan, Section 3.1 Eq. 3; Section 3.2).
//
// The paper stores the domain FDs in a height-balanced (AVL) tree and answers each range's
// query d_r - D_f <= d_d <= d_r + D_f by a tree search. The in-order traversal of such a tree
// is the sorted sequence of its keys, and a range query returns a contiguous run of it. Here
// the "tree" is that sorted sequence itself: a stable counting sort of the domains by LFD class
// (`dom_order`, `bin_off`), built in O(Dn), and each range's pool is the contiguous slice of the
// classes within w of its own. Ranges are sorted the same way so that ranges sharing a pool are
// adjacent (the tensor engine tiles them together).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "fic_internal.cuh"

namespace fic {

// Per-block class histograms of kSortChunk keys each, stored class-major: counts[k * nb4 + blk],
// nb4 = the block count rounded up to a multiple of 4 (pad entries zero), so that one class's
// counts over all blocks are contiguous 16-byte vectors for the scatter.
__global__ void __launch_bounds__(256) k_sort_hist(const uint8_t *__restrict__ keys, int n, int nb4, bool words,
                                                   int32_t *__restrict__ counts) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int base = blockIdx.x * kSortChunk;
    const int i0 = base + 4 * threadIdx.x;  // four keys per thread: kSortChunk = 4 x 256
    if (words && i0 + 3 < n) {  // words: keys is 4-byte aligned, so keys + i0 is
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(keys + i0));
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(&h[(w >> (8 * k)) & 0xFFu], 1);
    } else {
        for (int i = i0; i < n && i < i0 + 4; ++i) atomicAdd(&h[keys[i]], 1);
    }
    __syncthreads();
    counts[(size_t)threadIdx.x * nb4 + blockIdx.x] = h[threadIdx.x];
    if (blockIdx.x == gridDim.x - 1)
        for (int b = gridDim.x; b < nb4; ++b) counts[(size_t)threadIdx.x * nb4 + b] = 0;
}

// Stable scatter: block b places its kSortChunk keys, in index order, after the elements of the
// same class from blocks < b. Threads 0..255 first form the bases from every block's histogram:
// thread k sums class k over the blocks before b and over all blocks, an exclusive scan of the
// totals gives the class starts (block 0 also stores them as bin_off[0 .. K], bin_off[K] = n).
// One thread per key: its rank among equal keys is (earlier warps' counts of the key) + (earlier
// lanes with the same key).
__global__ void __launch_bounds__(kSortChunk) k_sort_scatter(const uint8_t *__restrict__ keys, int n, int nb4,
                                                             int K, const int32_t *__restrict__ counts,
                                                             int32_t *__restrict__ order,
                                                             int32_t *__restrict__ bin_off) {
    constexpr int NW = kSortChunk / 32;
    __shared__ int run[256];
    __shared__ int wtot[8];
    __shared__ int wc[NW][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int j = tid; j < NW * 256; j += kSortChunk) (&wc[0][0])[j] = 0;
    int tot = 0, incl = 0, before = 0;
    if (tid < 256) {
        const int4 *col = reinterpret_cast<const int4 *>(counts + (size_t)tid * nb4);
        const int b0 = blockIdx.x;
#pragma unroll 8
        for (int q = 0; q < nb4 / 4; ++q) {
            const int4 v = __ldg(col + q);
            const int bb = 4 * q;
            tot += (v.x + v.y) + (v.z + v.w);
            before += (bb < b0 ? v.x : 0) + (bb + 1 < b0 ? v.y : 0) + (bb + 2 < b0 ? v.z : 0) + (bb + 3 < b0 ? v.w : 0);
        }
        // exclusive scan of the class totals over the 256 classes (warps 0..7)
        incl = tot;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) wtot[warp] = incl;
    }
    const int i = blockIdx.x * kSortChunk + tid;
    const bool valid = i < n;
    const int key = valid ? (int)keys[i] : 256 + lane;  // invalid lanes never match others
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    __syncthreads();  // wc zeroed, wtot written
    if (valid && rank == 0) wc[warp][key] = __popc(peers);
    if (tid < 256) {
        int wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += wtot[w];
        const int start = wbase + incl - tot;
        run[tid] = start + before;
        if (blockIdx.x == 0) {
            if (tid < K) bin_off[tid] = start;
            if (tid == 0) bin_off[K] = n;
        }
    }
    __syncthreads();
    if (valid) {
        int pos = run[key] + rank;
        for (int w = 0; w < warp; ++w) pos += wc[w][key];
        order[pos] = i;
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

// ---- literal window (Eq. 3 on FD values) ----------------------------------------------------
// An 8x8 block's FD is L[N_2] - L[N_4] with 16 <= N_2 <= 64, 4 <= N_4 <= 8, so at most 245
// distinct values exist. They are sorted once on the host (computed with the same correctly
// rounded log2 table and one binary64 subtraction as the kernels), giving each (N_2, N_4) pair
// the rank of its value; domains and ranges are counting-sorted by that rank.
struct FdRanks {
    double vals[256];       // distinct FD values, ascending
    int n;
    uint8_t rank[65][9];    // rank[N_2][N_4]
};

static const FdRanks &fd_ranks() {
    static FdRanks t;
    static std::once_flag once;
    std::call_once(once, [] {
        const Log2Tab &L = log2_table();
        std::vector<double> v;
        for (int n2 = 16; n2 <= 64; ++n2)
            for (int n4 = 4; n4 <= 8; ++n4) v.push_back(L.v[n2] - L.v[n4]);
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        t.n = (int)v.size();
        for (int i = 0; i < 256; ++i) t.vals[i] = i < t.n ? v[i] : 0.0;
        memset(t.rank, 0, sizeof(t.rank));
        for (int n2 = 16; n2 <= 64; ++n2)
            for (int n4 = 4; n4 <= 8; ++n4)
                t.rank[n2][n4] = (uint8_t)(std::lower_bound(v.begin(), v.end(), L.v[n2] - L.v[n4]) - v.begin());
    });
    return t;
}

struct RankTab {
    uint8_t rank[65][9];
};

__global__ void k_fd_keys(int n, const int32_t *__restrict__ counts, RankTab t, uint8_t *__restrict__ key) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) key[i] = t.rank[counts[2 * i]][counts[2 * i + 1]];
}

struct ValTab {
    double vals[256];
};

// Pool window of every range: the domains (FD-rank-sorted) whose FD lies in
// [FD_r - D_f, FD_r + D_f], D_f = (F_m - F_l) / 3; all domains when that set is empty.
__global__ void k_windows_literal(Geo g, const double *__restrict__ rfd, const double *__restrict__ fd_extent,
                                  ValTab t, int nvals, const int32_t *__restrict__ off,
                                  int32_t *__restrict__ win_lo, int32_t *__restrict__ win_hi, long long *matches) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    long long m = 0;
    if (r < g.R) {
        const double Df = __ddiv_rn(__dsub_rn(fd_extent[1], fd_extent[0]), 3.0);
        const double lo_v = __dsub_rn(rfd[r], Df), hi_v = __dadd_rn(rfd[r], Df);
        int a = 0, b = nvals;  // first rank with value >= lo_v
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (t.vals[mid] >= lo_v) b = mid; else a = mid + 1;
        }
        const int rlo = a;
        a = 0;
        b = nvals;  // first rank with value > hi_v
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (t.vals[mid] > hi_v) b = mid; else a = mid + 1;
        }
        int lo = off[rlo], hi = off[a];
        if (lo >= hi) {
            lo = 0;
            hi = g.Dn;
        }
        win_lo[r] = lo;
        win_hi[r] = hi;
        m = (long long)(hi - lo) * 8;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd((unsigned long long *)matches, (unsigned long long)m);
}

// ---- literal window with 16x16 blocks ------------------------------------------------------
// A 16x16 block's FD is (L[N_2] - L[N_8]) / 2 (two binary64 operations, as in classification) with
// 64 <= N_2 <= 512 and 4 <= N_8 <= 8: 2245 pairs. The key of a pair is the number of pairs whose FD
// is smaller, so keys order blocks by FD and blocks of equal FD share a key; the keys are formed on
// the device from the same correctly rounded log2 table, one thread per pair.
__global__ void __launch_bounds__(256) k_fd_rank16(Log2Tab L, int32_t *__restrict__ rank) {
    __shared__ double v[kFdPairs16];
    for (int i = threadIdx.x; i < kFdPairs16; i += blockDim.x) {
        const int n2 = kFdN2Lo16 + i / (kFdN8Hi16 - kFdN8Lo16 + 1), n8 = kFdN8Lo16 + i % (kFdN8Hi16 - kFdN8Lo16 + 1);
        v[i] = __dmul_rn(__dsub_rn(L.v[n2], L.v[n8]), 0.5);
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kFdPairs16) return;
    const double x = v[i];
    int c = 0;
    for (int j = 0; j < kFdPairs16; ++j) c += v[j] < x;
    rank[i] = c;
}

// key[i] = the FD key of block i from its box counts (N_2, N_4, N_8 per block).
__global__ void k_fd_keys16(int n, const int32_t *__restrict__ counts, const int32_t *__restrict__ rank,
                            int32_t *__restrict__ key) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // box counts of 16x16 blocks lie in these ranges; caller-supplied statistics are clamped into
    // them so that no key is read outside the table
    const int n2 = min(max(counts[3 * i], kFdN2Lo16), kFdN2Hi16);
    const int n8 = min(max(counts[3 * i + 2], kFdN8Lo16), kFdN8Hi16);
    key[i] = rank[(n2 - kFdN2Lo16) * (kFdN8Hi16 - kFdN8Lo16 + 1) + (n8 - kFdN8Lo16)];
}

// off[k] = the first sorted position whose key is >= k, for k = 0 .. nk (binary search over the
// keys of the sorted order).
__global__ void k_key_offsets(int n, int nk, const int32_t *__restrict__ key, const int32_t *__restrict__ order,
                              int32_t *__restrict__ off) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nk) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key[order[mid]] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    off[k] = lo;
}

// sfd[j] = FD of the j-th domain in FD order.
__global__ void k_sorted_fd(int n, const double *__restrict__ fd, const int32_t *__restrict__ order,
                            double *__restrict__ sfd) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) sfd[j] = fd[order[j]];
}

// Pool window of every range, Eq. 3 on the FD values: the FD-sorted domains with
// FD_r - D_f <= FD_d <= FD_r + D_f (binary searches over their sorted FDs), every domain when
// none; these are whole runs of equal FD, so whole key buckets.
__global__ void k_windows_literal16(Geo g, const double *__restrict__ rfd, const double *__restrict__ fd_extent,
                                    const double *__restrict__ sfd, int32_t *__restrict__ win_lo,
                                    int32_t *__restrict__ win_hi, long long *matches) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    long long m = 0;
    if (r < g.R) {
        const double Df = __ddiv_rn(__dsub_rn(fd_extent[1], fd_extent[0]), 3.0);
        const double lo_v = __dsub_rn(rfd[r], Df), hi_v = __dadd_rn(rfd[r], Df);
        int a = 0, b = g.Dn;  // first position with FD >= lo_v
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (sfd[mid] >= lo_v) b = mid; else a = mid + 1;
        }
        int lo = a;
        a = lo;
        b = g.Dn;  // first position with FD > hi_v
        while (a < b) {
            const int mid = (a + b) >> 1;
            if (sfd[mid] > hi_v) b = mid; else a = mid + 1;
        }
        int hi = a;
        if (lo >= hi) {
            lo = 0;
            hi = g.Dn;
        }
        win_lo[r] = lo;
        win_hi[r] = hi;
        m = (long long)(hi - lo) * 8;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd((unsigned long long *)matches, (unsigned long long)m);
}

// Domains and ranges of a 16x16 encode in FD order (stable: equal FDs keep ascending ids), their
// key buckets' offsets and every range's literal window.
static cudaError_t launch_pools_literal16(const Geo &g, const EncodeBufs &b, cudaStream_t st) {
    cudaError_t e;
    k_fd_rank16<<<(kFdPairs16 + 255) / 256, 256, 0, st>>>(log2_table(), b.lit_rank);
    ++g_launches;
    struct Side {
        int n;
        const int32_t *counts;
        int32_t *order, *off;
    } sides[2] = {{g.Dn, b.dom_counts, b.dom_order, b.bin_off}, {g.R, b.range_counts, b.range_order, b.rbin_off}};
    for (const Side &sd : sides) {
        k_fd_keys16<<<(sd.n + 255) / 256, 256, 0, st>>>(sd.n, sd.counts, b.lit_rank, b.lit_key);
        ++g_launches;
        if ((e = launch_radix_sort(b.lit_key, sd.n, (uint32_t)(kFdPairs16 - 1), sd.order, b.lit_t1, b.lit_t2,
                                   b.lit_digit, b.lit_counts, st)))
            return e;
        k_key_offsets<<<(kFdPairs16 + 1 + 255) / 256, 256, 0, st>>>(sd.n, kFdPairs16, b.lit_key, sd.order, sd.off);
        ++g_launches;
        if (sd.order == b.dom_order) {
            k_sorted_fd<<<(g.Dn + 255) / 256, 256, 0, st>>>(g.Dn, b.dom_fd, b.dom_order, b.lit_sfd);
            ++g_launches;
        }
    }
    k_windows_literal16<<<(g.R + 255) / 256, 256, 0, st>>>(g, b.range_fd, b.fd_extent, b.lit_sfd, b.win_lo, b.win_hi,
                                                           b.matches);
    ++g_launches;
    return cudaGetLastError();
}

static cudaError_t counting_sort(const uint8_t *keys, int n, int K, int32_t *counts, int32_t *order,
                                 int32_t *bin_off, cudaStream_t st) {
    const int nblk = (n + kSortChunk - 1) / kSortChunk;
    const int nb4 = (nblk + 3) & ~3;
    // the scatter reads each class's histogram row as 16-byte vectors
    if ((uintptr_t)counts % 16 != 0) return cudaErrorMisalignedAddress;
    const bool words = (uintptr_t)keys % 4 == 0;
    k_sort_hist<<<nblk, 256, 0, st>>>(keys, n, nb4, words, counts);
    ++g_launches;
    k_sort_scatter<<<nblk, kSortChunk, 0, st>>>(keys, n, nb4, K, counts, order, bin_off);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_pools(const Geo &g, const EncodeBufs &b, cudaStream_t st) {
    cudaError_t e;
    if (g.literal && g.B == 16) return launch_pools_literal16(g, b, st);
    if (g.literal) {
        const FdRanks &fr = fd_ranks();
        RankTab rt;
        memcpy(rt.rank, fr.rank, sizeof(rt.rank));
        ValTab vt;
        memcpy(vt.vals, fr.vals, sizeof(vt.vals));
        k_fd_keys<<<(g.Dn + 255) / 256, 256, 0, st>>>(g.Dn, b.dom_counts, rt, b.dom_key);
        ++g_launches;
        k_fd_keys<<<(g.R + 255) / 256, 256, 0, st>>>(g.R, b.range_counts, rt, b.range_key);
        ++g_launches;
        if ((e = counting_sort(b.dom_key, g.Dn, fr.n, b.sort_counts, b.dom_order, b.bin_off, st))) return e;
        if ((e = counting_sort(b.range_key, g.R, fr.n, b.sort_offs, b.range_order, b.rbin_off, st))) return e;
        k_windows_literal<<<(g.R + 255) / 256, 256, 0, st>>>(g, b.range_fd, b.fd_extent, vt, fr.n, b.bin_off,
                                                             b.win_lo, b.win_hi, b.matches);
        ++g_launches;
        return cudaGetLastError();
    }
    if ((e = counting_sort(b.dom_bin, g.Dn, g.K, b.sort_counts, b.dom_order, b.bin_off, st))) return e;
    if ((e = counting_sort(b.range_bin, g.R, g.K, b.sort_offs, b.range_order, b.rbin_off, st))) return e;
    k_windows<<<(g.R + 255) / 256, 256, 0, st>>>(g, b.range_bin, b.bin_off, b.win_lo, b.win_hi,
                                                 b.matches);
    ++g_launches;
    return cudaGetLastError();
}

// The class-mode pools in two halves that can run on different streams: the domain sort
// (dom_order, bin_off), and the range sort plus the windows (which also need bin_off: the caller
// orders the second half after the first's domain sort). The two halves use separate sort
// scratch (sort_counts for domains, sort_offs for ranges).
cudaError_t launch_pools_domains(const Geo &g, const EncodeBufs &b, cudaStream_t st) {
    return counting_sort(b.dom_bin, g.Dn, g.K, b.sort_counts, b.dom_order, b.bin_off, st);
}

cudaError_t launch_pools_ranges_sort(const Geo &g, const EncodeBufs &b, cudaStream_t st) {
    return counting_sort(b.range_bin, g.R, g.K, b.sort_offs, b.range_order, b.rbin_off, st);
}

cudaError_t launch_pools_windows(const Geo &g, const EncodeBufs &b, cudaStream_t st) {
    k_windows<<<(g.R + 255) / 256, 256, 0, st>>>(g, b.range_bin, b.bin_off, b.win_lo, b.win_hi, b.matches);
    ++g_launches;
    return cudaGetLastError();
}

int sort_buckets(const Geo &g) { return g.literal ? (g.B == 16 ? kFdPairs16 : fd_ranks().n) : g.K; }

// ---- stable LSD radix sort of int keys, one byte per counting-sort pass ----------------------
// digit[i] = byte `shift / 8` of key[perm[i]] (of key[i] when perm is null).
__global__ void k_radix_digit(const int32_t *__restrict__ key, const int32_t *__restrict__ perm, int n, int shift,
                              uint8_t *__restrict__ digit) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) digit[i] = (uint8_t)((uint32_t)key[perm ? perm[i] : i] >> shift);
}

// out[j] = perm[order[j]]: the pass's stable order of positions, as indices into the keys.
__global__ void k_radix_compose(const int32_t *__restrict__ perm, const int32_t *__restrict__ order, int n,
                                int32_t *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = perm[order[j]];
}

size_t radix_counts_ints(int n) { return sort_counts_ints(n) + 257; }

// perm = the indices 0 .. n-1 ordered stably by key (0 <= key <= key_max): one counting-sort pass
// per byte of key_max, least significant first; each pass sorts stably by its byte the order the
// previous passes produced. Scratch: digit[n] bytes, t1[n], t2[n] ints, counts[radix_counts_ints(n)].
cudaError_t launch_radix_sort(const int32_t *key, int n, uint32_t key_max, int32_t *perm, int32_t *t1, int32_t *t2,
                              uint8_t *digit, int32_t *counts, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int passes = 1;
    while (passes < 4 && (key_max >> (8 * passes)) != 0) ++passes;
    int32_t *bin_off = counts + sort_counts_ints(n);  // the scatter's class offsets, not used here
    const unsigned g = (unsigned)((n + 255) / 256);
    // buffers: perm, t1, t2. The first pass's order is the current order; every later pass sorts
    // into one free buffer and composes into the other, which becomes current (perm on the last
    // pass when it is free, so that no copy is needed)
    int32_t *buf[3] = {perm, t1, t2};
    int cur = -1;
    for (int pass = 0; pass < passes; ++pass) {
        k_radix_digit<<<g, 256, 0, st>>>(key, cur < 0 ? nullptr : buf[cur], n, 8 * pass, digit);
        ++g_launches;
        if (cur < 0) {
            cur = passes == 1 ? 0 : 1;
            cudaError_t e = counting_sort(digit, n, 256, counts, buf[cur], bin_off, st);
            if (e) return e;
            continue;
        }
        const int nxt = (pass == passes - 1 && cur != 0) ? 0 : (cur == 1 ? 2 : 1);
        const int ord = 3 - cur - nxt;
        cudaError_t e = counting_sort(digit, n, 256, counts, buf[ord], bin_off, st);
        if (e) return e;
        k_radix_compose<<<g, 256, 0, st>>>(buf[cur], buf[ord], n, buf[nxt]);
        ++g_launches;
        cur = nxt;
    }
    if (cur != 0) return cudaMemcpyAsync(perm, buf[cur], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

}  // namespace fic
