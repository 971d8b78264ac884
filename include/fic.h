/*
 * fic.h - C ABI of the GB300 classified fractal image encoder.
 *
 * Method: K. Revathy and M. Jayamohan, "Dynamic Domain Classification for Fractal Image
 * Compression". An 8-bit grayscale image is cut into non-overlapping B x B range blocks
 * (Section 1); every 2B x 2B domain on a stride-sigma grid (Section 2) is contracted by 2x2
 * averaging; ranges and domains are classified by their local fractal dimension estimated with
 * differential box counting (Section 3.1); each range searches only the domains whose class is
 * within the fractal distance D_f = (F_m - F_l)/3 of its own (Section 3.1, Eq. 2-3), under the
 * 8 square isometries, with a least-squares contrast s (|s| <= 1) and brightness o, and keeps
 * the (domain, isometry, s, o) of least collage error (Section 1). Decoding iterates the maps
 * from an initial image (Section 1).
 *
 * Conventions for every entry point:
 *  - Image, code, statistics and workspace pointers are DEVICE pointers owned by the caller.
 *    The library allocates no device memory and frees none; it keeps no state between calls
 *    except a per-device cache of its own kernel attributes, the per-thread caches of captured
 *    graphs of fic_encode and fic_decode (see there), eight internal CUDA streams and events per
 *    host thread and device for fic_encode_batched and single encodes (created on the first call
 *    that is not inside a stream capture; the images' per-image stages run on them, joined back
 *    into `stream` by events), and two fixed device arrays with their addresses cached per
 *    device and context: the device error word that fic_check reads and fic_decode_static's
 *    scratch image.
 *  - `stream` is a cudaStream_t (passed as void*; NULL = the legacy default stream). All work
 *    is enqueued asynchronously on it; nothing synchronises the host.
 *  - Decode workspaces must be 256-byte aligned; encode workspaces may have any alignment (the
 *    library uses them from the first 1024-byte boundary; the size queries include that slack).
 *  - Arguments are validated on the host before anything is enqueued; a failed validation
 *    returns FIC_ERR_INVALID_ARG (or FIC_ERR_WORKSPACE) and enqueues nothing.
 *  - A launch failure returns FIC_ERR_CUDA. fic_last_error() returns a message for the last
 *    failure on the calling thread.
 *  - Each entry point marks its host call with an NVTX range named after it (seen by profilers
 *    that record NVTX; nothing is recorded otherwise).
 *  - Images are row-major uint8 with row pitch `pitch` >= W bytes. Ranges are numbered
 *    row-major: range r covers rows (r / (W/B))*B .. +B-1 and columns (r % (W/B))*B .. +B-1.
 *    Domains are numbered row-major over the stride grid: domain d has its top-left pixel at
 *    ((d / nDx) * sigma, (d % nDx) * sigma), nDy = (H - 2B)/sigma + 1, nDx = (W - 2B)/sigma + 1.
 *  - Isometry t maps a B x B block X to T_t X with (T_t X)[y][x] = X[sy][sx] where, with
 *    N = B-1: t=0 (y,x); 1 rotate 90 clockwise (N-x,y); 2 rotate 180 (N-y,N-x);
 *    3 rotate 270 clockwise (x,N-y); 4 mirror left-right (y,N-x); 5 mirror up-down (N-y,x);
 *    6 transpose (x,y); 7 anti-transpose (N-x,N-y).
 *
 * Supported in this version: B = 8 or 16 (16x16 ranges against 32x32 domains: the paper's
 * method at a second range size, with n = 256 pixels per block), 1 <= sigma, 1 <= K <= 255,
 * s_max = 1.0, the class window or the literal FD window (FIC_FLAG_LITERAL_WINDOW) for both.
 */
#ifndef FIC_H
#define FIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FIC_OK = 0,
    FIC_ERR_INVALID_ARG = 1,  /* bad geometry, parameters or null pointer */
    FIC_ERR_WORKSPACE = 2,    /* workspace missing, too small or (decode) not 256-byte aligned */
    FIC_ERR_CUDA = 3,         /* a CUDA runtime/driver call or launch failed */
    FIC_ERR_DEVICE_TIMEOUT = 4, /* a bounded device-side wait gave up (reported by fic_check) */
    FIC_ERR_UNSUPPORTED = 5   /* device or build lacks a required feature (sm_103a) */
} fic_status;

/* Matching engines. */
enum {
    FIC_ENGINE_TENSOR = 0, /* tcgen05 correlation GEMM + fused ranking + exact re-evaluation */
    FIC_ENGINE_SIMT = 1    /* exact search on CUDA cores (the plain GPU search) */
};

/* Pool window (fic_params.flags). Default: the class window |bin_d - bin_r| <= w. With
 * FIC_FLAG_LITERAL_WINDOW the pool is Section 3.1 Eq. 3 on the FD values themselves,
 * Pool(r) = {d : FD_r - D_f <= FD_d <= FD_r + D_f}, D_f = (F_m - F_l) / 3 (Eq. 2), each bound one
 * binary64 operation; domains and ranges are then ordered by FD value instead of class (stable:
 * equal FDs keep ascending ids), and num_classes / half_width only shape the reported classes. */
#define FIC_FLAG_LITERAL_WINDOW 1

typedef struct {
    int32_t H, W;   /* image height and width in pixels: multiples of B, >= 2B */
    int32_t pitch;  /* bytes between rows, >= W */
} fic_geom;

typedef struct {
    int32_t block;         /* B, range side: 8 or 16 */
    int32_t domain_stride; /* sigma >= 1: domain grid step in pixels */
    int32_t num_classes;   /* K in [1, 255]; K = 1 makes every pool the full domain set */
    int32_t half_width;    /* w >= 0 classes on each side; -1 selects floor(K/3) (Eq. 2) */
    double s_max;          /* contrast clamp; must be 1.0 */
    int32_t engine;        /* FIC_ENGINE_TENSOR or FIC_ENGINE_SIMT */
    int32_t flags;         /* 0, or FIC_FLAG_LITERAL_WINDOW */
    int32_t items_per_sm;  /* tensor engine scheduling: work items per SM the range tiles' domain
                              chunks are split into, 1..64; 0 selects 24 (block 8) or 48
                              (block 16) */
    int32_t group_chunks;  /* tensor engine scheduling: at most this many 512-domain chunks form one
                              domain group, the band of domain operand rows the SMs running together
                              stream (kept L2-resident), 1..1024; 0 selects 64 (block 8) or 16
                              (block 16). Smaller groups need a larger workspace (size queries take
                              it into account). */
    int32_t pipeline_stages; /* tensor engine: shared-memory stages of the streamed domain operand,
                                3 or 4 (block 8), 4 or 5 (block 16); 0 selects 3 (block 8) or 4
                                (block 16). Results do not depend on it. */
} fic_params;

/* Per-block statistics (Section 3.1: the fractal dimensions of the range blocks are computed and
 * kept in an array, then those of the overlapping domains). Device
 * arrays, R = (H/B)(W/B) entries for ranges and Dn = nDy*nDx for domains.
 *  range_sum = sum r, range_sumsq = sum r^2 over the B x B pixels;
 *  dom_sum = sum S, dom_sumsq = sum S^2 over the B x B integer 2x2 sums S of the domain;
 *  *_counts[ns*i + k] = differential box count N_s at s = 2^(k+1): ns = 2 scales (s = 2, 4)
 *  for B = 8, ns = 3 (s = 2, 4, 8) for B = 16; box height s*G/B with G = 256 grey levels for
 *  range pixels and G = 1024 for the domains' 2x2 sums;
 *  *_fd = the least-squares slope of log2 N_s against log2(B/s) in binary64 with correctly
 *  rounded log2: log2(N_2) - log2(N_4) for B = 8, (log2(N_2) - log2(N_8)) / 2 for B = 16 (the
 *  middle of three equally spaced abscissae has zero weight);
 *  fd_extent[0] = F_l (least domain FD), fd_extent[1] = F_m (largest domain FD);
 *  *_bin = class in [0, K): min(K-1, max(0, floor(K * ((f - F_l) / (F_m - F_l))))), or 0 if
 *  F_m == F_l, each operation a separate IEEE binary64 operation. */
typedef struct {
    int32_t *range_sum, *range_sumsq, *range_counts;
    double *range_fd;
    uint8_t *range_bin;
    int32_t *dom_sum, *dom_sumsq, *dom_counts;
    double *dom_fd;
    uint8_t *dom_bin;
    double *fd_extent;
} fic_blockstats;

/* Dynamic pools (Section 3.1 Eq. 3 in class units, replacing the paper's AVL tree by an
 * ordered array: a range query of the tree is a contiguous slice of the class-sorted domains).
 *  dom_order[Dn]   domain ids sorted by (class, id) - the in-order traversal of the tree;
 *  bin_off[257]    dom_order[bin_off[b] .. bin_off[b+1]) holds class b (257 entries). With
 *                  FIC_FLAG_LITERAL_WINDOW and B = 8: bucket b holds the b-th smallest distinct FD
 *                  value that 8x8 box counts can produce (up to 245 + 1 entries used); with B = 16
 *                  the array needs FIC_LITERAL16_OFFSETS entries, and bucket k holds the blocks whose
 *                  FD exceeds exactly k of the FDs of the 2245 (N_2, N_8) pairs 16x16 box counts
 *                  can produce (buckets of values no pair has are empty);
 *  range_order[R]  range ids sorted by (class, id); rbin_off[257] likewise;
 *  win_lo[R], win_hi[R]  Pool(r) = dom_order[win_lo[r] .. win_hi[r]) = the domains with
 *                  |bin_d - bin_r| <= w; when that set is empty the pool is every domain
 *                  (win_lo = 0, win_hi = Dn). */
typedef struct {
    int32_t *dom_order, *bin_off, *range_order, *rbin_off, *win_lo, *win_hi;
} fic_pools;

/* Entries of fic_pools.bin_off and rbin_off for the literal window with 16x16 blocks. */
#define FIC_LITERAL16_OFFSETS 2246

/* Fractal code per range r (device arrays of R entries): the best domain id, isometry, contrast
 * s, brightness o (binary64, unquantised) and collage error sse = sum (r - s T_t(D) - o)^2 with
 * D the 2x2-averaged domain. Ties in sse go to the smaller domain id, then the smaller t. */
typedef struct {
    int32_t *dom;
    int32_t *iso;
    double *s, *o, *sse;
} fic_codes;

/* Optional encode report, written to DEVICE memory when the pointer is non-null. */
typedef struct {
    int64_t matches;          /* sum over ranges of |Pool(r)| * 8: range-domain-isometry fits */
    int32_t fallback_ranges;  /* ranges re-searched exactly because ranking could not certify */
    int32_t work_items;       /* tensor engine: (range tile, domain chunk) items */
    int32_t device_error;     /* 0, or FIC_ERR_DEVICE_TIMEOUT if a bounded wait gave up (the
                                 codes are then marked invalid, see fic_encode) */
    int32_t reserved;
} fic_encode_info;

/* Bytes of workspace fic_encode / fic_classify / fic_build_pools need for this geometry. */
size_t fic_encode_workspace_size(const fic_geom *g, const fic_params *p);

/* Section 3.1: moments, differential box counts, FDs, F_l/F_m and classes of every range and
 * domain of `img`. Workspace: fic_encode_workspace_size bytes (may be NULL/0 for this call). */
fic_status fic_classify(const uint8_t *img, const fic_geom *g, const fic_params *p,
                        const fic_blockstats *out, void *workspace, size_t workspace_bytes,
                        void *stream);

/* Section 3.1 Eq. 3: class-sorted domain and range orders and every range's pool window, from
 * the classes in `st` (as written by fic_classify). Workspace: fic_encode_workspace_size. */
fic_status fic_build_pools(const fic_blockstats *st, const fic_geom *g, const fic_params *p,
                           const fic_pools *out, void *workspace, size_t workspace_bytes,
                           void *stream);

/* Sections 1 and 3: the whole encoder, image -> codes. Equal to the exact least-error search
 * over each range's pool (ties as in fic_codes). `info` (device, nullable) receives the
 * report. Device-side failure: every wait of the tensor matcher on another role of its CTA is
 * bounded (2 s); if one gives up, the kernel stops without leaving work in flight, every code of
 * the call is written as invalid (dom = iso = -1, s = o = sse = NaN), info->device_error (when
 * `info` is given) is FIC_ERR_DEVICE_TIMEOUT, and the next fic_check on the device returns
 * FIC_ERR_DEVICE_TIMEOUT. The call itself returns before the GPU runs, so it cannot report this.
 * The first call with a given argument set (pointers, geometry, parameters, device) on a host
 * thread runs its stages directly; the second captures its work into a CUDA graph on a private
 * stream, and it and later calls with the same arguments replay that graph on `stream` (up to 4
 * argument sets per thread, least recently used replaced). Calls with profiling on, or on a
 * stream the caller is capturing, run the stages directly. */
fic_status fic_encode(const uint8_t *img, const fic_geom *g, const fic_params *p,
                      const fic_codes *out, fic_encode_info *info, void *workspace,
                      size_t workspace_bytes, void *stream);

/* Instrumentation (not part of the method): after a fic_encode with this workspace, geometry and
 * parameters has run on `stream`, writes the ids of the ranges whose best code the tensor engine's
 * ranking could not certify and that were therefore re-searched exactly (Section 1's exhaustive
 * least squares over the uncertified part of the pool), in no particular order, to ids[0 ..
 * min(count, max_ids)) and their number to *count. ids and count are device pointers; 0 ranges
 * for the SIMT engine. Enqueued on `stream`. */
fic_status fic_encode_fallback_ranges(const fic_geom *g, const fic_params *p, void *workspace,
                                      size_t workspace_bytes, int32_t *ids, int32_t max_ids,
                                      int32_t *count, void *stream);

/* Bytes of workspace fic_encode_batched needs for these n images (1 <= n <= 4096). */
size_t fic_encode_batched_workspace_size(const fic_geom *geoms, int32_t n, const fic_params *p);

/* fic_encode over n images at once (Sections 1 and 3 applied to each image independently: every
 * image has its own classes, F_l/F_m and pools). imgs, geoms and outs are HOST arrays of n
 * entries (device image pointers, geometries, code structs of device arrays). The tensor engine
 * matches all images' pools in one persistent launch. `info` (device, nullable) receives the
 * totals over the batch. A device-side timeout marks every image's codes invalid, as in
 * fic_encode. */
fic_status fic_encode_batched(const uint8_t *const *imgs, const fic_geom *geoms, int32_t n,
                              const fic_params *p, const fic_codes *outs, fic_encode_info *info,
                              void *workspace, size_t workspace_bytes, void *stream);

/* Doubles `out` must hold for fic_quality. */
#define FIC_QUALITY_OUT_DOUBLES 1026

/* Table 4's quality metric: decoded 8-bit image clamp(round-half-even(x), 0, 255) (x: H*W floats,
 * dense) against the original `ref` (H x W bytes, row pitch g->pitch). Writes out[0] = mean
 * squared error, out[1] = PSNR = 10 log10(255^2 / MSE) in dB (+inf when MSE = 0); out[2..] is
 * scratch (FIC_QUALITY_OUT_DOUBLES entries in all, device memory). The sum runs in binary64 in
 * a fixed order, so the result does not depend on scheduling. */
fic_status fic_quality(const float *x, const uint8_t *ref, const fic_geom *g, double *out, void *stream);

/* Doubles `header` must hold for fic_quantize. */
#define FIC_QUANT_HEADER_DOUBLES 514

/* A code format for the per-range map coefficients of Section 1 (the paper fixes none): contrast
 * s in [-1, 1] quantised uniformly to 2^bits_s levels including both endpoints, brightness o
 * quantised uniformly to 2^bits_o levels over the codes' own [min o, max o]; 1 <= bits <= 16.
 * With Ls = 2^bits_s - 1 and Lo = 2^bits_o - 1, each a separate binary64 operation:
 *   q_s = clamp(rint(((s + 1) / 2) * Ls), 0, Ls),  s' = (q_s * 2) / Ls - 1,
 *   q_o = clamp(rint(((o - lo) / (hi - lo)) * Lo), 0, Lo) (0 if hi == lo),
 *   o' = lo + (q_o * (hi - lo)) / Lo,  rint rounding half to even.
 * Writes q_s, q_o (n entries), header[0] = lo, header[1] = hi (header holds
 * FIC_QUANT_HEADER_DOUBLES device doubles, the rest scratch) and the dequantised codes to `out`
 * (dom and iso copied from `in`; `out` may be `in`). All pointers are device pointers. */
fic_status fic_quantize(const fic_codes *in, int32_t n, int32_t bits_s, int32_t bits_o, uint16_t *q_s,
                        uint16_t *q_o, double *header, const fic_codes *out, void *stream);

/* Bytes of workspace fic_decode and fic_decode_backward need. */
size_t fic_decode_workspace_size(const fic_geom *g, const fic_params *p, int32_t iters,
                                 int32_t ckpt_every);

/* Section 1: decoding. x_0 = x0 (H*W float, row-major, dense) or 128 everywhere when x0 is
 * NULL; x_{k+1}[range r] = s_r T_{t_r}(D(x_k, dom_r)) + o_r for all ranges from x_k (Jacobi),
 * D the 2x2 average of the 2B x 2B domain; `out` (H*W float) receives x_iters, unclamped.
 * With an even domain stride the steps before the last run on the plane of 2x2 averages of x_k
 * (a quarter of the pixels; the same iterates in exact arithmetic, rounded in another order) and
 * only the last step writes full-resolution pixels.
 * iters >= 0. Workspace: fic_decode_workspace_size. Codes whose domain or isometry is out of range
 * (such as the invalid codes of an encode whose matcher gave up) give NaN pixels for their range.
 * Like fic_encode, the second call with a given argument set on a host thread captures its
 * launches into a CUDA graph (the first runs them directly); later calls with the same arguments
 * replay it (4 argument sets per thread; calls on a stream the caller is capturing run directly). */
fic_status fic_decode(const fic_codes *codes, const fic_geom *g, const fic_params *p,
                      int32_t iters, const float *x0, float *out, void *workspace,
                      size_t workspace_bytes, void *stream);

/* Bytes of workspace fic_decode_scaled needs at this scale. */
size_t fic_decode_scaled_workspace_size(const fic_geom *g, const fic_params *p, int32_t scale);

/* Section 1, resolution independence (decoding may start from an initial image of any size and
 * reconstruct at any size): decodes the codes
 * of the H x W encoding g on the (scale*H) x (scale*W) grid, 1 <= scale <= 16: range r covers the
 * (B scale)^2 block at scale times its position, domain d the (2B scale)^2 block at scale times
 * its position, contracted by 2x2 averaging, under the isometries of the larger square. x0 and out
 * are (scale H) x (scale W) floats (x0 NULL: 128 everywhere). With scale = 1 it is fic_decode;
 * 2x2 block averages of a scale-2 decode equal the scale-1 decode from the same constant start. */
fic_status fic_decode_scaled(const fic_codes *codes, const fic_geom *g, const fic_params *p,
                             int32_t scale, int32_t iters, const float *x0, float *out,
                             void *workspace, size_t workspace_bytes, void *stream);

/* Adjoint of fic_decode with respect to the per-range contrast and brightness: given
 * grad_out = dL/dx_iters (H*W float), writes grad_s[r] = dL/ds_r and grad_o[r] = dL/do_r
 * (R floats each). Iterates are recomputed from checkpoints kept every `ckpt_every` (>= 1)
 * iterations. W^T is applied as a deterministic gather (no floating-point atomics), so the
 * result does not depend on scheduling or on ckpt_every. With an even domain stride the
 * checkpoints, the recomputation and every reverse step but the last (the one that reads
 * grad_out) run on the plane of 2x2 averages, as in fic_decode. Workspace:
 * fic_decode_workspace_size with the same iters and ckpt_every. Like fic_decode, repeated calls
 * with the same arguments replay a CUDA graph of the launches, captured at the second such call
 * (4 argument sets per thread; calls on a stream the caller is capturing run directly). */
fic_status fic_decode_backward(const fic_codes *codes, const fic_geom *g, const fic_params *p,
                               int32_t iters, int32_t ckpt_every, const float *x0,
                               const float *grad_out, float *grad_s, float *grad_o,
                               void *workspace, size_t workspace_bytes, void *stream);

/* Instrumentation (not part of the method). When enabled on the calling thread, fic_encode
 * records CUDA events on its stream around each stage; fic_profile_read waits for the last
 * encode's events and writes the stage durations in milliseconds to ms[0..n):
 *   ms[0] classification, ms[1] pool build, ms[2] operand packing, ms[3] matching,
 *   ms[4] exact re-evaluation, ms[5] exact re-search of uncertified ranges
 * (0 for stages the engine does not run), and the number of kernels the last fic_encode on
 * this thread launched to *launches (nullable). The first enable creates the events on the
 * current device; they are kept for the thread's lifetime (an encode captured in a CUDA graph
 * with profiling on records into them at every replay, as event-record nodes). fic_profile_read
 * returns FIC_ERR_INVALID_ARG if profiling is off. */
fic_status fic_profile_enable(int32_t on);
fic_status fic_profile_read(float *ms, int32_t n, int32_t *launches);

/* Largest image (pixels) fic_decode_static accepts: 1024 x 1024. */
#define FIC_DECODE_STATIC_MAX_PIXELS (1 << 20)

/* fic_decode without any allocation. The paper has no counterpart: this is an interface for
 * callers that cannot call cudaMalloc (applications that reserve all device memory up front and
 * give libraries only the buffers they need, and latency-critical loops where an allocation
 * could block on or synchronise the device), who therefore cannot supply fic_decode's
 * workspace. It computes exactly what fic_decode computes (same arguments, no workspace) using
 * a fixed scratch image of FIC_DECODE_STATIC_MAX_PIXELS floats (4 MiB) kept in the library's
 * device memory, which every GPU that loads the library holds until the process exits. Images
 * with more pixels return FIC_ERR_INVALID_ARG. The first call made with a given device current
 * looks up the scratch's device address (cudaGetSymbolAddress) and caches it for that device and
 * its current CUDA context (a call after the context was destroyed and re-created, e.g. after
 * cudaDeviceReset, looks it up again); make that first call before any stream capture. All calls share the one scratch image: calls whose GPU work
 * overlaps (different streams, concurrent host threads) race on it and must be ordered by the
 * caller. x0 and out must not alias each other. */
fic_status fic_decode_static(const fic_codes *codes, const fic_geom *g, const fic_params *p,
                             int32_t iters, const float *x0, float *out, void *stream);

/* Waits for the work enqueued on `stream` (cudaStreamSynchronize), then reads and clears the
 * library's device error word on the current device: FIC_ERR_DEVICE_TIMEOUT if a bounded
 * device-side wait of any encode on this device gave up since the last fic_check (the codes of that
 * encode are marked invalid, see fic_encode), FIC_ERR_CUDA if the stream reported an error, else
 * FIC_OK. Synchronises the host; not for use on a stream that is being captured. */
fic_status fic_check(void *stream);

/* Testing hook for the device-side error path (not needed to use the library). With ns > 0, the
 * tensor matchers launched by this host thread's later fic_encode / fic_encode_batched calls first
 * wait up to ns nanoseconds (ns <= 1e9) on a barrier that nothing completes, before they issue any
 * copy or MMA, so the wait gives up and the call ends as a device timeout (see fic_encode) with no
 * work in flight. ns = 0 turns it off. While it is on, fic_encode does not use its graph cache. */
fic_status fic_debug_stall_matcher(int64_t ns);

/* 1 if `engine` (FIC_ENGINE_*) can run on the current device with this build, else 0. */
int32_t fic_engine_available(int32_t engine);

/* Message for the last failed call on this thread ("" if none). */
const char *fic_last_error(void);

/* Library version, (major << 16) | minor. */
int32_t fic_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FIC_H */
