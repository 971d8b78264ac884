// C ABI of the fic library (include/fic.h): argument validation, workspace carving and the
// order of launches. All device work is enqueued on the caller's stream.
#include <cuda.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "fic_internal.cuh"

namespace fic {
size_t adjoint_csr_ints(const Geo &g);
size_t adjoint_off_ints(const Geo &g);
size_t adjoint_entries(const Geo &g);
cudaError_t launch_dom_csr(const Geo &g, const fic_codes &c, const AdjointCsr &a, cudaStream_t st);
cudaError_t launch_adjoint_gather(const Geo &g, const fic_codes &c, const AdjointCsr &a, const float *lam,
                                  float *lam_prev, cudaStream_t st);
cudaError_t launch_adjoint_grads(const Geo &g, const fic_codes &c, const float *x, const float *lam,
                                 float2 *gs, float2 *go, cudaStream_t st);
cudaError_t launch_grads_out(int R, const float2 *gsf, const float2 *gof, float *gs, float *go,
                             cudaStream_t st);
cudaError_t launch_quality(const float *x, const uint8_t *ref, int H, int W, int pitch, double *out,
                           cudaStream_t st);
cudaError_t launch_decode_step_scaled(const fic_codes &c, const Geo &g, int z, const float *x, float *y,
                                      cudaStream_t st);
cudaError_t launch_quantize(const fic_codes &in, int n, int bits_s, int bits_o, uint16_t *q_s, uint16_t *q_o,
                            double *header, const fic_codes &out, cudaStream_t st);
bool tensor_engine_available(int device);
constexpr int kMaxBatch = 4096;
}  // namespace fic

using namespace fic;

static_assert(FIC_LITERAL16_OFFSETS == kFdPairs16 + 1, "bucket offsets of the 16x16 literal window");

namespace {

thread_local char g_err[512] = "";

// Testing hook of fic_debug_stall_matcher: the forced wait (ns) of the tensor matchers launched by
// this thread's encodes; 0 = off.
thread_local unsigned long long g_stall_ns = 0;

// Stage timing for fic_profile_*: events 0..6 bracket classify, pools, pack, match, re-evaluate,
// re-search.
struct Prof {
    bool on = false;
    bool made = false;  // events exist (created on the first enable, kept: a captured graph may
                        // record into them after profiling is switched off and on again)
    cudaEvent_t ev[7] = {};
    int launches = 0;
};
thread_local Prof g_prof;

fic_status fail(fic_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

// Internal streams on which the per-image stages of a batch run concurrently (fork/join through
// events on the caller's stream; inside a CUDA graph capture they become parallel branches). One
// set per host thread and device, created on first use outside a capture and kept.
constexpr int kSideStreams = 8;
struct SidePool {
    cudaStream_t s[kSideStreams];
    cudaEvent_t fork, join[kSideStreams];
    bool ready = false;
};
constexpr int kMaxDevices = 64;
thread_local SidePool g_side[kMaxDevices];

// The pool for `dev`, or nullptr (run serially) when it does not exist yet and `st` is capturing.
SidePool *side_pool(int dev, cudaStream_t st) {
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    SidePool &p = g_side[dev];
    if (p.ready) return &p;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    for (int k = 0; k < kSideStreams; ++k) {
        if (cudaStreamCreateWithFlags(&p.s[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p.join[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    }
    if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    p.ready = true;
    return &p;
}

cudaError_t side_fork(cudaStream_t st, SidePool *p, int ns) {
    cudaError_t e = cudaEventRecord(p->fork, st);
    for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p->s[k], p->fork, 0);
    return e;
}

cudaError_t side_join(cudaStream_t st, SidePool *p, int ns) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < ns && e == cudaSuccess; ++k) {
        e = cudaEventRecord(p->join[k], p->s[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->join[k], 0);
    }
    return e;
}

fic_status cuda_fail(cudaError_t e, const char *where) {
    return fail(FIC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define FIC_TRY(call, where)                                 \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);  \
    } while (0)

fic_status make_geo(const fic_geom *gm, const fic_params *p, Geo *g) {
    if (!gm || !p) return fail(FIC_ERR_INVALID_ARG, "null geometry or parameters");
    if (p->block != 8 && p->block != 16) return fail(FIC_ERR_INVALID_ARG, "block must be 8 or 16 (got %d)", p->block);
    const int B = p->block;
    if (gm->H < 2 * B || gm->W < 2 * B || gm->H % B || gm->W % B)
        return fail(FIC_ERR_INVALID_ARG, "H and W must be multiples of %d and >= %d (got %dx%d)",
                    B, 2 * B, gm->H, gm->W);
    if (gm->pitch < gm->W) return fail(FIC_ERR_INVALID_ARG, "pitch %d < W %d", gm->pitch, gm->W);
    if ((long long)gm->H * gm->W > (1LL << 30))
        return fail(FIC_ERR_INVALID_ARG, "image larger than 2^30 pixels");
    if (p->domain_stride < 1) return fail(FIC_ERR_INVALID_ARG, "domain_stride must be >= 1");
    if (p->num_classes < 1 || p->num_classes > kMaxClasses)
        return fail(FIC_ERR_INVALID_ARG, "num_classes must be in [1, %d]", kMaxClasses);
    if (p->half_width < -1) return fail(FIC_ERR_INVALID_ARG, "half_width must be >= -1");
    if (p->s_max != 1.0) return fail(FIC_ERR_INVALID_ARG, "s_max must be 1.0");
    if (p->engine != FIC_ENGINE_TENSOR && p->engine != FIC_ENGINE_SIMT)
        return fail(FIC_ERR_INVALID_ARG, "unknown engine %d", p->engine);
    if (p->flags != 0 && p->flags != FIC_FLAG_LITERAL_WINDOW)
        return fail(FIC_ERR_INVALID_ARG, "flags must be 0 or FIC_FLAG_LITERAL_WINDOW");
    if (p->items_per_sm < 0 || p->items_per_sm > 64)
        return fail(FIC_ERR_INVALID_ARG, "items_per_sm must be in [0, 64]");
    if (p->group_chunks < 0 || p->group_chunks > 1024)
        return fail(FIC_ERR_INVALID_ARG, "group_chunks must be in [0, 1024]");
    if (p->pipeline_stages != 0 && (B == 8 ? (p->pipeline_stages < 3 || p->pipeline_stages > 4)
                                           : (p->pipeline_stages < 4 || p->pipeline_stages > 5)))
        return fail(FIC_ERR_INVALID_ARG, "pipeline_stages must be 0 or in [%d, %d] for block %d", B == 8 ? 3 : 4,
                    B == 8 ? 4 : 5, B);
    g->H = gm->H;
    g->W = gm->W;
    g->pitch = gm->pitch;
    g->B = B;
    g->n = B * B;
    g->sigma = p->domain_stride;
    g->nRy = gm->H / B;
    g->nRx = gm->W / B;
    g->R = g->nRy * g->nRx;
    g->nDy = (gm->H - 2 * B) / g->sigma + 1;
    g->nDx = (gm->W - 2 * B) / g->sigma + 1;
    g->Dn = g->nDy * g->nDx;
    g->K = p->num_classes;
    g->w = p->half_width < 0 ? p->num_classes / 3 : p->half_width;
    g->literal = (p->flags & FIC_FLAG_LITERAL_WINDOW) ? 1 : 0;
    g->fRx = make_fastdiv((uint32_t)g->nRx);
    g->fDx = make_fastdiv((uint32_t)g->nDx);
    g->fS = make_fastdiv((uint32_t)g->sigma);
    g->group_chunks = p->group_chunks > 0 ? p->group_chunks : (B == 16 ? 16 : 64);
    g->stages = p->pipeline_stages;
    return FIC_OK;
}

}  // namespace

namespace fic {

thread_local int g_launches = 0;

// The library's device error word on every GPU that loads it: a matcher whose bounded wait gave up
// writes FIC_ERR_DEVICE_TIMEOUT here (besides the encode's own report); fic_check reads and clears
// it. Its address is looked up with the device current at each encode that launches a matcher.
__device__ int32_t g_device_error = 0;

void set_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

fic_status make_geometry(const fic_geom *gm, const fic_params *p, Geo *g) { return make_geo(gm, p, g); }

namespace {
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
        cudaGetLastError();
    });
    return fn;
}

std::mutex g_errword_mu;
struct SymbolEntry {
    void *ctx = nullptr;
    int32_t *ptr = nullptr;
};
SymbolEntry g_errword[kMaxDevices];
}  // namespace

bool current_context(void **ctx) {
    CtxGetCurrentFn get = ctx_get_current();
    CUcontext c = nullptr;
    if (!get || get(&c) != CUDA_SUCCESS) return false;
    *ctx = (void *)c;
    return true;
}

// Device address of g_device_error in the current device's current context, looked up once per
// (device, context); the encode paths look it up before they begin any stream capture.
cudaError_t device_error_word(int32_t **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *ctx = nullptr;
    if (!current_context(&ctx)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(g_errword_mu);
    SymbolEntry &ent = g_errword[dev];
    if (!ctx || !ent.ptr || ent.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_device_error);  // makes the primary context current if none is
        if (e != cudaSuccess) return e;
        if (!current_context(&ctx) || !ctx) return cudaErrorDeviceUninitialized;
        ent.ptr = static_cast<int32_t *>(p);
        ent.ctx = ctx;
    }
    *ptr = ent.ptr;
    return cudaSuccess;
}

size_t encode_workspace(const Geo *gs, int n, EncodeBufs *bs, TcBatch *tb, void *ws, size_t cap, bool *ok) {
    Carver c(ws, cap);
    long long R_pad_tot = 0, Dn_aux_tot = 0, mt_tot = 0, chunks_tot = 0;
    const int B = gs[0].B, TM = tile_rows(B), npx = B * B, H = B == 16 ? 1 : 2, NS = n_scales(B);
    // per image 8 int32 zeroed together at the start of an encode: [0] re-search count, [2..3] the
    // match count (int64), [4..7] the FD extent reduction words (2 x uint64)
    int32_t *img_counters = c.take<int32_t>(8 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        const Geo &g = gs[k];
        EncodeBufs *b = &bs[k];
        b->R_pad = (g.R + TM - 1) / TM * TM;
        b->Dn_pad = (g.Dn + kTileDom - 1) / kTileDom * kTileDom;
        b->Dn_aux = b->Dn_pad + kTileDom;  // a tile may start at any position < Dn
        b->n_mtiles = b->R_pad / TM;
        // chunks of the absolute grid a tile's window (within this image's Dn domains) can meet
        b->max_chunks = (g.Dn + kChunkDom - 1) / kChunkDom + 1;
        b->sort_blocks_dom = (g.Dn + kSortChunk - 1) / kSortChunk;
        b->sort_blocks_rng = (g.R + kSortChunk - 1) / kSortChunk;
        b->rng_off = (int)R_pad_tot;
        b->dom_off = (int)Dn_aux_tot;
        b->mt_off = (int)mt_tot;
        R_pad_tot += b->R_pad;
        Dn_aux_tot += b->Dn_aux;
        mt_tot += b->n_mtiles;
        chunks_tot += (long long)b->n_mtiles * b->max_chunks;
        const int sort_blocks = b->sort_blocks_dom > b->sort_blocks_rng ? b->sort_blocks_dom : b->sort_blocks_rng;
        b->range_sum = c.take<int32_t>(g.R);
        b->range_sumsq = c.take<int32_t>(g.R);
        b->range_counts = c.take<int32_t>((size_t)NS * g.R);
        b->range_fd = c.take<double>(g.R);
        b->range_bin = c.take<uint8_t>(g.R);
        b->dom_sum = c.take<int32_t>(g.Dn);
        b->dom_sumsq = c.take<int32_t>(g.Dn);
        b->dom_counts = c.take<int32_t>((size_t)NS * g.Dn);
        b->dom_fd = c.take<double>(g.Dn);
        b->dom_bin = c.take<uint8_t>(g.Dn);
        b->fd_extent = c.take<double>(2);
        b->dom_S = c.take<uint16_t>((size_t)g.Dn * npx);
        // bucket offsets: K + 1 classes, or one per FD key in literal mode (+ 1)
        const bool lit16 = g.literal && B == 16;
        const size_t n_off = lit16 ? (size_t)kFdPairs16 + 1 : (size_t)kMaxClasses + 2;
        b->dom_order = c.take<int32_t>(g.Dn);
        b->bin_off = c.take<int32_t>(n_off);
        b->range_order = c.take<int32_t>(g.R);
        b->rbin_off = c.take<int32_t>(n_off);
        b->win_lo = c.take<int32_t>(g.R);
        b->win_hi = c.take<int32_t>(g.R);
        b->dom_key = c.take<uint8_t>(g.Dn);
        b->range_key = c.take<uint8_t>(g.R);
        // per-block class histograms: of the domain sort and of the range sort
        b->sort_counts = c.take<int32_t>(sort_counts_ints(sort_blocks * kSortChunk));
        b->sort_offs = c.take<int32_t>(sort_counts_ints(sort_blocks * kSortChunk));
        b->fallback = c.take<int32_t>(g.R);
        b->fb_best = c.take<FallbackBest>(g.R);
        const int nmax = g.R > g.Dn ? g.R : g.Dn;
        b->lit_key = lit16 ? c.take<int32_t>(nmax) : nullptr;
        b->lit_t1 = lit16 ? c.take<int32_t>(nmax) : nullptr;
        b->lit_t2 = lit16 ? c.take<int32_t>(nmax) : nullptr;
        b->lit_counts = lit16 ? c.take<int32_t>(radix_counts_ints(nmax)) : nullptr;
        b->lit_rank = lit16 ? c.take<int32_t>(kFdPairs16) : nullptr;
        b->lit_digit = lit16 ? c.take<uint8_t>(nmax) : nullptr;
        b->lit_sfd = lit16 ? c.take<double>(g.Dn) : nullptr;
        b->counters = img_counters ? img_counters + 8 * k : nullptr;
        b->matches = img_counters ? reinterpret_cast<long long *>(img_counters + 8 * k + 2) : nullptr;
        b->extent_bits = img_counters ? reinterpret_cast<unsigned long long *>(img_counters + 8 * k + 4) : nullptr;
    }
    tb->B = B;
    tb->tm = TM;
    tb->halves = H;
    tb->R_pad = (int)R_pad_tot;
    tb->Dn_aux = (int)Dn_aux_tot;
    tb->n_mtiles = (int)mt_tot;
    // cpi_cap chunks per domain group: about 32 MB of B rows (512 KB per chunk for B = 8, 2 MB
    // for B = 16). A tile meets at most chunks / cpi + 2 groups, and cpi >= min(cap, total /
    // target), so items <= 2 tiles + max(target, chunks / cap); cutting the last two groups in
    // four adds at most 6 items per tile.
    tb->cpi_cap = gs[0].group_chunks;
    tb->stages = gs[0].stages;
    tb->max_items = (int)(8 * mt_tot + (chunks_tot / tb->cpi_cap + 1 > kMaxItemTarget ? chunks_tot / tb->cpi_cap + 1
                                                                                        : kMaxItemTarget));
    tb->max_chunks = (int)chunks_tot;
    // groups: at most ceil(chunks / cpi) + 6 (the last two cut in four) <= chunks + 6
    tb->ng_max = (int)(Dn_aux_tot / kChunkDom + 8);
    const size_t slice = B == 8 ? 16 : 0;  // correction slice columns (B = 16 corrects in the epilogue)
    tb->A_mat = c.take<__half>((size_t)R_pad_tot * npx, 1024);
    tb->B_mat = c.take<__half>((size_t)8 * Dn_aux_tot * npx, 1024);
    tb->A1_mat = c.take<__half>((size_t)R_pad_tot * slice, 1024);
    tb->B1_mat = c.take<__half>((size_t)8 * Dn_aux_tot * slice, 1024);
    tb->dom_aux = c.take<float4>((size_t)Dn_aux_tot);
    tb->rng_info = c.take<int4>((size_t)R_pad_tot);
    tb->tile_win = c.take<int4>((size_t)mt_tot);
    tb->n_chunks = c.take<int32_t>((size_t)mt_tot);
    tb->tile_items = c.take<int4>((size_t)mt_tot);
    tb->work = c.take<int4>((size_t)tb->max_items);
    tb->work_slot = c.take<int32_t>((size_t)tb->max_items);
    tb->grp = c.take<int32_t>((size_t)tb->ng_max);
    tb->cand = c.take<unsigned long long>((size_t)tb->max_items * TM * H * 2);
    tb->chunk_max = c.take<uint32_t>((size_t)chunks_tot * TM * H * 2);
    tb->gcounters = c.take<int32_t>(8);
    for (int k = 0; k < n; ++k) {
        EncodeBufs *b = &bs[k];
        const bool have = tb->A_mat != nullptr;
        b->A_mat = have ? tb->A_mat + (size_t)b->rng_off * npx : nullptr;
        b->A1_mat = have ? tb->A1_mat + (size_t)b->rng_off * slice : nullptr;
        b->B_mat = have ? tb->B_mat + (size_t)b->dom_off * 8 * npx : nullptr;
        b->B1_mat = have ? tb->B1_mat + (size_t)b->dom_off * 8 * slice : nullptr;
        b->dom_aux = have ? tb->dom_aux + b->dom_off : nullptr;
        b->rng_info = have ? tb->rng_info + b->rng_off : nullptr;
    }
    if (R_pad_tot * npx >= (1LL << 31) || 8 * Dn_aux_tot >= (1LL << 31)) c.ok = false;
    if (ok) *ok = c.ok;
    return c.off + 256;
}

// img_counters: 8 int32 per image ([0] re-search count, [2..3] match count, see encode_workspace)
__global__ void k_write_info(const int32_t *img_counters, int n, const int32_t *gcounters, fic_encode_info *info) {
    long long m = 0;
    int fb = 0;
    for (int k = 0; k < n; ++k) {
        m += *reinterpret_cast<const long long *>(img_counters + 8 * k + 2);
        fb += img_counters[8 * k];
    }
    info->matches = m;
    info->fallback_ranges = fb;
    info->work_items = gcounters[1];
    info->device_error = gcounters[2];
    info->reserved = 0;
}

// Range ids of the re-searched ranges: fallback[] holds class-sorted positions.
__global__ void k_fallback_ids(const int32_t *__restrict__ fallback, const int32_t *__restrict__ counters,
                               const int32_t *__restrict__ range_order, int max_ids, int32_t *__restrict__ ids,
                               int32_t *__restrict__ count) {
    const int n = counters[0];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n && k < max_ids; k += gridDim.x * blockDim.x)
        ids[k] = range_order[fallback[k]];
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

cudaError_t launch_info(const EncodeBufs *b, int n, const TcBatch &tb, fic_encode_info *info, cudaStream_t st) {
    k_write_info<<<1, 1, 0, st>>>(b[0].counters, n, tb.gcounters, info);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic

extern "C" {

const char *fic_last_error(void) { return g_err; }

int32_t fic_version(void) { return (0 << 16) | 1; }

int32_t fic_engine_available(int32_t engine) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (engine == FIC_ENGINE_SIMT) return 1;
    if (engine == FIC_ENGINE_TENSOR) return tensor_engine_available(dev) ? 1 : 0;
    return 0;
}

// Internal check hook for the host-side log2 table (no GPU needed).
double fic_debug_log2(int32_t n) { return log2_correctly_rounded(n); }

size_t fic_encode_workspace_size(const fic_geom *gm, const fic_params *p) {
    return fic_encode_batched_workspace_size(gm, 1, p);
}

size_t fic_encode_batched_workspace_size(const fic_geom *geoms, int32_t n, const fic_params *p) {
    if (!geoms || n < 1 || n > kMaxBatch) {
        fail(FIC_ERR_INVALID_ARG, "batch size must be in [1, %d]", kMaxBatch);
        return 0;
    }
    std::vector<Geo> g(n);
    for (int k = 0; k < n; ++k)
        if (make_geo(&geoms[k], p, &g[k]) != FIC_OK) return 0;
    std::vector<EncodeBufs> b(n);
    TcBatch tb;
    bool ok = true;
    const size_t need = encode_workspace(g.data(), n, b.data(), &tb, nullptr, (size_t)-1, &ok);
    if (!ok) {
        fail(FIC_ERR_INVALID_ARG, "batch too large for 32-bit tile indexing");
        return 0;
    }
    return need + 1024;
}

static fic_status carve_batch(const fic_geom *geoms, int n, const fic_params *p, void *ws, size_t bytes,
                              std::vector<Geo> &g, std::vector<EncodeBufs> &b, TcBatch *tb) {
    if (!geoms || n < 1 || n > kMaxBatch) return fail(FIC_ERR_INVALID_ARG, "batch size must be in [1, %d]", kMaxBatch);
    g.resize(n);
    b.resize(n);
    for (int k = 0; k < n; ++k) {
        fic_status s = make_geo(&geoms[k], p, &g[k]);
        if (s != FIC_OK) return s;
    }
    if (!ws) return fail(FIC_ERR_WORKSPACE, "workspace is null");
    // carve from the first 1024-byte boundary (TMA tiles); the size query includes the slack
    char *base = (char *)(((uintptr_t)ws + 1023) & ~(uintptr_t)1023);
    const size_t slack = (size_t)(base - (char *)ws);
    bool ok = false;
    const size_t need = encode_workspace(g.data(), n, b.data(), tb, base, bytes > slack ? bytes - slack : 0, &ok);
    if (!ok || bytes < need + 1024) return fail(FIC_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, need + 1024);
    return FIC_OK;
}

fic_status fic_classify(const uint8_t *img, const fic_geom *gm, const fic_params *p,
                        const fic_blockstats *out, void *ws, size_t bytes, void *stream) {
    NvtxRange nvtx_range("fic_classify");
    std::vector<Geo> gv;
    std::vector<EncodeBufs> bv;
    TcBatch tb;
    fic_status s = carve_batch(gm, 1, p, ws, bytes, gv, bv, &tb);
    if (s != FIC_OK) return s;
    const Geo &g = gv[0];
    EncodeBufs &b = bv[0];
    if (!img || !out || !out->range_sum || !out->range_sumsq || !out->range_counts ||
        !out->range_fd || !out->range_bin || !out->dom_sum || !out->dom_sumsq ||
        !out->dom_counts || !out->dom_fd || !out->dom_bin || !out->fd_extent)
        return fail(FIC_ERR_INVALID_ARG, "null image or statistics pointer");
    b.range_sum = out->range_sum;
    b.range_sumsq = out->range_sumsq;
    b.range_counts = out->range_counts;
    b.range_fd = out->range_fd;
    b.range_bin = out->range_bin;
    b.dom_sum = out->dom_sum;
    b.dom_sumsq = out->dom_sumsq;
    b.dom_counts = out->dom_counts;
    b.dom_fd = out->dom_fd;
    b.dom_bin = out->dom_bin;
    b.fd_extent = out->fd_extent;
    g_launches = 0;
    FIC_TRY(cudaMemsetAsync(b.counters, 0, 8 * sizeof(int32_t), (cudaStream_t)stream), "memset");
    FIC_TRY(launch_classify(img, g, b, (cudaStream_t)stream), "classify");
    return FIC_OK;
}

fic_status fic_build_pools(const fic_blockstats *st, const fic_geom *gm, const fic_params *p,
                           const fic_pools *out, void *ws, size_t bytes, void *stream) {
    NvtxRange nvtx_range("fic_build_pools");
    std::vector<Geo> gv;
    std::vector<EncodeBufs> bv;
    TcBatch tb;
    fic_status s = carve_batch(gm, 1, p, ws, bytes, gv, bv, &tb);
    if (s != FIC_OK) return s;
    const Geo &g = gv[0];
    EncodeBufs &b = bv[0];
    if (!st || !st->range_bin || !st->dom_bin || !out || !out->dom_order || !out->bin_off ||
        !out->range_order || !out->rbin_off || !out->win_lo || !out->win_hi)
        return fail(FIC_ERR_INVALID_ARG, "null statistics or pool pointer");
    b.range_bin = st->range_bin;
    b.dom_bin = st->dom_bin;
    if (g.literal) {
        if (!st->range_counts || !st->dom_counts || !st->range_fd || !st->fd_extent)
            return fail(FIC_ERR_INVALID_ARG, "the literal window needs box counts, range FDs and F_l/F_m");
        b.range_counts = st->range_counts;
        b.dom_counts = st->dom_counts;
        b.range_fd = st->range_fd;
        b.fd_extent = st->fd_extent;
    }
    b.dom_order = out->dom_order;
    b.bin_off = out->bin_off;
    b.range_order = out->range_order;
    b.rbin_off = out->rbin_off;
    b.win_lo = out->win_lo;
    b.win_hi = out->win_hi;
    g_launches = 0;
    FIC_TRY(cudaMemsetAsync(b.counters, 0, 8 * sizeof(int32_t), (cudaStream_t)stream), "memset");
    FIC_TRY(launch_pools(g, b, (cudaStream_t)stream), "build_pools");
    return FIC_OK;
}

static fic_status encode_batch(const uint8_t *const *imgs, const fic_geom *geoms, int n, const fic_params *p,
                               const fic_codes *outs, fic_encode_info *info, void *ws, size_t bytes,
                               void *stream) {
    std::vector<Geo> g;
    std::vector<EncodeBufs> b;
    TcBatch tb;
    fic_status s = carve_batch(geoms, n, p, ws, bytes, g, b, &tb);
    if (s != FIC_OK) return s;
    if (!imgs || !outs) return fail(FIC_ERR_INVALID_ARG, "null image or code array");
    for (int k = 0; k < n; ++k) {
        const fic_codes &o = outs[k];
        if (!imgs[k] || !o.dom || !o.iso || !o.s || !o.o || !o.sse)
            return fail(FIC_ERR_INVALID_ARG, "null image or code pointer (image %d)", k);
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    FIC_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (p->engine == FIC_ENGINE_TENSOR && !tensor_engine_available(dev))
        return fail(FIC_ERR_UNSUPPORTED, "tensor engine needs an sm_103 device");
    int sms = 0;
    FIC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr");
    if (p->engine == FIC_ENGINE_TENSOR) {
        FIC_TRY(device_error_word(&tb.lib_error), "device error word");
        tb.stall_ns = g_stall_ns;
    }
    g_launches = 0;
    // stage marks; inside a stream capture they become event-record nodes of the graph (external
    // records), so a replayed encode still reports its stage times
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    if (g_prof.on) FIC_TRY(cudaStreamIsCapturing(st, &capturing), "capture status");
    auto mark = [&](int i) -> cudaError_t {
        if (!g_prof.on) return cudaSuccess;
        return capturing == cudaStreamCaptureStatusActive
                   ? cudaEventRecordWithFlags(g_prof.ev[i], st, cudaEventRecordExternal)
                   : cudaEventRecord(g_prof.ev[i], st);
    };
    // a batch runs its per-image stages on internal streams, image k on stream k % ns, joined back
    // before the batch-wide matcher and at the end; a single image stays on the caller's stream
    SidePool *sp = n > 1 ? side_pool(dev, st) : nullptr;
    const int ns = sp ? (n < kSideStreams ? n : kSideStreams) : 0;
    auto on = [&](int k) -> cudaStream_t { return ns ? sp->s[k % ns] : st; };
    const bool tensor = p->engine != FIC_ENGINE_SIMT;
    const bool b16 = g[0].B == 16;
    const int ipsm = p->items_per_sm > 0 ? p->items_per_sm : (b16 ? kItemsPerSm16 : kItemsPerSm);
    // 8x8 ranges in class mode on internal streams: windows, range packing and tile windows fused
    const bool fused_tiles = ns && tensor && !b16 && !g[0].literal;
    FIC_TRY(mark(0), "event");
    FIC_TRY(cudaMemsetAsync(b[0].counters, 0, 8 * sizeof(int32_t) * n, st), "memset");
    FIC_TRY(cudaMemsetAsync(tb.gcounters, 0, 8 * sizeof(int32_t), st), "memset");
    // a single image in class mode on the tensor engine overlaps its independent stages: the range
    // sort with the domain sort, and the domain packing with windows, range packing and the work
    // list (which need the domain sort's class offsets)
    SidePool *sp1 = (n == 1 && tensor && !g[0].literal) ? side_pool(dev, st) : nullptr;
    if (sp1) {
        FIC_TRY(launch_classify(imgs[0], g[0], b[0], st), "classify");
        FIC_TRY(mark(1), "event");
        FIC_TRY(side_fork(st, sp1, 1), "fork");
        FIC_TRY(launch_pools_ranges_sort(g[0], b[0], sp1->s[0]), "pools");
        FIC_TRY(launch_pools_domains(g[0], b[0], st), "pools");
        FIC_TRY(cudaEventRecord(sp1->fork, st), "event");  // domain sort done
        FIC_TRY(cudaStreamWaitEvent(sp1->s[0], sp1->fork, 0), "event");
        FIC_TRY(mark(2), "event");
        if (b16) {
            FIC_TRY(launch_pools_windows(g[0], b[0], sp1->s[0]), "pools");
            FIC_TRY(launch_pack16(imgs[0], g[0], b[0], sp1->s[0], 1), "pack");
        } else {
            // windows, range packing and tile windows in one launch
            FIC_TRY(launch_pack_ranges_tiles(imgs[0], g[0], b[0], tb, sp1->s[0]), "pack");
        }
        // the work list needs only the packed ranges' windows: it runs beside the domain packing
        FIC_TRY(launch_work_list(tb, sms * ipsm, sp1->s[0], !b16), "work_list");
        FIC_TRY(b16 ? launch_pack16(imgs[0], g[0], b[0], st, 2) : launch_pack(imgs[0], g[0], b[0], st, 2), "pack");
        FIC_TRY(side_join(st, sp1, 1), "join");
    } else if (ns) {
        // classification, pools and packing per image (stage marks 1 and 2 coincide with 0)
        FIC_TRY(mark(1), "event");
        FIC_TRY(mark(2), "event");
        FIC_TRY(side_fork(st, sp, ns), "fork");
        for (int k = 0; k < n; ++k) {
            FIC_TRY(launch_classify(imgs[k], g[k], b[k], on(k)), "classify");
            if (fused_tiles) {
                // both sorts, then windows, range packing and tile windows in one launch
                FIC_TRY(launch_pools_domains(g[k], b[k], on(k)), "pools");
                FIC_TRY(launch_pools_ranges_sort(g[k], b[k], on(k)), "pools");
                FIC_TRY(launch_pack_ranges_tiles(imgs[k], g[k], b[k], tb, on(k)), "pack");
                FIC_TRY(launch_pack(imgs[k], g[k], b[k], on(k), 2), "pack");
                continue;
            }
            FIC_TRY(launch_pools(g[k], b[k], on(k)), "pools");
            if (tensor)
                FIC_TRY(b16 ? launch_pack16(imgs[k], g[k], b[k], on(k)) : launch_pack(imgs[k], g[k], b[k], on(k)),
                        "pack");
            else
                FIC_TRY(launch_match_simt(imgs[k], g[k], b[k], outs[k], on(k)), "match_simt");
        }
        FIC_TRY(side_join(st, sp, ns), "join");
    } else {
        for (int k = 0; k < n; ++k) FIC_TRY(launch_classify(imgs[k], g[k], b[k], st), "classify");
        FIC_TRY(mark(1), "event");
        for (int k = 0; k < n; ++k) FIC_TRY(launch_pools(g[k], b[k], st), "pools");
        FIC_TRY(mark(2), "event");
        if (tensor)
            for (int k = 0; k < n; ++k)
                FIC_TRY(b16 ? launch_pack16(imgs[k], g[k], b[k], st) : launch_pack(imgs[k], g[k], b[k], st), "pack");
        else
            for (int k = 0; k < n; ++k) FIC_TRY(launch_match_simt(imgs[k], g[k], b[k], outs[k], st), "match_simt");
    }
    if (!tensor) {
        FIC_TRY(mark(3), "event");
        FIC_TRY(mark(4), "event");
        FIC_TRY(mark(5), "event");
    } else {
        if (!sp1) FIC_TRY(launch_work_list(tb, sms * ipsm, st, fused_tiles), "work_list");
        FIC_TRY(mark(3), "event");
        FIC_TRY(b16 ? launch_match_tc16(tb, sms, st) : launch_match_tc(tb, sms, st), "match_tc");
        FIC_TRY(mark(4), "event");
        if (ns) {
            // re-evaluation and exact re-search per image (stage mark 5 coincides with 4)
            FIC_TRY(mark(5), "event");
            FIC_TRY(side_fork(st, sp, ns), "fork");
            for (int k = 0; k < n; ++k) {
                FIC_TRY(b16 ? launch_reeval16(imgs[k], g[k], b[k], tb, outs[k], on(k))
                            : launch_reeval(imgs[k], g[k], b[k], tb, outs[k], on(k)),
                        "reeval");
                FIC_TRY(launch_rescan(imgs[k], g[k], b[k], tb, outs[k], sms, on(k)), "rescan");
            }
            FIC_TRY(side_join(st, sp, ns), "join");
        } else {
            for (int k = 0; k < n; ++k)
                FIC_TRY(b16 ? launch_reeval16(imgs[k], g[k], b[k], tb, outs[k], st)
                            : launch_reeval(imgs[k], g[k], b[k], tb, outs[k], st),
                        "reeval");
            FIC_TRY(mark(5), "event");
            for (int k = 0; k < n; ++k) FIC_TRY(launch_rescan(imgs[k], g[k], b[k], tb, outs[k], sms, st), "rescan");
        }
    }
    FIC_TRY(mark(6), "event");
    if (info) FIC_TRY(launch_info(b.data(), n, tb, info, st), "info");
    g_prof.launches = g_launches;
    return FIC_OK;
}

}  // extern "C"

// ---- repeated calls: one cached CUDA graph per argument set ----------------------------------
// A fic_encode, fic_decode or fic_decode_backward call whose arguments (pointers, geometry,
// parameters, device) equal an earlier call's on this host thread replays that call's captured
// graph: one launch instead of the stage kernels, memsets and stream forks (encode), of the
// iterations (decode) or of the index build, recomputation and reverse steps (adjoint). The graph embeds
// every pointer and parameter, so equal arguments mean the same work on whatever the buffers hold
// now.
namespace {
constexpr int kGraphCache = 4;
template <class Key>
struct GraphCacheT {
    struct Entry {
        Key key;
        cudaGraphExec_t exec = nullptr;
        int launches = 0;
        unsigned long long used = 0;
    };
    Entry e[kGraphCache];
    unsigned long long tick = 0;
    Key seen[kGraphCache];  // argument sets met once and run directly: the next such call captures
    bool seen_valid[kGraphCache] = {};
    int seen_next = 0;
};
thread_local cudaStream_t g_capture_stream[kMaxDevices] = {};  // private capture streams

// Replays the graph cached for `k`; else, the first time an argument set is met, runs
// enqueue(st) directly and remembers the set, and the second time captures enqueue(capture
// stream) into a new graph (after prepare(), which creates whatever must exist before a capture
// begins) and replays that, so calls whose buffers change every time never pay for a capture. Keys
// compare as bytes, padding included, so callers zero them before filling them in.
template <class Key, class Prepare, class Enqueue>
fic_status replay_or_capture(GraphCacheT<Key> &cache, const Key &k, int dev, cudaStream_t st, Prepare prepare,
                             Enqueue enqueue) {
    typename GraphCacheT<Key>::Entry *hit = nullptr, *victim = nullptr;
    for (auto &e : cache.e) {
        if (e.exec && memcmp(&e.key, &k, sizeof k) == 0) {
            hit = &e;
            break;
        }
        if (!victim || !e.exec || (victim->exec && e.used < victim->used)) victim = &e;
    }
    if (!hit) {
        bool seen = false;
        for (int i = 0; i < kGraphCache && !seen; ++i)
            seen = cache.seen_valid[i] && memcmp(&cache.seen[i], &k, sizeof k) == 0;
        if (!seen) {
            const int i = cache.seen_next++ % kGraphCache;
            cache.seen[i] = k;
            cache.seen_valid[i] = true;
            return enqueue(st);
        }
        const fic_status ps = prepare();
        if (ps != FIC_OK) return ps;
        cudaStream_t &cap = g_capture_stream[dev];
        if (!cap) FIC_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
        FIC_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        const fic_status s = enqueue(cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cap, &graph);
        if (s != FIC_OK) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return s;
        }
        if (ce != cudaSuccess) return fail(FIC_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(FIC_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
        if (victim->exec) cudaGraphExecDestroy(victim->exec);
        victim->key = k;
        victim->exec = exec;
        victim->launches = g_launches;
        hit = victim;
    }
    hit->used = ++cache.tick;
    FIC_TRY(cudaGraphLaunch(hit->exec, st), "cudaGraphLaunch");
    g_launches = hit->launches;
    return FIC_OK;
}

// The current device, when a call on `st` may use the graph cache (not while `st` is capturing).
bool cacheable(cudaStream_t st, int *dev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone ||
        cudaGetDevice(dev) != cudaSuccess || *dev < 0 || *dev >= kMaxDevices) {
        cudaGetLastError();
        return false;
    }
    return true;
}

struct EncodeKey {
    const void *img, *ws, *info;
    size_t bytes;
    fic_geom g;
    fic_params p;
    fic_codes out;
    int dev;
};
thread_local GraphCacheT<EncodeKey> g_encode_graphs;
}  // namespace

extern "C" {

fic_status fic_encode(const uint8_t *img, const fic_geom *gm, const fic_params *p,
                      const fic_codes *out, fic_encode_info *info, void *ws, size_t bytes,
                      void *stream) {
    NvtxRange nvtx_range("fic_encode");
    const uint8_t *imgs[1] = {img};
    if (!out) return fail(FIC_ERR_INVALID_ARG, "null code pointer");
    cudaStream_t st = (cudaStream_t)stream;
    // profiling (stage events), the stall hook, a caller's own capture and bad arguments take the
    // direct path
    int dev = -1;
    if (g_prof.on || g_stall_ns || !gm || !p || !cacheable(st, &dev))
        return encode_batch(imgs, gm, 1, p, out, info, ws, bytes, stream);
    EncodeKey k;
    memset(&k, 0, sizeof k);  // padding included: keys compare as bytes
    k.img = img;
    k.ws = ws;
    k.info = info;
    k.bytes = bytes;
    k.g = *gm;
    k.p = *p;
    k.out = *out;
    k.dev = dev;
    const fic_status s = replay_or_capture(
        g_encode_graphs, k, dev, st,
        [&]() -> fic_status {
            // the internal streams and the error word's address exist before the capture starts
            side_pool(dev, st);
            int32_t *ew = nullptr;
            FIC_TRY(device_error_word(&ew), "device error word");
            return FIC_OK;
        },
        [&](cudaStream_t cap) { return encode_batch(imgs, gm, 1, p, out, info, ws, bytes, cap); });
    g_prof.launches = g_launches;
    return s;
}

fic_status fic_encode_fallback_ranges(const fic_geom *gm, const fic_params *p, void *ws, size_t bytes,
                                      int32_t *ids, int32_t max_ids, int32_t *count, void *stream) {
    NvtxRange nvtx_range("fic_encode_fallback_ranges");
    std::vector<Geo> gv;
    std::vector<EncodeBufs> bv;
    TcBatch tb;
    fic_status s = carve_batch(gm, 1, p, ws, bytes, gv, bv, &tb);
    if (s != FIC_OK) return s;
    if (!count || max_ids < 0 || (max_ids > 0 && !ids)) return fail(FIC_ERR_INVALID_ARG, "null output or max_ids < 0");
    g_launches = 0;
    k_fallback_ids<<<64, 256, 0, (cudaStream_t)stream>>>(bv[0].fallback, bv[0].counters, bv[0].range_order, max_ids,
                                                        ids, count);
    ++g_launches;
    FIC_TRY(cudaGetLastError(), "fallback_ranges");
    return FIC_OK;
}

fic_status fic_encode_batched(const uint8_t *const *imgs, const fic_geom *geoms, int32_t n,
                              const fic_params *p, const fic_codes *outs, fic_encode_info *info,
                              void *ws, size_t bytes, void *stream) {
    NvtxRange nvtx_range("fic_encode_batched");
    return encode_batch(imgs, geoms, n, p, outs, info, ws, bytes, stream);
}

fic_status fic_quality(const float *x, const uint8_t *ref, const fic_geom *gm, double *out, void *stream) {
    NvtxRange nvtx_range("fic_quality");
    if (!x || !ref || !gm || !out) return fail(FIC_ERR_INVALID_ARG, "null pointer");
    if (gm->H < 1 || gm->W < 1 || gm->pitch < gm->W) return fail(FIC_ERR_INVALID_ARG, "bad geometry");
    g_launches = 0;
    FIC_TRY(launch_quality(x, ref, gm->H, gm->W, gm->pitch, out, (cudaStream_t)stream), "quality");
    return FIC_OK;
}

fic_status fic_quantize(const fic_codes *in, int32_t n, int32_t bits_s, int32_t bits_o, uint16_t *q_s,
                        uint16_t *q_o, double *header, const fic_codes *out, void *stream) {
    NvtxRange nvtx_range("fic_quantize");
    if (!in || !in->dom || !in->iso || !in->s || !in->o || !out || !out->dom || !out->iso || !out->s ||
        !out->o || !q_s || !q_o || !header)
        return fail(FIC_ERR_INVALID_ARG, "null pointer");
    if (n < 1 || bits_s < 1 || bits_s > 16 || bits_o < 1 || bits_o > 16)
        return fail(FIC_ERR_INVALID_ARG, "n must be >= 1 and bits in [1, 16]");
    g_launches = 0;
    FIC_TRY(launch_quantize(*in, n, bits_s, bits_o, q_s, q_o, header, *out, (cudaStream_t)stream), "quantize");
    return FIC_OK;
}

fic_status fic_profile_enable(int32_t on) {
    if (on && !g_prof.made) {
        for (auto &e : g_prof.ev) FIC_TRY(cudaEventCreate(&e), "cudaEventCreate");
        g_prof.made = true;
    }
    g_prof.on = on != 0;
    return FIC_OK;
}

fic_status fic_profile_read(float *ms, int32_t n, int32_t *launches) {
    if (!g_prof.on) return fail(FIC_ERR_INVALID_ARG, "profiling is not enabled");
    if (n < 0 || (n > 0 && !ms)) return fail(FIC_ERR_INVALID_ARG, "bad output array");
    FIC_TRY(cudaEventSynchronize(g_prof.ev[6]), "cudaEventSynchronize");
    for (int i = 0; i < n && i < 6; ++i) FIC_TRY(cudaEventElapsedTime(&ms[i], g_prof.ev[i], g_prof.ev[i + 1]), "elapsed");
    for (int i = 6; i < n; ++i) ms[i] = 0.f;
    if (launches) *launches = g_prof.launches;
    return FIC_OK;
}

fic_status fic_check(void *stream) {
    NvtxRange nvtx_range("fic_check");
    FIC_TRY(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
    int32_t v = 0;
    FIC_TRY(cudaMemcpyFromSymbol(&v, g_device_error, sizeof v), "reading the device error word");
    if (v == 0) return FIC_OK;
    const int32_t zero = 0;
    FIC_TRY(cudaMemcpyToSymbol(g_device_error, &zero, sizeof zero), "clearing the device error word");
    return fail(FIC_ERR_DEVICE_TIMEOUT,
                "a bounded wait of the tensor matcher gave up; that encode's codes are marked invalid "
                "(dom = iso = -1, s = o = sse = NaN)");
}

fic_status fic_debug_stall_matcher(int64_t ns) {
    if (ns < 0 || ns > 1000000000LL) return fail(FIC_ERR_INVALID_ARG, "stall must be in [0, 1e9] ns");
    g_stall_ns = (unsigned long long)ns;
    return FIC_OK;
}

size_t fic_decode_workspace_size(const fic_geom *gm, const fic_params *p, int32_t iters,
                                 int32_t ckpt_every) {
    Geo g{};
    if (make_geo(gm, p, &g) != FIC_OK || iters < 0) return 0;
    const size_t img = (size_t)g.H * g.W;
    const int ck = ckpt_every < 1 ? 1 : ckpt_every;
    const int nseg = iters > 0 ? (iters + ck - 1) / ck : 1;
    Carver c(nullptr, (size_t)-1);
    c.take<float>(img);                       // decode ping-pong
    c.take<float>(img * (size_t)nseg);        // checkpoints
    c.take<float>(img * (size_t)(ck));        // segment iterates
    c.take<float>(2 * img);                   // adjoint vectors
    c.take<int32_t>(adjoint_csr_ints(g));     // domain -> ranges index: keys, list, sort buffers,
                                              // segment starts, radix histograms
    c.take<uint8_t>(g.R);                     // radix digits
    c.take<int4>(adjoint_entries(g));         // packed (range, isometry, s / 4) per list position
    c.take<float>((size_t)g.R * g.n);         // per-range cell blocks of W^T
    c.take<float2>(2 * (size_t)g.R);          // float-float gradient accumulators
    return c.off + 256;
}

static fic_status check_codes(const fic_codes *c) {
    if (!c || !c->dom || !c->iso || !c->s || !c->o)
        return fail(FIC_ERR_INVALID_ARG, "null code pointer");
    return FIC_OK;
}

}  // extern "C"

namespace {
// Enqueues x_iters = W^iters(x_0) into `out` (`tmp`: H * W floats of scratch).
fic_status decode_enqueue(const fic_codes &codes, const Geo &g, int iters, const float *x0, float *out, float *tmp,
                          cudaStream_t st) {
    const size_t img = (size_t)g.H * g.W;
    g_launches = 0;
    if (iters == 0) {
        if (x0) FIC_TRY(cudaMemcpyAsync(out, x0, img * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy");
        else FIC_TRY(launch_fill(out, img, 128.f, st), "fill");
        return FIC_OK;
    }
    FIC_TRY(launch_decode_iterate(codes, g, iters, x0, out, tmp, st), "decode");
    return FIC_OK;
}

struct DecodeKey {
    fic_codes codes;
    fic_geom g;
    fic_params p;
    const void *x0, *out, *ws;
    size_t bytes;
    int iters, dev;
};
thread_local GraphCacheT<DecodeKey> g_decode_graphs;
}  // namespace

extern "C" {

fic_status fic_decode(const fic_codes *codes, const fic_geom *gm, const fic_params *p,
                      int32_t iters, const float *x0, float *out, void *ws, size_t bytes,
                      void *stream) {
    NvtxRange nvtx_range("fic_decode");
    Geo g{};
    fic_status s = make_geo(gm, p, &g);
    if (s != FIC_OK) return s;
    if ((s = check_codes(codes)) != FIC_OK) return s;
    if (!out || iters < 0) return fail(FIC_ERR_INVALID_ARG, "null output or negative iters");
    if (!ws || (uintptr_t)ws % 256) return fail(FIC_ERR_WORKSPACE, "workspace null or misaligned");
    const size_t need = fic_decode_workspace_size(gm, p, iters, 1);
    const size_t img = (size_t)g.H * g.W;
    if (bytes < img * sizeof(float)) return fail(FIC_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    float *tmp = (float *)ws;
    int dev = -1;
    if (!cacheable(st, &dev)) return decode_enqueue(*codes, g, iters, x0, out, tmp, st);
    DecodeKey k;
    memset(&k, 0, sizeof k);  // padding included: keys compare as bytes
    k.codes = *codes;
    k.g = *gm;
    k.p = *p;
    k.x0 = x0;
    k.out = out;
    k.ws = ws;
    k.bytes = bytes;
    k.iters = iters;
    k.dev = dev;
    return replay_or_capture(
        g_decode_graphs, k, dev, st, []() { return FIC_OK; },
        [&](cudaStream_t cap) { return decode_enqueue(*codes, g, iters, x0, out, tmp, cap); });
}

size_t fic_decode_scaled_workspace_size(const fic_geom *gm, const fic_params *p, int32_t scale) {
    Geo g{};
    if (make_geo(gm, p, &g) != FIC_OK || scale < 1 || scale > 16) return 0;
    return (size_t)g.H * g.W * scale * scale * sizeof(float) + 256;
}

fic_status fic_decode_scaled(const fic_codes *codes, const fic_geom *gm, const fic_params *p, int32_t scale,
                             int32_t iters, const float *x0, float *out, void *ws, size_t bytes, void *stream) {
    NvtxRange nvtx_range("fic_decode_scaled");
    Geo g{};
    fic_status s = make_geo(gm, p, &g);
    if (s != FIC_OK) return s;
    if ((s = check_codes(codes)) != FIC_OK) return s;
    if (!out || iters < 0 || scale < 1 || scale > 16)
        return fail(FIC_ERR_INVALID_ARG, "null output, negative iters or scale outside [1, 16]");
    const size_t img = (size_t)g.H * g.W * scale * scale;
    if (!ws || (uintptr_t)ws % 256 || bytes < img * sizeof(float))
        return fail(FIC_ERR_WORKSPACE, "workspace null, misaligned or below %zu bytes", img * sizeof(float));
    cudaStream_t st = (cudaStream_t)stream;
    g_launches = 0;
    float *tmp = (float *)ws;
    if (iters == 0) {
        if (x0) FIC_TRY(cudaMemcpyAsync(out, x0, img * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy");
        else FIC_TRY(launch_fill(out, img, 128.f, st), "fill");
        return FIC_OK;
    }
    const float *cur = x0;
    if (!x0) {
        float *init = ((iters - 1) % 2 == 0) ? tmp : out;
        FIC_TRY(launch_fill(init, img, 128.f, st), "fill");
        cur = init;
    }
    for (int k = 0; k < iters; ++k) {
        float *dst = ((iters - 1 - k) % 2 == 0) ? out : tmp;
        FIC_TRY(launch_decode_step_scaled(*codes, g, scale, cur, dst, st), "decode_step_scaled");
        cur = dst;
    }
    return FIC_OK;
}

}  // extern "C"

namespace {
// Enqueues the adjoint of fic_decode_backward (arguments already checked) on st.
fic_status backward_enqueue(const fic_codes *codes, const Geo &g, int32_t iters, int32_t ckpt_every,
                            const float *x0, const float *grad_out, float *grad_s, float *grad_o, void *ws,
                            size_t bytes, cudaStream_t st) {
    const size_t img = (size_t)g.H * g.W;
    const int ck = ckpt_every;
    const int nseg = iters > 0 ? (iters + ck - 1) / ck : 1;
    Carver c(ws, bytes);
    float *pingpong = c.take<float>(img);
    float *ckpt = c.take<float>(img * (size_t)nseg);
    float *seg = c.take<float>(img * (size_t)ck);
    float *lam = c.take<float>(2 * img);
    AdjointCsr csr;
    int32_t *ints = c.take<int32_t>(adjoint_csr_ints(g));
    csr.key = ints;
    csr.list = ints + g.R;
    csr.t1 = ints + 2 * (size_t)g.R;
    csr.t2 = ints + 3 * (size_t)g.R;
    csr.off = ints + 4 * (size_t)g.R;
    csr.counts = csr.off + adjoint_off_ints(g);  // 16-byte aligned (the workspace is 256-byte aligned)
    csr.digit = c.take<uint8_t>(g.R);
    csr.ent = c.take<int4>(adjoint_entries(g));
    csr.acc = c.take<float>((size_t)g.R * g.n);
    float2 *gacc = c.take<float2>(2 * (size_t)g.R);  // float-float gradient accumulators
    g_launches = 0;
    FIC_TRY(cudaMemsetAsync(gacc, 0, sizeof(float2) * 2 * g.R, st), "memset");
    if (iters == 0) {
        FIC_TRY(launch_grads_out(g.R, gacc, gacc + g.R, grad_s, grad_o, st), "grads_out");
        return FIC_OK;
    }
    FIC_TRY(launch_dom_csr(g, *codes, csr, st), "csr");
    if (decode_on_plane(g)) {
        // even strides: checkpoints, recomputation and every step but the last on the plane of
        // 2x2 averages, as fic_decode iterates (the packed codes go where the full-resolution
        // ping-pong buffer would)
        FIC_TRY(launch_backward_plane(*codes, g, csr, iters, ck, x0, grad_out, ckpt, seg, lam,
                                      reinterpret_cast<int4 *>(pingpong), gacc, gacc + g.R, st),
                "backward_plane");
        FIC_TRY(launch_grads_out(g.R, gacc, gacc + g.R, grad_s, grad_o, st), "grads_out");
        return FIC_OK;
    }
    // forward: checkpoints x_0, x_ck, x_2ck, ...
    if (x0) FIC_TRY(cudaMemcpyAsync(ckpt, x0, img * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy");
    else FIC_TRY(launch_fill(ckpt, img, 128.f, st), "fill");
    auto seg_ptr = [&](int c0, int i) -> float * {  // iterate c0*ck + i within a segment
        return i == 0 ? ckpt + (size_t)c0 * img : seg + (size_t)i * img;
    };
    for (int c0 = 0; c0 + 1 < nseg; ++c0) {
        for (int i = 1; i <= ck; ++i) {
            float *dst = (i == ck) ? ckpt + (size_t)(c0 + 1) * img : seg_ptr(c0, i);
            FIC_TRY(launch_decode_step(*codes, g, seg_ptr(c0, i - 1), dst, st), "decode_step");
        }
    }
    // backward
    float *lcur = lam, *lprev = lam + img;
    FIC_TRY(cudaMemcpyAsync(lcur, grad_out, img * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy");
    for (int c0 = nseg - 1; c0 >= 0; --c0) {
        const int len = (c0 == nseg - 1) ? iters - c0 * ck : ck;
        for (int i = 1; i < len; ++i)
            FIC_TRY(launch_decode_step(*codes, g, seg_ptr(c0, i - 1), seg_ptr(c0, i), st), "decode_step");
        for (int i = len - 1; i >= 0; --i) {
            FIC_TRY(launch_adjoint_grads(g, *codes, seg_ptr(c0, i), lcur, gacc, gacc + g.R, st), "grads");
            if (c0 > 0 || i > 0) {
                FIC_TRY(launch_adjoint_gather(g, *codes, csr, lcur, lprev, st), "gather");
                float *t = lcur;
                lcur = lprev;
                lprev = t;
            }
        }
    }
    FIC_TRY(launch_grads_out(g.R, gacc, gacc + g.R, grad_s, grad_o, st), "grads_out");
    return FIC_OK;
}


struct BackwardKey {
    fic_codes codes;
    fic_geom g;
    fic_params p;
    const void *x0, *grad_out, *grad_s, *grad_o, *ws;
    size_t bytes;
    int iters, ckpt, dev;
};
thread_local GraphCacheT<BackwardKey> g_backward_graphs;
}  // namespace

extern "C" {

fic_status fic_decode_backward(const fic_codes *codes, const fic_geom *gm, const fic_params *p,
                               int32_t iters, int32_t ckpt_every, const float *x0,
                               const float *grad_out, float *grad_s, float *grad_o, void *ws,
                               size_t bytes, void *stream) {
    NvtxRange nvtx_range("fic_decode_backward");
    Geo g{};
    fic_status s = make_geo(gm, p, &g);
    if (s != FIC_OK) return s;
    if ((s = check_codes(codes)) != FIC_OK) return s;
    if (!grad_out || !grad_s || !grad_o || iters < 0 || ckpt_every < 1)
        return fail(FIC_ERR_INVALID_ARG, "null gradient pointer, iters < 0 or ckpt_every < 1");
    if (!ws || (uintptr_t)ws % 256) return fail(FIC_ERR_WORKSPACE, "workspace null or misaligned");
    const size_t need = fic_decode_workspace_size(gm, p, iters, ckpt_every);
    if (bytes < need) return fail(FIC_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = -1;
    if (!cacheable(st, &dev))
        return backward_enqueue(codes, g, iters, ckpt_every, x0, grad_out, grad_s, grad_o, ws, bytes, st);
    BackwardKey k;
    memset(&k, 0, sizeof k);  // padding included: keys compare as bytes
    k.codes = *codes;
    k.g = *gm;
    k.p = *p;
    k.x0 = x0;
    k.grad_out = grad_out;
    k.grad_s = grad_s;
    k.grad_o = grad_o;
    k.ws = ws;
    k.bytes = bytes;
    k.iters = iters;
    k.ckpt = ckpt_every;
    k.dev = dev;
    return replay_or_capture(
        g_backward_graphs, k, dev, st, []() { return FIC_OK; },
        [&](cudaStream_t cap) {
            return backward_enqueue(codes, g, iters, ckpt_every, x0, grad_out, grad_s, grad_o, ws, bytes, cap);
        });
}

}  // extern "C"
