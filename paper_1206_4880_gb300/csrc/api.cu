// C ABI of the fic library (include/fic.h): argument validation, workspace carving and the
// order of launches. All device work is enqueued on the caller's stream.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fic_internal.cuh"

namespace fic {
cudaError_t launch_dom_csr(const Geo &g, const int32_t *dom, int32_t *cnt, int32_t *off,
                           int32_t *cursor, int32_t *list, cudaStream_t st);
cudaError_t launch_adjoint_gather(const Geo &g, const fic_codes &c, const int32_t *off,
                                  const int32_t *list, const float *lam, float *lam_prev,
                                  cudaStream_t st);
cudaError_t launch_adjoint_grads(const Geo &g, const fic_codes &c, const float *x, const float *lam,
                                 double *gs, double *go, cudaStream_t st);
cudaError_t launch_grads_out(int R, const double *gs64, const double *go64, float *gs, float *go,
                             cudaStream_t st);
bool tensor_engine_available(int device);
}  // namespace fic

using namespace fic;

namespace {

thread_local char g_err[512] = "";

// Stage timing for fic_profile_*: events 0..6 bracket classify, pools, pack, match, re-evaluate,
// re-search.
struct Prof {
    bool on = false;
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
    if (p->block != 8) return fail(FIC_ERR_INVALID_ARG, "block must be 8 (got %d)", p->block);
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
    if (p->flags != 0) return fail(FIC_ERR_INVALID_ARG, "flags must be 0");
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
    return FIC_OK;
}

}  // namespace

namespace fic {

thread_local int g_launches = 0;

// Sets the message fic_last_error() returns on this thread.
void set_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

size_t encode_workspace(const Geo &g, EncodeBufs *b, void *ws, size_t cap, bool *ok) {
    Carver c(ws, cap);
    b->R_pad = (g.R + kTileM - 1) / kTileM * kTileM;
    b->Dn_pad = (g.Dn + kTileDom - 1) / kTileDom * kTileDom;
    b->Dn_aux = b->Dn_pad + kTileDom;  // a tile may start at any position < Dn
    b->n_mtiles = b->R_pad / kTileM;
    const int chunk_dom = kTileDom * kChunkTiles;
    b->max_chunks = (g.Dn + chunk_dom - 1) / chunk_dom;
    b->max_items = b->n_mtiles * b->max_chunks;
    b->sort_blocks_dom = (g.Dn + kSortChunk - 1) / kSortChunk;
    b->sort_blocks_rng = (g.R + kSortChunk - 1) / kSortChunk;
    const int sort_blocks = b->sort_blocks_dom > b->sort_blocks_rng ? b->sort_blocks_dom : b->sort_blocks_rng;
    b->range_sum = c.take<int32_t>(g.R);
    b->range_sumsq = c.take<int32_t>(g.R);
    b->range_counts = c.take<int32_t>(2 * (size_t)g.R);
    b->range_fd = c.take<double>(g.R);
    b->range_bin = c.take<uint8_t>(g.R);
    b->dom_sum = c.take<int32_t>(g.Dn);
    b->dom_sumsq = c.take<int32_t>(g.Dn);
    b->dom_counts = c.take<int32_t>(2 * (size_t)g.Dn);
    b->dom_fd = c.take<double>(g.Dn);
    b->dom_bin = c.take<uint8_t>(g.Dn);
    b->fd_extent = c.take<double>(2);
    b->extent_bits = c.take<unsigned long long>(2);
    b->dom_S = c.take<uint16_t>((size_t)g.Dn * 64);
    b->dom_order = c.take<int32_t>(g.Dn);
    b->bin_off = c.take<int32_t>(kMaxClasses + 2);
    b->range_order = c.take<int32_t>(g.R);
    b->rbin_off = c.take<int32_t>(kMaxClasses + 2);
    b->win_lo = c.take<int32_t>(g.R);
    b->win_hi = c.take<int32_t>(g.R);
    b->sort_counts = c.take<int32_t>((size_t)sort_blocks * 256);
    b->sort_offs = c.take<int32_t>((size_t)sort_blocks * 256);
    b->A_mat = c.take<__half>((size_t)b->R_pad * 64, 1024);
    b->B_mat = c.take<__half>((size_t)8 * b->Dn_aux * 64, 1024);
    b->dom_aux = c.take<float4>(b->Dn_aux);
    b->rng_info = c.take<int4>(b->R_pad);
    b->work = c.take<int4>(b->max_items);
    b->tile_win = c.take<int4>(b->n_mtiles);
    b->n_chunks = c.take<int32_t>(b->n_mtiles);
    b->cand = c.take<unsigned long long>((size_t)b->R_pad * b->max_chunks * 4);
    b->fallback = c.take<int32_t>(g.R);
    b->fb_best = c.take<FallbackBest>(g.R);
    b->counters = c.take<int32_t>(8);
    b->matches = c.take<long long>(1);
    if (ok) *ok = c.ok;
    return c.off + 256;
}

__global__ void k_write_info(const long long *matches, const int32_t *counters, fic_encode_info *info) {
    info->matches = *matches;
    info->fallback_ranges = counters[0];
    info->work_items = counters[1];
    info->device_error = counters[2];
    info->reserved = 0;
}

cudaError_t launch_info(const EncodeBufs &b, fic_encode_info *info, cudaStream_t st) {
    k_write_info<<<1, 1, 0, st>>>(b.matches, b.counters, info);
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
    Geo g;
    if (make_geo(gm, p, &g) != FIC_OK) return 0;
    EncodeBufs b;
    return encode_workspace(g, &b, nullptr, (size_t)-1, nullptr);
}

static fic_status carve_encode(const fic_geom *gm, const fic_params *p, void *ws, size_t bytes,
                               Geo *g, EncodeBufs *b) {
    fic_status s = make_geo(gm, p, g);
    if (s != FIC_OK) return s;
    if (!ws) return fail(FIC_ERR_WORKSPACE, "workspace is null");
    if ((uintptr_t)ws % 256) return fail(FIC_ERR_WORKSPACE, "workspace must be 256-byte aligned");
    bool ok = false;
    const size_t need = encode_workspace(*g, b, ws, bytes, &ok);
    if (!ok || bytes < need)
        return fail(FIC_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, need);
    return FIC_OK;
}

fic_status fic_classify(const uint8_t *img, const fic_geom *gm, const fic_params *p,
                        const fic_blockstats *out, void *ws, size_t bytes, void *stream) {
    Geo g;
    EncodeBufs b;
    fic_status s = carve_encode(gm, p, ws, bytes, &g, &b);
    if (s != FIC_OK) return s;
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
    FIC_TRY(launch_classify(img, g, b, (cudaStream_t)stream), "classify");
    return FIC_OK;
}

fic_status fic_build_pools(const fic_blockstats *st, const fic_geom *gm, const fic_params *p,
                           const fic_pools *out, void *ws, size_t bytes, void *stream) {
    Geo g;
    EncodeBufs b;
    fic_status s = carve_encode(gm, p, ws, bytes, &g, &b);
    if (s != FIC_OK) return s;
    if (!st || !st->range_bin || !st->dom_bin || !out || !out->dom_order || !out->bin_off ||
        !out->range_order || !out->rbin_off || !out->win_lo || !out->win_hi)
        return fail(FIC_ERR_INVALID_ARG, "null statistics or pool pointer");
    b.range_bin = st->range_bin;
    b.dom_bin = st->dom_bin;
    b.dom_order = out->dom_order;
    b.bin_off = out->bin_off;
    b.range_order = out->range_order;
    b.rbin_off = out->rbin_off;
    b.win_lo = out->win_lo;
    b.win_hi = out->win_hi;
    FIC_TRY(launch_pools(g, b, (cudaStream_t)stream), "build_pools");
    return FIC_OK;
}

fic_status fic_encode(const uint8_t *img, const fic_geom *gm, const fic_params *p,
                      const fic_codes *out, fic_encode_info *info, void *ws, size_t bytes,
                      void *stream) {
    Geo g;
    EncodeBufs b;
    fic_status s = carve_encode(gm, p, ws, bytes, &g, &b);
    if (s != FIC_OK) return s;
    if (!img || !out || !out->dom || !out->iso || !out->s || !out->o || !out->sse)
        return fail(FIC_ERR_INVALID_ARG, "null image or code pointer");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    FIC_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (p->engine == FIC_ENGINE_TENSOR && !tensor_engine_available(dev))
        return fail(FIC_ERR_UNSUPPORTED, "tensor engine needs an sm_103 device");
    g_launches = 0;
    auto mark = [&](int i) -> cudaError_t {
        return g_prof.on ? cudaEventRecord(g_prof.ev[i], st) : cudaSuccess;
    };
    FIC_TRY(mark(0), "event");
    FIC_TRY(cudaMemsetAsync(b.counters, 0, 8 * sizeof(int32_t), st), "memset");
    FIC_TRY(launch_classify(img, g, b, st), "classify");
    FIC_TRY(mark(1), "event");
    FIC_TRY(launch_pools(g, b, st), "pools");
    FIC_TRY(mark(2), "event");
    if (p->engine == FIC_ENGINE_SIMT) {
        FIC_TRY(mark(3), "event");
        FIC_TRY(launch_match_simt(img, g, b, *out, st), "match_simt");
        FIC_TRY(mark(4), "event");
        FIC_TRY(mark(5), "event");
    } else {
        int sms = 0;
        FIC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attr");
        FIC_TRY(launch_pack(img, g, b, st), "pack");
        FIC_TRY(mark(3), "event");
        FIC_TRY(launch_match_tc(g, b, sms, st), "match_tc");
        FIC_TRY(mark(4), "event");
        FIC_TRY(launch_reeval(img, g, b, *out, st), "reeval");
        FIC_TRY(mark(5), "event");
        FIC_TRY(launch_rescan(img, g, b, *out, sms, st), "rescan");
    }
    FIC_TRY(mark(6), "event");
    if (info) FIC_TRY(launch_info(b, info, st), "info");
    g_prof.launches = g_launches;
    return FIC_OK;
}

fic_status fic_profile_enable(int32_t on) {
    if (on && !g_prof.on) {
        for (auto &e : g_prof.ev) FIC_TRY(cudaEventCreate(&e), "cudaEventCreate");
        g_prof.on = true;
    } else if (!on && g_prof.on) {
        for (auto &e : g_prof.ev) cudaEventDestroy(e);
        g_prof.on = false;
    }
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

size_t fic_decode_workspace_size(const fic_geom *gm, const fic_params *p, int32_t iters,
                                 int32_t ckpt_every) {
    Geo g;
    if (make_geo(gm, p, &g) != FIC_OK || iters < 0) return 0;
    const size_t img = (size_t)g.H * g.W;
    const int ck = ckpt_every < 1 ? 1 : ckpt_every;
    const int nseg = iters > 0 ? (iters + ck - 1) / ck : 1;
    Carver c(nullptr, (size_t)-1);
    c.take<float>(img);                       // decode ping-pong
    c.take<float>(img * (size_t)nseg);        // checkpoints
    c.take<float>(img * (size_t)(ck));        // segment iterates
    c.take<float>(2 * img);                   // adjoint vectors
    c.take<int32_t>(3 * (size_t)g.Dn + 1);    // CSR counts, offsets, cursors
    c.take<int32_t>(g.R);                     // CSR list
    c.take<double>(2 * (size_t)g.R);          // FP64 gradient accumulators
    return c.off + 256;
}

static fic_status check_codes(const fic_codes *c) {
    if (!c || !c->dom || !c->iso || !c->s || !c->o)
        return fail(FIC_ERR_INVALID_ARG, "null code pointer");
    return FIC_OK;
}

fic_status fic_decode(const fic_codes *codes, const fic_geom *gm, const fic_params *p,
                      int32_t iters, const float *x0, float *out, void *ws, size_t bytes,
                      void *stream) {
    Geo g;
    fic_status s = make_geo(gm, p, &g);
    if (s != FIC_OK) return s;
    if ((s = check_codes(codes)) != FIC_OK) return s;
    if (!out || iters < 0) return fail(FIC_ERR_INVALID_ARG, "null output or negative iters");
    if (!ws || (uintptr_t)ws % 256) return fail(FIC_ERR_WORKSPACE, "workspace null or misaligned");
    const size_t need = fic_decode_workspace_size(gm, p, iters, 1);
    const size_t img = (size_t)g.H * g.W;
    if (bytes < img * sizeof(float)) return fail(FIC_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, need);
    (void)need;
    cudaStream_t st = (cudaStream_t)stream;
    float *tmp = (float *)ws;
    if (iters == 0) {
        if (x0) FIC_TRY(cudaMemcpyAsync(out, x0, img * sizeof(float), cudaMemcpyDeviceToDevice, st), "copy");
        else FIC_TRY(launch_fill(out, img, 128.f, st), "fill");
        return FIC_OK;
    }
    // step k writes out when (iters-1-k) is even, tmp otherwise, so x_iters lands in out
    const float *cur = x0;
    if (!x0) {
        float *init = ((iters - 1) % 2 == 0) ? tmp : out;
        FIC_TRY(launch_fill(init, img, 128.f, st), "fill");
        cur = init;
    }
    for (int k = 0; k < iters; ++k) {
        float *dst = ((iters - 1 - k) % 2 == 0) ? out : tmp;
        FIC_TRY(launch_decode_step(*codes, g, cur, dst, st), "decode_step");
        cur = dst;
    }
    return FIC_OK;
}

fic_status fic_decode_backward(const fic_codes *codes, const fic_geom *gm, const fic_params *p,
                               int32_t iters, int32_t ckpt_every, const float *x0,
                               const float *grad_out, float *grad_s, float *grad_o, void *ws,
                               size_t bytes, void *stream) {
    Geo g;
    fic_status s = make_geo(gm, p, &g);
    if (s != FIC_OK) return s;
    if ((s = check_codes(codes)) != FIC_OK) return s;
    if (!grad_out || !grad_s || !grad_o || iters < 0 || ckpt_every < 1)
        return fail(FIC_ERR_INVALID_ARG, "null gradient pointer, iters < 0 or ckpt_every < 1");
    if (!ws || (uintptr_t)ws % 256) return fail(FIC_ERR_WORKSPACE, "workspace null or misaligned");
    const size_t need = fic_decode_workspace_size(gm, p, iters, ckpt_every);
    if (bytes < need) return fail(FIC_ERR_WORKSPACE, "workspace of %zu bytes, need %zu", bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t img = (size_t)g.H * g.W;
    const int ck = ckpt_every;
    const int nseg = iters > 0 ? (iters + ck - 1) / ck : 1;
    Carver c(ws, bytes);
    float *pingpong = c.take<float>(img);
    float *ckpt = c.take<float>(img * (size_t)nseg);
    float *seg = c.take<float>(img * (size_t)ck);
    float *lam = c.take<float>(2 * img);
    int32_t *cnt = c.take<int32_t>(g.Dn);
    int32_t *off = c.take<int32_t>(g.Dn + 1);
    int32_t *cursor = c.take<int32_t>(g.Dn);
    int32_t *list = c.take<int32_t>(g.R);
    double *g64 = c.take<double>(2 * (size_t)g.R);
    (void)pingpong;
    g_launches = 0;
    FIC_TRY(cudaMemsetAsync(g64, 0, sizeof(double) * 2 * g.R, st), "memset");
    if (iters == 0) {
        FIC_TRY(launch_grads_out(g.R, g64, g64 + g.R, grad_s, grad_o, st), "grads_out");
        return FIC_OK;
    }
    FIC_TRY(launch_dom_csr(g, codes->dom, cnt, off, cursor, list, st), "csr");
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
            FIC_TRY(launch_adjoint_grads(g, *codes, seg_ptr(c0, i), lcur, g64, g64 + g.R, st), "grads");
            if (c0 > 0 || i > 0) {
                FIC_TRY(launch_adjoint_gather(g, *codes, off, list, lcur, lprev, st), "gather");
                float *t = lcur;
                lcur = lprev;
                lprev = t;
            }
        }
    }
    FIC_TRY(launch_grads_out(g.R, g64, g64 + g.R, grad_s, grad_o, st), "grads_out");
    return FIC_OK;
}

}  // extern "C"
