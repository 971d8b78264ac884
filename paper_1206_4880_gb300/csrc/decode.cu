// Fractal decoding and its adjoint (Revathy & Jayamohan, Section 1: decoding iterates the stored
// maps starting from an initial image; the adjoint differentiates a fixed number of iterations
// with respect to the per-range contrast s and brightness o).
//
// One Jacobi step: x_{k+1}[p] = s_r * D(x_k, d_r)[src_{t_r}(p)] + o_r for every pixel p of range
// r, with D the 2x2 average of the 2B x 2B domain. Adjoint of the linear part W:
// (W^T l)[q] = sum over ranges r whose domain covers q of (s_r / 4) * l[p_r(q)], where p_r(q)
// is the range pixel whose source cell contains q. It is evaluated as a gather per pixel q over
// the (at most (2B/sigma)^2) domains covering q and, through a domain -> ranges CSR whose
// segments are sorted, over the ranges using each domain: no atomics, so the result does not
// depend on scheduling.
#include "fic_internal.cuh"

namespace fic {

__global__ void k_fill(float *x, size_t n, float v) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

cudaError_t launch_fill(float *x, size_t n, float v, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, n, v);
    ++g_launches;
    return cudaGetLastError();
}

// One warp per range r: the warp reads the 2B x 2B source domain of x_k, forms the B x B averages
// D(x_k, d_r) in shared memory, and writes the range's B x B pixels of x_{k+1},
// y[p] = s_r * D[src_t(p)] + o_r, two (B = 8) or four (B = 16) adjacent pixels per store.
// LD selects the source loads: 4 = 16-byte loads, each the top or bottom row of two adjacent 2x2
// cells (every domain starts at a column that is a multiple of 4 and the image is 16-byte
// aligned); 2 = aligned pairs, one row of one cell; 1 = single floats. VS: the output is aligned for
// the vector stores (else single stores). The isometry is affine in the pixel coordinates, so a
// warp forms src_t(py, px) = c0 + ky py + kx px from three warp-uniform constants. The sum order
// ((x00 + x01) + x10) + x11, the scaling by 1/4 and the fma are those of the per-pixel definition,
// so every variant gives the same bits.
constexpr int kDecodeWarps = 8;

template <int B, int LD, bool VS>
__global__ void __launch_bounds__(32 * kDecodeWarps)
    k_decode_step(Geo g, const int32_t *__restrict__ dom, const int32_t *__restrict__ iso,
                  const double *__restrict__ s, const double *__restrict__ o, const float *__restrict__ x,
                  float *__restrict__ y) {
    constexpr int NC = B * B / 32;     // cells (and output pixels) per lane
    constexpr int PV = B == 8 ? 2 : 4;  // pixels per vector store
    __shared__ __align__(16) float cell[kDecodeWarps][B * B];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kDecodeWarps + warp;
    if (r >= g.R) return;  // whole warps leave together; the block has no block-wide barrier
    const int d = __ldg(dom + r), t = __ldg(iso + r);
    const int rq = fdiv(r, g.fRx), dq = fdiv(d, g.fDx);
    float *dst = y + (size_t)(rq * B) * g.W + (r - rq * g.nRx) * B;
    if (!valid_code(g, d, t)) {  // an invalid code (an encode that gave up): NaN pixels, no read
#pragma unroll
        for (int k = 0; k < NC; ++k)
            dst[(size_t)((lane + 32 * k) / B) * g.W + (lane + 32 * k) % B] = __int_as_float(0x7fc00000);
        return;
    }
    const float sr = (float)__ldg(s + r), orr = (float)__ldg(o + r);
    const float *src = x + (size_t)(dq * g.sigma) * g.W + (d - dq * g.nDx) * g.sigma;
    float *cw = cell[warp];
    if constexpr (LD == 4) {
#pragma unroll
        for (int k = 0; k < NC / 2; ++k) {
            const int q = lane + 32 * k, cy = q / (B / 2), cp = q % (B / 2);  // cells (cy, 2cp), (cy, 2cp + 1)
            const float4 *p = reinterpret_cast<const float4 *>(src + (size_t)(2 * cy) * g.W + 4 * cp);
            const float4 a = __ldg(p), b = __ldg(reinterpret_cast<const float4 *>(reinterpret_cast<const float *>(p) + g.W));
            *reinterpret_cast<float2 *>(&cw[cy * B + 2 * cp]) =
                make_float2((((a.x + a.y) + b.x) + b.y) * 0.25f, (((a.z + a.w) + b.z) + b.w) * 0.25f);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const int c = lane + 32 * k, cy = c / B, cx = c % B;
            const float *p = src + (size_t)(2 * cy) * g.W + 2 * cx;
            float v;
            if (LD == 2) {
                const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
                const float2 b = __ldg(reinterpret_cast<const float2 *>(p + g.W));
                v = (((a.x + a.y) + b.x) + b.y) * 0.25f;
            } else {
                v = (((__ldg(p) + __ldg(p + 1)) + __ldg(p + g.W)) + __ldg(p + g.W + 1)) * 0.25f;
            }
            cw[c] = v;
        }
    }
    __syncwarp();
    // src_t(py, px) = sy B + sx with (sy, sx) from iso_src: affine in (py, px)
    constexpr int N = B - 1;
    const bool swap = (0xCA >> t) & 1, fy = (0xA6 >> t) & 1, fx = (0x9C >> t) & 1;
    const int sgy = fy ? -1 : 1, sgx = fx ? -1 : 1;
    const int c0 = (fy ? N * B : 0) + (fx ? N : 0);
    const int ky = swap ? sgx : sgy * B, kx = swap ? sgy * B : sgx;
#pragma unroll
    for (int k = 0; k < NC / PV; ++k) {
        const int p0 = PV * (lane + 32 * k), py = p0 / B, px = p0 % B;
        const int s0 = c0 + ky * py + kx * px;
        float v[PV];
#pragma unroll
        for (int i = 0; i < PV; ++i) v[i] = fmaf(sr, cw[s0 + i * kx], orr);
        float *q = dst + (size_t)py * g.W + px;
        if constexpr (VS && PV == 2) {
            *reinterpret_cast<float2 *>(q) = make_float2(v[0], v[1]);
        } else if constexpr (VS && PV == 4) {
            *reinterpret_cast<float4 *>(q) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int i = 0; i < PV; ++i) q[i] = v[i];
        }
    }
}

template <int B, int LD>
void decode_step_vs(bool vs, unsigned blocks, const Geo &g, const fic_codes &c, const float *x, float *y,
                    cudaStream_t st) {
    if (vs)
        k_decode_step<B, LD, true><<<blocks, 32 * kDecodeWarps, 0, st>>>(g, c.dom, c.iso, c.s, c.o, x, y);
    else
        k_decode_step<B, LD, false><<<blocks, 32 * kDecodeWarps, 0, st>>>(g, c.dom, c.iso, c.s, c.o, x, y);
}

template <int B>
void decode_step_b(int ld, bool vs, unsigned blocks, const Geo &g, const fic_codes &c, const float *x, float *y,
                   cudaStream_t st) {
    if (ld == 4)
        decode_step_vs<B, 4>(vs, blocks, g, c, x, y, st);
    else if (ld == 2)
        decode_step_vs<B, 2>(vs, blocks, g, c, x, y, st);
    else
        decode_step_vs<B, 1>(vs, blocks, g, c, x, y, st);
}

cudaError_t launch_decode_step(const fic_codes &c, const Geo &g, const float *x, float *y,
                               cudaStream_t st) {
    const unsigned blocks = (unsigned)((g.R + kDecodeWarps - 1) / kDecodeWarps);
    // W is a multiple of B, so every row starts at a multiple of 8 floats: domain columns that are
    // multiples of 4 (2) and a 16-byte (8-byte) aligned base keep every source vector aligned, and
    // range blocks start at multiples of B floats, so an output aligned to the store width keeps
    // every store aligned
    const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
    const int ld = (g.sigma % 4 == 0 && xa % 16 == 0) ? 4 : (g.sigma % 2 == 0 && xa % 8 == 0) ? 2 : 1;
    const bool vs = ya % (g.B == 16 ? 16 : 8) == 0;
    if (g.B == 16)
        decode_step_b<16>(ld, vs, blocks, g, c, x, y, st);
    else
        decode_step_b<8>(ld, vs, blocks, g, c, x, y, st);
    ++g_launches;
    return cudaGetLastError();
}

// Resolution-independent step (Section 1): the codes of an H x W encoding applied on the
// (zH) x (zW) grid; range r covers the (Bz)^2 block at z times its position, domain d the (2Bz)^2
// block at z times its position, contracted by 2x2 averaging, with the isometries of the
// (Bz) x (Bz) square. One thread per output pixel.
__global__ void k_decode_step_scaled(Geo g, int z, const int32_t *__restrict__ dom, const int32_t *__restrict__ iso,
                                     const double *__restrict__ s, const double *__restrict__ o,
                                     const float *__restrict__ x, float *__restrict__ y) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int Wz = g.W * z, Bz = g.B * z;
    if (idx >= (long long)g.H * z * Wz) return;
    const int py = (int)(idx / Wz), px = (int)(idx - (long long)py * Wz);
    const int r = (py / Bz) * g.nRx + px / Bz;
    const int d = dom[r], t = iso[r];
    if (!valid_code(g, d, t)) {  // an invalid code: NaN, no read
        y[idx] = __int_as_float(0x7fc00000);
        return;
    }
    int sy, sx;
    iso_src(Bz, t, py % Bz, px % Bz, sy, sx);
    const int qy = (d / g.nDx) * g.sigma * z + 2 * sy, qx = (d % g.nDx) * g.sigma * z + 2 * sx;
    const float *p = x + (size_t)qy * Wz + qx;
    const float v = (((p[0] + p[1]) + p[Wz]) + p[Wz + 1]) * 0.25f;
    y[idx] = fmaf((float)s[r], v, (float)o[r]);
}

cudaError_t launch_decode_step_scaled(const fic_codes &c, const Geo &g, int z, const float *x, float *y,
                                      cudaStream_t st) {
    const long long n = (long long)g.H * g.W * z * z;
    k_decode_step_scaled<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, z, c.dom, c.iso, c.s, c.o, x, y);
    ++g_launches;
    return cudaGetLastError();
}

// ---- adjoint -------------------------------------------------------------------------------
// domain -> ranges CSR: cnt[d] = #ranges using d with s != 0 (a range with s = 0 contributes
// nothing to W^T l, and flat ranges, which all take the pool's smallest domain id, would otherwise
// pile onto one domain); off = exclusive scan; list sorted per segment.
__global__ void k_dom_count(Geo g, const int32_t *__restrict__ dom, const double *__restrict__ s, int32_t *cnt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < g.R && s[r] != 0.0 && valid_code(g, dom[r], 0)) atomicAdd(&cnt[dom[r]], 1);
}

// Single-block exclusive scan of cnt[0..n) into off[0..n], chunk by chunk.
__global__ void k_scan_single(const int32_t *__restrict__ cnt, int n, int32_t *__restrict__ off,
                              int32_t *__restrict__ cursor) {
    __shared__ int buf[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < n ? cnt[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int s = 1; s < 1024; s <<= 1) {
            const int a = threadIdx.x >= s ? buf[threadIdx.x - s] : 0;
            __syncthreads();
            buf[threadIdx.x] += a;
            __syncthreads();
        }
        const int incl = buf[threadIdx.x];
        if (i < n) {
            off[i] = carry + incl - v;
            cursor[i] = carry + incl - v;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void k_dom_fill(Geo g, const int32_t *__restrict__ dom, const double *__restrict__ s, int32_t *cursor,
                           int32_t *__restrict__ list) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < g.R && s[r] != 0.0 && valid_code(g, dom[r], 0)) list[atomicAdd(&cursor[dom[r]], 1)] = r;
}

// Insertion-sort each domain's segment so the gather order is fixed.
__global__ void k_dom_sortseg(int Dn, const int32_t *__restrict__ off, int32_t *__restrict__ list) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= Dn) return;
    const int a = off[d], b = off[d + 1];
    for (int i = a + 1; i < b; ++i) {
        const int v = list[i];
        int j = i - 1;
        while (j >= a && list[j] > v) {
            list[j + 1] = list[j];
            --j;
        }
        list[j + 1] = v;
    }
}

// l_prev = W^T l, one thread per pixel q.
template <int B>
__global__ void k_adjoint_gather(Geo g, const int32_t *__restrict__ iso, const double *__restrict__ s,
                                 const int32_t *__restrict__ off, const int32_t *__restrict__ list,
                                 const float *__restrict__ lam, float *__restrict__ lam_prev) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.H * g.W) return;
    const int qy = idx / g.W, qx = idx - qy * g.W;
    // domains (dy, dx) on the stride grid with dy <= qy < dy + 2B, likewise x
    const int jy_hi = min(qy / g.sigma, g.nDy - 1), jx_hi = min(qx / g.sigma, g.nDx - 1);
    const int jy_lo = max(0, (qy - (2 * B - 1) + g.sigma - 1) / g.sigma);
    const int jx_lo = max(0, (qx - (2 * B - 1) + g.sigma - 1) / g.sigma);
    float acc = 0.f;
    for (int jy = jy_lo; jy <= jy_hi; ++jy) {
        const int dy = jy * g.sigma;
        const int cy = (qy - dy) >> 1;
        for (int jx = jx_lo; jx <= jx_hi; ++jx) {
            const int dx = jx * g.sigma;
            const int cx = (qx - dx) >> 1;
            const int d = jy * g.nDx + jx;
            for (int k = off[d]; k < off[d + 1]; ++k) {
                const int r = list[k];
                const int t = iso[r] & 7;  // listed ranges have a valid domain; a bad isometry
                                           // makes the range's own gradients NaN (k_adjoint_grads)
                // range pixel p with src_t(p) = (cy, cx): p = src_{t^-1}(cy, cx)
                const int tinv = (t == 1) ? 3 : (t == 3 ? 1 : t);
                int py, px;
                iso_src(B, tinv, cy, cx, py, px);
                const int rq = fdiv(r, g.fRx);
                const int ry = rq * B, rx = (r - rq * g.nRx) * B;
                acc = fmaf((float)s[r] * 0.25f, lam[(size_t)(ry + py) * g.W + rx + px], acc);
            }
        }
    }
    lam_prev[idx] = acc;
}

// grad_s[r] += sum_p l[p] * T(D x)[p], grad_o[r] += sum_p l[p]; one warp per range. The terms
// are formed in FP32 and summed in FP64 (the sums cancel heavily: terms of a few hundred add up
// to gradients of order one), into per-range FP64 accumulators.
template <int B>
__global__ void k_adjoint_grads(Geo g, const int32_t *__restrict__ dom, const int32_t *__restrict__ iso,
                                const float *__restrict__ x, const float *__restrict__ lam,
                                double *__restrict__ gs, double *__restrict__ go) {
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= g.R) return;
    const int d = dom[r], t = iso[r];
    if (!valid_code(g, d, t)) {  // an invalid code: NaN gradients, no read
        if (lane == 0) gs[r] = go[r] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const int rq = fdiv(r, g.fRx), dq = fdiv(d, g.fDx);
    const int ry = rq * B, rx = (r - rq * g.nRx) * B;
    const int dy = dq * g.sigma, dx = (d - dq * g.nDx) * g.sigma;
    double a_s = 0.0, a_o = 0.0;
#pragma unroll
    for (int h = 0; h < B * B / 32; ++h) {
        const int p = lane + 32 * h;
        const int y = p / B, xx = p % B;
        int sy, sx;
        iso_src(B, t, y, xx, sy, sx);
        const float *q = x + (size_t)(dy + 2 * sy) * g.W + dx + 2 * sx;
        const float v = (((q[0] + q[1]) + q[g.W]) + q[g.W + 1]) * 0.25f;
        const float l = lam[(size_t)(ry + y) * g.W + rx + xx];
        a_s += (double)l * (double)v;
        a_o += (double)l;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a_s += __shfl_xor_sync(0xffffffffu, a_s, off);
        a_o += __shfl_xor_sync(0xffffffffu, a_o, off);
    }
    if (lane == 0) {
        gs[r] += a_s;
        go[r] += a_o;
    }
}

__global__ void k_grads_out(int R, const double *__restrict__ gs64, const double *__restrict__ go64,
                            float *__restrict__ gs, float *__restrict__ go) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) {
        gs[r] = (float)gs64[r];
        go[r] = (float)go64[r];
    }
}

cudaError_t launch_dom_csr(const Geo &g, const int32_t *dom, const double *s, int32_t *cnt, int32_t *off,
                           int32_t *cursor, int32_t *list, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * g.Dn, st))) return e;
    k_dom_count<<<(g.R + 255) / 256, 256, 0, st>>>(g, dom, s, cnt);
    ++g_launches;
    k_scan_single<<<1, 1024, 0, st>>>(cnt, g.Dn, off, cursor);
    ++g_launches;
    k_dom_fill<<<(g.R + 255) / 256, 256, 0, st>>>(g, dom, s, cursor, list);
    ++g_launches;
    k_dom_sortseg<<<(g.Dn + 255) / 256, 256, 0, st>>>(g.Dn, off, list);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_gather(const Geo &g, const fic_codes &c, const int32_t *off,
                                  const int32_t *list, const float *lam, float *lam_prev,
                                  cudaStream_t st) {
    const int n = g.H * g.W;
    if (g.B == 16)
        k_adjoint_gather<16><<<(n + 255) / 256, 256, 0, st>>>(g, c.iso, c.s, off, list, lam, lam_prev);
    else
        k_adjoint_gather<8><<<(n + 255) / 256, 256, 0, st>>>(g, c.iso, c.s, off, list, lam, lam_prev);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_adjoint_grads(const Geo &g, const fic_codes &c, const float *x, const float *lam,
                                 double *gs, double *go, cudaStream_t st) {
    const long long threads = (long long)g.R * 32;
    if (g.B == 16)
        k_adjoint_grads<16><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, c.dom, c.iso, x, lam, gs, go);
    else
        k_adjoint_grads<8><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(g, c.dom, c.iso, x, lam, gs, go);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_grads_out(int R, const double *gs64, const double *go64, float *gs, float *go,
                             cudaStream_t st) {
    k_grads_out<<<(R + 255) / 256, 256, 0, st>>>(R, gs64, go64, gs, go);
    ++g_launches;
    return cudaGetLastError();
}

// ---- quality (PSNR) --------------------------------------------------------------------------
constexpr int kQualBlocks = 1024;

__global__ void k_sqerr_partial(const float *__restrict__ x, const uint8_t *__restrict__ ref, int H, int W,
                                int pitch, double *__restrict__ partial) {
    __shared__ double red[256];
    double acc = 0.0;
    const long long n = (long long)H * W;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int py = (int)(i / W), px = (int)(i - (long long)py * W);
        const float q = fminf(fmaxf(rintf(x[i]), 0.f), 255.f);
        const double e = (double)q - (double)ref[(size_t)py * pitch + px];
        acc += e * e;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sqerr_final(const double *__restrict__ partial, int nb, long long n, double *out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mse = red[0] / (double)n;
        out[0] = mse;
        out[1] = mse > 0.0 ? 10.0 * log10(255.0 * 255.0 / mse) : __longlong_as_double(0x7ff0000000000000LL);
    }
}

cudaError_t launch_quality(const float *x, const uint8_t *ref, int H, int W, int pitch, double *out,
                           cudaStream_t st) {
    k_sqerr_partial<<<kQualBlocks, 256, 0, st>>>(x, ref, H, W, pitch, out + 2);
    ++g_launches;
    k_sqerr_final<<<1, 256, 0, st>>>(out + 2, kQualBlocks, (long long)H * W, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
