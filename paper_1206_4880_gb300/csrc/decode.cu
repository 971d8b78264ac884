// Fractal decoding and its adjoint (Revathy & Jayamohan, Section 1: decoding iterates the stored
// maps starting from an initial image; the adjoint differentiates a fixed number of iterations
// with respect to the per-range contrast s and brightness o).
//
// One Jacobi step: x_{k+1}[p] = s_r * D(x_k, d_r)[src_{t_r}(p)] + o_r for every pixel p of range
// r, with D the 2x2 average of the 2B x 2B domain. Adjoint of the linear part W:
// (W^T l)[q] = sum over ranges r whose domain covers q of (s_r / 4) * l[p_r(q)], where p_r(q)
// is the range pixel whose source cell contains q. It is formed per domain (the sum over the
// domain's ranges, in increasing id, for each of its cells) and then per pixel (the sum over the
// at most (2B/sigma)^2 domains covering it, in row-major order): no atomics, so the result does not
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

// The B x B 2x2 averages of the 2B x 2B block at src (row stride W) into cw (shared memory), by the
// lanes of one warp. LD = 4: 16-byte loads, each the top or bottom row of two adjacent cells (src
// and W keep every vector 16-byte aligned); 2: aligned pairs; 1: single floats. The sum order
// ((x00 + x01) + x10) + x11 and the scaling by 1/4 are the same in every form.
template <int B, int LD>
__device__ __forceinline__ void load_cells(const float *__restrict__ src, int W, int lane, float *cw) {
    constexpr int NC = B * B / 32;
    if constexpr (LD == 4) {
#pragma unroll
        for (int k = 0; k < NC / 2; ++k) {
            const int q = lane + 32 * k, cy = q / (B / 2), cp = q % (B / 2);  // cells (cy, 2cp), (cy, 2cp + 1)
            const float *p = src + (size_t)(2 * cy) * W + 4 * cp;
            const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
            const float4 b = __ldg(reinterpret_cast<const float4 *>(p + W));
            *reinterpret_cast<float2 *>(&cw[cy * B + 2 * cp]) =
                make_float2((((a.x + a.y) + b.x) + b.y) * 0.25f, (((a.z + a.w) + b.z) + b.w) * 0.25f);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const int c = lane + 32 * k, cy = c / B, cx = c % B;
            const float *p = src + (size_t)(2 * cy) * W + 2 * cx;
            float v;
            if constexpr (LD == 2) {
                const float2 a = __ldg(reinterpret_cast<const float2 *>(p));
                const float2 b = __ldg(reinterpret_cast<const float2 *>(p + W));
                v = (((a.x + a.y) + b.x) + b.y) * 0.25f;
            } else {
                v = (((__ldg(p) + __ldg(p + 1)) + __ldg(p + W)) + __ldg(p + W + 1)) * 0.25f;
            }
            cw[c] = v;
        }
    }
}

// Warp-uniform constants of src_t(py, px) = c0 + ky py + kx px, the index of the source cell of
// pixel (py, px) under isometry t (iso_src, which is affine in the pixel coordinates).
template <int B>
__device__ __forceinline__ void iso_affine(int t, int &c0, int &ky, int &kx) {
    constexpr int N = B - 1;
    const bool swap = (0xCA >> t) & 1, fy = (0xA6 >> t) & 1, fx = (0x9C >> t) & 1;
    const int sgy = fy ? -1 : 1, sgx = fx ? -1 : 1;
    c0 = (fy ? N * B : 0) + (fx ? N : 0);
    ky = swap ? sgx : sgy * B;
    kx = swap ? sgy * B : sgx;
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
    load_cells<B, LD>(src, g.W, lane, cw);
    __syncwarp();
    int c0, ky, kx;
    iso_affine<B>(t, c0, ky, kx);
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

// The same step for 8x8 ranges with 16-byte source loads: one half-warp per NR ranges (ranges
// hw, hw + 16, ... of the block's 16 NR), with every range's code and source rows loaded before
// any is used, so one warp's instructions keep 2 NR ranges' loads in flight. Lane hl of a half
// loads the top and bottom rows of cell pairs hl and hl + 16 (cell rows hl / 4 and hl / 4 + 4) of
// each range and writes four adjacent pixels of each.
constexpr int kDecodeNR = 1;  // measured at 4096^2: 1 -> 0.376 ms, 2 -> 0.423 ms (44 registers, fewer warps)

template <bool VS>
__global__ void __launch_bounds__(32 * kDecodeWarps)
    k_decode_step8h(Geo g, const int32_t *__restrict__ dom, const int32_t *__restrict__ iso,
                    const double *__restrict__ s, const double *__restrict__ o, const float *__restrict__ x,
                    float *__restrict__ y) {
    constexpr int NR = kDecodeNR, HW = 2 * kDecodeWarps;
    __shared__ __align__(16) float cell[HW][NR][64];
    const int hw = threadIdx.x >> 4, hl = threadIdx.x & 15;
    const unsigned hmask = 0xFFFFu << (threadIdx.x & 16);  // this half-warp
    int r[NR], d[NR], t[NR];
    bool use[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        r[k] = blockIdx.x * (HW * NR) + k * HW + hw;
        d[k] = t[k] = 0;
        use[k] = false;
        if (r[k] < g.R) {
            d[k] = __ldg(dom + r[k]);
            t[k] = __ldg(iso + r[k]);
            use[k] = valid_code(g, d[k], t[k]);
        }
    }
    float4 a[NR][2], b[NR][2];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (!use[k]) continue;
        const int dq = fdiv(d[k], g.fDx);
        const float *src = x + (size_t)(dq * g.sigma) * g.W + (d[k] - dq * g.nDx) * g.sigma;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = hl + 16 * h, cy = q >> 2, cp = q & 3;  // cells (cy, 2cp), (cy, 2cp + 1)
            const float *p = src + (size_t)(2 * cy) * g.W + 4 * cp;
            a[k][h] = __ldg(reinterpret_cast<const float4 *>(p));
            b[k][h] = __ldg(reinterpret_cast<const float4 *>(p + g.W));
        }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (!use[k]) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = hl + 16 * h, cy = q >> 2, cp = q & 3;
            *reinterpret_cast<float2 *>(&cell[hw][k][cy * 8 + 2 * cp]) =
                make_float2((((a[k][h].x + a[k][h].y) + b[k][h].x) + b[k][h].y) * 0.25f,
                            (((a[k][h].z + a[k][h].w) + b[k][h].z) + b[k][h].w) * 0.25f);
        }
    }
    __syncwarp(hmask);
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (r[k] >= g.R) continue;
        const int rq = fdiv(r[k], g.fRx);
        const int py = hl >> 1, px = 4 * (hl & 1);
        float *q = y + (size_t)(rq * 8 + py) * g.W + (r[k] - rq * g.nRx) * 8 + px;
        float v[4];
        if (use[k]) {
            const float sr = (float)__ldg(s + r[k]), orr = (float)__ldg(o + r[k]);
            int c0, ky, kx;
            iso_affine<8>(t[k], c0, ky, kx);
            const int s0 = c0 + ky * py + kx * px;
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = fmaf(sr, cell[hw][k][s0 + i * kx], orr);
        } else {  // an invalid code (an encode that gave up): NaN pixels, no read
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = __int_as_float(0x7fc00000);
        }
        if constexpr (VS) {
            *reinterpret_cast<float4 *>(q) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) q[i] = v[i];
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
    if (g.B == 16) {
        decode_step_b<16>(ld, vs, blocks, g, c, x, y, st);
    } else if (ld == 4) {
        const unsigned hblocks = (unsigned)((g.R + 2 * kDecodeWarps * kDecodeNR - 1) / (2 * kDecodeWarps * kDecodeNR));
        if (ya % 16 == 0)
            k_decode_step8h<true><<<hblocks, 32 * kDecodeWarps, 0, st>>>(g, c.dom, c.iso, c.s, c.o, x, y);
        else
            k_decode_step8h<false><<<hblocks, 32 * kDecodeWarps, 0, st>>>(g, c.dom, c.iso, c.s, c.o, x, y);
    } else {
        decode_step_b<8>(ld, vs, blocks, g, c, x, y, st);
    }
    ++g_launches;
    return cudaGetLastError();
}

// ---- iterating on the plane of 2x2 averages --------------------------------------------------
// With an even stride every domain starts at even coordinates, so its contracted block D(x_k, d)
// is the B x B window at (dy / 2, dx / 2) of the plane P_k of 2x2 averages of x_k
// (P_k[i][j] = the mean of x_k over rows 2i, 2i + 1 and columns 2j, 2j + 1). x_{k+1} depends on
// x_k only through P_k, and the 2x2 averages of a range's pixels at step k + 1 are
//   P_{k+1}[cell (u, v) of r] = s_r E[src'_t(u, v)] + o_r,
// E the 2x2 averages of r's window of P_k and src' the isometry of the (B/2)-square: an isometry
// of the B-square maps aligned 2x2 pixel blocks onto aligned 2x2 cell blocks, and averaging
// commutes with the map's affine part. So the iteration runs on P (a quarter of the pixels; the
// two planes stay in L2 up to 4096 x 4096 images) and only the last step writes x:
//   x_K[p] = s_r P_{K-1}[(dy / 2, dx / 2) + src_t(p)] + o_r.
// In exact arithmetic this is the Jacobi iteration of the maps; in FP32 it rounds in another order
// (s times the mean of four cells plus o, where the full-resolution steps average four results of
// s times a cell plus o). With one step it is the full-resolution step bit for bit: the first
// plane holds the same averages, summed in the same order.
constexpr int kHalfThreads = 128;

// P = the 2x2 averages of x (H x W, row stride W), two outputs per thread. V4: x is 16-byte
// aligned, so each pair's two source rows are two float4 loads; else single floats, same sums.
template <bool V4>
__global__ void __launch_bounds__(kHalfThreads) k_pool2(const float *__restrict__ x, int W, float *__restrict__ P) {
    const int Wh = W / 2, i = blockIdx.y, j = 2 * (blockIdx.x * kHalfThreads + threadIdx.x);
    if (j >= Wh) return;  // Wh is a multiple of 4 (W is a multiple of B >= 8), so j + 1 < Wh
    const float *a = x + (size_t)(2 * i) * W + 2 * j;
    float v0, v1;
    if constexpr (V4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(a));
        const float4 b = __ldg(reinterpret_cast<const float4 *>(a + W));
        v0 = (((t.x + t.y) + b.x) + b.y) * 0.25f;
        v1 = (((t.z + t.w) + b.z) + b.w) * 0.25f;
    } else {
        v0 = (((__ldg(a) + __ldg(a + 1)) + __ldg(a + W)) + __ldg(a + W + 1)) * 0.25f;
        v1 = (((__ldg(a + 2) + __ldg(a + 3)) + __ldg(a + W + 2)) + __ldg(a + W + 3)) * 0.25f;
    }
    *reinterpret_cast<float2 *>(P + (size_t)i * Wh + j) = make_float2(v0, v1);
}

// Each code once per decoding call, for the steps on the plane: (offset of the range's B x B window
// in P, or -1 for an invalid code; isometry; s and o rounded to FP32 bits). The steps then read one
// 16-byte record per range and convert nothing: an FP64 -> FP32 conversion runs on the FP64 pipe,
// a small fraction of the FP32 rate on this part, and every lane converting its range's
// coefficients at every step had been a large share of a step's time.
__global__ void k_pack_codes(Geo g, const int32_t *__restrict__ dom, const int32_t *__restrict__ iso,
                             const double *__restrict__ s, const double *__restrict__ o, int4 *__restrict__ pk) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.R) return;
    const int d = dom[r], t = iso[r];
    if (!valid_code(g, d, t)) {
        pk[r] = make_int4(-1, 0, 0, 0);
        return;
    }
    const int dq = fdiv(d, g.fDx);
    const int off = ((dq * g.sigma) / 2) * (g.W / 2) + ((d - dq * g.nDx) * g.sigma) / 2;
    pk[r] = make_int4(off, t, __float_as_int((float)s[r]), __float_as_int((float)o[r]));
}

template <int B>
struct PlaneShape {
    static constexpr int T = B == 8 ? 16 : 32;  // threads per range
    static constexpr int G = 256 / T;           // groups per block
    static constexpr int NR = B == 8 ? 4 : 2;   // ranges per group
};

// One step on the plane, by a group of T threads per NR ranges (T = 16 for B = 8, a warp for
// B = 16; in each of the NR rounds consecutive groups take consecutive ranges, so a warp's stores
// cover adjacent ranges of one range row); every range's record and source loads are issued before
// any is used. Lane l of a group forms the cells c = l + T j of the range's (B/2) x (B/2) grid of
// 2x2 means E of its window, row-major (each from two aligned float2 loads when V2 — the stride is
// a multiple of 4, so every window column is even — else four single loads; the lanes of one cell
// row read one contiguous run), summed ((w00 + w01) + w10) + w11 and scaled by 1/4, then writes
// the cells (u, v) = c of P_{k+1}: s * E[src'_t(u, v)] + o, taking E[src'] from the lane that
// formed it by a warp shuffle. C0: the plane is 128 everywhere (the mid-grey start, whose 2x2
// means are 128 exactly), so nothing is read.
template <int B, bool V2, bool C0>
__global__ void __launch_bounds__(256)
    k_plane_half(Geo g, const int4 *__restrict__ pk, const float *__restrict__ P, float *__restrict__ y) {
    constexpr int T = PlaneShape<B>::T, G = PlaneShape<B>::G, NR = PlaneShape<B>::NR;
    constexpr int OB = B / 2, J = OB * OB / T;  // cells per lane: 1 (B = 8), 2 (B = 16)
    const int grp = threadIdx.x / T, l = threadIdx.x % T, gbase = (threadIdx.x & 31) & ~(T - 1);
    const unsigned gmask = T == 32 ? 0xffffffffu : (0xFFFFu << (threadIdx.x & 16));
    const int Wh = g.W / 2;
    int r[NR];
    int4 c[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        r[k] = (blockIdx.x * NR + k) * G + grp;
        c[k] = r[k] < g.R ? __ldg(pk + r[k]) : make_int4(-1, 0, 0, 0);
    }
    float e[NR][J];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
#pragma unroll
        for (int j = 0; j < J; ++j) e[k][j] = 128.f;
        if (C0 || c[k].x < 0) continue;  // an invalid code (an encode that gave up): no read
        const float *w = P + c[k].x;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = l + T * j, cy = q / OB, cx = q % OB;
            const float *p = w + (size_t)(2 * cy) * Wh + 2 * cx;
            if constexpr (V2) {
                const float2 lo = __ldg(reinterpret_cast<const float2 *>(p));
                const float2 hi = __ldg(reinterpret_cast<const float2 *>(p + Wh));
                e[k][j] = (((lo.x + lo.y) + hi.x) + hi.y) * 0.25f;
            } else {
                e[k][j] = (((__ldg(p) + __ldg(p + 1)) + __ldg(p + Wh)) + __ldg(p + Wh + 1)) * 0.25f;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const bool live = r[k] < g.R;
        const int rq = live ? fdiv(r[k], g.fRx) : 0;
        float *dst = y + (size_t)(rq * OB) * Wh + (r[k] - rq * g.nRx) * OB;
        const float sr = __int_as_float(c[k].z), orr = __int_as_float(c[k].w);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = l + T * j, u = q / OB, v = q % OB;
            int sy, sx;
            iso_src(OB, c[k].y, u, v, sy, sx);
            const int src = sy * OB + sx;  // the cell to take: lane src % T, register src / T
            float val = __shfl_sync(gmask, e[k][0], gbase + src % T);
            if constexpr (J == 2) {
                const float hi = __shfl_sync(gmask, e[k][1], gbase + src % T);
                val = src >= T ? hi : val;
            }
            if (live) dst[(size_t)u * Wh + v] = c[k].x >= 0 ? fmaf(sr, val, orr) : __int_as_float(0x7fc00000);
        }
    }
}

// The last step: the B x B pixels of x_K, s * window[src_t(py, px)] + o, by the same groups; the
// group copies each range's window into shared memory (float2 loads when V2), then every lane
// writes B * B / T pixels (eight adjacent lanes cover 32 contiguous bytes of a pixel row).
template <int B, bool V2, bool C0>
__global__ void __launch_bounds__(256)
    k_plane_final(Geo g, const int4 *__restrict__ pk, const float *__restrict__ P, float *__restrict__ y) {
    constexpr int T = PlaneShape<B>::T, G = PlaneShape<B>::G, NR = PlaneShape<B>::NR;
    __shared__ __align__(16) float win[G][NR][B * B];
    const int grp = threadIdx.x / T, l = threadIdx.x % T;
    const unsigned gmask = T == 32 ? 0xffffffffu : (0xFFFFu << (threadIdx.x & 16));
    const int Wh = g.W / 2;
    int r[NR];
    int4 c[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        r[k] = (blockIdx.x * NR + k) * G + grp;
        c[k] = r[k] < g.R ? __ldg(pk + r[k]) : make_int4(-1, 0, 0, 0);
    }
    if constexpr (!C0) {
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            if (c[k].x < 0) continue;  // an invalid code: no read
            const float *w = P + c[k].x;
            float *wn = win[grp][k];
            if constexpr (V2) {
#pragma unroll
                for (int q = l; q < B * B / 2; q += T) {
                    const int row = q / (B / 2), c2 = q % (B / 2);
                    *reinterpret_cast<float2 *>(&wn[row * B + 2 * c2]) =
                        __ldg(reinterpret_cast<const float2 *>(w + (size_t)row * Wh + 2 * c2));
                }
            } else {
#pragma unroll
                for (int q = l; q < B * B; q += T) wn[q] = __ldg(w + (size_t)(q / B) * Wh + q % B);
            }
        }
        __syncwarp(gmask);
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        if (r[k] >= g.R) continue;
        const int rq = fdiv(r[k], g.fRx);
        float *dst = y + (size_t)(rq * B) * g.W + (r[k] - rq * g.nRx) * B;
        const float sr = __int_as_float(c[k].z), orr = __int_as_float(c[k].w);
        const float *wn = win[grp][k];
#pragma unroll
        for (int q = l; q < B * B; q += T) {
            const int u = q / B, v = q % B;
            float val = __int_as_float(0x7fc00000);  // an invalid code: NaN pixels
            if (c[k].x >= 0) {
                int sy, sx;
                iso_src(B, c[k].y, u, v, sy, sx);
                val = fmaf(sr, C0 ? 128.f : wn[sy * B + sx], orr);
            }
            dst[(size_t)u * g.W + v] = val;
        }
    }
}

template <int B, bool FINAL>
void launch_plane_step(bool v2, bool c0, const Geo &g, const int4 *pk, const float *P, float *y, cudaStream_t st) {
    constexpr int per_block = PlaneShape<B>::G * PlaneShape<B>::NR;
    const unsigned blocks = (unsigned)((g.R + per_block - 1) / per_block);
    if constexpr (!FINAL) {
        if (c0) k_plane_half<B, false, true><<<blocks, 256, 0, st>>>(g, pk, P, y);
        else if (v2) k_plane_half<B, true, false><<<blocks, 256, 0, st>>>(g, pk, P, y);
        else k_plane_half<B, false, false><<<blocks, 256, 0, st>>>(g, pk, P, y);
    } else {
        if (c0) k_plane_final<B, false, true><<<blocks, 256, 0, st>>>(g, pk, P, y);
        else if (v2) k_plane_final<B, true, false><<<blocks, 256, 0, st>>>(g, pk, P, y);
        else k_plane_final<B, false, false><<<blocks, 256, 0, st>>>(g, pk, P, y);
    }
}

bool decode_on_plane(const Geo &g) { return g.sigma % 2 == 0 && g.H <= 65535; }

cudaError_t launch_decode_iterate(const fic_codes &c, const Geo &g, int iters, const float *x0, float *out,
                                  float *tmp, cudaStream_t st) {
    const size_t img = (size_t)g.H * g.W;
    if (iters <= 0) return cudaErrorInvalidValue;
    if (!decode_on_plane(g)) {
        // odd strides: full-resolution steps, ping-pong between out and tmp ending in out
        const float *cur = x0;
        cudaError_t e = cudaSuccess;
        if (!x0) {
            float *init = ((iters - 1) % 2 == 0) ? tmp : out;
            e = launch_fill(init, img, 128.f, st);
            cur = init;
        }
        for (int k = 0; k < iters && e == cudaSuccess; ++k) {
            float *dst = ((iters - 1 - k) % 2 == 0) ? out : tmp;
            e = launch_decode_step(c, g, cur, dst, st);
            cur = dst;
        }
        return e;
    }
    // two planes of img / 4 floats in tmp (offset img bytes: a multiple of 256), then the packed
    // codes (R int4 <= img / 16 floats); with no x0 the first step reads the constant start
    // instead of a plane
    const int Wh = g.W / 2, Hh = g.H / 2;
    float *pa = tmp, *pb = tmp + img / 4;
    int4 *pk = reinterpret_cast<int4 *>(tmp + img / 2);
    k_pack_codes<<<(unsigned)((g.R + 255) / 256), 256, 0, st>>>(g, c.dom, c.iso, c.s, c.o, pk);
    ++g_launches;
    cudaError_t e = cudaGetLastError();
    if (x0 && e == cudaSuccess) {
        const dim3 grid((unsigned)((Wh / 2 + kHalfThreads - 1) / kHalfThreads), (unsigned)Hh);
        if ((uintptr_t)x0 % 16 == 0)
            k_pool2<true><<<grid, kHalfThreads, 0, st>>>(x0, g.W, pa);
        else
            k_pool2<false><<<grid, kHalfThreads, 0, st>>>(x0, g.W, pa);
        ++g_launches;
        e = cudaGetLastError();
    }
    const bool v2 = g.sigma % 4 == 0;
    bool c0 = !x0;
    for (int k = 1; k < iters && e == cudaSuccess; ++k, c0 = false) {
        if (g.B == 16) launch_plane_step<16, false>(v2, c0, g, pk, pa, pb, st);
        else launch_plane_step<8, false>(v2, c0, g, pk, pa, pb, st);
        ++g_launches;
        e = cudaGetLastError();
        float *t = pa;
        pa = pb;
        pb = t;
    }
    if (e != cudaSuccess) return e;
    if (g.B == 16) launch_plane_step<16, true>(v2, c0, g, pk, pa, out, st);
    else launch_plane_step<8, true>(v2, c0, g, pk, pa, out, st);
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
// W^T l (the adjoint of the linear part of one step) in two deterministic phases over the
// domain -> ranges index of the ranges that contribute (s != 0 and a valid code: a range with
// s = 0 contributes nothing, and flat ranges, which all take their pool's smallest domain, would
// otherwise pile onto a few domains):
//   cells: per listed range r (one warp each), its B x B cell block C_r[c] = (s_r / 4) l[p_r(c)],
//          p_r(c) the pixel of range r whose source cell under t_r is c, stored at r's list position;
//   pixels: (W^T l)[q] = sum over the domains d covering q, in row-major order, and over d's ranges
//          in increasing id, of C_r[cell of q in d].
// With an even stride every covering domain's cells are aligned 2x2 pixel blocks, so the sum is
// the same for the four pixels of each aligned 2x2 block and is formed once per block.
// The index is list = the range ids stably sorted by domain (a byte-wise radix sort) with
// off[d] = the first position of a domain >= d (off[Dn] = the number of listed ranges).
__global__ void k_csr_keys(Geo g, const int32_t *__restrict__ dom, const int32_t *__restrict__ iso,
                           const double *__restrict__ s, int32_t *__restrict__ key) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < g.R) key[r] = (s[r] != 0.0 && valid_code(g, dom[r], iso[r])) ? dom[r] : g.Dn;
}

// The sorted keys (for the segment starts) and, per list position, the range's packed entry
// (id, isometry, s / 4) that the cells phase reads at every step.
__global__ void k_csr_sorted_keys(int n, const int32_t *__restrict__ key, const int32_t *__restrict__ list,
                                  const int32_t *__restrict__ iso, const double *__restrict__ s,
                                  int32_t *__restrict__ skey, int4 *__restrict__ ent) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int r = list[j];
    skey[j] = key[r];
    ent[j] = make_int4(r, iso[r] & 7, __float_as_int((float)s[r] * 0.25f), 0);
}

// off[d] = the number of sorted keys below d, for d = 0 .. Dn (binary search).
__global__ void k_csr_offsets(int n, int Dn, const int32_t *__restrict__ skey, int32_t *__restrict__ off) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d > Dn) return;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (skey[mid] < d)
            lo = mid + 1;
        else
            hi = mid;
    }
    off[d] = lo;
}

// Phase "cells": one warp per listed range (B = 4: one half-warp). MUL = 4 gives s_r l[p_r(c)]
// (the transpose of a map without the 2x2 averaging: the packed entry holds s_r / 4, and the
// product by 4 is exact).
template <int B, int MUL = 1>
__global__ void __launch_bounds__(256)
    k_adjoint_cells(Geo g, const int4 *__restrict__ ent, const int32_t *__restrict__ off,
                    const float *__restrict__ lam, float *__restrict__ acc) {
    constexpr int LPR = B * B >= 32 ? 32 : B * B;  // lanes per range
    constexpr int NC = B * B / LPR;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = tid / LPR, lane = tid % LPR;
    if (k >= g.R) return;
    const int n = __ldg(off + g.Dn);  // listed ranges (the rest of the list holds the others)
    const int4 e = __ldg(ent + k);
    if (k >= n) return;
    const int r = e.x, t = e.y;
    const float sc = __int_as_float(e.z) * (float)MUL;
    const int rq = fdiv(r, g.fRx);
    const float *lr = lam + (size_t)(rq * B) * g.W + (r - rq * g.nRx) * B;
    // the pixel p with src_t(p) = c is p = src_{t^-1}(c)
    int c0, ky, kx;
    iso_affine<B>(t == 1 ? 3 : (t == 3 ? 1 : t), c0, ky, kx);
    float *dst = acc + (size_t)k * (B * B);
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const int c = lane + LPR * m, p = c0 + ky * (c / B) + kx * (c % B);
        dst[c] = sc * __ldg(lr + (size_t)(p / B) * g.W + p % B);
    }
}

// The sum of phase "pixels" for pixel (qy, qx) over the domains (jy, jx) covering it, row-major,
// and each domain's ranges in list order. MJ > 0: at most MJ domains cover a coordinate per axis,
// and every covering domain's segment bounds are loaded before any cell; MJ = 0: any number.
// WIN: the domains are windows of side 2B whose cells are single pixels (2B x 2B cells per range,
// cell (qy - jy sigma, qx - jx sigma)), the transpose of a map without the 2x2 averaging.
template <int B, int MJ, bool WIN = false>
__device__ __forceinline__ float adjoint_sum(const Geo &g, const int32_t *__restrict__ off,
                                             const float *__restrict__ acc, int jy_lo, int jy_hi, int jx_lo,
                                             int jx_hi, int qy, int qx) {
    constexpr int CB = WIN ? 2 * B : B;  // cells per side of a domain's block
    constexpr int SH = WIN ? 0 : 1;
    float a = 0.f;
    if constexpr (MJ > 0) {
        int o0[MJ * MJ], o1[MJ * MJ];
#pragma unroll
        for (int u = 0; u < MJ; ++u)
#pragma unroll
            for (int v = 0; v < MJ; ++v) {
                const bool in = jy_lo + u <= jy_hi && jx_lo + v <= jx_hi;
                const int d = (jy_lo + u) * g.nDx + jx_lo + v;
                o0[u * MJ + v] = in ? __ldg(off + d) : 0;
                o1[u * MJ + v] = in ? __ldg(off + d + 1) : 0;
            }
#pragma unroll
        for (int u = 0; u < MJ; ++u)
#pragma unroll
            for (int v = 0; v < MJ; ++v) {
                const float *cp = acc + ((qy - (jy_lo + u) * g.sigma) >> SH) * CB + ((qx - (jx_lo + v) * g.sigma) >> SH);
                for (int k = o0[u * MJ + v]; k < o1[u * MJ + v]; ++k) a += __ldg(cp + (size_t)k * (CB * CB));
            }
        return a;
    } else {
        for (int jy = jy_lo; jy <= jy_hi; ++jy) {
            const int cy = (qy - jy * g.sigma) >> SH;
            for (int jx = jx_lo; jx <= jx_hi; ++jx) {
                const int d = jy * g.nDx + jx;
                const int o1 = __ldg(off + d + 1);
                const float *cp = acc + cy * CB + ((qx - jx * g.sigma) >> SH);
                for (int k = __ldg(off + d); k < o1; ++k) a += __ldg(cp + (size_t)k * (CB * CB));
            }
        }
        return a;
    }
}

// First and last domain index along one axis covering coordinate q (domains at j * sigma span
// 2B pixels).
template <int B>
__device__ __forceinline__ void covering(const Geo &g, int q, int n, int &lo, int &hi) {
    hi = min(fdiv(q, g.fS), n - 1);
    const int num = q - (2 * B - 1) + g.sigma - 1;
    lo = num > 0 ? fdiv(num, g.fS) : 0;
}

// Phase "pixels", odd stride: l_prev = W^T l, one thread per pixel, blockIdx.y striding over rows.
template <int B, int MJ, bool WIN = false>
__global__ void __launch_bounds__(256)
    k_adjoint_gather(Geo g, const int32_t *__restrict__ off, const float *__restrict__ acc,
                     float *__restrict__ lam_prev) {
    const int qx = blockIdx.x * blockDim.x + threadIdx.x;
    if (qx >= g.W) return;
    int jx_lo, jx_hi;
    covering<B>(g, qx, g.nDx, jx_lo, jx_hi);
    for (int qy = blockIdx.y; qy < g.H; qy += gridDim.y) {
        int jy_lo, jy_hi;
        covering<B>(g, qy, g.nDy, jy_lo, jy_hi);
        lam_prev[(size_t)qy * g.W + qx] = adjoint_sum<B, MJ, WIN>(g, off, acc, jy_lo, jy_hi, jx_lo, jx_hi, qy, qx);
    }
}

// Phase "pixels", even stride: one thread per aligned 2x2 pixel block (bx, by), whose four pixels
// lie in the same cell of every covering domain and receive the same sum.
template <int B, int MJ>
__global__ void __launch_bounds__(256)
    k_adjoint_gather2(Geo g, const int32_t *__restrict__ off, const float *__restrict__ acc,
                      float *__restrict__ lam_prev) {
    const int bx = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * bx >= g.W) return;
    const int qx = 2 * bx;
    int jx_lo, jx_hi;
    covering<B>(g, qx, g.nDx, jx_lo, jx_hi);
    for (int by = blockIdx.y; 2 * by < g.H; by += gridDim.y) {
        const int qy = 2 * by;
        int jy_lo, jy_hi;
        covering<B>(g, qy, g.nDy, jy_lo, jy_hi);
        const float a = adjoint_sum<B, MJ>(g, off, acc, jy_lo, jy_hi, jx_lo, jx_hi, qy, qx);
        float *q = lam_prev + (size_t)qy * g.W + qx;
        *reinterpret_cast<float2 *>(q) = make_float2(a, a);
        *reinterpret_cast<float2 *>(q + g.W) = make_float2(a, a);
    }
}

// Float-float accumulation: hi + lo carries the running sum with about 44 significant bits
// (error-free two-sum of Knuth; exact products from the fused multiply-add residual).
struct FF {
    float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// a += (bh, bl): the high parts are added with their exact rounding error (two-sum), which goes into
// the low part with bl; the pair is renormalised once at the end (ff_norm). The low part only
// collects rounding errors, so its own rounding is of the order of the squared unit roundoff.
__device__ __forceinline__ void ff_add(FF &a, float bh, float bl) {
    float s, e;
    two_sum(a.hi, bh, s, e);
    a.hi = s;
    a.lo = (a.lo + bl) + e;
}
__device__ __forceinline__ void ff_norm(FF &a) {
    float s, e;
    two_sum(a.hi, a.lo, s, e);
    a.hi = s;
    a.lo = e;
}

// grad_s[r] += sum_p l[p] T(D x)[p], grad_o[r] += sum_p l[p]: one warp per range, the domain's
// averages staged in shared memory as in the decode step, exact FP32 products summed in float-float
// per lane, across the warp and into the per-range float-float accumulators (the sums cancel
// heavily: terms of a few hundred add up to gradients of order one; FP64 arithmetic, a small
// fraction of the FP32 rate on this part, is not used).
template <int B, int LD>
__global__ void __launch_bounds__(32 * kDecodeWarps)
    k_adjoint_grads(Geo g, const int32_t *__restrict__ dom, const int32_t *__restrict__ iso,
                    const float *__restrict__ x, const float *__restrict__ lam, float2 *__restrict__ gs,
                    float2 *__restrict__ go) {
    constexpr int NC = B * B / 32;
    constexpr int PV = B == 8 ? 2 : 4;
    __shared__ __align__(16) float cell[kDecodeWarps][B * B];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * kDecodeWarps + warp;
    if (r >= g.R) return;
    const int d = __ldg(dom + r), t = __ldg(iso + r);
    if (!valid_code(g, d, t)) {  // an invalid code: NaN gradients, no read
        if (lane == 0) gs[r] = go[r] = make_float2(__int_as_float(0x7fc00000), 0.f);
        return;
    }
    const int rq = fdiv(r, g.fRx), dq = fdiv(d, g.fDx);
    const float *lr = lam + (size_t)(rq * B) * g.W + (r - rq * g.nRx) * B;
    float *cw = cell[warp];
    load_cells<B, LD>(x + (size_t)(dq * g.sigma) * g.W + (d - dq * g.nDx) * g.sigma, g.W, lane, cw);
    __syncwarp();
    int c0, ky, kx;
    iso_affine<B>(t, c0, ky, kx);
    FF ss{0.f, 0.f}, so{0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NC / PV; ++k) {
        const int p0 = PV * (lane + 32 * k), py = p0 / B, px = p0 % B;
        const int s0 = c0 + ky * py + kx * px;
        float l[PV];
        if constexpr (PV == 2) {
            const float2 v2 = *reinterpret_cast<const float2 *>(lr + (size_t)py * g.W + px);
            l[0] = v2.x;
            l[1] = v2.y;
        } else {
            const float4 v4 = *reinterpret_cast<const float4 *>(lr + (size_t)py * g.W + px);
            l[0] = v4.x;
            l[1] = v4.y;
            l[2] = v4.z;
            l[3] = v4.w;
        }
#pragma unroll
        for (int i = 0; i < PV; ++i) {
            const float v = cw[s0 + i * kx];
            const float ph = l[i] * v;
            ff_add(ss, ph, fmaf(l[i], v, -ph));
            ff_add(so, l[i], 0.f);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float sh = __shfl_xor_sync(0xffffffffu, ss.hi, o), sl = __shfl_xor_sync(0xffffffffu, ss.lo, o);
        const float oh = __shfl_xor_sync(0xffffffffu, so.hi, o), ol = __shfl_xor_sync(0xffffffffu, so.lo, o);
        ff_add(ss, sh, sl);
        ff_add(so, oh, ol);
    }
    if (lane == 0) {
        FF a{gs[r].x, gs[r].y}, b{go[r].x, go[r].y};
        ff_add(a, ss.hi, ss.lo);
        ff_add(b, so.hi, so.lo);
        ff_norm(a);
        ff_norm(b);
        gs[r] = make_float2(a.hi, a.lo);
        go[r] = make_float2(b.hi, b.lo);
    }
}

__global__ void k_grads_out(int R, const float2 *__restrict__ gsf, const float2 *__restrict__ gof,
                            float *__restrict__ gs, float *__restrict__ go) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) {
        gs[r] = gsf[r].x + gsf[r].y;
        go[r] = gof[r].x + gof[r].y;
    }
}

// Dn + 1 segment starts, padded to a multiple of 4 ints so that the radix histograms after them
// start on a 16-byte boundary (the counting sort reads them as 16-byte vectors).
size_t adjoint_off_ints(const Geo &g) { return ((size_t)g.Dn + 1 + 3) & ~(size_t)3; }
size_t adjoint_csr_ints(const Geo &g) { return 4 * (size_t)g.R + adjoint_off_ints(g) + radix_counts_ints(g.R); }
size_t adjoint_entries(const Geo &g) { return (size_t)g.R; }

cudaError_t launch_dom_csr(const Geo &g, const fic_codes &c, const AdjointCsr &a, cudaStream_t st) {
    const unsigned gr = (unsigned)((g.R + 255) / 256);
    k_csr_keys<<<gr, 256, 0, st>>>(g, c.dom, c.iso, c.s, a.key);
    ++g_launches;
    cudaError_t e = launch_radix_sort(a.key, g.R, (uint32_t)g.Dn, a.list, a.t1, a.t2, a.digit, a.counts, st);
    if (e) return e;
    k_csr_sorted_keys<<<gr, 256, 0, st>>>(g.R, a.key, a.list, c.iso, c.s, a.t1, a.ent);
    ++g_launches;
    k_csr_offsets<<<(unsigned)((g.Dn + 1 + 255) / 256), 256, 0, st>>>(g.R, g.Dn, a.t1, a.off);
    ++g_launches;
    return cudaGetLastError();
}

// The pixel phase for this geometry: the 2x2-block form for even strides, with every covering
// domain's bounds loaded first when at most 2 or 4 domains cover a coordinate per axis.
template <int B, int MJ>
void gather_px(const Geo &g, const AdjointCsr &a, float *lam_prev, cudaStream_t st) {
    const bool even = g.sigma % 2 == 0;  // lam_prev is a workspace buffer: 8-byte aligned
    const int cols = even ? g.W / 2 : g.W, rows = even ? g.H / 2 : g.H;
    const dim3 px((unsigned)((cols + 255) / 256), (unsigned)min(rows, 65535));
    if (even)
        k_adjoint_gather2<B, MJ><<<px, 256, 0, st>>>(g, a.off, a.acc, lam_prev);
    else
        k_adjoint_gather<B, MJ><<<px, 256, 0, st>>>(g, a.off, a.acc, lam_prev);
}

template <int B>
void adjoint_gather_b(const Geo &g, const AdjointCsr &a, const float *lam, float *lam_prev, cudaStream_t st) {
    const unsigned cells = (unsigned)(((long long)g.R * (B * B >= 32 ? 32 : B * B) + 255) / 256);
    k_adjoint_cells<B><<<cells, 256, 0, st>>>(g, a.ent, a.off, lam, a.acc);
    // covering domains per axis: at most ceil(2B / sigma)
    const int mj = (2 * B + g.sigma - 1) / g.sigma;
    if (mj <= 2)
        gather_px<B, 2>(g, a, lam_prev, st);
    else if (mj <= 4)
        gather_px<B, 4>(g, a, lam_prev, st);
    else
        gather_px<B, 0>(g, a, lam_prev, st);
}

cudaError_t launch_adjoint_gather(const Geo &g, const fic_codes &c, const AdjointCsr &a, const float *lam,
                                  float *lam_prev, cudaStream_t st) {
    (void)c;
    if (g.B == 16)
        adjoint_gather_b<16>(g, a, lam, lam_prev, st);
    else
        adjoint_gather_b<8>(g, a, lam, lam_prev, st);
    g_launches += 2;
    return cudaGetLastError();
}

template <int B>
void adjoint_grads_b(int ld, unsigned blocks, const Geo &g, const fic_codes &c, const float *x, const float *lam,
                     float2 *gs, float2 *go, cudaStream_t st) {
    if (ld == 4)
        k_adjoint_grads<B, 4><<<blocks, 32 * kDecodeWarps, 0, st>>>(g, c.dom, c.iso, x, lam, gs, go);
    else if (ld == 2)
        k_adjoint_grads<B, 2><<<blocks, 32 * kDecodeWarps, 0, st>>>(g, c.dom, c.iso, x, lam, gs, go);
    else
        k_adjoint_grads<B, 1><<<blocks, 32 * kDecodeWarps, 0, st>>>(g, c.dom, c.iso, x, lam, gs, go);
}

cudaError_t launch_adjoint_grads(const Geo &g, const fic_codes &c, const float *x, const float *lam,
                                 float2 *gs, float2 *go, cudaStream_t st) {
    const unsigned blocks = (unsigned)((g.R + kDecodeWarps - 1) / kDecodeWarps);
    const uintptr_t xa = (uintptr_t)x;
    const int ld = (g.sigma % 4 == 0 && xa % 16 == 0) ? 4 : (g.sigma % 2 == 0 && xa % 8 == 0) ? 2 : 1;
    if (g.B == 16)
        adjoint_grads_b<16>(ld, blocks, g, c, x, lam, gs, go, st);
    else
        adjoint_grads_b<8>(ld, blocks, g, c, x, lam, gs, go, st);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_grads_out(int R, const float2 *gsf, const float2 *gof, float *gs, float *go, cudaStream_t st) {
    k_grads_out<<<(R + 255) / 256, 256, 0, st>>>(R, gsf, gof, gs, go);
    ++g_launches;
    return cudaGetLastError();
}

// ---- the adjoint on the plane of 2x2 averages ------------------------------------------------
// With an even stride one step is x_{k+1} = M P_k + b, P_k = A x_k the plane of 2x2 averages and M
// the per-range map s_r T_t of its window, so with nu_k = dL/dP_k = M^T l_{k+1}:
//   nu_{K-1} = M^T l_K (l_K = dL/dx_K, full resolution),
//   nu_k = H^T nu_{k+1} for k < K - 1, H = A M the plane step, which is the fractal map of ranges
//   B/2 and windows B on the plane at stride sigma/2 (so W^T's two phases on the plane geometry);
// and the gradient terms of step k, from l_{k+1} = A^T nu_{k+1} (nu_{k+1} / 4 over each 2x2 block):
//   k < K - 1: grad_s_r += sum over the cells c of r of nu_{k+1}[c] E_k[src'_t(c)] (E_k the 2x2 means
//              of r's window of P_k), grad_o_r += sum_c nu_{k+1}[c];
//   k = K - 1: grad_s_r += sum over the pixels p of r of l_K[p] P_{K-1}[window + src_t(p)],
//              grad_o_r += sum_p l_K[p].
// The checkpoints and the recomputed iterates are planes, and only the last step reads full-
// resolution data (l_K).

// Gradient terms of one step, a group of TG lanes per range (4 for 8x8 ranges, 8 for 16x16, so
// that a lane sums several terms before the float-float reduction across the group): FINAL =
// false takes lam = nu_{k+1} (a plane) and, for each cell (u, v) of the range, the 2x2 mean of the
// window of P = P_k at src'_t(u, v) (two aligned float2 loads when V2, else four single loads);
// FINAL = true takes lam = l_K (full resolution) and the window of P = P_{K-1} directly. Exact FP32
// products summed in float-float per lane, across the group and into the per-range accumulators.
template <int B>
struct GradShape {
    static constexpr int TG = B == 8 ? 4 : 8;  // lanes per range
    static constexpr int G = 256 / TG;         // ranges per block
};

template <int B, bool FINAL, bool V2>
__global__ void __launch_bounds__(256)
    k_plane_grads(Geo g, const int4 *__restrict__ pk, const float *__restrict__ P, const float *__restrict__ lam,
                  float2 *__restrict__ gs, float2 *__restrict__ go) {
    constexpr int TG = GradShape<B>::TG, G = GradShape<B>::G;
    constexpr int OB = B / 2, J = OB * OB / TG, JF = B * B / TG;
    const int grp = threadIdx.x / TG, l = threadIdx.x % TG;
    const unsigned gmask = ((1u << TG) - 1u) << ((threadIdx.x & 31) & ~(TG - 1));
    const int r = blockIdx.x * G + grp;
    if (r >= g.R) return;  // whole groups leave together
    const int4 c = __ldg(pk + r);
    if (c.x < 0) {  // an invalid code: NaN gradients, no read
        if (l == 0) gs[r] = go[r] = make_float2(__int_as_float(0x7fc00000), 0.f);
        return;
    }
    const int Wh = g.W / 2;
    const int rq = fdiv(r, g.fRx), rx = r - rq * g.nRx;
    const float *w = P + c.x;
    FF ss{0.f, 0.f}, so{0.f, 0.f};
    if constexpr (FINAL) {
#pragma unroll
        for (int j = 0; j < JF; ++j) {
            const int q = l + TG * j, py = q / B, px = q % B;
            int sy, sx;
            iso_src(B, c.y, py, px, sy, sx);
            const float v = __ldg(w + (size_t)sy * Wh + sx);
            const float lv = __ldg(lam + (size_t)(rq * B + py) * g.W + rx * B + px);
            const float ph = lv * v;
            ff_add(ss, ph, fmaf(lv, v, -ph));
            ff_add(so, lv, 0.f);
        }
    } else {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int q = l + TG * j, u = q / OB, v = q % OB;
            int sy, sx;
            iso_src(OB, c.y, u, v, sy, sx);
            const float *p = w + (size_t)(2 * sy) * Wh + 2 * sx;
            float e;
            if constexpr (V2) {
                const float2 lo = __ldg(reinterpret_cast<const float2 *>(p));
                const float2 hi = __ldg(reinterpret_cast<const float2 *>(p + Wh));
                e = (((lo.x + lo.y) + hi.x) + hi.y) * 0.25f;
            } else {
                e = (((__ldg(p) + __ldg(p + 1)) + __ldg(p + Wh)) + __ldg(p + Wh + 1)) * 0.25f;
            }
            const float lv = __ldg(lam + (size_t)(rq * OB + u) * Wh + rx * OB + v);
            const float ph = lv * e;
            ff_add(ss, ph, fmaf(lv, e, -ph));
            ff_add(so, lv, 0.f);
        }
    }
#pragma unroll
    for (int o = TG / 2; o > 0; o >>= 1) {
        const float sh = __shfl_xor_sync(gmask, ss.hi, o), sl = __shfl_xor_sync(gmask, ss.lo, o);
        const float oh = __shfl_xor_sync(gmask, so.hi, o), ol = __shfl_xor_sync(gmask, so.lo, o);
        ff_add(ss, sh, sl);
        ff_add(so, oh, ol);
    }
    if (l == 0) {
        FF a{gs[r].x, gs[r].y}, b{go[r].x, go[r].y};
        ff_add(a, ss.hi, ss.lo);
        ff_add(b, so.hi, so.lo);
        ff_norm(a);
        ff_norm(b);
        gs[r] = make_float2(a.hi, a.lo);
        go[r] = make_float2(b.hi, b.lo);
    }
}

// The gradient terms of a step k < K - 1 and the cell phase of H^T nu_{k+1} in one pass, a group
// of LPR lanes per list position of the domain -> ranges index (LPR = 16 for 8x8 ranges, a warp for
// 16x16; every range has a position, the listed ones first): lane l holds the cells l + LPR m of
// range r's (B/2) x (B/2) grid of nu_{k+1} in row-major order, forms the gradient terms of those
// cells against the 2x2 means of r's window of P_k (as k_plane_grads), and, when r is listed,
// writes the cell block (s_r / 4) nu_{k+1}[p_r(c)] of its position (as k_adjoint_cells on the
// plane geometry), taking nu_{k+1}[p_r(c)] from the lane that holds it by a shuffle.
template <int B, bool V2>
__global__ void __launch_bounds__(256)
    k_plane_grads_cells(Geo g, const int4 *__restrict__ pk, const int4 *__restrict__ ent,
                        const int32_t *__restrict__ off, const float *__restrict__ P,
                        const float *__restrict__ lam, float *__restrict__ acc, float2 *__restrict__ gs,
                        float2 *__restrict__ go) {
    constexpr int OB = B / 2, NCELL = OB * OB, LPR = NCELL >= 32 ? 32 : NCELL, M = NCELL / LPR;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int kpos = tid / LPR, l = tid % LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << ((threadIdx.x & 31) & ~(LPR - 1)));
    const int gbase = (threadIdx.x & 31) & ~(LPR - 1);
    if (kpos >= g.R) return;  // whole groups leave together
    const int n = __ldg(off + g.Dn);  // listed ranges
    const int4 e = __ldg(ent + kpos);
    const int r = e.x;
    const int4 c = __ldg(pk + r);
    const int Wh = g.W / 2;
    const int rq = fdiv(r, g.fRx), rx = r - rq * g.nRx;
    float nv[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int q = l + LPR * m;
        nv[m] = __ldg(lam + (size_t)(rq * OB + q / OB) * Wh + rx * OB + q % OB);
    }
    if (kpos < n) {
        // the cell block of this list position: cell q of the window block takes nu at the range
        // cell p = src'_{t^-1}(q)
        const float sc = __int_as_float(e.z);
        int c0, ky, kx;
        iso_affine<OB>(e.y == 1 ? 3 : (e.y == 3 ? 1 : e.y), c0, ky, kx);
        float *dst = acc + (size_t)kpos * NCELL;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int q = l + LPR * m, p = c0 + ky * (q / OB) + kx * (q % OB);
            float v = __shfl_sync(gmask, nv[0], gbase + p % LPR);
            if constexpr (M == 2) {
                const float hi = __shfl_sync(gmask, nv[1], gbase + p % LPR);
                v = p >= LPR ? hi : v;
            }
            dst[q] = sc * v;
        }
    }
    if (c.x < 0) {  // an invalid code: NaN gradients, no read
        if (l == 0) gs[r] = go[r] = make_float2(__int_as_float(0x7fc00000), 0.f);
        return;
    }
    const float *w = P + c.x;
    FF ss{0.f, 0.f}, so{0.f, 0.f};
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int q = l + LPR * m;
        int sy, sx;
        iso_src(OB, c.y, q / OB, q % OB, sy, sx);
        const float *p = w + (size_t)(2 * sy) * Wh + 2 * sx;
        float ev;
        if constexpr (V2) {
            const float2 lo = __ldg(reinterpret_cast<const float2 *>(p));
            const float2 hi = __ldg(reinterpret_cast<const float2 *>(p + Wh));
            ev = (((lo.x + lo.y) + hi.x) + hi.y) * 0.25f;
        } else {
            ev = (((__ldg(p) + __ldg(p + 1)) + __ldg(p + Wh)) + __ldg(p + Wh + 1)) * 0.25f;
        }
        const float ph = nv[m] * ev;
        ff_add(ss, ph, fmaf(nv[m], ev, -ph));
        ff_add(so, nv[m], 0.f);
    }
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) {
        const float sh = __shfl_xor_sync(gmask, ss.hi, o), sl = __shfl_xor_sync(gmask, ss.lo, o);
        const float oh = __shfl_xor_sync(gmask, so.hi, o), ol = __shfl_xor_sync(gmask, so.lo, o);
        ff_add(ss, sh, sl);
        ff_add(so, oh, ol);
    }
    if (l == 0) {
        FF a{gs[r].x, gs[r].y}, b{go[r].x, go[r].y};
        ff_add(a, ss.hi, ss.lo);
        ff_add(b, so.hi, so.lo);
        ff_norm(a);
        ff_norm(b);
        gs[r] = make_float2(a.hi, a.lo);
        go[r] = make_float2(b.hi, b.lo);
    }
}

// The plane geometry of H: ranges B/2 and windows B on the (H/2) x (W/2) plane at stride sigma/2,
// the same range and domain grids.
static Geo plane_geo(const Geo &g) {
    Geo p = g;
    p.H = g.H / 2;
    p.W = g.W / 2;
    p.pitch = p.W;
    p.B = g.B / 2;
    p.n = p.B * p.B;
    p.sigma = g.sigma / 2;
    p.fS = make_fastdiv((uint32_t)p.sigma);
    return p;
}

template <int B>
static void plane_grads(bool fin, bool v2, const Geo &g, const int4 *pk, const float *P, const float *lam,
                        float2 *gs, float2 *go, cudaStream_t st) {
    const unsigned blocks = (unsigned)((g.R + GradShape<B>::G - 1) / GradShape<B>::G);
    if (fin) k_plane_grads<B, true, false><<<blocks, 256, 0, st>>>(g, pk, P, lam, gs, go);
    else if (v2) k_plane_grads<B, false, true><<<blocks, 256, 0, st>>>(g, pk, P, lam, gs, go);
    else k_plane_grads<B, false, false><<<blocks, 256, 0, st>>>(g, pk, P, lam, gs, go);
}

// nu_{K-1} = M^T l_K: cell blocks s_r l_K[p_r(c)] of B x B window pixels per listed range, then
// per plane pixel the sum over the covering windows (side B at stride sigma/2) and their ranges.
template <int B>
static void plane_mt(const Geo &g, const Geo &gp, const AdjointCsr &a, const float *lK, float *nu,
                     cudaStream_t st) {
    const unsigned cells = (unsigned)(((long long)g.R * 32 + 255) / 256);
    k_adjoint_cells<B, 4><<<cells, 256, 0, st>>>(g, a.ent, a.off, lK, a.acc);
    const int mj = (B + gp.sigma - 1) / gp.sigma;  // covering windows per axis: at most ceil(B / (sigma/2))
    const dim3 px((unsigned)((gp.W + 255) / 256), (unsigned)min(gp.H, 65535));
    if (mj <= 2)
        k_adjoint_gather<B / 2, 2, true><<<px, 256, 0, st>>>(gp, a.off, a.acc, nu);
    else if (mj <= 4)
        k_adjoint_gather<B / 2, 4, true><<<px, 256, 0, st>>>(gp, a.off, a.acc, nu);
    else
        k_adjoint_gather<B / 2, 0, true><<<px, 256, 0, st>>>(gp, a.off, a.acc, nu);
}


// A reverse step k < K - 1 with its transpose: gradient terms and H^T's cell phase in one launch,
// then H^T's pixel phase on the plane geometry.
template <int B>
static void plane_step_back(bool v2, const Geo &g, const Geo &gp, const AdjointCsr &a, const int4 *pk, const float *P,
                            const float *nu, float *nu_prev, float2 *gs, float2 *go, cudaStream_t st) {
    constexpr int OB = B / 2, LPR = OB * OB >= 32 ? 32 : OB * OB;
    const unsigned blocks = (unsigned)(((long long)g.R * LPR + 255) / 256);
    if (v2) k_plane_grads_cells<B, true><<<blocks, 256, 0, st>>>(g, pk, a.ent, a.off, P, nu, a.acc, gs, go);
    else k_plane_grads_cells<B, false><<<blocks, 256, 0, st>>>(g, pk, a.ent, a.off, P, nu, a.acc, gs, go);
    const int mj = (2 * OB + gp.sigma - 1) / gp.sigma;
    if (mj <= 2)
        gather_px<OB, 2>(gp, a, nu_prev, st);
    else if (mj <= 4)
        gather_px<OB, 4>(gp, a, nu_prev, st);
    else
        gather_px<OB, 0>(gp, a, nu_prev, st);
}

cudaError_t launch_backward_plane(const fic_codes &c, const Geo &g, const AdjointCsr &a, int iters, int ck,
                                  const float *x0, const float *grad_out, float *ckpt, float *seg, float *nu,
                                  int4 *pk, float2 *gs, float2 *go, cudaStream_t st) {
    const size_t pl = (size_t)g.H * g.W / 4;  // floats per plane (a multiple of 64)
    const int nseg = (iters + ck - 1) / ck;
    const Geo gp = plane_geo(g);
    const bool v2 = g.sigma % 4 == 0;
    k_pack_codes<<<(unsigned)((g.R + 255) / 256), 256, 0, st>>>(g, c.dom, c.iso, c.s, c.o, pk);
    ++g_launches;
    // P_0 into the first checkpoint
    if (x0) {
        const dim3 grid((unsigned)((g.W / 4 + kHalfThreads - 1) / kHalfThreads), (unsigned)(g.H / 2));
        if ((uintptr_t)x0 % 16 == 0)
            k_pool2<true><<<grid, kHalfThreads, 0, st>>>(x0, g.W, ckpt);
        else
            k_pool2<false><<<grid, kHalfThreads, 0, st>>>(x0, g.W, ckpt);
        ++g_launches;
    } else {
        cudaError_t e = launch_fill(ckpt, pl, 128.f, st);
        if (e != cudaSuccess) return e;
    }
    auto plane = [&](int c0, int i) -> float * { return i == 0 ? ckpt + (size_t)c0 * pl : seg + (size_t)i * pl; };
    auto step = [&](const float *src, float *dst) {
        if (g.B == 16) launch_plane_step<16, false>(v2, false, g, pk, src, dst, st);
        else launch_plane_step<8, false>(v2, false, g, pk, src, dst, st);
        ++g_launches;
    };
    for (int c0 = 0; c0 + 1 < nseg; ++c0)
        for (int i = 1; i <= ck; ++i) step(plane(c0, i - 1), i == ck ? ckpt + (size_t)(c0 + 1) * pl : plane(c0, i));
    float *ncur = nu, *nprev = nu + pl;
    bool fin = true;  // the first reverse step is the last forward step
    for (int c0 = nseg - 1; c0 >= 0; --c0) {
        const int len = (c0 == nseg - 1) ? iters - c0 * ck : ck;
        for (int i = 1; i < len; ++i) step(plane(c0, i - 1), plane(c0, i));
        for (int i = len - 1; i >= 0; --i) {
            const bool more = c0 > 0 || i > 0;  // a transpose is needed (not the first step)
            if (fin || !more) {
                // the last step's terms (full-resolution l_K), or the first step's (no transpose)
                const float *lam = fin ? grad_out : ncur;
                if (g.B == 16) plane_grads<16>(fin, v2, g, pk, plane(c0, i), lam, gs, go, st);
                else plane_grads<8>(fin, v2, g, pk, plane(c0, i), lam, gs, go, st);
                ++g_launches;
                if (fin && more) {
                    if (g.B == 16) plane_mt<16>(g, gp, a, grad_out, ncur, st);
                    else plane_mt<8>(g, gp, a, grad_out, ncur, st);
                    g_launches += 2;
                }
            } else {
                if (g.B == 16) plane_step_back<16>(v2, g, gp, a, pk, plane(c0, i), ncur, nprev, gs, go, st);
                else plane_step_back<8>(v2, g, gp, a, pk, plane(c0, i), ncur, nprev, gs, go, st);
                g_launches += 2;
                float *t = ncur;
                ncur = nprev;
                nprev = t;
            }
            fin = false;
        }
    }
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
