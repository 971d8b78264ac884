// Code format and quantiser for the fractal codes. Section 1 stores each range's domain and map
// coefficients but the paper fixes no format; the library
// quantises the contrast s uniformly to 2^bits_s levels on [-1, 1] (both endpoints included) and
// the brightness o uniformly to 2^bits_o levels on the image's observed [min o, max o], rounding
// half to even, with the binary64 operations in the order the header documents.
#include "fic_internal.cuh"

namespace fic {

constexpr int kQuantBlocks = 256;

__global__ void k_minmax_partial(const double *__restrict__ o, int n, double *__restrict__ pmin,
                                 double *__restrict__ pmax) {
    __shared__ double smin[256], smax[256];
    double mn = __longlong_as_double(0x7ff0000000000000LL), mx = -mn;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        mn = fmin(mn, o[i]);
        mx = fmax(mx, o[i]);
    }
    smin[threadIdx.x] = mn;
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pmin[blockIdx.x] = smin[0];
        pmax[blockIdx.x] = smax[0];
    }
}

__global__ void k_minmax_final(const double *__restrict__ pmin, const double *__restrict__ pmax, double *header) {
    __shared__ double smin[256], smax[256];
    smin[threadIdx.x] = pmin[threadIdx.x];
    smax[threadIdx.x] = pmax[threadIdx.x];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        header[0] = smin[0];
        header[1] = smax[0];
    }
}

__global__ void k_quantize(fic_codes in, int n, int bits_s, int bits_o, const double *__restrict__ header,
                           uint16_t *__restrict__ q_s, uint16_t *__restrict__ q_o, fic_codes out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double Ls = (double)((1 << bits_s) - 1), Lo = (double)((1 << bits_o) - 1);
    const double lo = header[0], hi = header[1];
    double qs = rint(__dmul_rn(__ddiv_rn(__dadd_rn(in.s[i], 1.0), 2.0), Ls));
    qs = fmin(fmax(qs, 0.0), Ls);
    double qo = 0.0;
    if (hi > lo) {
        qo = rint(__dmul_rn(__ddiv_rn(__dsub_rn(in.o[i], lo), __dsub_rn(hi, lo)), Lo));
        qo = fmin(fmax(qo, 0.0), Lo);
    }
    q_s[i] = (uint16_t)qs;
    q_o[i] = (uint16_t)qo;
    out.dom[i] = in.dom[i];
    out.iso[i] = in.iso[i];
    out.s[i] = __dsub_rn(__ddiv_rn(__dmul_rn(qs, 2.0), Ls), 1.0);
    out.o[i] = __dadd_rn(lo, __ddiv_rn(__dmul_rn(qo, __dsub_rn(hi, lo)), Lo));
}

cudaError_t launch_quantize(const fic_codes &in, int n, int bits_s, int bits_o, uint16_t *q_s, uint16_t *q_o,
                            double *header, const fic_codes &out, cudaStream_t st) {
    k_minmax_partial<<<kQuantBlocks, 256, 0, st>>>(in.o, n, header + 2, header + 2 + kQuantBlocks);
    ++g_launches;
    k_minmax_final<<<1, 256, 0, st>>>(header + 2, header + 2 + kQuantBlocks, header);
    ++g_launches;
    k_quantize<<<(n + 255) / 256, 256, 0, st>>>(in, n, bits_s, bits_o, header, q_s, q_o, out);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace fic
