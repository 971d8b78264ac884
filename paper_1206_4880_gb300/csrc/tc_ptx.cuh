// Inline-PTX wrappers shared by the tensor-engine kernels (sm_103a: mbarrier, TMA, tcgen05,
// TMEM) and the key helpers of their epilogues. Internal to the fic library.
#pragma once

#include <cuda.h>

#include "fic_internal.cuh"

namespace fic {

// rows x cols fp16 row-major tensor map with a box of box_rows x box_cols (box_cols = 64:
// 128-byte rows with 128-byte swizzle; box_cols = 16: 32-byte rows with 32-byte swizzle).
cudaError_t make_map_f16(CUtensorMap *map, void *base, unsigned long long rows, unsigned cols, unsigned box_rows,
                         unsigned box_cols);

namespace {

constexpr unsigned long long kTimeoutNs = 2000000000ull;  // 2 s per wait

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
// Wait of at most limit_ns for the phase of parity `parity`; false on timeout or when another
// role gave up.
__device__ __forceinline__ bool mbar_wait_for(unsigned long long *b, uint32_t parity, volatile int *abort_flag,
                                              unsigned long long limit_ns) {
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_test(b, parity)) return true;
        if ((i & 63) == 0) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > limit_ns) return false;
        }
    }
}
// Bounded wait (kTimeoutNs) for the phase of parity `parity`.
__device__ __forceinline__ bool mbar_wait(unsigned long long *b, uint32_t parity, volatile int *abort_flag) {
    return mbar_wait_for(b, parity, abort_flag, kTimeoutNs);
}
// A role that gave up: records the timeout in the encode's error word and in the library's
// per-device word (read by fic_check), and tells the CTA's other roles to stop.
__device__ __forceinline__ void report_timeout(int32_t *err, int32_t *lib_err, volatile int *abort_flag) {
    atomicExch(err, (int)FIC_ERR_DEVICE_TIMEOUT);
    if (lib_err) atomicExch(lib_err, (int)FIC_ERR_DEVICE_TIMEOUT);
    *abort_flag = 1;
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
// The same for the 16-column correction slice: 32-byte rows, 32-byte swizzle (mode 6), 8-row
// groups 256 bytes apart.
__device__ __forceinline__ unsigned long long sw32_desc(uint32_t saddr) {
    return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((unsigned long long)(256 >> 4) << 32) |
           (1ull << 46) | (6ull << 61);
}
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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait(uint32_t (&v)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                   "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
                   "+r"(v[14]), "+r"(v[15])
                 :
                 : "memory");
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

// Three-input maxima (sm_100+ PTX forms; IEEE max, no flush of subnormals): max of three values,
// and max of their magnitudes.
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float max3_abs(float a, float b, float c) {
    float d;
    asm("max.abs.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Folds a chunk's 32-bit key (score bits, low 9 bits = 511 - domain offset in the chunk starting
// at batch-wide position cbase) into the running 64-bit keys (score bits << 32 | ~position).
__device__ __forceinline__ void merge_chunk_key(unsigned long long &b1, unsigned long long &b2, uint32_t t,
                                                int cbase) {
    const int j = cbase + 511 - (int)(t & 511u);
    const unsigned long long k =
        t ? (((unsigned long long)(t & 0xFFFFFE00u) << 32) | (unsigned long long)(uint32_t)(~j)) : 0ull;
    top2(b1, b2, k);
}

}  // namespace

}  // namespace fic
