// Fifth-generation tensor core (tcgen05) primitives for sm_100-family GPUs
// (GB300: sm_103a), as inline PTX: shared-memory matrix descriptors, the
// instruction descriptor of a dense bf16 x bf16 -> f32 MMA, tensor-memory
// allocation, the MMA itself, its completion through an mbarrier (with a
// bounded wait) and tensor-memory loads.  Operand layout: K-major, no
// swizzle ("interleaved"): an 8-row x 16-byte core matrix is 128 contiguous
// bytes; core matrices adjacent along K are LBO bytes apart and those
// adjacent along M (or N) SBO bytes apart.
#pragma once

#include <stdint.h>

namespace p2 {
namespace tc {


// Byte offset of element (row, k) of a K-major bf16 operand in the
// interleaved layout with the given SBO (LBO = 128: the core matrices of a
// row group follow each other along K).
static __host__ __device__ __forceinline__ uint32_t kmajor_off(int row, int k, uint32_t sbo) {
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, all in units of 16 bytes; version 1 (bits 46-47);
// base offset 0; layout "no swizzle" (bits 61-63 = 0).
static __device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16 with bf16 A and B, f32 D, both
// operands K-major, dense: D format bits 4-5 = 1 (f32), A format bits 7-9 =
// 1 (bf16), B format bits 10-12 = 1 (bf16), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
static __host__ __device__ __forceinline__ uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

#if defined(P2_CPU_EMU)
// CPU emulation (the library's kernels also run on the host, one thread per
// CUDA thread, for memory checking): shared-memory addresses are offsets into
// the block's dynamic shared memory, tensor memory is one host array (blocks
// run one after another), an MMA is computed at issue by the issuing thread
// from the operands the descriptors point at, and an mbarrier counts its
// completed phases.
static inline uint32_t smem_addr(const void *p) {
    return (uint32_t)((const unsigned char *)p - emu_dyn_smem_ptr);
}
static inline float (&emu_tmem())[128][512] {
    static float t[128][512];
    return t;
}
static inline void tmem_alloc(uint32_t *dst, uint32_t) {
    if ((threadIdx.x & 31) == 0) *dst = 0;
    __syncwarp();
}
static inline void tmem_relinquish() {}
static inline void tmem_dealloc(uint32_t, uint32_t) {}
static inline float emu_bf16(const unsigned char *p) {
    uint16_t h;
    memcpy(&h, p, 2);
    return __int_as_float((int)((uint32_t)h << 16));
}
static inline void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                            uint32_t accumulate) {
    const uint32_t aaddr = (uint32_t)(adesc & 0x3FFFu) << 4;
    const uint32_t alb = (uint32_t)((adesc >> 16) & 0x3FFFu) << 4;
    const uint32_t asb = (uint32_t)((adesc >> 32) & 0x3FFFu) << 4;
    const uint32_t baddr = (uint32_t)(bdesc & 0x3FFFu) << 4;
    const uint32_t blb = (uint32_t)((bdesc >> 16) & 0x3FFFu) << 4;
    const uint32_t bsb = (uint32_t)((bdesc >> 32) & 0x3FFFu) << 4;
    const int N = (int)((idesc >> 17) & 0x3Fu) << 3, M = (int)((idesc >> 24) & 0x1Fu) << 4;
    const int lane0 = (int)(d_tmem >> 16), col0 = (int)(d_tmem & 0xFFFFu);
    if (lane0 + M > 128 || col0 + N > 512) abort();
    const unsigned char *sm = emu_dyn_smem_ptr;
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
            float acc = accumulate ? emu_tmem()[lane0 + m][col0 + n] : 0.f;
            for (int k = 0; k < 16; ++k) {
                const float a = emu_bf16(sm + aaddr + (m >> 3) * asb + (k >> 3) * alb +
                                         (m & 7) * 16 + (k & 7) * 2);
                const float b = emu_bf16(sm + baddr + (n >> 3) * bsb + (k >> 3) * blb +
                                         (n & 7) * 16 + (k & 7) * 2);
                acc = fmaf(a, b, acc);
            }
            emu_tmem()[lane0 + m][col0 + n] = acc;
        }
}
static inline void mma_commit(uint64_t *bar) { __atomic_add_fetch(bar, 1, __ATOMIC_SEQ_CST); }
static inline void mbar_init(uint64_t *bar, uint32_t) { __atomic_store_n(bar, 0, __ATOMIC_SEQ_CST); }
static inline void mbar_inval(uint64_t *) {}
static inline bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t) {
    for (long n = 0; n < 200000000L; ++n) {
        if ((uint32_t)(__atomic_load_n(bar, __ATOMIC_SEQ_CST) & 1u) != parity) return true;
        std::this_thread::yield();
    }
    return false;
}
static inline void fence_async_smem() {}
static inline void fence_before_sync() {}
static inline void fence_after_sync() {}
static inline void tmem_ld16(uint32_t taddr, float *v) {
    const int lane = (int)(taddr >> 16) + (int)(threadIdx.x & 31), col = (int)(taddr & 0xFFFFu);
    if (lane >= 128 || col + 16 > 512) abort();
    for (int i = 0; i < 16; ++i) v[i] = emu_tmem()[lane][col + i];
}
static inline void tmem_ld8(uint32_t taddr, float *v) {
    const int lane = (int)(taddr >> 16) + (int)(threadIdx.x & 31), col = (int)(taddr & 0xFFFFu);
    if (lane >= 128 || col + 8 > 512) abort();
    for (int i = 0; i < 8; ++i) v[i] = emu_tmem()[lane][col + i];
}
static inline void tmem_wait_ld() {}
static inline long long f2ll_rn(float v) { return llrintf(v); }
#else
static __device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Tensor-memory allocation of ncols columns (a power of two >= 32) by one
// whole warp; the base address is written to *dst (shared memory).
static __device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
}
static __device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
static __device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// D[tmem] (+)= A[smem] B[smem]^T, issued by one thread.
static __device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                                uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The mbarrier at bar receives one arrival when every MMA issued so far by
// this thread has completed.
static __device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(bar))
        : "memory");
}

static __device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
static __device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Wait for the phase with the given parity to complete, at most `limit`
// polls; returns false when the limit ran out.
static __device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t n = 0; n < limit; ++n) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Generic-proxy shared-memory writes made visible to the tensor core.
static __device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
static __device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
static __device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive f32 columns of this thread's tensor-memory lane (the
// warp's 32-lane quadrant starts at taddr's lane field).
static __device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 8 consecutive f32 columns of this thread's tensor-memory lane
static __device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
static __device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// float -> int64, round to nearest
static __device__ __forceinline__ long long f2ll_rn(float v) { return __float2ll_rn(v); }
#endif

}  // namespace tc
}  // namespace p2
