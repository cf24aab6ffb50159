// Inline-PTX wrappers for the Blackwell (sm_103a) tensor-core path: mbarriers, 1-D bulk
// copies (the TMA unit, global -> shared), tensor-memory allocation, tcgen05.mma of
// kind::f16 with FP32 accumulation, commit, and tensor-memory loads.
//
// Operand layout in shared memory (K-major, 128-byte swizzle): a tile of R rows x 64
// K-elements of FP16 stores row r at byte r * 128, and the 16-byte chunk c (elements 8c ..
// 8c + 7) of row r at chunk position c XOR (r mod 8) -- the layout the tensor cores read
// without shared-memory bank conflicts.  Tiles start on 1024-byte boundaries (8 rows = one
// swizzle atom).  In the matrix descriptor the stride byte offset (between 8-row groups) is
// 1024 and the leading byte offset is unused; one MMA consumes K = 16 (32 bytes of a row),
// so the K step advances the start address by 32 bytes inside the atom.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sstc {

constexpr uint32_t kCoreLbo = 16;       // unused by the swizzled K-major layout (encoded 1)
constexpr uint32_t kCoreSbo = 1024;     // bytes between 8-row groups
constexpr int kTileK = 64;              // K elements per operand tile
constexpr uint32_t kRowGroupBytes = 1024;
constexpr uint32_t kKStepBytes = 32;    // start-address advance per MMA K step of 16

// byte offset of element (row, k) of an R x 64 FP16 tile in the swizzled layout
__host__ __device__ __forceinline__ uint32_t core_offset(int row, int k) {
    return (uint32_t)(row * 128 + ((((k >> 3) ^ row) & 7) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- mbarriers
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false after `limit` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        __nanosleep(32);
    }
    return false;
}

// ---- 1-D bulk copy global -> shared (TMA unit); dst, src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// ---- tensor memory (one warp executes alloc / dealloc)
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// ---- matrix descriptor of a K-major, 128-byte-swizzled operand tile at shared address saddr
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kCoreLbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kCoreSbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;     // descriptor version of the sm_100 family
    d |= (uint64_t)2 << 61;     // layout type: 128-byte swizzle
    return d;
}

// instruction descriptor of kind::f16: A, B FP16, D FP32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
    return (1u << 4)                          // D format: F32
           | (0u << 7) | (0u << 10)           // A, B format: F16
           | ((uint32_t)(N >> 3) << 17)       // N / 8
           | ((uint32_t)(M >> 4) << 24);      // M / 16
}

// D[tmem] (+)= A B^T, one thread issues
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// the mbarrier's arrive fires when every MMA this thread issued before has completed
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// The 112 MMAs of one 64-wide piece of a digit-sliced product (7 slices per operand):
// accumulator d (tensor-memory columns d * kNCols ..) gets sum_{p + q = d} A_p B_q^T.  da, db
// are the descriptors of slice 0 of A and B, the slices kAStride / kBStride bytes apart.  The
// descriptors advance by additions to the start-address field (16-byte units), a few
// instructions per MMA, so one thread keeps the tensor pipe fed; the (d, p) loops stay
// rolled so the 224 descriptors are not all held in registers.  fresh: the first MMA into
// each accumulator overwrites it.
template <uint32_t kAStride, uint32_t kBStride, uint32_t kNCols>
__device__ __forceinline__ void issue_digit_mmas(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                                 bool fresh) {
    const uint32_t keep_first = fresh ? 0u : 1u;
#pragma unroll 1
    for (int d = 0; d < 7; ++d) {
        const uint32_t t = tmem + (uint32_t)d * kNCols;
#pragma unroll 1
        for (int p = 0; p <= d; ++p) {
            const uint64_t a = da + (uint64_t)(p * (kAStride >> 4));
            const uint64_t b = db + (uint64_t)((d - p) * (kBStride >> 4));
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_f16(t, a + (uint64_t)(kk * (kKStepBytes >> 4)), b + (uint64_t)(kk * (kKStepBytes >> 4)), idesc,
                        (kk == 0 && p == 0) ? keep_first : 1u);
        }
    }
}

// 32 lanes x 32 bits, 16 consecutive columns per thread (warp w reads lanes 32 w .. 32 w + 31).
// The load and its wait sit in one asm statement, so no use of the registers can be
// scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace sstc
