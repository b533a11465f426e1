// Inline-PTX wrappers for the 5th-generation tensor cores (tcgen05), TMEM,
// mbarriers and bulk async copies on sm_103a. Used by the BF16 network.
//
// Shared-memory operand layout used throughout ("core-matrix blocked"): a
// BF16 matrix X[R x C] stores element (r, c) at
//     (r / 8) * (C / 8) * 128 + (c / 8) * 128 + (r % 8) * 16 + (c % 8) * 2
// i.e. 8 x 8 core matrices of 128 contiguous bytes, 16-byte rows along C,
// core matrices adjacent in C 128 B apart and 8-row groups (C / 8) * 128 B
// apart. With no swizzle, a matrix descriptor's leading byte offset is the
// distance between core matrices adjacent along K and its stride byte offset
// the distance between core matrices adjacent along M/N. The same bytes are a
// K-major operand with K = C (LBO = 128, SBO = (C/8)*128) or an MN-major
// operand with MN = C and K = R (LBO = (C/8)*128, SBO = 128).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace sssgs {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t blk_offset(int r, int c, int C) {
    return (uint32_t)((r >> 3) * (C >> 3) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// Instruction descriptor of kind::f16 with BF16 A/B, FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn_major, bool b_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) | ((b_mn_major ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Wait for the mbarrier phase with parity `parity` for at most `limit` SM
// clock cycles (cheap to read). Returns false when the limit runs out (the
// caller records a timeout and stops).
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, long long limit) {
    long long t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it == 0) t0 = clock64();
        else if ((it & 15) == 0 && clock64() - t0 > limit) return false;
    }
}

// The kernels' wait: about 2 s at the maximum clock.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    return mbar_wait_for(bar, parity, 4000000000ll);
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk (non-tensor) async copy global -> shared, completing on an mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor (no swizzle, descriptor version 1) as its
// two 32-bit words: bits 0-13 start address >> 4, 16-29 leading byte offset
// >> 4, 32-45 stride byte offset >> 4, bit 46 the version. Stepping an operand
// by a byte offset is one 32-bit add to the start-address field: shared-memory
// addresses stay below 256 KB, so the field never carries into the next one.
struct Desc2 {
    uint32_t lo, hi;
};
__device__ __forceinline__ Desc2 desc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return Desc2{((saddr >> 4) & 0x3FFFu) | (((lbo >> 4) & 0x3FFFu) << 16), ((sbo >> 4) & 0x3FFFu) | (1u << 14)};
}

// D(tmem) (+)= A(smem) * B(smem)^T issued from a converged warp: every lane
// evaluates the warp-uniform operands and lane 0 alone executes the MMA.
// a_step / b_step are byte offsets added to the operands' start addresses.
__device__ __forceinline__ void mma_bf16_w(uint32_t d_tmem, Desc2 a, uint32_t a_step, Desc2 b, uint32_t b_step,
                                           uint32_t idesc, uint32_t accumulate, uint32_t lane) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t.reg .b64 da, db;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "setp.eq.u32 e, %7, 0;\n\t"
        "mov.b64 da, {%1, %2};\n\t"
        "mov.b64 db, {%3, %4};\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n\t}\n" ::"r"(d_tmem),
        "r"(a.lo + (a_step >> 4)), "r"(a.hi), "r"(b.lo + (b_step >> 4)), "r"(b.hi), "r"(idesc), "r"(accumulate),
        "r"(lane)
        : "memory");
}

// tcgen05.commit from lane 0 of a converged warp (the lane that issued the
// warp's MMAs through mma_bf16_w): the mbarrier arrives once every tcgen05
// operation that lane issued so far has completed.
__device__ __forceinline__ void mma_commit_w(uint32_t bar, uint32_t lane) {
    asm volatile(
        "{\n\t.reg .pred e;\n\t"
        "setp.eq.u32 e, %1, 0;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(bar),
        "r"(lane)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 columns (two x32 loads, one wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
    uint32_t r[64];
#define SSSGS_LD32(OFF, BASE)                                                                              \
    asm volatile(                                                                                          \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                                          \
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"                                        \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                        \
        : "=r"(r[BASE + 0]), "=r"(r[BASE + 1]), "=r"(r[BASE + 2]), "=r"(r[BASE + 3]), "=r"(r[BASE + 4]),   \
          "=r"(r[BASE + 5]), "=r"(r[BASE + 6]), "=r"(r[BASE + 7]), "=r"(r[BASE + 8]), "=r"(r[BASE + 9]),   \
          "=r"(r[BASE + 10]), "=r"(r[BASE + 11]), "=r"(r[BASE + 12]), "=r"(r[BASE + 13]),                  \
          "=r"(r[BASE + 14]), "=r"(r[BASE + 15]), "=r"(r[BASE + 16]), "=r"(r[BASE + 17]),                  \
          "=r"(r[BASE + 18]), "=r"(r[BASE + 19]), "=r"(r[BASE + 20]), "=r"(r[BASE + 21]),                  \
          "=r"(r[BASE + 22]), "=r"(r[BASE + 23]), "=r"(r[BASE + 24]), "=r"(r[BASE + 25]),                  \
          "=r"(r[BASE + 26]), "=r"(r[BASE + 27]), "=r"(r[BASE + 28]), "=r"(r[BASE + 29]),                  \
          "=r"(r[BASE + 30]), "=r"(r[BASE + 31])                                                           \
        : "r"(taddr + OFF));
    SSSGS_LD32(0, 0)
    SSSGS_LD32(32, 32)
#undef SSSGS_LD32
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// ReLU(a), ReLU(b) rounded to BF16 (nearest even), packed with a in the low
// half: one conversion with the clamp built in. Its zeros can differ from
// rounding fmaxf(x, 0) only in sign, which no product or comparison sees.
__device__ __forceinline__ uint32_t pack_bf16_relu(float a, float b) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

// BF16 roundings of (a, b), packed, each kept where the matching half of the
// packed BF16 pair h is > 0 and 0 elsewhere: the same bits as rounding
// (h > 0 ? x : 0).
__device__ __forceinline__ uint32_t pack_bf16_mask(float a, float b, uint32_t h) {
    __nv_bfloat162 hv;
    *reinterpret_cast<uint32_t*>(&hv) = h;
    return pack_bf16(a, b) & __hgt2_mask(hv, __float2bfloat162_rn(0.f));
}

// Leaky-ReLU derivative applied to a packed pair: the BF16 roundings of
// (a, b) where the matching half of the packed BF16 pair h is > 0, of
// (slope a, slope b) elsewhere (the same bits as rounding h > 0 ? x : slope x).
__device__ __forceinline__ uint32_t pack_bf16_leaky(float a, float b, uint32_t h, float slope) {
    __nv_bfloat162 hv;
    *reinterpret_cast<uint32_t*>(&hv) = h;
    const uint32_t m = __hgt2_mask(hv, __float2bfloat162_rn(0.f));
    const float2 s = __fmul2_rn(make_float2(a, b), make_float2(slope, slope));
    return (pack_bf16(a, b) & m) | (pack_bf16(s.x, s.y) & ~m);
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

}  // namespace tc
}  // namespace sssgs
