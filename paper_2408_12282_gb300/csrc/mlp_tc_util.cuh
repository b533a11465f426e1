// Helpers shared by the tensor-core network kernels: BF16 operand tiles in
// the core-matrix blocked layout of tc.cuh, per-warpgroup named barriers, the
// item -> pair lookup, and the list of rows with a nonzero upstream gradient.
#pragma once
#include "mlp_common.cuh"
#include "tc.cuh"

namespace sssgs {

// Store 8 consecutive FP32 values of row r (columns c..c+7) as BF16.
__device__ __forceinline__ void store8_bf16(uint8_t* base, int r, int c, int C, const float* v) {
    uint4 q;
    q.x = tc::pack_bf16(v[0], v[1]);
    q.y = tc::pack_bf16(v[2], v[3]);
    q.z = tc::pack_bf16(v[4], v[5]);
    q.w = tc::pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(base + tc::blk_offset(r, c, C)) = q;
}

// Store one FP32 value of row r, column c as BF16.
__device__ __forceinline__ void store1_bf16(uint8_t* base, int r, int c, int C, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + tc::blk_offset(r, c, C)) = __float2bfloat16_rn(v);
}

constexpr int TC_MAX_SMEM_PAIRS = 256;

// Item -> pair lookup against a shared-memory copy of the pairs' item offsets
// (falls back to the global table for very large batches).
__device__ __forceinline__ int pair_lookup(const int64_t* s_off, const sssgs_pair* __restrict__ pairs, int n_pairs,
                                           int64_t item) {
    if (n_pairs > TC_MAX_SMEM_PAIRS) return pair_of_item(pairs, n_pairs, item);
    int lo = 0, hi = n_pairs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Store 8 consecutive BF16 values (already packed) of row r.
__device__ __forceinline__ void store8_packed(uint8_t* base, int r, int c, int C, uint4 q) {
    *reinterpret_cast<uint4*>(base + tc::blk_offset(r, c, C)) = q;
}

__device__ __forceinline__ uint4 load8_packed(const uint8_t* base, int r, int c, int C) {
    return *reinterpret_cast<const uint4*>(base + tc::blk_offset(r, c, C));
}

// Hidden-layer epilogue of 8 consecutive columns: ReLU(v + bias) rounded to
// BF16 and stored at (r, c..c+7). The bias adds are paired FP32 additions
// (each rounded as the scalar one); bias8 is 16-byte aligned.
__device__ __forceinline__ void store8_bias_relu(uint8_t* base, int r, int c, int C, const float* v,
                                                 const float* bias8) {
    const float4 b0 = *reinterpret_cast<const float4*>(bias8), b1 = *reinterpret_cast<const float4*>(bias8 + 4);
    const float2 s0 = __fadd2_rn(make_float2(v[0], v[1]), make_float2(b0.x, b0.y));
    const float2 s1 = __fadd2_rn(make_float2(v[2], v[3]), make_float2(b0.z, b0.w));
    const float2 s2 = __fadd2_rn(make_float2(v[4], v[5]), make_float2(b1.x, b1.y));
    const float2 s3 = __fadd2_rn(make_float2(v[6], v[7]), make_float2(b1.z, b1.w));
    uint4 q;
    q.x = tc::pack_bf16_relu(s0.x, s0.y);
    q.y = tc::pack_bf16_relu(s1.x, s1.y);
    q.z = tc::pack_bf16_relu(s2.x, s2.y);
    q.w = tc::pack_bf16_relu(s3.x, s3.y);
    store8_packed(base, r, c, C, q);
}

// The same with Leaky-ReLU: max(x, slope x) for slope < 1 equals
// (x > 0 ? x : slope x) bit for bit, taken on paired FP32 products.
__device__ __forceinline__ void store8_bias_lrelu(uint8_t* base, int r, int c, int C, const float* v,
                                                  const float* bias8, float slope) {
    const float4 b0 = *reinterpret_cast<const float4*>(bias8), b1 = *reinterpret_cast<const float4*>(bias8 + 4);
    const float2 sl = make_float2(slope, slope);
    const float2 s[4] = {__fadd2_rn(make_float2(v[0], v[1]), make_float2(b0.x, b0.y)),
                         __fadd2_rn(make_float2(v[2], v[3]), make_float2(b0.z, b0.w)),
                         __fadd2_rn(make_float2(v[4], v[5]), make_float2(b1.x, b1.y)),
                         __fadd2_rn(make_float2(v[6], v[7]), make_float2(b1.z, b1.w))};
    uint32_t q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 t = __fmul2_rn(s[k], sl);
        q[k] = tc::pack_bf16(fmaxf(s[k].x, t.x), fmaxf(s[k].y, t.y));
    }
    store8_packed(base, r, c, C, make_uint4(q[0], q[1], q[2], q[3]));
}

// Write n TMEM columns [col, col + n) of this warp's 32 lanes with zeros
// (n a multiple of 32); the whole warp calls it.
__device__ __forceinline__ void tmem_zero(uint32_t taddr, int n) {
    for (int c = 0; c < n; c += 32) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
            "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
            "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr + (uint32_t)c), "r"(0u)
            : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Rows of the network backward: the items whose upstream gradient (drec
// fields 16..19) is not all zero, in item order, into active[] with their
// count in *nact; dx_items of the other items is set to 0. Scratch: flag[n],
// cnt/off[ceil(n / 1024)]. Returns the number of launches made.
int launch_active_rows(const float* dout, int64_t dstride, int64_t n, uint8_t* flag, uint32_t* cnt, uint32_t* off,
                       uint32_t* nact,
                       uint32_t* active, float* dx_items, cudaStream_t st);

}  // namespace sssgs
