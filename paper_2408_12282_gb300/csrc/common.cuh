// Shared device helpers of libsssgs (sm_103a). Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sssgs.h"

#define SSSGS_FULL 0xffffffffu

namespace sssgs {

constexpr float kPi = 3.14159265358979323846f;

// Number of kernels this library has launched (process-wide, host side).
void note_launches(int n);

// Launch-status helper used by every entry point.
// Number of SMs of the current device (at least 1).
static inline int device_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

static inline int launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SSSGS_OK : SSSGS_ERR_CUDA;
}

// Index of the pair owning `item` (pairs ordered by item_offset).
__device__ __forceinline__ int pair_of_item(const sssgs_pair* __restrict__ pairs, int n_pairs, int64_t item) {
    int lo = 0, hi = n_pairs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pairs[mid].item_offset <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Index of the pair owning global tile `tile`.
__device__ __forceinline__ int pair_of_tile(const sssgs_pair* __restrict__ pairs, int n_pairs, int tile) {
    int lo = 0, hi = n_pairs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pairs[mid].tile_offset <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Camera centre C = -R^T t.
__device__ __forceinline__ float3 cam_center(const sssgs_pair& P) {
    return make_float3(-(P.R[0] * P.t[0] + P.R[3] * P.t[1] + P.R[6] * P.t[2]),
                       -(P.R[1] * P.t[0] + P.R[4] * P.t[1] + P.R[7] * P.t[2]),
                       -(P.R[2] * P.t[0] + P.R[5] * P.t[1] + P.R[8] * P.t[2]));
}

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }

// Per-pixel alpha of one splat (Eq. 3 and the alpha definition after it).
// Every compositing kernel, forward and backward replay alike, calls this or
// its two-pixel form below (whose paired instructions round each component
// as these scalar ones do), so their float32 decisions agree bit for bit.
struct AlphaEval {
    float alpha;     // clamped alpha
    float G;         // exp(-p)
    float dx, dy;
    bool use;        // contributes (p >= 0 and alpha >= alpha_min)
    bool clamped;    // o * G > alpha_max
};

__device__ __forceinline__ AlphaEval eval_alpha(float4 g0, float4 g1, float px, float py,
                                                float a_min, float a_max) {
    // Every rounding step is spelled out (no contraction choices left to the
    // compiler), so all kernels that call this take identical decisions.
    AlphaEval r;
    r.dx = __fsub_rn(g0.x, px);
    r.dy = __fsub_rn(g0.y, py);
    const float dxx = __fmul_rn(r.dx, r.dx), dyy = __fmul_rn(r.dy, r.dy), dxy = __fmul_rn(r.dx, r.dy);
    const float p = __fmaf_rn(__fmul_rn(0.5f, g0.z), dxx, __fmaf_rn(__fmul_rn(0.5f, g1.x), dyy, __fmul_rn(g0.w, dxy)));
    r.G = __expf(-p);
    const float araw = __fmul_rn(g1.y, r.G);
    r.clamped = araw > a_max;
    r.alpha = fminf(a_max, araw);
    r.use = (p >= 0.f) && (r.alpha >= a_min);
    return r;
}

// The same for two pixels of one column (x = px, y = py0 and py1): the
// per-pixel steps run as paired FP32 instructions, each component rounded
// exactly like the scalar operation above (a - b as a + (-b), which is the
// same IEEE result), so both pixels get eval_alpha's results bit for bit.
__device__ __forceinline__ void eval_alpha2(float4 g0, float4 g1, float px, float py0, float py1, float a_min,
                                            float a_max, AlphaEval& r0, AlphaEval& r1) {
    const float dx = __fsub_rn(g0.x, px);
    const float dxx = __fmul_rn(dx, dx);
    const float2 dy = __fadd2_rn(make_float2(g0.y, g0.y), make_float2(-py0, -py1));
    const float2 dyy = __fmul2_rn(dy, dy);
    const float2 dxy = __fmul2_rn(make_float2(dx, dx), dy);
    const float hc = __fmul_rn(0.5f, g1.x), ha = __fmul_rn(0.5f, g0.z);
    const float2 inner = __ffma2_rn(make_float2(hc, hc), dyy, __fmul2_rn(make_float2(g0.w, g0.w), dxy));
    const float2 p = __ffma2_rn(make_float2(ha, ha), make_float2(dxx, dxx), inner);
    r0.dx = dx;
    r1.dx = dx;
    r0.dy = dy.x;
    r1.dy = dy.y;
    r0.G = __expf(-p.x);
    r1.G = __expf(-p.y);
    const float2 araw = __fmul2_rn(make_float2(g1.y, g1.y), make_float2(r0.G, r1.G));
    r0.clamped = araw.x > a_max;
    r1.clamped = araw.y > a_max;
    r0.alpha = fminf(a_max, araw.x);
    r1.alpha = fminf(a_max, araw.y);
    r0.use = (p.x >= 0.f) && (r0.alpha >= a_min);
    r1.use = (p.y >= 0.f) && (r1.alpha >= a_min);
}

}  // namespace sssgs
