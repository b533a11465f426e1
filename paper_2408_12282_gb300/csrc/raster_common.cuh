// Device helpers shared by the render kernels (raster.cu, raster_ml.cu):
// deferred shading of one pixel and its backward, the splat / sub-tile
// culling test, and cp.async wrappers.
#pragma once
#include "common.cuh"

namespace sssgs {

// ---------------------------------------------------------------- shading

// Shading of one surface point (Eq. 4 BRDF: GGX D, Schlick F, separable
// Smith V; Eq. 7 blend): Lc = sss L_SSS + (1 - sss) (f_s + f_d) L_in
// max(n . w_i, 0) at the point x seen from the camera centre C under the point
// light Lp, with the (unnormalised) normal nbar. With BWD, back-propagates
// gL = dLoss/dLc into dg (feature layout of the G-buffer: 1..3 n, 4..6 base,
// 7 rough, 8 metal, 9 sss, 10..12 L_SSS, 13 L_in; other entries untouched)
// and dx = dLoss/dx.
template <bool BWD>
__device__ __forceinline__ void shade_point(float3 nbar, const float* bb, float rb, float mb, float sb,
                                            const float* Ls, float Li, float3 x, float3 C, float3 Lp, float* Lc,
                                            const float* gL, float* dg, float3* dxo) {
    const float3 Vo = C - x;
    const float3 Vi = make_float3(Lp.x - x.x, Lp.y - x.y, Lp.z - x.z);
    const float lo = sqrtf(dot3(Vo, Vo)), li = sqrtf(dot3(Vi, Vi));
    const float3 wo = (1.f / lo) * Vo, wi = (1.f / li) * Vi;
    const float nn = fmaxf(sqrtf(dot3(nbar, nbar)), 1e-12f);
    const float3 nh = (1.f / nn) * nbar;
    const float3 Hv = wo + wi;
    const float lh = fmaxf(sqrtf(dot3(Hv, Hv)), 1e-12f);
    const float3 h = (1.f / lh) * Hv;
    const float co = dot3(nh, wo), ci = dot3(nh, wi), ch = dot3(nh, h), cv = dot3(wo, h);
    const float no = fmaxf(co, 0.f), ni = fmaxf(ci, 0.f), nhc = fmaxf(ch, 0.f), vh = fmaxf(cv, 0.f);
    const float ar = rb * rb, a2 = ar * ar;
    const float den = nhc * nhc * (a2 - 1.f) + 1.f;
    const float D = a2 / (kPi * den * den);
    const float so = sqrtf(a2 + (1.f - a2) * no * no), si = sqrtf(a2 + (1.f - a2) * ni * ni);
    const float Lo = no + so, Lm = ni + si;
    const float Vis = 1.f / (Lo * Lm);
    const float om = 1.f - vh, om2 = om * om, w5 = om2 * om2 * om;
    float F0[3], Fr[3], fs[3], fd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        F0[c] = 0.04f * (1.f - mb) + bb[c] * mb;
        Fr[c] = F0[c] + (1.f - F0[c]) * w5;
        fs[c] = D * Fr[c] * Vis;
        fd[c] = (1.f - mb) * bb[c] * (1.f / kPi);
        Lc[c] = sb * Ls[c] + (1.f - sb) * (fs[c] + fd[c]) * Li * ni;
    }
    if constexpr (BWD) {
        float dni = 0.f, dD = 0.f, dVis = 0.f, dw5 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float g = gL[c];
            const float fsd = fs[c] + fd[c];
            dg[9] += g * (Ls[c] - fsd * Li * ni);
            dg[10 + c] += g * sb;
            dg[13] += g * (1.f - sb) * fsd * ni;
            dni += g * (1.f - sb) * fsd * Li;
            const float cm = g * (1.f - sb) * Li * ni;
            dg[8] -= cm * bb[c] * (1.f / kPi);
            dg[4 + c] += cm * (1.f - mb) * (1.f / kPi);
            dD += cm * Fr[c] * Vis;
            dVis += cm * D * Fr[c];
            const float dFr = cm * D * Vis;
            const float dF0 = dFr * (1.f - w5);
            dw5 += dFr * (1.f - F0[c]);
            dg[8] += dF0 * (bb[c] - 0.04f);
            dg[4 + c] += dF0 * mb;
        }
        const float dvh = -5.f * om2 * om2 * dw5;
        const float dLo = -dVis * Vis / Lo, dLm = -dVis * Vis / Lm;
        const float dno = dLo * (1.f + (1.f - a2) * no / so);
        float da2 = dLo * (1.f - no * no) / (2.f * so) + dLm * (1.f - ni * ni) / (2.f * si);
        dni += dLm * (1.f + (1.f - a2) * ni / si);
        const float iden3 = 1.f / (kPi * den * den * den);
        da2 += dD * (den - 2.f * a2 * nhc * nhc) * iden3;
        const float dnh = dD * (-4.f * a2 * nhc * (a2 - 1.f)) * iden3;
        dg[7] += da2 * 4.f * rb * rb * rb;
        const float dco = co > 0.f ? dno : 0.f, dci = ci > 0.f ? dni : 0.f;
        const float dch = ch > 0.f ? dnh : 0.f, dcv = cv > 0.f ? dvh : 0.f;
        float3 dn = dco * wo + dci * wi + dch * h;
        float3 dwo = dco * nh + dcv * h;
        float3 dwi = dci * nh;
        const float3 dh = dch * nh + dcv * wo;
        const float hd = dot3(h, dh);
        const float3 dHv = (1.f / lh) * (dh - hd * h);
        dwo = dwo + dHv;
        dwi = dwi + dHv;
        const float3 dVo = (1.f / lo) * (dwo - dot3(wo, dwo) * wo);
        const float3 dVi = (1.f / li) * (dwi - dot3(wi, dwi) * wi);
        *dxo = make_float3(-dVo.x - dVi.x, -dVo.y - dVi.y, -dVo.z - dVi.z);
        const float3 dnb = (1.f / nn) * (dn - dot3(nh, dn) * nh);
        dg[1] += dnb.x; dg[2] += dnb.y; dg[3] += dnb.z;
    }
}

// Deferred shading of one pixel (Eq. 4 BRDF, Eq. 7 blend) under the point
// light at Lp. F: composited features, T: final transmittance, (u, v): pixel
// centre, P: the camera. The normalised features shade the surface point
// back-projected from the pixel at the composited depth; out = A Lc. With BWD
// it also back-propagates g3 = dLoss/d(out) to dF (15) and dT.
template <bool BWD>
__device__ __forceinline__ void shade_px_at(const float* F, float T, float u, float v, const sssgs_pair& P,
                                            float3 Lp, float A_eps, float* out, const float* g3, float* dF,
                                            float* dT) {
    out[0] = out[1] = out[2] = 0.f;
    if (BWD) {
#pragma unroll
        for (int k = 0; k < SSSGS_NF; ++k) dF[k] = 0.f;
        *dT = 0.f;
    }
    if (!(T < 1.f)) return;                      // no contribution: black, no gradient
    const float A = 1.f - T;
    const float Ad = fmaxf(A, A_eps);
    const float iA = 1.f / Ad;
    float g[SSSGS_NF];
#pragma unroll
    for (int k = 0; k < SSSGS_NF; ++k) g[k] = F[k] * iA;
    const float dbar = g[0], rb = g[7], mb = g[8], sb = g[9], Li = g[13];
    const float3 nbar = make_float3(g[1], g[2], g[3]);
    const float bb[3] = {g[4], g[5], g[6]};
    const float Ls[3] = {g[10], g[11], g[12]};
    // back-projected surface point x = R^T (dbar * ray - t)
    const float3 ray = make_float3((u - P.cx) / P.fx, (v - P.cy) / P.fy, 1.f);
    const float3 Xc = make_float3(dbar * ray.x - P.t[0], dbar * ray.y - P.t[1], dbar * ray.z - P.t[2]);
    const float3 x = make_float3(P.R[0] * Xc.x + P.R[3] * Xc.y + P.R[6] * Xc.z,
                                 P.R[1] * Xc.x + P.R[4] * Xc.y + P.R[7] * Xc.z,
                                 P.R[2] * Xc.x + P.R[5] * Xc.y + P.R[8] * Xc.z);
    float Lc[3];
    if constexpr (!BWD) {
        shade_point<false>(nbar, bb, rb, mb, sb, Ls, Li, x, cam_center(P), Lp, Lc, nullptr, nullptr, nullptr);
#pragma unroll
        for (int c = 0; c < 3; ++c) out[c] = A * Lc[c];
    } else {
        float gL[3], dg[SSSGS_NF];
#pragma unroll
        for (int k = 0; k < SSSGS_NF; ++k) dg[k] = 0.f;
        // out = A Lc: dLoss/dLc = A g3, dLoss/dA = g3 . Lc
#pragma unroll
        for (int c = 0; c < 3; ++c) gL[c] = g3[c] * A;
        float3 dx;
        shade_point<true>(nbar, bb, rb, mb, sb, Ls, Li, x, cam_center(P), Lp, Lc, gL, dg, &dx);
        float dA = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            out[c] = A * Lc[c];
            dA += g3[c] * Lc[c];
        }
        const float3 dXc = make_float3(P.R[0] * dx.x + P.R[1] * dx.y + P.R[2] * dx.z,
                                       P.R[3] * dx.x + P.R[4] * dx.y + P.R[5] * dx.z,
                                       P.R[6] * dx.x + P.R[7] * dx.y + P.R[8] * dx.z);
        dg[0] += dot3(dXc, ray);
        float dAd = 0.f;
#pragma unroll
        for (int k = 0; k < SSSGS_NF; ++k) {
            dF[k] = dg[k] * iA;
            dAd -= dg[k] * g[k] * iA;
        }
        if (A > A_eps) dA += dAd;
        *dT = -dA;
    }
}

// The same under the pair's own light.
template <bool BWD>
__device__ __forceinline__ void shade_px(const float* F, float T, float u, float v, const sssgs_pair& P,
                                         float A_eps, float* out, const float* g3, float* dF, float* dT) {
    shade_px_at<BWD>(F, T, u, v, P, make_float3(P.light[0], P.light[1], P.light[2]), A_eps, out, g3, dF, dT);
}

// ---------------------------------------------------------------- helpers

// 1/x for x = 1 - alpha in [1 - alpha_max, 1]: the hardware reciprocal
// estimate refined by one Newton-Raphson step r <- r + r (1 - x r), which
// squares its relative error (well below one float32 ulp afterwards).
__device__ __forceinline__ float rcp_newton(float x) {
    const float r = __fdividef(1.f, x);
    return __fmaf_rn(r, __fmaf_rn(-x, r, 1.f), r);
}

struct TilePix {
    int i, j;
    bool inside;
    int64_t pix;
};

// Pixel of this thread. Each warp covers an 8 x 4 sub-tile (TILE / 8 sub-tiles
// across), so the per-warp culling mask below is selective.
__device__ __forceinline__ TilePix tile_pixel(const sssgs_pair& P, int tile, int TILE) {
    TilePix r;
    int lt = tile - P.tile_offset;
    int tx = lt % P.tiles_x, ty = lt / P.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per_row = TILE / 8;
    r.i = tx * TILE + (warp % per_row) * 8 + (lane & 7);
    r.j = ty * TILE + (warp / per_row) * 4 + (lane >> 3);
    r.inside = r.i < P.W && r.j < P.H;
    r.pix = P.pixel_offset + (int64_t)r.j * P.W + r.i;
    return r;
}

// Conservative test: does the support ellipse {p <= L} of a splat (mean m,
// conic (a, b, c)) reach the box of pixel centres [x0,x1] x [y0,y1]? The
// minimum of the convex p over the box is at the mean if it lies inside,
// else on an edge (1-D minimum clamped to the edge). ia = 1/a, ic = 1/c and
// lim = 1.001 L + 0.01 come precomputed in the record (fields 21..23); the
// padding keeps float32 rounding of the per-pixel test from passing where
// this one fails.
__device__ __forceinline__ bool ellipse_meets_box(float mx, float my, float a, float b, float c, float ia, float ic,
                                                  float lim, float x0, float x1, float y0, float y1) {
    // both cases evaluated, no early return: the lanes of a warp do not diverge
    const bool inside = (mx >= x0) & (mx <= x1) & (my >= y0) & (my <= y1);
    float best = 3.0e38f;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dx = (e ? x1 : x0) - mx;
        const float dy = fminf(fmaxf(-b * dx * ic, y0 - my), y1 - my);
        best = fminf(best, 0.5f * (a * dx * dx + c * dy * dy) + b * dx * dy);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dy = (e ? y1 : y0) - my;
        const float dx = fminf(fmaxf(-b * dy * ia, x0 - mx), x1 - mx);
        best = fminf(best, 0.5f * (a * dx * dx + c * dy * dy) + b * dx * dy);
    }
    return inside | (best <= lim);
}

// Bit w set: the splat can reach warp w's SW x SH sub-tile of this tile
// (sub-tiles numbered row-major, TILE / SW across).
template <int TILE, int SW = 8, int SH = 4>
__device__ __forceinline__ uint32_t subtile_mask(const sssgs_pair& P, int tile, float4 g0, float4 g1, float4 g5) {
    constexpr int PER_ROW = TILE / SW, NW = (TILE / SW) * (TILE / SH);
    const int lt = tile - P.tile_offset;
    const float bx = (float)((lt % P.tiles_x) * TILE) + 0.5f, by = (float)((lt / P.tiles_x) * TILE) + 0.5f;
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const float x0 = bx + (float)((w % PER_ROW) * SW), y0 = by + (float)((w / PER_ROW) * SH);
        if (ellipse_meets_box(g0.x, g0.y, g0.z, g0.w, g1.x, g5.y, g5.z, g5.w, x0, x0 + (float)(SW - 1), y0,
                              y0 + (float)(SH - 1)))
            m |= 1u << w;
    }
    return m;
}

__device__ __forceinline__ void load_pair_shared(const sssgs_pair* __restrict__ pairs, int n_pairs, int tile,
                                                 sssgs_pair* sP) {
    if (threadIdx.x < 32) {
        int p = pair_of_tile(pairs, n_pairs, tile);
        reinterpret_cast<float4*>(sP)[threadIdx.x & 7] = reinterpret_cast<const float4*>(pairs + p)[threadIdx.x & 7];
    }
    __syncthreads();
}

// cp.async wrappers (16-byte copies into shared memory, groups, waits).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace sssgs
