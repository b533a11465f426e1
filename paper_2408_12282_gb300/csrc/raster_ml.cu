// Many lights per view: fused composite + shade, forward and backward, for a
// camera view rendered under n_lights point lights at once.
//
// A light-stage training batch holds one view under several lights (Sec. 4.1
// "Dataset"), and a relit view under an environment map is a weighted sum of
// such OLAT renders (App. C "Image Based Lighting"). Everything geometric is
// the same for all lights of a view: the projection, the tile lists and every
// alpha of the compositing (Eq. 3), hence also the compositing weights
// w_i = T_i alpha_i. Only the network output (L_SSS, L_in; Eq. 6) differs per
// light, and the shading (Eq. 4, Eq. 7) with it. So a pixel walks its tile's
// list once, accumulates the 11 light-independent features (depth, n, base,
// rough, metal, sss, vis) once and the four light channels (L_SSS, L_in) of
// every light, then shades each light. The result equals rendering each
// (view, light) pair on its own.
//
// Kernels: one 32-thread block per 8 x 4 sub-tile of a 16 x 16 tile, one pixel
// per lane; the tile's list is walked in batches of 32 splats whose records
// and per-light network outputs arrive by cp.async into a double buffer; a
// ballot of the exact sub-tile test lists the splats to visit. The backward
// replays each pixel back to front from the stored final T with the summed
// per-light upstream gradients; per-splat gradients are reduced over the
// warp through a shared-memory transpose, light-independent ones into the
// view's gradient records, per-light ones into the network-output gradient
// rows of the (view, light) pairs.
#include "raster_common.cuh"

namespace sssgs {
namespace {

constexpr int ML_TILE = 16, ML_NSUB = 8;          // 8 x 4 sub-tiles of a 16 x 16 tile
constexpr int ML_GEO = 12;                        // view G-buffer: depth, n 3, base 3, rough, metal, sss, vis, T
constexpr uint32_t ML_NONE = 0xFFFFFFFFu;

// Row of the (view, light) network output holding light l of view item `it`
// (pair v * L + l of the pair table: view v's camera and scene, light l).
__device__ __forceinline__ int64_t ml_row(const sssgs_pair& V, int L, int l, int64_t it) {
    return it + (int64_t)(L - 1) * V.item_offset + (int64_t)l * V.g_count;
}

// Pixel of (view, light l) in the pair-ordered image layout.
__device__ __forceinline__ int64_t ml_pair_pixel(const sssgs_pair& V, int L, int l, int i, int j) {
    return (int64_t)L * V.pixel_offset + (int64_t)l * V.W * V.H + (int64_t)j * V.W + i;
}

// The 15 features of light l in the layout shade_px_at takes.
template <int L>
__device__ __forceinline__ void ml_features(const float* geo, float vis, const float (&lf)[L][4], int l, float* F) {
#pragma unroll
    for (int k = 0; k < 10; ++k) F[k] = geo[k];
#pragma unroll
    for (int c = 0; c < 4; ++c) F[10 + c] = lf[l][c];
    F[14] = vis;
}

#ifndef SSSGS_ML_BWD_BLOCKS8      // resident one-warp blocks per SM the L = 8 backward is built for
#define SSSGS_ML_BWD_BLOCKS8 8
#endif
template <int L>
struct MlBlocks {
    static constexpr int FWD = L <= 2 ? 16 : (L == 4 ? 14 : 10);
    static constexpr int BWD = L <= 2 ? 16 : (L == 4 ? 12 : SSSGS_ML_BWD_BLOCKS8);
};

// Record float4s the many-light kernels read: 0..3 and 5 (4 holds L_SSS, L_in,
// which live in the per-light network output instead).
__device__ __forceinline__ int ml_rec_q(int q) { return q < 4 ? q : 5; }

template <int L>
__global__ void __launch_bounds__(32, MlBlocks<L>::FWD) k_render_ml_fwd(
    sssgs_cfg cfg, const sssgs_pair* __restrict__ views, int n_views, const float* __restrict__ lights,
    const float4* __restrict__ rec, const float4* __restrict__ mlp_out, const uint32_t* __restrict__ vals,
    const uint2* __restrict__ ranges, float* __restrict__ gbuf, uint32_t* __restrict__ last,
    float* __restrict__ img, const float* __restrict__ env_w, unsigned long long* __restrict__ stats) {
    constexpr int GB = ML_GEO + 4 * L;
    __shared__ __align__(16) float4 s_rec[2][5][32];     // record float4s 0..3, 5
    __shared__ __align__(16) float4 s_lf[2][L][32];
    __shared__ __align__(16) sssgs_pair sP;
    __shared__ float s_light[L * 3];
    const int tile = blockIdx.x / ML_NSUB, sub = blockIdx.x % ML_NSUB;
    const int lane = threadIdx.x;
    const int vi = pair_of_tile(views, n_views, tile);
    if (lane < 8) reinterpret_cast<float4*>(&sP)[lane] = reinterpret_cast<const float4*>(views + vi)[lane];
    for (int k = lane; k < 3 * L; k += 32) s_light[k] = lights[(int64_t)vi * 3 * L + k];
    __syncwarp();
    const int lt = tile - sP.tile_offset;
    const int bx = (lt % sP.tiles_x) * ML_TILE + (sub & 1) * 8, by = (lt / sP.tiles_x) * ML_TILE + (sub >> 1) * 4;
    const int i = bx + (lane & 7), j = by + (lane >> 3);
    const bool inside = i < sP.W && j < sP.H;
    const uint2 rg = ranges[tile];
    const float a_min = cfg.alpha_min, a_max = cfg.alpha_max, T_min = cfg.T_min;
    const float x0 = bx + 0.5f, y0 = by + 0.5f, px = i + 0.5f, py = j + 0.5f;
    // Accumulators as component pairs for the paired FP32 FMA (each component
    // rounds as a scalar fmaf): geometry features (2k, 2k+1), light channels
    // (0, 1) and (2, 3) of every light.
    float T = 1.f, vis = 0.f;
    float2 geo2[5], lf2[L][2];
#pragma unroll
    for (int k = 0; k < 5; ++k) geo2[k] = make_float2(0.f, 0.f);
#pragma unroll
    for (int l = 0; l < L; ++l) lf2[l][0] = lf2[l][1] = make_float2(0.f, 0.f);
    uint32_t lastc = 0, stop = inside ? rg.y : rg.x, n_use = 0;
    bool done = !inside;
    const int nb = (int)((rg.y - rg.x + 31) >> 5);
    auto entry = [&](int t) -> uint32_t {
        if (t >= nb) return ML_NONE;
        const uint32_t idx = rg.x + 32u * t + lane;
        return idx < rg.y ? vals[idx] : ML_NONE;
    };
    auto fetch = [&](uint32_t item, int buf) {
        if (item != ML_NONE) {
            const float4* r = rec + 6 * (int64_t)item;
#pragma unroll
            for (int q = 0; q < 5; ++q)
                cp_async16((uint32_t)__cvta_generic_to_shared(&s_rec[buf][q][lane]), r + ml_rec_q(q));
#pragma unroll
            for (int l = 0; l < L; ++l)
                cp_async16((uint32_t)__cvta_generic_to_shared(&s_lf[buf][l][lane]), mlp_out + ml_row(sP, L, l, item));
        }
        cp_async_commit();
    };
    if (nb > 0 && !__all_sync(SSSGS_FULL, done)) {
        uint32_t it0 = entry(0);
        fetch(it0, 0);
        uint32_t it1 = entry(1);
        for (int t = 0; t < nb; ++t) {
            const int buf = t & 1;
            fetch(it1, buf ^ 1);
            const uint32_t it2 = entry(t + 2);
            cp_async_wait1();
            bool pass = false;
            if (it0 != ML_NONE) {
                const float4 g0 = s_rec[buf][0][lane], g1 = s_rec[buf][1][lane], g5 = s_rec[buf][4][lane];
                pass = ellipse_meets_box(g0.x, g0.y, g0.z, g0.w, g1.x, g5.y, g5.z, g5.w, x0, x0 + 7.f, y0, y0 + 3.f);
            }
            uint32_t bits = __ballot_sync(SSSGS_FULL, pass);
            __syncwarp();
            const uint32_t base = rg.x + 32u * t;
            while (bits) {
                const int k = __ffs(bits) - 1;
                bits &= bits - 1;
                // warp-uniform visit: a lane that does not take the splat adds
                // weight 0 (exact: the sums are never -0), so lanes never diverge
                const float4 g0 = s_rec[buf][0][k], g1 = s_rec[buf][1][k];
                const AlphaEval e = eval_alpha(g0, g1, px, py, a_min, a_max);
                bool u = !done && e.use;
                const float Tn = T * (1.f - e.alpha);
                if (u && Tn < T_min) {
                    done = true;
                    stop = base + k + 1;
                    u = false;
                }
                if (!__any_sync(SSSGS_FULL, u)) continue;
                n_use += (uint32_t)u;
                const float w = u ? T * e.alpha : 0.f;
                const float2 ww = make_float2(w, w);
                const float4 g2 = s_rec[buf][2][k], g3 = s_rec[buf][3][k];
                geo2[0] = __ffma2_rn(ww, make_float2(g1.z, g1.w), geo2[0]);
                geo2[1] = __ffma2_rn(ww, make_float2(g2.x, g2.y), geo2[1]);
                geo2[2] = __ffma2_rn(ww, make_float2(g2.z, g2.w), geo2[2]);
                geo2[3] = __ffma2_rn(ww, make_float2(g3.x, g3.y), geo2[3]);
                geo2[4] = __ffma2_rn(ww, make_float2(g3.z, g3.w), geo2[4]);
                vis = __fmaf_rn(w, s_rec[buf][4][k].x, vis);
#pragma unroll
                for (int l = 0; l < L; ++l) {
                    const float4 v = s_lf[buf][l][k];
                    lf2[l][0] = __ffma2_rn(ww, make_float2(v.x, v.y), lf2[l][0]);
                    lf2[l][1] = __ffma2_rn(ww, make_float2(v.z, v.w), lf2[l][1]);
                }
                T = u ? Tn : T;
                lastc = u ? base + k + 1 : lastc;
            }
            if (__all_sync(SSSGS_FULL, done)) break;
            __syncwarp();
            it0 = it1;
            it1 = it2;
        }
        cp_async_wait_all();
    }
    if (stats) {
        unsigned long long u = n_use, v = stop - rg.x;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            u += __shfl_xor_sync(SSSGS_FULL, u, o);
            v += __shfl_xor_sync(SSSGS_FULL, v, o);
        }
        if (lane == 0) {
            atomicAdd(stats, u);
            atomicAdd(stats + 1, v);
        }
    }
    if (!inside) return;
    float geo[10], lf[L][4];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        geo[2 * k] = geo2[k].x;
        geo[2 * k + 1] = geo2[k].y;
    }
#pragma unroll
    for (int l = 0; l < L; ++l) {
        lf[l][0] = lf2[l][0].x;
        lf[l][1] = lf2[l][0].y;
        lf[l][2] = lf2[l][1].x;
        lf[l][3] = lf2[l][1].y;
    }
    const int64_t vpix = sP.pixel_offset + (int64_t)j * sP.W + i;
    float4* go = reinterpret_cast<float4*>(gbuf + (int64_t)GB * vpix);
    go[0] = make_float4(geo[0], geo[1], geo[2], geo[3]);
    go[1] = make_float4(geo[4], geo[5], geo[6], geo[7]);
    go[2] = make_float4(geo[8], geo[9], vis, T);
#pragma unroll
    for (int l = 0; l < L; ++l) go[3 + l] = make_float4(lf[l][0], lf[l][1], lf[l][2], lf[l][3]);
    last[vpix] = lastc;
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int l = 0; l < L; ++l) {
        float F[SSSGS_NF], o[3];
        ml_features<L>(geo, vis, lf, l, F);
        shade_px_at<false>(F, T, px, py, sP, make_float3(s_light[3 * l], s_light[3 * l + 1], s_light[3 * l + 2]),
                           cfg.A_eps, o, nullptr, nullptr, nullptr);
        if (env_w) {
            const float we = env_w[(int64_t)vi * L + l];
            acc[0] += we * o[0];
            acc[1] += we * o[1];
            acc[2] += we * o[2];
        } else {
            const int64_t q = ml_pair_pixel(sP, L, l, i, j);
            img[3 * q] = o[0];
            img[3 * q + 1] = o[1];
            img[3 * q + 2] = o[2];
        }
    }
    if (env_w) {
        img[3 * vpix] = acc[0];
        img[3 * vpix + 1] = acc[1];
        img[3 * vpix + 2] = acc[2];
    }
}

// Backward. Per pixel, the shading backward of every light gives dL/dF: the
// light-independent part summed over the lights (dgeo 10), the light
// channels per light (dlf), and dL/dT_final summed. The replay then follows
// the single-light kernel: T_i = T_{i+1} / (1 - alpha_i), dL/dalpha_i =
// T_i (dF . f_i) - Q / (1 - alpha_i), Q accumulating w (dF . f) from
// dL/dT_final * T_final, with dF . f running over the 10 + 4 L channels the
// shading reads.
// Reduction rows per splat: 0..5 geometry (mean 2, conic 3, opacity),
// 6..15 the ten light-independent features, 16 + 4 l + c light l's channel c.
// The visibility channel has no row: the shading does not read it, so its
// upstream gradient is exactly zero (the caller's cleared drec keeps it).
template <int L>
__global__ void __launch_bounds__(32, MlBlocks<L>::BWD) k_render_ml_bwd(
    sssgs_cfg cfg, const sssgs_pair* __restrict__ views, int n_views, const float* __restrict__ lights,
    const float4* __restrict__ rec, const float4* __restrict__ mlp_out, const uint32_t* __restrict__ vals,
    const uint2* __restrict__ ranges, const float* __restrict__ gbuf, const uint32_t* __restrict__ last,
    const float* __restrict__ img, const float* __restrict__ dimg, const float* __restrict__ target,
    float l1_scale, float* __restrict__ drec, float* __restrict__ dmlp, unsigned long long* __restrict__ stats) {
    constexpr int GB = ML_GEO + 4 * L, NG = 16 + 4 * L, RS = 36;
    constexpr int NR = NG < 32 ? NG : 32;                 // rows the transpose buffer holds at once
    __shared__ __align__(16) float4 s_rec[2][5][32];     // record float4s 0..3, 5
    __shared__ __align__(16) float4 s_lf[2][L][32];
    __shared__ uint32_t s_item[2][32];
    __shared__ __align__(16) float s_red[NR * RS];
    __shared__ __align__(16) sssgs_pair sP;
    __shared__ float s_light[L * 3];
    const int tile = blockIdx.x / ML_NSUB, sub = blockIdx.x % ML_NSUB;
    const int lane = threadIdx.x;
    const int vi = pair_of_tile(views, n_views, tile);
    if (lane < 8) reinterpret_cast<float4*>(&sP)[lane] = reinterpret_cast<const float4*>(views + vi)[lane];
    for (int k = lane; k < 3 * L; k += 32) s_light[k] = lights[(int64_t)vi * 3 * L + k];
    __syncwarp();
    const int lt = tile - sP.tile_offset;
    const int bx = (lt % sP.tiles_x) * ML_TILE + (sub & 1) * 8, by = (lt / sP.tiles_x) * ML_TILE + (sub >> 1) * 4;
    const int i = bx + (lane & 7), j = by + (lane >> 3);
    const bool inside = i < sP.W && j < sP.H;
    const uint2 rg = ranges[tile];
    const float px = i + 0.5f, py = j + 0.5f;
    // per-pixel upstream: shading backward of every light
    float dgeo[10], dlf[L][4], T = 1.f, Q = 0.f;
    uint32_t lastc = 0;
#pragma unroll
    for (int k = 0; k < 10; ++k) dgeo[k] = 0.f;
#pragma unroll
    for (int l = 0; l < L; ++l)
#pragma unroll
        for (int c = 0; c < 4; ++c) dlf[l][c] = 0.f;
    if (inside) {
        const int64_t vpix = sP.pixel_offset + (int64_t)j * sP.W + i;
        lastc = last[vpix];
        const float4* gi = reinterpret_cast<const float4*>(gbuf + (int64_t)GB * vpix);
        float geo[10], lfv[L][4];
        const float4 a = gi[0], b = gi[1], c2 = gi[2];
        geo[0] = a.x; geo[1] = a.y; geo[2] = a.z; geo[3] = a.w;
        geo[4] = b.x; geo[5] = b.y; geo[6] = b.z; geo[7] = b.w;
        geo[8] = c2.x; geo[9] = c2.y;
        const float vs = c2.z;
        T = c2.w;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const float4 v = gi[3 + l];
            lfv[l][0] = v.x; lfv[l][1] = v.y; lfv[l][2] = v.z; lfv[l][3] = v.w;
        }
        float dT = 0.f;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const int64_t q = ml_pair_pixel(sP, L, l, i, j);
            float g3[3];
            if (dimg) {
                g3[0] = dimg[3 * q]; g3[1] = dimg[3 * q + 1]; g3[2] = dimg[3 * q + 2];
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float d = img[3 * q + c] - target[3 * q + c];
                    g3[c] = d > 0.f ? l1_scale : (d < 0.f ? -l1_scale : 0.f);
                }
            }
            float F[SSSGS_NF], dF[SSSGS_NF], o[3], dTl;
            ml_features<L>(geo, vs, lfv, l, F);
            shade_px_at<true>(F, T, px, py, sP, make_float3(s_light[3 * l], s_light[3 * l + 1], s_light[3 * l + 2]),
                              cfg.A_eps, o, g3, dF, &dTl);
#pragma unroll
            for (int k = 0; k < 10; ++k) dgeo[k] += dF[k];
#pragma unroll
            for (int c = 0; c < 4; ++c) dlf[l][c] = dF[10 + c];
            dT += dTl;
        }
        Q = dT * T;
    }
    const uint32_t wmax = __reduce_max_sync(SSSGS_FULL, lastc);
    const float a_min = cfg.alpha_min, a_max = cfg.alpha_max;
    const float x0 = bx + 0.5f, y0 = by + 0.5f;
    uint32_t n_use = 0;
    if (wmax > rg.x) {
        const int nb = (int)((wmax - rg.x + 31) >> 5);
        auto entry = [&](int t) -> uint32_t {
            if (t >= nb) return ML_NONE;
            const int64_t hi = (int64_t)wmax - 32 * t, lo = max((int64_t)rg.x, hi - 32);
            const int64_t idx = lo + lane;
            return idx < hi ? vals[idx] : ML_NONE;
        };
        auto fetch = [&](uint32_t item, int buf) {
            if (item != ML_NONE) {
                const float4* r = rec + 6 * (int64_t)item;
#pragma unroll
                for (int q = 0; q < 5; ++q)
                    cp_async16((uint32_t)__cvta_generic_to_shared(&s_rec[buf][q][lane]), r + ml_rec_q(q));
#pragma unroll
                for (int l = 0; l < L; ++l)
                    cp_async16((uint32_t)__cvta_generic_to_shared(&s_lf[buf][l][lane]),
                               mlp_out + ml_row(sP, L, l, item));
            }
            cp_async_commit();
        };
        uint32_t it0 = entry(0);
        fetch(it0, 0);
        uint32_t it1 = entry(1);
        for (int t = 0; t < nb; ++t) {
            const int buf = t & 1;
            fetch(it1, buf ^ 1);
            const uint32_t it2 = entry(t + 2);
            cp_async_wait1();
            bool pass = false;
            if (it0 != ML_NONE) {
                const float4 g0 = s_rec[buf][0][lane], g1 = s_rec[buf][1][lane], g5 = s_rec[buf][4][lane];
                pass = ellipse_meets_box(g0.x, g0.y, g0.z, g0.w, g1.x, g5.y, g5.z, g5.w, x0, x0 + 7.f, y0, y0 + 3.f);
            }
            s_item[buf][lane] = it0;
            uint32_t bits = __ballot_sync(SSSGS_FULL, pass);
            __syncwarp();
            const uint32_t lo = (uint32_t)max((int64_t)rg.x, (int64_t)wmax - 32 * t - 32);
            while (bits) {
                const int k = 31 - __clz(bits);
                bits ^= 1u << k;
                const uint32_t pos = lo + k;
                const float4 g0 = s_rec[buf][0][k], g1 = s_rec[buf][1][k];
                const AlphaEval e = eval_alpha(g0, g1, px, py, a_min, a_max);
                const bool act = (pos < lastc) && e.use;
                if (!__any_sync(SSSGS_FULL, act)) continue;
                float wk;                              // this lane's compositing weight of the splat
                {
                    const float4 g2 = s_rec[buf][2][k], g3 = s_rec[buf][3][k];
                    const float f[10] = {g1.z, g1.w, g2.x, g2.y, g2.z, g2.w, g3.x, g3.y, g3.z, g3.w};
                    float dot = 0.f;
#pragma unroll
                    for (int kk = 0; kk < 10; ++kk) dot = fmaf(dgeo[kk], f[kk], dot);
#pragma unroll
                    for (int l = 0; l < L; ++l) {
                        const float4 v = s_lf[buf][l][k];
                        dot = fmaf(dlf[l][0], v.x, dot);
                        dot = fmaf(dlf[l][1], v.y, dot);
                        dot = fmaf(dlf[l][2], v.z, dot);
                        dot = fmaf(dlf[l][3], v.w, dot);
                    }
                    const float ia = rcp_newton(1.f - e.alpha);
                    const float Ti = T * ia;
                    const float da = Ti * dot - Q * ia;
                    const bool geo_ok = act && !e.clamped;
                    const float w = act ? e.alpha * Ti : 0.f;
                    const float dp = geo_ok ? -da * e.alpha : 0.f;
                    const float dg = geo_ok ? da * e.G : 0.f;
                    Q = fmaf(w, dot, Q);
                    T = act ? Ti : T;
                    n_use += (uint32_t)act;
                    float* col = s_red + lane;
                    const float dx = e.dx, dy = e.dy;
                    const float ca = g0.z, cb = g0.w, cc = g1.x;
                    col[0] = dp * (ca * dx + cb * dy);
                    col[RS] = dp * (cb * dx + cc * dy);
                    col[2 * RS] = 0.5f * dx * dx * dp;
                    col[3 * RS] = dx * dy * dp;
                    col[4 * RS] = 0.5f * dy * dy * dp;
                    col[5 * RS] = dg;
#pragma unroll
                    for (int kk = 0; kk < 10; ++kk) col[(6 + kk) * RS] = w * dgeo[kk];
                    if constexpr (NG <= NR) {          // all rows in one transpose
#pragma unroll
                        for (int l = 0; l < L; ++l)
#pragma unroll
                            for (int c = 0; c < 4; ++c) col[(16 + 4 * l + c) * RS] = w * dlf[l][c];
                    }
                    wk = w;
                }
                __syncwarp();
                const uint32_t item = s_item[buf][k];
                // sum of the 32 lanes' terms of row r of the transpose buffer
                auto row_sum = [&](int r) -> float {
                    const float4* row = reinterpret_cast<const float4*>(s_red + r * RS);
                    float2 a[16];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 v = row[q];
                        a[2 * q] = make_float2(v.x, v.y);
                        a[2 * q + 1] = make_float2(v.z, v.w);
                    }
#pragma unroll
                    for (int h = 8; h >= 1; h >>= 1)
#pragma unroll
                        for (int q = 0; q < h; ++q) a[q] = __fadd2_rn(a[q], a[q + h]);
                    return a[0].x + a[0].y;
                };
                auto light_add = [&](int r, float sum) {   // light row r = 4 l + c
                    atomicAdd(dmlp + 4 * ml_row(sP, L, r >> 2, item) + (r & 3), sum);
                };
                if (lane < 16) {
                    atomicAdd(drec + (int64_t)SSSGS_REC * item + lane, row_sum(lane));
                } else if (NG <= NR && lane < NG) {
                    light_add(lane - 16, row_sum(lane));
                }
                if constexpr (NG > NR) {               // light channels in a second transpose
                    __syncwarp();
#pragma unroll
                    for (int l = 0; l < L; ++l)
#pragma unroll
                        for (int c = 0; c < 4; ++c) s_red[(4 * l + c) * RS + lane] = wk * dlf[l][c];
                    __syncwarp();
                    if (lane < 4 * L) light_add(lane, row_sum(lane));
                }
                __syncwarp();
            }
            __syncwarp();
            it0 = it1;
            it1 = it2;
        }
    }
    if (stats) {
        unsigned long long u = n_use, v = lastc > rg.x ? lastc - rg.x : 0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            u += __shfl_xor_sync(SSSGS_FULL, u, o);
            v += __shfl_xor_sync(SSSGS_FULL, v, o);
        }
        if (lane == 0) {
            atomicAdd(stats, u);
            atomicAdd(stats + 1, v);
        }
    }
}

int ml_tiles(const sssgs_pair* h, int n) { return h[n - 1].tile_offset + h[n - 1].tiles_x * h[n - 1].tiles_y; }

bool ml_args_ok(const sssgs_cfg* cfg, const sssgs_pair* h, const sssgs_pair* d, int n, int L, const float* lights,
                const float* rec, const float* mlp_out, const uint32_t* vals, const uint32_t* ranges,
                const void* gbuf, const uint32_t* last) {
    if (!cfg || !h || !d || n <= 0 || !lights || !rec || !mlp_out || !vals || !ranges || !gbuf || !last) return false;
    if (!(L == 1 || L == 2 || L == 4 || L == 8)) return false;
    if (((uintptr_t)rec & 15) || ((uintptr_t)mlp_out & 15) || ((uintptr_t)gbuf & 15) || ((uintptr_t)ranges & 7))
        return false;
    return true;
}

template <int L>
int launch_ml_fwd(const sssgs_cfg* cfg, const sssgs_pair* d, int n, int tiles, const float* lights, const float* rec,
                  const float* mlp_out, const uint32_t* vals, const uint32_t* ranges, float* gbuf, uint32_t* last,
                  float* img, const float* env_w, uint64_t* stats, cudaStream_t st) {
    k_render_ml_fwd<L><<<(unsigned)tiles * ML_NSUB, 32, 0, st>>>(
        *cfg, d, n, lights, reinterpret_cast<const float4*>(rec), reinterpret_cast<const float4*>(mlp_out), vals,
        reinterpret_cast<const uint2*>(ranges), gbuf, last, img, env_w, reinterpret_cast<unsigned long long*>(stats));
    sssgs::note_launches(1);
    return launch_status();
}

template <int L>
int launch_ml_bwd(const sssgs_cfg* cfg, const sssgs_pair* d, int n, int tiles, const float* lights, const float* rec,
                  const float* mlp_out, const uint32_t* vals, const uint32_t* ranges, const float* gbuf,
                  const uint32_t* last, const float* img, const float* dimg, const float* target, float l1_scale,
                  float* drec, float* dmlp, uint64_t* stats, cudaStream_t st) {
    k_render_ml_bwd<L><<<(unsigned)tiles * ML_NSUB, 32, 0, st>>>(
        *cfg, d, n, lights, reinterpret_cast<const float4*>(rec), reinterpret_cast<const float4*>(mlp_out), vals,
        reinterpret_cast<const uint2*>(ranges), gbuf, last, img, dimg, target, l1_scale, drec, dmlp,
        reinterpret_cast<unsigned long long*>(stats));
    sssgs::note_launches(1);
    return launch_status();
}

}  // namespace
}  // namespace sssgs

using namespace sssgs;

extern "C" int sssgs_render_ml_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_views, const sssgs_pair* d_views,
                                   int n_views, int n_lights, const float* lights, const float* rec,
                                   const float* mlp_out, const uint32_t* vals, const uint32_t* ranges, float* gbuf,
                                   uint32_t* last, float* img, const float* env_w, uint64_t* d_stats,
                                   sssgs_stream stream) {
    if (!ml_args_ok(cfg, h_views, d_views, n_views, n_lights, lights, rec, mlp_out, vals, ranges, gbuf, last) || !img)
        return SSSGS_ERR_INVALID_ARG;
    if (cfg->tile != ML_TILE) return SSSGS_ERR_UNSUPPORTED;
    const int tiles = ml_tiles(h_views, n_views);
    if (tiles == 0) return SSSGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    switch (n_lights) {
        case 1: return launch_ml_fwd<1>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, env_w, d_stats, st);
        case 2: return launch_ml_fwd<2>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, env_w, d_stats, st);
        case 4: return launch_ml_fwd<4>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, env_w, d_stats, st);
        default: return launch_ml_fwd<8>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, env_w, d_stats, st);
    }
}

extern "C" int sssgs_render_ml_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_views, const sssgs_pair* d_views,
                                   int n_views, int n_lights, const float* lights, const float* rec,
                                   const float* mlp_out, const uint32_t* vals, const uint32_t* ranges,
                                   const float* gbuf, const uint32_t* last, const float* img, const float* dimg,
                                   const float* target, float l1_scale, float* drec, float* dmlp, uint64_t* d_stats,
                                   sssgs_stream stream) {
    if (!ml_args_ok(cfg, h_views, d_views, n_views, n_lights, lights, rec, mlp_out, vals, ranges, gbuf, last) ||
        !drec || !dmlp || (!dimg && (!img || !target)))
        return SSSGS_ERR_INVALID_ARG;
    if (cfg->tile != ML_TILE) return SSSGS_ERR_UNSUPPORTED;
    const int tiles = ml_tiles(h_views, n_views);
    if (tiles == 0) return SSSGS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    switch (n_lights) {
        case 1: return launch_ml_bwd<1>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, dimg, target, l1_scale, drec, dmlp, d_stats, st);
        case 2: return launch_ml_bwd<2>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, dimg, target, l1_scale, drec, dmlp, d_stats, st);
        case 4: return launch_ml_bwd<4>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, dimg, target, l1_scale, drec, dmlp, d_stats, st);
        default: return launch_ml_bwd<8>(cfg, d_views, n_views, tiles, lights, rec, mlp_out, vals, ranges, gbuf, last, img, dimg, target, l1_scale, drec, dmlp, d_stats, st);
    }
}
