// Per-pixel compositing (Eq. 3) into the deferred G-buffer and deferred
// shading (Eq. 4, Eq. 7), forward and backward.
//
// The fused kernels run one 32-thread block per 8 x 8 sub-tile of an image
// tile, two pixels per lane. Each walks its tile's depth-ordered instance
// list in batches: every lane loads packed 96-B records (six 16-B copies)
// into a shared-memory double buffer, a ballot of the lanes' sub-tile tests
// lists the splats the warp visits, and the warp reads each visited record
// by broadcast. The forward stops a pixel when its transmittance would drop
// below T_min and the warp once all its pixels have stopped.
//
// The backward replays each pixel's list back to front starting from the final
// transmittance stored by the forward (T_i = T_{i+1} / (1 - alpha_i)), so no
// per-pixel list is kept. Per-Gaussian gradients are summed over the pixels
// of a warp through a shared-memory transpose (each lane stores its values in
// a column, lane k then sums row k with eight 16-byte loads) and issued as
// one fire-and-forget add per reduced row and warp, instead of one atomic per
// pixel. A block-per-tile backward (one thread per pixel) serves the unfused
// path, whose upstream is a G-buffer gradient.
#include "raster_common.cuh"

// Resident one-warp blocks per SM the fused kernels are built for (the
// register cap follows): the forward at 32, the SM's block limit (64
// registers, a small spill), measured faster than 20-28; the backward at 20
// (96 registers), measured faster than 24.
#ifndef SSSGS_FWD_MINB
#define SSSGS_FWD_MINB 32
#endif
#ifndef SSSGS_BWD_MINB
#define SSSGS_BWD_MINB 20
#endif

namespace sssgs {

// ---------------------------------------------------------------- composite forward, one warp per sub-tile
//
// Each block is a single warp that owns an 8 x 8 sub-tile of a TILE x TILE
// tile (TILE = 8, 16 or 32: (TILE/8)^2 sub-tiles per tile); there is no
// block barrier and a warp stops as soon as its own pixels are done. The
// tile's list is walked front to back in batches of BATCH splats (32 or 64:
// one or two per lane) through a cp.async double buffer in shared memory; a
// ballot of each lane's exact sub-tile test lists the splats the warp visits.

// Sub-tile origin of block `blk` for SW x SH sub-tiles of TILE x TILE tiles.
template <int TILE, int SW, int SH>
struct SubTile {
    static constexpr int PER_ROW = TILE / SW, NSUB = (TILE / SW) * (TILE / SH);
    int tile, bx, by;
    __device__ __forceinline__ SubTile(int blk, const sssgs_pair& P) {
        tile = blk / NSUB;
        const int sub = blk - tile * NSUB;
        const int lt = tile - P.tile_offset;
        bx = (lt % P.tiles_x) * TILE + (sub % PER_ROW) * SW;
        by = (lt / P.tiles_x) * TILE + (sub / PER_ROW) * SH;
    }
};

// Lane l holds pixels (l & 7, 2 (l >> 3)) and the one below, as in the
// backward. A visited splat's records are read once for both pixels, the
// two alpha evaluations share their column terms and run as paired FP32
// instructions, the G-buffer sums advance as pairs (one paired FMA per
// feature) and the two pixels' chains are independent work for the
// scheduler. A pixel that does not take the splat adds w = 0 (F + 0 * g = F
// exactly: F is never -0), so each pixel's float32 result is the one a lane
// of its own would compute, and the warp skips a visit only when none of its
// pixels takes the splat: lanes never diverge inside a visit.
template <int TILE, int BATCH, bool SHADE, bool STATS>
__global__ void __launch_bounds__(32, SSSGS_FWD_MINB) k_composite_fwd_warp(sssgs_cfg cfg, const sssgs_pair* __restrict__ pairs,
                                                              int n_pairs, const float4* __restrict__ rec,
                                                              const uint32_t* __restrict__ vals,
                                                              const uint2* __restrict__ ranges,
                                                              float* __restrict__ gbuf, uint32_t* __restrict__ last,
                                                              float* __restrict__ img,
                                                              unsigned long long* __restrict__ stats) {
    constexpr int R = BATCH / 32;                 // records per lane per batch
    using ST = SubTile<TILE, 8, 8>;
    constexpr uint32_t NONE = 0xFFFFFFFFu;
    __shared__ __align__(16) float4 s_rec[2][6][BATCH];
    __shared__ __align__(16) sssgs_pair sP;
    const int lane = threadIdx.x;
    if (lane < 8) {
        const int pi = pair_of_tile(pairs, n_pairs, (int)(blockIdx.x / ST::NSUB));
        reinterpret_cast<float4*>(&sP)[lane] = reinterpret_cast<const float4*>(pairs + pi)[lane];
    }
    __syncwarp();
    const ST st(blockIdx.x, sP);
    const int tile = st.tile, bx = st.bx, by = st.by;
    const int i = bx + (lane & 7), j0 = by + (lane >> 3) * 2;
    const uint2 rg = ranges[tile];
    const float a_min = cfg.alpha_min, a_max = cfg.alpha_max, T_min = cfg.T_min;
    const float x0 = bx + 0.5f, y0 = by + 0.5f;
    const float px = (float)i + 0.5f, py0 = (float)j0 + 0.5f, py1 = py0 + 1.f;
    const bool in0 = i < sP.W && j0 < sP.H, in1 = i < sP.W && j0 + 1 < sP.H;
    float2 F[SSSGS_NF];                           // (pixel 0, pixel 1) of each G-buffer channel
    float T0 = 1.f, T1 = 1.f;
    uint32_t last0 = 0, last1 = 0;
    bool done0 = !in0, done1 = !in1;
    uint32_t stop0 = done0 ? rg.x : rg.y, stop1 = done1 ? rg.x : rg.y;   // read only with STATS
#pragma unroll
    for (int k = 0; k < SSSGS_NF; ++k) F[k] = make_float2(0.f, 0.f);
    uint32_t n_use = 0;
    const int nb = (int)((rg.y - rg.x + BATCH - 1) / BATCH);
    auto entry = [&](int t, int r) -> uint32_t {
        if (t >= nb) return NONE;
        const uint32_t idx = rg.x + (uint32_t)BATCH * t + 32u * r + lane;
        return idx < rg.y ? vals[idx] : NONE;
    };
    auto fetch = [&](const uint32_t* item, int buf) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (item[r] != NONE) {
                const float4* src = rec + 6 * (int64_t)item[r];
#pragma unroll
                for (int q = 0; q < 6; ++q)
                    cp_async16((uint32_t)__cvta_generic_to_shared(&s_rec[buf][q][32 * r + lane]), src + q);
            }
        }
        cp_async_commit();
    };
    if (nb > 0 && !__all_sync(SSSGS_FULL, done0 && done1)) {
        uint32_t it0[R], it1[R], it2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) it0[r] = entry(0, r);
        fetch(it0, 0);
#pragma unroll
        for (int r = 0; r < R; ++r) it1[r] = entry(1, r);
        for (int t = 0; t < nb; ++t) {
            const int buf = t & 1;
            fetch(it1, buf ^ 1);
#pragma unroll
            for (int r = 0; r < R; ++r) it2[r] = entry(t + 2, r);
            cp_async_wait1();
            uint32_t bits[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                // every slot is tested (an empty slot holds stale or
                // unwritten shared data, harmless to compare) and empty ones are masked out
                const int s = 32 * r + lane;
                const float4 g0 = s_rec[buf][0][s], g1 = s_rec[buf][1][s], g5 = s_rec[buf][5][s];
                const bool pass = (it0[r] != NONE) &
                                  ellipse_meets_box(g0.x, g0.y, g0.z, g0.w, g1.x, g5.y, g5.z, g5.w, x0, x0 + 7.f,
                                                    y0, y0 + 7.f);
                bits[r] = __ballot_sync(SSSGS_FULL, pass);
            }
            __syncwarp();
            const uint32_t base = rg.x + (uint32_t)BATCH * t;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                while (bits[r]) {          // warp-uniform loop; finished lanes idle
                    const int k = 32 * r + __ffs(bits[r]) - 1;
                    bits[r] &= bits[r] - 1;
                    const float4 g0 = s_rec[buf][0][k], g1 = s_rec[buf][1][k];
                    AlphaEval e0, e1;
                    eval_alpha2(g0, g1, px, py0, py1, a_min, a_max, e0, e1);
                    bool u0 = !done0 && e0.use, u1 = !done1 && e1.use;
                    const float Tn0 = T0 * (1.f - e0.alpha), Tn1 = T1 * (1.f - e1.alpha);
                    if (u0 && Tn0 < T_min) {
                        done0 = true;
                        if (STATS) stop0 = base + k + 1;
                        u0 = false;
                    }
                    if (u1 && Tn1 < T_min) {
                        done1 = true;
                        if (STATS) stop1 = base + k + 1;
                        u1 = false;
                    }
                    // warp-uniform skip: the lanes never diverge inside a visit
                    if (!__any_sync(SSSGS_FULL, u0 || u1)) continue;
                    if (STATS) n_use += (uint32_t)u0 + (uint32_t)u1;
                    const float2 w = make_float2(u0 ? T0 * e0.alpha : 0.f, u1 ? T1 * e1.alpha : 0.f);
                    const float4 g2 = s_rec[buf][2][k], g3 = s_rec[buf][3][k], g4 = s_rec[buf][4][k];
                    const float g5 = s_rec[buf][5][k].x;
                    const float f[SSSGS_NF] = {g1.z, g1.w, g2.x, g2.y, g2.z, g2.w, g3.x, g3.y,
                                               g3.z, g3.w, g4.x, g4.y, g4.z, g4.w, g5};
#pragma unroll
                    for (int c = 0; c < SSSGS_NF; ++c) F[c] = __ffma2_rn(w, make_float2(f[c], f[c]), F[c]);
                    T0 = u0 ? Tn0 : T0;
                    T1 = u1 ? Tn1 : T1;
                    last0 = u0 ? base + k + 1 : last0;
                    last1 = u1 ? base + k + 1 : last1;
                }
            }
            if (__all_sync(SSSGS_FULL, done0 && done1)) break;
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                it0[r] = it1[r];
                it1[r] = it2[r];
            }
        }
        cp_async_wait_all();
    }
    if (STATS) {   // contributions, and list positions each pixel considered
        unsigned long long u = n_use, v = (unsigned long long)(in0 ? stop0 - rg.x : 0) + (in1 ? stop1 - rg.x : 0);
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
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (!(q ? in1 : in0)) continue;
        const int j = j0 + q;
        const int64_t pix = sP.pixel_offset + (int64_t)j * sP.W + i;
        float Fq[SSSGS_NF];
#pragma unroll
        for (int c = 0; c < SSSGS_NF; ++c) Fq[c] = q ? F[c].y : F[c].x;
        const float T = q ? T1 : T0;
        float4* go = reinterpret_cast<float4*>(gbuf + SSSGS_GBUF * pix);
        go[0] = make_float4(Fq[0], Fq[1], Fq[2], Fq[3]);
        go[1] = make_float4(Fq[4], Fq[5], Fq[6], Fq[7]);
        go[2] = make_float4(Fq[8], Fq[9], Fq[10], Fq[11]);
        go[3] = make_float4(Fq[12], Fq[13], Fq[14], T);
        last[pix] = q ? last1 : last0;
        if (SHADE) {
            float o[3];
            shade_px<false>(Fq, T, px, q ? py1 : py0, sP, cfg.A_eps, o, nullptr, nullptr, nullptr);
            img[3 * pix] = o[0];
            img[3 * pix + 1] = o[1];
            img[3 * pix + 2] = o[2];
        }
    }
}

// ---------------------------------------------------------------- shade only

template <int TILE, bool BWD>
__global__ void __launch_bounds__(TILE * TILE) k_shade(sssgs_cfg cfg, const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                       const float* __restrict__ gbuf, float* __restrict__ img,
                                                       const float* __restrict__ dimg, float* __restrict__ dgbuf) {
    __shared__ __align__(16) sssgs_pair sP;
    const int tile = blockIdx.x;
    load_pair_shared(pairs, n_pairs, tile, &sP);
    const TilePix px = tile_pixel(sP, tile, TILE);
    if (!px.inside) return;
    const float4* gi = reinterpret_cast<const float4*>(gbuf + SSSGS_GBUF * px.pix);
    float F[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float4 v = gi[q];
        F[4 * q] = v.x; F[4 * q + 1] = v.y; F[4 * q + 2] = v.z; F[4 * q + 3] = v.w;
    }
    float o[3];
    if (!BWD) {
        shade_px<false>(F, F[15], px.i + 0.5f, px.j + 0.5f, sP, cfg.A_eps, o, nullptr, nullptr, nullptr);
        img[3 * px.pix] = o[0];
        img[3 * px.pix + 1] = o[1];
        img[3 * px.pix + 2] = o[2];
    } else {
        float g3[3] = {dimg[3 * px.pix], dimg[3 * px.pix + 1], dimg[3 * px.pix + 2]};
        float dF[SSSGS_NF], dT;
        shade_px<true>(F, F[15], px.i + 0.5f, px.j + 0.5f, sP, cfg.A_eps, o, g3, dF, &dT);
        float4* go = reinterpret_cast<float4*>(dgbuf + SSSGS_GBUF * px.pix);
        go[0] = make_float4(dF[0], dF[1], dF[2], dF[3]);
        go[1] = make_float4(dF[4], dF[5], dF[6], dF[7]);
        go[2] = make_float4(dF[8], dF[9], dF[10], dF[11]);
        go[3] = make_float4(dF[12], dF[13], dF[14], dT);
    }
}

// ---------------------------------------------------------------- composite backward

enum { UPSTREAM_DGBUF = 0, UPSTREAM_DIMG = 1, UPSTREAM_L1 = 2 };

#ifndef SSSGS_BWD_MIN_BLOCKS
#define SSSGS_BWD_MIN_BLOCKS 3     // resident CTAs per SM the register budget is sized for
#endif

template <int TILE, int MODE>
__global__ void __launch_bounds__(TILE * TILE, SSSGS_BWD_MIN_BLOCKS) k_composite_bwd(sssgs_cfg cfg, const sssgs_pair* __restrict__ pairs,
                                                               int n_pairs, const float4* __restrict__ rec,
                                                               const uint32_t* __restrict__ vals,
                                                               const uint2* __restrict__ ranges,
                                                               const float* __restrict__ gbuf,
                                                               const uint32_t* __restrict__ last,
                                                               const float* __restrict__ dgbuf,
                                                               const float* __restrict__ img,
                                                               const float* __restrict__ dimg,
                                                               const float* __restrict__ target,
                                                               const float* __restrict__ weight, float l1_scale,
                                                               float* __restrict__ drec,
                                                               unsigned long long* __restrict__ stats) {
    constexpr int B = TILE * TILE;
    constexpr int NG = 6 + SSSGS_NF;                        // gradient components per Gaussian
    constexpr int RS = 36;                                  // row stride of the transpose scratch (floats)
    extern __shared__ float4 s_rec[];                       // [6][B], item ids, masks, reduction scratch
    uint32_t* s_item = reinterpret_cast<uint32_t*>(s_rec + 6 * B);
    uint32_t* s_mask = s_item + B;
    float* s_red = reinterpret_cast<float*>(s_mask + B) + (threadIdx.x >> 5) * (NG * RS);
    const uint32_t wbit = 1u << (threadIdx.x >> 5);
    __shared__ __align__(16) sssgs_pair sP;
    __shared__ uint32_t s_max;
    const int tile = blockIdx.x;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_max = 0;
    load_pair_shared(pairs, n_pairs, tile, &sP);
    const TilePix px = tile_pixel(sP, tile, TILE);
    const float fx = px.i + 0.5f, fy = px.j + 0.5f;
    const uint2 rg = ranges[tile];
    float dF[SSSGS_NF];
    float dT = 0.f, T = 1.f;
    uint32_t lastc = 0;
#pragma unroll
    for (int k = 0; k < SSSGS_NF; ++k) dF[k] = 0.f;
    if (px.inside) {
        lastc = last[px.pix];
        const float4* gi = reinterpret_cast<const float4*>(gbuf + SSSGS_GBUF * px.pix);
        float F[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 v = gi[q];
            F[4 * q] = v.x; F[4 * q + 1] = v.y; F[4 * q + 2] = v.z; F[4 * q + 3] = v.w;
        }
        T = F[15];
        if (MODE == UPSTREAM_DGBUF) {
            const float4* di = reinterpret_cast<const float4*>(dgbuf + SSSGS_GBUF * px.pix);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 v = di[q];
                float t4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (4 * q + c < SSSGS_NF) dF[4 * q + c] = t4[c]; else dT = t4[c];
                }
            }
        } else {
            float g3[3], o[3];
            if (MODE == UPSTREAM_DIMG) {
                g3[0] = dimg[3 * px.pix]; g3[1] = dimg[3 * px.pix + 1]; g3[2] = dimg[3 * px.pix + 2];
            } else {
                const float wgt = l1_scale * (weight ? weight[px.pix] : 1.f);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float d = img[3 * px.pix + c] - target[3 * px.pix + c];
                    g3[c] = d > 0.f ? wgt : (d < 0.f ? -wgt : 0.f);
                }
            }
            shade_px<true>(F, T, fx, fy, sP, cfg.A_eps, o, g3, dF, &dT);
        }
        if (lastc > 0) atomicMax(&s_max, lastc);
    }
    __syncthreads();
    const uint32_t maxlast = s_max;
    const float dTT = dT * T;        // dLoss/dT_final * T_final
    float Q = 0.f;                   // sum_k dF_k * (suffix sum of w_j f_jk)
    uint32_t n_use = 0;
    const float a_min = cfg.alpha_min, a_max = cfg.alpha_max;
    for (uint32_t b1 = maxlast; b1 > rg.x;) {
        const uint32_t b0 = b1 - rg.x > (uint32_t)B ? b1 - B : rg.x;
        __syncthreads();
        const uint32_t idx = b0 + threadIdx.x;
        if (idx < b1) {
            const uint32_t item = vals[idx];
            s_item[threadIdx.x] = item;
            const float4* r = rec + 6 * (int64_t)item;
#pragma unroll
            for (int q = 0; q < 6; ++q) s_rec[q * B + threadIdx.x] = __ldg(r + q);
            s_mask[threadIdx.x] =
                subtile_mask<TILE>(sP, tile, s_rec[threadIdx.x], s_rec[B + threadIdx.x], s_rec[5 * B + threadIdx.x]);
        }
        __syncthreads();
        if (__any_sync(SSSGS_FULL, lastc > b0)) {
            for (int k = (int)(b1 - b0) - 1; k >= 0; --k) {
                if (!(s_mask[k] & wbit)) continue;       // splat misses this warp's sub-tile
                const uint32_t pos = b0 + k;
                const float4 g0 = s_rec[k], g1 = s_rec[B + k];
                AlphaEval e = eval_alpha(g0, g1, fx, fy, a_min, a_max);
                const bool act = (pos < lastc) && e.use;
                if (!__any_sync(SSSGS_FULL, act)) continue;
                // column `lane` of the per-warp scratch holds this pixel's 21 values
                if (act) {
                    ++n_use;
                    const float4 g2 = s_rec[2 * B + k], g3 = s_rec[3 * B + k], g4 = s_rec[4 * B + k];
                    const float g5 = s_rec[5 * B + k].x;
                    const float f[SSSGS_NF] = {g1.z, g1.w, g2.x, g2.y, g2.z, g2.w, g3.x, g3.y,
                                               g3.z, g3.w, g4.x, g4.y, g4.z, g4.w, g5};
                    const float ia = rcp_newton(1.f - e.alpha);
                    const float Ti = T * ia;
                    const float w = e.alpha * Ti;
                    float dot = 0.f;
#pragma unroll
                    for (int c = 0; c < SSSGS_NF; ++c) {
                        dot += dF[c] * f[c];
                        s_red[(6 + c) * RS + lane] = w * dF[c];
                    }
                    const float da = Ti * dot - (Q + dTT) * ia;
                    Q += w * dot;
                    float dp = 0.f, gdo = 0.f;
                    if (!e.clamped) {
                        dp = -da * e.alpha;
                        gdo = da * e.G;
                    }
                    s_red[0 * RS + lane] = dp * (g0.z * e.dx + g0.w * e.dy);
                    s_red[1 * RS + lane] = dp * (g0.w * e.dx + g1.x * e.dy);
                    s_red[2 * RS + lane] = dp * 0.5f * e.dx * e.dx;
                    s_red[3 * RS + lane] = dp * e.dx * e.dy;
                    s_red[4 * RS + lane] = dp * 0.5f * e.dy * e.dy;
                    s_red[5 * RS + lane] = gdo;
                    T = Ti;
                } else {
#pragma unroll
                    for (int c = 0; c < NG; ++c) s_red[c * RS + lane] = 0.f;
                }
                __syncwarp();
                if (lane < NG) {
                    const float4* row = reinterpret_cast<const float4*>(s_red + lane * RS);
                    float4 a = row[0];
#pragma unroll
                    for (int q = 1; q < 8; ++q) {
                        const float4 b = row[q];
                        a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
                    }
                    atomicAdd(drec + (int64_t)SSSGS_REC * s_item[k] + lane, (a.x + a.y) + (a.z + a.w));
                }
                __syncwarp();
            }
        }
        b1 = b0;
    }
    if (stats) {   // contributions replayed and alpha evaluations (positions below each pixel's end)
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

// ---------------------------------------------------------------- composite backward, one warp per sub-tile
//
// Used for 16 x 16 tiles with the fused upstream gradient. Each block is a
// single warp that owns one 8 x 8 sub-tile of a 16 x 16 tile, each lane two
// vertically adjacent pixels; both pixels' contributions to a splat are summed
// in registers before the warp reduction. The hardware block scheduler
// balances work at warp granularity and no warp ever waits for another. The
// warp walks its tile's list back to front in batches of 32 splats. While it
// processes batch i, the records of batch i+1 are in flight into the other
// half of a shared-memory double buffer (cp.async, no registers held) and the
// list entries of batch i+2 are being loaded. Each lane tests its splat
// against the sub-tile with the exact padded ellipse/box test; the warp then
// visits only the splats that passed (ballot bits, highest position first).

// Replay state of one pixel. Q starts at dL/dT_final * T_final and
// accumulates w * (dF . f) over the splats replayed so far, so that
// dL/dalpha_i = T_i (dF . f_i) - Q / (1 - alpha_i).
struct PixBwd {
    float dF[SSSGS_NF];
    float T, Q;
    uint32_t lastc;
};

template <int MODE>
__device__ __forceinline__ void bwd_pixel_setup(PixBwd& p, bool inside, int64_t pix, float fx, float fy,
                                                const sssgs_pair& P,
                                                const sssgs_cfg& cfg, const float* __restrict__ gbuf,
                                                const uint32_t* __restrict__ last, const float* __restrict__ img,
                                                const float* __restrict__ dimg, const float* __restrict__ target,
                                                const float* __restrict__ weight, float l1_scale) {
    float dT = 0.f;
    p.T = 1.f;
    p.lastc = 0;
#pragma unroll
    for (int k = 0; k < SSSGS_NF; ++k) p.dF[k] = 0.f;
    if (inside) {
        p.lastc = last[pix];
        const float4* gi = reinterpret_cast<const float4*>(gbuf + SSSGS_GBUF * pix);
        float F[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 v = gi[q];
            F[4 * q] = v.x; F[4 * q + 1] = v.y; F[4 * q + 2] = v.z; F[4 * q + 3] = v.w;
        }
        p.T = F[15];
        float g3[3], o[3];
        if (MODE == UPSTREAM_DIMG) {
            g3[0] = dimg[3 * pix]; g3[1] = dimg[3 * pix + 1]; g3[2] = dimg[3 * pix + 2];
        } else {
            const float wgt = l1_scale * (weight ? weight[pix] : 1.f);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float d = img[3 * pix + c] - target[3 * pix + c];
                g3[c] = d > 0.f ? wgt : (d < 0.f ? -wgt : 0.f);
            }
        }
        shade_px<true>(F, p.T, fx, fy, P, cfg.A_eps, o, g3, p.dF, &dT);
    }
    p.Q = dT * p.T;
}


// 20 resident blocks per SM: 96 registers (a 40-byte spill) and ~21 warps per
// SM measured faster than 124 registers and 16 warps (29.4 vs 31.7 ms).
// One block per 8 x 8 sub-tile of a TILE x TILE tile ((TILE/8)^2 per tile).
// The composited visibility channel (feature 14) is a G-buffer output that
// the deferred shading does not read, so its upstream gradient is exactly 0
// with the fused upstreams (dimg, L1): the kernel leaves it out of the dot
// products and reduces 20 gradient values per splat (field 20 of the
// gradient record stays as the caller zeroed it). STATS adds the work
// counters.
template <int TILE, int BATCH, int MODE, bool STATS>
__global__ void __launch_bounds__(32, SSSGS_BWD_MINB) k_composite_bwd_warp(sssgs_cfg cfg, const sssgs_pair* __restrict__ pairs,
                                                         int n_pairs, const float4* __restrict__ rec,
                                                         const uint32_t* __restrict__ vals,
                                                         const uint2* __restrict__ ranges,
                                                         const float* __restrict__ gbuf,
                                                         const uint32_t* __restrict__ last,
                                                         const float* __restrict__ img,
                                                         const float* __restrict__ dimg,
                                                         const float* __restrict__ target,
                                                         const float* __restrict__ weight, float l1_scale,
                                                         float* __restrict__ drec,
                                                         unsigned long long* __restrict__ stats) {
    constexpr int NG = 5 + SSSGS_NF, RS = 36, R = BATCH / 32;    // geometry 6 + features 0..13
    using ST = SubTile<TILE, 8, 8>;
    constexpr uint32_t NONE = 0xFFFFFFFFu;
    __shared__ __align__(16) float4 s_rec[2][6][BATCH];
    __shared__ uint32_t s_item[2][BATCH];
    __shared__ __align__(16) float s_red[NG * RS];
    __shared__ __align__(16) sssgs_pair sP;
    const int lane = threadIdx.x;
    if (lane < 8) {
        const int pi = pair_of_tile(pairs, n_pairs, (int)(blockIdx.x / ST::NSUB));
        reinterpret_cast<float4*>(&sP)[lane] = reinterpret_cast<const float4*>(pairs + pi)[lane];
    }
    __syncwarp();
    const ST st(blockIdx.x, sP);
    const int tile = st.tile, bx = st.bx, by = st.by;
    const int i = bx + (lane & 7), j0 = by + (lane >> 3) * 2;
    const uint2 rg = ranges[tile];
    PixBwd p[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = j0 + q;
        const bool inside = i < sP.W && j < sP.H;
        const int64_t pix = sP.pixel_offset + (int64_t)j * sP.W + i;
        bwd_pixel_setup<MODE>(p[q], inside, pix, i + 0.5f, j + 0.5f, sP, cfg, gbuf, last, img, dimg, target,
                              weight, l1_scale);
    }
    const uint32_t wmax = __reduce_max_sync(SSSGS_FULL, max(p[0].lastc, p[1].lastc));
    const float a_min = cfg.alpha_min, a_max = cfg.alpha_max;
    const float px_x = i + 0.5f, px_y0 = j0 + 0.5f;     // centres of this lane's two pixels (y and y + 1)
    // The two pixels' replay state in float2 form for the paired FP32
    // instructions: dF of each pixel as component pairs (2k, 2k+1) of
    // features 0..13; T and Q as (pixel 0, pixel 1).
    float2 dF0[7], dF1[7];
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) {
        dF0[kk] = make_float2(p[0].dF[2 * kk], p[0].dF[2 * kk + 1]);
        dF1[kk] = make_float2(p[1].dF[2 * kk], p[1].dF[2 * kk + 1]);
    }
    float2 Tp = make_float2(p[0].T, p[1].T), Qp = make_float2(p[0].Q, p[1].Q);
    const uint32_t last0 = p[0].lastc, last1 = p[1].lastc;
    const float x0 = bx + 0.5f, y0 = by + 0.5f;
    uint32_t n_use = 0;
    if (wmax > rg.x) {
        const int nb = (int)((wmax - rg.x + BATCH - 1) / BATCH);
        // Batch t covers list positions [lo(t), wmax - BATCH t); slot s of a
        // batch holds position lo(t) + s.
        auto lo_of = [&](int t) -> int64_t { return max((int64_t)rg.x, (int64_t)wmax - (int64_t)BATCH * (t + 1)); };
        auto entry = [&](int t, int r) -> uint32_t {
            if (t >= nb) return NONE;
            const int64_t hi = (int64_t)wmax - (int64_t)BATCH * t;
            const int64_t idx = lo_of(t) + 32 * r + lane;
            return idx < hi ? vals[idx] : NONE;
        };
        auto fetch = [&](const uint32_t* item, int buf) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (item[r] != NONE) {
                    const float4* src = rec + 6 * (int64_t)item[r];
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        cp_async16((uint32_t)__cvta_generic_to_shared(&s_rec[buf][q][32 * r + lane]), src + q);
                }
            }
            cp_async_commit();
        };
        uint32_t it0[R], it1[R], it2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) it0[r] = entry(0, r);
        fetch(it0, 0);
#pragma unroll
        for (int r = 0; r < R; ++r) it1[r] = entry(1, r);
        for (int t = 0; t < nb; ++t) {
            const int buf = t & 1;
            fetch(it1, buf ^ 1);
#pragma unroll
            for (int r = 0; r < R; ++r) it2[r] = entry(t + 2, r);
            cp_async_wait1();
            uint32_t bits[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int sl = 32 * r + lane;
                const float4 g0 = s_rec[buf][0][sl], g1 = s_rec[buf][1][sl], g5 = s_rec[buf][5][sl];
                const bool pass = (it0[r] != NONE) &
                                  ellipse_meets_box(g0.x, g0.y, g0.z, g0.w, g1.x, g5.y, g5.z, g5.w, x0, x0 + 7.f,
                                                    y0, y0 + 7.f);
                s_item[buf][sl] = it0[r];
                bits[r] = __ballot_sync(SSSGS_FULL, pass);
            }
            __syncwarp();
            const uint32_t lo = (uint32_t)lo_of(t);
#pragma unroll
            for (int r = R - 1; r >= 0; --r) {
            while (bits[r]) {
                const int kb = 31 - __clz(bits[r]);
                bits[r] ^= 1u << kb;
                const int k = 32 * r + kb;
                const uint32_t pos = lo + k;
                const float4 g0 = s_rec[buf][0][k], g1 = s_rec[buf][1][k];
                AlphaEval e0, e1;
                eval_alpha2(g0, g1, px_x, px_y0, px_y0 + 1.f, a_min, a_max, e0, e1);
                const bool act0 = (pos < last0) && e0.use;
                const bool act1 = (pos < last1) && e1.use;
                if (!__any_sync(SSSGS_FULL, act0 || act1)) continue;
                {   // both pixels' terms, summed, straight into this lane's reduction column
                    const float4 g2 = s_rec[buf][2][k], g3 = s_rec[buf][3][k], g4 = s_rec[buf][4][k];
                    const float2 fp[7] = {make_float2(g1.z, g1.w), make_float2(g2.x, g2.y), make_float2(g2.z, g2.w),
                                          make_float2(g3.x, g3.y), make_float2(g3.z, g3.w), make_float2(g4.x, g4.y),
                                          make_float2(g4.z, g4.w)};
                    // dF . f of each pixel (even and odd components summed separately)
                    float2 d0 = __fmul2_rn(dF0[0], fp[0]), d1 = __fmul2_rn(dF1[0], fp[0]);
#pragma unroll
                    for (int kk = 1; kk < 7; ++kk) {
                        d0 = __ffma2_rn(dF0[kk], fp[kk], d0);
                        d1 = __ffma2_rn(dF1[kk], fp[kk], d1);
                    }
                    const float2 dot = make_float2(d0.x + d0.y, d1.x + d1.y);
                    // replay step: T_i = T_{i+1} / (1 - alpha), dL/dalpha = T_i dot - Q / (1 - alpha)
                    const float2 ia = make_float2(rcp_newton(1.f - e0.alpha), rcp_newton(1.f - e1.alpha));
                    const float2 alp = make_float2(e0.alpha, e1.alpha);
                    const float2 Ti = __fmul2_rn(Tp, ia);
                    const float2 qa = __fmul2_rn(Qp, ia);
                    const float2 da = __ffma2_rn(Ti, dot, make_float2(-qa.x, -qa.y));
                    const float2 wr = __fmul2_rn(alp, Ti);
                    const float2 dpr = __fmul2_rn(make_float2(-da.x, -da.y), alp);
                    const float2 dgr = __fmul2_rn(da, make_float2(e0.G, e1.G));
                    const bool geo0 = act0 && !e0.clamped, geo1 = act1 && !e1.clamped;
                    const float2 w = make_float2(act0 ? wr.x : 0.f, act1 ? wr.y : 0.f);
                    const float2 dp = make_float2(geo0 ? dpr.x : 0.f, geo1 ? dpr.y : 0.f);
                    const float2 dg = make_float2(geo0 ? dgr.x : 0.f, geo1 ? dgr.y : 0.f);
                    Qp = __ffma2_rn(w, dot, Qp);
                    Tp = make_float2(act0 ? Ti.x : Tp.x, act1 ? Ti.y : Tp.y);
                    if (STATS) n_use += (uint32_t)act0 + (uint32_t)act1;
                    float* col = s_red + lane;
                    // features: w0 dF0 + w1 dF1, component pairs
                    const float2 w0b = make_float2(w.x, w.x), w1b = make_float2(w.y, w.y);
#pragma unroll
                    for (int kk = 0; kk < 7; ++kk) {
                        const float2 cv = __ffma2_rn(w1b, dF1[kk], __fmul2_rn(w0b, dF0[kk]));
                        col[(6 + 2 * kk) * RS] = cv.x;
                        col[(7 + 2 * kk) * RS] = cv.y;
                    }
                    // geometry: the two pixels share dx (same column)
                    const float dx = e0.dx;
                    const float2 dy = make_float2(e0.dy, e1.dy);
                    const float ca = g0.z, cb = g0.w, cc = g1.x;
                    const float2 u = __ffma2_rn(make_float2(cb, cb), dy, make_float2(ca * dx, ca * dx));
                    const float2 v = __ffma2_rn(make_float2(cc, cc), dy, make_float2(cb * dx, cb * dx));
                    const float2 pdy = __fmul2_rn(dp, dy);
                    col[0] = dp.x * u.x + dp.y * u.y;
                    col[RS] = dp.x * v.x + dp.y * v.y;
                    col[2 * RS] = 0.5f * dx * dx * (dp.x + dp.y);
                    col[3 * RS] = dx * (pdy.x + pdy.y);
                    col[4 * RS] = 0.5f * (pdy.x * dy.x + pdy.y * dy.y);
                    col[5 * RS] = dg.x + dg.y;
                }
                __syncwarp();
                if (lane < NG) {   // sum of the 32 lanes' terms, in pairs
                    const float4* row = reinterpret_cast<const float4*>(s_red + lane * RS);
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
                    atomicAdd(drec + (int64_t)SSSGS_REC * s_item[buf][k] + lane, a[0].x + a[0].y);
                }
                __syncwarp();
            }
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < R; ++r) {
                it0[r] = it1[r];
                it1[r] = it2[r];
            }
        }
    }
    if (STATS) {
        unsigned long long u = n_use;
        unsigned long long v = (last0 > rg.x ? last0 - rg.x : 0) + (last1 > rg.x ? last1 - rg.x : 0);
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

template <int TILE>
static size_t bwd_smem() {
    return (size_t)6 * TILE * TILE * sizeof(float4) + (size_t)TILE * TILE * 8 +
           (size_t)(TILE * TILE / 32) * (6 + SSSGS_NF) * 36 * 4;
}

}  // namespace sssgs

using namespace sssgs;

namespace {
bool args_ok(const sssgs_cfg* cfg, const sssgs_pair* h, const sssgs_pair* d, int n) {
    return cfg && h && d && n > 0 && (cfg->tile == 8 || cfg->tile == 16 || cfg->tile == 32) &&
           (cfg->batch == 0 || cfg->batch == 32 || cfg->batch == 64);
}
int tiles_of(const sssgs_pair* h, int n) { return h[n - 1].tile_offset + h[n - 1].tiles_x * h[n - 1].tiles_y; }
bool a16(const void* p) { return ((uintptr_t)p & 15) == 0; }

// One-warp forward: (TILE/8)^2 blocks of 32 threads per tile.
template <int TILE, int BATCH, bool SHADE>
int launch_fwd_warp_t(const sssgs_cfg* cfg, const sssgs_pair* d, int n, int tiles, const float* rec,
                      const uint32_t* vals, const uint32_t* ranges, float* gbuf, uint32_t* last, float* img,
                      cudaStream_t st, unsigned long long* stats) {
    constexpr int NSUB = (TILE / 8) * (TILE / 8);
    if (stats)
        k_composite_fwd_warp<TILE, BATCH, SHADE, true><<<NSUB * tiles, 32, 0, st>>>(
            *cfg, d, n, (const float4*)rec, vals, (const uint2*)ranges, gbuf, last, img, stats);
    else
        k_composite_fwd_warp<TILE, BATCH, SHADE, false><<<NSUB * tiles, 32, 0, st>>>(
            *cfg, d, n, (const float4*)rec, vals, (const uint2*)ranges, gbuf, last, img, nullptr);
    sssgs::note_launches(1);
    return launch_status();
}

template <bool SHADE>
int launch_fwd_warp(const sssgs_cfg* cfg, const sssgs_pair* d, int n, int tiles, const float* rec,
                    const uint32_t* vals, const uint32_t* ranges, float* gbuf, uint32_t* last, float* img,
                    cudaStream_t st, unsigned long long* stats = nullptr) {
    const bool b64 = cfg->batch == 64;
    switch (cfg->tile) {
        case 8: return b64 ? launch_fwd_warp_t<8, 64, SHADE>(cfg, d, n, tiles, rec, vals, ranges, gbuf, last, img, st, stats)
                           : launch_fwd_warp_t<8, 32, SHADE>(cfg, d, n, tiles, rec, vals, ranges, gbuf, last, img, st, stats);
        case 16: return b64 ? launch_fwd_warp_t<16, 64, SHADE>(cfg, d, n, tiles, rec, vals, ranges, gbuf, last, img, st, stats)
                            : launch_fwd_warp_t<16, 32, SHADE>(cfg, d, n, tiles, rec, vals, ranges, gbuf, last, img, st, stats);
        default: return b64 ? launch_fwd_warp_t<32, 64, SHADE>(cfg, d, n, tiles, rec, vals, ranges, gbuf, last, img, st, stats)
                            : launch_fwd_warp_t<32, 32, SHADE>(cfg, d, n, tiles, rec, vals, ranges, gbuf, last, img, st, stats);
    }
}

// Block-per-tile backward with a G-buffer gradient upstream (the unfused path).
template <int TILE>
int launch_bwd_dgbuf(const sssgs_cfg* cfg, const sssgs_pair* d, int n, int tiles, const float* rec,
                     const uint32_t* vals, const uint32_t* ranges, const float* gbuf, const uint32_t* last,
                     const float* dgbuf, float* drec, cudaStream_t st) {
    size_t sm = bwd_smem<TILE>();
    cudaFuncSetAttribute(k_composite_bwd<TILE, UPSTREAM_DGBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_composite_bwd<TILE, UPSTREAM_DGBUF><<<tiles, TILE * TILE, sm, st>>>(*cfg, d, n, (const float4*)rec, vals,
                                                                         (const uint2*)ranges, gbuf, last, dgbuf,
                                                                         nullptr, nullptr, nullptr, nullptr, 0.f,
                                                                         drec, nullptr);
    sssgs::note_launches(1);
    return launch_status();
}

// One-warp backward with the fused upstream (dimg or L1): (TILE/8)^2 blocks per tile.
template <int TILE, int BATCH, int MODE>
int launch_bwd_warp_t(const sssgs_cfg* cfg, const sssgs_pair* d, int n, int tiles, const float* rec,
                      const uint32_t* vals, const uint32_t* ranges, const float* gbuf, const uint32_t* last,
                      const float* img, const float* dimg, const float* target, const float* weight, float l1,
                      float* drec, cudaStream_t st, unsigned long long* stats) {
    constexpr int NSUB = (TILE / 8) * (TILE / 8);
    if (stats)
        k_composite_bwd_warp<TILE, BATCH, MODE, true><<<NSUB * tiles, 32, 0, st>>>(
            *cfg, d, n, (const float4*)rec, vals, (const uint2*)ranges, gbuf, last, img, dimg, target, weight, l1,
            drec, stats);
    else
        k_composite_bwd_warp<TILE, BATCH, MODE, false><<<NSUB * tiles, 32, 0, st>>>(
            *cfg, d, n, (const float4*)rec, vals, (const uint2*)ranges, gbuf, last, img, dimg, target, weight, l1,
            drec, nullptr);
    sssgs::note_launches(1);
    return launch_status();
}

template <int MODE>
int launch_bwd_warp(const sssgs_cfg* cfg, const sssgs_pair* d, int n, int tiles, const float* rec,
                    const uint32_t* vals, const uint32_t* ranges, const float* gbuf, const uint32_t* last,
                    const float* img, const float* dimg, const float* target, const float* weight, float l1,
                    float* drec, cudaStream_t st, unsigned long long* stats) {
    const bool b64 = cfg->batch == 64;
#define SSSGS_BWD_ARGS cfg, d, n, tiles, rec, vals, ranges, gbuf, last, img, dimg, target, weight, l1, drec, st, stats
    switch (cfg->tile) {
        case 8: return b64 ? launch_bwd_warp_t<8, 64, MODE>(SSSGS_BWD_ARGS) : launch_bwd_warp_t<8, 32, MODE>(SSSGS_BWD_ARGS);
        case 16: return b64 ? launch_bwd_warp_t<16, 64, MODE>(SSSGS_BWD_ARGS) : launch_bwd_warp_t<16, 32, MODE>(SSSGS_BWD_ARGS);
        default: return b64 ? launch_bwd_warp_t<32, 64, MODE>(SSSGS_BWD_ARGS) : launch_bwd_warp_t<32, 32, MODE>(SSSGS_BWD_ARGS);
    }
#undef SSSGS_BWD_ARGS
}
}  // namespace

extern "C" int sssgs_composite_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                   int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                                   float* gbuf, uint32_t* last, sssgs_stream stream) {
    if (!args_ok(cfg, h_pairs, d_pairs, n_pairs) || !rec || !ranges || !gbuf || !last) return SSSGS_ERR_INVALID_ARG;
    if (!a16(rec) || !a16(gbuf) || !a16(d_pairs) || !a16(ranges)) return SSSGS_ERR_INVALID_ARG;
    int tiles = tiles_of(h_pairs, n_pairs);
    cudaStream_t st = (cudaStream_t)stream;
    return launch_fwd_warp<false>(cfg, d_pairs, n_pairs, tiles, rec, vals, ranges, gbuf, last, nullptr, st);
}

extern "C" int sssgs_render_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                                float* gbuf, uint32_t* last, float* img, uint64_t* d_stats, sssgs_stream stream) {
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(d_stats);
    if (!args_ok(cfg, h_pairs, d_pairs, n_pairs) || !rec || !ranges || !gbuf || !last || !img)
        return SSSGS_ERR_INVALID_ARG;
    if (!a16(rec) || !a16(gbuf) || !a16(d_pairs) || !a16(ranges)) return SSSGS_ERR_INVALID_ARG;
    int tiles = tiles_of(h_pairs, n_pairs);
    cudaStream_t st = (cudaStream_t)stream;
    return launch_fwd_warp<true>(cfg, d_pairs, n_pairs, tiles, rec, vals, ranges, gbuf, last, img, st, stats);
}

extern "C" int sssgs_shade_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                               int n_pairs, const float* gbuf, float* img, sssgs_stream stream) {
    if (!args_ok(cfg, h_pairs, d_pairs, n_pairs) || !gbuf || !img) return SSSGS_ERR_INVALID_ARG;
    if (!a16(gbuf) || !a16(d_pairs)) return SSSGS_ERR_INVALID_ARG;
    int tiles = tiles_of(h_pairs, n_pairs);
    cudaStream_t st = (cudaStream_t)stream;
    switch (cfg->tile) {
        case 8: k_shade<8, false><<<tiles, 64, 0, st>>>(*cfg, d_pairs, n_pairs, gbuf, img, nullptr, nullptr); sssgs::note_launches(1); break;
        case 16: k_shade<16, false><<<tiles, 256, 0, st>>>(*cfg, d_pairs, n_pairs, gbuf, img, nullptr, nullptr); sssgs::note_launches(1); break;
        default: k_shade<32, false><<<tiles, 1024, 0, st>>>(*cfg, d_pairs, n_pairs, gbuf, img, nullptr, nullptr); sssgs::note_launches(1); break;
    }
    return launch_status();
}

extern "C" int sssgs_shade_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                               int n_pairs, const float* gbuf, const float* dimg, float* dgbuf, sssgs_stream stream) {
    if (!args_ok(cfg, h_pairs, d_pairs, n_pairs) || !gbuf || !dimg || !dgbuf) return SSSGS_ERR_INVALID_ARG;
    if (!a16(gbuf) || !a16(dgbuf) || !a16(d_pairs)) return SSSGS_ERR_INVALID_ARG;
    int tiles = tiles_of(h_pairs, n_pairs);
    cudaStream_t st = (cudaStream_t)stream;
    switch (cfg->tile) {
        case 8: k_shade<8, true><<<tiles, 64, 0, st>>>(*cfg, d_pairs, n_pairs, gbuf, nullptr, dimg, dgbuf); sssgs::note_launches(1); break;
        case 16: k_shade<16, true><<<tiles, 256, 0, st>>>(*cfg, d_pairs, n_pairs, gbuf, nullptr, dimg, dgbuf); sssgs::note_launches(1); break;
        default: return SSSGS_ERR_UNSUPPORTED;
    }
    return launch_status();
}

extern "C" int sssgs_composite_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                   int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                                   const float* gbuf, const uint32_t* last, const float* dgbuf, float* drec,
                                   sssgs_stream stream) {
    if (!args_ok(cfg, h_pairs, d_pairs, n_pairs) || !rec || !ranges || !gbuf || !last || !dgbuf || !drec)
        return SSSGS_ERR_INVALID_ARG;
    if (!a16(rec) || !a16(gbuf) || !a16(dgbuf) || !a16(d_pairs) || !a16(ranges)) return SSSGS_ERR_INVALID_ARG;
    const int tiles = tiles_of(h_pairs, n_pairs);
    cudaStream_t st = (cudaStream_t)stream;
    switch (cfg->tile) {
        case 8: return launch_bwd_dgbuf<8>(cfg, d_pairs, n_pairs, tiles, rec, vals, ranges, gbuf, last, dgbuf, drec, st);
        case 16: return launch_bwd_dgbuf<16>(cfg, d_pairs, n_pairs, tiles, rec, vals, ranges, gbuf, last, dgbuf, drec, st);
        default: return SSSGS_ERR_UNSUPPORTED;   // 32 x 32 tiles: the block-per-tile kernel would need 1024 threads
    }
}

extern "C" int sssgs_render_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                                const float* gbuf, const uint32_t* last, const float* img, const float* dimg,
                                const float* target, const float* weight, float l1_scale, float* drec,
                                uint64_t* d_stats, sssgs_stream stream) {
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(d_stats);
    if (!args_ok(cfg, h_pairs, d_pairs, n_pairs) || !rec || !ranges || !gbuf || !last || !drec)
        return SSSGS_ERR_INVALID_ARG;
    if (!a16(rec) || !a16(gbuf) || !a16(d_pairs) || !a16(ranges)) return SSSGS_ERR_INVALID_ARG;
    int tiles = tiles_of(h_pairs, n_pairs);
    cudaStream_t st = (cudaStream_t)stream;
    if (dimg)
        return launch_bwd_warp<UPSTREAM_DIMG>(cfg, d_pairs, n_pairs, tiles, rec, vals, ranges, gbuf, last, nullptr,
                                              dimg, nullptr, nullptr, 0.f, drec, st, stats);
    if (!img || !target) return SSSGS_ERR_INVALID_ARG;
    return launch_bwd_warp<UPSTREAM_L1>(cfg, d_pairs, n_pairs, tiles, rec, vals, ranges, gbuf, last, img, nullptr,
                                        target, weight, l1_scale, drec, st, stats);
}
