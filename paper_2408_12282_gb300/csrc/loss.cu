// Training losses of Appendix E ("Losses"), fused into the backward step:
//   image loss  L_img = (1 - lambda) L1 + lambda (1 - SSIM)  per view/light pair
//   incident    L_inc = lambda_inc * mean_i |min(L_in_i, 1) - v_i|  per pair
// SSIM: Wang et al. (2004) with an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2,
// averaged over the pair's pixels and channels.
//
// Image loss, two passes over every pair's tiles (the render tile grid; the
// tile, its 5-pixel window halo and all three channels staged in shared
// memory; separable windowed sums, rows then columns):
//   A: windowed moments mu_x, mu_y, E[x^2], E[y^2], E[xy], the per-pixel SSIM
//      and L1 terms of the loss, and three coefficient planes per channel of
//      the gradient (dS/dmu_x, dS/dE[x^2], dS/dE[xy] for the mean over the
//      pair) into the workspace (9 planes of n_pixels floats);
//   B: the windowed sums of those planes give
//      dSSIM/dx = W*a + 2 x (W*b) + y (W*c)  (the window is symmetric);
//      dimg = (1 - lambda) sign(x - y) / n - lambda dSSIM/dx.
#include <cmath>

#include "common.cuh"

namespace sssgs {
namespace {

constexpr int R = 5;             // window radius
constexpr float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
struct Win {
    float w[2 * R + 1];
};

template <int TILE>
struct SsimTile {
    static constexpr int E = TILE + 2 * R;          // staged edge (tile + halo)
    static constexpr int ES = E + (E & 1);          // even row stride: float2 pairs stay 16-B aligned
    static constexpr int NT = TILE * TILE;          // threads per block
    static constexpr int NW = NT / 32;
    static constexpr int KH = TILE == 32 ? 4 : 2;   // outputs per item of the row pass
    static constexpr int KV = 4;                    // outputs per item of the column pass
    static constexpr int GH = TILE / KH, GV = TILE / KV;
    static constexpr int STAGE = 3 * E * ES;        // staged elements per buffer
    static constexpr int HSZ = 3 * E * TILE;        // row-pass outputs per plane
    // shared memory of the two passes (bytes): staging buffer + row-pass planes
    static constexpr int SMEM_A = 8 * STAGE + (8 + 8 + 4) * HSZ + 4 * NW;
    static constexpr int SMEM_B = (8 + 4) * STAGE + (8 + 4) * HSZ;
};

// Where a tile lies: its pair, pixel origin and the pair's image.
struct TileGeo {
    int pair, x0, y0, W, H;
    int64_t pix0;
    bool first;
};

template <int TILE>
__device__ __forceinline__ TileGeo tile_geo(const sssgs_pair* __restrict__ pairs, int n_pairs, int tile) {
    TileGeo g;
    g.pair = pair_of_tile(pairs, n_pairs, tile);
    const sssgs_pair& P = pairs[g.pair];
    const int lt = tile - P.tile_offset;
    g.x0 = (lt % P.tiles_x) * TILE;
    g.y0 = (lt / P.tiles_x) * TILE;
    g.W = P.W;
    g.H = P.H;
    g.pix0 = P.pixel_offset;
    g.first = lt == 0;
    return g;
}

__device__ __forceinline__ float2 f2(float w) { return make_float2(w, w); }

// 4-byte asynchronous copy global -> shared; zero-fills when !ok (src is then
// not read).
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Pass A staging: the tile and its halo, all three channels, as (x, y) pairs
// xy[(c E + r) ES + col]; one warp per staged row reads the row's 3E
// interleaved floats (coalesced), zero outside the image.
template <int TILE>
__device__ __forceinline__ void stage_xy(float2* xy, const TileGeo& g, const float* __restrict__ img,
                                         const float* __restrict__ target) {
    using T = SsimTile<TILE>;
    constexpr int E = T::E, ES = T::ES;
    constexpr int PER = (3 * E + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < E; r += T::NW) {
        const int gy = g.y0 - R + r;
        const bool rok = gy >= 0 && gy < g.H;
        const int64_t base = 3 * (g.pix0 + (int64_t)gy * g.W + (g.x0 - R));
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int f = lane + 32 * u;
            if (f < 3 * E) {
                const int col = f / 3, ch = f - 3 * col, gx = g.x0 - R + col;
                const bool ok = rok && gx >= 0 && gx < g.W;
                float2* d = xy + (ch * E + r) * ES + col;
                cp_async4(&d->x, ok ? img + base + f : img, ok);
                cp_async4(&d->y, ok ? target + base + f : target, ok);
            }
        }
    }
}

// Pass A, one block per tile: all staging copies are issued at once
// (cp.async, no registers held), then the block waits for them. Row pass: every item slides the 11-tap window
// over KH adjacent outputs of one staged row, forming (W*x, W*y),
// (W*x^2, W*y^2) with paired FP32 FMAs and W*xy. Column pass: KV adjacent
// outputs of one column, then per pixel and channel the SSIM, the loss terms
// and the coefficients
//   coef plane 3c+0: dS/dmu_x, 3c+1: dS/dE[x^2], 3c+2: dS/dE[xy]
// (for the mean over the pair), planar over all pixels (n_pix_total apart).
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_ssim_moments(const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                              int n_tiles, int64_t n_pix_total,
                                                              const float* __restrict__ img,
                                                              const float* __restrict__ target, Win win,
                                                              float lambda, float* __restrict__ coef,
                                                              float* __restrict__ d_loss) {
    using T = SsimTile<TILE>;
    constexpr int E = T::E, ES = T::ES, NT = T::NT, KH = T::KH, KV = T::KV;
    extern __shared__ __align__(16) float smem[];
    float2* xy = reinterpret_cast<float2*>(smem);            // [3][E][ES]
    float2* hm = xy + T::STAGE;                             // [3][E][TILE]  row sums of (x, y)
    float2* hs = hm + T::HSZ;                               // [3][E][TILE]  row sums of (x^2, y^2)
    float* hp = reinterpret_cast<float*>(hs + T::HSZ);      // [3][E][TILE]  row sums of xy
    float* red = hp + T::HSZ;                               // [NW]
    const int tid = threadIdx.x;
    float2 w2[2 * R + 1];
#pragma unroll
    for (int t = 0; t <= 2 * R; ++t) w2[t] = f2(win.w[t]);
    const int tile = blockIdx.x;
    const TileGeo g = tile_geo<TILE>(pairs, n_pairs, tile);
    stage_xy<TILE>(xy, g, img, target);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    {
        const float2* X = xy;
        for (int k = tid; k < 3 * E * T::GH; k += NT) {
            const int gi = k % T::GH, rc = k / T::GH;         // rc = channel * E + staged row
            const float4* src = reinterpret_cast<const float4*>(X + rc * ES + gi * KH);
            float2 m[KH], sq[KH];
            float p[KH];
#pragma unroll
            for (int o = 0; o < KH; ++o) {
                m[o] = make_float2(0.f, 0.f);
                sq[o] = make_float2(0.f, 0.f);
                p[o] = 0.f;
            }
#pragma unroll
            for (int jj = 0; jj < (KH + 2 * R) / 2; ++jj) {
                const float4 q4 = src[jj];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 2 * jj + h;
                    const float2 v = h ? make_float2(q4.z, q4.w) : make_float2(q4.x, q4.y);
                    const float2 v2 = __fmul2_rn(v, v);
                    const float pr = v.x * v.y;
#pragma unroll
                    for (int o = 0; o < KH; ++o) {
                        const int t = j - o;
                        if (t >= 0 && t <= 2 * R) {
                            m[o] = __ffma2_rn(w2[t], v, m[o]);
                            sq[o] = __ffma2_rn(w2[t], v2, sq[o]);
                            p[o] = fmaf(w2[t].x, pr, p[o]);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < KH; ++o) {
                const int d = rc * TILE + gi * KH + o;
                hm[d] = m[o];
                hs[d] = sq[o];
                hp[d] = p[o];
            }
        }
        __syncthreads();
        const float inv_n = 1.f / (3.f * (float)g.W * (float)g.H);
        float part = 0.f;
        for (int k = tid; k < 3 * TILE * T::GV; k += NT) {
            const int col = k % TILE, rest = k / TILE;
            const int ch = rest % 3, rb = (rest / 3) * KV;
            float2 m[KV], sq[KV];
            float p[KV];
#pragma unroll
            for (int o = 0; o < KV; ++o) {
                m[o] = make_float2(0.f, 0.f);
                sq[o] = make_float2(0.f, 0.f);
                p[o] = 0.f;
            }
#pragma unroll
            for (int j = 0; j < KV + 2 * R; ++j) {
                const int d = (ch * E + rb + j) * TILE + col;
                const float2 a = hm[d], b = hs[d];
                const float c = hp[d];
#pragma unroll
                for (int o = 0; o < KV; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t <= 2 * R) {
                        m[o] = __ffma2_rn(w2[t], a, m[o]);
                        sq[o] = __ffma2_rn(w2[t], b, sq[o]);
                        p[o] = fmaf(w2[t].x, c, p[o]);
                    }
                }
            }
            const int i = g.x0 + col;
#pragma unroll
            for (int o = 0; o < KV; ++o) {
                const int j = g.y0 + rb + o;
                if (i < g.W && j < g.H) {
                    const float mx = m[o].x, my = m[o].y;
                    const float sxx = sq[o].x - mx * mx, syy = sq[o].y - my * my, sxy = p[o] - mx * my;
                    const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
                    const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
                    const float iB = 1.f / (B1 * B2);
                    const float S = A1 * A2 * iB;
                    const float sn = S * iB * inv_n;
                    const float dA1 = A2 * iB * inv_n, dA2 = A1 * iB * inv_n;
                    const float d_sxx = -sn * B1, d_sxy = 2.f * dA2;          // dS/dB2 = -S / B2
                    const float d_mx = 2.f * (dA1 * my - sn * B2 * mx) - 2.f * mx * d_sxx - my * d_sxy;
                    const int64_t pix = g.pix0 + (int64_t)j * g.W + i;
                    coef[(3 * ch + 0) * n_pix_total + pix] = d_mx;
                    coef[(3 * ch + 1) * n_pix_total + pix] = d_sxx;
                    coef[(3 * ch + 2) * n_pix_total + pix] = d_sxy;
                    const float2 v = X[(ch * E + rb + o + R) * ES + col + R];
                    part += ((1.f - lambda) * fabsf(v.x - v.y) - lambda * S) * inv_n;
                }
            }
        }
        // block sum of the loss terms; the pair's first tile also adds lambda (the 1 of 1 - SSIM)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(SSSGS_FULL, part, o);
        if ((tid & 31) == 0) red[tid >> 5] = part;
        __syncthreads();
        if (tid == 0) {
            float s = 0.f;
            for (int w = 0; w < T::NW; ++w) s += red[w];
            if (g.first) s += lambda;
            atomicAdd(d_loss + g.pair, s);
        }
    }
}

// Pass B staging: the coefficient planes of the tile and its halo,
// sab[(c E + r) ES + col] = (a, b), sc[...] = c; one warp per (channel, row).
template <int TILE>
__device__ __forceinline__ void stage_coef(float2* sab, float* sc, const TileGeo& g, int64_t n_pix_total,
                                           const float* __restrict__ coef) {
    using T = SsimTile<TILE>;
    constexpr int E = T::E, ES = T::ES;
    constexpr int PER = (E + 31) / 32;
    const int lane = threadIdx.x & 31;
    for (int rc = threadIdx.x >> 5; rc < 3 * E; rc += T::NW) {
        const int ch = rc / E, r = rc - ch * E, gy = g.y0 - R + r;
        const bool rok = gy >= 0 && gy < g.H;
        const float* cf = coef + 3 * ch * n_pix_total + g.pix0 + (int64_t)gy * g.W + (g.x0 - R);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int col = lane + 32 * u, gx = g.x0 - R + col;
            if (col < E) {
                const bool ok = rok && gx >= 0 && gx < g.W;
                float2* d = sab + rc * ES + col;
                cp_async4(&d->x, ok ? cf + col : coef, ok);
                cp_async4(&d->y, ok ? cf + n_pix_total + col : coef, ok);
                cp_async4(sc + rc * ES + col, ok ? cf + 2 * n_pix_total + col : coef, ok);
            }
        }
    }
}

// Pass B: dimg = (1 - lambda) sign(x - y) / n - lambda (W*a + 2 x W*b + y W*c)
// with a, b, c the coefficient planes of pass A (the window is symmetric, so
// the adjoint of the windowed mean is the same correlation). Same staging,
// one block per tile, two separable passes with (a, b) paired.
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_ssim_grad(const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                           int n_tiles, int64_t n_pix_total,
                                                           const float* __restrict__ img,
                                                           const float* __restrict__ target, Win win, float lambda,
                                                           const float* __restrict__ coef, float* __restrict__ dimg) {
    using T = SsimTile<TILE>;
    constexpr int E = T::E, ES = T::ES, NT = T::NT, KH = T::KH, KV = T::KV;
    extern __shared__ __align__(16) float smem[];
    float2* sab = reinterpret_cast<float2*>(smem);              // [3][E][ES]  (a, b)
    float* sc = reinterpret_cast<float*>(sab + T::STAGE);       // [3][E][ES]  c
    float2* h2 = reinterpret_cast<float2*>(sc + T::STAGE);      // [3][E][TILE]
    float* h1 = reinterpret_cast<float*>(h2 + T::HSZ);          // [3][E][TILE]
    const int tid = threadIdx.x;
    float2 w2[2 * R + 1];
#pragma unroll
    for (int t = 0; t <= 2 * R; ++t) w2[t] = f2(win.w[t]);
    const int tile = blockIdx.x;
    const TileGeo g = tile_geo<TILE>(pairs, n_pairs, tile);
    stage_coef<TILE>(sab, sc, g, n_pix_total, coef);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    {
        const float2* SAB = sab;
        const float* SC = sc;
        for (int k = tid; k < 3 * E * T::GH; k += NT) {
            const int gi = k % T::GH, rc = k / T::GH;
            const float4* s4 = reinterpret_cast<const float4*>(SAB + rc * ES + gi * KH);
            const float2* c2 = reinterpret_cast<const float2*>(SC + rc * ES + gi * KH);
            float2 u[KH];
            float v[KH];
#pragma unroll
            for (int o = 0; o < KH; ++o) {
                u[o] = make_float2(0.f, 0.f);
                v[o] = 0.f;
            }
#pragma unroll
            for (int jj = 0; jj < (KH + 2 * R) / 2; ++jj) {
                const float4 q4 = s4[jj];
                const float2 cc = c2[jj];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 2 * jj + h;
                    const float2 ab = h ? make_float2(q4.z, q4.w) : make_float2(q4.x, q4.y);
                    const float c = h ? cc.y : cc.x;
#pragma unroll
                    for (int o = 0; o < KH; ++o) {
                        const int t = j - o;
                        if (t >= 0 && t <= 2 * R) {
                            u[o] = __ffma2_rn(w2[t], ab, u[o]);
                            v[o] = fmaf(w2[t].x, c, v[o]);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < KH; ++o) {
                h2[rc * TILE + gi * KH + o] = u[o];
                h1[rc * TILE + gi * KH + o] = v[o];
            }
        }
        __syncthreads();
        const float inv_n = 1.f / (3.f * (float)g.W * (float)g.H);
        for (int k = tid; k < 3 * TILE * T::GV; k += NT) {
            const int col = k % TILE, rest = k / TILE;
            const int ch = rest % 3, rb = (rest / 3) * KV;
            const int i = g.x0 + col;
            float2 u[KV], xyv[KV];
            float v[KV];
#pragma unroll
            for (int o = 0; o < KV; ++o) {             // image values first: their latency hides under the taps
                u[o] = make_float2(0.f, 0.f);
                v[o] = 0.f;
                const int j = g.y0 + rb + o;
                xyv[o] = make_float2(0.f, 0.f);
                if (i < g.W && j < g.H) {
                    const int64_t q = 3 * (g.pix0 + (int64_t)j * g.W + i) + ch;
                    xyv[o] = make_float2(img[q], target[q]);
                }
            }
#pragma unroll
            for (int j = 0; j < KV + 2 * R; ++j) {
                const int d = (ch * E + rb + j) * TILE + col;
                const float2 ab = h2[d];
                const float c = h1[d];
#pragma unroll
                for (int o = 0; o < KV; ++o) {
                    const int t = j - o;
                    if (t >= 0 && t <= 2 * R) {
                        u[o] = __ffma2_rn(w2[t], ab, u[o]);
                        v[o] = fmaf(w2[t].x, c, v[o]);
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < KV; ++o) {
                const int j = g.y0 + rb + o;
                if (i < g.W && j < g.H) {
                    const int64_t q = 3 * (g.pix0 + (int64_t)j * g.W + i) + ch;
                    const float xv = xyv[o].x, yv = xyv[o].y;
                    const float d = xv - yv;
                    const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
                    dimg[q] = (1.f - lambda) * sg * inv_n - lambda * (u[o].x + 2.f * xv * u[o].y + yv * v[o]);
                }
            }
        }
    }
}

// Incident-light constraint: per item m of pair p with n_p items,
// L += lambda |min(L_in, 1) - v| / n_p; drec[19] += dL/dL_in, drec[20] += dL/dv.
__global__ void __launch_bounds__(256) k_incident(const sssgs_pair* __restrict__ pairs, int n_pairs, int64_t n_items,
                                                  const float* __restrict__ rec, float lambda,
                                                  float* __restrict__ drec, float* __restrict__ d_loss) {
    __shared__ float s_sum[2];
    __shared__ int s_p0;
    const int64_t m0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t m = m0 + threadIdx.x;
    if (threadIdx.x == 0) {
        s_p0 = pair_of_item(pairs, n_pairs, m0);
        s_sum[0] = s_sum[1] = 0.f;
    }
    __syncthreads();
    if (m < n_items) {
        const int p = pair_of_item(pairs, n_pairs, m);
        const float inv = 1.f / (float)pairs[p].g_count;
        const float Lin = rec[(int64_t)SSSGS_REC * m + 19], v = rec[(int64_t)SSSGS_REC * m + 20];
        const float d = fminf(Lin, 1.f) - v;
        const float sg = d > 0.f ? lambda * inv : (d < 0.f ? -lambda * inv : 0.f);
        if (Lin < 1.f) drec[(int64_t)SSSGS_REC * m + 19] += sg;
        drec[(int64_t)SSSGS_REC * m + 20] -= sg;
        const float l = lambda * fabsf(d) * inv;
        if (p == s_p0) atomicAdd(&s_sum[0], l);
        else if (p == s_p0 + 1) atomicAdd(&s_sum[1], l);
        else atomicAdd(d_loss + p, l);                    // a block spanning more than two pairs
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(d_loss + s_p0, s_sum[0]);
        if (s_p0 + 1 < n_pairs) atomicAdd(d_loss + s_p0 + 1, s_sum[1]);
    }
}

Win gaussian_window() {
    Win w;
    double t[2 * R + 1], s = 0.0;
    for (int k = 0; k <= 2 * R; ++k) {
        const double r = k - R;
        t[k] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
        s += t[k];
    }
    for (int k = 0; k <= 2 * R; ++k) w.w[k] = (float)(t[k] / s);
    return w;
}

template <int TILE>
int launch_image_loss(const sssgs_pair* d, int n, int tiles, int64_t n_pix, const float* img, const float* target,
                      float lambda, float* dimg, float* d_loss, float* coef, cudaStream_t st) {
    using T = SsimTile<TILE>;
    const Win w = gaussian_window();
    cudaFuncSetAttribute(k_ssim_moments<TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM_A);
    cudaFuncSetAttribute(k_ssim_grad<TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM_B);
    k_ssim_moments<TILE><<<tiles, T::NT, T::SMEM_A, st>>>(d, n, tiles, n_pix, img, target, w, lambda, coef, d_loss);
    k_ssim_grad<TILE><<<tiles, T::NT, T::SMEM_B, st>>>(d, n, tiles, n_pix, img, target, w, lambda, coef, dimg);
    sssgs::note_launches(2);
    return launch_status();
}

}  // namespace
}  // namespace sssgs

using namespace sssgs;

extern "C" size_t sssgs_image_loss_workspace_bytes(int64_t n_pixels) {
    return n_pixels < 0 ? 0 : (size_t)n_pixels * 9 * sizeof(float) + 256;
}

extern "C" int sssgs_image_loss(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                int n_pairs, const float* img, const float* target, float lambda_dssim,
                                float* dimg, float* d_loss, void* workspace, size_t workspace_bytes,
                                sssgs_stream stream) {
    if (!cfg || !h_pairs || !d_pairs || n_pairs <= 0 || !img || !target || !dimg || !d_loss)
        return SSSGS_ERR_INVALID_ARG;
    if (!(lambda_dssim >= 0.f && lambda_dssim <= 1.f)) return SSSGS_ERR_INVALID_ARG;
    const sssgs_pair& L = h_pairs[n_pairs - 1];
    const int64_t n_pix = L.pixel_offset + (int64_t)L.W * L.H;
    const int tiles = L.tile_offset + L.tiles_x * L.tiles_y;
    if (!workspace || workspace_bytes < sssgs_image_loss_workspace_bytes(n_pix)) return SSSGS_ERR_WORKSPACE;
    float* coef = (float*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    cudaStream_t st = (cudaStream_t)stream;
    switch (cfg->tile) {
        case 8: return launch_image_loss<8>(d_pairs, n_pairs, tiles, n_pix, img, target, lambda_dssim, dimg, d_loss, coef, st);
        case 16: return launch_image_loss<16>(d_pairs, n_pairs, tiles, n_pix, img, target, lambda_dssim, dimg, d_loss, coef, st);
        case 32: return launch_image_loss<32>(d_pairs, n_pairs, tiles, n_pix, img, target, lambda_dssim, dimg, d_loss, coef, st);
        default: return SSSGS_ERR_INVALID_ARG;
    }
}

extern "C" int sssgs_incident_loss(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                                   const float* rec, float lambda_incident, float* drec, float* d_loss,
                                   sssgs_stream stream) {
    if (!h_pairs || !d_pairs || n_pairs <= 0 || !rec || !drec || !d_loss) return SSSGS_ERR_INVALID_ARG;
    const int64_t n = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    if (n == 0) return SSSGS_OK;
    k_incident<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_pairs, n_pairs, n, rec,
                                                                              lambda_incident, drec, d_loss);
    sssgs::note_launches(1);
    return launch_status();
}
