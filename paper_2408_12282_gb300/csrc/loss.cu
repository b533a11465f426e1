// Training losses of Appendix E ("Losses"), fused into the backward step:
//   image loss  L_img = (1 - lambda) L1 + lambda (1 - SSIM)  per view/light pair
//   incident    L_inc = lambda_inc * mean_i |min(L_in_i, 1) - v_i|  per pair
// SSIM: Wang et al. (2004) with an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2,
// averaged over the pair's pixels and channels.
//
// Image loss, two passes over every pair's tiles (the render tile grid, one
// pixel per thread, the window halo of 5 pixels staged in shared memory):
//   A: windowed moments mu_x, mu_y, E[x^2], E[y^2], E[xy] (separable: rows,
//      then columns), the per-pixel SSIM and L1 terms of the loss, and the
//      three coefficient maps of the gradient (dS/dmu_x, dS/dE[x^2],
//      dS/dE[xy] for the mean over the pair) into the workspace;
//   B: the windowed sums of those maps give
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
struct LossTile {
    static constexpr int E = TILE + 2 * R;     // staged edge
};

// Pixel (i, j) of this block's tile and the staged window origin.
template <int TILE>
__device__ __forceinline__ void tile_origin(const sssgs_pair& P, int tile, int& x0, int& y0) {
    const int lt = tile - P.tile_offset;
    x0 = (lt % P.tiles_x) * TILE;
    y0 = (lt / P.tiles_x) * TILE;
}

// Pass A. coef[pix * 9 + 3 c + (0, 1, 2)] = (dS/dmu_x, dS/dE[x^2], dS/dE[xy])
// of channel c for the mean SSIM of the pair; d_loss[pair] += loss terms.
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_ssim_moments(const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                              const float* __restrict__ img,
                                                              const float* __restrict__ target, Win win,
                                                              float lambda, float* __restrict__ coef,
                                                              float* __restrict__ d_loss) {
    constexpr int E = LossTile<TILE>::E;
    __shared__ float sx[E * E], sy[E * E];
    __shared__ float sh[5][E * TILE];
    __shared__ float s_red[TILE * TILE / 32];
    __shared__ __align__(16) sssgs_pair sP;
    const int tile = blockIdx.x, tid = threadIdx.x;
    if (tid < 8) {
        const int pi = pair_of_tile(pairs, n_pairs, tile);
        reinterpret_cast<float4*>(&sP)[tid] = reinterpret_cast<const float4*>(pairs + pi)[tid];
    }
    __syncthreads();
    int x0, y0;
    tile_origin<TILE>(sP, tile, x0, y0);
    const int ti = tid % TILE, tj = tid / TILE;
    const int i = x0 + ti, j = y0 + tj;
    const bool inside = i < sP.W && j < sP.H;
    const int64_t pix = sP.pixel_offset + (int64_t)j * sP.W + i;
    const float inv_n = 1.f / (3.f * (float)sP.W * (float)sP.H);
    float part = 0.f;
    for (int c = 0; c < 3; ++c) {
        for (int k = tid; k < E * E; k += TILE * TILE) {
            const int gi = x0 - R + k % E, gj = y0 - R + k / E;
            float xv = 0.f, yv = 0.f;
            if (gi >= 0 && gi < sP.W && gj >= 0 && gj < sP.H) {
                const int64_t q = sP.pixel_offset + (int64_t)gj * sP.W + gi;
                xv = img[3 * q + c];
                yv = target[3 * q + c];
            }
            sx[k] = xv;
            sy[k] = yv;
        }
        __syncthreads();
        for (int k = tid; k < E * TILE; k += TILE * TILE) {       // rows: all E staged rows, TILE columns
            const int r = k / TILE, cc = k % TILE;
            float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t <= 2 * R; ++t) {
                const float xv = sx[r * E + cc + t], yv = sy[r * E + cc + t], w = win.w[t];
                a[0] += w * xv;
                a[1] += w * yv;
                a[2] += w * xv * xv;
                a[3] += w * yv * yv;
                a[4] += w * xv * yv;
            }
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][r * TILE + cc] = a[q];
        }
        __syncthreads();
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};                   // columns
#pragma unroll
        for (int t = 0; t <= 2 * R; ++t)
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] += win.w[t] * sh[q][(tj + t) * TILE + ti];
        if (inside) {
            const float mx = m[0], my = m[1];
            const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
            const float A1 = 2.f * mx * my + C1, A2 = 2.f * sxy + C2;
            const float B1 = mx * mx + my * my + C1, B2 = sxx + syy + C2;
            const float iB = 1.f / (B1 * B2);
            const float S = A1 * A2 * iB;
            const float dA1 = A2 * iB * inv_n, dA2 = A1 * iB * inv_n;
            const float dB1 = -S / B1 * inv_n, dB2 = -S / B2 * inv_n;
            const float d_sxx = dB2, d_sxy = 2.f * dA2;
            const float d_mx = dA1 * 2.f * my + dB1 * 2.f * mx - 2.f * mx * d_sxx - my * d_sxy;
            float* cf = coef + 9 * pix + 3 * c;
            cf[0] = d_mx;
            cf[1] = d_sxx;
            cf[2] = d_sxy;
            const float xv = sx[(tj + R) * E + ti + R], yv = sy[(tj + R) * E + ti + R];
            part += ((1.f - lambda) * fabsf(xv - yv) - lambda * S) * inv_n;
        }
        __syncthreads();
    }
    // block sum of the loss terms; the pair's first tile also adds lambda (the 1 of 1 - SSIM)
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(SSSGS_FULL, part, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
        float s = 0.f;
        for (int w = 0; w < TILE * TILE / 32; ++w) s += s_red[w];
        if (tile == sP.tile_offset) s += lambda;
        atomicAdd(d_loss + pair_of_tile(pairs, n_pairs, tile), s);
    }
}

// Pass B: dimg = (1 - lambda) sign(x - y) / n - lambda (W*a + 2 x W*b + y W*c).
template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_ssim_grad(const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                           const float* __restrict__ img,
                                                           const float* __restrict__ target, Win win, float lambda,
                                                           const float* __restrict__ coef, float* __restrict__ dimg) {
    constexpr int E = LossTile<TILE>::E;
    __shared__ float sc[3][E * E];
    __shared__ float sh[3][E * TILE];
    __shared__ __align__(16) sssgs_pair sP;
    const int tile = blockIdx.x, tid = threadIdx.x;
    if (tid < 8) {
        const int pi = pair_of_tile(pairs, n_pairs, tile);
        reinterpret_cast<float4*>(&sP)[tid] = reinterpret_cast<const float4*>(pairs + pi)[tid];
    }
    __syncthreads();
    int x0, y0;
    tile_origin<TILE>(sP, tile, x0, y0);
    const int ti = tid % TILE, tj = tid / TILE;
    const int i = x0 + ti, j = y0 + tj;
    const bool inside = i < sP.W && j < sP.H;
    const int64_t pix = sP.pixel_offset + (int64_t)j * sP.W + i;
    const float inv_n = 1.f / (3.f * (float)sP.W * (float)sP.H);
    for (int c = 0; c < 3; ++c) {
        for (int k = tid; k < E * E; k += TILE * TILE) {
            const int gi = x0 - R + k % E, gj = y0 - R + k / E;
            float a = 0.f, b = 0.f, d = 0.f;
            if (gi >= 0 && gi < sP.W && gj >= 0 && gj < sP.H) {
                const float* cf = coef + 9 * (sP.pixel_offset + (int64_t)gj * sP.W + gi) + 3 * c;
                a = cf[0];
                b = cf[1];
                d = cf[2];
            }
            sc[0][k] = a;
            sc[1][k] = b;
            sc[2][k] = d;
        }
        __syncthreads();
        for (int k = tid; k < E * TILE; k += TILE * TILE) {
            const int r = k / TILE, cc = k % TILE;
            float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t <= 2 * R; ++t)
#pragma unroll
                for (int q = 0; q < 3; ++q) s[q] += win.w[t] * sc[q][r * E + cc + t];
#pragma unroll
            for (int q = 0; q < 3; ++q) sh[q][r * TILE + cc] = s[q];
        }
        __syncthreads();
        if (inside) {
            float s[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int t = 0; t <= 2 * R; ++t)
#pragma unroll
                for (int q = 0; q < 3; ++q) s[q] += win.w[t] * sh[q][(tj + t) * TILE + ti];
            const float xv = img[3 * pix + c], yv = target[3 * pix + c];
            const float d = xv - yv;
            const float sg = d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f);
            dimg[3 * pix + c] = (1.f - lambda) * sg * inv_n - lambda * (s[0] + 2.f * xv * s[1] + yv * s[2]);
        }
        __syncthreads();
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
int launch_image_loss(const sssgs_pair* d, int n, int tiles, const float* img, const float* target, float lambda,
                      float* dimg, float* d_loss, float* coef, cudaStream_t st) {
    const Win w = gaussian_window();
    k_ssim_moments<TILE><<<tiles, TILE * TILE, 0, st>>>(d, n, img, target, w, lambda, coef, d_loss);
    k_ssim_grad<TILE><<<tiles, TILE * TILE, 0, st>>>(d, n, img, target, w, lambda, coef, dimg);
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
        case 8: return launch_image_loss<8>(d_pairs, n_pairs, tiles, img, target, lambda_dssim, dimg, d_loss, coef, st);
        case 16: return launch_image_loss<16>(d_pairs, n_pairs, tiles, img, target, lambda_dssim, dimg, d_loss, coef, st);
        case 32: return launch_image_loss<32>(d_pairs, n_pairs, tiles, img, target, lambda_dssim, dimg, d_loss, coef, st);
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
