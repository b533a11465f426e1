// Per-Gaussian shading: the paper's "w/o Deferred" ablation (appendix
// "Ablation": the method without the deferred shading stage). Each Gaussian
// is shaded on its own at its mean x = mu with its own attributes (Eq. 4 BRDF,
// Eq. 7 blend; shade_point, the same arithmetic the deferred path applies per
// pixel), and the colours are alpha-composited (Eq. 3) into the image.
//
// The path reuses the unfused compositing kernels: sssgs_shade_gaussians_fwd
// writes a copy of the records whose feature slots carry the colour (6..8)
// and zeros (9..20); the composite of those records puts the image in G-buffer
// channels 0..2 (sssgs_colors_to_image copies it out, black background). The
// backward turns dL/dimg into a G-buffer gradient (sssgs_colors_to_image_bwd),
// the composite backward gives dL/dcolour per Gaussian in gradient-record
// slots 6..8, and sssgs_shade_gaussians_bwd replaces them by the gradients of
// the shaded attributes (slots 7..19, the network outputs included) and of the
// mean (slots 21..23, which sssgs_project_bwd adds to dL/dmu).
#include "raster_common.cuh"

namespace sssgs {
namespace {

__device__ __forceinline__ void gauss_inputs(const float* __restrict__ r, float3& nbar, float* bb, float& rb,
                                             float& mb, float& sb, float* Ls, float& Li) {
    nbar = make_float3(r[7], r[8], r[9]);
    bb[0] = r[10]; bb[1] = r[11]; bb[2] = r[12];
    rb = r[13]; mb = r[14]; sb = r[15];
    Ls[0] = r[16]; Ls[1] = r[17]; Ls[2] = r[18];
    Li = r[19];
}

__global__ void __launch_bounds__(256) k_shade_gauss_fwd(const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                         int64_t n_items, sssgs_scene sc,
                                                         const float* __restrict__ rec, float* __restrict__ out) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_items) return;
    const int p = pair_of_item(pairs, n_pairs, m);
    const sssgs_pair& P = pairs[p];
    const int64_t g = P.g_begin + (m - P.item_offset);
    const float* r = rec + (int64_t)SSSGS_REC * m;
    float3 nbar;
    float bb[3], Ls[3], rb, mb, sb, Li, Lc[3];
    gauss_inputs(r, nbar, bb, rb, mb, sb, Ls, Li);
    const float3 x = make_float3(sc.mu[3 * g], sc.mu[3 * g + 1], sc.mu[3 * g + 2]);
    shade_point<false>(nbar, bb, rb, mb, sb, Ls, Li, x, cam_center(P),
                       make_float3(P.light[0], P.light[1], P.light[2]), Lc, nullptr, nullptr, nullptr);
    float* o = out + (int64_t)SSSGS_REC * m;
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = r[k];
    o[6] = Lc[0]; o[7] = Lc[1]; o[8] = Lc[2];
#pragma unroll
    for (int k = 9; k <= 20; ++k) o[k] = 0.f;
    o[21] = r[21]; o[22] = r[22]; o[23] = r[23];
}

__global__ void __launch_bounds__(256) k_shade_gauss_bwd(const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                         int64_t n_items, sssgs_scene sc,
                                                         const float* __restrict__ rec, float* __restrict__ drec) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_items) return;
    const int p = pair_of_item(pairs, n_pairs, m);
    const sssgs_pair& P = pairs[p];
    const int64_t g = P.g_begin + (m - P.item_offset);
    const float* r = rec + (int64_t)SSSGS_REC * m;
    float* d = drec + (int64_t)SSSGS_REC * m;
    const float gL[3] = {d[6], d[7], d[8]};
    float3 nbar, dx = make_float3(0.f, 0.f, 0.f);
    float bb[3], Ls[3], rb, mb, sb, Li, Lc[3], dg[SSSGS_NF];
#pragma unroll
    for (int k = 0; k < SSSGS_NF; ++k) dg[k] = 0.f;
    if (gL[0] != 0.f || gL[1] != 0.f || gL[2] != 0.f) {
        gauss_inputs(r, nbar, bb, rb, mb, sb, Ls, Li);
        const float3 x = make_float3(sc.mu[3 * g], sc.mu[3 * g + 1], sc.mu[3 * g + 2]);
        shade_point<true>(nbar, bb, rb, mb, sb, Ls, Li, x, cam_center(P),
                          make_float3(P.light[0], P.light[1], P.light[2]), Lc, gL, dg, &dx);
    }
    d[6] = 0.f;                                   // the composited depth is not used here
#pragma unroll
    for (int k = 1; k <= 13; ++k) d[6 + k] = dg[k];
    d[20] = 0.f;
    d[21] = dx.x; d[22] = dx.y; d[23] = dx.z;
}

__global__ void __launch_bounds__(256) k_colors_to_image(int64_t n_pix, const float* __restrict__ gbuf,
                                                         float* __restrict__ img) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_pix) return;
    const float4 v = reinterpret_cast<const float4*>(gbuf + (int64_t)SSSGS_GBUF * q)[0];
    img[3 * q] = v.x;
    img[3 * q + 1] = v.y;
    img[3 * q + 2] = v.z;
}

__global__ void __launch_bounds__(256) k_colors_to_image_bwd(int64_t n_pix, const float* __restrict__ dimg,
                                                             float* __restrict__ dgbuf) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_pix) return;
    float4* o = reinterpret_cast<float4*>(dgbuf + (int64_t)SSSGS_GBUF * q);
    o[0] = make_float4(dimg[3 * q], dimg[3 * q + 1], dimg[3 * q + 2], 0.f);
    o[1] = o[2] = o[3] = make_float4(0.f, 0.f, 0.f, 0.f);     // other features and T: no gradient
}

int64_t items_of(const sssgs_pair* h, int n) { return h[n - 1].item_offset + h[n - 1].g_count; }
int64_t pixels_of(const sssgs_pair* h, int n) { return h[n - 1].pixel_offset + (int64_t)h[n - 1].W * h[n - 1].H; }

}  // namespace
}  // namespace sssgs

using namespace sssgs;

extern "C" int sssgs_shade_gaussians_fwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                                         const sssgs_scene* scene, const float* rec, float* rec_colors,
                                         sssgs_stream stream) {
    if (!h_pairs || !d_pairs || n_pairs <= 0 || !scene || !scene->mu || !rec || !rec_colors || rec == rec_colors)
        return SSSGS_ERR_INVALID_ARG;
    const int64_t n = items_of(h_pairs, n_pairs);
    if (n == 0) return SSSGS_OK;
    k_shade_gauss_fwd<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_pairs, n_pairs, n, *scene,
                                                                                    rec, rec_colors);
    sssgs::note_launches(1);
    return launch_status();
}

extern "C" int sssgs_shade_gaussians_bwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                                         const sssgs_scene* scene, const float* rec, float* drec,
                                         sssgs_stream stream) {
    if (!h_pairs || !d_pairs || n_pairs <= 0 || !scene || !scene->mu || !rec || !drec)
        return SSSGS_ERR_INVALID_ARG;
    const int64_t n = items_of(h_pairs, n_pairs);
    if (n == 0) return SSSGS_OK;
    k_shade_gauss_bwd<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_pairs, n_pairs, n, *scene,
                                                                                    rec, drec);
    sssgs::note_launches(1);
    return launch_status();
}

extern "C" int sssgs_colors_to_image(const sssgs_pair* h_pairs, int n_pairs, const float* gbuf, float* img,
                                     sssgs_stream stream) {
    if (!h_pairs || n_pairs <= 0 || !gbuf || !img || ((uintptr_t)gbuf & 15)) return SSSGS_ERR_INVALID_ARG;
    const int64_t n = pixels_of(h_pairs, n_pairs);
    k_colors_to_image<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, gbuf, img);
    sssgs::note_launches(1);
    return launch_status();
}

extern "C" int sssgs_colors_to_image_bwd(const sssgs_pair* h_pairs, int n_pairs, const float* dimg, float* dgbuf,
                                         sssgs_stream stream) {
    if (!h_pairs || n_pairs <= 0 || !dimg || !dgbuf || ((uintptr_t)dgbuf & 15)) return SSSGS_ERR_INVALID_ARG;
    const int64_t n = pixels_of(h_pairs, n_pairs);
    k_colors_to_image_bwd<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, dimg, dgbuf);
    sssgs::note_launches(1);
    return launch_status();
}
