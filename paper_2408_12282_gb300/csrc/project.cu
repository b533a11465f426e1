// EWA projection of every (pair, Gaussian) item and its backward.
//   Eq. 1: G(x) = exp(-0.5 (x - mu)^T Sigma^-1 (x - mu))
//   Eq. 2: Sigma' = J W Sigma W^T J^T, J the Jacobian of the affine
//          approximation of the perspective projection, W the view rotation.
//   Sigma = R(q) diag(s)^2 R(q)^T with s = exp(log_s) and q normalised
//   (Section 3.1, "3D Gaussian Splatting").
#include "common.cuh"

namespace sssgs {

struct ProjGeom {
    float q[4], qn;      // normalised quaternion and the norm of the raw one
    float R[9];          // rotation of q
    float s[3];          // scales
    float Sig[6];        // 3D covariance (00, 01, 02, 11, 12, 22)
    float t[3];          // camera-space mean
    float T[6];          // J * Rc (2 x 3)
    float a, b, c;       // dilated 2D covariance
    float det;
    float o;             // opacity
    bool valid;
};

__device__ __forceinline__ void project_geom(const sssgs_pair& P, const sssgs_cfg& cfg,
                                             const float* __restrict__ mu, const float* __restrict__ log_s,
                                             const float* __restrict__ quat, const float* __restrict__ logit_o,
                                             int64_t g, ProjGeom& G) {
    float m0 = mu[3 * g], m1 = mu[3 * g + 1], m2 = mu[3 * g + 2];
    // view-space mean; z by the fixed fused chain that also defines the depth order
    G.t[0] = fmaf(P.R[0], m0, fmaf(P.R[1], m1, fmaf(P.R[2], m2, P.t[0])));
    G.t[1] = fmaf(P.R[3], m0, fmaf(P.R[4], m1, fmaf(P.R[5], m2, P.t[1])));
    G.t[2] = fmaf(P.R[6], m0, fmaf(P.R[7], m1, fmaf(P.R[8], m2, P.t[2])));
    G.o = 1.f / (1.f + expf(-logit_o[g]));
    float qw = quat[4 * g], qx = quat[4 * g + 1], qy = quat[4 * g + 2], qz = quat[4 * g + 3];
    G.qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    float iq = 1.f / G.qn;
    float w = qw * iq, x = qx * iq, y = qy * iq, z = qz * iq;
    G.q[0] = w; G.q[1] = x; G.q[2] = y; G.q[3] = z;
    float* R = G.R;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
    for (int k = 0; k < 3; ++k) G.s[k] = expf(log_s[3 * g + k]);
    // Sigma = M M^T, M = R diag(s)
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * G.s[j];
    G.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    G.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    G.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    G.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    G.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    G.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    G.valid = G.t[2] >= cfg.z_near;
    float tz = fmaxf(G.t[2], cfg.z_near);
    float iz = 1.f / tz;
    float J00 = P.fx * iz, J02 = -P.fx * G.t[0] * iz * iz;
    float J11 = P.fy * iz, J12 = -P.fy * G.t[1] * iz * iz;
    for (int j = 0; j < 3; ++j) {
        G.T[j] = J00 * P.R[j] + J02 * P.R[6 + j];
        G.T[3 + j] = J11 * P.R[3 + j] + J12 * P.R[6 + j];
    }
    // Sigma' = T Sigma T^T
    const float* S = G.Sig;
    float u0 = S[0] * G.T[0] + S[1] * G.T[1] + S[2] * G.T[2];
    float u1 = S[1] * G.T[0] + S[3] * G.T[1] + S[4] * G.T[2];
    float u2 = S[2] * G.T[0] + S[4] * G.T[1] + S[5] * G.T[2];
    float v0 = S[0] * G.T[3] + S[1] * G.T[4] + S[2] * G.T[5];
    float v1 = S[1] * G.T[3] + S[3] * G.T[4] + S[4] * G.T[5];
    float v2 = S[2] * G.T[3] + S[4] * G.T[4] + S[5] * G.T[5];
    G.a = G.T[0] * u0 + G.T[1] * u1 + G.T[2] * u2 + cfg.dilation;
    G.b = G.T[3] * u0 + G.T[4] * u1 + G.T[5] * u2;
    G.c = G.T[3] * v0 + G.T[4] * v1 + G.T[5] * v2 + cfg.dilation;
    G.det = G.a * G.c - G.b * G.b;
    G.valid = G.valid && (G.det > cfg.det_eps);
}

__global__ void __launch_bounds__(256) k_project_fwd(sssgs_cfg cfg, const sssgs_pair* __restrict__ pairs,
                                                     int n_pairs, int64_t n_items, sssgs_scene sc,
                                                     const float* __restrict__ mlp_out,
                                                     float4* __restrict__ rec, int4* __restrict__ rect) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_items) return;
    int p = pair_of_item(pairs, n_pairs, m);
    const sssgs_pair& P = pairs[p];
    int64_t g = P.g_begin + (m - P.item_offset);
    ProjGeom G;
    project_geom(P, cfg, sc.mu, sc.log_s, sc.quat, sc.logit_o, g, G);
    float id = 1.f / G.det;
    float ca = G.c * id, cb = -G.b * id, cc = G.a * id;
    float iz = 1.f / G.t[2];
    float mx = P.fx * G.t[0] * iz + P.cx;
    float my = P.fy * G.t[1] * iz + P.cy;
    float L = logf(G.o / cfg.alpha_min);
    bool valid = G.valid && (L > 0.f);
    int4 r = make_int4(1, 0, 1, 0);
    if (valid) {
        // AABB of the support ellipse {p <= L}, padded for float32 rounding
        float ex = sqrtf(2.f * L * G.a) * 1.001f + 0.01f;
        float ey = sqrtf(2.f * L * G.c) * 1.001f + 0.01f;
        float fi0 = fmaxf(ceilf(mx - ex - 0.5f), 0.f);
        float fi1 = fminf(floorf(mx + ex - 0.5f), (float)(P.W - 1));
        float fj0 = fmaxf(ceilf(my - ey - 0.5f), 0.f);
        float fj1 = fminf(floorf(my + ey - 0.5f), (float)(P.H - 1));
        if (fi0 <= fi1 && fj0 <= fj1) {
            int tile = cfg.tile;
            r = make_int4((int)fi0 / tile, (int)fi1 / tile, (int)fj0 / tile, (int)fj1 / tile);
        }
    }
    rect[m] = r;
    const float* n = sc.normal + 3 * g;
    const float* b = sc.base + 3 * g;
    const float4 mo = mlp_out ? reinterpret_cast<const float4*>(mlp_out)[m] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4* o = rec + 6 * m;
    o[0] = make_float4(mx, my, ca, cb);
    o[1] = make_float4(cc, G.o, G.t[2], n[0]);
    o[2] = make_float4(n[1], n[2], b[0], b[1]);
    o[3] = make_float4(b[2], sc.rough[g], sc.metal[g], sc.sss[g]);
    o[4] = mo;
    // tile / sub-tile culling constants of the render kernels: 1/ca, 1/cc and
    // the padded support level of {p <= ln(o / alpha_min)}
    o[5] = make_float4(sc.vis_item ? sc.vis_item[m] : sc.vis[g], 1.f / ca, 1.f / cc, L * 1.001f + 0.01f);
}

// One thread per scene Gaussian; sums the gradient of every pair rendering it.
__global__ void __launch_bounds__(128) k_project_bwd(sssgs_cfg cfg, const sssgs_pair* __restrict__ pairs,
                                                     int n_pairs, sssgs_scene sc, const float* __restrict__ drec,
                                                     const float* __restrict__ dx_items, sssgs_scene_grad gr) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sc.n) return;
    float dmu[3] = {0, 0, 0}, dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0}, dlo = 0;
    float dn[3] = {0, 0, 0}, db[3] = {0, 0, 0}, dr = 0, dm = 0, dss = 0, dv = 0;
    for (int p = 0; p < n_pairs; ++p) {
        const sssgs_pair& P = pairs[p];
        if (g < P.g_begin || g >= (int64_t)P.g_begin + P.g_count) continue;
        int64_t m = P.item_offset + (g - P.g_begin);
        float dvm = 0.f;                 // dL/dv of this item (record and network input)
        if (dx_items) {
            const float* x = dx_items + SSSGS_DX * m;
            dmu[0] += x[0]; dmu[1] += x[1]; dmu[2] += x[2];
            dn[0] += x[3]; dn[1] += x[4]; dn[2] += x[5];
            dvm += x[6];
            dq[0] += x[7]; dq[1] += x[8]; dq[2] += x[9]; dq[3] += x[10];
            dls[0] += x[11]; dls[1] += x[12]; dls[2] += x[13];
        }
        const float* d = drec ? drec + (int64_t)SSSGS_REC * m : nullptr;
        if (d) {
            dn[0] += d[7]; dn[1] += d[8]; dn[2] += d[9];
            db[0] += d[10]; db[1] += d[11]; db[2] += d[12];
            dr += d[13]; dm += d[14]; dss += d[15]; dvm += d[20];
        }
        if (gr.vis_item) gr.vis_item[m] += dvm;      // per-item visibility: its gradient stays per item
        else dv += dvm;
        if (!d) continue;
        dmu[0] += d[21]; dmu[1] += d[22]; dmu[2] += d[23];   // per-Gaussian shading at the mean (zero otherwise)
        float dmx = d[0], dmy = d[1], dca = d[2], dcb = d[3], dcc = d[4], dop = d[5], dz = d[6];
        if (dmx == 0.f && dmy == 0.f && dca == 0.f && dcb == 0.f && dcc == 0.f && dop == 0.f && dz == 0.f)
            continue;
        ProjGeom G;
        project_geom(P, cfg, sc.mu, sc.log_s, sc.quat, sc.logit_o, g, G);
        if (!G.valid) continue;
        dlo += dop * G.o * (1.f - G.o);
        float tx = G.t[0], ty = G.t[1], tz = G.t[2];
        float iz = 1.f / tz, iz2 = iz * iz, iz3 = iz2 * iz;
        float dt0 = dmx * P.fx * iz;
        float dt1 = dmy * P.fy * iz;
        float dt2 = -(dmx * P.fx * tx + dmy * P.fy * ty) * iz2 + dz;
        // conic (ca, cb, cc) = (c, -b, a) / det  ->  symmetric dSigma' = -C Gb C
        float id = 1.f / G.det;
        float ca = G.c * id, cb = -G.b * id, cc = G.a * id;
        float hb = 0.5f * dcb;
        float x00 = ca * dca + cb * hb, x01 = ca * hb + cb * dcc;   // C * Gb
        float x10 = cb * dca + cc * hb, x11 = cb * hb + cc * dcc;
        float g00 = -(x00 * ca + x01 * cb);                        // -(C Gb) C
        float g01 = -(x00 * cb + x01 * cc);
        float g11 = -(x10 * cb + x11 * cc);
        const float* T = G.T;
        const float* S = G.Sig;
        // GT = Gs T (2x3)
        float GT0[3], GT1[3];
        for (int j = 0; j < 3; ++j) {
            GT0[j] = g00 * T[j] + g01 * T[3 + j];
            GT1[j] = g01 * T[j] + g11 * T[3 + j];
        }
        // dT = 2 GT Sigma ; dJ = dT Rc^T
        float Sf[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
        float dT0[3], dT1[3];
        for (int j = 0; j < 3; ++j) {
            dT0[j] = 2.f * (GT0[0] * Sf[j] + GT0[1] * Sf[3 + j] + GT0[2] * Sf[6 + j]);
            dT1[j] = 2.f * (GT1[0] * Sf[j] + GT1[1] * Sf[3 + j] + GT1[2] * Sf[6 + j]);
        }
        float dJ00 = dT0[0] * P.R[0] + dT0[1] * P.R[1] + dT0[2] * P.R[2];
        float dJ02 = dT0[0] * P.R[6] + dT0[1] * P.R[7] + dT0[2] * P.R[8];
        float dJ11 = dT1[0] * P.R[3] + dT1[1] * P.R[4] + dT1[2] * P.R[5];
        float dJ12 = dT1[0] * P.R[6] + dT1[1] * P.R[7] + dT1[2] * P.R[8];
        dt0 += -dJ02 * P.fx * iz2;
        dt1 += -dJ12 * P.fy * iz2;
        dt2 += -dJ00 * P.fx * iz2 + 2.f * dJ02 * P.fx * tx * iz3 - dJ11 * P.fy * iz2 + 2.f * dJ12 * P.fy * ty * iz3;
        for (int i = 0; i < 3; ++i) dmu[i] += P.R[i] * dt0 + P.R[3 + i] * dt1 + P.R[6 + i] * dt2;
        // dSigma = T^T Gs T ; dM = 2 dSigma M ; M = R diag(s)
        float dS[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dS[3 * i + j] = T[i] * GT0[j] + T[3 + i] * GT1[j];
        const float* R = G.R;
        float M[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * G.s[j];
        float dR[9];
        for (int j = 0; j < 3; ++j) {
            float ds = 0.f;
            for (int i = 0; i < 3; ++i) {
                float dMij = 2.f * (dS[3 * i] * M[j] + dS[3 * i + 1] * M[3 + j] + dS[3 * i + 2] * M[6 + j]);
                dR[3 * i + j] = dMij * G.s[j];
                ds += dMij * R[3 * i + j];
            }
            dls[j] += ds * G.s[j];
        }
        float w = G.q[0], x = G.q[1], y = G.q[2], z = G.q[3];
        float e0 = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        float e1 = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2.f * x * dR[8]);
        float e2 = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
        float e3 = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
        float qd = w * e0 + x * e1 + y * e2 + z * e3;
        float iq = 1.f / G.qn;
        dq[0] += (e0 - w * qd) * iq;
        dq[1] += (e1 - x * qd) * iq;
        dq[2] += (e2 - y * qd) * iq;
        dq[3] += (e3 - z * qd) * iq;
    }
    if (gr.mu) for (int k = 0; k < 3; ++k) gr.mu[3 * g + k] += dmu[k];
    if (gr.log_s) for (int k = 0; k < 3; ++k) gr.log_s[3 * g + k] += dls[k];
    if (gr.quat) for (int k = 0; k < 4; ++k) gr.quat[4 * g + k] += dq[k];
    if (gr.logit_o) gr.logit_o[g] += dlo;
    if (gr.normal) for (int k = 0; k < 3; ++k) gr.normal[3 * g + k] += dn[k];
    if (gr.base) for (int k = 0; k < 3; ++k) gr.base[3 * g + k] += db[k];
    if (gr.rough) gr.rough[g] += dr;
    if (gr.metal) gr.metal[g] += dm;
    if (gr.sss) gr.sss[g] += dss;
    if (gr.vis) gr.vis[g] += dv;
}

}  // namespace sssgs

using namespace sssgs;

static bool cfg_ok(const sssgs_cfg* c) {
    return c && (c->tile == 8 || c->tile == 16 || c->tile == 32) && (c->batch == 0 || c->batch == 32 || c->batch == 64) &&
           c->alpha_min > 0.f && c->alpha_max <= 1.f && c->alpha_min < c->alpha_max && c->T_min > 0.f;
}

static int64_t items_of(const sssgs_pair* h, int n) {
    return n > 0 ? h[n - 1].item_offset + h[n - 1].g_count : 0;
}

extern "C" int sssgs_project_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                 int n_pairs, const sssgs_scene* scene, const float* mlp_out,
                                 float* rec, int32_t* rect, sssgs_stream stream) {
    if (!cfg_ok(cfg) || !h_pairs || !d_pairs || n_pairs <= 0 || !scene || !rec || !rect)
        return SSSGS_ERR_INVALID_ARG;
    if (((uintptr_t)rec & 15) || ((uintptr_t)rect & 15) || ((uintptr_t)mlp_out & 15)) return SSSGS_ERR_INVALID_ARG;
    int64_t n = items_of(h_pairs, n_pairs);
    if (n == 0) return SSSGS_OK;
    unsigned blocks = (unsigned)((n + 255) / 256);
    k_project_fwd<<<blocks, 256, 0, (cudaStream_t)stream>>>(*cfg, d_pairs, n_pairs, n, *scene, mlp_out,
                                                           (float4*)rec, (int4*)rect);
    sssgs::note_launches(1);
    return launch_status();
}

extern "C" int sssgs_project_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                 int n_pairs, const sssgs_scene* scene, const float* drec,
                                 const float* dx_items, const sssgs_scene_grad* grad, sssgs_stream stream) {
    if (!cfg_ok(cfg) || !h_pairs || !d_pairs || n_pairs <= 0 || !scene || (!drec && !dx_items) || !grad)
        return SSSGS_ERR_INVALID_ARG;
    if (scene->n == 0) return SSSGS_OK;
    unsigned blocks = (unsigned)((scene->n + 127) / 128);
    k_project_bwd<<<blocks, 128, 0, (cudaStream_t)stream>>>(*cfg, d_pairs, n_pairs, *scene, drec, dx_items, *grad);
    sssgs::note_launches(1);
    return launch_status();
}
