// Network input encoding shared by the CUDA-core and tensor-core networks.
#pragma once
#include "common.cuh"

namespace sssgs {

// Leaky-ReLU negative slope of the paper's network (App. E; the slope is not
// stated, 0.01 is taken).
constexpr float kLReluSlope = 0.01f;

struct MlpDev {
    int kind, L;
    int w[SSSGS_MAX_LAYERS + 1];
    const float* W[SSSGS_MAX_LAYERS];
    const float* b[SSSGS_MAX_LAYERS];
};

// Network input of item m (row of width w[0]) written to x.
// Visibility v of item m (Gaussian g): the per-item array when the scene has
// one (SH visibility at the pair's light direction), else the Gaussian's.
__device__ __forceinline__ float vis_of(const sssgs_scene& sc, int64_t g, int64_t m) {
    return sc.vis_item ? __ldg(sc.vis_item + m) : __ldg(sc.vis + g);
}

// pad = false: the caller has zeroed x, so the columns past the features are
// left alone (a register array then sees no runtime index).
__device__ __forceinline__ void build_input(const MlpDev& net, const sssgs_pair& P, const sssgs_scene& sc,
                                            int64_t g, int64_t m, float* x, bool pad = true) {
    const float m0 = sc.mu[3 * g], m1 = sc.mu[3 * g + 1], m2 = sc.mu[3 * g + 2];
    const float3 C = cam_center(P);
    float3 Vo = make_float3(C.x - m0, C.y - m1, C.z - m2);
    float3 Vi = make_float3(P.light[0] - m0, P.light[1] - m1, P.light[2] - m2);
    const float lo = sqrtf(dot3(Vo, Vo)), li = sqrtf(dot3(Vi, Vi));
    const float3 wo = (1.f / lo) * Vo, wi = (1.f / li) * Vi;
    if (net.kind == SSSGS_MLP_BASIC) {
        x[0] = m0; x[1] = m1; x[2] = m2;
        x[3] = wo.x; x[4] = wo.y; x[5] = wo.z;
        x[6] = wi.x; x[7] = wi.y; x[8] = wi.z;
        return;
    }
    if (net.kind == SSSGS_MLP_PAPER) {   // [n, q/|q|, exp(log_s), w_in, w_out, |light - mu|, v, PE4(mu)]
        const float* q = sc.quat + 4 * g;
        const float iq = 1.f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        x[0] = sc.normal[3 * g]; x[1] = sc.normal[3 * g + 1]; x[2] = sc.normal[3 * g + 2];
        x[3] = q[0] * iq; x[4] = q[1] * iq; x[5] = q[2] * iq; x[6] = q[3] * iq;
        x[7] = expf(sc.log_s[3 * g]); x[8] = expf(sc.log_s[3 * g + 1]); x[9] = expf(sc.log_s[3 * g + 2]);
        x[10] = wi.x; x[11] = wi.y; x[12] = wi.z;
        x[13] = wo.x; x[14] = wo.y; x[15] = wo.z;
        x[16] = li;
        x[17] = vis_of(sc, g, m);
        const float mm[3] = {m0, m1, m2};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float s, co;
                sincospif(ldexpf(mm[c], k), &s, &co);
                x[18 + 6 * k + c] = s;
                x[21 + 6 * k + c] = co;
            }
        }
        if (pad)
            for (int k = 42; k < net.w[0]; ++k) x[k] = 0.f;
        return;
    }
    const float mm[3] = {m0, m1, m2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // sin(2^k pi mu) via sinpi of the exact product 2^k mu: no rounding of pi
            float s, co;
            sincospif(ldexpf(mm[c], k), &s, &co);
            x[6 * k + c] = s;
            x[6 * k + 3 + c] = co;
        }
    }
    x[36] = m0; x[37] = m1; x[38] = m2;
    x[39] = wo.x; x[40] = wo.y; x[41] = wo.z;
    x[42] = wi.x; x[43] = wi.y; x[44] = wi.z;
    x[45] = sc.normal[3 * g]; x[46] = sc.normal[3 * g + 1]; x[47] = sc.normal[3 * g + 2];
    x[48] = li;
    x[49] = vis_of(sc, g, m);
    if (pad)
        for (int k = 50; k < net.w[0]; ++k) x[k] = 0.f;
}

// Input gradient dX (row) -> (dmu, dn, dv, dquat, dlog_s) of item m, written
// to dx[SSSGS_DX] (the last 7 are zero for the BASIC and PE6 inputs).
// KIND is the network kind (compile time, so a register array dX sees no
// runtime index); input_backward dispatches on net.kind.
template <int KIND>
__device__ __forceinline__ void input_backward_k(const sssgs_pair& P, const sssgs_scene& sc, int64_t g,
                                                 const float* dX, float* dx) {
    const float m0 = sc.mu[3 * g], m1 = sc.mu[3 * g + 1], m2 = sc.mu[3 * g + 2];
    const float3 C = cam_center(P);
    float3 Vo = make_float3(C.x - m0, C.y - m1, C.z - m2);
    float3 Vi = make_float3(P.light[0] - m0, P.light[1] - m1, P.light[2] - m2);
    const float lo = sqrtf(dot3(Vo, Vo)), li = sqrtf(dot3(Vi, Vi));
    const float3 wo = (1.f / lo) * Vo, wi = (1.f / li) * Vi;
    constexpr int o_mu = KIND == SSSGS_MLP_BASIC ? 0 : (KIND == SSSGS_MLP_PAPER ? -1 : 36);
    constexpr int o_wo = KIND == SSSGS_MLP_BASIC ? 3 : (KIND == SSSGS_MLP_PAPER ? 13 : 39);
    constexpr int o_wi = KIND == SSSGS_MLP_BASIC ? 6 : (KIND == SSSGS_MLP_PAPER ? 10 : 42);
    float dmu[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 7; k < SSSGS_DX; ++k) dx[k] = 0.f;
    if constexpr (KIND == SSSGS_MLP_BASIC) {
        dx[3] = dx[4] = dx[5] = dx[6] = 0.f;
    } else if constexpr (KIND == SSSGS_MLP_PAPER) {
        const float mm[3] = {m0, m1, m2};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float f = ldexpf(kPi, k);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float s, co;
                sincospif(ldexpf(mm[c], k), &s, &co);
                dmu[c] += f * (dX[18 + 6 * k + c] * co - dX[21 + 6 * k + c] * s);
            }
        }
        dmu[0] -= dX[16] * wi.x; dmu[1] -= dX[16] * wi.y; dmu[2] -= dX[16] * wi.z;
        dx[3] = dX[0]; dx[4] = dX[1]; dx[5] = dX[2];
        dx[6] = dX[17];
        // q/|q|: dq = (g - qn (qn . g)) / |q| ; exp(log_s): dlog_s = g * s
        const float* q = sc.quat + 4 * g;
        const float iq = 1.f / sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float qn[4] = {q[0] * iq, q[1] * iq, q[2] * iq, q[3] * iq};
        const float qg = qn[0] * dX[3] + qn[1] * dX[4] + qn[2] * dX[5] + qn[3] * dX[6];
#pragma unroll
        for (int k = 0; k < 4; ++k) dx[7 + k] = (dX[3 + k] - qn[k] * qg) * iq;
#pragma unroll
        for (int k = 0; k < 3; ++k) dx[11 + k] = dX[7 + k] * expf(sc.log_s[3 * g + k]);
    } else {
        const float mm[3] = {m0, m1, m2};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float f = ldexpf(kPi, k);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float s, co;
                sincospif(ldexpf(mm[c], k), &s, &co);
                dmu[c] += f * (dX[6 * k + c] * co - dX[6 * k + 3 + c] * s);
            }
        }
        dx[3] = dX[45]; dx[4] = dX[46]; dx[5] = dX[47];
        dx[6] = dX[49];
        dmu[0] -= dX[48] * wi.x; dmu[1] -= dX[48] * wi.y; dmu[2] -= dX[48] * wi.z;
    }
    if constexpr (o_mu >= 0) {
        dmu[0] += dX[o_mu]; dmu[1] += dX[o_mu + 1]; dmu[2] += dX[o_mu + 2];
    }
    // d unit(P - mu) / d mu applied to g:  -(g - w (w.g)) / |P - mu|
    const float3 go = make_float3(dX[o_wo], dX[o_wo + 1], dX[o_wo + 2]);
    const float3 gi = make_float3(dX[o_wi], dX[o_wi + 1], dX[o_wi + 2]);
    const float3 bo = (-1.f / lo) * (go - dot3(wo, go) * wo);
    const float3 bi = (-1.f / li) * (gi - dot3(wi, gi) * wi);
    dx[0] = dmu[0] + bo.x + bi.x;
    dx[1] = dmu[1] + bo.y + bi.y;
    dx[2] = dmu[2] + bo.z + bi.z;
}

__device__ __forceinline__ void input_backward(const MlpDev& net, const sssgs_pair& P, const sssgs_scene& sc,
                                               int64_t g, const float* dX, float* dx) {
    if (net.kind == SSSGS_MLP_BASIC) input_backward_k<SSSGS_MLP_BASIC>(P, sc, g, dX, dx);
    else if (net.kind == SSSGS_MLP_PAPER) input_backward_k<SSSGS_MLP_PAPER>(P, sc, g, dX, dx);
    else input_backward_k<SSSGS_MLP_PE6>(P, sc, g, dX, dx);
}

// PE6 input (64 features, fixed layout) with compile-time indices, so the
// row stays in registers.
// Fourier part of the PE6 input, frequencies k in [K0, K1): x[6 (k - K0) + c]
// = sin(2^k pi mu_c), x[6 (k - K0) + 3 + c] = cos(2^k pi mu_c), i.e. x[0] is
// input column 6 K0.
template <int K0, int K1>
__device__ __forceinline__ void pe6_fourier(const float (&mm)[3], float* x) {
#pragma unroll
    for (int k = K0; k < K1; ++k) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sn, cs;
            sincospif(ldexpf(mm[c], k), &sn, &cs);
            x[6 * (k - K0) + c] = sn;
            x[6 * (k - K0) + 3 + c] = cs;
        }
    }
}

// Input columns [36, 64) (x[0] is column 36): mu, unit(camera - mu),
// unit(light - mu), n, |light - mu|, v, zero padding.
__device__ __forceinline__ void pe6_direct(const sssgs_pair& P, const float (&mm)[3], const float (&nn)[3], float vv,
                                           float* x) {
    const float3 C = cam_center(P);
    const float3 Vo = make_float3(C.x - mm[0], C.y - mm[1], C.z - mm[2]);
    const float3 Vi = make_float3(P.light[0] - mm[0], P.light[1] - mm[1], P.light[2] - mm[2]);
    const float lo = sqrtf(dot3(Vo, Vo)), li = sqrtf(dot3(Vi, Vi));
    const float3 wo = (1.f / lo) * Vo, wi = (1.f / li) * Vi;
    x[0] = mm[0]; x[1] = mm[1]; x[2] = mm[2];
    x[3] = wo.x; x[4] = wo.y; x[5] = wo.z;
    x[6] = wi.x; x[7] = wi.y; x[8] = wi.z;
    x[9] = nn[0]; x[10] = nn[1]; x[11] = nn[2];
    x[12] = li;
    x[13] = vv;
#pragma unroll
    for (int k = 14; k < 28; ++k) x[k] = 0.f;
}

// The per-Gaussian network inputs of one item.
struct Pe6Params {
    float mu[3], n[3], v;
};
__device__ __forceinline__ Pe6Params load_pe6_params(const sssgs_scene& sc, int64_t g, int64_t m) {
    Pe6Params q;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        q.mu[c] = __ldg(sc.mu + 3 * g + c);
        q.n[c] = __ldg(sc.normal + 3 * g + c);
    }
    q.v = vis_of(sc, g, m);
    return q;
}

__device__ __forceinline__ void build_input_pe6(const sssgs_pair& P, const sssgs_scene& sc, int64_t g, int64_t m,
                                                float (&x)[64]) {
    const Pe6Params q = load_pe6_params(sc, g, m);
    pe6_fourier<0, 6>(q.mu, x);
    pe6_direct(P, q.mu, q.n, q.v, x + 36);
}

// Backward of pe6_fourier<K0, K1>: adds the Fourier columns' contribution to
// dL/dmu (dX[0] is input column 6 K0).
template <int K0, int K1>
__device__ __forceinline__ void pe6_fourier_bwd(const float (&mm)[3], const float* dX, float (&dmu)[3]) {
#pragma unroll
    for (int k = K0; k < K1; ++k) {
        const float f = ldexpf(kPi, k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float sn, cs;
            sincospif(ldexpf(mm[c], k), &sn, &cs);
            dmu[c] += f * (dX[6 * (k - K0) + c] * cs - dX[6 * (k - K0) + 3 + c] * sn);
        }
    }
}

// Backward of pe6_direct (dX[0] is input column 36): dx = (dL/dmu from the
// direct columns, dL/dn, dL/dv).
__device__ __forceinline__ void pe6_direct_bwd(const sssgs_pair& P, const float (&mm)[3], const float* dX,
                                               float (&dx)[7]) {
    const float3 C = cam_center(P);
    const float3 Vo = make_float3(C.x - mm[0], C.y - mm[1], C.z - mm[2]);
    const float3 Vi = make_float3(P.light[0] - mm[0], P.light[1] - mm[1], P.light[2] - mm[2]);
    const float lo = sqrtf(dot3(Vo, Vo)), li = sqrtf(dot3(Vi, Vi));
    const float3 wo = (1.f / lo) * Vo, wi = (1.f / li) * Vi;
    const float3 go = make_float3(dX[3], dX[4], dX[5]);
    const float3 gi = make_float3(dX[6], dX[7], dX[8]);
    const float3 bo = (-1.f / lo) * (go - dot3(wo, go) * wo);
    const float3 bi = (-1.f / li) * (gi - dot3(wi, gi) * wi);
    dx[0] = dX[0] - dX[12] * wi.x + bo.x + bi.x;
    dx[1] = dX[1] - dX[12] * wi.y + bo.y + bi.y;
    dx[2] = dX[2] - dX[12] * wi.z + bo.z + bi.z;
    dx[3] = dX[9]; dx[4] = dX[10]; dx[5] = dX[11];
    dx[6] = dX[13];
}

}  // namespace sssgs
