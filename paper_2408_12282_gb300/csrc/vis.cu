// Ray-traced per-Gaussian visibility and the SH visibility term (Sec. 3.2
// "Incident Light": visibility estimated by tracing rays through the
// Gaussians with a BVH and learnt as a per-Gaussian SH visibility term;
// App. E "Losses": the ray-traced visibility loss, lambda_raytrace = 0.01).
//
// Tracing: the visibility of item m (pair p, Gaussian i) is the transmittance
// of the segment from mu_i to p's light through every other Gaussian j of the
// same scene, prod_j (1 - alpha_j), with alpha_j = min(alpha_max,
// o_j exp(-q/2)) at the Gaussian's peak along the ray (q the minimum over the
// ray of the Mahalanobis distance), counted when that peak lies inside the
// segment and alpha_j >= alpha_min.
//
// BVH: a linear BVH (Karras 2012) over the boxes that bound each Gaussian's
// support {alpha >= alpha_min} = {q <= 2 ln(o / alpha_min)} (half extent along
// axis a: sqrt(2 ln(o / alpha_min) Sigma_aa)); a ray whose peak response
// reaches alpha_min passes through that box, so the box test never drops a
// contributing Gaussian. Build: scene bounds, 30-bit Morton codes of the means,
// the library's radix sort, one thread per internal node for the hierarchy,
// and one thread per leaf walking up with an arrival counter per node to
// fit the boxes (the second child to arrive writes the union). Traversal: one
// thread per item in Morton order of the origins, a depth-first walk with an
// explicit stack, nearer child first (the depth of this hierarchy is at most
// 62: 30 code bits and 32 index bits).
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace sssgs {
size_t radix_sort_u32_workspace(int64_t n);
int radix_sort_u32(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, int64_t n, int bits, void* ws,
                   cudaStream_t st);

namespace {

// Layout of the BVH buffer (floats):
//   nodes [2N-1][8]: (lo.x, lo.y, lo.z, hi.x), (hi.y, hi.z, a, b) with a, b
//     bit-cast int32: internal node k < N-1: children a, b (node indices);
//     leaf N-1+i (i-th Gaussian in Morton order): a = Gaussian index, b = -1;
//   tracing records [N][16] in Morton order: (mu, o), then M = S^-1 R^T
//     row-major (9), then pad: q' = M (x - mu) is x in the Gaussian's frame.
constexpr int NODE_F = 8, TREC_F = 16, STACK = 64;
constexpr float VIS_T_STOP = 1e-5f;

struct BvhWs {
    size_t kA, vA, kB, vB, parent, flags, part, bounds, sort, total;
};
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr int BOUND_BLOCKS = 256;

BvhWs bvh_ws(int64_t n) {
    BvhWs W;
    size_t o = 0;
    W.kA = o; o += al256(4 * (size_t)n);
    W.vA = o; o += al256(4 * (size_t)n);
    W.kB = o; o += al256(4 * (size_t)n);
    W.vB = o; o += al256(4 * (size_t)n);
    W.parent = o; o += al256(4 * (size_t)(2 * n));
    W.flags = o; o += al256(4 * (size_t)n);
    W.part = o; o += al256(4 * 6 * (size_t)BOUND_BLOCKS);
    W.bounds = o; o += al256(4 * 6);
    W.sort = o; o += al256(radix_sort_u32_workspace(n));
    W.total = o;
    return W;
}

__device__ __forceinline__ int f2i(float f) { return __float_as_int(f); }
__device__ __forceinline__ float i2f(int i) { return __int_as_float(i); }

// Rotation of the normalised quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_rot(const float* q4, float* R) {
    const float n = rsqrtf(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
    const float w = q4[0] * n, x = q4[1] * n, y = q4[2] * n, z = q4[3] * n;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Per-block min / max of the means, then one block over the partials.
__global__ void __launch_bounds__(256) k_bounds_part(const float* __restrict__ mu, int64_t n, float* __restrict__ part) {
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = mu[3 * g + c];
            lo[c] = fminf(lo[c], v);
            hi[c] = fmaxf(hi[c], v);
        }
    __shared__ float s[6][8];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(SSSGS_FULL, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(SSSGS_FULL, hi[c], o));
        }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            s[c][w] = lo[c];
            s[3 + c][w] = hi[c];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        float v = s[threadIdx.x][0];
        for (int k = 1; k < 8; ++k) v = threadIdx.x < 3 ? fminf(v, s[threadIdx.x][k]) : fmaxf(v, s[threadIdx.x][k]);
        part[6 * blockIdx.x + threadIdx.x] = v;
    }
}

__global__ void k_bounds_final(const float* __restrict__ part, int nb, float* __restrict__ bounds) {
    if (threadIdx.x < 6) {
        float v = part[threadIdx.x];
        for (int k = 1; k < nb; ++k) {
            const float u = part[6 * k + threadIdx.x];
            v = threadIdx.x < 3 ? fminf(v, u) : fmaxf(v, u);
        }
        bounds[threadIdx.x] = v;
    }
}

// 10-bit integer -> its bits spread to every third position.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void __launch_bounds__(256) k_morton(const float* __restrict__ mu, int64_t n,
                                                const float* __restrict__ bounds, uint32_t* __restrict__ code,
                                                uint32_t* __restrict__ idx) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    uint32_t q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float ext = bounds[3 + c] - bounds[c];
        const float u = ext > 0.f ? (mu[3 * g + c] - bounds[c]) / ext : 0.f;
        q[c] = (uint32_t)fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
    }
    code[g] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    idx[g] = (uint32_t)g;
}

// Common prefix length of sorted keys i and j (ties broken by position).
__device__ __forceinline__ int bvh_delta(const uint32_t* __restrict__ code, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const uint32_t a = code[i], b = code[j];
    return a == b ? 32 + __clz((uint32_t)(i ^ j)) : __clz(a ^ b);
}

// Internal node i (Karras 2012): the range of sorted leaves it covers, its
// split, and its two children.
__global__ void __launch_bounds__(256) k_bvh_internal(const uint32_t* __restrict__ code, int n,
                                                      float* __restrict__ nodes, int* __restrict__ parent) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = bvh_delta(code, n, i, i + 1) - bvh_delta(code, n, i, i - 1) >= 0 ? 1 : -1;
    const int dmin = bvh_delta(code, n, i, i - d);
    int lmax = 2;
    while (bvh_delta(code, n, i, i + lmax * d) > dmin) lmax <<= 1;       // at most 32 doublings
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (bvh_delta(code, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = bvh_delta(code, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (bvh_delta(code, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    const int gamma = i + s * d + min(d, 0);
    const int left = min(i, j) == gamma ? (n - 1) + gamma : gamma;
    const int right = max(i, j) == gamma + 1 ? (n - 1) + gamma + 1 : gamma + 1;
    nodes[NODE_F * i + 6] = i2f(left);
    nodes[NODE_F * i + 7] = i2f(right);
    parent[left] = i;
    parent[right] = i;
}

// Leaves: box and tracing record of the i-th Gaussian in Morton order, then a
// walk towards the root; the second child to reach a node writes its box.
__global__ void __launch_bounds__(256) k_bvh_fit(sssgs_cfg cfg, sssgs_scene sc, const uint32_t* __restrict__ idx,
                                                 int n, float* __restrict__ nodes, float* __restrict__ trec,
                                                 const int* __restrict__ parent, int* __restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int g = (int)idx[i];
    float R[9];
    quat_rot(sc.quat + 4 * g, R);
    const float s[3] = {expf(sc.log_s[3 * g]), expf(sc.log_s[3 * g + 1]), expf(sc.log_s[3 * g + 2])};
    const float o = 1.f / (1.f + expf(-sc.logit_o[g]));
    const float Q = o > cfg.alpha_min ? 2.f * logf(o / cfg.alpha_min) : -1.f;
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float saa = R[3 * a] * R[3 * a] * s[0] * s[0] + R[3 * a + 1] * R[3 * a + 1] * s[1] * s[1] +
                          R[3 * a + 2] * R[3 * a + 2] * s[2] * s[2];
        const float h = Q >= 0.f ? sqrtf(Q * saa) * 1.001f + 1e-6f : -1.f;     // padded for float rounding
        lo[a] = Q >= 0.f ? sc.mu[3 * g + a] - h : 3.0e38f;
        hi[a] = Q >= 0.f ? sc.mu[3 * g + a] + h : -3.0e38f;
    }
    const int leaf = (n - 1) + i;
    float* nd = nodes + (int64_t)NODE_F * leaf;
    nd[0] = lo[0]; nd[1] = lo[1]; nd[2] = lo[2]; nd[3] = hi[0];
    nd[4] = hi[1]; nd[5] = hi[2]; nd[6] = i2f(g); nd[7] = i2f(-1);
    float* tr = trec + (int64_t)TREC_F * i;
    tr[0] = sc.mu[3 * g]; tr[1] = sc.mu[3 * g + 1]; tr[2] = sc.mu[3 * g + 2]; tr[3] = o;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) tr[4 + 3 * r + c] = R[3 * c + r] / s[r];      // (S^-1 R^T)[r][c]
    tr[13] = tr[14] = tr[15] = 0.f;
    __threadfence();
    int node = parent[leaf];
    while (node >= 0) {                                    // at most the tree depth (< 64) steps
        if (atomicAdd(flags + node, 1) == 0) return;       // the sibling finishes this node
        __threadfence();
        const float* p = nodes + (int64_t)NODE_F * node;
        const int a = f2i(__ldcg(p + 6)), b = f2i(__ldcg(p + 7));
        const float* A = nodes + (int64_t)NODE_F * a;
        const float* B = nodes + (int64_t)NODE_F * b;
        float box[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) box[k] = fminf(__ldcg(A + k), __ldcg(B + k));
        box[3] = fmaxf(__ldcg(A + 3), __ldcg(B + 3));
        box[4] = fmaxf(__ldcg(A + 4), __ldcg(B + 4));
        box[5] = fmaxf(__ldcg(A + 5), __ldcg(B + 5));
        float* q = nodes + (int64_t)NODE_F * node;
#pragma unroll
        for (int k = 0; k < 6; ++k) q[k] = box[k];
        __threadfence();
        node = parent[node];
    }
}

__global__ void k_bvh_init(int* __restrict__ parent, int* __restrict__ flags, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * n - 1) parent[i] = -1;
    if (i < n) flags[i] = 0;
}

// One ray per item: transmittance of the segment mu_i -> light. Thread t
// takes pair t / N and the Gaussian at Morton position t % N (the BVH's leaf
// order), so a warp traces from neighbouring origins toward one light and
// walks the hierarchy coherently; threads whose Gaussian belongs to another
// scene than the pair's return at once. At an internal node both children's
// boxes are tested and the nearer hit is visited first (the farther one is
// pushed), so dense occluders near the origin end the ray early.
__global__ void __launch_bounds__(128) k_trace(sssgs_cfg cfg, const sssgs_pair* __restrict__ pairs, int n_pairs,
                                               const float* __restrict__ mu, const float4* __restrict__ nodes,
                                               const float4* __restrict__ trec, int n, float* __restrict__ vis) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_pairs * n) return;
    const int p = (int)(t / n), k = (int)(t - (int64_t)p * n);
    const sssgs_pair& P = pairs[p];
    const int gi = f2i(nodes[2 * ((n - 1) + k) + 1].z);
    const int g0 = P.g_begin, g1 = P.g_begin + P.g_count;
    if (gi < g0 || gi >= g1) return;
    const int64_t m = P.item_offset + (gi - g0);
    const float ox = mu[3 * gi], oy = mu[3 * gi + 1], oz = mu[3 * gi + 2];
    float dx = P.light[0] - ox, dy = P.light[1] - oy, dz = P.light[2] - oz;
    const float tL = sqrtf(dx * dx + dy * dy + dz * dz);
    const float il = 1.f / tL;
    dx *= il; dy *= il; dz *= il;
    auto inv = [](float v) { return fabsf(v) > 1e-20f ? 1.f / v : copysignf(1e20f, v); };
    const float ix = inv(dx), iy = inv(dy), iz = inv(dz);
    // entry distance of the segment into node nd's box, or -1 when it misses
    auto enter = [&](int nd) -> float {
        const float4 A = nodes[2 * nd], B = nodes[2 * nd + 1];     // lo = (A.x, A.y, A.z), hi = (A.w, B.x, B.y)
        float t0 = 0.f, t1 = tL;
        float u0 = (A.x - ox) * ix, u1 = (A.w - ox) * ix;
        t0 = fmaxf(t0, fminf(u0, u1)); t1 = fminf(t1, fmaxf(u0, u1));
        u0 = (A.y - oy) * iy; u1 = (B.x - oy) * iy;
        t0 = fmaxf(t0, fminf(u0, u1)); t1 = fminf(t1, fmaxf(u0, u1));
        u0 = (A.z - oz) * iz; u1 = (B.y - oz) * iz;
        t0 = fmaxf(t0, fminf(u0, u1)); t1 = fminf(t1, fmaxf(u0, u1));
        return t0 <= t1 ? t0 : -1.f;
    };
    const float a_min = cfg.alpha_min, a_max = cfg.alpha_max;
    float T = 1.f;
    int stack[STACK];
    int sp = 0, node = 0;
    if (enter(0) < 0.f) node = -1;
    while (node >= 0) {
        if (node >= n - 1) {                                   // leaf (its box was hit)
            const int j = f2i(nodes[2 * node + 1].z);
            if (j != gi && j >= g0 && j < g1) {
                const int li = node - (n - 1);
                const float4 r0 = trec[4 * li], r1 = trec[4 * li + 1], r2 = trec[4 * li + 2], r3 = trec[4 * li + 3];
                const float ex = ox - r0.x, ey = oy - r0.y, ez = oz - r0.z;
                const float px = r1.x * ex + r1.y * ey + r1.z * ez;
                const float py = r1.w * ex + r2.x * ey + r2.y * ez;
                const float pz = r2.z * ex + r2.w * ey + r3.x * ez;
                const float qx = r1.x * dx + r1.y * dy + r1.z * dz;
                const float qy = r1.w * dx + r2.x * dy + r2.y * dz;
                const float qz = r2.z * dx + r2.w * dy + r3.x * dz;
                const float dd = qx * qx + qy * qy + qz * qz;
                const float tt = -(px * qx + py * qy + pz * qz) / dd;
                const float cx = px + tt * qx, cy = py + tt * qy, cz = pz + tt * qz;
                const float alpha = fminf(a_max, r0.w * expf(-0.5f * (cx * cx + cy * cy + cz * cz)));
                if (tt > 0.f && tt < tL && alpha >= a_min) {
                    T *= 1.f - alpha;
                    if (T < VIS_T_STOP) break;
                }
            }
            node = sp > 0 ? stack[--sp] : -1;
            continue;
        }
        const float4 B = nodes[2 * node + 1];
        const int ca = f2i(B.z), cb = f2i(B.w);
        const float ta = enter(ca), tb = enter(cb);
        if (ta >= 0.f && tb >= 0.f) {
            const bool a_first = ta <= tb;
            if (sp < STACK) stack[sp++] = a_first ? cb : ca;
            node = a_first ? ca : cb;
        } else if (ta >= 0.f) {
            node = ca;
        } else if (tb >= 0.f) {
            node = cb;
        } else {
            node = sp > 0 ? stack[--sp] : -1;
        }
    }
    vis[m] = T;
}

// ---------------------------------------------------------------- SH visibility

constexpr float SH_C0 = 0.28209479177387814f;   // 1 / (2 sqrt(pi))
constexpr float SH_C1 = 0.4886025119029199f;    // sqrt(3 / (4 pi))
constexpr float SH_C2a = 1.0925484305920792f;   // sqrt(15 / pi) / 2
constexpr float SH_C2b = 0.31539156525252005f;  // sqrt(5 / pi) / 4
constexpr float SH_C2c = 0.5462742152960396f;   // sqrt(15 / pi) / 4
constexpr float SH_C3a = 0.5900435899266435f;   // sqrt(35 / (2 pi)) / 4
constexpr float SH_C3b = 2.890611442640554f;    // sqrt(105 / pi) / 2
constexpr float SH_C3c = 0.4570457994644658f;   // sqrt(21 / (2 pi)) / 4
constexpr float SH_C3d = 0.3731763325901154f;   // sqrt(7 / pi) / 4
constexpr float SH_C3e = 1.445305721320277f;    // sqrt(105 / pi) / 4

// Real SH of degree <= 3 at the unit vector (x, y, z), index l^2 + l + m.
__device__ __forceinline__ void sh16(float x, float y, float z, float* Y) {
    Y[0] = SH_C0;
    Y[1] = SH_C1 * y; Y[2] = SH_C1 * z; Y[3] = SH_C1 * x;
    Y[4] = SH_C2a * x * y; Y[5] = SH_C2a * y * z; Y[6] = SH_C2b * (3.f * z * z - 1.f);
    Y[7] = SH_C2a * x * z; Y[8] = SH_C2c * (x * x - y * y);
    Y[9] = SH_C3a * y * (3.f * x * x - y * y); Y[10] = SH_C3b * x * y * z;
    Y[11] = SH_C3c * y * (5.f * z * z - 1.f); Y[12] = SH_C3d * z * (5.f * z * z - 3.f);
    Y[13] = SH_C3c * x * (5.f * z * z - 1.f); Y[14] = SH_C3e * z * (x * x - y * y);
    Y[15] = SH_C3a * x * (x * x - 3.f * y * y);
}

// Gradient of u = sum_k c_k Y_k with respect to (x, y, z) (the polynomials).
__device__ __forceinline__ float3 sh16_grad(const float* c, float x, float y, float z) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    gy += c[1] * SH_C1; gz += c[2] * SH_C1; gx += c[3] * SH_C1;
    gx += c[4] * SH_C2a * y; gy += c[4] * SH_C2a * x;
    gy += c[5] * SH_C2a * z; gz += c[5] * SH_C2a * y;
    gz += c[6] * SH_C2b * 6.f * z;
    gx += c[7] * SH_C2a * z; gz += c[7] * SH_C2a * x;
    gx += c[8] * SH_C2c * 2.f * x; gy -= c[8] * SH_C2c * 2.f * y;
    gx += c[9] * SH_C3a * 6.f * x * y; gy += c[9] * SH_C3a * 3.f * (x * x - y * y);
    gx += c[10] * SH_C3b * y * z; gy += c[10] * SH_C3b * x * z; gz += c[10] * SH_C3b * x * y;
    gy += c[11] * SH_C3c * (5.f * z * z - 1.f); gz += c[11] * SH_C3c * 10.f * y * z;
    gz += c[12] * SH_C3d * (15.f * z * z - 3.f);
    gx += c[13] * SH_C3c * (5.f * z * z - 1.f); gz += c[13] * SH_C3c * 10.f * x * z;
    gx += c[14] * SH_C3e * 2.f * x * z; gy -= c[14] * SH_C3e * 2.f * y * z; gz += c[14] * SH_C3e * (x * x - y * y);
    gx += c[15] * SH_C3a * 3.f * (x * x - y * y); gy -= c[15] * SH_C3a * 6.f * x * y;
    return make_float3(gx, gy, gz);
}

__global__ void __launch_bounds__(256) k_vis_sh_fwd(const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                    int64_t n_items, const float* __restrict__ mu,
                                                    const float* __restrict__ sh, float* __restrict__ vis_item) {
    const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_items) return;
    const int p = pair_of_item(pairs, n_pairs, m);
    const sssgs_pair& P = pairs[p];
    const int64_t g = P.g_begin + (m - P.item_offset);
    float vx = P.light[0] - mu[3 * g], vy = P.light[1] - mu[3 * g + 1], vz = P.light[2] - mu[3 * g + 2];
    const float ir = rsqrtf(vx * vx + vy * vy + vz * vz);
    float Y[16];
    sh16(vx * ir, vy * ir, vz * ir, Y);
    float u = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) u = fmaf(sh[16 * g + k], Y[k], u);
    vis_item[m] = fminf(fmaxf(u, 0.f), 1.f);
}

// One thread per Gaussian; sums over the pairs that hold it (no atomics).
__global__ void __launch_bounds__(128) k_vis_sh_bwd(const sssgs_pair* __restrict__ pairs, int n_pairs, int64_t n,
                                                    const float* __restrict__ mu, const float* __restrict__ sh,
                                                    const float* __restrict__ dvis_item, float* __restrict__ dsh,
                                                    float* __restrict__ dmu) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    float c[16], dc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        c[k] = sh[16 * g + k];
        dc[k] = 0.f;
    }
    float dm[3] = {0.f, 0.f, 0.f};
    bool any = false;
    for (int p = 0; p < n_pairs; ++p) {
        const sssgs_pair& P = pairs[p];
        if (g < P.g_begin || g >= (int64_t)P.g_begin + P.g_count) continue;
        const float dv = dvis_item[P.item_offset + (g - P.g_begin)];
        if (dv == 0.f) continue;
        const float vx = P.light[0] - mu[3 * g], vy = P.light[1] - mu[3 * g + 1], vz = P.light[2] - mu[3 * g + 2];
        const float r = sqrtf(vx * vx + vy * vy + vz * vz), ir = 1.f / r;
        const float x = vx * ir, y = vy * ir, z = vz * ir;
        float Y[16];
        sh16(x, y, z, Y);
        float u = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) u = fmaf(c[k], Y[k], u);
        if (!(u > 0.f && u < 1.f)) continue;                // clamped: no gradient
        any = true;
#pragma unroll
        for (int k = 0; k < 16; ++k) dc[k] = fmaf(dv, Y[k], dc[k]);
        const float3 gu = sh16_grad(c, x, y, z);
        const float wx = dv * gu.x, wy = dv * gu.y, wz = dv * gu.z;    // dL/dw
        const float wd = x * wx + y * wy + z * wz;
        // w = V / |V|, V = light - mu: dL/dmu = -(dL/dw - (w . dL/dw) w) / |V|
        dm[0] -= (wx - wd * x) * ir;
        dm[1] -= (wy - wd * y) * ir;
        dm[2] -= (wz - wd * z) * ir;
    }
    if (!any) return;
    if (dsh)
#pragma unroll
        for (int k = 0; k < 16; ++k) dsh[16 * g + k] += dc[k];
    if (dmu)
#pragma unroll
        for (int k = 0; k < 3; ++k) dmu[3 * g + k] += dm[k];
}

// Ray-traced visibility loss: lambda * |v - v_traced| / n_p per item.
__global__ void __launch_bounds__(256) k_vis_loss(const sssgs_pair* __restrict__ pairs, int n_pairs, int64_t n_items,
                                                  const float* __restrict__ v, const float* __restrict__ vt,
                                                  float lambda, float* __restrict__ dv, float* __restrict__ d_loss) {
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
        const float d = v[m] - vt[m];
        dv[m] += d > 0.f ? lambda * inv : (d < 0.f ? -lambda * inv : 0.f);
        const float l = lambda * fabsf(d) * inv;
        if (p == s_p0) atomicAdd(&s_sum[0], l);
        else if (p == s_p0 + 1) atomicAdd(&s_sum[1], l);
        else atomicAdd(d_loss + p, l);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(d_loss + s_p0, s_sum[0]);
        if (s_p0 + 1 < n_pairs) atomicAdd(d_loss + s_p0 + 1, s_sum[1]);
    }
}

int64_t items_of(const sssgs_pair* h, int n) { return h[n - 1].item_offset + h[n - 1].g_count; }

}  // namespace
}  // namespace sssgs

using namespace sssgs;

extern "C" int64_t sssgs_bvh_floats(int64_t n) {
    return n <= 0 ? 0 : (int64_t)NODE_F * (2 * n - 1) + (int64_t)TREC_F * n;
}

extern "C" size_t sssgs_bvh_workspace_bytes(int64_t n) { return n <= 0 ? 256 : bvh_ws(n).total; }

extern "C" int sssgs_bvh_build(const sssgs_cfg* cfg, const sssgs_scene* scene, float* bvh, void* workspace,
                               size_t workspace_bytes, sssgs_stream stream) {
    if (!cfg || !scene || !bvh || !scene->mu || !scene->log_s || !scene->quat || !scene->logit_o)
        return SSSGS_ERR_INVALID_ARG;
    const int64_t n = scene->n;
    if (n <= 0) return SSSGS_OK;
    if (n >= ((int64_t)1 << 30)) return SSSGS_ERR_TOO_LARGE;
    if (((uintptr_t)bvh & 15) || ((uintptr_t)workspace & 255)) return SSSGS_ERR_INVALID_ARG;
    const BvhWs W = bvh_ws(n);
    if (!workspace || workspace_bytes < W.total) return SSSGS_ERR_WORKSPACE;
    uint8_t* w = (uint8_t*)workspace;
    uint32_t *kA = (uint32_t*)(w + W.kA), *vA = (uint32_t*)(w + W.vA);
    uint32_t *kB = (uint32_t*)(w + W.kB), *vB = (uint32_t*)(w + W.vB);
    int* parent = (int*)(w + W.parent);
    int* flags = (int*)(w + W.flags);
    float* part = (float*)(w + W.part);
    float* bounds = (float*)(w + W.bounds);
    cudaStream_t st = (cudaStream_t)stream;
    const int nn = (int)n;
    const unsigned nb = (unsigned)((n + 255) / 256), nb2 = (unsigned)((2 * n + 255) / 256);
    const int bb = (int)std::min<int64_t>(BOUND_BLOCKS, (n + 255) / 256);
    k_bounds_part<<<bb, 256, 0, st>>>(scene->mu, n, part);
    k_bounds_final<<<1, 32, 0, st>>>(part, bb, bounds);
    k_morton<<<nb, 256, 0, st>>>(scene->mu, n, bounds, kA, vA);
    sssgs::note_launches(3);
    const int which = radix_sort_u32(kA, vA, kB, vB, n, 30, w + W.sort, st);
    const uint32_t* codes = which ? kB : kA;
    const uint32_t* idx = which ? vB : vA;
    float* nodes = bvh;
    float* trec = bvh + (int64_t)NODE_F * (2 * n - 1);
    k_bvh_init<<<nb2, 256, 0, st>>>(parent, flags, nn);
    if (nn > 1) k_bvh_internal<<<(unsigned)((n - 1 + 255) / 256), 256, 0, st>>>(codes, nn, nodes, parent);
    k_bvh_fit<<<nb, 256, 0, st>>>(*cfg, *scene, idx, nn, nodes, trec, parent, flags);
    sssgs::note_launches(nn > 1 ? 3 : 2);
    return launch_status();
}

extern "C" int sssgs_trace_visibility(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                      int n_pairs, const sssgs_scene* scene, const float* bvh, float* vis_traced,
                                      sssgs_stream stream) {
    if (!cfg || !h_pairs || !d_pairs || n_pairs <= 0 || !scene || !scene->mu || !bvh || !vis_traced)
        return SSSGS_ERR_INVALID_ARG;
    if ((uintptr_t)bvh & 15) return SSSGS_ERR_INVALID_ARG;
    const int64_t n_items = items_of(h_pairs, n_pairs), n = scene->n;
    if (n_items == 0 || n <= 0) return SSSGS_OK;
    const float* nodes = bvh;
    const float* trec = bvh + (int64_t)NODE_F * (2 * n - 1);
    const int64_t threads = (int64_t)n_pairs * n;
    k_trace<<<(unsigned)((threads + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        *cfg, d_pairs, n_pairs, scene->mu, reinterpret_cast<const float4*>(nodes),
        reinterpret_cast<const float4*>(trec), (int)n, vis_traced);
    sssgs::note_launches(1);
    return launch_status();
}

extern "C" int sssgs_vis_sh_fwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                                const sssgs_scene* scene, const float* vis_sh, float* vis_item, sssgs_stream stream) {
    if (!h_pairs || !d_pairs || n_pairs <= 0 || !scene || !scene->mu || !vis_sh || !vis_item)
        return SSSGS_ERR_INVALID_ARG;
    const int64_t n_items = items_of(h_pairs, n_pairs);
    if (n_items == 0) return SSSGS_OK;
    k_vis_sh_fwd<<<(unsigned)((n_items + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_pairs, n_pairs, n_items,
                                                                                     scene->mu, vis_sh, vis_item);
    sssgs::note_launches(1);
    return launch_status();
}

extern "C" int sssgs_vis_sh_bwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                                const sssgs_scene* scene, const float* vis_sh, const float* dvis_item,
                                float* dvis_sh, float* dmu, sssgs_stream stream) {
    if (!h_pairs || !d_pairs || n_pairs <= 0 || !scene || !scene->mu || !vis_sh || !dvis_item)
        return SSSGS_ERR_INVALID_ARG;
    const int64_t n = scene->n;
    if (n <= 0) return SSSGS_OK;
    k_vis_sh_bwd<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(d_pairs, n_pairs, n, scene->mu,
                                                                               vis_sh, dvis_item, dvis_sh, dmu);
    sssgs::note_launches(1);
    return launch_status();
}

extern "C" int sssgs_vis_loss(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                              const float* vis_item, const float* vis_traced, float lambda_raytrace,
                              float* dvis_item, float* d_loss, sssgs_stream stream) {
    if (!h_pairs || !d_pairs || n_pairs <= 0 || !vis_item || !vis_traced || !dvis_item || !d_loss)
        return SSSGS_ERR_INVALID_ARG;
    const int64_t n_items = items_of(h_pairs, n_pairs);
    if (n_items == 0) return SSSGS_OK;
    k_vis_loss<<<(unsigned)((n_items + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        d_pairs, n_pairs, n_items, vis_item, vis_traced, lambda_raytrace, dvis_item, d_loss);
    sssgs::note_launches(1);
    return launch_status();
}
