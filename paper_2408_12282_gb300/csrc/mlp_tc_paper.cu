// The paper's network (Appendix E "Network", SSSGS_MLP_PAPER) on the 5th-
// generation tensor cores: BF16 operands in shared memory, FP32 accumulators
// in TMEM, one fused kernel for the forward and one for the backward (which
// recomputes the forward of its rows first).
//
// Device chain (rows = 128 items per tile, MMA M = 128):
//   L0  X  [48]  -> 64   Leaky-ReLU        (W0)
//   L1  H1 [64]  -> 32   Leaky-ReLU        (W1)
//   L2  H2 [32]  -> 32   Leaky-ReLU = T    (W2, trunk output)
//   L3  T  [32]  -> 48   columns 0..31: incident hidden G (W3, Leaky-ReLU);
//                        columns 32..34: SSS logits (W5) -> sigmoid -> L_SSS
//   L4  G  [32]  -> 16   column 0: incident output (W4) -> ReLU -> L_in
// Numerics as for the other BF16 network: inputs, weights and hidden
// activations rounded to bfloat16, FP32 accumulation; biases and heads FP32;
// in the backward every pre-activation gradient dZ is rounded to bfloat16
// once and used for dW = dZ^T H, db = sum dZ and dH = dZ W.
//
// A CTA runs two independent tile lanes (one warpgroup each, its own
// activation tiles, TMEM working columns and mbarrier), so one lane's
// epilogue overlaps the other's MMAs. All weights stay resident (16 KB). The
// backward accumulates dW and db of every layer across all tiles of the CTA
// in TMEM (lane = output unit; dW_l = dZ^T H_l with M = 128 output units, of
// which the first out_l are real: the operand rows past them read other data
// of the dZ tile and land in TMEM lanes that are never read), zeroed once and
// added to the caller's gradients at the end.
#include <algorithm>

#include "mlp_tc_util.cuh"

namespace sssgs {
namespace {

constexpr int PR = 128;          // rows per tile
constexpr int PLANES = 2;        // tile lanes per CTA
constexpr int PT = 128;          // threads per lane
constexpr int NCH = 5;           // chain layers
__host__ __device__ constexpr int kin(int l) { return l == 0 ? 48 : (l == 1 ? 64 : 32); }
__host__ __device__ constexpr int nout(int l) { return l == 0 ? 64 : (l == 3 ? 48 : (l == 4 ? 16 : 32)); }

// TMEM columns. Backward: dW / db accumulators, then 64 working columns per
// lane. Forward: only the working columns.
__host__ __device__ constexpr uint32_t acc_w(int l) {            // widths kin(l): 48, 64, 32, 32, 32
    return l == 0 ? 0u : (l == 1 ? 48u : (l == 2 ? 112u : (l == 3 ? 144u : 176u)));
}
__host__ __device__ constexpr uint32_t acc_b(int l) { return 208u + 16u * (uint32_t)l; }   // 16 columns each
constexpr uint32_t ACC_END = 288;
__host__ __device__ constexpr uint32_t work_col(bool bwd, int g) { return (bwd ? ACC_END : 0u) + 64u * g; }
__host__ __device__ constexpr uint32_t tmem_cols(bool bwd) { return bwd ? 512u : 128u; }

// Shared memory (bytes). Weight images: [nout(l) x kin(l)] BF16 blocked with
// C = kin(l). Per lane: X (C 48), H1 (C 64), H2, T, G (C 32), DZ (C 64, plus
// 1 KB that the M = 128 dW operands may read past its end).
struct PSmem {
    static constexpr uint32_t W(int l) {
        uint32_t o = 0;
        for (int q = 0; q < l; ++q) o += (uint32_t)(nout(q) * kin(q) * 2);
        return o;
    }
    static constexpr uint32_t ONES = 16384;                     // 16 x 128 BF16 ones, K-major
    static constexpr uint32_t BIAS = ONES + 16 * PR * 2;         // b0 64, b1 32, b2 32, bc 48, b4 16 floats
    static constexpr uint32_t BIAS_OFF(int l) { return l == 0 ? 0 : (l == 1 ? 64 : (l == 2 ? 96 : (l == 3 ? 128 : 176))); }
    static constexpr uint32_t BAR = BIAS + 192 * 4;              // mbarriers, TMEM address, fail flags
    static constexpr uint32_t PAIRS = BAR + 64;                  // item offsets of up to 256 pairs
    static constexpr uint32_t LANE0 = (PAIRS + 8 * TC_MAX_SMEM_PAIRS + 1023) & ~1023u;
    static constexpr uint32_t X = 0, H1 = X + PR * 48 * 2, H2 = H1 + PR * 64 * 2, T = H2 + PR * 32 * 2,
                              G = T + PR * 32 * 2, DZ = G + PR * 32 * 2;
    static constexpr uint32_t LANE_BYTES = DZ + PR * 64 * 2 + 1024;
    static constexpr uint32_t TOTAL = LANE0 + PLANES * LANE_BYTES;
};
static_assert(PSmem::W(NCH) <= PSmem::ONES, "weight images overlap");

// Offset of chain layer l's input tile within a lane. Computed, not looked
// up: a runtime index into a local array of tile pointers is served from local
// memory, and with this kernel's shared-memory carve-out such loads miss L1.
__host__ __device__ constexpr uint32_t act_off(int l) {
    return l == 0 ? PSmem::X : (l == 1 ? PSmem::H1 : (l == 2 ? PSmem::H2 : (l == 3 ? PSmem::T : PSmem::G)));
}
static_assert(PSmem::TOTAL <= 227 * 1024, "shared memory budget");

// Weight (n, k) of chain layer l and bias n, from the caller's six matrices.
__device__ __forceinline__ float pw(const MlpDev& net, int l, int n, int k) {
    if (l < 3) return net.W[l][n * kin(l) + k];
    if (l == 3) return n < 32 ? net.W[3][n * 32 + k] : (n < 35 ? net.W[5][(n - 32) * 32 + k] : 0.f);
    return n == 0 ? net.W[4][k] : 0.f;
}
__device__ __forceinline__ float pb(const MlpDev& net, int l, int n) {
    if (l < 3) return net.b[l][n];
    if (l == 3) return n < 32 ? net.b[3][n] : (n < 35 ? net.b[5][n - 32] : 0.f);
    return n == 0 ? net.b[4][0] : 0.f;
}


// Forward (BWD = false: rows are the items, writes out) or backward (BWD =
// true: rows are the active items, recompute + back-propagate, gradients).
template <bool BWD>
__global__ void __launch_bounds__(PLANES * PT, 1) k_mlp_paper_tc(MlpDev net, const sssgs_pair* __restrict__ pairs,
                                                                 int n_pairs, int64_t n_items, sssgs_scene sc,
                                                                 float* __restrict__ out,
                                                                 const float* __restrict__ dout, int64_t dstride,
                                                                 sssgs_mlp_grad gr, float* __restrict__ dx_items,
                                                                 const uint32_t* __restrict__ active,
                                                                 const uint32_t* __restrict__ n_active,
                                                                 int32_t* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int tid = threadIdx.x, wg = tid >> 7, t = tid & 127, warp = (tid >> 5) & 3;
    float* sbias = reinterpret_cast<float*>(smem + PSmem::BIAS);
    const uint32_t bar = tc::smem_u32(smem + PSmem::BAR) + 8 * wg;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + PSmem::BAR + 32);
    volatile int* s_fail = reinterpret_cast<volatile int*>(smem + PSmem::BAR + 40);
    int64_t* s_off = reinterpret_cast<int64_t*>(smem + PSmem::PAIRS);
    uint8_t* lane = smem + PSmem::LANE0 + wg * PSmem::LANE_BYTES;
    uint8_t* sDZ = lane + PSmem::DZ;

    if (tid < 32) {
        tc::tmem_alloc(tc::smem_u32(s_tmem), tmem_cols(BWD));
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int g = 0; g < PLANES; ++g) {
            tc::mbar_init(tc::smem_u32(smem + PSmem::BAR) + 8 * g, 1);
            s_fail[g] = 0;
        }
        tc::fence_mbar_init();
    }
    for (int p = tid; p < n_pairs && p < TC_MAX_SMEM_PAIRS; p += blockDim.x) s_off[p] = pairs[p].item_offset;
    for (int l = 0; l < NCH; ++l) {
        const int N = nout(l), K = kin(l);
        uint8_t* wb = smem + PSmem::W(l);
        for (int i = tid; i < N * K; i += blockDim.x) {
            const int n = i / K, k = i - n * K;
            *reinterpret_cast<__nv_bfloat16*>(wb + tc::blk_offset(n, k, K)) = __float2bfloat16_rn(pw(net, l, n, k));
        }
        for (int n = tid; n < N; n += blockDim.x) sbias[PSmem::BIAS_OFF(l) + n] = pb(net, l, n);
    }
    for (int i = tid; i < 16 * PR / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(smem + PSmem::ONES)[i] = 0x3F803F80u;   // two bf16 1.0
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    if (BWD && wg == 0) tmem_zero(tmem + lane_off, (int)ACC_END);   // dW / db accumulators
    tc::fence_before();
    __syncthreads();
    tc::fence_after();

    const uint32_t work = tmem + work_col(BWD, wg);
    const uint32_t work_l = work + lane_off;
    const int64_t n_rows = BWD ? (int64_t)*n_active : n_items;
    const int64_t n_tiles = (n_rows + PR - 1) / PR;
    uint32_t phase = 0;
    bool ok = true;
    auto round_wait = [&]() {
        const bool got = tc::mbar_wait(bar, phase);
        phase ^= 1u;
        tc::fence_after();
        if (!got) s_fail[wg] = 1;
    };
    auto round_end = [&]() -> bool {
        tc::fence_before();
        tc::fence_async_smem();
        named_sync(1 + wg, PT);
        return s_fail[wg] == 0;
    };
    // Issued from the lane group's first warp (t < 32), lane 0 executing:
    // D(work) = A(kin(l)) W_l^T
    auto mma_fwd = [&](int l) {
        const int K = kin(l);
        const uint32_t idesc = tc::idesc_bf16(PR, nout(l), false, false);
        const tc::Desc2 a = tc::desc2(tc::smem_u32(lane + act_off(l)), 128, (uint32_t)(K / 8) * 128u);
        const tc::Desc2 w = tc::desc2(tc::smem_u32(smem + PSmem::W(l)), 128, (uint32_t)(K / 8) * 128u);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < K / 16) tc::mma_bf16_w(work, a, k * 256, w, k * 256, idesc, k > 0 ? 1u : 0u, t);
    };
    // dW_l += dZ^T H_l, db_l += dZ^T 1, D(work) = dZ W_l (dZ in sDZ, C = 64)
    auto mma_bwd = [&](int l) {
        const int K = kin(l), No = nout(l);
        const uint32_t dz = tc::smem_u32(sDZ), h = tc::smem_u32(lane + act_off(l));
        const uint32_t ones = tc::smem_u32(smem + PSmem::ONES), w = tc::smem_u32(smem + PSmem::W(l));
        const uint32_t hsr = (uint32_t)(K / 8) * 128u;
        const uint32_t idw = tc::idesc_bf16(PR, K, true, true), idb = tc::idesc_bf16(PR, 16, true, false);
        const tc::Desc2 dzm = tc::desc2(dz, 8 * 128, 128), hm = tc::desc2(h, hsr, 128);
        const tc::Desc2 on = tc::desc2(ones, 128, (PR / 8) * 128);
#pragma unroll
        for (int k = 0; k < PR / 16; ++k) {
            tc::mma_bf16_w(tmem + acc_w(l), dzm, k * 2048, hm, k * 2 * hsr, idw, 1u, t);
            tc::mma_bf16_w(tmem + acc_b(l), dzm, k * 2048, on, k * 256, idb, 1u, t);
        }
        const uint32_t idh = tc::idesc_bf16(PR, K, false, true);
        const tc::Desc2 dzk = tc::desc2(dz, 128, 8 * 128), wm = tc::desc2(w, hsr, 128);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (k < No / 16) tc::mma_bf16_w(work, dzk, k * 256, wm, k * 2 * hsr, idh, k > 0 ? 1u : 0u, t);
    };

    for (int64_t tile = PLANES * (int64_t)blockIdx.x + wg; tile < n_tiles && ok;
         tile += PLANES * (int64_t)gridDim.x) {
        // ---- this thread's row: item, pair, network input
        const int64_t row = tile * PR + t;
        const bool valid = row < n_rows;
        int64_t m = 0;
        int pidx = 0;
        if (valid) {
            m = BWD ? (int64_t)active[row] : row;
            pidx = pair_lookup(s_off, pairs, n_pairs, m);
        }
        {
            float x[48];
#pragma unroll
            for (int k = 0; k < 48; ++k) x[k] = 0.f;
            if (valid)
                build_input(net, pairs[pidx], sc, pairs[pidx].g_begin + (m - pairs[pidx].item_offset), m, x, false);
#pragma unroll
            for (int c = 0; c < 48; c += 8) store8_bf16((lane + act_off(0)), t, c, 48, x + c);
        }
        ok = round_end();
        // ---- forward
        float ls[3] = {0.f, 0.f, 0.f}, zi = 0.f;
        for (int l = 0; l < NCH && ok; ++l) {
            if (t < 32) {
                tc::fence_after();
                mma_fwd(l);
                tc::mma_commit_w(bar, t);
            }
            round_wait();
            if (s_fail[wg] == 0) {
                const float* bl = sbias + PSmem::BIAS_OFF(l);
                if (l == 0) {
                    float v[64];
                    tc::tmem_ld64(work_l, v);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        store8_bias_lrelu(lane + act_off(1), t, 8 * q, 64, v + 8 * q, bl + 8 * q, kLReluSlope);
                } else if (l < 4) {
                    float v[32];
                    tc::tmem_ld32(work_l, v);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        store8_bias_lrelu(lane + act_off(l + 1), t, 8 * q, 32, v + 8 * q, bl + 8 * q, kLReluSlope);
                    if (l == 3) {   // SSS head: logits in columns 32..34
                        float h[16];
                        tc::tmem_ld16(work_l + 32, h);
#pragma unroll
                        for (int c = 0; c < 3; ++c) ls[c] = 1.f / (1.f + expf(-(h[c] + bl[32 + c])));
                    }
                } else {            // incident output: column 0
                    float h[16];
                    tc::tmem_ld16(work_l, h);
                    zi = h[0] + bl[0];
                    if (!BWD && valid)
                        reinterpret_cast<float4*>(out)[m] = make_float4(ls[0], ls[1], ls[2], fmaxf(zi, 0.f));
                    if (BWD) {      // head gradients: dZ of the incident output (column 0 of 16)
                        float dz[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        if (valid) {
                            const float* up = dout + dstride * m;
                            dz[0] = zi > 0.f ? up[3] : 0.f;
#pragma unroll
                            for (int c = 0; c < 3; ++c) ls[c] = up[c] * ls[c] * (1.f - ls[c]);   // now dL/d(logit)
                        } else {
                            ls[0] = ls[1] = ls[2] = 0.f;
                        }
                        const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        store8_bf16(sDZ, t, 0, 64, dz);
                        store8_bf16(sDZ, t, 8, 64, zero8);
                    }
                }
            }
            ok = round_end();
        }
        // ---- backward, chain layer 4 down to 0
        for (int l = NCH - 1; BWD && l >= 0 && ok; --l) {
            if (t < 32) {
                tc::fence_after();
                mma_bwd(l);
                tc::mma_commit_w(bar, t);
            }
            round_wait();
            if (s_fail[wg] == 0) {
                const int K = kin(l);   // width of dH_l
                if (l > 0) {
                    // dZ_l = bf16(dH_l * act'(H_l)), H_l = (lane + act_off(l)) (Leaky-ReLU output)
                    float v[64];
                    if (K == 64) tc::tmem_ld64(work_l, v); else tc::tmem_ld32(work_l, v);
#pragma unroll
                    for (int c0 = 0; c0 < 64; c0 += 8) {
                        if (c0 >= K) break;
                        const uint4 hq = load8_packed((lane + act_off(l)), t, c0, K);
                        uint4 o;
                        o.x = tc::pack_bf16_leaky(v[c0 + 0], v[c0 + 1], hq.x, kLReluSlope);
                        o.y = tc::pack_bf16_leaky(v[c0 + 2], v[c0 + 3], hq.y, kLReluSlope);
                        o.z = tc::pack_bf16_leaky(v[c0 + 4], v[c0 + 5], hq.z, kLReluSlope);
                        o.w = tc::pack_bf16_leaky(v[c0 + 6], v[c0 + 7], hq.w, kLReluSlope);
                        store8_packed(sDZ, t, c0, 64, o);
                    }
                    if (l == 4) {   // the layer-3 output also carries the SSS logits' dZ
                        const float d8[8] = {ls[0], ls[1], ls[2], 0.f, 0.f, 0.f, 0.f, 0.f};
                        const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                        store8_bf16(sDZ, t, 32, 64, d8);
                        store8_bf16(sDZ, t, 40, 64, zero8);
                    }
                } else {            // dX -> (d mu, d n, d v, d quat, d log_s)
                    float dX[48];
                    tc::tmem_ld32(work_l, dX);
                    tc::tmem_ld16(work_l + 32, dX + 32);
                    if (valid) {
                        float dx[SSSGS_DX];
                        const sssgs_pair& P = pairs[pidx];
                        input_backward_k<SSSGS_MLP_PAPER>(P, sc, P.g_begin + (m - P.item_offset), dX, dx);
#pragma unroll
                        for (int k = 0; k < SSSGS_DX; ++k) dx_items[(int64_t)SSSGS_DX * m + k] = dx[k];
                    }
                }
            }
            ok = round_end();
        }
    }
    if (!ok && t == 0 && status) atomicOr(status, SSSGS_STATUS_TIMEOUT);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (BWD && wg == 0 && s_fail[0] == 0 && s_fail[PLANES - 1] == 0) {
        // flush: lane = output unit of the chain layer
        float v[64];
        tc::tmem_ld32(tmem + lane_off + acc_w(0), v);
        tc::tmem_ld16(tmem + lane_off + acc_w(0) + 32, v + 32);
        if (t < 64)
            for (int c = 0; c < 48; ++c) atomicAdd(&gr.W[0][t * 48 + c], v[c]);
        tc::tmem_ld64(tmem + lane_off + acc_w(1), v);
        if (t < 32)
            for (int c = 0; c < 64; ++c) atomicAdd(&gr.W[1][t * 64 + c], v[c]);
        tc::tmem_ld32(tmem + lane_off + acc_w(2), v);
        if (t < 32)
            for (int c = 0; c < 32; ++c) atomicAdd(&gr.W[2][t * 32 + c], v[c]);
        tc::tmem_ld32(tmem + lane_off + acc_w(3), v);
        if (t < 32)
            for (int c = 0; c < 32; ++c) atomicAdd(&gr.W[3][t * 32 + c], v[c]);
        else if (t < 35)
            for (int c = 0; c < 32; ++c) atomicAdd(&gr.W[5][(t - 32) * 32 + c], v[c]);
        tc::tmem_ld32(tmem + lane_off + acc_w(4), v);
        if (t == 0)
            for (int c = 0; c < 32; ++c) atomicAdd(&gr.W[4][c], v[c]);
        float b[NCH];
#pragma unroll
        for (int l = 0; l < NCH; ++l) {
            float h[16];
            tc::tmem_ld16(tmem + lane_off + acc_b(l), h);
            b[l] = h[0];
        }
        if (t < 64 && gr.b[0]) atomicAdd(&gr.b[0][t], b[0]);
        if (t < 32 && gr.b[1]) atomicAdd(&gr.b[1][t], b[1]);
        if (t < 32 && gr.b[2]) atomicAdd(&gr.b[2][t], b[2]);
        if (t < 32 && gr.b[3]) atomicAdd(&gr.b[3][t], b[3]);
        else if (t >= 32 && t < 35 && gr.b[5]) atomicAdd(&gr.b[5][t - 32], b[3]);
        if (t == 0 && gr.b[4]) atomicAdd(&gr.b[4][0], b[4]);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_dealloc(tmem, tmem_cols(BWD));
}

}  // namespace

namespace {
MlpDev paper_dev(const sssgs_mlp* m) {
    MlpDev d;
    d.kind = SSSGS_MLP_PAPER;
    d.L = NCH;
    for (int l = 0; l <= SSSGS_MAX_LAYERS; ++l) d.w[l] = l <= NCH ? (l < NCH ? kin(l) : 16) : 0;
    for (int l = 0; l < SSSGS_MAX_LAYERS; ++l) {
        d.W[l] = l < 6 ? m->W[l] : nullptr;
        d.b[l] = l < 6 ? m->b[l] : nullptr;
    }
    return d;
}

int num_sms_paper() { return device_sm_count(); }

// Backward workspace: the active-row list, its flags, per-block counts and
// offsets, and the row count.
struct PaperWs {
    size_t active, flag, cnt, off, nact, total;
};
PaperWs paper_ws(int64_t n) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nb = (size_t)((n + 1023) / 1024);
    PaperWs w;
    size_t o = 0;
    w.active = o; o += al(4 * (size_t)n);
    w.flag = o;   o += al((size_t)n);
    w.cnt = o;    o += al(4 * nb);
    w.off = o;    o += al(4 * nb);
    w.nact = o;   o += 256;
    w.total = o + 256;
    return w;
}
}  // namespace

size_t paper_tc_workspace_bytes(int64_t n_items) { return paper_ws(std::max<int64_t>(n_items, 1)).total; }

int paper_tc_fwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                 const sssgs_scene* scene, float* out, int32_t* d_status, cudaStream_t st) {
    if ((uintptr_t)out & 15) return SSSGS_ERR_INVALID_ARG;
    const int64_t n = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    if (n == 0) return SSSGS_OK;
    cudaFuncSetAttribute(k_mlp_paper_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PSmem::TOTAL);
    const int64_t tiles = (n + PR - 1) / PR;
    const int grid = (int)std::min<int64_t>((tiles + PLANES - 1) / PLANES, (int64_t)num_sms_paper());
    sssgs_mlp_grad none{};
    k_mlp_paper_tc<false><<<grid, PLANES * PT, PSmem::TOTAL, st>>>(paper_dev(mlp), d_pairs, n_pairs, n, *scene, out,
                                                                    nullptr, 0, none, nullptr, nullptr, nullptr,
                                                                    d_status);
    sssgs::note_launches(1);
    return launch_status();
}

int paper_tc_bwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                 const sssgs_scene* scene, const float* dout, int64_t dstride, const sssgs_mlp_grad* grad,
                 float* dx_items, void* workspace, size_t workspace_bytes, int32_t* d_status, cudaStream_t st) {
    const int64_t n = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    if (n == 0) return SSSGS_OK;
    if (n >= ((int64_t)1 << 32)) return SSSGS_ERR_INVALID_ARG;
    const PaperWs W = paper_ws(n);
    if (!workspace || workspace_bytes < W.total) return SSSGS_ERR_WORKSPACE;
    uint8_t* base = (uint8_t*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    uint32_t* active = (uint32_t*)(base + W.active);
    uint32_t* nact = (uint32_t*)(base + W.nact);
    int launches = launch_active_rows(dout, dstride, n, base + W.flag, (uint32_t*)(base + W.cnt),
                                      (uint32_t*)(base + W.off), nact, active, dx_items, st);
    cudaFuncSetAttribute(k_mlp_paper_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PSmem::TOTAL);
    const int64_t tiles = (n + PR - 1) / PR;
    const int grid = (int)std::min<int64_t>((tiles + PLANES - 1) / PLANES, (int64_t)num_sms_paper());
    k_mlp_paper_tc<true><<<grid, PLANES * PT, PSmem::TOTAL, st>>>(paper_dev(mlp), d_pairs, n_pairs, n, *scene,
                                                                   nullptr, dout, dstride, *grad, dx_items, active,
                                                                   nact, d_status);
    sssgs::note_launches(launches + 1);
    return launch_status();
}

}  // namespace sssgs
