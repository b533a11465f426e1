// Joint SSS-residual / incident-light network f_Theta (Eq. 6) on the tensor
// cores: BF16 operands, FP32 accumulation in TMEM (tcgen05.mma, cta_group::1).
//
// Forward: one persistent CTA of 4 warps per SM. The CTA converts every
// layer's weights to BF16 once into shared memory (core-matrix layout, see
// tc.cuh). Per 128-row tile of (pair, Gaussian) items, each thread builds its
// row's network input, then for every layer one thread issues K/16 MMAs
// (M = 128 rows, N = layer width, K = 16) into a 128-column TMEM accumulator
// and commits them to an mbarrier; the four warps read their 32 TMEM lanes
// back (tcgen05.ld), add the bias, apply ReLU, round to BF16 and write the
// next layer's A operand to shared memory. The 4-wide output layer is padded
// to N = 16; its epilogue applies the heads (sigmoid -> L_SSS, ReLU -> L_in).
//
// Numerics: inputs, weights and hidden activations are rounded to BF16 (round
// to nearest even); products accumulate in FP32; biases and heads in FP32.
#include "mlp_common.cuh"
#include "tc.cuh"

namespace sssgs {

constexpr int TC_ROWS = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_MAXW = 128;

struct TcLayout {
    uint32_t offW[SSSGS_MAX_LAYERS];   // weight images
    uint32_t offA;                     // activation tile
    uint32_t offBias;                  // FP32 biases
    uint32_t offBar;                   // mbarrier + TMEM address
    uint32_t total;
    int Np[SSSGS_MAX_LAYERS];          // padded output widths
    int biasOff[SSSGS_MAX_LAYERS];
};

__host__ __device__ inline TcLayout tc_layout(const MlpDev& net) {
    TcLayout T;
    uint32_t o = 0;
    int bo = 0;
    for (int l = 0; l < net.L; ++l) {
        T.Np[l] = (net.w[l + 1] + 15) & ~15;
        T.offW[l] = o;
        o += (uint32_t)(T.Np[l] * net.w[l] * 2);
        o = (o + 127) & ~127u;
        T.biasOff[l] = bo;
        bo += T.Np[l];
    }
    T.offA = o;
    o += TC_ROWS * TC_MAXW * 2;
    T.offBias = o;
    o += (uint32_t)(bo * 4);
    o = (o + 15) & ~15u;
    T.offBar = o;
    o += 16;
    T.total = o;
    return T;
}

// Convert layer weights (FP32, out x in, row-major) into BF16 operand images.
__device__ __forceinline__ void stage_weights_bf16(const MlpDev& net, const TcLayout& T, uint8_t* smem, float* sbias) {
    for (int l = 0; l < net.L; ++l) {
        const int K = net.w[l], N = net.w[l + 1], Np = T.Np[l];
        const float* W = net.W[l];
        uint8_t* base = smem + T.offW[l];
        for (int i = threadIdx.x; i < Np * K; i += blockDim.x) {
            const int n = i / K, k = i - n * K;
            const float v = n < N ? W[n * K + k] : 0.f;
            *reinterpret_cast<__nv_bfloat16*>(base + tc::blk_offset(n, k, K)) = __float2bfloat16_rn(v);
        }
        for (int n = threadIdx.x; n < Np; n += blockDim.x) sbias[T.biasOff[l] + n] = n < N ? net.b[l][n] : 0.f;
    }
}

// Store 8 consecutive FP32 values of row r (columns c..c+7) as BF16.
__device__ __forceinline__ void store8_bf16(uint8_t* base, int r, int c, int C, const float* v) {
    uint4 q;
    q.x = tc::pack_bf16(v[0], v[1]);
    q.y = tc::pack_bf16(v[2], v[3]);
    q.z = tc::pack_bf16(v[4], v[5]);
    q.w = tc::pack_bf16(v[6], v[7]);
    *reinterpret_cast<uint4*>(base + tc::blk_offset(r, c, C)) = q;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_fwd_tc(MlpDev net, const sssgs_pair* __restrict__ pairs,
                                                              int n_pairs, int64_t n_items, sssgs_scene sc,
                                                              float* __restrict__ out, int32_t* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const TcLayout T = tc_layout(net);
    const int tid = threadIdx.x, warp = tid >> 5;
    float* sbias = reinterpret_cast<float*>(smem + T.offBias);
    const uint32_t bar = tc::smem_u32(smem + T.offBar);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + T.offBar + 8);
    uint8_t* sA = smem + T.offA;
    const uint32_t a_addr = tc::smem_u32(sA);

    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(s_tmem), 128);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    stage_weights_bf16(net, T, smem, sbias);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t n_tiles = (n_items + TC_ROWS - 1) / TC_ROWS;
    const int K0 = net.w[0];
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t m = tile * TC_ROWS + tid;
        {
            float x[TC_MAXW];
#pragma unroll
            for (int k = 0; k < 64; ++k) x[k] = 0.f;
            if (m < n_items) {
                const int p = pair_of_item(pairs, n_pairs, m);
                const sssgs_pair& P = pairs[p];
                build_input(net, P, sc, P.g_begin + (m - P.item_offset), x);
            }
            for (int c = 0; c < K0; c += 8) store8_bf16(sA, tid, c, K0, x + c);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        for (int l = 0; l < net.L; ++l) {
            const int K = net.w[l], N = T.Np[l];
            if (tid == 0) {
                tc::fence_after();
                const uint32_t idesc = tc::idesc_bf16(TC_ROWS, N, false, false);
                const uint32_t w_addr = tc::smem_u32(smem + T.offW[l]);
                const uint32_t sbo = (uint32_t)(K / 8) * 128u;
                for (int k = 0; k < K / 16; ++k) {
                    const uint64_t ad = tc::make_desc(a_addr + k * 256, 128, sbo);
                    const uint64_t bd = tc::make_desc(w_addr + k * 256, 128, sbo);
                    tc::mma_bf16(tmem, ad, bd, idesc, k > 0 ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            __syncwarp();
            bool got = tc::mbar_wait(bar, phase);
            phase ^= 1;
            tc::fence_after();
            if (got) {
                const float* bl = sbias + T.biasOff[l];
                if (l < net.L - 1) {
                    for (int c0 = 0; c0 < N; c0 += 32) {
                        float v[32];
                        tc::tmem_ld32(lane_base + c0, v);
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + bl[c0 + j], 0.f);
#pragma unroll
                        for (int q = 0; q < 4; ++q) store8_bf16(sA, tid, c0 + 8 * q, N, v + 8 * q);
                    }
                } else {
                    float v[16];
                    tc::tmem_ld16(lane_base, v);
                    if (m < n_items) {
                        float4 o4;
                        o4.x = 1.f / (1.f + expf(-(v[0] + bl[0])));
                        o4.y = 1.f / (1.f + expf(-(v[1] + bl[1])));
                        o4.z = 1.f / (1.f + expf(-(v[2] + bl[2])));
                        o4.w = fmaxf(v[3] + bl[3], 0.f);
                        reinterpret_cast<float4*>(out)[m] = o4;
                    }
                }
            }
            tc::fence_before();
            tc::fence_async_smem();
            ok = __syncthreads_and(got) != 0;
            if (!ok) break;
        }
    }
    if (!ok && tid == 0 && status) atomicOr(status, SSSGS_STATUS_TIMEOUT);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

}  // namespace sssgs

using namespace sssgs;

namespace {
bool tc_supported(const sssgs_mlp* m) {
    if (m->kind != SSSGS_MLP_PE6 || m->width[0] != 64 || m->width[m->n_layers] != 4) return false;
    for (int l = 1; l < m->n_layers; ++l)
        if (m->width[l] < 16 || m->width[l] > TC_MAXW || m->width[l] % 32) return false;
    return true;
}

MlpDev to_dev_tc(const sssgs_mlp* m) {
    MlpDev d;
    d.kind = m->kind;
    d.L = m->n_layers;
    for (int l = 0; l <= SSSGS_MAX_LAYERS; ++l) d.w[l] = l <= m->n_layers ? m->width[l] : 0;
    for (int l = 0; l < SSSGS_MAX_LAYERS; ++l) {
        d.W[l] = l < m->n_layers ? m->W[l] : nullptr;
        d.b[l] = l < m->n_layers ? m->b[l] : nullptr;
    }
    return d;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}
}  // namespace

int sssgs_mlp_fwd_tc(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                     const sssgs_scene* scene, float* out, int32_t* d_status, sssgs_stream stream) {
    if (!tc_supported(mlp)) return SSSGS_ERR_UNSUPPORTED;
    if ((uintptr_t)out & 15) return SSSGS_ERR_INVALID_ARG;
    int64_t n = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    if (n == 0) return SSSGS_OK;
    MlpDev net = to_dev_tc(mlp);
    TcLayout T = tc_layout(net);
    if (T.total > 227 * 1024) return SSSGS_ERR_UNSUPPORTED;
    cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T.total);
    int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    int grid = (int)std::min<int64_t>(tiles, (int64_t)sm_count());
    k_mlp_fwd_tc<<<grid, TC_THREADS, T.total, (cudaStream_t)stream>>>(net, d_pairs, n_pairs, n, *scene, out,
                                                                        d_status);
    sssgs::note_launches(1);
    return launch_status();
}

int sssgs_mlp_bwd_tc(const sssgs_mlp*, const sssgs_pair*, const sssgs_pair*, int, const sssgs_scene*, const float*,
                     const sssgs_mlp_grad*, float*, void*, size_t, int32_t*, sssgs_stream) {
    return SSSGS_ERR_UNSUPPORTED;
}
