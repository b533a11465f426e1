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
#include "mlp_tc_util.cuh"

namespace sssgs {

constexpr int TC_ROWS = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_MAXW = 128;
// Tile lanes per forward CTA: three (216 KB of shared memory with the
// resident weights, 384 TMEM columns) measured 4.21 ms against 4.61 for two.
constexpr int TC_FWD_LANES = 3;
constexpr int TC_FWD_TMEM = TC_FWD_LANES * 128 <= 256 ? 256 : 512;  // TMEM columns (power of two)

struct TcLayout {
    uint32_t offW[SSSGS_MAX_LAYERS];   // weight images
    uint32_t offA;                     // activation tile
    uint32_t offBias;                  // FP32 biases
    uint32_t offBar;                   // mbarrier + TMEM address
    uint32_t offTab;                   // per-layer table (TcLayerTab) in shared memory
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
    o += TC_FWD_LANES * TC_ROWS * TC_MAXW * 2;  // one activation tile per lane
    T.offBias = o;
    o += (uint32_t)(bo * 4);
    o = (o + 15) & ~15u;
    T.offBar = o;
    o += 64 + 8 * 256;                           // mbarriers, TMEM address, flags, pair offsets
    T.offTab = o;
    o += SSSGS_MAX_LAYERS * 16;
    T.total = o;
    return T;
}

// One layer's geometry, copied to shared memory at kernel start: a runtime
// index into the parameter tables would be served from local memory, and with
// the shared-memory carve-out these kernels take nearly every such load misses
// L1 and waits on L2 inside each layer round.
struct TcLayerTab {
    int K, Np, offW, bias;
};

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


// TC_FWD_LANES independent tile lanes per CTA: warpgroup g (4 warps) owns
// activation buffer g, TMEM columns [128 g, 128 g + 128) and mbarrier g, and
// processes every TC_FWD_LANES-th tile; the tensor core interleaves the lanes'
// MMAs, so one lane's epilogue overlaps the others' matrix work. Weights are
// shared.
__global__ void __launch_bounds__(TC_FWD_LANES * TC_THREADS, 1) k_mlp_fwd_tc(MlpDev net, const sssgs_pair* __restrict__ pairs,
                                                                  int n_pairs, int64_t n_items, sssgs_scene sc,
                                                                  float* __restrict__ out,
                                                                  int32_t* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const TcLayout T = tc_layout(net);
    const int tid = threadIdx.x, wg = tid >> 7, t = tid & 127, warp = (tid >> 5) & 3;
    float* sbias = reinterpret_cast<float*>(smem + T.offBias);
    const uint32_t bar = tc::smem_u32(smem + T.offBar) + 8 * wg;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + T.offBar + 32);
    volatile int* s_fail = reinterpret_cast<volatile int*>(smem + T.offBar + 40);
    int64_t* s_off = reinterpret_cast<int64_t*>(smem + T.offBar + 64);
    uint8_t* sA = smem + T.offA + wg * (TC_ROWS * TC_MAXW * 2);
    const uint32_t a_addr = tc::smem_u32(sA);

    if (tid < 32) {
        tc::tmem_alloc(tc::smem_u32(s_tmem), TC_FWD_TMEM);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int g = 0; g < TC_FWD_LANES; ++g) {
            tc::mbar_init(tc::smem_u32(smem + T.offBar) + 8 * g, 1);
            s_fail[g] = 0;
        }
        tc::fence_mbar_init();
    }
    for (int p = tid; p < n_pairs && p < TC_MAX_SMEM_PAIRS; p += blockDim.x) s_off[p] = pairs[p].item_offset;
    TcLayerTab* s_tab = reinterpret_cast<TcLayerTab*>(smem + T.offTab);
    if (tid == 0)
        for (int l = 0; l < net.L; ++l) s_tab[l] = TcLayerTab{net.w[l], T.Np[l], (int)T.offW[l], T.biasOff[l]};
    stage_weights_bf16(net, T, smem, sbias);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *s_tmem + (uint32_t)(wg * 128);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t n_tiles = (n_items + TC_ROWS - 1) / TC_ROWS;
    for (int64_t tile = TC_FWD_LANES * (int64_t)blockIdx.x + wg; tile < n_tiles && ok;
         tile += TC_FWD_LANES * (int64_t)gridDim.x) {
        const int64_t m = tile * TC_ROWS + t;
        {
            float x[64];
#pragma unroll
            for (int k = 0; k < 64; ++k) x[k] = 0.f;
            if (m < n_items) {
                const int p = pair_lookup(s_off, pairs, n_pairs, m);
                const sssgs_pair& P = pairs[p];
                build_input_pe6(P, sc, P.g_begin + (m - P.item_offset), m, x);
            }
#pragma unroll
            for (int c = 0; c < 64; c += 8) store8_bf16(sA, t, c, 64, x + c);
        }
        tc::fence_async_smem();
        tc::fence_before();
        named_sync(1 + wg, 128);
        for (int l = 0; l < net.L; ++l) {
            const TcLayerTab lt = s_tab[l];
            const int K = lt.K, N = lt.Np;
            if (t < 32) {   // the lane group's first warp; lane 0 issues
                tc::fence_after();
                const uint32_t idesc = tc::idesc_bf16(TC_ROWS, N, false, false);
                const uint32_t sbo = (uint32_t)(K / 8) * 128u;
                const tc::Desc2 da = tc::desc2(a_addr, 128, sbo);
                const tc::Desc2 dw = tc::desc2(tc::smem_u32(smem + lt.offW), 128, sbo);
#pragma unroll
                for (int k = 0; k < TC_MAXW / 16; ++k)
                    if (k < K / 16) tc::mma_bf16_w(tmem, da, k * 256, dw, k * 256, idesc, k > 0 ? 1u : 0u, t);
                tc::mma_commit_w(bar, t);
            }
            const bool got = tc::mbar_wait(bar, phase);
            phase ^= 1;
            tc::fence_after();
            if (!got) s_fail[wg] = 1;
            if (got) {
                const float* bl = sbias + lt.bias;
                if (l < net.L - 1) {
                    for (int c0 = 0; c0 < N; c0 += 64) {
                        float v[64];
                        tc::tmem_ld64(lane_base + c0, v);
#pragma unroll
                        for (int q = 0; q < 8; ++q) store8_bias_relu(sA, t, c0 + 8 * q, N, v + 8 * q, bl + c0 + 8 * q);
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
            named_sync(1 + wg, 128);
            ok = s_fail[wg] == 0;
            if (!ok) break;
        }
    }
    if (!ok && t == 0 && status) atomicOr(status, SSSGS_STATUS_TIMEOUT);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_dealloc(*s_tmem, TC_FWD_TMEM);
}

// ---------------------------------------------------------------- backward
//
// Per 128-row tile: recompute the forward from the input H_0 keeping every
// layer input H_l (BF16) in shared memory, form the head gradient dZ_L, then
// for l = L-1 .. 0 (lane 0 of warp 0 issues, all warps run epilogues):
//   dW_l (+)= dZ_{l+1}^T H_l   hidden layers: accumulated across tiles in TMEM
//                              first/last layer: per tile, summed in registers
//   dH_l  = dZ_{l+1} W_l       (hidden layers in one 128-column round, the
//                              last layer in two 64-column halves), then
//   dZ_l  = bf16(dH_l * [H_l > 0]) written in place over H_l; dH_0 is the
//   network-input gradient, mapped to (d mu, d n, d v) per item.
// A last round forms every bias gradient db_l (+)= dZ_{l+1}^T 1 (MMAs against
// a ones operand; dZ_{l+1} stays in place of H_{l+1} until then) while the
// next tile's H_0 is built.
// Weight images (BF16, operand layout) stream from global memory with
// cp.async.bulk into two shared-memory slots, two uses ahead.
// TMEM columns: [0, 128) recompute and dH, [64, 128) the per-tile dW of the
// first and last layers (with a 64-wide dH), [0, 16 (L-1)) the bias round,
// [128, 512) the hidden layers' dW accumulators.

struct TcBwdLayout {
    uint32_t offH[SSSGS_MAX_LAYERS];   // layer inputs (later dZ, in place)
    uint32_t offDZL, offOnes, offW[2], offBias, offDbL, offDx, offBar, offPairs, offGb;
    uint32_t total;
    uint32_t gW[SSSGS_MAX_LAYERS];     // weight image offsets in the global workspace
    uint32_t wbytes[SSSGS_MAX_LAYERS];
    uint32_t gtotal;
    int Np[SSSGS_MAX_LAYERS];
    int biasOff[SSSGS_MAX_LAYERS];
    int colW[SSSGS_MAX_LAYERS];        // TMEM column of dW_l (hidden layers)
};

__host__ __device__ inline TcBwdLayout tc_bwd_layout(const MlpDev& net) {
    TcBwdLayout T;
    uint32_t o = 0, g = 0, wmax = 0;
    int bo = 0, col = 128;
    for (int l = 0; l < net.L; ++l) {
        T.Np[l] = (net.w[l + 1] + 15) & ~15;
        T.offH[l] = o;
        o += (uint32_t)(TC_ROWS * net.w[l] * 2);
        T.wbytes[l] = (uint32_t)(T.Np[l] * net.w[l] * 2);
        T.gW[l] = g;
        g += (T.wbytes[l] + 127) & ~127u;
        wmax = T.wbytes[l] > wmax ? T.wbytes[l] : wmax;
        T.biasOff[l] = bo;
        bo += T.Np[l];
        T.colW[l] = -1;
        if (l >= 1 && l <= net.L - 2) {
            T.colW[l] = col;
            col += net.w[l];
        }
    }
    T.offDZL = o;  o += TC_ROWS * 16 * 2;
    T.offOnes = o; o += 16 * TC_ROWS * 2;
    T.offW[0] = o; o += wmax;
    T.offW[1] = o; o += wmax;
    T.offBias = o; o += (uint32_t)(bo * 4);
    T.offDbL = o;  o += 16 * 4;
    T.offDx = o;   o += 7 * TC_ROWS * 4;
    T.offBar = o;  o += 32;
    T.offPairs = o; o += 8 * 256;
    T.offGb = o;   o += 4 * 256;
    T.total = o;
    T.gtotal = g;
    T.colW[0] = col;          // > 512 signals "does not fit" to the host check
    return T;
}

__global__ void k_mlp_weights_bf16(MlpDev net, TcBwdLayout T, uint8_t* __restrict__ gimg) {
    const int l = blockIdx.y;
    const int K = net.w[l], N = net.w[l + 1], Np = T.Np[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Np * K; i += gridDim.x * blockDim.x) {
        const int n = i / K, k = i - n * K;
        const float v = n < N ? net.W[l][n * K + k] : 0.f;
        *reinterpret_cast<__nv_bfloat16*>(gimg + T.gW[l] + tc::blk_offset(n, k, K)) = __float2bfloat16_rn(v);
    }
}


// ---------------------------------------------------------------- active rows
//
// A row whose upstream gradient (its four dL/d(L_SSS, L_in)) is exactly zero adds
// exactly zero to every dW, db and to its own input gradient: all dZ of the
// chain are 0 * finite = 0, and bf16(0) = 0. Gaussians hidden behind the
// surface in a view never contribute to a pixel, so their rows are zero. The
// backward therefore runs on the list of the other rows, in item order
// (deterministic: count with a flag byte per item, scan, write); dx_items is
// cleared first, so the rest keep dx = 0.
constexpr int ACT_BLOCK = 1024;

__device__ __forceinline__ bool row_active(const float* __restrict__ dout, int64_t dstride, int64_t m) {
    const float4 u = *reinterpret_cast<const float4*>(dout + dstride * m);
    return (u.x != 0.f) | (u.y != 0.f) | (u.z != 0.f) | (u.w != 0.f);
}

__global__ void __launch_bounds__(ACT_BLOCK) k_active_count(const float* __restrict__ dout, int64_t dstride,
                                                            int64_t n, uint32_t* __restrict__ cnt,
                                                            uint8_t* __restrict__ flag) {
    const int64_t m = (int64_t)blockIdx.x * ACT_BLOCK + threadIdx.x;
    const bool a = m < n && row_active(dout, dstride, m);
    if (m < n) flag[m] = a ? 1 : 0;
    const int c = __syncthreads_count(a);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (uint32_t)c;
}

// Exclusive scan of the block counts (one block, carried over chunks of 1024);
// n_active = the total.
__global__ void __launch_bounds__(1024) k_active_scan(const uint32_t* __restrict__ cnt, int nb,
                                                      uint32_t* __restrict__ off, uint32_t* __restrict__ n_active) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nb ? cnt[b] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(SSSGS_FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(SSSGS_FULL, w, o);
                if (lane >= o) w += y;
            }
            wsum[lane] = w;
        }
        __syncthreads();
        const uint32_t c = carry;
        const uint32_t incl = x + (warp > 0 ? wsum[warp - 1] : 0u);
        if (b < nb) off[b] = c + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_active = carry;
}

__global__ void __launch_bounds__(ACT_BLOCK) k_active_write(const uint8_t* __restrict__ flag, int64_t n,
                                                            const uint32_t* __restrict__ off,
                                                            uint32_t* __restrict__ active) {
    __shared__ uint32_t wcnt[ACT_BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t m = (int64_t)blockIdx.x * ACT_BLOCK + threadIdx.x;
    const bool a = m < n && flag[m] != 0;
    const uint32_t bal = __ballot_sync(SSSGS_FULL, a);
    if (lane == 0) wcnt[warp] = (uint32_t)__popc(bal);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wcnt[w];
    if (a) active[off[blockIdx.x] + before + (uint32_t)__popc(bal & ((1u << lane) - 1u))] = (uint32_t)m;
}

int launch_active_rows(const float* dout, int64_t dstride, int64_t n, uint8_t* flag, uint32_t* cnt, uint32_t* off,
                       uint32_t* nact, uint32_t* active, float* dx_items, cudaStream_t st) {
    const int nb = (int)((n + ACT_BLOCK - 1) / ACT_BLOCK);
    // every row's input gradient starts at zero (one contiguous clear); the
    // backward then overwrites the active rows
    cudaMemsetAsync(dx_items, 0, (size_t)n * SSSGS_DX * sizeof(float), st);
    k_active_count<<<nb, ACT_BLOCK, 0, st>>>(dout, dstride, n, cnt, flag);
    k_active_scan<<<1, 1024, 0, st>>>(cnt, nb, off, nact);
    k_active_write<<<nb, ACT_BLOCK, 0, st>>>(flag, n, off, active);
    return 3;
}

// Per-layer geometry of the backward network in closed form. The backward
// runs the fixed widths w = [64, 128, ..., 128, 4] (the host checks them and
// this geometry against tc_bwd_layout), so a layer's input width, activation
// and weight-image offsets, bias offset and TMEM column follow from its
// index. A runtime index into the kernel's parameter tables would be served
// from local memory, and with the shared-memory carve-out this kernel takes
// nearly every such load misses L1 and waits on L2 inside each round.
struct BwdGeom {
    int L;
    __host__ __device__ __forceinline__ int kin(int l) const { return l == 0 ? 64 : 128; }
    __host__ __device__ __forceinline__ int np(int l) const { return l == L - 1 ? 16 : 128; }
    // H_l in shared memory, and weight image l in the global workspace
    __host__ __device__ __forceinline__ uint32_t off(int l) const {
        return l == 0 ? 0u : 16384u + (uint32_t)(l - 1) * 32768u;
    }
    __host__ __device__ __forceinline__ uint32_t wbytes(int l) const {
        return l == 0 ? 16384u : (l == L - 1 ? 4096u : 32768u);
    }
    __host__ __device__ __forceinline__ int bias(int l) const { return 128 * l; }
    __host__ __device__ __forceinline__ int colw(int l) const { return 128 * l; }   // hidden layers 1 .. L-2
};

__global__ void __launch_bounds__(2 * TC_THREADS, 1) k_mlp_bwd_tc(MlpDev net, TcBwdLayout T,
                                                              const uint8_t* __restrict__ gimg,
                                                              const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                              int64_t n_items, sssgs_scene sc,
                                                              const float* __restrict__ dout, int64_t dstride,
                                                              sssgs_mlp_grad gr,
                                                              float* __restrict__ dx_items,
                                                              const uint32_t* __restrict__ active,
                                                              const uint32_t* __restrict__ n_active,
                                                              int32_t* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    // 8 warps: warpgroup wg handles half of the columns of every column-parallel
    // epilogue; per-row scalar work (input, heads, input gradient) runs on wg 0.
    const int tid = threadIdx.x, lane = tid & 31, wg = tid >> 7, t = tid & 127, warp = (tid >> 5) & 3;
    const int L = net.L;
    int64_t* s_off = reinterpret_cast<int64_t*>(smem + T.offPairs);
    int* s_gb = reinterpret_cast<int*>(smem + T.offGb);
    float* sbias = reinterpret_cast<float*>(smem + T.offBias);
    float* sdbL = reinterpret_cast<float*>(smem + T.offDbL);
    const uint32_t bar_m = tc::smem_u32(smem + T.offBar);
    const uint32_t bar_w0 = bar_m + 8, bar_w1 = bar_m + 16;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + T.offBar + 24);
    uint8_t* sDZL = smem + T.offDZL;
    float* s_dx = reinterpret_cast<float*>(smem + T.offDx);   // [7][TC_ROWS]

    if (tid < 32) {
        tc::tmem_alloc(tc::smem_u32(s_tmem), 512);
        tc::tmem_relinquish();
    }
    for (int p = tid; p < n_pairs && p < TC_MAX_SMEM_PAIRS; p += blockDim.x) {
        s_off[p] = pairs[p].item_offset;
        s_gb[p] = pairs[p].g_begin;
    }
    if (tid == 0) {
        tc::mbar_init(bar_m, 1);
        tc::mbar_init(bar_w0, 1);
        tc::mbar_init(bar_w1, 1);
        tc::fence_mbar_init();
    }
    // constants: ones operand (16 x 128, K-major), biases, last-layer db partials
    for (int i = tid; i < 16 * TC_ROWS / 2; i += blockDim.x)
        reinterpret_cast<uint32_t*>(smem + T.offOnes)[i] = 0x3F803F80u;   // two bf16 1.0
    const BwdGeom G{L};
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        const float* bsrc = l == 0 ? net.b[0] : l == 1 ? net.b[1] : l == 2 ? net.b[2] : l == 3 ? net.b[3]
                          : l == 4 ? net.b[4] : l == 5 ? net.b[5] : l == 6 ? net.b[6] : net.b[7];
        const int nw = l == L - 1 ? 4 : 128;
        for (int n = tid; n < G.np(l); n += blockDim.x) sbias[G.bias(l) + n] = n < nw ? bsrc[n] : 0.f;
    }
    if (tid < 16) sdbL[tid] = 0.f;
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;

    // per-thread accumulators: dW_0 row (thread = output unit), dW_{L-1}^T row
    // (thread = input unit of the last layer), db of layers 0..L-2
    float acc0[32];                    // this warpgroup's 32 of dW_0's 64 input columns
    float accL[4] = {0.f, 0.f, 0.f, 0.f};
    float dbacc[SSSGS_MAX_LAYERS];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc0[j] = 0.f;
#pragma unroll
    for (int j = 0; j < SSSGS_MAX_LAYERS; ++j) dbacc[j] = 0.f;

    uint32_t ph_m = 0;
    uint32_t use = 0;            // weight uses begun (2L per tile); use u reads slot u & 1
    bool ok = true, any_tile = false;
    const int uses_per_tile = 2 * L;
    auto layer_of_use = [&](uint32_t u) -> int {
        const int k = (int)(u % (uint32_t)uses_per_tile);
        return k < L ? k : 2 * L - 1 - k;
    };
    // rows = the active items (see k_active_count)
    const int64_t n_rows = *n_active;
    const int64_t n_tiles = (n_rows + TC_ROWS - 1) / TC_ROWS;
    const uint32_t wslot0 = tc::smem_u32(smem + T.offW[0]), wslot1 = tc::smem_u32(smem + T.offW[1]);
    // Weight images stream into two slots. The copy for use u + 2 starts as
    // soon as the MMAs of use u have completed (its slot's release), so it
    // has the rest of use u and all of use u + 1 to land. Thread 0 copies;
    // fetched = one past the last use copied.
    uint32_t fetched = 0;
    auto fetch_use = [&](uint32_t u) {
        const int64_t tl = (int64_t)blockIdx.x + (int64_t)(u / (uint32_t)uses_per_tile) * gridDim.x;
        if (tl < n_tiles) {
            const int lu = layer_of_use(u);
            const uint32_t b = (u & 1) ? bar_w1 : bar_w0;
            tc::mbar_arrive_expect_tx(b, G.wbytes(lu));
            tc::bulk_g2s((u & 1) ? wslot1 : wslot0, gimg + G.off(lu), G.wbytes(lu), b);
            fetched = u + 1;
        }
    };
    if (tid == 0) {
        fetch_use(0);
        fetch_use(1);
    }
    // warp 0 (which issues the MMAs): wait for this use's weights
    auto begin_use = [&]() -> bool {
        bool got = true;
        if (tid < 32) {
            got = tc::mbar_wait((use & 1) ? bar_w1 : bar_w0, (use >> 1) & 1u);
            tc::fence_after();
        }
        return got;
    };
    auto release_use = [&](uint32_t u) {
        if (tid == 0) fetch_use(u + 2);
    };
    auto wait_mma = [&]() -> bool {
        const bool got = tc::mbar_wait(bar_m, ph_m);
        ph_m ^= 1u;
        tc::fence_after();
        return got;
    };
    auto sync_all = [&](bool mine) -> bool {
        tc::fence_before();
        tc::fence_async_smem();
        return __syncthreads_and(mine) != 0;
    };

    // Per-row inputs (network parameters and upstream gradient) of a tile:
    // the row ids two tiles ahead and the inputs of the next tile are loaded
    // while the current one is processed, so no load waits on another load
    // inside a tile.
    // Item ids fit 32 bits (the host checks n < 2^32); NO_ROW marks a
    // padding row past the list.
    constexpr uint32_t NO_ROW = 0xFFFFFFFFu;
    struct RowIn {
        Pe6Params q;
        float up[4];
        uint32_t m;
        int pidx;
        bool valid;
    };
    auto load_act = [&](int64_t tl) -> uint32_t {
        const int64_t row = tl * TC_ROWS + t;
        return (tl < n_tiles && row < n_rows) ? active[row] : NO_ROW;
    };
    auto load_row = [&](uint32_t mr) -> RowIn {
        RowIn r;
        r.valid = mr != NO_ROW;
        r.pidx = 0;
        r.m = 0;
        if (r.valid) {
            r.m = mr;
            r.pidx = pair_lookup(s_off, pairs, n_pairs, mr);
            const int gb = n_pairs <= TC_MAX_SMEM_PAIRS ? s_gb[r.pidx] : pairs[r.pidx].g_begin;
            const int64_t io = n_pairs <= TC_MAX_SMEM_PAIRS ? s_off[r.pidx] : pairs[r.pidx].item_offset;
            r.q = load_pe6_params(sc, gb + ((int64_t)mr - io), mr);
            const float4 u = *reinterpret_cast<const float4*>(dout + dstride * (int64_t)mr);
            r.up[0] = u.x;
            r.up[1] = u.y;
            r.up[2] = u.z;
            r.up[3] = u.w;
        }
        return r;
    };
    RowIn cur = load_row(load_act(blockIdx.x));
    uint32_t act1 = load_act((int64_t)blockIdx.x + gridDim.x);
    float dmu_a[3] = {0.f, 0.f, 0.f};     // Fourier part of dL/dmu (frequencies 0..2, warpgroup 0)
    const uint32_t ones = tc::smem_u32(smem + T.offOnes);

    // H_0 of a tile: the network input, split between the warpgroups: columns
    // [0, 18) (frequencies 0..2) on warpgroup 0, [18, 64) on warpgroup 1.
    auto build_h0 = [&](const RowIn& r) {
        if (wg == 0) {
            float x[18];
#pragma unroll
            for (int k = 0; k < 18; ++k) x[k] = 0.f;
            if (r.valid) pe6_fourier<0, 3>(r.q.mu, x);
            store8_bf16(smem + G.off(0), t, 0, 64, x);
            store8_bf16(smem + G.off(0), t, 8, 64, x + 8);
            store1_bf16(smem + G.off(0), t, 16, 64, x[16]);
            store1_bf16(smem + G.off(0), t, 17, 64, x[17]);
        } else {
            float x[46];
#pragma unroll
            for (int k = 0; k < 46; ++k) x[k] = 0.f;
            if (r.valid) {
                pe6_fourier<3, 6>(r.q.mu, x);
                pe6_direct(pairs[r.pidx], r.q.mu, r.q.n, r.q.v, x + 18);
            }
#pragma unroll
            for (int c = 18; c < 24; ++c) store1_bf16(smem + G.off(0), t, c, 64, x[c - 18]);
#pragma unroll
            for (int q = 0; q < 5; ++q) store8_bf16(smem + G.off(0), t, 24 + 8 * q, 64, x + 6 + 8 * q);
        }
    };
    // the first tile's input; every later tile's is built during the previous
    // tile's bias round (H_0 is free once layer 0's MMAs are done)
    if ((int64_t)blockIdx.x < n_tiles) {
        build_h0(cur);
        ok = sync_all(true);
    }

    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t m = (int64_t)cur.m;
        const bool valid = cur.valid;
        const int pidx = cur.pidx;
        const uint32_t act2 = load_act(tile + 2 * (int64_t)gridDim.x);
        const RowIn nxt = load_row(act1);
        // ---------------- forward recompute
        for (int l = 0; l < L && ok; ++l) {
            const int K = G.kin(l), Np = G.np(l);
            bool mine = begin_use();
            ++use;
            if (tid < 32) {
                const uint32_t idesc = tc::idesc_bf16(TC_ROWS, Np, false, false);
                const uint32_t sbo = (uint32_t)(K / 8) * 128u;
                const tc::Desc2 da = tc::desc2(tc::smem_u32(smem + G.off(l)), 128, sbo);
                const tc::Desc2 dw = tc::desc2(((use - 1) & 1) ? wslot1 : wslot0, 128, sbo);
#pragma unroll
                for (int k = 0; k < TC_MAXW / 16; ++k)
                    if (k < K / 16) tc::mma_bf16_w(tmem, da, k * 256, dw, k * 256, idesc, k > 0 ? 1u : 0u, lane);
                tc::mma_commit_w(bar_m, lane);
            }
            mine = wait_mma() && mine;
            release_use(use - 1);
            const float* bl = sbias + G.bias(l);
            if (l < L - 1) {
                const int N = 128;
                if (N == 128) {
                    const int c0 = wg * 64;
                    float v[64];
                    tc::tmem_ld64(tmem + lane_off + c0, v);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        store8_bias_relu(smem + G.off(l + 1), t, c0 + 8 * q, N, v + 8 * q, bl + c0 + 8 * q);
                } else {
                    for (int c0 = wg * (N / 2); c0 < (wg + 1) * (N / 2); c0 += 32) {
                        float v[32];
                        tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            store8_bias_relu(smem + G.off(l + 1), t, c0 + 8 * q, N, v + 8 * q, bl + c0 + 8 * q);
                    }
                }
            } else if (wg == 0) {
                // heads and their gradient: dZ_L (padded to 16 columns), db_{L-1}
                float v[16];
                tc::tmem_ld16(tmem + lane_off, v);
                float dz[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) dz[j] = 0.f;
                if (valid) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float s = 1.f / (1.f + expf(-(v[c] + bl[c])));
                        dz[c] = cur.up[c] * s * (1.f - s);
                    }
                    dz[3] = (v[3] + bl[3]) > 0.f ? cur.up[3] : 0.f;
                }
                uint4 q0, q1;
                q0.x = tc::pack_bf16(dz[0], dz[1]); q0.y = tc::pack_bf16(dz[2], dz[3]);
                q0.z = tc::pack_bf16(dz[4], dz[5]); q0.w = tc::pack_bf16(dz[6], dz[7]);
                q1.x = tc::pack_bf16(dz[8], dz[9]); q1.y = tc::pack_bf16(dz[10], dz[11]);
                q1.z = tc::pack_bf16(dz[12], dz[13]); q1.w = tc::pack_bf16(dz[14], dz[15]);
                store8_packed(sDZL, t, 0, 16, q0);
                store8_packed(sDZL, t, 8, 16, q1);
                // db_{L-1} = sum over rows of bf16(dZ_L)
                float r4[4] = {tc::bf16_lo(q0.x), tc::bf16_hi(q0.x), tc::bf16_lo(q0.y), tc::bf16_hi(q0.y)};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float a = r4[c];
#pragma unroll
                    for (int off = 16; off >= 1; off >>= 1) a += __shfl_xor_sync(SSSGS_FULL, a, off);
                    if (lane == 0) atomicAdd(&sdbL[c], a);
                }
            }
            ok = sync_all(mine);
        }
        // ---------------- backward
        for (int l = L - 1; l >= 0 && ok; --l) {
            const int Kin = G.kin(l);
            const bool last = (l == L - 1);
            const bool hidden = l >= 1 && l <= L - 2;
            const int Nout = last ? 16 : 128;        // dZ_{l+1} columns (padded for the last layer)
            const uint8_t* dzbuf = last ? sDZL : smem + G.off(l + 1);
            const uint32_t dz_addr = tc::smem_u32(dzbuf);
            const uint32_t dz_sr = (uint32_t)(Nout / 8) * 128u;
            const uint32_t h_addr = tc::smem_u32(smem + G.off(l));
            const uint32_t h_sr = (uint32_t)(Kin / 8) * 128u;
            bool mine = begin_use();
            ++use;
            const uint32_t w_addr = tc::smem_u32(smem + (((use - 1) & 1) ? T.offW[1] : T.offW[0]));
            const uint32_t w_sr = (uint32_t)(Kin / 8) * 128u;    // weight image: rows = outputs, C = Kin
            // dH_l in one 128-column round on the hidden layers (their bias
            // gradients wait for the tile's last round, so TMEM columns
            // [0, 128) are free); the last layer (dW^T at columns [64, 80))
            // takes two 64-column halves, layer 0 has 64 columns
            const int halves = (!hidden && Kin > 64) ? 2 : 1;
            const int ncols_round = hidden ? 128 : (Kin > 64 ? 64 : Kin);
            if (tid < 32) {
                // per-tile or accumulated weight gradient, K' = 128 rows
                const tc::Desc2 dzm = tc::desc2(dz_addr, dz_sr, 128);    // dZ, MN-major (K = rows)
                const tc::Desc2 hm = tc::desc2(h_addr, h_sr, 128);       // H_l, MN-major (K = rows)
                if (hidden) {
                    const uint32_t idesc = tc::idesc_bf16(TC_ROWS, Kin, true, true);
#pragma unroll
                    for (int k = 0; k < TC_ROWS / 16; ++k)
                        tc::mma_bf16_w(tmem + G.colw(l), dzm, k * 2 * dz_sr, hm, k * 2 * h_sr, idesc,
                                       (any_tile || k > 0) ? 1u : 0u, lane);
                } else if (last) {      // dW_{L-1}^T = H_{L-1}^T dZ_L  -> [Kin x 16]
                    const uint32_t idesc = tc::idesc_bf16(TC_ROWS, 16, true, true);
#pragma unroll
                    for (int k = 0; k < TC_ROWS / 16; ++k)
                        tc::mma_bf16_w(tmem + 64, hm, k * 2 * h_sr, dzm, k * 2 * dz_sr, idesc, k > 0 ? 1u : 0u, lane);
                } else {                // l == 0: dW_0 = dZ_1^T H_0 -> [w1 x Kin]
                    const uint32_t idesc = tc::idesc_bf16(TC_ROWS, Kin, true, true);
#pragma unroll
                    for (int k = 0; k < TC_ROWS / 16; ++k)
                        tc::mma_bf16_w(tmem + 64, dzm, k * 2 * dz_sr, hm, k * 2 * h_sr, idesc, k > 0 ? 1u : 0u, lane);
                }
                // dH_l (hidden: all 128 columns; else the first half): dZ_{l+1} W_l
                const uint32_t idesc = tc::idesc_bf16(TC_ROWS, ncols_round, false, true);
                const tc::Desc2 dzk = tc::desc2(dz_addr, 128, dz_sr);    // dZ, K-major (K = outputs)
                const tc::Desc2 wm = tc::desc2(w_addr, w_sr, 128);       // W_l, MN-major (K = outputs)
#pragma unroll
                for (int k = 0; k < TC_MAXW / 16; ++k)
                    if (k < Nout / 16)
                        tc::mma_bf16_w(tmem, dzk, k * 256, wm, k * 2 * w_sr, idesc, k > 0 ? 1u : 0u, lane);
                tc::mma_commit_w(bar_m, lane);
            }
            mine = wait_mma() && mine;
            if (halves == 1) release_use(use - 1);
            // epilogue of the per-tile weight gradients
            if (last) {
                if (wg == 0) {
                    float v[16];
                    tc::tmem_ld16(tmem + lane_off + 64, v);
#pragma unroll
                    for (int c = 0; c < 4; ++c) accL[c] += v[c];
                }
            } else if (l == 0) {
                float v[32];
                tc::tmem_ld32(tmem + lane_off + 64 + 32 * wg, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc0[j] += v[j];
            }
            for (int h = 0; h < 2; ++h) {
                if (h == 1) {
                    if (halves == 1) break;
                    mine = sync_all(mine);
                    if (tid < 32) {
                        tc::fence_after();
                        const uint32_t idesc = tc::idesc_bf16(TC_ROWS, 64, false, true);
                        const tc::Desc2 dzk = tc::desc2(dz_addr, 128, dz_sr);
                        const tc::Desc2 wm = tc::desc2(w_addr + 8 * 128, w_sr, 128);
#pragma unroll
                        for (int k = 0; k < TC_MAXW / 16; ++k)
                            if (k < Nout / 16)
                                tc::mma_bf16_w(tmem, dzk, k * 256, wm, k * 2 * w_sr, idesc, k > 0 ? 1u : 0u, lane);
                        tc::mma_commit_w(bar_m, lane);
                    }
                    mine = wait_mma() && mine;
                    release_use(use - 1);
                }
                const int cbase = 64 * h;
                if (l > 0) {
                    // dZ_l = bf16(dH_l * [H_l > 0]) in place over H_l; warpgroup wg
                    // takes 32-column chunks wg, wg + 2, ... of the columns this MMA pass formed
                    uint8_t* hb = smem + G.off(l);
                    for (int c0 = 32 * wg; c0 < ncols_round; c0 += 64) {
                        float v[32];
                        tc::tmem_ld32(tmem + lane_off + c0, v);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int c = cbase + c0 + 8 * q;
                            const uint4 hq = load8_packed(hb, t, c, Kin);
                            uint4 o;
                            o.x = tc::pack_bf16_mask(v[8 * q + 0], v[8 * q + 1], hq.x);
                            o.y = tc::pack_bf16_mask(v[8 * q + 2], v[8 * q + 3], hq.y);
                            o.z = tc::pack_bf16_mask(v[8 * q + 4], v[8 * q + 5], hq.z);
                            o.w = tc::pack_bf16_mask(v[8 * q + 6], v[8 * q + 7], hq.w);
                            store8_packed(hb, t, c, Kin, o);
                        }
                    }
                } else {
                    // network-input gradient (64 columns) -> (d mu, d n, d v), split
                    // like the input: warpgroup 0 keeps the Fourier part of
                    // frequencies 0..2, warpgroup 1 leaves the rest in s_dx.
                    float dX[64];
                    tc::tmem_ld64(tmem + lane_off, dX);
                    if (wg == 0) {
                        dmu_a[0] = dmu_a[1] = dmu_a[2] = 0.f;
                        if (valid) pe6_fourier_bwd<0, 3>(cur.q.mu, dX, dmu_a);
                    } else if (valid) {
                        float dm[3] = {0.f, 0.f, 0.f}, dx[7];
                        pe6_fourier_bwd<3, 6>(cur.q.mu, dX + 18, dm);
                        pe6_direct_bwd(pairs[pidx], cur.q.mu, dX + 36, dx);
                        dx[0] += dm[0]; dx[1] += dm[1]; dx[2] += dm[2];
#pragma unroll
                        for (int k = 0; k < 7; ++k) s_dx[k * TC_ROWS + t] = dx[k];
                    }
                }
            }
            mine = sync_all(mine);
            if (l == 0) {
                if (wg == 0 && valid) {   // combine the two halves of the input gradient
#pragma unroll
                    for (int k = 0; k < 7; ++k)
                        dx_items[SSSGS_DX * m + k] = s_dx[k * TC_ROWS + t] + (k < 3 ? dmu_a[k] : 0.f);
                    // columns 7..13 (no q, log_s inputs) stay as cleared
                }
                // the tile's bias gradients of layers 0 .. L-2 in one round:
                // db_j = dZ_{j+1}^T 1 (dZ_{j+1} stays where H_{j+1} was) into
                // TMEM columns [16 j, 16 j + 16)
                if (tid < 32) {
                    tc::fence_after();
                    const uint32_t idesc = tc::idesc_bf16(TC_ROWS, 16, true, false);
                    const tc::Desc2 on = tc::desc2(ones, 128, (TC_ROWS / 8) * 128);
                    for (int j = 0; j <= L - 2; ++j) {
                        const tc::Desc2 dzm = tc::desc2(tc::smem_u32(smem + G.off(j + 1)), 2048, 128);
#pragma unroll
                        for (int k = 0; k < TC_ROWS / 16; ++k)
                            tc::mma_bf16_w(tmem + 16 * j, dzm, k * 2 * 2048, on, k * 256, idesc, k > 0 ? 1u : 0u, lane);
                    }
                    tc::mma_commit_w(bar_m, lane);
                }
                if (tile + gridDim.x < n_tiles) build_h0(nxt);   // next tile's input, under the bias MMAs
                mine = wait_mma() && mine;
                if (wg == 0) {
#pragma unroll
                    for (int j = 0; j < SSSGS_MAX_LAYERS - 1; ++j)
                        if (j <= L - 2) {
                            float v[16];
                            tc::tmem_ld16(tmem + lane_off + 16 * j, v);
                            dbacc[j] += v[0];
                        }
                }
                mine = sync_all(mine);
            }
            ok = mine;
        }
        any_tile = true;
        cur = nxt;
        act1 = act2;
    }
    // copies still in flight after a failed wait: let them land (bounded)
    if (tid == 0)
        for (uint32_t u = use; u < fetched; ++u) tc::mbar_wait((u & 1) ? bar_w1 : bar_w0, (u >> 1) & 1u);
    if (!ok) {
        if (tid == 0 && status) atomicOr(status, SSSGS_STATUS_TIMEOUT);
    } else if (any_tile) {
        // flush: dW of hidden layers from TMEM, dW_0 / dW_{L-1} / db from registers
        // (layer indices unrolled, so no parameter table is indexed at run time)
#pragma unroll
        for (int l = 1; l < SSSGS_MAX_LAYERS - 1; ++l) {
            if (l > L - 2) break;
            for (int c0 = 32 * wg; c0 < 128; c0 += 64) {
                float v[32];
                tc::tmem_ld32(tmem + lane_off + G.colw(l) + c0, v);
                for (int j = 0; j < 32; ++j) atomicAdd(&gr.W[l][t * 128 + c0 + j], v[j]);
            }
        }
        for (int j = 0; j < 32; ++j) atomicAdd(&gr.W[0][t * 64 + 32 * wg + j], acc0[j]);
        float* dWL = gr.W[0];
        float* dbL = gr.b[0];
#pragma unroll
        for (int l = 1; l < SSSGS_MAX_LAYERS; ++l)
            if (l == L - 1) {
                dWL = gr.W[l];
                dbL = gr.b[l];
            }
        if (wg == 0) {
            for (int c = 0; c < 4; ++c) atomicAdd(&dWL[c * 128 + t], accL[c]);
#pragma unroll
            for (int j = 0; j < SSSGS_MAX_LAYERS; ++j)
                if (j <= L - 2 && gr.b[j]) atomicAdd(&gr.b[j][t], dbacc[j]);
        }
        __syncthreads();
        if (dbL && tid < 4) atomicAdd(&dbL[tid], sdbL[tid]);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_dealloc(tmem, 512);
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

int sm_count() { return device_sm_count(); }
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
    int grid = (int)std::min<int64_t>((tiles + TC_FWD_LANES - 1) / TC_FWD_LANES, (int64_t)sm_count());
    k_mlp_fwd_tc<<<grid, TC_FWD_LANES * TC_THREADS, T.total, (cudaStream_t)stream>>>(net, d_pairs, n_pairs, n, *scene, out,
                                                                            d_status);
    sssgs::note_launches(1);
    return launch_status();
}


namespace {
// Backward workspace: BF16 weight images, then the active-row list, the
// per-block counts and offsets, and the active-row count.
struct TcBwdWs {
    size_t img, active, flag, cnt, off, nact, total;
};
TcBwdWs tc_bwd_ws(const TcBwdLayout& T, int64_t n_items) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nb = (size_t)((n_items + ACT_BLOCK - 1) / ACT_BLOCK);
    TcBwdWs w;
    size_t o = 0;
    w.img = o;    o += al(T.gtotal);
    w.active = o; o += al(4 * (size_t)n_items);
    w.flag = o;   o += al((size_t)n_items);
    w.cnt = o;    o += al(4 * nb);
    w.off = o;    o += al(4 * nb);
    w.nact = o;   o += 256;
    w.total = o + 256;    // room to align the base
    return w;
}
}  // namespace

size_t sssgs_mlp_workspace_bytes_tc(const sssgs_mlp* mlp, int64_t n_items) {
    if (!tc_supported(mlp)) return 0;
    return tc_bwd_ws(tc_bwd_layout(to_dev_tc(mlp)), n_items).total;
}

int sssgs_mlp_bwd_tc(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                     const sssgs_scene* scene, const float* dout, int64_t dstride, const sssgs_mlp_grad* grad,
                     float* dx_items, void* workspace, size_t workspace_bytes, int32_t* d_status,
                     sssgs_stream stream) {
    if (!tc_supported(mlp)) return SSSGS_ERR_UNSUPPORTED;
    MlpDev net = to_dev_tc(mlp);
    TcBwdLayout T = tc_bwd_layout(net);
    if (T.colW[0] > 512 || T.total > 227 * 1024 || net.w[1] != 128) return SSSGS_ERR_UNSUPPORTED;
    for (int l = 1; l < net.L; ++l)
        if (net.w[l] != 128) return SSSGS_ERR_UNSUPPORTED;
    const BwdGeom G{net.L};
    for (int l = 0; l < net.L; ++l)
        if (G.kin(l) != net.w[l] || G.np(l) != T.Np[l] || G.off(l) != T.offH[l] || G.off(l) != T.gW[l] ||
            G.wbytes(l) != T.wbytes[l] || G.bias(l) != T.biasOff[l] ||
            (l >= 1 && l <= net.L - 2 && G.colw(l) != T.colW[l]))
            return SSSGS_ERR_UNSUPPORTED;
    int64_t n = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    if (n == 0) return SSSGS_OK;
    if (n >= ((int64_t)1 << 32)) return SSSGS_ERR_INVALID_ARG;    // row list holds u32 item ids
    const TcBwdWs W = tc_bwd_ws(T, n);
    if (!workspace || workspace_bytes < W.total) return SSSGS_ERR_WORKSPACE;
    uint8_t* base = (uint8_t*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    uint8_t* gimg = base + W.img;
    uint32_t* active = (uint32_t*)(base + W.active);
    uint8_t* flag = base + W.flag;
    uint32_t* cnt = (uint32_t*)(base + W.cnt);
    uint32_t* off = (uint32_t*)(base + W.off);
    uint32_t* nact = (uint32_t*)(base + W.nact);
    cudaStream_t st = (cudaStream_t)stream;
    k_mlp_weights_bf16<<<dim3(32, net.L), 256, 0, st>>>(net, T, gimg);
    sssgs::note_launches(1 + launch_active_rows(dout, dstride, n, flag, cnt, off, nact, active, dx_items, st));
    cudaFuncSetAttribute(k_mlp_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T.total);
    int64_t tiles = (n + TC_ROWS - 1) / TC_ROWS;
    int grid = (int)std::min<int64_t>(tiles, (int64_t)sm_count());
    k_mlp_bwd_tc<<<grid, 2 * TC_THREADS, T.total, st>>>(net, T, gimg, d_pairs, n_pairs, n, *scene, dout, dstride,
                                                    *grad, dx_items, active, nact, d_status);
    sssgs::note_launches(1);
    return launch_status();
}
