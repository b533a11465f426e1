// Joint SSS-residual / incident-light network f_Theta (Eq. 6) on CUDA cores, FP32.
//
// Every (pair, Gaussian) item is one row. Its input is built in the kernel
// from the Gaussian's mean (Fourier-encoded in the PE6 form, as the paper
// does for mu), normal and visibility, and the pair's camera and light
// (w_out, w_in, light distance). A CTA runs a 64-row tile through all layers
// with activations and the current layer's weights in shared memory and a
// 4 x (N/16) register micro-tile per thread. Heads: sigmoid -> L_SSS (rgb),
// ReLU -> L_in (Appendix E "Network").
//
// The paper's network (SSSGS_MLP_PAPER) runs on the same chain machinery as
// five chain layers built while staging: the three trunk layers; a 32 -> 64
// layer holding the incident hidden units (Leaky-ReLU, columns 0..31) next to
// the SSS logits (identity, columns 32..34); and a final layer that copies the
// three logits through (weights exactly 1 and 0, so the copy is exact) and
// forms the incident output in column 3. Gradients of the packed layers are
// scattered back to the six matrices.
//
// Backward, per chunk of rows: phase A recomputes the forward of a 32-row tile,
// back-propagates to every layer's pre-activation gradient dZ and to the
// network input (mapped to d mu, d n, d v per item), storing H and dZ in the
// workspace; phase B reduces dW = sum_rows dZ^T H and db = sum_rows dZ with a
// register micro-tile per thread and one atomic per weight per CTA.
#include <algorithm>

#include "mlp_common.cuh"

namespace sssgs {

constexpr int MLP_THREADS = 256;
constexpr int MLP_MAXW = 128;
constexpr int MLP_LDA = MLP_MAXW + 4;
constexpr int FWD_ROWS = 64;
constexpr int BWD_ROWS = 32;
constexpr int64_t MLP_CHUNK = 131072;


// Activation codes of a chain layer's output: 0 none, 1 ReLU, 2 Leaky-ReLU,
// 3 Leaky-ReLU on columns < 32 and none above (the paper network's packed
// head layer).
__device__ __forceinline__ float activate(float v, int act, int col) {
    if (act == 1) return fmaxf(v, 0.f);
    if (act == 2 || (act == 3 && col < 32)) return v > 0.f ? v : kLReluSlope * v;
    return v;
}

// Backward of activation `act` at an output whose activated value is h (same
// sign as the pre-activation): dh -> dz.
__device__ __forceinline__ float activate_bwd(float dh, float h, int act, int col) {
    if (act == 1) return h > 0.f ? dh : 0.f;
    if (act == 2 || (act == 3 && col < 32)) return h > 0.f ? dh : kLReluSlope * dh;
    return dh;
}

// out[r][j] = act(bias[j] + sum_i in[r][i] * M[i*J + j]) over a ROWS-row tile;
// with mask != null, out = activate_bwd(out, mask[r][j], mact). J multiple of 16.
template <int ROWS, int CJ>
__device__ __forceinline__ void tile_gemm16(const float* in, int I, const float* M, const float* bias, float* out,
                                            int act, const float* mask, int mact) {
    constexpr int J = 16 * CJ;
    constexpr int RR = ROWS / 16;
    const int t = threadIdx.x, rg = t >> 4, cg = t & 15;
    float acc[RR][CJ];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int c = 0; c < CJ; ++c) acc[r][c] = bias ? bias[cg * CJ + c] : 0.f;
    for (int i = 0; i < I; ++i) {
        float a[RR], w[CJ];
#pragma unroll
        for (int r = 0; r < RR; ++r) a[r] = in[(rg * RR + r) * MLP_LDA + i];
#pragma unroll
        for (int c = 0; c < CJ; ++c) w[c] = M[i * J + cg * CJ + c];
#pragma unroll
        for (int r = 0; r < RR; ++r)
#pragma unroll
            for (int c = 0; c < CJ; ++c) acc[r][c] = fmaf(a[r], w[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int c = 0; c < CJ; ++c) {
            const int row = rg * RR + r, col = cg * CJ + c;
            float v = activate(acc[r][c], act, col);
            if (mask) v = activate_bwd(v, mask[row * MLP_LDA + col], mact, col);
            out[row * MLP_LDA + col] = v;
        }
}

// Generic (any J) variant: one output per thread-iteration.
template <int ROWS>
__device__ __forceinline__ void tile_gemm_any(const float* in, int I, const float* M, int J, const float* bias,
                                              float* out, int act, const float* mask, int mact) {
    for (int o = threadIdx.x; o < ROWS * J; o += MLP_THREADS) {
        const int row = o / J, col = o % J;
        float v = bias ? bias[col] : 0.f;
        for (int i = 0; i < I; ++i) v = fmaf(in[row * MLP_LDA + i], M[i * J + col], v);
        v = activate(v, act, col);
        if (mask) v = activate_bwd(v, mask[row * MLP_LDA + col], mact, col);
        out[row * MLP_LDA + col] = v;
    }
}

template <int ROWS>
__device__ __forceinline__ void tile_gemm(const float* in, int I, const float* M, int J, const float* bias,
                                          float* out, int act, const float* mask, int mact = 1) {
    switch (J) {   // every multiple of 16 up to MLP_MAXW has its register-tiled form
        case 16: tile_gemm16<ROWS, 1>(in, I, M, bias, out, act, mask, mact); break;
        case 32: tile_gemm16<ROWS, 2>(in, I, M, bias, out, act, mask, mact); break;
        case 48: tile_gemm16<ROWS, 3>(in, I, M, bias, out, act, mask, mact); break;
        case 64: tile_gemm16<ROWS, 4>(in, I, M, bias, out, act, mask, mact); break;
        case 80: tile_gemm16<ROWS, 5>(in, I, M, bias, out, act, mask, mact); break;
        case 96: tile_gemm16<ROWS, 6>(in, I, M, bias, out, act, mask, mact); break;
        case 112: tile_gemm16<ROWS, 7>(in, I, M, bias, out, act, mask, mact); break;
        case 128: tile_gemm16<ROWS, 8>(in, I, M, bias, out, act, mask, mact); break;
        default: tile_gemm_any<ROWS>(in, I, M, J, bias, out, act, mask, mact); break;
    }
}

// Activation code of chain layer l's output (the last layer feeds the heads).
__device__ __forceinline__ int layer_act(const MlpDev& net, int l) {
    if (l == net.L - 1) return 0;
    if (net.kind != SSSGS_MLP_PAPER) return 1;
    return l < 3 ? 2 : 3;
}

// Weight (n, k) and bias n of chain layer l (N x K): the user's matrices, or
// for the paper network the packed head layers described above.
__device__ __forceinline__ float chain_w(const MlpDev& net, int l, int n, int k, int K) {
    if (net.kind != SSSGS_MLP_PAPER || l < 3) return net.W[l][n * K + k];
    if (l == 3) return n < 32 ? net.W[3][n * 32 + k] : (n < 35 ? net.W[5][(n - 32) * 32 + k] : 0.f);
    if (n < 3) return k == 32 + n ? 1.f : 0.f;
    return k < 32 ? net.W[4][k] : 0.f;
}
__device__ __forceinline__ float chain_b(const MlpDev& net, int l, int n) {
    if (net.kind != SSSGS_MLP_PAPER || l < 3) return net.b[l][n];
    if (l == 3) return n < 32 ? net.b[3][n] : (n < 35 ? net.b[5][n - 32] : 0.f);
    return n == 3 ? net.b[4][0] : 0.f;
}
// Where the gradient of chain weight (n, k) / bias n goes (null: a fixed entry).
__device__ __forceinline__ float* chain_dw(const MlpDev& net, const sssgs_mlp_grad& gr, int l, int n, int k, int K) {
    if (net.kind != SSSGS_MLP_PAPER || l < 3) return gr.W[l] + n * K + k;
    if (l == 3) return n < 32 ? gr.W[3] + n * 32 + k : (n < 35 ? gr.W[5] + (n - 32) * 32 + k : nullptr);
    return (n == 3 && k < 32) ? gr.W[4] + k : nullptr;
}
__device__ __forceinline__ float* chain_db(const MlpDev& net, const sssgs_mlp_grad& gr, int l, int n) {
    if (net.kind != SSSGS_MLP_PAPER || l < 3) return gr.b[l] ? gr.b[l] + n : nullptr;
    if (l == 3) return n < 32 ? (gr.b[3] ? gr.b[3] + n : nullptr) : (n < 35 && gr.b[5] ? gr.b[5] + n - 32 : nullptr);
    return (n == 3 && gr.b[4]) ? gr.b[4] : nullptr;
}

// Stage chain layer l's weights in shared memory: transposed (K x N, for
// H W^T) or as stored (N x K, for dZ W).
__device__ __forceinline__ void stage_weights(const MlpDev& net, int l, int N, int K, bool transpose, float* sW) {
    for (int i = threadIdx.x; i < N * K; i += MLP_THREADS) {
        const int n = i / K, k = i - n * K;
        const float v = chain_w(net, l, n, k, K);
        if (transpose) sW[k * N + n] = v; else sW[i] = v;
    }
}

__global__ void __launch_bounds__(MLP_THREADS) k_mlp_fwd(MlpDev net, const sssgs_pair* __restrict__ pairs, int n_pairs,
                                                         int64_t n_items, sssgs_scene sc, float* __restrict__ out) {
    extern __shared__ float smem[];
    float* sA = smem;
    float* sB = sA + FWD_ROWS * MLP_LDA;
    float* sW = sB + FWD_ROWS * MLP_LDA;
    float* sb = sW + MLP_MAXW * MLP_MAXW;
    const int64_t n_tiles = (n_items + FWD_ROWS - 1) / FWD_ROWS;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t row0 = tile * FWD_ROWS;
        if (threadIdx.x < FWD_ROWS) {
            const int64_t m = row0 + threadIdx.x;
            float* x = sA + threadIdx.x * MLP_LDA;
            if (m < n_items) {
                const int p = pair_of_item(pairs, n_pairs, m);
                const sssgs_pair& P = pairs[p];
                build_input(net, P, sc, P.g_begin + (m - P.item_offset), m, x);
            } else {
                for (int k = 0; k < net.w[0]; ++k) x[k] = 0.f;
            }
        }
        float* cur = sA;
        float* nxt = sB;
        for (int l = 0; l < net.L; ++l) {
            const int K = net.w[l], N = net.w[l + 1];
            __syncthreads();
            stage_weights(net, l, N, K, true, sW);
            for (int i = threadIdx.x; i < N; i += MLP_THREADS) sb[i] = chain_b(net, l, i);
            __syncthreads();
            tile_gemm<FWD_ROWS>(cur, K, sW, N, sb, nxt, layer_act(net, l), nullptr);
            float* t = cur; cur = nxt; nxt = t;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < FWD_ROWS * 4; o += MLP_THREADS) {
            const int r = o >> 2, c = o & 3;
            const int64_t m = row0 + r;
            if (m >= n_items) continue;
            const float y = cur[r * MLP_LDA + c];
            out[4 * m + c] = c < 3 ? 1.f / (1.f + expf(-y)) : fmaxf(y, 0.f);
        }
        __syncthreads();   // the next tile overwrites the buffers read above
    }
}

// Phase A: recompute, back-propagate, store H_l and dZ_{l+1} for the chunk.
__global__ void __launch_bounds__(MLP_THREADS) k_mlp_bwd_a(MlpDev net, const sssgs_pair* __restrict__ pairs,
                                                           int n_pairs, int64_t row_begin, int64_t rows,
                                                           sssgs_scene sc, const float* __restrict__ dout,
                                                           int64_t dstride, float* __restrict__ ws, int64_t chunk,
                                                           float* __restrict__ dx_items) {
    extern __shared__ float smem[];
    float* sH = smem;                                          // [L][BWD_ROWS][LDA]
    float* sD0 = sH + net.L * BWD_ROWS * MLP_LDA;
    float* sD1 = sD0 + BWD_ROWS * MLP_LDA;
    float* sW = sD1 + BWD_ROWS * MLP_LDA;
    float* sb = sW + MLP_MAXW * MLP_MAXW;
    // workspace offsets (floats): H_l then dZ_{l+1}, each chunk x width
    int64_t offH[SSSGS_MAX_LAYERS], offD[SSSGS_MAX_LAYERS];
    {
        int64_t o = 0;
        for (int l = 0; l < net.L; ++l) { offH[l] = o; o += chunk * net.w[l]; }
        for (int l = 0; l < net.L; ++l) { offD[l] = o; o += chunk * net.w[l + 1]; }
    }
    const int64_t n_tiles = (rows + BWD_ROWS - 1) / BWD_ROWS;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t r0 = tile * BWD_ROWS;           // row within the chunk
        if (threadIdx.x < BWD_ROWS) {
            const int64_t m = row_begin + r0 + threadIdx.x;
            float* x = sH + threadIdx.x * MLP_LDA;
            if (r0 + threadIdx.x < rows) {
                const int p = pair_of_item(pairs, n_pairs, m);
                const sssgs_pair& P = pairs[p];
                build_input(net, P, sc, P.g_begin + (m - P.item_offset), m, x);
            } else {
                for (int k = 0; k < net.w[0]; ++k) x[k] = 0.f;
            }
        }
        // forward, keeping every layer input
        for (int l = 0; l < net.L; ++l) {
            const int K = net.w[l], N = net.w[l + 1];
            __syncthreads();
            stage_weights(net, l, N, K, true, sW);
            for (int i = threadIdx.x; i < N; i += MLP_THREADS) sb[i] = chain_b(net, l, i);
            __syncthreads();
            float* dst = (l < net.L - 1) ? sH + (l + 1) * BWD_ROWS * MLP_LDA : sD0;
            tile_gemm<BWD_ROWS>(sH + l * BWD_ROWS * MLP_LDA, K, sW, N, sb, dst, layer_act(net, l), nullptr);
        }
        __syncthreads();
        // heads: dZ_L from dL/d(L_SSS, L_in)
        for (int o = threadIdx.x; o < BWD_ROWS * 4; o += MLP_THREADS) {
            const int r = o >> 2, c = o & 3;
            const float y = sD0[r * MLP_LDA + c];
            float d = 0.f;
            if (r0 + r < rows) {
                const float up = dout[dstride * (row_begin + r0 + r) + c];
                if (c < 3) {
                    const float s = 1.f / (1.f + expf(-y));
                    d = up * s * (1.f - s);
                } else {
                    d = y > 0.f ? up : 0.f;
                }
            }
            sD0[r * MLP_LDA + c] = d;
        }
        float* dcur = sD0;
        float* dnxt = sD1;
        for (int l = net.L - 1; l >= 0; --l) {
            const int K = net.w[l], N = net.w[l + 1];
            __syncthreads();
            // store H_l and dZ_{l+1} rows of this tile
            for (int o = threadIdx.x; o < BWD_ROWS * K; o += MLP_THREADS) {
                const int r = o / K, k = o - r * K;
                if (r0 + r < rows) ws[offH[l] + (r0 + r) * K + k] = sH[(l * BWD_ROWS + r) * MLP_LDA + k];
            }
            for (int o = threadIdx.x; o < BWD_ROWS * N; o += MLP_THREADS) {
                const int r = o / N, n = o - r * N;
                if (r0 + r < rows) ws[offD[l] + (r0 + r) * N + n] = dcur[r * MLP_LDA + n];
            }
            stage_weights(net, l, N, K, false, sW);
            __syncthreads();
            // dH_l = dZ_{l+1} W_l ; dZ_l = dH_l * act'(H_l) (l > 0)
            tile_gemm<BWD_ROWS>(dcur, N, sW, K, nullptr, dnxt, 0,
                                l > 0 ? sH + l * BWD_ROWS * MLP_LDA : nullptr, l > 0 ? layer_act(net, l - 1) : 1);
            float* t = dcur; dcur = dnxt; dnxt = t;
        }
        __syncthreads();
        if (threadIdx.x < BWD_ROWS && r0 + threadIdx.x < rows) {
            const int64_t m = row_begin + r0 + threadIdx.x;
            const int p = pair_of_item(pairs, n_pairs, m);
            const sssgs_pair& P = pairs[p];
            float dx[SSSGS_DX];
            input_backward(net, P, sc, P.g_begin + (m - P.item_offset), dcur + threadIdx.x * MLP_LDA, dx);
            for (int k = 0; k < SSSGS_DX; ++k) dx_items[(int64_t)SSSGS_DX * m + k] = dx[k];
        }
        __syncthreads();   // the next tile overwrites the buffers read above
    }
}

// Phase B: dW_l += sum_rows dZ_{l+1}^T H_l, db_l += sum_rows dZ_{l+1}.
template <int TN, int TK>
__device__ __forceinline__ void reduce_dw16(const float* sD, const float* sHt, int rows_here, int N, int K,
                                            const MlpDev& net, const sssgs_mlp_grad& gr, int l) {
    const int t = threadIdx.x, ng = t >> 4, kg = t & 15;
    float acc[TN][TK];
#pragma unroll
    for (int a = 0; a < TN; ++a)
#pragma unroll
        for (int b = 0; b < TK; ++b) acc[a][b] = 0.f;
    for (int r = 0; r < rows_here; ++r) {
        float d[TN], h[TK];
#pragma unroll
        for (int a = 0; a < TN; ++a) d[a] = sD[r * MLP_LDA + ng * TN + a];
#pragma unroll
        for (int b = 0; b < TK; ++b) h[b] = sHt[r * MLP_LDA + kg * TK + b];
#pragma unroll
        for (int a = 0; a < TN; ++a)
#pragma unroll
            for (int b = 0; b < TK; ++b) acc[a][b] = fmaf(d[a], h[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < TN; ++a)
#pragma unroll
        for (int b = 0; b < TK; ++b) {
            float* dst = chain_dw(net, gr, l, ng * TN + a, kg * TK + b, K);
            if (dst) atomicAdd(dst, acc[a][b]);
        }
}

template <int TN>
__device__ __forceinline__ void reduce_dw_tk(const float* sD, const float* sH, int rows_here, int N, int K,
                                             const MlpDev& net, const sssgs_mlp_grad& gr, int l) {
    switch (K / 16) {   // K is a multiple of 16 in 16..MLP_MAXW here (tiled layers)
        case 1: reduce_dw16<TN, 1>(sD, sH, rows_here, N, K, net, gr, l); break;
        case 2: reduce_dw16<TN, 2>(sD, sH, rows_here, N, K, net, gr, l); break;
        case 3: reduce_dw16<TN, 3>(sD, sH, rows_here, N, K, net, gr, l); break;
        case 4: reduce_dw16<TN, 4>(sD, sH, rows_here, N, K, net, gr, l); break;
        case 5: reduce_dw16<TN, 5>(sD, sH, rows_here, N, K, net, gr, l); break;
        case 6: reduce_dw16<TN, 6>(sD, sH, rows_here, N, K, net, gr, l); break;
        case 7: reduce_dw16<TN, 7>(sD, sH, rows_here, N, K, net, gr, l); break;
        default: reduce_dw16<TN, 8>(sD, sH, rows_here, N, K, net, gr, l); break;
    }
}

__global__ void __launch_bounds__(MLP_THREADS) k_mlp_bwd_b(MlpDev net, int64_t rows, const float* __restrict__ ws,
                                                           int64_t chunk, sssgs_mlp_grad gr) {
    extern __shared__ float smem[];
    float* sD = smem;                                   // [32][LDA]
    float* sHs = sD + 32 * MLP_LDA;                     // [32][LDA]
    const int l = blockIdx.y;
    const int K = net.w[l], N = net.w[l + 1];
    int64_t offH = 0, offD = 0;
    {
        int64_t o = 0;
        for (int q = 0; q < net.L; ++q) { if (q == l) offH = o; o += chunk * net.w[q]; }
        for (int q = 0; q < net.L; ++q) { if (q == l) offD = o; o += chunk * net.w[q + 1]; }
    }
    const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
    const int64_t rb = (int64_t)blockIdx.x * per;
    const int64_t re = min(rows, rb + per);
    const bool tiled = (N % 16 == 0) && (K % 16 == 0);
    constexpr int GQ = 4;              // generic path: up to GQ * 256 outputs per layer
    float accs[GQ] = {0.f, 0.f, 0.f, 0.f};
    float dbias = 0.f;
    for (int64_t r0 = rb; r0 < re; r0 += 32) {
        const int rows_here = (int)min((int64_t)32, re - r0);
        __syncthreads();
        for (int o = threadIdx.x; o < rows_here * N; o += MLP_THREADS) {
            const int r = o / N, n = o - r * N;
            sD[r * MLP_LDA + n] = ws[offD + (r0 + r) * N + n];
        }
        for (int o = threadIdx.x; o < rows_here * K; o += MLP_THREADS) {
            const int r = o / K, k = o - r * K;
            sHs[r * MLP_LDA + k] = ws[offH + (r0 + r) * K + k];
        }
        __syncthreads();
        if (threadIdx.x < N)
            for (int r = 0; r < rows_here; ++r) dbias += sD[r * MLP_LDA + threadIdx.x];
        if (tiled) {
            switch (N / 16) {
                case 1: reduce_dw_tk<1>(sD, sHs, rows_here, N, K, net, gr, l); break;
                case 2: reduce_dw_tk<2>(sD, sHs, rows_here, N, K, net, gr, l); break;
                case 3: reduce_dw_tk<3>(sD, sHs, rows_here, N, K, net, gr, l); break;
                case 4: reduce_dw_tk<4>(sD, sHs, rows_here, N, K, net, gr, l); break;
                case 5: reduce_dw_tk<5>(sD, sHs, rows_here, N, K, net, gr, l); break;
                case 6: reduce_dw_tk<6>(sD, sHs, rows_here, N, K, net, gr, l); break;
                case 7: reduce_dw_tk<7>(sD, sHs, rows_here, N, K, net, gr, l); break;
                default: reduce_dw_tk<8>(sD, sHs, rows_here, N, K, net, gr, l); break;
            }
        } else {
            for (int q = 0; q < GQ; ++q) {
                const int o = threadIdx.x + q * MLP_THREADS;
                if (o >= N * K) break;
                const int n = o / K, k = o - n * K;
                float v = 0.f;
                for (int r = 0; r < rows_here; ++r) v = fmaf(sD[r * MLP_LDA + n], sHs[r * MLP_LDA + k], v);
                accs[q] += v;
            }
        }
    }
    if (!tiled)
        for (int q = 0; q < GQ; ++q) {
            const int o = threadIdx.x + q * MLP_THREADS;
            if (o >= N * K) break;
            float* dst = chain_dw(net, gr, l, o / K, o % K, K);
            if (dst) atomicAdd(dst, accs[q]);
        }
    if (threadIdx.x < N) {
        float* dst = chain_db(net, gr, l, threadIdx.x);
        if (dst) atomicAdd(dst, dbias);
    }
}

}  // namespace sssgs

using namespace sssgs;

namespace {
bool paper_ok(const sssgs_mlp* m) {
    static const int w[7] = {48, 64, 32, 32, 32, 1, 3};
    if (m->n_layers != 6) return false;
    for (int l = 0; l < 7; ++l)
        if (m->width[l] != w[l]) return false;
    for (int l = 0; l < 6; ++l)
        if (!m->W[l] || !m->b[l]) return false;
    return true;
}

bool mlp_ok(const sssgs_mlp* m) {
    if (!m) return false;
    if (m->kind == SSSGS_MLP_PAPER) return paper_ok(m);
    if (m->n_layers < 2 || m->n_layers > SSSGS_MAX_LAYERS) return false;
    if (m->kind == SSSGS_MLP_BASIC && m->width[0] != 9) return false;
    if (m->kind == SSSGS_MLP_PE6 && m->width[0] != 64) return false;
    if (m->kind != SSSGS_MLP_BASIC && m->kind != SSSGS_MLP_PE6) return false;
    if (m->width[m->n_layers] != 4) return false;
    for (int l = 1; l < m->n_layers; ++l)
        if (m->width[l] < 16 || m->width[l] > MLP_MAXW || m->width[l] % 16) return false;
    for (int l = 0; l < m->n_layers; ++l) {
        if (!m->W[l] || !m->b[l]) return false;
        const bool tiled = m->width[l] % 16 == 0 && m->width[l + 1] % 16 == 0;
        if (!tiled && m->width[l] * m->width[l + 1] > 4 * MLP_THREADS) return false;
    }
    return true;
}

// Device view of the network: the chain the kernels run (for the paper network
// five packed layers 48-64-32-32-64-4) over the user's matrices.
MlpDev to_dev(const sssgs_mlp* m) {
    MlpDev d;
    d.kind = m->kind;
    d.L = m->n_layers;
    for (int l = 0; l <= SSSGS_MAX_LAYERS; ++l) d.w[l] = l <= m->n_layers ? m->width[l] : 0;
    if (m->kind == SSSGS_MLP_PAPER) {
        static const int w[6] = {48, 64, 32, 32, 64, 4};
        d.L = 5;
        for (int l = 0; l <= SSSGS_MAX_LAYERS; ++l) d.w[l] = l < 6 ? w[l] : 0;
    }
    for (int l = 0; l < SSSGS_MAX_LAYERS; ++l) {
        d.W[l] = l < m->n_layers ? m->W[l] : nullptr;
        d.b[l] = l < m->n_layers ? m->b[l] : nullptr;
    }
    return d;
}

int64_t floats_per_row(const sssgs_mlp* m) {
    const MlpDev d = to_dev(m);
    int64_t f = 0;
    for (int l = 0; l < d.L; ++l) f += d.w[l] + d.w[l + 1];
    return f;
}

int num_sms() { return device_sm_count(); }
}  // namespace

int sssgs_mlp_fwd_tc(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                     const sssgs_scene* scene, float* out, int32_t* d_status, sssgs_stream stream);
namespace sssgs {
size_t paper_tc_workspace_bytes(int64_t n_items);
int paper_tc_fwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                 const sssgs_scene* scene, float* out, int32_t* d_status, cudaStream_t st);
int paper_tc_bwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                 const sssgs_scene* scene, const float* dout, int64_t dstride, const sssgs_mlp_grad* grad,
                 float* dx_items, void* workspace, size_t workspace_bytes, int32_t* d_status, cudaStream_t st);
}  // namespace sssgs

extern "C" int sssgs_mlp_fwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                             int n_pairs, const sssgs_scene* scene, float* out, int32_t* d_status,
                             sssgs_stream stream) {
    if (!mlp_ok(mlp) || !h_pairs || !d_pairs || n_pairs <= 0 || !scene || !out) return SSSGS_ERR_INVALID_ARG;
    if (mlp->precision == SSSGS_BF16 && mlp->kind == SSSGS_MLP_PAPER)
        return sssgs::paper_tc_fwd(mlp, h_pairs, d_pairs, n_pairs, scene, out, d_status, (cudaStream_t)stream);
    if (mlp->precision == SSSGS_BF16)
        return sssgs_mlp_fwd_tc(mlp, h_pairs, d_pairs, n_pairs, scene, out, d_status, stream);
    if (mlp->precision != SSSGS_FP32) return SSSGS_ERR_INVALID_ARG;
    int64_t n = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    if (n == 0) return SSSGS_OK;
    size_t sm = (size_t)(2 * FWD_ROWS * MLP_LDA + MLP_MAXW * MLP_MAXW + MLP_MAXW) * 4;
    cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int64_t tiles = (n + FWD_ROWS - 1) / FWD_ROWS;
    int grid = (int)std::min<int64_t>(tiles, (int64_t)num_sms());
    k_mlp_fwd<<<grid, MLP_THREADS, sm, (cudaStream_t)stream>>>(to_dev(mlp), d_pairs, n_pairs, n, *scene, out);
    sssgs::note_launches(1);
    return launch_status();
}

size_t sssgs_mlp_workspace_bytes_tc(const sssgs_mlp* mlp, int64_t n_items);

extern "C" size_t sssgs_mlp_workspace_bytes(const sssgs_mlp* mlp, int64_t n_items) {
    if (!mlp_ok(mlp) || n_items < 0) return 0;
    if (mlp->precision == SSSGS_BF16 && mlp->kind == SSSGS_MLP_PAPER) return sssgs::paper_tc_workspace_bytes(n_items);
    if (mlp->precision == SSSGS_BF16) return sssgs_mlp_workspace_bytes_tc(mlp, n_items);
    int64_t chunk = std::min<int64_t>(std::max<int64_t>(n_items, 1), MLP_CHUNK);
    return (size_t)(chunk * floats_per_row(mlp) * 4) + 256;
}

int sssgs_mlp_bwd_tc(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                     const sssgs_scene* scene, const float* dout, int64_t dstride, const sssgs_mlp_grad* grad,
                     float* dx_items, void* workspace, size_t workspace_bytes, int32_t* d_status,
                     sssgs_stream stream);

extern "C" int sssgs_mlp_bwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                             int n_pairs, const sssgs_scene* scene, const float* drec,
                             const sssgs_mlp_grad* grad, float* dx_items, void* workspace,
                             size_t workspace_bytes, int32_t* d_status, sssgs_stream stream) {
    if (!drec) return SSSGS_ERR_INVALID_ARG;
    return sssgs_mlp_bwd_strided(mlp, h_pairs, d_pairs, n_pairs, scene, drec + 16, SSSGS_REC, grad, dx_items,
                                 workspace, workspace_bytes, d_status, stream);
}

extern "C" int sssgs_mlp_bwd_strided(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                     int n_pairs, const sssgs_scene* scene, const float* dout, int64_t dstride,
                                     const sssgs_mlp_grad* grad, float* dx_items, void* workspace,
                                     size_t workspace_bytes, int32_t* d_status, sssgs_stream stream) {
    if (!mlp_ok(mlp) || !h_pairs || !d_pairs || n_pairs <= 0 || !scene || !dout || !grad || !dx_items)
        return SSSGS_ERR_INVALID_ARG;
    if (dstride < 4 || (dstride & 3) || ((uintptr_t)dout & 15)) return SSSGS_ERR_INVALID_ARG;
    for (int l = 0; l < mlp->n_layers; ++l)
        if (!grad->W[l]) return SSSGS_ERR_INVALID_ARG;
    if (mlp->precision == SSSGS_BF16 && mlp->kind == SSSGS_MLP_PAPER)
        return sssgs::paper_tc_bwd(mlp, h_pairs, d_pairs, n_pairs, scene, dout, dstride, grad, dx_items,
                                   workspace, workspace_bytes, d_status, (cudaStream_t)stream);
    if (mlp->precision == SSSGS_BF16)
        return sssgs_mlp_bwd_tc(mlp, h_pairs, d_pairs, n_pairs, scene, dout, dstride, grad, dx_items, workspace,
                                workspace_bytes, d_status, stream);
    int64_t n = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    if (n == 0) return SSSGS_OK;
    if (!workspace || workspace_bytes < sssgs_mlp_workspace_bytes(mlp, n)) return SSSGS_ERR_WORKSPACE;
    int64_t chunk = std::min<int64_t>(n, MLP_CHUNK);
    float* ws = (float*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    cudaStream_t st = (cudaStream_t)stream;
    MlpDev net = to_dev(mlp);
    size_t smA = (size_t)((net.L + 2) * BWD_ROWS * MLP_LDA + MLP_MAXW * MLP_MAXW + MLP_MAXW) * 4;
    size_t smB = (size_t)(2 * 32 * MLP_LDA) * 4;
    cudaFuncSetAttribute(k_mlp_bwd_a, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smA);
    int sms = num_sms();
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        int64_t rows = std::min(chunk, n - r0);
        int64_t tiles = (rows + BWD_ROWS - 1) / BWD_ROWS;
        int grid = (int)std::min<int64_t>(tiles, (int64_t)sms);
        k_mlp_bwd_a<<<grid, MLP_THREADS, smA, st>>>(net, d_pairs, n_pairs, r0, rows, *scene, dout, dstride, ws,
                                                    chunk, dx_items);
        sssgs::note_launches(1);
        int splits = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 255) / 256, (int64_t)(2 * sms / net.L + 1)));
        dim3 gb((unsigned)splits, (unsigned)net.L);
        k_mlp_bwd_b<<<gb, MLP_THREADS, smB, st>>>(net, rows, ws, chunk, *grad);
        sssgs::note_launches(1);
    }
    return launch_status();
}
