// Tensor-core (tcgen05, BF16 operands, FP32 accumulation in TMEM) network.
#include "common.cuh"

int sssgs_mlp_fwd_tc(const sssgs_mlp*, const sssgs_pair*, const sssgs_pair*, int, const sssgs_scene*, float*,
                     sssgs_stream) {
    return SSSGS_ERR_UNSUPPORTED;
}

int sssgs_mlp_bwd_tc(const sssgs_mlp*, const sssgs_pair*, const sssgs_pair*, int, const sssgs_scene*, const float*,
                     const sssgs_mlp_grad*, float*, void*, size_t, sssgs_stream) {
    return SSSGS_ERR_UNSUPPORTED;
}
