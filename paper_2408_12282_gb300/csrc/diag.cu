// Diagnostics of the failure-detection path. The tensor-core kernels bound
// every mbarrier wait; when a wait runs out they set SSSGS_STATUS_TIMEOUT in
// the caller's status word and return, leaving the context usable. This entry
// point exercises exactly that path: one thread waits on an mbarrier that no
// thread ever arrives on, with a short limit, and reports the timeout.
#include "common.cuh"
#include "tc.cuh"

namespace sssgs {
namespace {

__global__ void k_wait_selftest(int32_t* __restrict__ status, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = tc::smem_u32(&bar);
    if (threadIdx.x == 0) {
        tc::mbar_init(b, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait_for(b, 0, limit)) atomicOr(status, (int32_t)SSSGS_STATUS_TIMEOUT);
}

}  // namespace
}  // namespace sssgs

extern "C" int sssgs_selftest_wait_timeout(int32_t* d_status, int64_t limit_cycles, sssgs_stream stream) {
    if (!d_status || limit_cycles <= 0 || limit_cycles > 4000000000ll) return SSSGS_ERR_INVALID_ARG;
    sssgs::k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(d_status, (long long)limit_cycles);
    sssgs::note_launches(1);
    return sssgs::launch_status();
}
