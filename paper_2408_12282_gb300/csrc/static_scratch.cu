// Allocation-free variant of sssgs_bin_sort.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// all device memory and hands out none, and real-time loops that must not pay
// cudaMalloc's implicit device-wide synchronisation. They still own their
// inputs and outputs, but cannot provide the bin/sort workspace. This entry
// point uses a scratch array compiled into the library instead.
//
// The scratch is a file-scope __device__ array of SSSGS_STATIC_SCRATCH_BYTES
// (9 MiB). Every GPU that loads the library holds it until the process
// exits. In host code the array's name only stands for the symbol, not for a
// device address, so its address is looked up with cudaGetSymbolAddress, once
// per device, on the first call made while that device is current, and cached.
// Make that first call before any stream capture begins. The cached address
// belongs to the device's primary context: after cudaDeviceReset the array
// lives at a new address, so do not call this entry point again in that
// process after a reset.
//
// All calls share the one array and it keeps whatever the last call wrote.
// Nothing in it has to start at zero: every region is written by the sort
// before it is read. Calls whose work overlaps on the GPU (different streams,
// or different host threads, on the same device) race on the array; serialise
// them.
#include <mutex>

#include "common.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)SSSGS_STATIC_SCRATCH_BYTES;
static_assert(kScratchBytes % 256 == 0, "scratch size must keep 256-byte alignment");

__device__ __align__(256) unsigned char g_bin_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (nullptr on error).
void* scratch_on_current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace

extern "C" int sssgs_bin_sort_static(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                                     int n_pairs, const float* rec, const int32_t* rect, int64_t capacity,
                                     uint32_t* vals, uint32_t* ranges, int64_t* d_count, int32_t* d_status,
                                     sssgs_stream stream) {
    if (!cfg || !h_pairs || !d_pairs || n_pairs <= 0 || !rec || !rect || !vals || !ranges || !d_count)
        return SSSGS_ERR_INVALID_ARG;
    const sssgs_pair& lastp = h_pairs[n_pairs - 1];
    const int64_t n_items = lastp.item_offset + lastp.g_count;
    const int64_t n_tiles = (int64_t)lastp.tile_offset + (int64_t)lastp.tiles_x * lastp.tiles_y;
    // a pair table that sssgs_plan did not fill (negative counts or offsets)
    if (lastp.item_offset < 0 || lastp.g_count < 0 || n_tiles <= 0 || n_tiles > INT32_MAX || capacity < 0)
        return SSSGS_ERR_INVALID_ARG;
    if (n_items > SSSGS_STATIC_MAX_ITEMS || capacity > SSSGS_STATIC_MAX_INSTANCES) return SSSGS_ERR_TOO_LARGE;
    if (sssgs_bin_workspace_bytes(n_items, capacity, (int32_t)n_tiles) > kScratchBytes) return SSSGS_ERR_TOO_LARGE;
    void* ws = scratch_on_current_device();
    if (!ws) return SSSGS_ERR_CUDA;
    return sssgs_bin_sort(cfg, h_pairs, d_pairs, n_pairs, rec, rect, capacity, vals, ranges, d_count, d_status, ws,
                          kScratchBytes, stream);
}
