// Tile binning and depth ordering of the splats (the ordered sequence of Eq. 3).
//
// Two stable LSD radix sorts replace one wide-key sort:
//   1. items (pair, Gaussian) by (pair, float32 depth bits)   -- n_items keys
//   2. instances, emitted in that order, by the tile index within their pair
//      (the instances already come out pair by pair, so the pair needs no
//      pass)                                                  -- ~12 key bits
// Stability of (2) keeps the depth order inside every (pair, tile) run, so
// every tile's list is in (depth, item) order; runs of the same local tile
// of different pairs sit next to each other and the per-tile ranges point
// to them.
//
// Each radix pass is reduce-then-scan: a per-block digit histogram (one
// shared-memory histogram per warp, plain atomics), a device scan of the
// (digit-major, block-minor) histogram, then a scatter in which every warp
// ranks its keys stably (the lanes sharing a digit are found with one ballot
// per digit bit), blocks stage keys in shared memory in digit order and write
// each digit run contiguously. No kernel waits on another block, so nothing
// can spin.
#include <algorithm>

#include "common.cuh"

namespace sssgs {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;   // keys per block
constexpr int RS_WARPS = RS_THREADS / 32;

constexpr int SC_THREADS = 512;
constexpr int SC_PER = 8;
constexpr int SC_CHUNK = SC_THREADS * SC_PER;

__device__ __forceinline__ int64_t eff_n(const int64_t* d_n, int64_t cap) {
    return d_n ? min(*d_n, cap) : cap;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(SSSGS_FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Inclusive scan over the block; `sh` needs blockDim/32 entries.
template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T* sh) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_incl_scan(v, lane);
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? sh[lane] : T(0);
        w = warp_incl_scan(w, lane);
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v += sh[warp - 1];
    __syncthreads();
    return v;
}

// ---------------------------------------------------------------- scan

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const T* __restrict__ in, int64_t L, T* __restrict__ part) {
    __shared__ T sh[SC_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SC_CHUNK;
    T s = 0;
    for (int k = 0; k < SC_PER; ++k) {
        int64_t i = base + (int64_t)k * SC_THREADS + threadIdx.x;
        if (i < L) s += in[i];
    }
    s = block_incl_scan(s, sh);
    if (threadIdx.x == SC_THREADS - 1) part[blockIdx.x] = s;
}

template <typename T>
__global__ void __launch_bounds__(1024) k_scan_top(T* __restrict__ part, int64_t nb) {
    __shared__ T sh[32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < nb; b += 1024) {
        int64_t i = b + threadIdx.x;
        T v = i < nb ? part[i] : T(0);
        T inc = block_incl_scan(v, sh);
        T c = carry;
        if (i < nb) part[i] = c + inc - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + inc;
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_scan_apply(const T* __restrict__ in, T* __restrict__ out, int64_t L,
                                                          const T* __restrict__ part) {
    __shared__ T sh[SC_THREADS / 32];
    int64_t base = (int64_t)blockIdx.x * SC_CHUNK + (int64_t)threadIdx.x * SC_PER;
    T v[SC_PER];
    T s = 0;
#pragma unroll
    for (int k = 0; k < SC_PER; ++k) {
        v[k] = (base + k < L) ? in[base + k] : T(0);
        s += v[k];
    }
    T inc = block_incl_scan(s, sh);
    T run = part[blockIdx.x] + inc - s;
#pragma unroll
    for (int k = 0; k < SC_PER; ++k) {
        if (base + k < L) out[base + k] = run;
        run += v[k];
    }
}

template <typename T>
static void exclusive_scan(const T* in, T* out, int64_t L, T* part, cudaStream_t st) {
    int64_t nb = (L + SC_CHUNK - 1) / SC_CHUNK;
    if (nb == 0) return;
    k_scan_reduce<T><<<(unsigned)nb, SC_THREADS, 0, st>>>(in, L, part);
    sssgs::note_launches(1);
    k_scan_top<T><<<1, 1024, 0, st>>>(part, nb);
    sssgs::note_launches(1);
    k_scan_apply<T><<<(unsigned)nb, SC_THREADS, 0, st>>>(in, out, L, part);
    sssgs::note_launches(1);
}

// ---------------------------------------------------------------- radix pass

template <typename K, int NB>
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const K* __restrict__ keys, const int64_t* d_n, int64_t cap,
                                                        int shift, uint32_t mask, uint32_t* __restrict__ hist,
                                                        int nblocks) {
    // One histogram per warp; plain shared-memory atomics (lanes with the
    // same digit serialise only within their warp).
    __shared__ uint32_t h[RS_WARPS * NB];
    for (int d = threadIdx.x; d < RS_WARPS * NB; d += RS_THREADS) h[d] = 0;
    __syncthreads();
    const int64_t n = eff_n(d_n, cap);
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    uint32_t* hw = h + (threadIdx.x >> 5) * NB;
    uint32_t dig[RS_ITEMS];
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k) {
        const int64_t idx = base + (int64_t)k * RS_THREADS + threadIdx.x;
        dig[k] = idx < n ? ((uint32_t)(keys[idx] >> shift) & mask) : 0xFFFFu;
    }
#pragma unroll
    for (int k = 0; k < RS_ITEMS; ++k)
        if (dig[k] != 0xFFFFu) atomicAdd(&hw[dig[k]], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < NB; d += RS_THREADS) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) c += h[w * NB + d];
        hist[(int64_t)d * nblocks + blockIdx.x] = c;
    }
}

template <typename K, int NB>
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                           K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           const int64_t* d_n, int64_t cap, int shift, uint32_t mask,
                                                           const uint32_t* __restrict__ hoff, int nblocks) {
    constexpr int DPT = NB / RS_THREADS;          // digits per thread in the digit scans
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* skey = reinterpret_cast<K*>(smem_raw);
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + RS_TILE);
    uint32_t* wcnt = sval + RS_TILE;               // [RS_WARPS][NB]
    uint32_t* bstart = wcnt + RS_WARPS * NB;       // [NB]
    uint32_t* gbase = bstart + NB;                 // [NB]
    uint32_t* sh = gbase + NB;                     // [RS_WARPS]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < RS_WARPS * NB; i += RS_THREADS) wcnt[i] = 0;
    for (int d = tid; d < NB; d += RS_THREADS) gbase[d] = hoff[(int64_t)d * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t n = eff_n(d_n, cap);
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    if (base >= n) return;                          // uniform over the block
    const int64_t wbase = base + (int64_t)warp * (RS_ITEMS * 32);
    const uint32_t lt = (1u << lane) - 1u;
    const int nbits = 32 - __clz(mask);
    K key[RS_ITEMS];
    uint32_t val[RS_ITEMS], rank[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {   // all loads first, so they are in flight together
        const int64_t idx = wbase + j * 32 + lane;
        key[j] = idx < n ? kin[idx] : K(0);
        val[j] = idx < n ? vin[idx] : 0u;
    }
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        int64_t idx = wbase + j * 32 + lane;
        bool ok = idx < n;
        uint32_t d = ok ? ((uint32_t)(key[j] >> shift) & mask) : 0xFFFFu;
        // lanes with the same digit: one ballot per digit bit
        uint32_t peers = __ballot_sync(SSSGS_FULL, ok);
        for (int b = 0; b < nbits; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t bal = __ballot_sync(SSSGS_FULL, bit);
            peers &= bit ? bal : ~bal;
        }
        rank[j] = ok ? wcnt[warp * NB + d] + __popc(peers & lt) : 0u;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[warp * NB + d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // digits [DPT*tid, DPT*tid + DPT): exclusive over warps, then over digits
        uint32_t tot[DPT];
        uint32_t sum = 0;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = DPT * tid + q;
            uint32_t run = 0;
            for (int w = 0; w < RS_WARPS; ++w) {
                uint32_t c = wcnt[w * NB + d];
                wcnt[w * NB + d] = run;
                run += c;
            }
            tot[q] = run;
            sum += run;
        }
        uint32_t inc = block_incl_scan(sum, sh);
        uint32_t start = inc - sum;
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            bstart[DPT * tid + q] = start;
            start += tot[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        int64_t idx = wbase + j * 32 + lane;
        if (idx < n) {
            uint32_t d = (uint32_t)(key[j] >> shift) & mask;
            uint32_t lpos = bstart[d] + wcnt[warp * NB + d] + rank[j];
            skey[lpos] = key[j];
            sval[lpos] = val[j];
        }
    }
    __syncthreads();
    int cnt = (int)min((int64_t)RS_TILE, n - base);
    for (int i = tid; i < cnt; i += RS_THREADS) {
        K k = skey[i];
        uint32_t d = (uint32_t)(k >> shift) & mask;
        int64_t g = (int64_t)gbase[d] + (uint32_t)(i - bstart[d]);
        kout[g] = k;
        vout[g] = sval[i];
    }
}

template <typename K, int NB>
static size_t scatter_smem() {
    return (size_t)RS_TILE * (sizeof(K) + 4) + (size_t)(RS_WARPS * NB + 2 * NB + RS_WARPS) * 4;
}

template <typename K, int NB>
static void radix_pass(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, const int64_t* d_n, int64_t cap,
                       int shift, int nb, uint32_t* hist, uint32_t* part32, int nblocks, cudaStream_t st) {
    const uint32_t mask = (1u << nb) - 1u;
    const size_t sm = scatter_smem<K, NB>();
    cudaFuncSetAttribute(k_rs_scatter<K, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_rs_hist<K, NB><<<nblocks, RS_THREADS, 0, st>>>(kin, d_n, cap, shift, mask, hist, nblocks);
    sssgs::note_launches(1);
    exclusive_scan<uint32_t>(hist, hist, (int64_t)NB * nblocks, part32, st);
    k_rs_scatter<K, NB><<<nblocks, RS_THREADS, sm, st>>>(kin, vin, kout, vout, d_n, cap, shift, mask, hist, nblocks);
    sssgs::note_launches(1);
}

// Stable sort of (key, value) pairs over `bits` low key bits, in the fewest
// passes of at most 10 bits (<= 1024 buckets), bits spread evenly. Buffers
// ping-pong; returns the index (0: kA/vA, 1: kB/vB) holding the result.
template <typename K>
static int radix_sort(K* kA, uint32_t* vA, K* kB, uint32_t* vB, const int64_t* d_n, int64_t cap, int bits,
                      uint32_t* hist, uint32_t* part32, cudaStream_t st, int lo = 0) {
    int nblocks = (int)((cap + RS_TILE - 1) / RS_TILE);
    if (nblocks == 0 || bits <= 0) return 0;
    const int np = (bits + 9) / 10;
    const int per = (bits + np - 1) / np;
    int cur = 0;
    for (int shift = lo; shift < lo + bits; shift += per) {
        const int nb = lo + bits - shift < per ? lo + bits - shift : per;
        K* kin = cur ? kB : kA;
        uint32_t* vin = cur ? vB : vA;
        K* kout = cur ? kA : kB;
        uint32_t* vout = cur ? vA : vB;
        if (nb <= 8) radix_pass<K, 256>(kin, vin, kout, vout, d_n, cap, shift, nb, hist, part32, nblocks, st);
        else if (nb == 9) radix_pass<K, 512>(kin, vin, kout, vout, d_n, cap, shift, nb, hist, part32, nblocks, st);
        else radix_pass<K, 1024>(kin, vin, kout, vout, d_n, cap, shift, nb, hist, part32, nblocks, st);
        cur ^= 1;
    }
    return cur;
}

static int passes(int bits) {
    if (bits <= 0) return 0;
    const int np = (bits + 9) / 10;
    const int per = (bits + np - 1) / np;
    return (bits + per - 1) / per;
}

// Stable sort of n (u32 key, u32 value) pairs by the low `bits` key bits, for
// other parts of the library (the BVH builder's Morton codes). Workspace:
// radix_sort_u32_workspace(n) bytes, 256-byte aligned. Returns 0 when kA/vA
// hold the result, 1 when kB/vB do.
size_t radix_sort_u32_workspace(int64_t n) {
    const int64_t nb = std::max<int64_t>((n + RS_TILE - 1) / RS_TILE, 1);
    const int64_t np = (1024 * nb + SC_CHUNK - 1) / SC_CHUNK;
    return ((4 * (size_t)1024 * (size_t)nb + 255) & ~(size_t)255) + 4 * (size_t)(np + 1);
}

int radix_sort_u32(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, int64_t n, int bits, void* ws,
                   cudaStream_t st) {
    const int64_t nb = std::max<int64_t>((n + RS_TILE - 1) / RS_TILE, 1);
    uint32_t* hist = (uint32_t*)ws;
    uint32_t* part32 = (uint32_t*)((uint8_t*)ws + ((4 * (size_t)1024 * (size_t)nb + 255) & ~(size_t)255));
    return radix_sort<uint32_t>(kA, vA, kB, vB, nullptr, n, bits, hist, part32, st);
}

// ---------------------------------------------------------------- binning kernels

__global__ void k_depth_keys(const sssgs_pair* __restrict__ pairs, int n_pairs, int64_t n_items,
                             const float* __restrict__ rec, const int4* __restrict__ rect,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_items) return;
    int p = pair_of_item(pairs, n_pairs, m);
    int4 r = rect[m];
    uint32_t bits = 0xffffffffu;
    if (r.x <= r.y && r.z <= r.w) bits = __float_as_uint(rec[(int64_t)SSSGS_REC * m + 6]);
    keys[m] = ((uint64_t)p << 32) | bits;
    vals[m] = (uint32_t)m;
}

__global__ void k_count_tiles(int64_t n_items, const uint32_t* __restrict__ vals, const int4* __restrict__ rect,
                              uint64_t* __restrict__ cnt) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > n_items) return;
    uint64_t c = 0;
    if (s < n_items) {
        int4 r = rect[vals[s]];
        if (r.x <= r.y && r.z <= r.w) c = (uint64_t)(r.y - r.x + 1) * (uint64_t)(r.w - r.z + 1);
    }
    cnt[s] = c;    // cnt[n_items] = 0 so the exclusive scan ends with the total
}

__global__ void k_set_count(const uint64_t* __restrict__ off, int64_t n_items, int64_t cap, int64_t* d_count,
                            int32_t* d_status) {
    uint64_t total = off[n_items];
    *d_count = (int64_t)total;
    if (total > (uint64_t)cap && d_status) atomicOr(d_status, SSSGS_STATUS_CAPACITY);
}

// Writes the instances of a block of 256 depth-ordered items. The block's
// output is the contiguous range [off[s0], off[s0 + 256]), so the block fills
// it position by position (coalesced stores): each position finds its item by
// binary search over the block's offsets, then its tile inside the item's
// rectangle (row-major order). The instance key is the pair-local tile index
// above the pair index, (local tile << pbits) | pair: instances come out in
// pair order (items are sorted by pair first), so a stable sort of the keys'
// pair bits would leave them in place, and sorting the local-tile bits alone
// gives every (pair, tile) its contiguous, depth-ordered run.
__global__ void __launch_bounds__(256) k_emit(const sssgs_pair* __restrict__ pairs, int64_t n_items,
                                              const uint64_t* __restrict__ dkeys, const uint32_t* __restrict__ dvals,
                                              const int4* __restrict__ rect, const uint64_t* __restrict__ off,
                                              int64_t cap, int pbits, uint32_t* __restrict__ ikeys,
                                              uint32_t* __restrict__ ivals) {
    __shared__ uint32_t s_off[257], s_item[256], s_base[256], s_w[256], s_tx[256], s_pair[256];
    const int t = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * 256;
    const int nb = (int)min((int64_t)256, n_items - s0);
    const uint64_t B0 = off[s0];
    if (t < nb) {
        const int64_t s = s0 + t;
        const uint32_t m = dvals[s];
        const int4 r = rect[m];
        s_off[t] = (uint32_t)(off[s] - B0);
        s_item[t] = m;
        if (r.x <= r.y && r.z <= r.w) {
            const int p = (int)(dkeys[s] >> 32);
            const sssgs_pair& P = pairs[p];
            s_base[t] = (uint32_t)(r.z * P.tiles_x + r.x);
            s_w[t] = (uint32_t)(r.y - r.x + 1);
            s_tx[t] = (uint32_t)P.tiles_x;
            s_pair[t] = (uint32_t)p;
        } else {
            s_base[t] = 0;
            s_w[t] = 1;
            s_tx[t] = 0;
            s_pair[t] = 0;
        }
    }
    if (t == 0) s_off[nb] = (uint32_t)(off[s0 + nb] - B0);
    __syncthreads();
    const uint32_t total = s_off[nb];
    for (uint32_t rel = t; rel < total; rel += 256) {
        const uint64_t pos = B0 + rel;
        if (pos >= (uint64_t)cap) break;
        int lo = 0, hi = nb - 1;            // last item whose range starts at or before rel
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= rel) lo = mid; else hi = mid - 1;
        }
        const uint32_t q = rel - s_off[lo], w = s_w[lo];
        const uint32_t dy = q / w, dx = q - dy * w;
        ikeys[pos] = ((s_base[lo] + dy * s_tx[lo] + dx) << pbits) | s_pair[lo];
        ivals[pos] = s_item[lo];
    }
}

// Per-tile [start, end) from the sorted instance keys, four keys per thread;
// a key (local tile << pbits) | pair names global tile tile_offset[pair] +
// local tile.
__global__ void k_ranges(const uint32_t* __restrict__ keys, const int64_t* d_n, int64_t cap,
                         const sssgs_pair* __restrict__ pairs, int pbits, uint2* __restrict__ ranges) {
    const int64_t n = eff_n(d_n, cap);
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (s >= n) return;
    const uint4 q = *reinterpret_cast<const uint4*>(keys + s);
    const uint32_t k[6] = {s > 0 ? keys[s - 1] : 0xFFFFFFFFu, q.x, q.y, q.z, q.w,
                           s + 4 < n ? keys[s + 4] : 0xFFFFFFFFu};
#pragma unroll
    for (int j = 1; j <= 4; ++j) {
        const int64_t i = s + j - 1;
        if (i >= n) break;
        const uint32_t kj = k[j];
        const bool first = i == 0 || k[j - 1] != kj;
        const bool lastk = i == n - 1 || (j < 4 ? k[j + 1] : k[5]) != kj;
        if (first || lastk) {
            const uint32_t g = (uint32_t)pairs[kj & ((1u << pbits) - 1u)].tile_offset + (kj >> pbits);
            if (first) ranges[g].x = (uint32_t)i;
            if (lastk) ranges[g].y = (uint32_t)(i + 1);
        }
    }
}

}  // namespace sssgs

using namespace sssgs;

namespace {
struct BinLayout {
    size_t dkA, dkB, dvA, dvB, cnt, ikA, ikB, ivW, hist, part32, part64, total;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

BinLayout bin_layout(int64_t n_items, int64_t cap) {
    BinLayout L;
    size_t o = 0;
    L.dkA = o; o += al(8 * (size_t)n_items);
    L.dkB = o; o += al(8 * (size_t)n_items);
    L.dvA = o; o += al(4 * (size_t)n_items);
    L.dvB = o; o += al(4 * (size_t)n_items);
    L.cnt = o; o += al(8 * (size_t)(n_items + 1));
    L.ikA = o; o += al(4 * (size_t)cap);
    L.ikB = o; o += al(4 * (size_t)cap);
    L.ivW = o; o += al(4 * (size_t)cap);
    int64_t nb = std::max((n_items + RS_TILE - 1) / RS_TILE, (cap + RS_TILE - 1) / RS_TILE);
    L.hist = o; o += al(4 * (size_t)1024 * (size_t)std::max<int64_t>(nb, 1));
    int64_t np = std::max<int64_t>((1024 * nb + SC_CHUNK - 1) / SC_CHUNK, (n_items + 1 + SC_CHUNK - 1) / SC_CHUNK);
    L.part32 = o; o += al(4 * (size_t)(np + 1));
    L.part64 = o; o += al(8 * (size_t)(np + 1));
    L.total = o;
    return L;
}

int bits_for(int64_t n) {
    int b = 1;
    while (b < 40 && ((int64_t)1 << b) < n) ++b;
    return b;
}
}  // namespace

extern "C" size_t sssgs_bin_workspace_bytes(int64_t n_items, int64_t capacity, int32_t n_tiles) {
    (void)n_tiles;
    if (n_items < 0 || capacity < 0) return 0;
    return bin_layout(n_items, capacity).total;
}

extern "C" int sssgs_bin_sort(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                              int n_pairs, const float* rec, const int32_t* rect, int64_t capacity,
                              uint32_t* vals, uint32_t* ranges, int64_t* d_count, int32_t* d_status,
                              void* workspace, size_t workspace_bytes, sssgs_stream stream) {
    if (!cfg || !h_pairs || !d_pairs || n_pairs <= 0 || !rec || !rect || !vals || !ranges || !d_count)
        return SSSGS_ERR_INVALID_ARG;
    if (capacity < 0 || capacity >= ((int64_t)1 << 32) || ((uintptr_t)rect & 15)) return SSSGS_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t n_items = h_pairs[n_pairs - 1].item_offset + h_pairs[n_pairs - 1].g_count;
    int64_t n_tiles = (int64_t)h_pairs[n_pairs - 1].tile_offset +
                      (int64_t)h_pairs[n_pairs - 1].tiles_x * h_pairs[n_pairs - 1].tiles_y;
    if (n_items >= ((int64_t)1 << 32)) return SSSGS_ERR_INVALID_ARG;
    int64_t max_local = 1;
    for (int p = 0; p < n_pairs; ++p)
        max_local = std::max<int64_t>(max_local, (int64_t)h_pairs[p].tiles_x * h_pairs[p].tiles_y);
    const int local_tile_bits = max_local > 1 ? bits_for(max_local) : 0;
    if ((n_pairs > 1 ? bits_for(n_pairs) : 0) + local_tile_bits > 32) return SSSGS_ERR_INVALID_ARG;
    BinLayout L = bin_layout(n_items, capacity);
    if (!workspace || workspace_bytes < L.total) return SSSGS_ERR_WORKSPACE;
    if ((uintptr_t)workspace & 255) return SSSGS_ERR_INVALID_ARG;
    unsigned char* ws = (unsigned char*)workspace;
    uint64_t* dkA = (uint64_t*)(ws + L.dkA);
    uint64_t* dkB = (uint64_t*)(ws + L.dkB);
    uint32_t* dvA = (uint32_t*)(ws + L.dvA);
    uint32_t* dvB = (uint32_t*)(ws + L.dvB);
    uint64_t* cnt = (uint64_t*)(ws + L.cnt);
    uint32_t* ikA = (uint32_t*)(ws + L.ikA);
    uint32_t* ikB = (uint32_t*)(ws + L.ikB);
    uint32_t* ivW = (uint32_t*)(ws + L.ivW);
    uint32_t* hist = (uint32_t*)(ws + L.hist);
    uint32_t* part32 = (uint32_t*)(ws + L.part32);
    uint64_t* part64 = (uint64_t*)(ws + L.part64);

    cudaMemsetAsync(ranges, 0, sizeof(uint32_t) * 2 * (size_t)n_tiles, st);
    if (n_items == 0) {
        cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
        return launch_status();
    }
    const int4* rect4 = (const int4*)rect;
    // 1. depth order per pair
    unsigned gb = (unsigned)((n_items + 255) / 256);
    k_depth_keys<<<gb, 256, 0, st>>>(d_pairs, n_pairs, n_items, rec, rect4, dkA, dvA);
    sssgs::note_launches(1);
    int pbits = n_pairs > 1 ? bits_for(n_pairs) : 0;
    int r1 = radix_sort<uint64_t>(dkA, dvA, dkB, dvB, nullptr, n_items, 32 + pbits, hist, part32, st);
    uint64_t* dk = r1 ? dkB : dkA;
    uint32_t* dv = r1 ? dvB : dvA;
    // 2. instance offsets in depth order
    unsigned gc = (unsigned)((n_items + 1 + 255) / 256);
    k_count_tiles<<<gc, 256, 0, st>>>(n_items, dv, rect4, cnt);
    sssgs::note_launches(1);
    exclusive_scan<uint64_t>(cnt, cnt, n_items + 1, part64, st);
    k_set_count<<<1, 1, 0, st>>>(cnt, n_items, capacity, d_count, d_status);
    sssgs::note_launches(1);
    if (capacity == 0) return launch_status();
    // 3. emit into the buffer that the tile sort will finish in `vals`
    const int tpbits = n_pairs > 1 ? bits_for(n_pairs) : 0;   // pair bits of the instance keys
    const int lbits = local_tile_bits;                         // pair-local tile bits
    int np = passes(lbits);
    uint32_t* v0 = (np % 2 == 0) ? vals : ivW;
    uint32_t* v1 = (np % 2 == 0) ? ivW : vals;
    k_emit<<<gb, 256, 0, st>>>(d_pairs, n_items, dk, dv, rect4, cnt, capacity, tpbits, ikA, v0);
    sssgs::note_launches(1);
    // 4. stable sort by the local tile bits (the pair bits are in order already)
    int r2 = radix_sort<uint32_t>(ikA, v0, ikB, v1, d_count, capacity, lbits, hist, part32, st, tpbits);
    uint32_t* ik = r2 ? ikB : ikA;
    // 5. per-tile ranges
    unsigned gr = (unsigned)((capacity + 1023) / 1024);
    k_ranges<<<gr, 256, 0, st>>>(ik, d_count, capacity, d_pairs, tpbits, (uint2*)ranges);
    sssgs::note_launches(1);
    return launch_status();
}
