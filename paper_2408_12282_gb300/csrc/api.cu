// Host-side entry points of libsssgs that launch nothing: version, error
// strings, default conventions and the layout planner of a batch of pairs.
#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace {
std::atomic<unsigned long long> g_launches{0};
}

void sssgs::note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

extern "C" uint64_t sssgs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char* sssgs_version(void) { return "sssgs 0.1 (sm_103a)"; }

extern "C" const char* sssgs_strerror(int code) {
    switch (code) {
        case SSSGS_OK: return "ok";
        case SSSGS_ERR_INVALID_ARG: return "invalid argument";
        case SSSGS_ERR_CUDA: return "CUDA launch or API error";
        case SSSGS_ERR_UNSUPPORTED: return "configuration not supported";
        case SSSGS_ERR_WORKSPACE: return "workspace too small";
        case SSSGS_ERR_TOO_LARGE: return "problem exceeds the static scratch limits";
        default: return "unknown error";
    }
}

extern "C" void sssgs_cfg_default(sssgs_cfg* c) {
    if (!c) return;
    c->tile = 16;
    c->batch = 32;
    c->dilation = 0.3f;
    c->det_eps = 1e-6f;
    c->z_near = 0.2f;
    c->alpha_min = 1.0f / 255.0f;
    c->alpha_max = 0.99f;
    c->T_min = 1e-4f;
    c->A_eps = 1e-6f;
}

extern "C" int sssgs_plan(sssgs_pair* pairs, int n_pairs, const sssgs_cfg* cfg, sssgs_plan_info* info) {
    if (!pairs || n_pairs <= 0 || !cfg || !info) return SSSGS_ERR_INVALID_ARG;
    if (cfg->tile != 8 && cfg->tile != 16 && cfg->tile != 32) return SSSGS_ERR_INVALID_ARG;
    int64_t items = 0, pixels = 0, tiles = 0;
    for (int p = 0; p < n_pairs; ++p) {
        sssgs_pair& P = pairs[p];
        if (P.W < 1 || P.H < 1 || P.W > 16384 || P.H > 16384 || P.g_count < 0 || P.g_begin < 0)
            return SSSGS_ERR_INVALID_ARG;
        if (!(P.fx > 0.f) || !(P.fy > 0.f)) return SSSGS_ERR_INVALID_ARG;
        P.tiles_x = (P.W + cfg->tile - 1) / cfg->tile;
        P.tiles_y = (P.H + cfg->tile - 1) / cfg->tile;
        P.tile_offset = (int32_t)tiles;
        P.pad0 = P.pad1 = 0;
        P.pixel_offset = pixels;
        P.item_offset = items;
        items += P.g_count;
        pixels += (int64_t)P.W * P.H;
        tiles += (int64_t)P.tiles_x * P.tiles_y;
        if (tiles >= ((int64_t)1 << 31)) return SSSGS_ERR_INVALID_ARG;
    }
    info->n_items = items;
    info->n_pixels = pixels;
    info->n_tiles = (int32_t)tiles;
    int b = 1;
    while (((int64_t)1 << b) < tiles) ++b;
    info->tile_bits = b;
    return SSSGS_OK;
}
