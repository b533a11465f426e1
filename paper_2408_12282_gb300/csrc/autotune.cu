// Schedule autotuner: picks the tile edge and the per-block splat batch of the
// render kernels for one scene's pairs by timing every candidate on the
// device with CUDA events.
//
// Only the stages whose work depends on the schedule are timed: the
// projection (its tile rectangles), tile binning + sort (instances grow as
// tiles shrink), and the fused composite + shade forward and backward (list
// lengths and sub-tile culling). The network runs before and after them and
// does not depend on the schedule, so its output is an input here.
#include <vector>

#include "common.cuh"

namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok = false;
    EventPair() { ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess; }
    ~EventPair() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// One pass of the schedule-dependent stages.
int run_pass(const sssgs_cfg* c, const sssgs_pair* h, int n, const sssgs_scene* scene, const float* mlp_out,
             const sssgs_tune_buffers* B, sssgs_stream st) {
    int rc = sssgs_project_fwd(c, h, B->d_pairs, n, scene, mlp_out, B->rec, B->rect, st);
    if (rc) return rc;
    rc = sssgs_bin_sort(c, h, B->d_pairs, n, B->rec, B->rect, B->capacity, B->vals, B->ranges, B->d_count,
                        B->d_status, B->workspace, B->workspace_bytes, st);
    if (rc) return rc;
    rc = sssgs_render_fwd(c, h, B->d_pairs, n, B->rec, B->vals, B->ranges, B->gbuf, B->last, B->img, nullptr, st);
    if (rc) return rc;
    return sssgs_render_bwd(c, h, B->d_pairs, n, B->rec, B->vals, B->ranges, B->gbuf, B->last, B->img, B->dimg,
                            nullptr, nullptr, 1.f, B->drec, nullptr, st);
}

}  // namespace

extern "C" int sssgs_autotune(const sssgs_cfg* base, const sssgs_pair* h_pairs, int n_pairs, const sssgs_scene* scene,
                              const float* mlp_out, const sssgs_tune_buffers* buf, const int32_t* tiles, int n_tiles,
                              const int32_t* batches, int n_batches, int reps, sssgs_tune_result* results,
                              sssgs_cfg* best, sssgs_stream stream) {
    if (!base || !h_pairs || n_pairs <= 0 || !scene || !mlp_out || !buf || !tiles || n_tiles <= 0 || !batches ||
        n_batches <= 0 || reps < 1 || reps > 1000 || !results || !best)
        return SSSGS_ERR_INVALID_ARG;
    if (!buf->d_pairs || !buf->rec || !buf->rect || !buf->vals || buf->capacity < 0 || !buf->ranges ||
        !buf->d_count || !buf->d_status || !buf->gbuf || !buf->last || !buf->img || !buf->drec || !buf->dimg)
        return SSSGS_ERR_INVALID_ARG;
    if (((uintptr_t)buf->d_pairs & 15) != 0) return SSSGS_ERR_INVALID_ARG;
    // Plan every candidate on the host first: each must fit the caller's tile
    // ranges and bin/sort workspace, otherwise nothing runs.
    std::vector<std::vector<sssgs_pair>> plans;
    std::vector<sssgs_cfg> cfgs;
    for (int ti = 0; ti < n_tiles; ++ti)
        for (int bi = 0; bi < n_batches; ++bi) {
            sssgs_cfg c = *base;
            c.tile = tiles[ti];
            c.batch = batches[bi];
            if (c.batch != 32 && c.batch != 64) return SSSGS_ERR_INVALID_ARG;
            std::vector<sssgs_pair> P(h_pairs, h_pairs + n_pairs);
            sssgs_plan_info info;
            const int rc = sssgs_plan(P.data(), n_pairs, &c, &info);
            if (rc) return rc;
            if (info.n_tiles > buf->max_tiles) return SSSGS_ERR_INVALID_ARG;
            if (sssgs_bin_workspace_bytes(info.n_items, buf->capacity, info.n_tiles) > buf->workspace_bytes)
                return SSSGS_ERR_WORKSPACE;
            plans.push_back(std::move(P));
            cfgs.push_back(c);
        }
    cudaStream_t st = (cudaStream_t)stream;
    EventPair ev;
    if (!ev.ok) return SSSGS_ERR_CUDA;
    int best_k = -1;
    for (size_t k = 0; k < plans.size(); ++k) {
        sssgs_tune_result& R = results[k];
        R.tile = cfgs[k].tile;
        R.batch = cfgs[k].batch;
        R.status = 0;
        R.reps = 0;
        R.instances = 0;
        R.ms = -1.f;
        R.reserved = 0.f;
        const sssgs_pair* h = plans[k].data();
        // the pair table for this candidate (pageable host memory: wait for the copy)
        if (cudaMemcpyAsync(buf->d_pairs, h, sizeof(sssgs_pair) * (size_t)n_pairs, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemsetAsync(buf->d_status, 0, sizeof(int32_t), st) != cudaSuccess)
            return SSSGS_ERR_CUDA;
        // warm-up pass; its instance count decides whether the candidate fits
        int rc = sssgs_project_fwd(&cfgs[k], h, buf->d_pairs, n_pairs, scene, mlp_out, buf->rec, buf->rect, stream);
        if (!rc)
            rc = sssgs_bin_sort(&cfgs[k], h, buf->d_pairs, n_pairs, buf->rec, buf->rect, buf->capacity, buf->vals,
                                buf->ranges, buf->d_count, buf->d_status, buf->workspace, buf->workspace_bytes,
                                stream);
        if (rc) return rc;
        int64_t count = 0;
        int32_t status = 0;
        if (cudaMemcpyAsync(&count, buf->d_count, sizeof(count), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&status, buf->d_status, sizeof(status), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SSSGS_ERR_CUDA;
        R.instances = count;
        if (count > buf->capacity || (status & SSSGS_STATUS_CAPACITY)) {
            R.status = SSSGS_STATUS_CAPACITY;
            continue;
        }
        rc = run_pass(&cfgs[k], h, n_pairs, scene, mlp_out, buf, stream);
        if (rc) return rc;
        if (cudaEventRecord(ev.a, st) != cudaSuccess) return SSSGS_ERR_CUDA;
        for (int r = 0; r < reps; ++r) {
            rc = run_pass(&cfgs[k], h, n_pairs, scene, mlp_out, buf, stream);
            if (rc) return rc;
        }
        float ms = 0.f;
        if (cudaEventRecord(ev.b, st) != cudaSuccess || cudaEventSynchronize(ev.b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess)
            return SSSGS_ERR_CUDA;
        R.reps = reps;
        R.ms = ms / (float)reps;
        if (best_k < 0 || R.ms < results[best_k].ms) best_k = (int)k;
    }
    if (best_k < 0) return SSSGS_ERR_WORKSPACE;   // no candidate fitted the instance capacity
    *best = cfgs[best_k];
    return SSSGS_OK;
}
