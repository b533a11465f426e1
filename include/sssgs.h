/*
 * libsssgs -- differentiable OLAT render of relightable 3D Gaussians with a
 * learned subsurface-scattering residual, for one NVIDIA GB300 (sm_103a).
 *
 * Method: "Subsurface Scattering for 3D Gaussian Splatting" (arXiv 2408.12282).
 * One view/light pair ("pair") is rendered per camera + OLAT point light
 * (Section 3.2, "Incident Light"). The stages of the forward pass are
 *
 *   mlp      (L_SSS, L_in) = f_Theta(mu, Sigma, n, w_in, w_out, v)        Eq. 6
 *   project  EWA splat: Sigma' = J W Sigma W^T J^T, conic, mean, depth    Eq. 1, Eq. 2
 *   bin_sort tile binning + stable radix sort by (tile, depth)            Eq. 3 ordering
 *   composite front-to-back alpha compositing of 15 features             Eq. 3, Fig. 2
 *   shade    per-pixel Cook-Torrance/Lambert BRDF + SSS blend             Eq. 4, Eq. 7
 *
 * and the backward of each (gradients accumulate, "+=", into caller-zeroed
 * buffers).
 *
 * Conventions (the paper is silent on each; both this library and its test
 * oracle use them):
 *   camera  OpenCV pinhole, x_cam = R x_world + t, +z forward, pixel (i, j)
 *           sampled at (i + 0.5, j + 0.5);
 *   alpha   = min(alpha_max, o exp(-p)), p = 0.5 (ca dx^2 + cc dy^2) + cb dx dy,
 *           skipped if p < 0 or alpha < alpha_min; compositing stops before the
 *           Gaussian that would take T below T_min;
 *   order   float32 view depth z = fmaf(R20, mx, fmaf(R21, my, fmaf(R22, mz, t2))),
 *           ties by item index;
 *   BRDF    GGX D, Schlick F (F0 = 0.04 (1 - m) + b m), separable Smith-GGX as
 *           V = G / (4 n.wo n.wi), alpha_r = roughness^2; Lambert (1 - m) b / pi;
 *   output  image = A * L_out(G / A), A = 1 - T (black background).
 *
 * Ownership: the caller allocates every buffer (device memory unless stated)
 * and the workspace; the library never allocates or frees. All calls enqueue
 * asynchronous work on `stream` and return immediately.
 *
 * Errors: each entry point returns SSSGS_OK (0) or a negative code detected on
 * the host before any launch (bad argument, launch failure). Conditions found
 * on the device (instance capacity overflow) are written to the caller's
 * device status word and never trap; read it after the stream synchronises.
 */
#ifndef SSSGS_H
#define SSSGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sssgs_stream;   /* == cudaStream_t; NULL = legacy default stream */

enum {
    SSSGS_OK = 0,
    SSSGS_ERR_INVALID_ARG = -1,   /* host-side argument check failed; nothing launched */
    SSSGS_ERR_CUDA = -2,          /* a CUDA launch or API call failed */
    SSSGS_ERR_UNSUPPORTED = -3,   /* configuration not compiled in (tile size, MLP shape) */
    SSSGS_ERR_WORKSPACE = -4,     /* workspace smaller than sssgs_*_workspace_bytes */
    SSSGS_ERR_TOO_LARGE = -5      /* problem exceeds the fixed scratch of sssgs_bin_sort_static */
};

/* Device status bits (written with atomicOr into the caller's int32 word). */
enum {
    SSSGS_STATUS_CAPACITY = 1,    /* more tile instances than `capacity`; lists truncated */
    SSSGS_STATUS_TIMEOUT = 2      /* a bounded wait inside a tensor-core kernel ran out (~1 s);
                                     that kernel stopped early and its outputs are incomplete */
};

#define SSSGS_NF 15          /* composited features: depth, n3, base3, rough, metal, sss, Lsss3, Lin, vis */
#define SSSGS_REC 24         /* floats per packed (pair, Gaussian) record (96 B, 16-B aligned) */
#define SSSGS_GBUF 16        /* floats per G-buffer pixel: 15 features + final transmittance T */
#define SSSGS_MAX_LAYERS 8
#define SSSGS_DX 14          /* floats per item of the network-input gradient: dmu 3, dn 3, dv 1, dquat 4, dlog_s 3 */

/* Record layout (floats): 0 mx, 1 my, 2 ca, 3 cb, 4 cc, 5 opacity,
 * 6..20 features (6 depth, 7-9 n, 10-12 base, 13 rough, 14 metal, 15 sss,
 * 16-18 L_SSS, 19 L_in, 20 vis), 21 1/ca, 22 1/cc, 23 1.001 ln(o/alpha_min)
 * + 0.01 (culling constants the render kernels read; sssgs_project_fwd
 * writes them). The gradient record has the layout of fields 0..20
 * (d/dmx ... d/dvis); its fields 21..23 hold dL/dmu of the per-Gaussian
 * shading (sssgs_shade_gaussians_bwd) and are zero otherwise. */

/* Render conventions. Defaults (sssgs_cfg_default): tile 16, batch 32, dilation 0.3 px^2,
 * det_eps 1e-6 px^4, z_near 0.2, alpha_min 1/255, alpha_max 0.99, T_min 1e-4,
 * A_eps 1e-6. All values are float32. */
typedef struct sssgs_cfg {
    int32_t tile;        /* tile edge in pixels: 8, 16 or 32 */
    int32_t batch;       /* splats staged per round by the one-warp render kernels: 32 or 64 (0 = 32) */
    float dilation;      /* low-pass dilation added to the 2D covariance diagonal */
    float det_eps;       /* cull if det(Sigma') <= det_eps (guards the conic inverse) */
    float z_near;        /* cull if view depth < z_near */
    float alpha_min;     /* skip contributions below this alpha */
    float alpha_max;     /* clamp alpha */
    float T_min;         /* stop before transmittance falls below T_min */
    float A_eps;         /* shading normalises by max(A, A_eps) */
} sssgs_cfg;

/* One view/light pair. The caller fills the first block; sssgs_plan fills
 * the layout block. The same array must be passed as host copy (h_pairs) and
 * device copy (d_pairs, 16-byte aligned) to every call. 128 bytes. */
typedef struct sssgs_pair {
    float R[9];          /* world->camera rotation, row-major */
    float t[3];          /* x_cam = R x_world + t */
    float fx, fy, cx, cy;
    float light[3];      /* OLAT point-light position (world) */
    int32_t W, H;        /* image size in pixels */
    int32_t g_begin;     /* this pair renders Gaussians [g_begin, g_begin + g_count) */
    int32_t g_count;     /*   of the scene arrays */
    /* --- filled by sssgs_plan --- */
    int32_t tiles_x, tiles_y;
    int32_t tile_offset;   /* first global tile id of this pair */
    int32_t pad0, pad1;
    int64_t pixel_offset;  /* first global pixel of this pair (row-major within the pair) */
    int64_t item_offset;   /* first (pair, Gaussian) item row of this pair */
} sssgs_pair;

/* Totals of a planned batch. */
typedef struct sssgs_plan_info {
    int64_t n_items;       /* sum of g_count */
    int64_t n_pixels;      /* sum of W*H */
    int32_t n_tiles;       /* sum of tiles_x*tiles_y */
    int32_t tile_bits;     /* bits needed for a global tile id */
} sssgs_plan_info;

/* Per-Gaussian parameters (float32 device arrays, concatenated over scenes):
 * mu N*3, log_s N*3, quat N*4 (w,x,y,z; normalised inside), logit_o N,
 * normal N*3, base N*3, rough N, metal N, sss N, vis N.
 * vis_item (optional, NULL: unused): the visibility per item (pair,
 * Gaussian) instead of per Gaussian, e.g. the SH visibility term evaluated at
 * each pair's light direction (sssgs_vis_sh_fwd); when set, the projection and
 * the network read v from it and vis is not read. */
typedef struct sssgs_scene {
    const float *mu, *log_s, *quat, *logit_o, *normal, *base, *rough, *metal, *sss, *vis;
    int64_t n;
    const float* vis_item;
} sssgs_scene;

/* Gradients of the same shapes (accumulated). Any pointer may be NULL to skip.
 * vis_item: with a per-item visibility, sssgs_project_bwd accumulates dL/dv
 * per item here (n_items floats) instead of into vis. */
typedef struct sssgs_scene_grad {
    float *mu, *log_s, *quat, *logit_o, *normal, *base, *rough, *metal, *sss, *vis;
    float* vis_item;
} sssgs_scene_grad;

enum { SSSGS_MLP_BASIC = 0, SSSGS_MLP_PE6 = 1, SSSGS_MLP_PAPER = 2 };
enum { SSSGS_FP32 = 0, SSSGS_BF16 = 1 };

/* Residual / incident-light MLP (Eq. 6; Appendix E "Network"). Input per
 * (pair, Gaussian), with w_out = unit(camera - mu), w_in = unit(light - mu):
 *   BASIC: [mu, w_out, w_in] (width[0] = 9)
 *   PE6:   [sin(2^k pi mu), cos(2^k pi mu) (k<6, 36), mu, w_out, w_in, n,
 *           |light - mu|, v] = 50, zero-padded (width[0] = 64)
 * BASIC / PE6: linear layers W[l] (width[l+1] x width[l], row-major, float32)
 * + b[l], ReLU between layers; width[n_layers] = 4: sigmoid -> L_SSS (3),
 * ReLU -> L_in.
 *   PAPER (the network of Appendix E): input [n, q/|q| (4), exp(log_s) (3),
 *           w_in, w_out, |light - mu|, v, sin(2^k pi mu), cos(2^k pi mu)
 *           (k<4, 24)] = 42, zero-padded to 48. n_layers = 6 and width =
 *           {48, 64, 32, 32, 32, 1, 3} (checked); the matrices by role:
 *           W[0] 64x48, W[1] 32x64, W[2] 32x32 (trunk, Leaky-ReLU slope 0.01
 *           after each), W[3] 32x32 (incident hidden, Leaky-ReLU), W[4] 1x32
 *           (incident output, ReLU -> L_in), W[5] 3x32 on the trunk output
 *           (sigmoid -> L_SSS). FP32 precision only. */
typedef struct sssgs_mlp {
    int32_t kind;        /* SSSGS_MLP_BASIC, SSSGS_MLP_PE6 or SSSGS_MLP_PAPER */
    int32_t n_layers;    /* 2 .. SSSGS_MAX_LAYERS */
    int32_t precision;   /* SSSGS_FP32 (CUDA cores) or SSSGS_BF16 (tensor cores, FP32 accumulate) */
    int32_t width[SSSGS_MAX_LAYERS + 1];
    const float* W[SSSGS_MAX_LAYERS];
    const float* b[SSSGS_MAX_LAYERS];
} sssgs_mlp;

typedef struct sssgs_mlp_grad {
    float* W[SSSGS_MAX_LAYERS];
    float* b[SSSGS_MAX_LAYERS];
} sssgs_mlp_grad;

/* ---------------------------------------------------------------------- */

const char* sssgs_version(void);

/* Number of kernels libsssgs has launched in this process (host-side counter,
 * incremented at every launch site; for accounting in benchmarks). */
uint64_t sssgs_launch_count(void);
const char* sssgs_strerror(int code);
void sssgs_cfg_default(sssgs_cfg* cfg);

/* Fill the layout fields of pairs[0..n_pairs) (host memory) and the totals.
 * Pairs must have W, H in 1..16384 and g_count >= 0. Host only. */
int sssgs_plan(sssgs_pair* pairs, int n_pairs, const sssgs_cfg* cfg, sssgs_plan_info* info);

/* a0 -- network forward (Eq. 6). out[n_items*4] = (L_SSS rgb, L_in) per item
 * (16-byte aligned). d_status (device int32, may be NULL) receives
 * SSSGS_STATUS_TIMEOUT if a tensor-core wait ran out. */
int sssgs_mlp_fwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                  int n_pairs, const sssgs_scene* scene, float* out, int32_t* d_status,
                  sssgs_stream stream);

/* a5 -- network backward. Reads dL/d(L_SSS, L_in) from the gradient records
 * drec (fields 16..19), accumulates weight/bias gradients into grad and
 * writes (overwrites) the per-item input gradients
 * dx_items[n_items*SSSGS_DX] = (dmu 3, dn 3, dv 1, dquat 4, dlog_s 3); the
 * last two are nonzero only for SSSGS_MLP_PAPER. Items whose four upstream values
 * are all exactly zero (Gaussians that reach no pixel of their view) add
 * exactly zero to every gradient; the BF16 path leaves them out of the
 * network and writes their dx_items as 0. BF16 path: n_items < 2^32.
 * workspace: sssgs_mlp_workspace_bytes(mlp, n_items) bytes (any alignment >= 256). */
size_t sssgs_mlp_workspace_bytes(const sssgs_mlp* mlp, int64_t n_items);
int sssgs_mlp_bwd(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                  int n_pairs, const sssgs_scene* scene, const float* drec,
                  const sssgs_mlp_grad* grad, float* dx_items,
                  void* workspace, size_t workspace_bytes, int32_t* d_status, sssgs_stream stream);

/* sssgs_mlp_bwd with the upstream gradient read from dout: item m's four
 * values dL/d(L_SSS 3, L_in) at dout[m * dout_stride + 0..3] (dout 16-byte
 * aligned, dout_stride a multiple of 4 and >= 4). sssgs_mlp_bwd is this call
 * with dout = drec + 16, dout_stride = SSSGS_REC; the many-light path passes
 * its per-(view, light, item) gradient rows with stride 4. */
int sssgs_mlp_bwd_strided(const sssgs_mlp* mlp, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                          int n_pairs, const sssgs_scene* scene, const float* dout, int64_t dout_stride,
                          const sssgs_mlp_grad* grad, float* dx_items,
                          void* workspace, size_t workspace_bytes, int32_t* d_status, sssgs_stream stream);

/* a1 -- EWA projection (Eq. 1, Eq. 2). Per item writes the packed record
 * (rec[n_items*24], features copied from the scene and from mlp_out[n_items*4];
 * mlp_out == NULL leaves fields 16..19 zero, as the many-light path wants)
 * and the inclusive tile rectangle rect[n_items*4] = (tx0, tx1, ty0, ty1) of
 * the ellipse {p <= ln(o / alpha_min)}; tx0 > tx1 marks a culled item. */
int sssgs_project_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                      int n_pairs, const sssgs_scene* scene, const float* mlp_out,
                      float* rec, int32_t* rect, sssgs_stream stream);

/* a2 -- tile binning + stable radix sort. Orders the items of each pair by
 * (float32 depth bits of rec[6], item), emits one instance per tile of each
 * rectangle, and stably sorts instances by global tile id, giving the order
 * (tile, depth, item). Outputs: vals[capacity] item id per instance,
 * ranges[n_tiles*2] = [start, end) per global tile, d_count = number of
 * instances (device int64). If more than `capacity` instances arise,
 * SSSGS_STATUS_CAPACITY is set in *d_status and lists are truncated.
 * workspace: sssgs_bin_workspace_bytes(n_items, capacity, n_tiles) bytes,
 * 256-byte aligned (SSSGS_ERR_INVALID_ARG otherwise). */
size_t sssgs_bin_workspace_bytes(int64_t n_items, int64_t capacity, int32_t n_tiles);
int sssgs_bin_sort(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                   int n_pairs, const float* rec, const int32_t* rect, int64_t capacity,
                   uint32_t* vals, uint32_t* ranges, int64_t* d_count, int32_t* d_status,
                   void* workspace, size_t workspace_bytes, sssgs_stream stream);

/* Allocation-free sssgs_bin_sort. The paper has no counterpart: this is an
 * interface for callers that cannot call cudaMalloc -- plug-ins whose host
 * application owns all device memory, and real-time loops that cannot afford
 * cudaMalloc's implicit device synchronisation. Same arguments and results as
 * sssgs_bin_sort, without the workspace: the sort runs in a scratch array of
 * SSSGS_STATIC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library keeps until the process exits.
 * Limits: n_items <= SSSGS_STATIC_MAX_ITEMS and capacity <=
 * SSSGS_STATIC_MAX_INSTANCES; larger problems return SSSGS_ERR_TOO_LARGE
 * before anything is launched and leave every output untouched. A missing
 * buffer, a negative capacity or a pair table with negative counts or no
 * tiles returns SSSGS_ERR_INVALID_ARG, also before any launch.
 * The first call on a device (with that device current) looks up the
 * scratch address and caches it; make it before any stream capture. The
 * cached address belongs to the device's primary context: after
 * cudaDeviceReset do not call this entry point again in that process. All
 * calls share the scratch, which keeps the last call's contents (nothing in
 * it needs to start at zero); calls that overlap on the GPU race, so
 * serialise them. */
#define SSSGS_STATIC_MAX_ITEMS 65536
#define SSSGS_STATIC_MAX_INSTANCES 524288
#define SSSGS_STATIC_SCRATCH_BYTES 9437184
int sssgs_bin_sort_static(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                          int n_pairs, const float* rec, const int32_t* rect, int64_t capacity,
                          uint32_t* vals, uint32_t* ranges, int64_t* d_count, int32_t* d_status,
                          sssgs_stream stream);

/* a3 -- front-to-back compositing (Eq. 3) into gbuf[n_pixels*16] (15 features
 * weighted by w_i = T_i alpha_i, then the final T) and last[n_pixels] (one past
 * the list position of the last contribution). */
int sssgs_composite_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                        int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                        float* gbuf, uint32_t* last, sssgs_stream stream);

/* a4 -- deferred shading (Eq. 4, Eq. 7): img[n_pixels*3] from gbuf. */
int sssgs_shade_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                    int n_pairs, const float* gbuf, float* img, sssgs_stream stream);

/* a4 backward: dgbuf[n_pixels*16] (written, not accumulated) from dimg. */
int sssgs_shade_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                    int n_pairs, const float* gbuf, const float* dimg, float* dgbuf,
                    sssgs_stream stream);

/* a3 backward: back-to-front replay from the stored final T (no per-pixel
 * lists kept). Accumulates per-item gradient records into drec[n_items*24].
 * The unfused path: 8 x 8 and 16 x 16 tiles (SSSGS_ERR_UNSUPPORTED for 32 x
 * 32; the fused sssgs_render_bwd takes every tile edge). */
int sssgs_composite_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                        int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                        const float* gbuf, const uint32_t* last, const float* dgbuf,
                        float* drec, sssgs_stream stream);

/* Fused a3+a4 forward: composite then shade in one pass; writes gbuf, last, img.
 * One 32-thread block per 8 x 8 sub-tile (two pixels per thread) of every
 * tile of every pair (tile edge cfg->tile: 8, 16 or 32; cfg->batch splats
 * staged per round); images are bit-identical across tile edges and batches.
 * d_stats (device uint64[2], may be NULL) accumulates the number of
 * contributions (pixel-Gaussian pairs composited) and the tile-list positions
 * each pixel considered (up to the splat that stopped it, else the list end). */
int sssgs_render_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                     int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                     float* gbuf, uint32_t* last, float* img, uint64_t* d_stats, sssgs_stream stream);

/* Fused a4+a3 backward. Upstream gradient either dimg[n_pixels*3], or (dimg ==
 * NULL) the L1 loss  l1_scale * sum |img - target|  with optional per-pixel
 * weights (NULL = 1): dimg = l1_scale * w * sign(img - target). Accumulates drec;
 * its visibility field (20) is left untouched, since the shading does not read
 * the visibility channel and its gradient is exactly zero.
 * One 32-thread block per 8 x 8 sub-tile (tile edge 8, 16 or 32). Errors:
 * SSSGS_ERR_INVALID_ARG for a missing buffer, misaligned records, G-buffer,
 * pair table or ranges (16 bytes), a tile edge other than 8/16/32 or a batch
 * other than 0/32/64; SSSGS_ERR_CUDA if the launch fails.
 * d_stats (device uint64[2], may be NULL) accumulates the contributions
 * replayed and the alpha evaluations (list positions below each pixel's end). */
int sssgs_render_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                     int n_pairs, const float* rec, const uint32_t* vals, const uint32_t* ranges,
                     const float* gbuf, const uint32_t* last, const float* img,
                     const float* dimg, const float* target, const float* weight, float l1_scale,
                     float* drec, uint64_t* d_stats, sssgs_stream stream);

/* Schedule autotuner. The paper renders with the tile rasterizer of 3D
 * Gaussian splatting (Sec. 4.1 "Implementation Details") and fixes no tile
 * shape; here the tile edge (cfg.tile: 8, 16, 32) and the per-block splat
 * batch of the one-warp render kernels (cfg.batch: 32, 64) are chosen per
 * scene by measurement. For the pairs of one scene, every candidate
 * (tiles[i], batches[j]) runs the stages whose work depends on the schedule
 * -- sssgs_project_fwd, sssgs_bin_sort, sssgs_render_fwd and sssgs_render_bwd
 * with the upstream gradient dimg -- once to warm up and check the instance
 * count, then `reps` times between two CUDA events on `stream`.
 * results[i * n_batches + j] receives the candidate's mean milliseconds per
 * pass (ms, -1 if not run), its instance count and status (0, or
 * SSSGS_STATUS_CAPACITY when its instances exceed buf->capacity; enlarge the
 * buffers and call again for it); *best becomes *base with the fastest
 * candidate's tile and batch.
 * h_pairs: the scene's pairs with the caller-filled fields (camera, light,
 * W, H, g_begin, g_count); the layout fields are planned per candidate and
 * the planned table is copied into buf->d_pairs. mlp_out: the network output
 * of these pairs (sssgs_mlp_fwd; it does not depend on the schedule).
 * Buffers (device, the caller's scratch; their contents are overwritten):
 * sized for the largest candidate -- ranges for max_tiles tiles (the smallest
 * tile edge), vals for `capacity` instances and the bin/sort workspace for
 * (n_items, capacity, max_tiles); records, rectangles, G-buffer, last index,
 * image and gradient records for the pairs' items and pixels.
 * Blocking: the call synchronises `stream` (it reads the instance counts and
 * the events), so it runs outside stream capture, at set-up.
 * Errors: SSSGS_ERR_INVALID_ARG for a missing buffer, reps outside 1..1000, a
 * batch other than 32 or 64, or a candidate needing more than max_tiles
 * tiles; SSSGS_ERR_WORKSPACE for a bin/sort workspace too small for a
 * candidate, or when no candidate fits `capacity`; errors of the stages
 * above as they return them. */
typedef struct sssgs_tune_buffers {
    sssgs_pair* d_pairs;        /* n_pairs entries, 16-byte aligned */
    float* rec;                 /* n_items * SSSGS_REC */
    int32_t* rect;              /* n_items * 4 */
    uint32_t* vals;             /* capacity */
    int64_t capacity;
    uint32_t* ranges;           /* max_tiles * 2 */
    int32_t max_tiles;
    int32_t pad;
    int64_t* d_count;
    int32_t* d_status;
    void* workspace;            /* bin/sort workspace, 256-byte aligned */
    size_t workspace_bytes;
    float* gbuf;                /* n_pixels * SSSGS_GBUF */
    uint32_t* last;             /* n_pixels */
    float* img;                 /* n_pixels * 3 */
    float* drec;                /* n_items * SSSGS_REC (accumulated into; scratch) */
    const float* dimg;          /* n_pixels * 3 upstream gradient */
} sssgs_tune_buffers;

typedef struct sssgs_tune_result {
    int32_t tile, batch;
    int32_t status;             /* 0 measured, SSSGS_STATUS_CAPACITY not run */
    int32_t reps;
    int64_t instances;
    float ms;                   /* mean milliseconds per pass of the four stages; -1 if not run */
    float reserved;
} sssgs_tune_result;

int sssgs_autotune(const sssgs_cfg* base, const sssgs_pair* h_pairs, int n_pairs, const sssgs_scene* scene,
                   const float* mlp_out, const sssgs_tune_buffers* buf, const int32_t* tiles, int n_tiles,
                   const int32_t* batches, int n_batches, int reps, sssgs_tune_result* results,
                   sssgs_cfg* best, sssgs_stream stream);

/* Many lights per view. A training batch of the paper's light-stage data
 * holds one camera view under several point lights (Sec. 4.1 "Dataset": fixed
 * light positions, each view captured under all of them), and a relit view
 * under an environment map is a sum of such renders weighted by environment
 * samples (App. C "Image Based Lighting"). The geometry of a view does not
 * depend on the light: projection, tile binning/sort and every alpha of the
 * compositing (Eq. 3) are computed once per view; the network output
 * (L_SSS, L_in; Eq. 6), its composited channels and the shading (Eq. 4,
 * Eq. 7) are per light. Results equal rendering each (view, light) pair on its
 * own.
 *
 * Views: h_views/d_views[n_views] planned with sssgs_plan (their light field
 * is unused); rec, vals, ranges from sssgs_project_fwd (mlp_out NULL) and
 * sssgs_bin_sort on the views. n_lights: 1, 2, 4 or 8 lights per view, with
 * positions lights[(v * n_lights + l) * 3] (device). mlp_out: the network
 * output of the (view, light) pair table, pair v * n_lights + l being view v's
 * camera and scene with light l, as sssgs_mlp_fwd on that table writes it:
 * row n_lights * item_offset_v + l * g_count_v + k for item k of view v.
 * G-buffer per view pixel: gbuf[n_view_pixels * (12 + 4 n_lights)] = depth,
 * n 3, base 3, rough, metal, sss, vis, T, then (L_SSS 3, L_in) per light.
 * Images: with env_w == NULL one image per (view, light) pair in pair order
 * (pixel n_lights * pixel_offset_v + l * W_v * H_v + j * W_v + i); with
 * env_w[n_views * n_lights] (device weights) one image per view (view pixel
 * layout) holding sum_l env_w[v * n_lights + l] * image of light l.
 * d_stats as for sssgs_render_fwd.
 * Errors: SSSGS_ERR_INVALID_ARG for a missing buffer, n_lights not 1, 2, 4
 * or 8, or rec / mlp_out / gbuf not 16-byte (ranges not 8-byte) aligned;
 * SSSGS_ERR_UNSUPPORTED unless cfg->tile == 16; SSSGS_ERR_CUDA if a launch
 * fails. */
int sssgs_render_ml_fwd(const sssgs_cfg* cfg, const sssgs_pair* h_views, const sssgs_pair* d_views, int n_views,
                        int n_lights, const float* lights, const float* rec, const float* mlp_out,
                        const uint32_t* vals, const uint32_t* ranges, float* gbuf, uint32_t* last, float* img,
                        const float* env_w, uint64_t* d_stats, sssgs_stream stream);

/* Backward of sssgs_render_ml_fwd (per-light images, env_w NULL). Upstream
 * gradient per (view, light) image in pair pixel order: dimg, or (dimg ==
 * NULL) the L1 loss l1_scale * sum |img - target|. Accumulates the per-view
 * gradient records drec[n_view_items * 24] (geometry and the light-independent
 * features; fields 16..20 untouched, 20 being the visibility feature, whose
 * gradient is exactly zero because the shading does not read it) and
 * dmlp[rows * 4] = dL/d(L_SSS 3, L_in)
 * per (view, light, item) row in mlp_out's layout, for
 * sssgs_mlp_bwd_strided(dout = dmlp, dout_stride = 4) on the pair table.
 * Errors as for sssgs_render_ml_fwd, and SSSGS_ERR_INVALID_ARG without drec,
 * dmlp, or an upstream (dimg, or img and target). */
int sssgs_render_ml_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_views, const sssgs_pair* d_views, int n_views,
                        int n_lights, const float* lights, const float* rec, const float* mlp_out,
                        const uint32_t* vals, const uint32_t* ranges, const float* gbuf, const uint32_t* last,
                        const float* img, const float* dimg, const float* target, float l1_scale, float* drec,
                        float* dmlp, uint64_t* d_stats, sssgs_stream stream);

/* Ray-traced visibility and the SH visibility term (Sec. 3.2 "Incident
 * Light": visibility is estimated by tracing rays through the Gaussians with a
 * BVH and learnt as a per-Gaussian SH visibility term v; App. E "Losses":
 * lambda_raytrace = 0.01).
 *
 * Tracing: the visibility of item m (pair p, Gaussian i) is the transmittance
 * of the segment from mu_i to p's light through every other Gaussian j:
 * prod_j (1 - alpha_j), alpha_j = min(alpha_max, o_j exp(-q/2)), q the
 * minimum of the Mahalanobis distance (x - mu_j)^T Sigma_j^-1 (x - mu_j) over
 * the ray, counted when that minimum lies inside the segment and alpha_j >=
 * alpha_min. Stops once the product is below 1e-5.
 *
 * sssgs_bvh_build: a linear BVH (Morton order of the means, 30-bit codes) over
 * the boxes bounding each Gaussian's support {alpha >= alpha_min}. Writes
 * bvh[sssgs_bvh_floats(n)] (nodes and per-Gaussian tracing records); the
 * caller allocates it and the workspace (sssgs_bvh_workspace_bytes, 256-byte
 * aligned). The BVH holds the scene's geometry as it is when built.
 * Errors: SSSGS_ERR_INVALID_ARG for missing scene arrays or bvh, bvh not
 * 16-byte or workspace not 256-byte aligned; SSSGS_ERR_WORKSPACE for a
 * missing or short workspace; SSSGS_ERR_TOO_LARGE for n >= 2^30. n == 0 is a
 * no-op. */
int64_t sssgs_bvh_floats(int64_t n_gaussians);
size_t sssgs_bvh_workspace_bytes(int64_t n_gaussians);
int sssgs_bvh_build(const sssgs_cfg* cfg, const sssgs_scene* scene, float* bvh, void* workspace,
                    size_t workspace_bytes, sssgs_stream stream);
/* One ray per item of the pairs: vis_traced[n_items] (overwritten), from a
 * BVH of the same scene. SSSGS_ERR_INVALID_ARG for a missing buffer or a bvh
 * not 16-byte aligned. */
int sssgs_trace_visibility(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                           const sssgs_scene* scene, const float* bvh, float* vis_traced, sssgs_stream stream);

/* SH visibility: vis_sh[N*16] real spherical-harmonic coefficients per
 * Gaussian (degree 3, orthonormal, no Condon-Shortley phase; index l^2 + l + m).
 * Forward: vis_item[m] = clamp(sum_k c_k Y_k(w), 0, 1), w = unit(light - mu)
 * of item m's pair. Backward: from dvis_item[n_items] accumulates dvis_sh and
 * the mean gradient dmu (through w); zero where the clamp is active.
 * SSSGS_ERR_INVALID_ARG for a missing buffer. */
int sssgs_vis_sh_fwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs, const sssgs_scene* scene,
                     const float* vis_sh, float* vis_item, sssgs_stream stream);
int sssgs_vis_sh_bwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs, const sssgs_scene* scene,
                     const float* vis_sh, const float* dvis_item, float* dvis_sh, float* dmu, sssgs_stream stream);

/* Ray-traced visibility loss per pair p: lambda_raytrace * mean over its items
 * of |vis_item - vis_traced| (the traced value a constant target). Adds
 * dL/dvis_item to dvis_item and the loss to d_loss[p] (caller-zeroed).
 * SSSGS_ERR_INVALID_ARG for a missing buffer. */
int sssgs_vis_loss(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs, const float* vis_item,
                   const float* vis_traced, float lambda_raytrace, float* dvis_item, float* d_loss,
                   sssgs_stream stream);

/* Diagnostic of the failure-detection path: one thread waits on an mbarrier
 * that nothing arrives on, for at most limit_cycles SM clock cycles (1 ..
 * 4e9), then sets SSSGS_STATUS_TIMEOUT in *d_status (device int32) and
 * returns, as the tensor-core kernels do when a wait runs out. The context
 * stays usable. */
int sssgs_selftest_wait_timeout(int32_t* d_status, int64_t limit_cycles, sssgs_stream stream);

/* Per-Gaussian shading: the paper's "w/o Deferred" ablation (appendix
 * "Ablation"). Each Gaussian is shaded at its own mean with its own attributes
 * (Eq. 4 BRDF, Eq. 7 blend) and the colours are composited (Eq. 3), black
 * background. Forward: sssgs_project_fwd -> sssgs_bin_sort (on rec) ->
 * sssgs_shade_gaussians_fwd (rec -> rec_colors: a copy of the records whose
 * feature fields carry the colour (6..8) and zeros (9..20)) ->
 * sssgs_composite_fwd on rec_colors -> sssgs_colors_to_image (img = G-buffer
 * channels 0..2). Backward: sssgs_colors_to_image_bwd (dimg -> dgbuf) ->
 * sssgs_composite_bwd on rec_colors -> sssgs_shade_gaussians_bwd (replaces
 * drec fields 6..8, dL/dcolour, by the gradients of the shaded attributes in
 * fields 7..19 and of the mean in 21..23) -> sssgs_mlp_bwd ->
 * sssgs_project_bwd. Errors: SSSGS_ERR_INVALID_ARG for a missing buffer,
 * rec_colors aliasing rec, or a G-buffer / dgbuf not 16-byte aligned. */
int sssgs_shade_gaussians_fwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                              const sssgs_scene* scene, const float* rec, float* rec_colors, sssgs_stream stream);
int sssgs_shade_gaussians_bwd(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                              const sssgs_scene* scene, const float* rec, float* drec, sssgs_stream stream);
int sssgs_colors_to_image(const sssgs_pair* h_pairs, int n_pairs, const float* gbuf, float* img,
                          sssgs_stream stream);
int sssgs_colors_to_image_bwd(const sssgs_pair* h_pairs, int n_pairs, const float* dimg, float* dgbuf,
                              sssgs_stream stream);

/* Training losses (Appendix E "Losses").
 * Image loss per pair p: L_img = (1 - lambda_dssim) L1 + lambda_dssim (1 - SSIM)
 * over the pair's pixels and channels (L1: mean |img - target|; SSIM: Wang et
 * al. 2004, 11 x 11 Gaussian window with sigma 1.5, zero padding, C1 = 0.01^2,
 * C2 = 0.03^2, mean over pixels and channels). Writes (overwrites)
 * dimg[n_pixels*3] = dL/dimg (sum over pairs of L_img) for sssgs_render_bwd
 * with a dimg upstream, and adds each pair's L_img to d_loss[p] (device
 * float[n_pairs], caller-zeroed). workspace: sssgs_image_loss_workspace_bytes
 * (9 floats per pixel). lambda_dssim in [0, 1] (the paper uses 0.2). */
size_t sssgs_image_loss_workspace_bytes(int64_t n_pixels);
int sssgs_image_loss(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs,
                     const float* img, const float* target, float lambda_dssim, float* dimg, float* d_loss,
                     void* workspace, size_t workspace_bytes, sssgs_stream stream);

/* Incident-light constraint per pair p (App. E): L_inc = lambda_incident *
 * mean over the pair's items of |min(L_in, 1) - v|, with L_in and v read from
 * the records (fields 19, 20). Adds dL/dL_in to drec field 19 and dL/dv to
 * field 20 (call after sssgs_render_bwd, before sssgs_mlp_bwd) and L_inc to
 * d_loss[p]. The paper uses lambda_incident = 0.02. */
int sssgs_incident_loss(const sssgs_pair* h_pairs, const sssgs_pair* d_pairs, int n_pairs, const float* rec,
                        float lambda_incident, float* drec, float* d_loss, sssgs_stream stream);

/* a5 -- projection backward. For every Gaussian of the scene, sums over the
 * pairs that render it: the gradient records drec (geometry via Eq. 2 and the
 * covariance parameterisation, features directly) and, if dx_items != NULL,
 * the network-input gradients from sssgs_mlp_bwd (dx_items[n_items*SSSGS_DX]).
 * Either may be NULL (the many-light path sums its view records and its
 * (view, light) network-input gradients in two calls). Accumulates into grad. */
int sssgs_project_bwd(const sssgs_cfg* cfg, const sssgs_pair* h_pairs, const sssgs_pair* d_pairs,
                      int n_pairs, const sssgs_scene* scene, const float* drec,
                      const float* dx_items, const sssgs_scene_grad* grad, sssgs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SSSGS_H */
