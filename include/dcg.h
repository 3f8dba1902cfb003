/*
 * dcg.h -- C ABI of the B300 (sm_103a) chunked Gaussian-splatting mapper hot path.
 *
 * The calls follow the optimisation pass of a chunk-based 3DGS mapper
 * (DiskChunGS, Sec. III-D "Chunk 3DGS Mapping" and Sec. III-E "Optimization",
 * Fig. 2): compute chunk ids of new Gaussians (Eq. 5, Eq. 6), cull chunks
 * against a keyframe frustum, make the visible chunks resident under a
 * Gaussian budget with LRU eviction to a slower tier, gather the visible
 * Gaussians into one active buffer, rasterise RGB and depth, back-propagate
 * the loss of Eq. 2-4 to every Gaussian parameter and the camera pose, and
 * write the updated Gaussians back to their chunks.
 *
 * Conventions shared by every call
 *  - Pointers marked (dev) are CUDA device pointers, (host) are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are stream-ordered and asynchronous unless stated otherwise.
 *  - Argument and capacity errors are returned synchronously.  Errors found
 *    by a kernel (a chunk coordinate outside the +-2^20 range, an instance or
 *    list capacity overflow, a bounded wait that gave up) are written to a
 *    device error word; dcg_sync() and the calls documented as synchronising
 *    return them.  No kernel traps or asserts.
 *  - A dcg_ctx is not thread-safe; use one per host thread.
 *  - All device memory the library needs is allocated in dcg_create /
 *    dcg_state_create from the capacities in dcg_config; the render and chunk
 *    calls allocate nothing.
 */
#ifndef DCG_H
#define DCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DCG_OK = 0,
  DCG_ERR_ARG = 1,       /* invalid argument (null pointer, size <= 0, too many views ...) */
  DCG_ERR_OOM = 2,       /* allocation at create time failed */
  DCG_ERR_CUDA = 3,      /* a CUDA runtime call failed; dcg_last_error has the text */
  DCG_ERR_BUDGET = 4,    /* the visible chunks alone exceed the device Gaussian budget */
  DCG_ERR_KEY_RANGE = 5, /* a chunk coordinate lies outside [-2^20, 2^20-1] (Eq. 6) */
  DCG_ERR_CAPACITY = 6,  /* a configured capacity (instances, pixels, chunks, host tier) was exceeded */
  DCG_ERR_TIMEOUT = 7,   /* a bounded device-side wait gave up: the MLP's tcgen05 GEMM waits on
                            its own mbarriers (TMA arrivals, MMA completion) for at most about two
                            seconds each; no render kernel waits on another block or on a flag */
  DCG_ERR_FAULT = 8,     /* a chunk load failed verification, or an injected host-side fault */
  DCG_ERR_STATE = 9,     /* call order violated (e.g. backward without a forward) */
  DCG_ERR_BOUNDS = 10    /* bounds-check build only (libdcg_checks.so): a kernel met an index outside
                            its buffer, skipped the access and recorded it; reported by the next
                            dcg_sync */
} dcg_status;

typedef struct dcg_ctx dcg_ctx;
typedef struct dcg_render_state dcg_render_state;

/* Pinhole camera, x right, y down, z forward.  Pixel (x, y) is sampled at
 * image-plane point (x, y) with u = fx X/Z + cx, v = fy Y/Z + cy.
 * Tcw is the row-major 4x4 world->camera rigid transform. */
typedef struct {
  float fx, fy, cx, cy;
  int32_t W, H;
  float Tcw[16];
  float znear, zfar;
} dcg_camera;

/* Gaussians, component-major ("planar"): component c of Gaussian i is
 * data[c * stride + i].  F = 11 + 3 (deg+1)^2 components:
 *   0..2 mean, 3..5 log-scale, 6..9 quaternion (w,x,y,z; normalised on use),
 *   10 opacity logit, 11 + 3k + ch SH coefficient k of channel ch.
 * The 3DGS representation with SH up to degree 3 (Sec. II). */
typedef struct {
  float* data;       /* (dev) */
  int64_t stride;    /* >= number of Gaussians */
  int32_t sh_degree; /* 0..3 */
  int32_t pad;
} dcg_gaussians;

typedef struct {
  float chunk_size;        /* s of Eq. 5, metres (the paper uses 10 m) */
  int32_t sh_degree;       /* 0..3 */
  int64_t device_budget;   /* max resident Gaussians on the device (paper: 1.5 M) */
  int64_t host_capacity;   /* Gaussians the pinned host tier (stand-in for disk) can hold */
  int32_t max_chunks;      /* chunk table capacity */
  int32_t max_views;       /* views per render call (<= 16) */
  int64_t max_active;      /* Gaussians per render call / active buffer; max_views max_active <= 2^28 */
  int64_t max_pixels;      /* total pixels over the views of one render call */
  int64_t max_instances;   /* (view, tile, Gaussian) instances per render call */
  int32_t tile_w, tile_h;  /* default blend tile: 16x16, 32x16 or 32x32 */
  int32_t stage;           /* default Gaussians staged per block batch: 64..256; 32 selects the
                              warp-per-block blend kernels, 16 the half-warp-per-half-block ones */
  float dfar;              /* distance filter of the chunk cull, metres */
  int32_t page_gaussians;  /* Gaussians per device/host page (power of two) */
  int32_t flags;           /* bit 0: backward blend accumulates per-lane shared slots instead of
                              reducing each Gaussian across the warp (same result); bit 1: the
                              half-warp backward (stage 16) puts pixels on the lanes, one Gaussian
                              per half block and step, instead of Gaussians on the lanes with the
                              half block's pixels in turn (same result); bit 2: verify every chunk
                              load (a checksum of the host pages against one of the pages that
                              arrived, compared before dcg_gather_active returns; a chunk that
                              fails is dropped and the call returns DCG_ERR_FAULT, so a retry
                              loads it again); others 0 */
  int32_t with_moments;    /* 1: every Gaussian stores its Adam moments m and v beside its
                              parameters (pages, host tier and active buffer hold 3 F components);
                              0 (default): parameters only */
} dcg_config;

/* Fill *cfg with defaults (s = 4 m, degree 3, budget 6 M, 8 views, 16x16
 * tiles with the half-warp blends (stage 16) ...). */
void dcg_config_default(dcg_config* cfg);

/* Create a context on the current CUDA device; allocates the chunk table,
 * the device page pool (device_budget), the pinned host tier (host_capacity),
 * the active buffer (max_active) and one render state.  Synchronous. */
dcg_status dcg_create(const dcg_config* cfg, dcg_ctx** out);
dcg_status dcg_destroy(dcg_ctx* ctx);

/* Text of the last error on this context (valid until the next call). */
const char* dcg_last_error(const dcg_ctx* ctx);

/* Synchronise `stream` and return the first device-detected error since the
 * last dcg_sync (then clear it). */
dcg_status dcg_sync(dcg_ctx* ctx, void* stream);

/* ---------------------------------------------------------------- chunks
 * Eq. 5 / Eq. 6: chunk coordinate floor((p + s/2)/s) per axis, evaluated in
 * FP32 (one rounding for the add, one for the divide, then floor), and
 * EncodedID = (cx+2^20) 2^42 + (cy+2^20) 2^21 + (cz+2^20).
 * dcg_chunk_keys: keys_out[i] (dev, n) for means (dev, [n,3] row-major);
 * a coordinate outside [-2^20, 2^20-1] or a non-finite mean writes key 0 and
 * raises DCG_ERR_KEY_RANGE at the next dcg_sync. */
dcg_status dcg_chunk_keys(dcg_ctx* ctx, const float* means, int64_t n, uint64_t* keys_out, void* stream);

/* dcg_chunk_table_update: insert n new Gaussians (dev, planar with `stride`,
 * the context's SH degree) into the chunk table (Sec. III-D: "an O(1) chunk
 * location" keyed by EncodedID).  Their keys are computed on the device, the
 * Gaussians are grouped by chunk (stable, in input order) and appended to
 * their chunks in the pinned host tier; new chunks are created.  A resident
 * chunk that receives Gaussians is written back (if dirty) and dropped from
 * the device so that the next gather reloads it whole.  keys_out (dev, n)
 * may be NULL.  Synchronises `stream`. */
dcg_status dcg_chunk_table_update(dcg_ctx* ctx, const float* params, int64_t stride, int64_t n,
                                  uint64_t* keys_out, void* stream);

/* Number of chunks, and per chunk (host arrays of length dcg_chunk_count, in
 * ascending EncodedID order -- the order every chunk index of this API uses):
 * integer coordinates [C,3], ids, Gaussian counts, resident flag, last access
 * step.  Any output may be NULL.  Synchronous host query. */
int32_t dcg_chunk_count(const dcg_ctx* ctx);
dcg_status dcg_chunk_info(const dcg_ctx* ctx, int32_t* coords, uint64_t* keys, int64_t* counts,
                          uint8_t* resident, int64_t* last_access);

/* Frustum cull of chunks (Sec. III-D "Frustum Culling"): six planes are
 * extracted from the view-projection matrix P Tcw (P maps u in [0,W],
 * v in [0,H], Z in [znear, zfar] to the clip cube); chunk k (the cube
 * [c s - s/2, c s + s/2)^3) is visible in view v iff for every plane the cube
 * vertex furthest along the plane normal is on the inner side, and the
 * distance from the camera centre to the cube is <= dfar.  FP64, fixed
 * evaluation order.  Outputs: mask_out (dev, [n_views, C] u8, may be NULL),
 * list_out (host, capacity C) = ascending chunk indices visible in any view,
 * *n_out (host) = their number.  The list is needed on the host by
 * dcg_gather_active, so the call waits for the cull: with mask_out it runs on
 * `stream` and synchronises it; without, it runs on a stream of the context
 * and waits for that only (work the caller queued keeps running). */
dcg_status dcg_cull_chunks(dcg_ctx* ctx, const dcg_camera* cams, int32_t n_views, uint8_t* mask_out,
                           int32_t* list_out, int32_t* n_out, void* stream);

/* The same cull, left on the device and not waited for: list_out (dev,
 * capacity = chunk count) ascending indices visible in any view, *n_out (dev)
 * their number, mask_out as above (dev, may be NULL).  Asynchronous on
 * `stream`; cams (1 to 16 views, independent of max_views) is copied into
 * the launch's parameters before return.  For
 * work that overlaps rendering (prefetch proposals on a side stream).  It has
 * its own scratch, so it may overlap dcg_cull_chunks, but two calls of it on
 * one context must not overlap on the GPU. */
dcg_status dcg_cull_chunks_async(dcg_ctx* ctx, const dcg_camera* cams, int32_t n_views, uint8_t* mask_out,
                                 int32_t* list_out, int32_t* n_out, void* stream);

/* Make the listed chunks (host, ascending chunk indices) resident and gather
 * their Gaussians into the library-owned active buffer (Sec. III-E: load
 * visible chunks, evict with LRU when over budget, index the visible
 * Gaussians).  Missing chunks are copied host->device on the context's copy
 * stream; when the budget would be exceeded, resident chunks not in the list
 * are evicted oldest first (ties by id), the fewest that make room, and dirty
 * ones are copied back to the host tier.  Active order: listed chunks in
 * ascending id, each in stored order.  *active_out receives a view of the
 * active buffer (stride = max_active), *n_active_out its size.
 * When the last call on the active buffer was a dcg_scatter_back of the
 * buffer itself and the list names the same chunks (all still resident), the
 * buffer is handed out again without a copy (it already holds their stored
 * values); otherwise a deferred write-back is completed first.
 * DCG_ERR_BUDGET if the listed chunks alone exceed the budget. */
dcg_status dcg_gather_active(dcg_ctx* ctx, const int32_t* chunk_list, int32_t n_chunks,
                             dcg_gaussians* active_out, int64_t* n_active_out, void* stream);

/* Inverse of the last dcg_gather_active: copy `active` (dev, planar, n must
 * equal the gathered count) back into the resident chunks and mark them
 * dirty, so that an eviction writes them to the host tier.  When `active` is
 * the library's own active buffer the copy is deferred (write-back): from
 * then on the buffer is the stored value of the gathered chunks, and writes
 * to it reach the map, until the library copies it into the chunk pages, which
 * it does before anything else reads, moves or replaces them (a gather of a
 * different list, dcg_flush, dcg_chunk_table_update, dcg_loop_closure).
 * A caller buffer is copied at once (the moments from the active buffer). */
dcg_status dcg_scatter_back(dcg_ctx* ctx, const dcg_gaussians* active, int64_t n, void* stream);

/* For every row j of the last gathered active set (n_active rows): the
 * chunk it belongs to (its index in the table now, as in dcg_chunk_info) in
 * chunk_out[j] and its row in that chunk's stored order in row_out[j] (dev
 * [n_active] each, either may be NULL).  Rows follow the gather: listed
 * chunks in ascending id, each with the count it had when gathered.
 * DCG_ERR_STATE without a valid gathered set (none yet, or after a loop
 * closure).  Asynchronous on `stream`; the table goes up from pinned staging
 * that the next call reuses once this upload has run.  The device copy of the
 * table is per context, so calls on one context must not overlap on the GPU
 * (one stream, or the caller orders them). */
dcg_status dcg_active_map(dcg_ctx* ctx, int32_t* chunk_out, int32_t* row_out, void* stream);

/* Complete a deferred write-back of the active buffer, copy every resident
 * dirty chunk back to the host tier and wait. */
dcg_status dcg_flush(dcg_ctx* ctx, void* stream);

/* Asynchronous load of proposed chunks (host, chunk indices in the order to load) on the copy
 * stream, overlapping the caller's rendering: listed non-resident chunks are
 * loaded in order while they fit in the budget and the page pool, evicting
 * (oldest first) only resident chunks that are neither listed nor part of the
 * last gather.  Loaded chunks count as accessed now.  *n_loaded (host, may be
 * NULL) receives the number of chunks whose load was started.  The exact cull
 * still decides what dcg_gather_active uses: a prefetch changes only where
 * the data already is, never what is rendered. */
dcg_status dcg_prefetch(dcg_ctx* ctx, const int32_t* chunk_list, int32_t n_chunks, int32_t* n_loaded, void* stream);

/* Chunks whose cube lies within `radius` of point `p` (host, 3 floats),
 * optionally only non-resident ones; ascending indices into list_out (host,
 * capacity dcg_chunk_count), count into *n_out.  Host query, synchronous. */
dcg_status dcg_chunks_near(const dcg_ctx* ctx, const float* p, float radius, int32_t only_nonresident,
                           int32_t* list_out, int32_t* n_out);

/* Tier statistics since creation (host outputs, any may be NULL): chunk
 * loads and evictions, bytes copied host->device and device->host, Gaussians
 * resident now. */
dcg_status dcg_tier_stats(const dcg_ctx* ctx, int64_t* loads, int64_t* evictions, int64_t* bytes_h2d,
                          int64_t* bytes_d2h, int64_t* resident);

/* Read n Gaussians of chunk `chunk` (ascending-id index) from the host tier
 * into params_out (host, planar with stride n).  For checks and checkpoints. */
dcg_status dcg_chunk_read(dcg_ctx* ctx, int32_t chunk, float* params_out, int64_t n);

/* Adam moments of chunk `chunk` as last written to the host tier (m_out and
 * v_out host, planar with stride n, n = the chunk's count; fresh Gaussians
 * start at zero).  Contexts with with_moments only (DCG_ERR_ARG otherwise). */
dcg_status dcg_chunk_read_moments(dcg_ctx* ctx, int32_t chunk, float* m_out, float* v_out, int64_t n);

/* ---------------------------------------------------------------- optimizer
 * The paper optimises the parameters of the active chunks against the loss
 * of Eq. 2-4 (Sec. III-E "Optimization") and keeps optimizer state per
 * Gaussian (Sec. III-F resets it after a loop closure).  With with_moments,
 * the Adam moments travel with their Gaussians: dcg_gather_active copies
 * them into the active buffer beside the parameters, dcg_scatter_back and
 * evictions write them back. */

/* Views of the active set's moments (library-owned device memory, planar
 * like the parameters, in the order of the last dcg_gather_active; valid
 * until dcg_destroy).  DCG_ERR_ARG without with_moments. */
dcg_status dcg_active_moments(dcg_ctx* ctx, dcg_gaussians* m, dcg_gaussians* v);

/* One Adam step (Kingma & Ba, bias-corrected) over the n Gaussians of the
 * gathered active set, in place on `params` (dev, usually the active view
 * from dcg_gather_active) and the active moments, with gradients `grads`
 * (dev, planar):
 *   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *   p <- p - lr[c] / (1 - b1^step) * m / (sqrt(v) / sqrt(1 - b2^step) + eps)
 * lr: host, F learning rates, one per component.  step >= 1 counts the steps
 * taken so far including this one.  Errors: DCG_ERR_ARG (hyper-parameters,
 * degree, strides, no moments), DCG_ERR_STATE (n differs from the gathered
 * set).  Stream-ordered; call dcg_scatter_back afterwards to keep the result. */
dcg_status dcg_adam_step(dcg_ctx* ctx, const dcg_gaussians* params, const dcg_gaussians* grads, int64_t n,
                         const float* lr, float beta1, float beta2, float eps, int64_t step, void* stream);

/* ---------------------------------------------------------------- loop closure
 * Sec. III-F "Cross-Chunk Transformation" and "Chunk Redistribution". */

/* Corrects the map after a loop closure.  kf: the K affected keyframes
 * (1 <= K <= 16) with their poses before the correction; corr (host,
 * [K][16] row-major) the correction of each keyframe, a rigid transform
 * (typically Tcw_new^-1 Tcw_old).  The chunks that keyframe k's frustum cull
 * keeps (pose before the correction) are batch-loaded together (their union
 * must fit the device budget: DCG_ERR_BUDGET otherwise, the table is then
 * unchanged; the paper's keyframe-by-keyframe fallback is not provided).  A
 * Gaussian of such a chunk whose centre projects into keyframe k's image
 * (znear < z <= zfar, 0 <= u < W, 0 <= v < H; FP32, one rounding per
 * operation) moves rigidly with it: x' = C_k x, q' = q(C_k) (x) q (SH
 * coefficients and scales unchanged); a Gaussian seen by several keyframes
 * moves with the first of them only (the global transformation mask).
 * Then chunk ids (Eq. 5/6) are recomputed for the loaded Gaussians and those
 * whose chunk changed are redistributed: a chunk keeps its remaining
 * Gaussians in stored order and receives incoming ones after them in gather
 * order; chunks are created as needed (emptied chunks stay, with count 0).
 * Optimizer moments travel with their Gaussians.  Chunk indices may change
 * (new chunks keep the table in ascending key order) and the active set is
 * invalidated.  n_transformed / n_moved (host, may be NULL): Gaussians moved
 * rigidly / moved to another chunk.  DCG_ERR_KEY_RANGE if a corrected position
 * leaves the Eq. 6 range (table unchanged).  Synchronous. */
dcg_status dcg_loop_closure(dcg_ctx* ctx, const dcg_camera* kf, const float* corr, int32_t K, int64_t* n_transformed,
                            int64_t* n_moved, void* stream);

/* Post-correction reset of Sec. III-F for the gathered active set: opacity
 * capped at max_opacity (logit <- min(logit, logit(max_opacity))) and, with
 * with_moments, the Adam moments zeroed.  params: the active view (dev).
 * DCG_ERR_STATE if n differs from the gathered set.  Stream-ordered. */
dcg_status dcg_reset_active(dcg_ctx* ctx, const dcg_gaussians* params, int64_t n, float max_opacity, void* stream);

/* ---------------------------------------------------------------- LoG sampling (Sec. III-B, Eq. 1) */

/* Sampling probability of Eq. 1 for one view and the pixels it samples:
 * P_s = max(P_L - P~, 0) with P_L, P~ the norms over the three channels of
 * the Laplacian-of-Gaussian responses of `image` and of `rendered` (dev,
 * [3][H][W] each).  The paper leaves the operator open; here: sigma 1 on a
 * 7 x 7 support as g2(dx) g(dy) + g(dx) g2(dy) (g the normalised Gaussian,
 * g2 its second derivative shifted to sum 0), the nearest edge pixel repeated
 * outside the image.  Pixel p = y W + x is sampled iff
 * u[p] < min(1, kappa P_s(p)) (u: dev [H W], the caller's uniform numbers in
 * [0, 1)).  ps_out (dev [H W], may be NULL) receives P_s; idx_out (dev,
 * max_out entries) the sampled pixels in ascending order, *n_out (host)
 * their number (DCG_ERR_CAPACITY if more than max_out, the first max_out are
 * written).  H W <= max_pixels.  Synchronous. */
dcg_status dcg_log_sample(dcg_ctx* ctx, const float* image, const float* rendered, int32_t W, int32_t H, float kappa,
                          const float* u, float* ps_out, int32_t* idx_out, int32_t max_out, int32_t* n_out,
                          void* stream);

/* New Gaussians at n sampled pixels idx (dev) of a view with camera `cam`:
 * centre at depth[p] (dev [H W], metres along the optical axis, > 0) on the
 * pixel's ray, log-scale log(depth / fx) on all three axes (one pixel
 * footprint), identity rotation, the given opacity logit, SH DC
 * (image[p] - 0.5) / Y00 from the pixel colour (dev [3][H][W]) and the other
 * coefficients 0, written planar to params_out (dev, [F][stride], stride >= n)
 * for dcg_chunk_table_update.  The paper places sampled Gaussians at depths
 * from its depth networks (Sec. III-B); those are outside this library. */
dcg_status dcg_backproject(dcg_ctx* ctx, const int32_t* idx, int32_t n, const float* depth, const float* image,
                           const dcg_camera* cam, float opacity_logit, float* params_out, int64_t stride,
                           void* stream);

/* dcg_log_sample over the n_views (1..16) views of a keyframe window in one
 * call.  The views sit back to back as in dcg_render_fwd's outputs: with
 * off_v = sum_{w<v} W_w H_w, image and rendered (dev) hold view v's
 * [3][H_v][W_v] block at 3 off_v floats, u and ps_out (dev, ps_out may be
 * NULL) its [H_v W_v] pixels at off_v.  Only W and H of cams (host
 * [n_views]) are read.  idx_out (dev, max_out entries) receives the sampled
 * pixels as window indices off_v + y W_v + x, ascending (views in order);
 * counts (host [n_views], may be NULL) the samples per view; *n_out (host)
 * their total (DCG_ERR_CAPACITY if more than max_out: the first max_out are
 * written and counted per view).  The same penalty and
 * sampling rule as the one-view call, view by view; sum of W_v H_v <=
 * max_pixels (DCG_ERR_CAPACITY) and < 2^31 (DCG_ERR_ARG).  Synchronous. */
dcg_status dcg_log_sample_views(dcg_ctx* ctx, const dcg_camera* cams, int32_t n_views, const float* image,
                                const float* rendered, float kappa, const float* u, float* ps_out, int32_t* idx_out,
                                int64_t max_out, int64_t* counts, int64_t* n_out, void* stream);

/* dcg_backproject for window indices idx (dev [n], as written by
 * dcg_log_sample_views) of the n_views views cams (host): a sample's view is
 * the last one whose first window pixel off_v is <= its index; depth (dev,
 * [off_V] pixels) and image (dev, view blocks of [3][H_v][W_v]) are laid out
 * as in dcg_log_sample_views.  Output as in dcg_backproject. */
dcg_status dcg_backproject_views(dcg_ctx* ctx, const int32_t* idx, int64_t n, const float* depth, const float* image,
                                 const dcg_camera* cams, int32_t n_views, float opacity_logit, float* params_out,
                                 int64_t stride, void* stream);

/* ---------------------------------------------------------------- rendering
 * Differentiable rasterisation of RGB and depth (Sec. III-E: the selected
 * Gaussians are rasterised into RGB and depth images; Eq. 4 needs the depth)
 * with the 3DGS representation.  Per view and Gaussian: camera point
 * t = R mu + t_cw, culled if t_z <= znear; u, v as in dcg_camera; the 2D
 * covariance J R Sigma R^T J^T + 0.3 I with Sigma = R(q) S S^T R(q)^T and
 * the perspective Jacobian J (x/z, y/z clamped to the image extended by 15%);
 * colour max(0, sum_k c_k Y_k(dir) + 0.5) with real SH (Condon-Shortley
 * phase) of the direction from the camera centre; opacity sigmoid(logit).
 * Per pixel (sample point (x, y)): Gaussians with q = d^T Sigma'^-1 d <= 9
 * and alpha = min(0.99, o exp(-q/2)) >= 1/255, in ascending (depth, index)
 * order, front to back; stop before T (1 - alpha) < 1e-4; background 0;
 * depth = sum T alpha t_z.
 *
 * Output layout: views are stacked; view v starts at pixel offset
 * off_v = sum_{w<v} W_w H_w; rgb (dev) holds [3][H_v][W_v] at 3 off_v,
 * depth (dev) holds [H_v][W_v] at off_v.  The state keeps what the backward
 * needs (sorted per-tile lists, per-pixel final transmittance and last
 * contributor); it refers to `g` and `cams`, which must stay unchanged until
 * the backward. */
dcg_status dcg_state_create(dcg_ctx* ctx, dcg_render_state** out);
/* The state every context creates for itself (used when a call gets NULL). */
dcg_render_state* dcg_default_state(dcg_ctx* ctx);
dcg_status dcg_state_destroy(dcg_render_state* st);

dcg_status dcg_render_fwd(dcg_ctx* ctx, const dcg_gaussians* g, int64_t n, const dcg_camera* cams,
                          int32_t n_views, float* rgb, float* depth, dcg_render_state* state, void* stream);

/* Gradient of L through the last forward of `state`: dL_drgb and dL_ddepth
 * (dev, layouts as rgb / depth) in; grads (dev, planar, same n and degree as
 * the forward, overwritten) and dL_dpose (dev, [n_views, 6], overwritten; may
 * be NULL) out.  The pose gradient is w.r.t. the left perturbation
 * Tcw <- exp(xi^) Tcw, xi = (v, w): a camera-frame point moves by v + w x t.
 * Transmittance is recomputed front-from-back from the stored final value.
 * A forward may be followed by several backward calls (other loss seeds):
 * each computes its gradient afresh. */
dcg_status dcg_render_bwd(dcg_ctx* ctx, dcg_render_state* state, const float* dL_drgb, const float* dL_ddepth,
                          dcg_gaussians* grads, float* dL_dpose, void* stream);

/* L1 parts of Eq. 2-4 summed over views: L = sum_v [ mean|C - C_gt| +
 * lambda_depth mean|D - D_gt| ]; writes dL/dC and dL/dD (dev, layouts as
 * rgb / depth; sign(0) = 0) and adds L to *loss (dev, one float, caller
 * zeroes). */
dcg_status dcg_loss_l1(dcg_ctx* ctx, const float* rgb, const float* depth, const float* tgt_rgb,
                       const float* tgt_depth, const dcg_camera* cams, int32_t n_views, float lambda_depth,
                       float* dL_drgb, float* dL_ddepth, float* loss, void* stream);

/* The loss of Eq. 2-4 with the SSIM term of Eq. 3, summed over views:
 *   L = sum_v [ (1 - lambda_s) mean|C - C_gt| + lambda_s (1 - SSIM(C, C_gt))
 *               + lambda_depth mean|D - D_gt| ],
 * SSIM with an 11 x 11 Gaussian window (sigma 1.5), C1 = 0.01^2,
 * C2 = 0.03^2, zero padding, averaged over pixels and channels (the 3DGS
 * form; the paper does not define it further).  Writes dL/dC and dL/dD
 * (dev, layouts as rgb / depth) and adds L to *loss (dev, caller zeroes).
 * lambda_s in [0, 1]; 0 gives dcg_loss_l1.  DCG_ERR_CAPACITY if the views
 * need more 16x16 SSIM tiles than max_pixels / 16 + 64 max_views + 64. */
dcg_status dcg_loss(dcg_ctx* ctx, const float* rgb, const float* depth, const float* tgt_rgb, const float* tgt_depth,
                    const dcg_camera* cams, int32_t n_views, float lambda_s, float lambda_depth, float* dL_drgb,
                    float* dL_ddepth, float* loss, void* stream);

/* Blend launch shape used by the next render calls: tile 16x16, 32x16 or
 * 32x32 pixels and 64..256 Gaussians staged per block batch (one block per
 * tile, warps of a tile synchronised per batch); stage 32 selects the
 * warp-per-block kernels (every warp takes one 8-column block of a tile from
 * a device queue on its own, no block barriers), stage 16 the half-warp
 * kernels (as 32, but the two half-warps walk separate lists for the two
 * 4-column halves of the block).  Results do not depend on it (gradients up
 * to FP32 atomic order). */
dcg_status dcg_set_launch(dcg_ctx* ctx, int32_t tile_w, int32_t tile_h, int32_t stage);

/* Batched keyframe window as one CUDA graph.  dcg_window_capture records,
 * on `stream`, the forward render of all n_views views of `g`, the loss of
 * Eq. 2-4 against tgt_rgb / tgt_depth (as dcg_loss with lambda_s and
 * lambda_depth), and the
 * backward to `grads` and dL_dpose, with every item count read from device
 * memory, and instantiates the graph (replacing a previous one).
 * dcg_window_run replays it on `stream` with the camera poses and
 * intrinsics of `cams`; view count and image sizes, buffers, n and the launch
 * shape must equal those of the capture (DCG_ERR_ARG otherwise).  *loss is
 * zeroed by the graph.  The render state used is the context's default one. */
dcg_status dcg_window_capture(dcg_ctx* ctx, const dcg_gaussians* g, int64_t n, const dcg_camera* cams,
                              int32_t n_views, float* rgb, float* depth, const float* tgt_rgb, const float* tgt_depth,
                              float lambda_depth, float lambda_s, float* dL_drgb, float* dL_ddepth, float* loss,
                              dcg_gaussians* grads, float* dL_dpose, void* stream);
dcg_status dcg_window_run(dcg_ctx* ctx, const dcg_camera* cams, int32_t n_views, void* stream);

/* Generation of a render state: incremented by every forward into it (a
 * backward can tell whether the state still holds its forward). */
int64_t dcg_state_generation(const dcg_render_state* st);

/* Autotuner of the blend launch shape: times render_fwd + render_bwd of this
 * call (default state, `reps` repetitions after one warm-up, CUDA events on
 * `stream`) for every tile {16x16, 32x16, 32x32} x stage
 * {64, 96, 128, 192, 256, 32 (warp-per-block), 16 (half-warp)}, keeps the
 * fastest as the context's launch shape and returns it.  ms_out (21 floats, tile-major in
 * that order, may be NULL) receives the mean time of each.  rgb/depth/grads
 * are overwritten; dL_drgb and dL_ddepth are the seeds used for the
 * backward.  Synchronous. */
dcg_status dcg_autotune(dcg_ctx* ctx, const dcg_gaussians* g, int64_t n, const dcg_camera* cams, int32_t n_views,
                        float* rgb, float* depth, const float* dL_drgb, const float* dL_ddepth, dcg_gaussians* grads,
                        int32_t reps, int32_t* tile_w, int32_t* tile_h, int32_t* stage, float* ms_out, void* stream);

/* Diagnostics of the last forward of `state` (host copies; any may be NULL):
 * visible (view, Gaussian) pairs, instances, tiles. Synchronises `stream`. */
dcg_status dcg_state_stats(dcg_render_state* st, int64_t* n_visible, int64_t* n_instances, int64_t* n_tiles,
                           void* stream);

/* Work of the last forward blend of `st`: *n_eval (pixel, Gaussian) pairs
 * whose support test ran while the pixel was still blending (depends on the
 * kernel's culling), *n_blend (may be NULL) pairs actually composited
 * (alpha >= 1/255, before termination: the method's own unit of blending
 * work, independent of the kernel).  Synchronises `stream`. */
dcg_status dcg_state_evals(dcg_render_state* st, int64_t* n_eval, int64_t* n_blend, void* stream);

/* Copies of the state's per-tile sorted lists for checks (host outputs; any
 * may be NULL): ranges [n_tiles, 2] (start, end) into ids, ids [n_instances]
 * (pair index v n + i), masks [n_instances] (bit 2 b + h: the instance's
 * Gaussian may reach the left (h = 0) or right (h = 1) 4-pixel-wide half of
 * warp block b of the tile; blocks are 8 pixels wide and tile_w tile_h / 64
 * high, numbered row-major), per (view, Gaussian) FP32
 * depth [n_views * n], 3-sigma tile rectangle [n_views * n, 4] (x0, y0, x1,
 * y1 inclusive; x1 < x0 if culled), per-pixel final transmittance and
 * contributor count.  A tile lists the Gaussians whose rectangle covers it
 * and whose support ellipse reaches its pixel rectangle.  Synchronises. */
dcg_status dcg_state_read(dcg_render_state* st, uint32_t* ranges, uint32_t* ids, uint16_t* masks, float* depth,
                          int32_t* rect, float* T_final, int32_t* n_contrib, void* stream);

/* ---------------------------------------------------------------- learned chunk prefetch
 * A small MLP proposes chunks that the next ~20 frames will need, so that
 * their host->device copies (Sec. III-E loads) can start early with
 * dcg_prefetch; the exact frustum cull still decides what is rendered.
 * Network: 128 inputs (99 used) -> 256 -> 256 -> 256 -> 1, GELU (erf form)
 * after each hidden layer, sigmoid output, binary cross-entropy (mean over
 * the batch) and Adam (beta 0.9 / 0.999, eps 1e-8).  Matrix products in BF16
 * on the tensor cores with FP32 accumulation; FP32 master parameters.  On
 * sm_100 and later the products use tcgen05.mma into tensor memory with
 * operands staged by TMA; dcg_mlp_set_gemm selects the mma.sync kernels
 * instead (same products, FP32 sums in another order).  The tcgen05 kernel
 * bounds its waits; if one gives up, the next dcg_mlp_get_params returns
 * DCG_ERR_TIMEOUT (and the affected outputs are not written).
 * Parameters, flat FP32 (dcg_mlp_num_params() = 164865 values):
 *   W1[128][256] b1[256] W2[256][256] b2[256] W3[256][256] b3[256] w4[256] b4
 * (W[i][j]: input i -> output j).  Inputs x are BF16 rows of 128 (dev);
 * batch sizes B are multiples of 64 up to max_batch. */
typedef struct dcg_mlp dcg_mlp;
enum { DCG_MLP_GEMM_TCGEN05 = 0, DCG_MLP_GEMM_MMA_SYNC = 1 };
dcg_status dcg_mlp_create(int32_t max_batch, dcg_mlp** out);
dcg_status dcg_mlp_set_gemm(dcg_mlp* m, int32_t kind);
dcg_status dcg_mlp_destroy(dcg_mlp* m);
int32_t dcg_mlp_num_params(void);
dcg_status dcg_mlp_set_params(dcg_mlp* m, const float* host_params); /* also resets Adam */
dcg_status dcg_mlp_get_params(dcg_mlp* m, float* host_params);
/* prob (dev, B) = sigmoid(MLP(x)) */
dcg_status dcg_mlp_forward(dcg_mlp* m, const uint16_t* x, int32_t B, float* prob, void* stream);
/* gradient of the mean BCE against labels y (dev, B, 0/1) into grads (dev,
 * num_params, may be NULL); the loss is added to *loss (dev) */
dcg_status dcg_mlp_grads(dcg_mlp* m, const uint16_t* x, const float* y, int32_t B, float* grads, float* loss,
                         void* stream);
/* dcg_mlp_grads followed by one Adam step with learning rate lr */
dcg_status dcg_mlp_train_step(dcg_mlp* m, const uint16_t* x, const float* y, int32_t B, float lr, float* loss,
                              void* stream);
/* Feature rows for one frame (x, dev, n_rows x 128 BF16; rows >= n_cand are
 * zero): columns 0..95 the SE(3) logarithms log(T_t^-1 T_{t-k}), k = 0..15,
 * of the camera-to-world poses (translation / 16 m, rotation in radians),
 * 96..98 the centre of candidate chunk cand[r] (dev) in the current camera
 * frame / 60 m.  pose_hist (host) holds 16 world->camera 3x4 row-major
 * matrices, current frame first; coords (dev) the chunk coordinates. */
dcg_status dcg_mlp_features(const float* pose_hist, const int32_t* coords, float chunk_size, const int32_t* cand,
                            int32_t n_cand, int32_t n_rows, uint16_t* x, void* stream);
/* x_out[r] = x[perm[r]], y_out[r] = y[perm[r]] for r < n (dev arrays). */
dcg_status dcg_mlp_gather_rows(const uint16_t* x, const float* y, const int32_t* perm, int32_t n, uint16_t* x_out,
                               float* y_out, void* stream);

/* ---------------------------------------------------------------- cull without allocation
 * The paper has no counterpart of this call; it exists for callers that
 * cannot allocate device memory: programs whose device memory is owned by
 * their own allocator or pool, or that run under a memory budget fixed in
 * advance, and so can neither let the library call cudaMalloc nor create a
 * dcg_ctx (whose creation allocates).
 * Same result as dcg_cull_chunks for chunk cubes of side chunk_size with
 * integer coordinates coords (dev, [n_chunks, 3] int32, any order; indices
 * below refer to this order) and distance filter dfar: mask_out (dev,
 * [n_views, n_chunks] u8, may be NULL), list_out (dev, capacity n_chunks)
 * ascending indices visible in any view, *n_out (dev, one int32).
 * Asynchronous on `stream`; cams is a host array, copied into the kernel's
 * launch parameters before return (pageable or pinned, it may be reused at
 * once).  Its scratch (one flag per chunk) is a fixed 1 MiB array in device
 * memory that every GPU loading the library keeps until the process exits:
 * at most 2^20 chunks and 16 views per call, larger requests return
 * DCG_ERR_CAPACITY without doing anything.  The first call on a device, and
 * the first after a cudaDeviceReset, looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the previous call's contents (the
 * call clears the flags before use), so calls that overlap on the GPU -- on
 * different streams, or from different host threads -- race and must be
 * serialised by the caller.  A failed launch or clear returns DCG_ERR_CUDA. */
dcg_status dcg_cull_chunks_noalloc(const int32_t* coords, int32_t n_chunks, float chunk_size, float dfar,
                                   const dcg_camera* cams, int32_t n_views, uint8_t* mask_out, int32_t* list_out,
                                   int32_t* n_out, void* stream);

/* ---------------------------------------------------------------- failure injection (testing)
 * Host-side faults of the chunk tier, for testing how a caller recovers; no
 * fault touches the GPU beyond ordinary copies.  An armed fault fires once,
 * on the (skip + 1)-th opportunity, and is then disarmed:
 *   DCG_FAULT_H2D_FAIL   a chunk load fails before its copies are issued
 *                        (dcg_gather_active / dcg_prefetch return DCG_ERR_FAULT;
 *                        the chunk stays in the host tier only);
 *   DCG_FAULT_SHORT_COPY the last page of a chunk load is copied only half
 *                        (the rest of the page holds a fill pattern); arming
 *                        it turns on load verification, which detects it:
 *                        the next dcg_gather_active drops the chunk and returns
 *                        DCG_ERR_FAULT before anything is rendered from it;
 *   DCG_FAULT_BUDGET     dcg_gather_active returns DCG_ERR_BUDGET as if the
 *                        listed chunks exceeded the device budget.
 * After any of them the context stays usable and a repeated call succeeds
 * with the same result as without the fault.  The environment variable
 * DCG_FAULT=h2d_fail|short_copy|budget[:skip] arms one at dcg_create. */
enum { DCG_FAULT_NONE = 0, DCG_FAULT_H2D_FAIL = 1, DCG_FAULT_SHORT_COPY = 2, DCG_FAULT_BUDGET = 3 };
dcg_status dcg_inject_fault(dcg_ctx* ctx, int32_t kind, int32_t skip);
/* Parses "none|h2d_fail|short_copy|budget[:skip]" (host only, no context). */
dcg_status dcg_fault_parse(const char* spec, int32_t* kind, int32_t* skip);

/* ---------------------------------------------------------------- profiling
 * Optional per-phase device timers.  When enabled, every call records CUDA
 * events around its phases on the stream it runs on; dcg_profile_read
 * synchronises on those events and returns, per phase, the summed
 * milliseconds (ms, DCG_PH_COUNT floats) and the number of timed intervals
 * (counts, may be NULL) since the last read.  Enabling creates the events;
 * the timed calls allocate nothing.  The pool holds 8192 events (two per
 * interval) between reads: intervals past it are not recorded, and the next
 * dcg_profile_read still writes ms and counts of the recorded ones but
 * returns DCG_ERR_CAPACITY, so a long run reads the timers every few hundred
 * steps and sums them. */
enum {
  DCG_PH_CULL = 0,
  DCG_PH_GATHER = 1,
  DCG_PH_PRE_FWD = 2,   /* per-Gaussian projection, conic, SH colour, tile rectangle */
  DCG_PH_BINNING = 3,   /* compaction, depth sort, instance emission, tile sort, ranges */
  DCG_PH_BLEND_FWD = 4, /* per-tile front-to-back blending */
  DCG_PH_LOSS = 5,
  DCG_PH_BLEND_BWD = 6, /* per-tile reverse traversal, 2D gradients */
  DCG_PH_PRE_BWD = 7,   /* chain rule to the parameters and the pose */
  DCG_PH_SCATTER = 8,
  DCG_PH_STALL = 9,     /* compute stream idle in dcg_gather_active, waiting for chunk copies */
  DCG_PH_SAMPLE = 10,   /* dcg_log_sample(_views) (LoG penalty, flags, ordered compaction, per-view counts)
                           and dcg_backproject(_views) */
  DCG_PH_LOOP = 11,     /* device work of dcg_loop_closure: cull, transform and keys, row permutation
                           and page writes (its gather is timed as DCG_PH_GATHER / DCG_PH_STALL) */
  DCG_PH_COUNT = 12
};
dcg_status dcg_profile(dcg_ctx* ctx, int32_t enable);
dcg_status dcg_profile_read(dcg_ctx* ctx, float* ms, int32_t* counts);

/* Kernel launches issued by the library in this process so far. */
uint64_t dcg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* DCG_H */
