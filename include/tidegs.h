/*
 * tidegs.h -- C ABI of the B300 (sm_103a) implementation of the TideGS
 * out-of-core 3D Gaussian Splatting training step (arXiv 2605.20150).
 *
 * Conventions shared by every entry point
 *   - Every call returns a tgs_status; TGS_OK is 0.  On failure nothing is
 *     thrown or aborted across the boundary: the status says what went wrong
 *     and tgs_last_error() returns a thread-local message.
 *   - Pointers marked "host" point to CPU memory, "device" to memory of the
 *     current CUDA device.  Input buffers are borrowed for the duration of the
 *     call unless stated otherwise; output buffers are owned by the caller.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).  Device work is ordered after work already
 *     queued on that stream; results are ready when that stream reaches the
 *     point after the call.
 *   - A Gaussian row has D = 59 floats in the paper's logical layout
 *     (Sec. 2 "Per-Gaussian parameter table", D = 59): mean (3), log-scale (3),
 *     rotation quaternion w,x,y,z (4), opacity logit (1), SH DC rgb (3), SH rest
 *     (45 = 15 coefficients x rgb, coefficient-major, l=1..3, m=-l..l).
 *   - Images are H x W x 3 float32, row-major, pixel (px, py) sampled at its
 *     integer coordinates.
 *   - A table is not thread-safe: one calling thread per table.
 */
#ifndef TIDEGS_H
#define TIDEGS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TGS_D 59
#define TGS_TILE 16

typedef int32_t tgs_status;
enum {
  TGS_OK = 0,
  TGS_ERR_INVALID = 1,  /* bad argument (null pointer, size out of range) */
  TGS_ERR_OOM = 2,      /* device or pinned host allocation failed */
  TGS_ERR_CUDA = 3,     /* a CUDA runtime call failed */
  TGS_ERR_CAPACITY = 4, /* a working set or buffer exceeds its configured capacity */
  TGS_ERR_TIMEOUT = 5,  /* a bounded wait ran out */
  TGS_ERR_STATE = 6     /* call not valid in the table's current state */
};

/* Thread-local description of the last failure on this thread ("" if none). */
const char* tgs_last_error(void);

/* Pinhole camera.  A world point x maps to camera coordinates
 * c = R x + t with world_to_cam = [R | t] (row-major 3x4); the camera looks
 * down +z, y points down; pixel u = fx c_x / c_z + cx, v = fy c_y / c_z + cy.
 * znear / zfar bound the visible depth (Sec. 3.3, "6-plane frustum test"). */
typedef struct tgs_camera {
  uint32_t width, height;
  float fx, fy, cx, cy;
  float znear, zfar;
  float world_to_cam[12];
} tgs_camera;

/* Training-table configuration.  Defaults from tgs_default_config(). */
typedef struct tgs_config {
  uint32_t block_size;     /* B, Gaussians per block (Sec. 3.3 uses 4096) */
  uint32_t moments_policy; /* 0: Adam moments stream with their block (persistent);
                              1: moments dropped on eviction, zeroed on re-admission
                              (the paper's default "cold restart", Sec. 3.5) */
  uint32_t prefetch_mode;  /* 0: reactive -- batch t's working set is selected and
                              streamed at step t (copies exposed);
                              1: exact next batch (Sec. 3.4-3.5) -- batch t+1's delta is
                              selected and streamed while batch t computes;
                              2: learned (tgs_set_predictor); 3: exact lookahead over a
                              schedule (tgs_set_schedule) */
  uint32_t overlap;        /* 1: copies on dedicated streams overlap compute (Sec. 3.4);
                              0: copies serialised with compute */
  uint64_t cache_blocks;   /* C, resident-set capacity in blocks; 0 = all blocks */
  uint32_t spare_slots;    /* extra HBM slots that receive incoming blocks while the
                              current step still uses its resident set */
  uint32_t max_batch;      /* largest camera batch J */
  uint32_t max_width, max_height;  /* largest image; (ceil(w/16) + 1) x (ceil(h/16) + 1) <= 40,960
                              (the tile binning's difference array in shared memory: up
                              to 3840 x 2160 and beyond); larger is TGS_ERR_INVALID */
  uint32_t quota;          /* per-camera quota of the camera-balanced Top-C;
                              0xFFFFFFFF = floor(C / (2 J)) */
  float lambda;            /* residency mix lambda of s(k) (Sec. 3.5) */
  float lr, beta1, beta2, eps; /* Adam, one learning rate for all 59 columns */
  float cull_margin_px;    /* Level-1 side-plane margin in pixels */
  float bg[3];             /* background colour */
  uint32_t loss;           /* photometric loss f_i (App. A.1): 0 L1 mean, 1 L2 mean,
                              2 the 3DGS recipe (1 - 0.2) L1 + 0.2 (1 - SSIM), SSIM over an
                              11 x 11 Gaussian window (sigma 1.5), zero padding */
  uint32_t host_bf16;      /* 1: the 45 SH-rest coefficients and both Adam moments are
                              BF16 in the host tier and the cache (382 instead of 708
                              bytes per Gaussian; not in the paper); projection, blending
                              and accumulation stay FP32.  Needs an even block_size. */
  uint32_t stochastic_round; /* BF16 stores of Adam: 1 stochastic rounding (counter hash
                              of seed, Gaussian id, field, step), 0 round to nearest */
  uint32_t seed;
  uint64_t pair_capacity;  /* initial (tile, Gaussian) pair capacity per camera; 0 = the larger
                              of 2 x the render-list capacity and 16 x max_width x max_height.  A render whose pairs exceed it is
                              completed on the device without the excess, its step's update
                              is skipped, and the capacity grows once the host sees the
                              count (tgs_stats.pair_overflows / dropped_steps). */
  uint64_t max_render_blocks; /* most blocks one batch renders (the per-camera buffers scale
                              with it); 0 = cache_blocks.  A batch with more visible resident
                              blocks is a TGS_ERR_CAPACITY error. */
  /* Learning-rate schedule (Sec. 4 trains with "the 3DGS learning-rate
   * schedule"): lr_schedule 0 = `lr` for all 59 columns; 1 = one rate per
   * group (means, log-scales, quaternion, opacity, SH DC, SH rest) from
   * lr_groups, the means' rate decaying log-linearly to lr_means_final over
   * lr_decay_steps training steps (then constant). */
  uint32_t lr_schedule;
  float lr_groups[6];
  float lr_means_final;
  uint32_t lr_decay_steps;
  /* Ablations (Tab. 5): differential 0 = every selection evicts the whole
   * cache and streams the selected set again ("w/o Tide"); morton 0 = blocks
   * are runs of the input order ("w/o Morton").  overlap 0 above is "w/o
   * Overlap". */
  uint32_t differential;
  uint32_t morton;
  /* Host second tier (Sec. 3.4, "CPU tiered cache" over storage):
   * host_cache_blocks = 0 (or >= the block count) keeps every block record in
   * pinned host memory; otherwise the records live in an append-only log file
   * at backing_path (created or replaced; removed with the table) and a pool
   * of host_cache_blocks pinned record slots caches them (LRU): a block
   * streamed to the GPU is read from the log on a pool miss, a dirty block
   * written back from the GPU stays in the pool and is appended to the log
   * when the pool recycles its slot.  backing_path: borrowed during
   * tgs_create / tgs_resume (copied). */
  uint64_t host_cache_blocks;
  const char* backing_path;
} tgs_config;

void tgs_default_config(tgs_config* cfg);

typedef struct tgs_table tgs_table;

/* Creates a block-virtualised table of n Gaussians (Sec. 3.3, Eq. block_def):
 * Morton-orders the rows by the codes of their centres, cuts blocks of B rows
 * (the last block truncated at n), writes the block records to pinned host
 * memory (the host tier), computes the block bounding spheres and allocates
 * the HBM working-set cache.
 * params_host: host, n x 59 row-major, borrowed (copied).
 * Errors: TGS_ERR_INVALID (n == 0, bad config), TGS_ERR_OOM. */
tgs_status tgs_create(const tgs_config* cfg, uint64_t n, const float* params_host, tgs_table** out);

void tgs_destroy(tgs_table* t);

/* Checkpoint and resume of the training state (Sec. 3.5's consistency
 * barrier: every dirty resident block is written back first).  The file holds
 * the Morton order, the host tier (parameters and Adam moments of every
 * block), the per-block Adam step counters, the residency ages and the block
 * bounds.  tgs_resume creates a table from it with an empty HBM cache (blocks
 * stream in as they are needed); cfg must give the checkpoint's block_size
 * and host_bf16, the other fields (cache size, prefetch, image limits) may
 * differ.  path: host string, the file is created or replaced.
 * Errors: TGS_ERR_INVALID (unreadable, truncated or mismatching file),
 * TGS_ERR_OOM, TGS_ERR_CUDA. */
tgs_status tgs_checkpoint(tgs_table* t, const char* path);
tgs_status tgs_resume(const tgs_config* cfg, const char* path, tgs_table** out);

/* One training step on a camera batch (Sec. 3.2 stages 1-4, Algorithm 1):
 * culls the batch's blocks, makes its working set resident (streaming only the
 * delta S+ and writing back dirty evicted blocks S-), renders each camera over
 * the resident visible blocks, computes the photometric loss against the
 * targets, back-propagates, applies masked Adam to the touched Gaussians
 * (App. A.1, Eq. masked_update), marks their blocks dirty and refreshes their
 * bounds.  With prefetch_mode 1 and next_cams given, it also selects and
 * starts streaming the next batch's delta while this batch computes.
 * cams: host, batch cameras (batch <= max_batch).
 * next_cams: host, the next batch (may be NULL).
 * targets_dev: device, batch x H x W x 3, or NULL when targets_host is given;
 *   read after `stream`'s prior work.
 * targets_host: host (pinned or pageable), used when targets_dev is NULL; copied
 *   inside the call on the copy stream (pinned memory: asynchronously, into one
 *   of two device buffers, overlapping the previous step; pinned targets must
 *   then stay unchanged until the step has run, e.g. until tgs_sync or a later
 *   step's loss is read).
 * loss_out: host, may be NULL; when given the call waits for the step and writes
 *   the batch loss (mean over cameras, pixels and channels).
 * Errors: TGS_ERR_INVALID, TGS_ERR_CAPACITY (a batch's working set exceeds the
 *   cache), TGS_ERR_CUDA. */
tgs_status tgs_step(tgs_table* t, const tgs_camera* cams, uint32_t batch, const tgs_camera* next_cams,
                    uint32_t next_batch, const float* targets_dev, const float* targets_host, void* stream,
                    float* loss_out);

/* Renders one camera from the current parameters (forward only).  The camera's
 * working set is made resident first (it counts as a step of the residency
 * policy, without parameter updates).  image_dev: device, H x W x 3. */
tgs_status tgs_render(tgs_table* t, const tgs_camera* cam, float* image_dev, void* stream);

/* Losses of the training steps since the previous call, oldest first (the
 * photometric loss f_i of App. A.1, mean over cameras, pixels and channels).
 * Every step copies its loss to pinned host memory asynchronously, so a
 * caller can read them without waiting on each step; the call waits for the
 * compute stream.  At most the last 4096 steps are kept.
 * out_host: host, room for max_count floats; count: host, receives the number
 * written.  Errors: TGS_ERR_INVALID. */
tgs_status tgs_losses(tgs_table* t, float* out_host, uint64_t max_count, uint64_t* count);

/* Changes prefetch_mode (0 reactive, 1 exact next batch, 2 learned) between
 * steps; a pending prefetch is kept and used if it matches the next batch. */
tgs_status tgs_set_prefetch_mode(tgs_table* t, uint32_t mode);

/* Known trajectory for the exact lookahead prefetch (prefetch_mode 3; not in
 * the paper, the upper bound the learned form is measured against): each step
 * moves a cursor past its batch and, while the batch computes, selects
 * (Algorithm 1, no access update) and streams the Level-1 visible blocks of
 * the next `horizon` scheduled cameras.  cams: host, n cameras in step order
 * (copied); horizon: 1..8.  Errors: TGS_ERR_INVALID. */
tgs_status tgs_set_schedule(tgs_table* t, const tgs_camera* cams, uint64_t n, uint32_t horizon);

/* Waits for all queued work of the table. */
tgs_status tgs_sync(tgs_table* t);

/* Replaces all parameters (params_host: host, n x 59 in the original row
 * order given to tgs_create), zeroes the Adam moments and step counters,
 * empties the HBM cache and recomputes the block bounds.  The block order
 * (Morton permutation) of the table is kept. */
tgs_status tgs_set_params(tgs_table* t, const float* params_host);

/* Flushes dirty resident blocks to the host tier (a consistency barrier,
 * Sec. 3.4) and writes the parameters in the caller's original row order.
 * out_host: host, n x 59. */
tgs_status tgs_get_params(tgs_table* t, float* out_host);

/* Same barrier; writes the state in block (Morton) order: params, first and
 * second Adam moments (each n x 59, any may be NULL), and the per-block Adam
 * step counters (K values, may be NULL). */
tgs_status tgs_get_state(tgs_table* t, float* params_host, float* m1_host, float* m2_host, uint32_t* steps_host);

/* The same barrier, then selected rows of that state: ids (host, count
 * block-order ids, any order, repeats allowed); params / m1 / m2 (host,
 * count x 59 each, any may be NULL) receive those rows in the order of ids.
 * For checking a table of 10^8 Gaussians without reading all of it.
 * Errors: TGS_ERR_INVALID (an id >= n). */
tgs_status tgs_get_state_rows(tgs_table* t, const int64_t* ids, uint64_t count, float* params_host, float* m1_host,
                              float* m2_host);

/* perm_host[g] = original row of the Gaussian with block-order id g (n values). */
tgs_status tgs_get_block_order(tgs_table* t, int64_t* perm_host);

/* Block bounding spheres (cx, cy, cz, r), K x 4, as the next cull uses them. */
tgs_status tgs_get_spheres(tgs_table* t, float* spheres_host);

/* Sizes: n Gaussians, K blocks, number of HBM slots. */
tgs_status tgs_get_sizes(tgs_table* t, uint64_t* n, uint64_t* k, uint64_t* slots);

/* Set state of the last step, as K-byte arrays (1 = member): the visible set
 * K_t of the computed batch, the resident set R_t it rendered from, and the
 * per-camera visible sets (batch x K); s_plus / s_minus receive the block ids
 * streamed in / evicted to make R_t resident (ascending) with their counts.
 * Any pointer may be NULL. */
tgs_status tgs_get_sets(tgs_table* t, uint8_t* k_visible, uint8_t* r_resident, uint8_t* k_per_camera,
                        int64_t* s_plus, uint64_t* n_plus, int64_t* s_minus, uint64_t* n_minus);

/* Per-camera intermediates of the last step (camera index j of the batch), in
 * render-list order (ascending Gaussian id over the blocks of R_t & K_t):
 *   ids (int64 Gaussian ids), splat (float x 12: u, v, depth, A, B, C, opacity,
 *   r, g, b, radius, visible), rect (int32 x 4: x0, y0, x1, y1);
 *   pair_vals (uint32 render-list positions of the sorted pairs),
 *   ranges (uint32 x 2 per tile); image (H x W x 3), t_final (H x W),
 *   n_last (int32, H x W); grad2d (float x 9 per Gaussian: u, v, A, B, C,
 *   opacity, r, g, b).  Call with all array pointers NULL to get the counts. */
tgs_status tgs_get_camera_record(tgs_table* t, uint32_t j, uint64_t* n_gauss, uint64_t* n_pairs,
                                 int64_t* ids, float* splat, int32_t* rect, uint32_t* pair_vals,
                                 uint32_t* ranges, float* image, float* t_final, int32_t* n_last,
                                 float* grad2d);

/* Counters (Tab. 4/5/9 style): steps, bytes and blocks moved each way,
 * write-backs, re-admissions, cold restarts, kernel launches of the library,
 * exposed copy time, copy-engine busy time, and the last render's sizes. */
typedef struct tgs_stats {
  uint64_t steps;
  uint64_t bytes_h2d, bytes_d2h;
  uint64_t blocks_in, blocks_out, writebacks, readmissions, cold_restarts;
  uint64_t kernel_launches;
  double stall_ms;          /* compute stream waiting for incoming blocks */
  double h2d_ms, d2h_ms;    /* CUDA-event time of the copy batches on the copy streams */
  uint64_t demand_blocks;   /* sum over computed batches of their visible blocks */
  uint64_t demand_hits;     /* ... of those already resident before the batch's own selection */
  uint64_t predicted_blocks; /* blocks streamed in on a prediction (learned prefetch) */
  uint64_t last_pairs, last_visible, last_render_blocks;
  /* Tile/Gaussian pair capacity: renders whose pairs exceeded it (the
   * capacity then grows), and training steps whose update was skipped
   * because a render of theirs, or of an earlier step not yet seen by the
   * host, overflowed. */
  uint64_t pair_overflows, dropped_steps;
  /* Host time inside tgs_step, and of it the time blocked on the control
   * stream's selections (Algorithm 1 lists read back). */
  double host_step_ms, host_wait_ms;
  /* Residency churn (App. A.4, Tab. 9): resident_block_steps = sum over
   * training steps of the resident blocks |R_t|; block_updates = blocks with
   * an updated Gaussian, summed over steps; cold_updates = of those, the
   * first update of a block after a re-admission (the update that starts
   * from zeroed moments under moments_policy 1; counted under either
   * policy, the residency decisions do not depend on it); streaks /
   * streak_steps = completed residencies (a
   * block's stay from admission to eviction) and their total length in
   * steps. */
  uint64_t resident_block_steps, block_updates, cold_updates, streaks, streak_steps;
  /* Host second tier (host_cache_blocks > 0): pool hits and misses of block
   * accesses, bytes read from and appended to the log. */
  uint64_t host_cache_hits, host_cache_misses, log_bytes_read, log_bytes_written;
} tgs_stats;
tgs_status tgs_get_stats(tgs_table* t, tgs_stats* out);

/* Stage timing (tracing): when enabled, CUDA events on the compute stream
 * bracket each stage of every step.  Stages, in order: 0 Level-2 preprocess,
 * 1 binning + depth/tile sort, 2 forward raster, 3 loss, 4 backward raster,
 * 5 backward preprocess, 6 masked Adam, 7 bound refresh.
 * tgs_get_stage_ms waits for the recorded events and returns the accumulated
 * milliseconds and launch counts per stage (8 values each); reset = 1 clears
 * the accumulators after reading. */
tgs_status tgs_set_stage_timing(tgs_table* t, int enable);
tgs_status tgs_get_stage_ms(tgs_table* t, double* ms8, uint64_t* counts8, int reset);

/* Level-1 visibility only (Sec. 3.3, Eq. Kt_def) of J cameras against the
 * current block bounds: vis_host (host, J x K bytes) gets 1 for visible
 * blocks.  Used to log visibility for the learned predictor. */
tgs_status tgs_visible_blocks(tgs_table* t, const tgs_camera* cams, uint32_t J, uint8_t* vis_host);

/* ---------------------------------------------------------------------------
 * Learned block-prefetch predictor (the paper has none; it is the learned
 * prefetch form of this implementation).  A 3-layer MLP, 102 -> 256 -> 256
 * -> 4 (ReLU, sigmoid outputs), predicts for each block whether it will be
 * visible 1..4 iterations ahead from the last 8 camera poses (each as the
 * rotation and translation / zfar of that camera in the current camera's
 * frame) and 6 block features (centroid in the current camera frame / zfar,
 * radius / zfar, distance / zfar, radius / max(distance, radius)).  Layer 2
 * runs on the tensor cores (BF16 weights and activations, FP32 accumulation).
 * Parameters: flat FP32 [W1 (102 x 256), b1 (256), W2 (256 x 256), b2 (256),
 * W3 (256 x 4), b3 (4)], row-major, input index first.
 * ------------------------------------------------------------------------- */
typedef struct tgs_mlp tgs_mlp;
/* max_blocks: largest K; seed: initial weights N(0, 1/sqrt(fan_in)), zero biases. */
tgs_status tgs_mlp_create(uint64_t max_blocks, uint32_t seed, tgs_mlp** out);
void tgs_mlp_destroy(tgs_mlp* m);
uint64_t tgs_mlp_num_params(void);
tgs_status tgs_mlp_get_params(tgs_mlp* m, float* params_host);
tgs_status tgs_mlp_set_params(tgs_mlp* m, const float* params_host);
/* Logits (device, K x 4) of K blocks with spheres (device, K x 4: cx, cy, cz,
 * r) for the camera history hist (host, 8 cameras, oldest first, the last the
 * current one). */
tgs_status tgs_mlp_forward(tgs_mlp* m, const float* spheres_dev, uint64_t K, const tgs_camera* hist,
                           float* logits_dev, void* stream);
/* One training step on K labelled blocks (labels_dev: device, K x 4, 1 = visible
 * at t+h): forward, BCE with pos_weight (mean over K x 4), backward, and, if
 * apply != 0, AdamW (lr, weight_decay, betas 0.9 / 0.999, eps 1e-8).
 * loss_out (host) gets the loss before the update; grads_host (host, flat, may
 * be NULL) the gradient. */
tgs_status tgs_mlp_train_step(tgs_mlp* m, const float* spheres_dev, uint64_t K, const tgs_camera* hist,
                              const float* labels_dev, float pos_weight, float lr, float weight_decay, int apply,
                              float* loss_out, float* grads_host, void* stream);
/* Attaches a predictor to a table for prefetch_mode 2: after each step's
 * culling, blocks whose predicted probability exceeds `threshold` for a
 * horizon in horizon_mask (bit h-1 = t+h) are selected by Algorithm 1 and
 * streamed while the step computes; the next step culls its actual batch
 * and fetches what was missed.  The predictor must outlive its use. */
tgs_status tgs_set_predictor(tgs_table* t, tgs_mlp* m, float threshold, uint32_t horizon_mask);

/* ---------------------------------------------------------------------------
 * Resident (fully in-HBM) rasteriser for autograd frameworks: the standard
 * 3DGS forward/backward that Sec. 3.3 "Level 2" runs on the resident blocks.
 * Parameters live in caller-owned device memory in block layout
 * [ceil(n/B)][59][B] float (field-major inside a block); Gaussian id g is
 * block g / B, lane g % B; lanes past n are ignored.
 * ------------------------------------------------------------------------- */
typedef struct tgs_raster tgs_raster;

/* max_gaussians: largest n; max_width / max_height: largest image (the same
 * bound as tgs_config's max_width / max_height). */
tgs_status tgs_raster_create(uint64_t max_gaussians, uint32_t max_width, uint32_t max_height, tgs_raster** out);
void tgs_raster_destroy(tgs_raster* r);

/* Forward render of one camera over all n Gaussians of params_dev.
 * image_dev: device, H x W x 3.  The context keeps what the backward needs
 * for this one camera until the next forward. */
tgs_status tgs_raster_forward(tgs_raster* r, const float* params_dev, uint64_t n, uint32_t block_size,
                              const tgs_camera* cam, const float* bg3, float* image_dev, void* stream);

/* Backward of the last forward (same params, camera and background):
 * dl_dimage_dev (device, H x W x 3) -> grad_dev (device, params layout,
 * ACCUMULATED with +=).  touched_dev (device, n bytes, may be NULL) is set to 1
 * for Gaussians with a non-empty tile rect. */
tgs_status tgs_raster_backward(tgs_raster* r, const float* params_dev, uint64_t n, uint32_t block_size,
                               const tgs_camera* cam, const float* bg3, const float* dl_dimage_dev,
                               float* grad_dev, uint8_t* touched_dev, void* stream);

/* Forward render like tgs_raster_forward for callers that cannot allocate
 * device memory when they render (under a fixed memory budget owned by another
 * allocator, where an allocation of their own would fail or fragment it; in
 * real-time loops that must not allocate).  The paper has no counterpart.
 * All intermediates live in one 16 MiB file-scope device array that every GPU
 * loading the library holds until exit; nothing is allocated per call.
 * Limits: ceil(n / block_size) * block_size <= 32768, width * height <=
 * 512 * 512 (at most 1024 tiles), at most 524288 (tile, Gaussian) pairs;
 * beyond them the call returns TGS_ERR_CAPACITY and renders nothing.
 * The first call on a device looks the array up (cudaGetSymbolAddress) with
 * that device current: make it before any stream capture.  The call reads
 * the visible and pair counts back to the host (it waits on `stream`) and
 * returns when its work on `stream` has completed.  Calls share the array
 * and keep its last contents; calls whose GPU work overlaps race.
 * params_dev, image_dev, bg3: as for tgs_raster_forward. */
tgs_status tgs_raster_forward_noalloc(const float* params_dev, uint64_t n, uint32_t block_size,
                                      const tgs_camera* cam, const float* bg3, float* image_dev, void* stream);

/* Masked Adam (App. A.1, Eq. masked_update) on block-layout device arrays:
 * rows with touched[g] != 0 update m, v and params; step_dev holds per-block
 * step counters (ceil(n/B) uint32), incremented for blocks with a touched row
 * before their rows use them for bias correction. */
tgs_status tgs_adam(float* params_dev, const float* grad_dev, float* m1_dev, float* m2_dev,
                    const uint8_t* touched_dev, uint32_t* step_dev, uint64_t n, uint32_t block_size, float lr,
                    float beta1, float beta2, float eps, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TIDEGS_H */
