// Level-2 rendering (Sec. 3.3 "Level 2"): the standard 3DGS projection,
// tile binning, depth sort, front-to-back compositing and their backward,
// run over the Gaussians of a render list of resident blocks.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "stage_timer.cuh"

namespace tgs {

// Gaussians addressed through a list of resident blocks.  Block j of the list
// lives in slot item_slot[j] of a pool whose slots are `slot_stride` floats
// apart; inside a slot, field f of lane l is at f * B + l (params), and at
// m_off + f * B + l / v_off + f * B + l for the Adam moments when present.
// Render-list position of lane l of item j: j * B + l.
// BF16 form (bf16 != 0): fields 0..13 (mean, log-scale, quaternion,
// opacity, SH DC) stay FP32 at f * B + l; the 45 SH-rest coefficients are
// BF16 at (bf16*)(slot + 14 B) + (f - 14) * B + l; both moments are BF16 at
// (bf16*)(slot + m_off / v_off) + f * B + l.  Adam's BF16 stores round
// stochastically (sr != 0, counter hash of seed, Gaussian id, field, step) or
// to nearest.
constexpr int F_BF16 = 14;
struct RenderList {
  float* base;
  uint64_t slot_stride;
  uint32_t B;
  uint32_t n_items;
  const uint32_t* item_slot;   // device [n_items]
  const uint32_t* item_count;  // device [n_items], Gaussians in the block
  const uint32_t* item_block;  // device [n_items], block id
  uint64_t m_off, v_off;       // moment offsets inside a slot (floats)
  uint32_t bf16 = 0, sr = 0, seed = 0;
  uint64_t capacity() const { return (uint64_t)n_items * B; }
};

// List segments of the backward work split.  A tile whose list is longer
// than R_SEG is composited backward as ceil(length / R_SEG) segments (at most
// R_NSEG_MAX, the last one taking the rest), each an independent CTA; the
// forward records per pixel (T, accumulated colour) at every segment boundary
// and, in one more slot, (T_final, final colour).  One tile's backward is
// otherwise a single CTA whose serial work can exceed the share of an SM slot
// several times (the longest lists are a few percent of the tiles).
constexpr int R_SEG = 256;  // a multiple of 32 (one staging batch)
constexpr uint32_t R_NSEG_MAX = 255;
__host__ __device__ __forceinline__ uint32_t seg_count(uint32_t len) {
  const uint32_t n = (len + R_SEG - 1) / R_SEG;
  return n <= 1 ? 1u : (n < R_NSEG_MAX ? n : R_NSEG_MAX);
}

// Per-camera state of one render (capacities fixed at allocation).
struct CamState {
  uint64_t cap_v = 0, cap_pairs = 0, cap_pix = 0, cap_tiles = 0;
  // per render-list position
  float2* xy = nullptr;
  float* depth = nullptr;
  float4* conic_o = nullptr;   // A, B, C, opacity
  float4* rgb = nullptr;       // r, g, b, clamp bits (as float)
  ushort4* rect = nullptr;     // x0, y0, x1, y1 (tiles)
  int* radius = nullptr;
  uint32_t* ntiles = nullptr;
  uint32_t* scan = nullptr;    // V: visibility scan, then pair offsets
  uint32_t* dkeys = nullptr;   // V x 2 (ping-pong): depth keys / positions
  uint32_t* dvals = nullptr;
  float* g2 = nullptr;         // 9 x g2_stride: dL/d(u, v, A, B, C, opacity, r, g, b)
  uint64_t g2_stride = 0;      // the last backward's render-list size
  // per pair
  uint32_t* pkeys = nullptr;   // 2 x cap_pairs (ping-pong)
  uint32_t* pvals = nullptr;
  // per tile / pixel
  uint2* ranges = nullptr;
  int32_t* tdiff = nullptr;    // (max TX + 1) x (max TY + 1) tile difference array, zero between renders
  uint32_t* tfill = nullptr;   // cap_tiles: pairs placed per tile
  uint32_t* tbig = nullptr;    // cap_tiles: tiles sorted by the large-tile sort
  uint32_t* torder = nullptr;  // 2 x cap_tiles: tiles, longest pair list first
  bool order_valid = false;
  // backward work split: a tile with a long list is composited backward as
  // several independent list segments, each started from the forward's
  // per-pixel state (T, accumulated colour) at its upper boundary
  uint32_t ck_cap = 0;         // checkpoint slots (TILE_PIX float4 each)
  float4* ck = nullptr;        // ck_cap x TILE_PIX
  uint32_t* tck = nullptr;     // cap_tiles: first checkpoint slot of a split tile, ~0u otherwise
  uint32_t* units = nullptr;   // cap_tiles + ck_cap: backward units, tile | segment << 24
  float* t_final = nullptr;
  int* n_last = nullptr;
  // scratch for scans and sorts
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  uint32_t* counters = nullptr;  // device [16]: n_vis, n_pairs (before the clamp), overflow, pairs needed, -,
                                 // backward units, binning consistency error, -, then the tile
                                 // binning's words (this render's overflow, long-list counts)
  uint32_t* counters_host = nullptr;  // pinned mirror (8 words), copied at the end of each render
  cudaEvent_t ev_counts = nullptr;    // recorded after that copy
  cudaStream_t aux = nullptr;         // the tile order's stream beside the binning (render_forward)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  uint32_t* step_flag = nullptr;      // optional device word raised with the overflow flag
  // results of the last render (valid after cam_state_counts)
  uint64_t n_vis = 0, n_pairs = 0, pairs_needed = 0;
  uint64_t hint_nv = 0, hint_np = 0;  // counts of the latest harvested render (grid sizes)
  bool overflow = false, counts_pending = false, counts_valid = false;
  int W = 0, H = 0, TX = 0, TY = 0;
};

void cam_state_alloc(CamState& cs, uint64_t cap_v, uint64_t cap_pairs, int max_w, int max_h);

// Tile binning (tiles.cu) of a render whose preprocess has run with the
// tile difference array (V render-list positions, TX x TY tiles): per-tile
// counts and ranges, pair emission, per-tile depth order, the tile order of
// the raster launches and the backward units.  The counts stay on the device
// (cs.counters).  The tile scan holds the (TX + 1) x (TY + 1) difference
// array in shared memory, which bounds the image to TILE_SCAN_SMEM_MAX bytes
// of it (40,960 cells: 3840 x 2160 uses 32,776).
constexpr size_t TILE_SCAN_SMEM_MAX = 160 * 1024;
size_t tile_scan_smem_bytes(int TX, int TY);
void bin_tiles(uint64_t V, int TX, int TY, CamState& cs, cudaStream_t s);
void cam_state_free(CamState& cs);
void cam_state_grow_pairs(CamState& cs, uint64_t need, cudaStream_t s);
// Reads the last render's counts into n_vis / n_pairs / overflow; wait =
// false returns false if they have not reached the host yet.
bool cam_state_counts(CamState& cs, bool wait);

// Forward: preprocess -> tile binning (counts, ranges, pair emission,
// per-tile depth sort) -> compositing.  touched (render-list bytes, may be
// null) gets 1 for visible Gaussians; item_touched (per item, may be null)
// gets 1 for items with a visible Gaussian.  No host synchronisation: the
// visible and pair counts stay on the device, pairs beyond cs.cap_pairs are
// dropped and flag an overflow (counters[2], and *cs.step_flag if set); the
// counts reach the host asynchronously.
void render_forward(const RenderList& rl, const DevCam& cam, const float bg[3], CamState& cs, float* image,
                    uint8_t* touched, uint32_t* item_touched, cudaStream_t s, StageTimer* tm = nullptr);

// render_forward on fixed caller-provided buffers (no allocation; pairs
// beyond cs.cap_pairs are a TGS_ERR_CAPACITY error).
void render_forward_fixed(const RenderList& rl, const DevCam& cam, const float bg[3], CamState& cs, float* image,
                          cudaStream_t s);

// Backward of the compositing into cs.g2 (zeroed here).
void render_backward_2d(const RenderList& rl, const DevCam& cam, const float bg[3], CamState& cs,
                        const float* dl_dimage, cudaStream_t s);

// Chain rule from cs.g2 to the 59 parameters.  mode 0 stores every valid
// position's gradient (zero when invisible) into a local [59][rl.capacity()] array,
// mode 1 adds visible gradients to it, mode 2 adds into a pool with the
// render list's slot layout (grad = pool base).
// rows / nrows (device, may be null): work on the listed render-list
// positions only (touched_rows); mode 0 then stores exactly those rows.
void render_backward_params(const RenderList& rl, const DevCam& cam, const CamState& cs, float* grad, int mode,
                            cudaStream_t s, const uint32_t* rows = nullptr, const uint32_t* nrows = nullptr);

// The chain rule of a batch of J cameras in one pass over the listed rows
// (their gradients summed in registers, stored once).
struct BatchGrad {
  static constexpr int MAXJ = 8;
  int J = 0;
  DevCam cam[MAXJ];
  const uint32_t* ntiles[MAXJ];
  const float4* rgb[MAXJ];
  const float4* conic[MAXJ];
  const float* g2[MAXJ];
  uint64_t stride[MAXJ];
};
void render_backward_params_batch(const RenderList& rl, const DevCam* cams, CamState* const* cs, int J, float* grad,
                                  const uint32_t* rows, const uint32_t* nrows, cudaStream_t s);

// rows[0..*nrows) = the render-list positions with touched != 0 (groups of
// 128 positions in ascending order, groups in any order).  prows (may be
// null): the even positions i whose pair (i, i + 1) has a touched member, as
// i | (touched[i] | touched[i + 1] << 1) << 30, their count in *nprows.
void touched_rows(const RenderList& rl, const uint8_t* touched, uint32_t* rows, uint32_t* nrows, cudaStream_t s,
                  uint32_t* prows = nullptr, uint32_t* nprows = nullptr);

// Masked Adam over the listed (touched) rows of the render list: params and
// moments in the pool are updated; `grad` is the local [59][rl.capacity()] array; step counters per
// block id (already incremented for this step).  Nothing is updated while
// *abort_flag (device, may be null) is set.
// Learning rates of the six parameter groups (means, log-scales, quaternion,
// opacity, SH DC, SH rest) for one step.
struct LrSet {
  float g[6];
};
__host__ __device__ inline int lr_group(int f) {
  return f < 3 ? 0 : f < 6 ? 1 : f < 10 ? 2 : f < 11 ? 3 : f < 14 ? 4 : 5;
}

// bias: per item (1 / (1 - b1^step), 1 / (1 - b2^step)) from mark_touched_blocks.
// prows / nprows (may be null; used when B is even): the pair list of
// touched_rows -- each thread then updates two adjacent Gaussians.
void adam_render_list(const RenderList& rl, const float* grad, const uint32_t* rows, const uint32_t* nrows,
                      const float2* bias, const uint32_t* block_step, const LrSet& lr, float b1, float b2, float eps,
                      cudaStream_t s, const uint32_t* abort_flag = nullptr, const uint32_t* prows = nullptr,
                      const uint32_t* nprows = nullptr);

// Per-item bookkeeping before Adam: for items with item_touched != 0,
// block_step[block] += 1 and dirty[slot] = 1.  While abort_flag[0] is set
// (device, may be null) nothing is marked and abort_flag[1] counts the step.
// bias (per item, may be null) receives the Adam bias corrections of the
// incremented step.
// readmit (per block, may be null): set for a re-admitted block; its next
// update counts as cold-restarted (Tab. 9) and clears it.  churn (may be null): [0] += updated blocks, [1] += cold-restarted ones.
void mark_touched_blocks(const RenderList& rl, const uint32_t* item_touched, uint32_t* block_step, uint8_t* dirty,
                         cudaStream_t s, uint32_t* abort_flag = nullptr, float b1 = 0.9f, float b2 = 0.999f,
                         float2* bias = nullptr, uint8_t* readmit = nullptr, unsigned long long* churn = nullptr);

// touched[j * B + l] |= (Gaussian l of item j had a non-empty tile rect in cs).
void mark_visible_bytes(const RenderList& rl, const CamState& cs, uint8_t* touched, cudaStream_t s);

// The 3DGS photometric loss with the D-SSIM term on J images (H x W x 3,
// interleaved): adds the loss sum ((1 - 0.2) |x - y| + 0.2 (1 - SSIM) over
// every value) to *loss_sum and writes dL/dimage of the mean into grad.
// scratch: device, 3 x J x H x W x 3 floats.
void photometric_loss_ssim(const float* img, const float* target, int J, int W, int H, float* grad, float* loss_sum,
                           float* scratch, cudaStream_t s);

// Masked Adam on block-layout arrays [ceil(n/B)][59][B]: per-block step
// counters are incremented for blocks with a touched row, then touched rows
// update m, v and params.
void adam_dense(float* params, const float* grad, float* m1, float* m2, const uint8_t* touched, uint32_t* step,
                uint64_t n, uint32_t B, float lr, float b1, float b2, float eps, cudaStream_t s);

// Bounding spheres (Sec. 3.3 "Level 1") of the listed blocks: centre = middle
// of the means' box, radius = max(|mu - c| + 3 max exp(log-scale)); written to
// spheres[block].  only_flag (per item, may be null) restricts to flagged items.
void block_bounds(const RenderList& rl, const uint32_t* only_flag, float4* spheres, cudaStream_t s,
                  const uint32_t* abort_flag = nullptr);

// Photometric loss over n values: writes dL/dimage and accumulates the sum of
// per-value losses into *loss_sum (device float, zeroed by the caller).
void photometric_loss(const float* img, const float* target, uint64_t n, int kind, float* grad, float* loss_sum,
                      cudaStream_t s);

}  // namespace tgs
