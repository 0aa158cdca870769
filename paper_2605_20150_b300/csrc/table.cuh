// The block-virtualised training table: pinned host tier, HBM working-set
// cache, copy streams and the training step (Sec. 3.2-3.5).
#pragma once
#include <cstdio>
#include <vector>

#include <deque>

#include "host_tier.cuh"
#include "predictor.cuh"
#include "raster.cuh"
#include "visibility.cuh"

namespace tgs {

void ck_read(std::FILE* f, void* dst, uint64_t bytes);

struct CopyPlan {
  std::vector<uint32_t> early_block, early_slot;  // into free slots, may start now
  std::vector<uint32_t> evict_block, evict_slot;  // S-, after the compute that last used them
  std::vector<uint32_t> late_block, late_slot;    // into slots freed by S-
};

struct Prepared {
  bool valid = false;
  bool enqueued = false;
  bool predicted = false;  // selection for a predicted (learned) visible set
  std::vector<tgs_camera> cams;
  std::vector<uint32_t> render_blocks;  // R & K of the batch, ascending
  std::vector<uint32_t> render_slots;   // their slots, fixed when the batch is selected
  std::vector<uint32_t> s_plus, s_minus;
  std::vector<uint32_t> kvis_host, r_host;  // per-camera visible sets, R after selection
  CopyPlan plan;
};

struct Table {
  tgs_config cfg{};
  uint64_t N = 0, K = 0, words = 0;
  uint32_t B = 0;
  uint64_t C = 0, n_slots = 0;
  uint64_t rec_floats = 0;   // floats per block record (params, m, v)
  uint64_t p_floats = 0, m_floats = 0;  // params part, one moment part (floats)
  uint64_t V_cap = 0;        // render-list Gaussians capacity
  uint32_t max_items = 0;

  // host tier: K records pinned, or a pinned pool over a log file
  HostTier tier;
  std::vector<uint32_t> perm;

  // device state
  float* pool = nullptr;
  float4* spheres = nullptr;
  float4* spheres_snap = nullptr;  // bounds as of the start of the latest compute
  uint32_t* ages = nullptr;
  uint32_t* block_step = nullptr;
  uint8_t* dirty_dev = nullptr;
  uint32_t *r_bits = nullptr, *r_next_bits = nullptr, *acc_bits = nullptr, *acc_next_bits = nullptr;
  uint32_t *kvis = nullptr, *kvis_union = nullptr;  // of the last prepared batch
  Planes* planes_dev = nullptr;
  Planes* planes_host = nullptr;
  ResidencyBuffers rb{};
  uint32_t* lists_dev = nullptr;   // s_plus | s_minus | render (K each)
  uint32_t* lists_host = nullptr;  // pinned
  uint32_t* kvis_host_pinned = nullptr;  // pinned, max_batch x words
  uint32_t* r_host_pinned = nullptr;     // pinned, words
  uint32_t *lists_map = nullptr, *kvis_map = nullptr, *r_map = nullptr;  // device views of the three (mapped)
  uint32_t* rl_dev = nullptr;      // item_slot | item_count | item_block
  static constexpr uint32_t RL_RING = 4;
  uint32_t* rl_host = nullptr;     // pinned, RL_RING staging slots of 3 x max_items
  cudaEvent_t rl_ev[RL_RING] = {};  // after the copy from each slot
  int rl_ev_used[RL_RING] = {};
  uint64_t rl_seq = 0;
  std::vector<CamState> cams;
  float* images = nullptr;
  float* dl_dimg = nullptr;
  float* targets_buf = nullptr;
  uint8_t* touched = nullptr;
  uint32_t* item_touched = nullptr;
  float* grad_local = nullptr;
  float* loss_dev = nullptr;
  float* ssim_buf = nullptr;       // loss 2: the three D-SSIM partial maps
  float* loss_host = nullptr;
  static constexpr uint64_t LOSS_RING = 4096;
  float* loss_ring = nullptr;      // pinned: the loss sum of the last LOSS_RING steps
  std::vector<float> loss_norm;    // element counts of those steps
  uint64_t loss_enq = 0, loss_read = 0;
  int tgt_parity = 0;              // host targets: double buffer in targets_buf
  int tgt_used[2] = {0, 0};
  cudaEvent_t ev_tgt_ready = nullptr, ev_tgt_used[2] = {nullptr, nullptr};
  float2* item_bias = nullptr;     // per render-list item: Adam bias corrections of this step
  uint32_t* rows_dev = nullptr;    // touched render-list rows of this step, count at rows_dev[V_cap_rows]
  uint64_t V_cap_rows = 0;
  uint32_t* prows_dev = nullptr;   // pairs of adjacent positions with a touched member, count at prows_dev[V_cap / 2 + 1]
  uint32_t* abort_dev = nullptr;   // [2]: a render of a step overflowed its pairs; steps dropped since
  uint32_t* abort_host = nullptr;  // pinned

  // host mirrors
  std::vector<int64_t> slot_of;          // K
  std::vector<int64_t> block_of_slot;    // n_slots
  std::vector<uint8_t> dirty_host;       // n_slots
  std::vector<cudaEvent_t> slot_free_ev; // n_slots (null = no pending use)
  std::vector<uint8_t> slot_has_ev;
  std::vector<uint8_t> ever_loaded;      // K: for the re-admission counter
  std::vector<uint8_t> wb_pending;       // K: write-back to the host tier issued, not yet waited on
  std::vector<uint64_t> admitted_at;     // K: stats.steps when the block was last admitted (Tab. 9 streaks)
  uint64_t resident_count = 0;           // blocks holding a slot
  uint8_t* readmit_dev = nullptr;        // K: moments zeroed by a re-admission, not yet updated
  unsigned long long* churn_dev = nullptr;  // [2]: block updates, cold-restarted block updates
  std::deque<uint32_t> free_fifo;        // free slots, longest free first
  cudaEvent_t ev_wb = nullptr;           // recorded after each write-back batch on d2h
  cudaEvent_t ev_snap = nullptr;         // recorded after the bounds snapshot on comp

  // last computed batch (for the debug getters)
  std::vector<tgs_camera> last_cams;
  std::vector<uint32_t> last_render, last_splus, last_sminus;
  std::vector<uint32_t> last_kvis_host;  // J x words
  std::vector<uint32_t> last_r_host;     // words
  Prepared prep;

  // h2d: loads into free slots; h2d_late: loads into slots S- frees (they
  // wait for that write-back), kept off h2d so that later loads into free
  // slots never queue behind them; tgtq: host targets of a step
  cudaStream_t comp = nullptr, h2d = nullptr, h2d_late = nullptr, tgtq = nullptr, d2h = nullptr, ctl = nullptr;
  cudaEvent_t ev_comp = nullptr, ev_h2d = nullptr, ev_h2d_late = nullptr, ev_ctl = nullptr, ev_user = nullptr;
  cudaEvent_t ev_stall_a = nullptr, ev_stall_b = nullptr;
  bool stall_pending = false;

  tgs_stats stats{};
  // learned prefetch
  Mlp* predictor = nullptr;
  float pred_threshold = 0.5f;
  uint32_t pred_mask = 1u;
  std::deque<tgs_camera> hist;
  // exact lookahead (prefetch mode 3): the camera schedule and its cursor
  static constexpr uint32_t MAX_LOOKAHEAD = 8;
  uint32_t vis_rows = 0;
  std::vector<tgs_camera> schedule;
  uint64_t sched_pos = 0;
  uint32_t sched_horizon = 0;
  std::vector<uint32_t> r_host_prev;  // resident set before the latest selection
  StageTimer timer;
  StageTimer copy_timer;  // stage 0: H2D batches, stage 1: D2H batches (always on)

  // ck (may be null): read the Morton order, host tier and state from a
  // checkpoint file instead of ordering params_host
  void create(const tgs_config& c, uint64_t n, const float* params_host, std::FILE* ck = nullptr);
  void save(const char* path);
  void resume(const tgs_config& c, const char* path);
  void destroy();
  void fill_host(const float* params);
  void init_spheres();
  void set_params(const float* params);
  void prepare_enqueue(const tgs_camera* cams, uint32_t J, Prepared& out, bool own_batch);
  void prepare_enqueue_predicted(Prepared& out);
  void prepare_enqueue_lookahead(Prepared& out);
  void select_enqueue(uint32_t J, Prepared& out, bool accessed);
  void cull_only(const tgs_camera* cams, uint32_t J, uint8_t* vis_host);
  void prepare_finish(Prepared& out);
  void issue_early(Prepared& p);
  void issue_evictions_and_late(Prepared& p);
  void compute(const Prepared& p, const float* targets_dev, const float* targets_host, cudaStream_t user,
               bool backward, float* image_out);
  void step(const tgs_camera* cams, uint32_t J, const tgs_camera* next, uint32_t nJ, const float* targets_dev,
            const float* targets_host, cudaStream_t user, float* loss_out);
  void render(const tgs_camera& cam, float* image_dev, cudaStream_t user);
  void flush();
  void collect_stall();
  void wait_ctl();
  // Handles a pair-capacity overflow seen by a render (wait: block until the
  // last renders' counts are on the host): grows the pair buffers, counts
  // the dropped steps and clears the flag.  Returns true if one was handled.
  bool check_overflow(bool wait);
  // the learning rates of the step about to run (schedule at stats.steps)
  LrSet step_lrs() const;
  // the losses (mean per step) of the steps since the last call, oldest
  // first, at most the last LOSS_RING; waits for the compute stream
  uint64_t losses(float* out, uint64_t max_count);
  RenderList render_list(uint32_t n_items) const;
};

}  // namespace tgs
