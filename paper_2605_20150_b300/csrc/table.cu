// Block-virtualised training table (Sec. 3.2-3.5): the pinned host tier, the
// HBM working-set cache of block slots, the copy streams and the step.
//
// Streams: `ctl` runs Level-1 culling and Algorithm 1, `h2d` streams S+ into
// free slots, `h2d_late` into the slots S- frees (after their write-back),
// `d2h` writes dirty S- blocks back, `tgtq` uploads host targets, `comp`
// renders and trains.  With the exact next-batch prefetch, batch t+1's delta
// is selected at the start of step t and its incoming blocks are copied into
// spare slots while batch t computes (Sec. 3.4 "Hierarchical asynchronous
// execution"); blocks that can only go into slots freed by S- are copied
// after that write-back.  Every copy waits only for what it needs (the slot's
// last reader and write-back, the block's own pending write-back), so no
// copy queues behind one that waits for compute.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>

#include <cuda_bf16.h>

#include "sort.cuh"
#include "table.cuh"

namespace tgs {

// Distance between the centres (-R^T t) of two cameras.
static double camera_distance(const tgs_camera& a, const tgs_camera& b) {
  double d2 = 0.0;
  for (int i = 0; i < 3; ++i) {
    double ca = 0.0, cb = 0.0;
    for (int j = 0; j < 3; ++j) {
      ca -= (double)a.world_to_cam[4 * j + i] * a.world_to_cam[4 * j + 3];
      cb -= (double)b.world_to_cam[4 * j + i] * b.world_to_cam[4 * j + 3];
    }
    d2 += (ca - cb) * (ca - cb);
  }
  return std::sqrt(d2);
}

namespace {

// Device allocations of the table start zeroed: no state is ever read from
// memory a previous owner left behind.
template <class T>
void dalloc(T*& p, uint64_t count) {
  const uint64_t bytes = (count > 0 ? count : 1) * sizeof(T);
  TGS_CUDA(cudaMalloc((void**)&p, bytes));
  TGS_CUDA(cudaMemset(p, 0, bytes));
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

}  // namespace

RenderList Table::render_list(uint32_t n_items) const {
  RenderList rl;
  rl.base = pool;
  rl.slot_stride = rec_floats;
  rl.B = B;
  rl.n_items = n_items;
  rl.item_slot = rl_dev;
  rl.item_count = rl_dev + max_items;
  rl.item_block = rl_dev + 2 * (uint64_t)max_items;
  rl.m_off = p_floats;
  rl.v_off = p_floats + m_floats;
  rl.bf16 = cfg.host_bf16 ? 1u : 0u;
  rl.sr = cfg.stochastic_round ? 1u : 0u;
  rl.seed = cfg.seed;
  return rl;
}

void Table::create(const tgs_config& c, uint64_t n, const float* params, std::FILE* ck) {
  cfg = c;
  TGS_CHECK(n > 0 && (params || ck), TGS_ERR_INVALID, "tgs_create: n must be > 0 and params non-null");
  TGS_CHECK(c.block_size >= 1 && c.block_size <= 65536, TGS_ERR_INVALID, "block_size out of range [1, 65536]");
  TGS_CHECK(c.max_batch >= 1 && c.max_width >= 1 && c.max_height >= 1, TGS_ERR_INVALID, "bad batch/image limits");
  TGS_CHECK(n < (1ull << 32), TGS_ERR_INVALID, "n must be below 2^32");
  TGS_CHECK(c.host_bf16 == 0 || c.block_size % 2 == 0, TGS_ERR_INVALID, "host_bf16 needs an even block_size");
  TGS_CHECK(c.loss <= 2, TGS_ERR_INVALID, "loss must be 0 (L1), 1 (L2) or 2 (L1 + D-SSIM)");
  N = n;
  B = c.block_size;
  K = (N + B - 1) / B;
  words = (K + 31) / 32;
  C = c.cache_blocks == 0 || c.cache_blocks > K ? K : c.cache_blocks;
  n_slots = C + (C < K ? c.spare_slots : 0);
  if (n_slots > K) n_slots = K;
  // FP32 record: params 59 B + m 59 B + v 59 B floats (708 bytes per Gaussian).
  // BF16 record: 14 FP32 fields + 45 BF16 SH-rest + BF16 m and v (382 bytes).
  if (c.host_bf16) {
    p_floats = (uint64_t)(F_BF16 * 4 + (D - F_BF16) * 2) * B / 4;
    m_floats = (uint64_t)D * 2 * B / 4;
  } else {
    p_floats = (uint64_t)D * B;
    m_floats = (uint64_t)D * B;
  }
  rec_floats = p_floats + 2 * m_floats;
  // render-list capacity (the per-camera buffers scale with it): the cache
  // capacity unless a smaller bound on one batch's visible blocks is given
  max_items = (uint32_t)(c.max_render_blocks && c.max_render_blocks < C ? c.max_render_blocks : C);
  V_cap = (uint64_t)max_items * B;

  // the control stream's short selection kernels are scheduled ahead of the
  // compute stream's long raster kernels (the host waits on the former)
  int prio_low = 0, prio_high = 0;
  TGS_CUDA(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high));
  TGS_CUDA(cudaStreamCreateWithPriority(&comp, cudaStreamNonBlocking, prio_low));
  TGS_CUDA(cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking));
  TGS_CUDA(cudaStreamCreateWithFlags(&h2d_late, cudaStreamNonBlocking));
  TGS_CUDA(cudaStreamCreateWithFlags(&tgtq, cudaStreamNonBlocking));
  TGS_CUDA(cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking));
  TGS_CUDA(cudaStreamCreateWithPriority(&ctl, cudaStreamNonBlocking, prio_high));
  for (cudaEvent_t* e : {&ev_comp, &ev_h2d, &ev_h2d_late, &ev_ctl, &ev_user, &ev_wb, &ev_snap, &ev_tgt_ready, &ev_tgt_used[0],
                         &ev_tgt_used[1]})
    TGS_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  TGS_CUDA(cudaEventCreate(&ev_stall_a));
  TGS_CUDA(cudaEventCreate(&ev_stall_b));
  copy_timer.on = true;

  if (ck) {
    // a checkpoint brings its own Morton order
    perm.resize(N);
    ck_read(ck, perm.data(), N * sizeof(uint32_t));
  } else {
    // ---- Morton order on the device (Sec. 3.3): centres -> codes -> stable sort
    {
      float* means = nullptr;
      uint32_t *codes = nullptr, *pm = nullptr;
      void* scr = nullptr;
      float* aabb = nullptr;
      dalloc(means, 3 * N);
      dalloc(codes, 2 * N);
      dalloc(pm, 2 * N);
      TGS_CUDA(cudaMalloc(&scr, radix_scratch_bytes(N)));
      dalloc(aabb, 16);
      perm.resize(N);
      if (c.morton) {
        TGS_CUDA(cudaMemcpy2DAsync(means, 3 * sizeof(float), params, D * sizeof(float), 3 * sizeof(float), N,
                                   cudaMemcpyHostToDevice, comp));
        morton_order(means, N, pm, codes, codes + N, pm + N, scr, aabb, comp);
        TGS_CUDA(cudaMemcpyAsync(perm.data(), pm, N * sizeof(uint32_t), cudaMemcpyDeviceToHost, comp));
        TGS_CUDA(cudaStreamSynchronize(comp));
      } else {
        // ablation (Tab. 5 "w/o Morton"): blocks are runs of the input order
        for (uint64_t g = 0; g < N; ++g) perm[g] = (uint32_t)g;
      }
      dfree(means); dfree(codes); dfree(pm); dfree(scr); dfree(aabb);
    }
  }

  // ---- host tier: K block records [params | m | v], field-major inside
  tier.init(K, rec_floats, c.host_cache_blocks, c.backing_path);
  if (ck) {
    if (!tier.tiered) {
      ck_read(ck, tier.pinned, K * rec_floats * sizeof(float));
    } else {
      std::vector<float> rec(rec_floats);
      for (uint64_t k = 0; k < K; ++k) {
        ck_read(ck, rec.data(), rec_floats * sizeof(float));
        tier.put_initial((uint32_t)k, rec.data());
      }
      tier.finish_initial();
    }
  } else {
    fill_host(params);
  }

  // ---- device cache and state
  dalloc(pool, n_slots * rec_floats);
  dalloc(spheres, K);
  dalloc(spheres_snap, K);
  dalloc(ages, K);
  dalloc(block_step, K);
  dalloc(readmit_dev, K);
  dalloc(churn_dev, 2);
  dalloc(dirty_dev, n_slots);
  TGS_CUDA(cudaMemsetAsync(ages, 0, K * sizeof(uint32_t), comp));
  {
    // never-accessed blocks start with the oldest age
    std::vector<uint32_t> a(K, 126u);
    TGS_CUDA(cudaMemcpy(ages, a.data(), K * sizeof(uint32_t), cudaMemcpyHostToDevice));
  }
  TGS_CUDA(cudaMemsetAsync(block_step, 0, K * sizeof(uint32_t), comp));
  TGS_CUDA(cudaMemsetAsync(dirty_dev, 0, n_slots, comp));
  for (uint32_t** b : {&r_bits, &r_next_bits, &acc_bits, &acc_next_bits, &kvis_union}) {
    dalloc(*b, words);
    TGS_CUDA(cudaMemsetAsync(*b, 0, words * sizeof(uint32_t), comp));
  }
  // visibility rows: a batch, or the cameras of an exact lookahead
  vis_rows = std::max<uint32_t>(cfg.max_batch, MAX_LOOKAHEAD);
  dalloc(kvis, (uint64_t)vis_rows * words);
  dalloc(planes_dev, vis_rows);
  TGS_CUDA(cudaMallocHost(&planes_host, vis_rows * sizeof(Planes)));
  dalloc(rb.flag, K);
  dalloc(rb.pos, K);
  dalloc(rb.key, 2 * K);
  dalloc(rb.blk, 2 * K);
  dalloc(rb.sel, K);
  dalloc(rb.tmp, K);
  dalloc(rb.tmp2, K);
  dalloc(rb.counters, 16);
  TGS_CUDA(cudaMalloc(&rb.scratch, residency_scratch_bytes(K)));
  dalloc(lists_dev, 3 * K + 16);
  // the selection's results arrive in mapped pinned memory (device stores)
  TGS_CUDA(cudaHostAlloc((void**)&lists_host, (3 * K + 16) * sizeof(uint32_t), cudaHostAllocMapped));
  TGS_CUDA(cudaHostAlloc((void**)&kvis_host_pinned, (uint64_t)vis_rows * words * sizeof(uint32_t), cudaHostAllocMapped));
  TGS_CUDA(cudaHostAlloc((void**)&r_host_pinned, words * sizeof(uint32_t), cudaHostAllocMapped));
  std::memset(lists_host, 0, (3 * K + 16) * sizeof(uint32_t));
  TGS_CUDA(cudaHostGetDevicePointer((void**)&lists_map, lists_host, 0));
  TGS_CUDA(cudaHostGetDevicePointer((void**)&kvis_map, kvis_host_pinned, 0));
  TGS_CUDA(cudaHostGetDevicePointer((void**)&r_map, r_host_pinned, 0));
  dalloc(rl_dev, 3ull * max_items);
  TGS_CUDA(cudaMallocHost(&rl_host, RL_RING * 3ull * max_items * sizeof(uint32_t)));
  for (auto& e : rl_ev) TGS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const uint64_t pix = (uint64_t)cfg.max_width * cfg.max_height;
  cams.resize(cfg.max_batch);
  dalloc(abort_dev, 2);
  TGS_CUDA(cudaMallocHost(&abort_host, 2 * sizeof(uint32_t)));
  for (auto& cs : cams) {
    // default pair capacity: two pairs per render-list Gaussian or 16 per
    // pixel (a mean tile list of 4,096 splats), whichever is larger
    const uint64_t def_pairs = std::max<uint64_t>(2 * V_cap, 16 * pix);
    cam_state_alloc(cs, V_cap, cfg.pair_capacity ? cfg.pair_capacity : def_pairs, (int)cfg.max_width,
                    (int)cfg.max_height);
    cs.step_flag = abort_dev;
  }
  dalloc(images, cfg.max_batch * pix * 3);
  dalloc(dl_dimg, cfg.max_batch * pix * 3);
  dalloc(targets_buf, 2 * cfg.max_batch * pix * 3);  // double buffer for host targets
  if (cfg.loss == 2) dalloc(ssim_buf, 3 * cfg.max_batch * pix * 3);
  TGS_CUDA(cudaMallocHost(&loss_ring, LOSS_RING * sizeof(float)));
  loss_norm.assign(LOSS_RING, 1.f);
  dalloc(touched, V_cap);
  dalloc(item_touched, max_items);
  dalloc(item_bias, max_items);
  V_cap_rows = V_cap;
  dalloc(rows_dev, V_cap + 1);  // touched rows, then their count
  dalloc(prows_dev, V_cap / 2 + 2);  // touched pairs, then their count
  dalloc(grad_local, (uint64_t)D * V_cap);
  dalloc(loss_dev, 4);
  TGS_CUDA(cudaMallocHost(&loss_host, 4 * sizeof(float)));

  init_spheres();
  if (ck) {
    // optimiser and residency state, then the bounds as the saved table had them
    std::vector<uint32_t> u(K);
    ck_read(ck, u.data(), K * sizeof(uint32_t));
    TGS_CUDA(cudaMemcpy(block_step, u.data(), K * sizeof(uint32_t), cudaMemcpyHostToDevice));
    ck_read(ck, u.data(), K * sizeof(uint32_t));
    TGS_CUDA(cudaMemcpy(ages, u.data(), K * sizeof(uint32_t), cudaMemcpyHostToDevice));
    std::vector<float4> sp(K);
    ck_read(ck, sp.data(), K * sizeof(float4));
    TGS_CUDA(cudaMemcpy(spheres, sp.data(), K * sizeof(float4), cudaMemcpyHostToDevice));
    ck_read(ck, sp.data(), K * sizeof(float4));
    TGS_CUDA(cudaMemcpy(spheres_snap, sp.data(), K * sizeof(float4), cudaMemcpyHostToDevice));
  }
  slot_of.assign(K, -1);
  block_of_slot.assign(n_slots, -1);
  free_fifo.clear();
  for (uint64_t sl = 0; sl < n_slots; ++sl) free_fifo.push_back((uint32_t)sl);
  dirty_host.assign(n_slots, 0);
  ever_loaded.assign(K, 0);
  wb_pending.assign(K, 0);
  admitted_at.assign(K, 0);
  resident_count = 0;
  slot_free_ev.assign(n_slots, nullptr);
  slot_has_ev.assign(n_slots, 0);
  for (auto& e : slot_free_ev) TGS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  TGS_CUDA(cudaEventRecord(ev_comp, comp));
  TGS_CUDA(cudaDeviceSynchronize());
}

// Host tier from caller rows (original order): block records with the
// parameters of ids kB.. in Morton order and zero moments (lanes past n zero).
void Table::fill_host(const float* params) {
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  const bool bf = cfg.host_bf16 != 0;
  for (unsigned w = 0; w < nt; ++w)
    th.emplace_back([&, w]() {
      // tiered: the record is built here and written to the log
      std::vector<float> buf(tier.tiered ? rec_floats : 0);
      for (uint64_t k = w; k < K; k += nt) {
        float* rec = tier.tiered ? buf.data() : tier.pinned + k * rec_floats;
        __nv_bfloat16* rec16 = reinterpret_cast<__nv_bfloat16*>(rec + (uint64_t)F_BF16 * B);
        std::memset(rec + p_floats, 0, 2 * m_floats * sizeof(float));
        for (uint32_t l = 0; l < B; ++l) {
          uint64_t g = k * B + l;
          const float* row = g < N ? params + (uint64_t)perm[g] * D : nullptr;
          for (int f = 0; f < D; ++f) {
            float x = row ? row[f] : 0.f;
            if (bf && f >= F_BF16)
              rec16[(uint64_t)(f - F_BF16) * B + l] = __float2bfloat16_rn(x);
            else
              rec[(uint64_t)f * B + l] = x;
          }
        }
        if (tier.tiered) tier.put_initial((uint32_t)k, rec);
      }
    });
  for (auto& t : th) t.join();
  tier.finish_initial();
}

// Bounding spheres of every block: means and log-scales of the host records
// are streamed through the first slots of the pool.
void Table::init_spheres() {
  uint64_t chunk = std::min<uint64_t>(n_slots, max_items);
  for (uint64_t k0 = 0; k0 < K; k0 += chunk) {
    uint64_t m = std::min(chunk, K - k0);
    if (!tier.tiered) {
      TGS_CUDA(cudaMemcpy2DAsync(pool, rec_floats * sizeof(float), tier.pinned + k0 * rec_floats,
                                 rec_floats * sizeof(float), 6ull * B * sizeof(float), m, cudaMemcpyHostToDevice, comp));
    } else {
      for (uint64_t j = 0; j < m; ++j) {
        const uint32_t blk = (uint32_t)(k0 + j);
        TGS_CUDA(cudaMemcpyAsync(pool + j * rec_floats, tier.acquire_read(blk), 6ull * B * sizeof(float),
                                 cudaMemcpyHostToDevice, comp));
        tier.record_use(blk, comp);
      }
    }
    for (uint64_t j = 0; j < m; ++j) {
      uint64_t blk = k0 + j;
      rl_host[j] = (uint32_t)j;
      rl_host[max_items + j] = (uint32_t)std::min<uint64_t>(B, N - blk * B);
      rl_host[2ull * max_items + j] = (uint32_t)blk;
    }
    TGS_CUDA(cudaMemcpyAsync(rl_dev, rl_host, 3ull * max_items * sizeof(uint32_t), cudaMemcpyHostToDevice, comp));
    block_bounds(render_list((uint32_t)m), nullptr, spheres, comp);
    TGS_CUDA(cudaStreamSynchronize(comp));
  }
  TGS_CUDA(cudaMemcpyAsync(spheres_snap, spheres, K * sizeof(float4), cudaMemcpyDeviceToDevice, comp));
  TGS_CUDA(cudaEventRecord(ev_snap, comp));
  TGS_CUDA(cudaStreamSynchronize(comp));
}

// Replaces every parameter (rows in the caller's original order), zeroes the
// moments and step counters and empties the cache.
void Table::set_params(const float* params) {
  TGS_CHECK(params, TGS_ERR_INVALID, "tgs_set_params: null params");
  for (cudaStream_t st : {comp, h2d, h2d_late, tgtq, d2h, ctl}) TGS_CUDA(cudaStreamSynchronize(st));
  tier.reset_log();
  fill_host(params);
  std::vector<uint32_t> a(K, 126u);
  TGS_CUDA(cudaMemcpy(ages, a.data(), K * sizeof(uint32_t), cudaMemcpyHostToDevice));
  TGS_CUDA(cudaMemset(block_step, 0, K * sizeof(uint32_t)));
  TGS_CUDA(cudaMemset(dirty_dev, 0, n_slots));
  TGS_CUDA(cudaMemset(abort_dev, 0, 2 * sizeof(uint32_t)));
  for (uint32_t* b : {r_bits, r_next_bits, acc_bits, acc_next_bits}) TGS_CUDA(cudaMemset(b, 0, words * sizeof(uint32_t)));
  slot_of.assign(K, -1);
  block_of_slot.assign(n_slots, -1);
  free_fifo.clear();
  for (uint64_t sl = 0; sl < n_slots; ++sl) free_fifo.push_back((uint32_t)sl);
  dirty_host.assign(n_slots, 0);
  slot_has_ev.assign(n_slots, 0);
  ever_loaded.assign(K, 0);
  wb_pending.assign(K, 0);
  admitted_at.assign(K, 0);
  resident_count = 0;
  TGS_CUDA(cudaMemset(readmit_dev, 0, K));
  prep = Prepared();
  init_spheres();
  TGS_CUDA(cudaEventRecord(ev_comp, comp));
  TGS_CUDA(cudaDeviceSynchronize());
}

void Table::destroy() {
  if (comp) cudaStreamSynchronize(comp);
  if (h2d) cudaStreamSynchronize(h2d);
  if (h2d_late) cudaStreamSynchronize(h2d_late);
  if (tgtq) cudaStreamSynchronize(tgtq);
  if (d2h) cudaStreamSynchronize(d2h);
  if (ctl) cudaStreamSynchronize(ctl);
  for (auto& cs : cams) cam_state_free(cs);
  void* dev[] = {pool, spheres, spheres_snap, ages, block_step, readmit_dev, churn_dev, dirty_dev, r_bits, r_next_bits, acc_bits, acc_next_bits, kvis,
                 kvis_union, planes_dev, rb.flag, rb.pos, rb.key, rb.blk, rb.sel, rb.tmp, rb.tmp2, rb.counters,
                 rb.scratch, lists_dev, rl_dev, images, dl_dimg, targets_buf, ssim_buf, touched, item_touched, item_bias, rows_dev, prows_dev, grad_local,
                 loss_dev, abort_dev};
  for (void* p : dev) dfree(p);
  tier.release();
  void* hst[] = {planes_host, lists_host, rl_host, loss_host, kvis_host_pinned, r_host_pinned, abort_host,
                 loss_ring};
  for (void* p : hst)
    if (p) cudaFreeHost(p);
  for (auto& e : slot_free_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : rl_ev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {ev_comp, ev_h2d, ev_h2d_late, ev_ctl, ev_user, ev_stall_a, ev_stall_b, ev_wb, ev_snap, ev_tgt_ready,
                        ev_tgt_used[0], ev_tgt_used[1]})
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : {comp, h2d, h2d_late, tgtq, d2h, ctl})
    if (s) cudaStreamDestroy(s);
}

// Stage 1 + Algorithm 1 for a batch, enqueued on the control stream: cull,
// select R_next, derive S+ / S- and the render list; their counts are copied
// back asynchronously.  prepare_finish() reads the lists and assigns slots.
void Table::prepare_enqueue(const tgs_camera* cs, uint32_t J, Prepared& out, bool own_batch) {
  TGS_CHECK(J >= 1 && J <= cfg.max_batch, TGS_ERR_INVALID, "batch size out of range");
  for (uint32_t j = 0; j < J; ++j) {
    TGS_CHECK(cs[j].width == cs[0].width && cs[j].height == cs[0].height, TGS_ERR_INVALID,
              "cameras of a batch must share the image size");
    TGS_CHECK(cs[j].width <= cfg.max_width && cs[j].height <= cfg.max_height, TGS_ERR_INVALID,
              "camera larger than max_width x max_height");
    TGS_CHECK(cs[j].znear > 0.f && cs[j].zfar > cs[j].znear && cs[j].fx > 0.f && cs[j].fy > 0.f,
              TGS_ERR_INVALID, "bad camera intrinsics");
    planes_host[j] = frustum_planes(cs[j], cfg.cull_margin_px);
  }
  out = Prepared();
  out.cams.assign(cs, cs + J);
  // Batch t is culled with the bounds refreshed through step t-2: a batch
  // selected at its own step reads the snapshot taken when step t-1 started;
  // the next batch selected at the start of step t reads the bounds after
  // step t-1 (the control stream waits for that step, the host does not).
  TGS_CUDA(cudaMemcpyAsync(planes_dev, planes_host, J * sizeof(Planes), cudaMemcpyHostToDevice, ctl));
  if (own_batch) {
    TGS_CUDA(cudaStreamWaitEvent(ctl, ev_snap, 0));
    cull_blocks(spheres_snap, K, planes_dev, (int)J, kvis, kvis_union, ctl);
  } else {
    TGS_CUDA(cudaStreamWaitEvent(ctl, ev_comp, 0));
    cull_blocks(spheres, K, planes_dev, (int)J, kvis, kvis_union, ctl);
  }
  select_enqueue(J, out, true);
}

// Learned prefetch: the predictor's visible set for the coming iterations
// (probability above the threshold for a horizon in pred_mask) replaces the
// culled set of a known next batch.  Ages and the accessed set are left alone:
// nothing has been rendered from the prediction yet.
void Table::prepare_enqueue_predicted(Prepared& out) {
  TGS_CHECK(predictor && !hist.empty(), TGS_ERR_STATE, "no predictor or camera history");
  out = Prepared();
  out.predicted = true;
  tgs_camera h[MLP_HIST];
  for (int s = 0; s < MLP_HIST; ++s) {
    int idx = (int)hist.size() - MLP_HIST + s;
    h[s] = hist[idx < 0 ? 0 : idx];
  }
  // reach: twice the longest camera move of the history per predicted step
  int hmax = 0;
  for (int q = 0; q < MLP_OUT; ++q)
    if (pred_mask >> q & 1u) hmax = q + 1;
  double vmax = 0.0;
  for (int s = 1; s < MLP_HIST; ++s) vmax = std::max(vmax, camera_distance(h[s - 1], h[s]));
  const float reach = (float)(2.0 * hmax * vmax);
  TGS_CUDA(cudaStreamWaitEvent(ctl, ev_comp, 0));
  mlp_predict_near(*predictor, spheres, K, h, reach, pred_mask, pred_threshold, kvis, ctl);
  TGS_CUDA(cudaMemcpyAsync(kvis_union, kvis, words * sizeof(uint32_t), cudaMemcpyDeviceToDevice, ctl));
  select_enqueue(1, out, false);
}

// Exact lookahead: the Level-1 visible sets of the next `horizon` cameras of
// the schedule replace the prediction (the upper bound the learned form is
// compared with); no ages or access are updated.
void Table::prepare_enqueue_lookahead(Prepared& out) {
  const uint64_t first = sched_pos;
  const uint32_t H = (uint32_t)std::min<uint64_t>(sched_horizon, schedule.size() - std::min(first, (uint64_t)schedule.size()));
  out = Prepared();
  if (H == 0) return;
  out.predicted = true;
  for (uint32_t j = 0; j < H; ++j) planes_host[j] = frustum_planes(schedule[first + j], cfg.cull_margin_px);
  TGS_CUDA(cudaMemcpyAsync(planes_dev, planes_host, H * sizeof(Planes), cudaMemcpyHostToDevice, ctl));
  TGS_CUDA(cudaStreamWaitEvent(ctl, ev_comp, 0));
  cull_blocks(spheres, K, planes_dev, (int)H, kvis, kvis_union, ctl);
  select_enqueue(H, out, false);
}

// Algorithm 1 on the visible sets in kvis (J rows); counts and sets are copied
// back asynchronously.  accessed = false: a prediction (no ages, no access).
void Table::select_enqueue(uint32_t J, Prepared& out, bool accessed) {
  uint64_t quota = cfg.quota == 0xFFFFFFFFu ? C / (2 * J) : cfg.quota;
  if (quota * J > C) quota = C / J;
  residency(acc_bits, r_bits, kvis, kvis_union, (int)J, K, ages, C, cfg.lambda, quota, r_next_bits,
            lists_dev, lists_dev + K, lists_dev + 2 * K, acc_next_bits, rb, ctl, accessed);
  // the selected set becomes the current one for the next selection
  std::swap(r_bits, r_next_bits);
  if (accessed) std::swap(acc_bits, acc_next_bits);
  // counts, the used list prefixes, the visible rows and the selected set
  // reach the host by device stores into mapped memory (one host wait)
  publish_sets(rb.counters, lists_dev, K, kvis, (uint64_t)J * words, r_bits, words, lists_map, kvis_map, r_map, ctl);
  TGS_CUDA(cudaEventRecord(ev_ctl, ctl));
  out.enqueued = true;
}

void Table::cull_only(const tgs_camera* cs, uint32_t J, uint8_t* vis_host) {
  TGS_CHECK(J >= 1 && J <= cfg.max_batch, TGS_ERR_INVALID, "batch size out of range");
  for (uint32_t j = 0; j < J; ++j) planes_host[j] = frustum_planes(cs[j], cfg.cull_margin_px);
  TGS_CUDA(cudaStreamWaitEvent(ctl, ev_comp, 0));
  TGS_CUDA(cudaMemcpyAsync(planes_dev, planes_host, J * sizeof(Planes), cudaMemcpyHostToDevice, ctl));
  // the union buffer of the selection is not touched: use the residency
  // scratch for the per-camera words
  cull_blocks(spheres, K, planes_dev, (int)J, rb.tmp, rb.tmp2, ctl);
  std::vector<uint32_t> w((uint64_t)J * words);
  TGS_CUDA(cudaMemcpyAsync(w.data(), rb.tmp, w.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctl));
  TGS_CUDA(cudaStreamSynchronize(ctl));
  for (uint32_t j = 0; j < J; ++j)
    for (uint64_t k = 0; k < K; ++k) vis_host[(uint64_t)j * K + k] = (w[(uint64_t)j * words + (k >> 5)] >> (k & 31)) & 1u;
}

// Host time blocked on the control stream (tracing counter).
void Table::wait_ctl() {
  const auto t0 = std::chrono::steady_clock::now();
  TGS_CUDA(cudaStreamSynchronize(ctl));
  stats.host_wait_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void Table::prepare_finish(Prepared& out) {
  TGS_CHECK(out.enqueued, TGS_ERR_STATE, "prepare_finish without prepare_enqueue");
  wait_ctl();
  const uint32_t J = (uint32_t)out.cams.size();
  const uint32_t np = lists_host[0], nm = lists_host[1], nr = lists_host[2];
  out.kvis_host.assign(kvis_host_pinned, kvis_host_pinned + (uint64_t)J * words);
  out.r_host.assign(r_host_pinned, r_host_pinned + words);
  const uint32_t* lists = lists_host + 16;
  out.s_plus.assign(lists, lists + np);
  out.s_minus.assign(lists + K, lists + K + nm);
  out.render_blocks.assign(lists + 2 * K, lists + 2 * K + nr);
  if (!cfg.differential && !out.predicted) {
    // ablation (Tab. 5 "w/o Tide"): no differential streaming -- every
    // resident block leaves (dirty ones written back) and the whole selected
    // set streams in again
    out.s_minus.clear();
    for (uint64_t b = 0; b < K; ++b)
      if (slot_of[b] >= 0) out.s_minus.push_back((uint32_t)b);
    out.s_plus.clear();
    for (uint64_t w = 0; w < words; ++w)
      for (uint32_t m = out.r_host[w]; m; m &= m - 1) out.s_plus.push_back((uint32_t)(w * 32 + __builtin_ctz(m)));
  }
  // demand hit counters: blocks of an actual batch already resident before
  // its selection (for the learned mode: after the prediction's copies)
  if (!out.predicted) {
    if (r_host_prev.size() != words) r_host_prev.assign(words, 0u);
    for (uint64_t w = 0; w < words; ++w) {
      uint32_t u = 0;
      for (uint32_t j = 0; j < J; ++j) u |= out.kvis_host[(uint64_t)j * words + w];
      stats.demand_blocks += __builtin_popcount(u);
      stats.demand_hits += __builtin_popcount(u & r_host_prev[w]);
    }
  } else {
    stats.predicted_blocks += np;
  }
  r_host_prev = out.r_host;

  // ---- slot assignment: S+ in ascending id order takes the free slots that
  // have been free the longest (a FIFO: their last write-back and reads are
  // long done, so an early copy never waits behind them on the copy stream),
  // the rest take the slots S- frees (ascending); S- slots not reused join
  // the back of the FIFO.
  CopyPlan& pl = out.plan;
  std::vector<uint32_t> ev_slots;
  for (uint32_t b : out.s_minus) {
    TGS_CHECK(slot_of[b] >= 0, TGS_ERR_STATE, "evicted block is not resident");
    ev_slots.push_back((uint32_t)slot_of[b]);
    pl.evict_block.push_back(b);
    pl.evict_slot.push_back((uint32_t)slot_of[b]);
  }
  std::sort(ev_slots.begin(), ev_slots.end());
  size_t ei = 0;
  for (uint32_t b : out.s_plus) {
    if (!free_fifo.empty()) {
      pl.early_block.push_back(b);
      pl.early_slot.push_back(free_fifo.front());
      free_fifo.pop_front();
    } else {
      TGS_CHECK(ei < ev_slots.size(), TGS_ERR_CAPACITY, "no slot left for an incoming block");
      pl.late_block.push_back(b);
      pl.late_slot.push_back(ev_slots[ei++]);
    }
  }
  for (; ei < ev_slots.size(); ++ei) free_fifo.push_back(ev_slots[ei]);
  if (!cfg.differential) {
    // a block may leave and come back in the same selection: every load goes
    // after the write-backs (late), so a reload sees its written-back record
    pl.late_block.insert(pl.late_block.begin(), pl.early_block.begin(), pl.early_block.end());
    pl.late_slot.insert(pl.late_slot.begin(), pl.early_slot.begin(), pl.early_slot.end());
    pl.early_block.clear();
    pl.early_slot.clear();
  }
  // host mirrors describe the state after this selection's copies
  for (size_t i = 0; i < pl.evict_block.size(); ++i) {
    slot_of[pl.evict_block[i]] = -1;
    block_of_slot[pl.evict_slot[i]] = -1;
  }
  for (size_t i = 0; i < pl.early_block.size(); ++i) {
    slot_of[pl.early_block[i]] = pl.early_slot[i];
    block_of_slot[pl.early_slot[i]] = pl.early_block[i];
  }
  for (size_t i = 0; i < pl.late_block.size(); ++i) {
    slot_of[pl.late_block[i]] = pl.late_slot[i];
    block_of_slot[pl.late_slot[i]] = pl.late_block[i];
  }
  out.render_slots.resize(out.render_blocks.size());
  for (size_t j = 0; j < out.render_blocks.size(); ++j) {
    int64_t s = slot_of[out.render_blocks[j]];
    TGS_CHECK(s >= 0, TGS_ERR_STATE, "render block without a slot");
    out.render_slots[j] = (uint32_t)s;
  }
  out.valid = true;
}

static void copy_block_in(Table& t, uint32_t b, uint32_t s, cudaStream_t st) {
  const uint64_t pf = t.p_floats;
  float* dst = t.pool + (uint64_t)s * t.rec_floats;
  const float* src = t.tier.acquire_read(b);
  if (t.slot_has_ev[s]) TGS_CUDA(cudaStreamWaitEvent(st, t.slot_free_ev[s], 0));
  // a block evicted earlier may still be on its way back to the host tier:
  // wait for the latest write-back batch (it includes this block's)
  if (t.wb_pending[b]) {
    TGS_CUDA(cudaStreamWaitEvent(st, t.ev_wb, 0));
    t.wb_pending[b] = 0;
  }
  if (t.cfg.moments_policy == 1) {
    TGS_CUDA(cudaMemcpyAsync(dst, src, pf * sizeof(float), cudaMemcpyHostToDevice, st));
    t.tier.record_use(b, st);
    TGS_CUDA(cudaMemsetAsync(dst + pf, 0, 2 * t.m_floats * sizeof(float), st));
    TGS_CUDA(cudaMemsetAsync(t.block_step + b, 0, sizeof(uint32_t), st));
    t.stats.bytes_h2d += pf * sizeof(float);
    t.stats.cold_restarts++;
  } else {
    TGS_CUDA(cudaMemcpyAsync(dst, src, t.rec_floats * sizeof(float), cudaMemcpyHostToDevice, st));
    t.tier.record_use(b, st);
    t.stats.bytes_h2d += t.rec_floats * sizeof(float);
  }
  // Tab. 9: the block's next update is its first after a re-admission
  // (under moments_policy 1 it starts from zeroed moments)
  if (t.ever_loaded[b]) TGS_CUDA(cudaMemsetAsync(t.readmit_dev + b, 1, 1, st));
  t.dirty_host[s] = 0;
  t.stats.blocks_in++;
  if (t.ever_loaded[b]) t.stats.readmissions++;
  t.ever_loaded[b] = 1;
  t.admitted_at[b] = t.stats.steps;
  t.resident_count++;
}

void Table::issue_early(Prepared& p) {
  if (!cfg.overlap) TGS_CUDA(cudaStreamWaitEvent(h2d, ev_comp, 0));
  if (!p.plan.early_block.empty()) {
    copy_timer.begin(0, h2d);
    for (size_t i = 0; i < p.plan.early_block.size(); ++i)
      copy_block_in(*this, p.plan.early_block[i], p.plan.early_slot[i], h2d);
    copy_timer.end(0, h2d);
  }
  TGS_CUDA(cudaEventRecord(ev_h2d, h2d));
}

// Write-back of S- after the compute that used them (ev_comp must be the last
// compute that may read those slots), then the loads into their slots.
void Table::issue_evictions_and_late(Prepared& p) {
  TGS_CUDA(cudaStreamWaitEvent(d2h, ev_comp, 0));
  const uint64_t pf = p_floats;
  bool any_wb = false;
  for (size_t i = 0; i < p.plan.evict_block.size(); ++i)
    if (dirty_host[p.plan.evict_slot[i]]) any_wb = true;
  if (any_wb) copy_timer.begin(1, d2h);
  for (size_t i = 0; i < p.plan.evict_block.size(); ++i) {
    uint32_t b = p.plan.evict_block[i], s = p.plan.evict_slot[i];
    if (dirty_host[s]) {
      uint64_t nf = cfg.moments_policy == 1 ? pf : rec_floats;
      TGS_CUDA(cudaMemcpyAsync(tier.acquire_write(b, nf == rec_floats), pool + (uint64_t)s * rec_floats,
                               nf * sizeof(float), cudaMemcpyDeviceToHost, d2h));
      tier.record_use(b, d2h);
      stats.bytes_d2h += nf * sizeof(float);
      stats.writebacks++;
      wb_pending[b] = 1;
    }
    dirty_host[s] = 0;
    TGS_CUDA(cudaEventRecord(slot_free_ev[s], d2h));
    slot_has_ev[s] = 1;
    stats.blocks_out++;
    stats.streaks++;
    stats.streak_steps += stats.steps - admitted_at[b];
    resident_count--;
  }
  if (any_wb) {
    copy_timer.end(1, d2h);
    TGS_CUDA(cudaEventRecord(ev_wb, d2h));
  }
  // loads into the slots S- frees wait (slot_free_ev) for the compute that
  // last read those slots and for their write-back; on their own stream,
  // so that the next selection's loads into free slots (and the host
  // targets) do not queue behind them
  if (!cfg.overlap) TGS_CUDA(cudaStreamWaitEvent(h2d_late, ev_comp, 0));
  if (!p.plan.late_block.empty()) {
    copy_timer.begin(0, h2d_late);
    for (size_t i = 0; i < p.plan.late_block.size(); ++i)
      copy_block_in(*this, p.plan.late_block[i], p.plan.late_slot[i], h2d_late);
    copy_timer.end(0, h2d_late);
  }
  TGS_CUDA(cudaEventRecord(ev_h2d_late, h2d_late));
}

void Table::collect_stall() {
  if (!stall_pending) return;
  TGS_CUDA(cudaEventSynchronize(ev_stall_b));
  float ms = 0.f;
  TGS_CUDA(cudaEventElapsedTime(&ms, ev_stall_a, ev_stall_b));
  stats.stall_ms += ms;
  stall_pending = false;
}

void Table::compute(const Prepared& p, const float* targets_dev, const float* targets_host, cudaStream_t user,
                    bool backward, float* image_out) {
  const uint32_t J = (uint32_t)p.cams.size();
  const uint32_t n_items = (uint32_t)p.render_blocks.size();
  TGS_CHECK(n_items <= max_items, TGS_ERR_CAPACITY, "render list exceeds the render-list capacity");
  const int W = (int)p.cams[0].width, H = (int)p.cams[0].height;
  const uint64_t pix = (uint64_t)W * H;
  collect_stall();
  // wait for this batch's incoming blocks; the wait is the exposed copy time
  TGS_CUDA(cudaEventRecord(ev_stall_a, comp));
  TGS_CUDA(cudaStreamWaitEvent(comp, ev_h2d, 0));
  TGS_CUDA(cudaStreamWaitEvent(comp, ev_h2d_late, 0));
  TGS_CUDA(cudaEventRecord(ev_stall_b, comp));
  stall_pending = true;
  const float* tgt = targets_dev;
  int tgt_buf = -1;
  if (backward) {
    // the bounds as this step starts: the next own-batch cull reads them while
    // this step refreshes the live copy
    TGS_CUDA(cudaMemcpyAsync(spheres_snap, spheres, K * sizeof(float4), cudaMemcpyDeviceToDevice, comp));
    TGS_CUDA(cudaEventRecord(ev_snap, comp));
    if (!tgt) {
      // host targets go up on the copy stream into the buffer the step before
      // last used, overlapping the work still queued ahead of this step
      TGS_CHECK(targets_host != nullptr, TGS_ERR_INVALID, "targets are required for a training step");
      tgt_buf = tgt_parity;
      tgt_parity ^= 1;
      float* dst = targets_buf + (uint64_t)tgt_buf * cfg.max_batch * pix * 3;
      if (tgt_used[tgt_buf]) TGS_CUDA(cudaStreamWaitEvent(tgtq, ev_tgt_used[tgt_buf], 0));
      TGS_CUDA(cudaMemcpyAsync(dst, targets_host, (uint64_t)J * pix * 3 * sizeof(float), cudaMemcpyHostToDevice, tgtq));
      TGS_CUDA(cudaEventRecord(ev_tgt_ready, tgtq));
      tgt = dst;
    }
  }
  // the render list goes up from a ring of pinned staging slots: a slot is
  // rewritten only after the copy that last read it has run
  const uint32_t rs = (uint32_t)(rl_seq++ % RL_RING);
  if (rl_ev_used[rs]) TGS_CUDA(cudaEventSynchronize(rl_ev[rs]));
  uint32_t* rlh = rl_host + (uint64_t)rs * 3 * max_items;
  for (uint32_t j = 0; j < n_items; ++j) {
    uint32_t b = p.render_blocks[j];
    rlh[j] = p.render_slots[j];
    rlh[max_items + j] = (uint32_t)std::min<uint64_t>(B, N - (uint64_t)b * B);
    rlh[2ull * max_items + j] = b;
  }
  if (n_items) {
    for (int q = 0; q < 3; ++q)
      TGS_CUDA(cudaMemcpyAsync(rl_dev + (uint64_t)q * max_items, rlh + (uint64_t)q * max_items,
                               n_items * sizeof(uint32_t), cudaMemcpyHostToDevice, comp));
    TGS_CUDA(cudaEventRecord(rl_ev[rs], comp));
    rl_ev_used[rs] = 1;
  }
  RenderList rl = render_list(n_items);
  const uint64_t V = rl.capacity();
  if (V) {
    TGS_CUDA(cudaMemsetAsync(touched, 0, V, comp));
    TGS_CUDA(cudaMemsetAsync(item_touched, 0, n_items * sizeof(uint32_t), comp));
  }
  for (uint32_t j = 0; j < J; ++j) {
    DevCam dc = make_devcam(p.cams[j]);
    float* img = image_out && J == 1 ? image_out : images + (uint64_t)j * pix * 3;
    render_forward(rl, dc, cfg.bg, cams[j], img, touched, item_touched, comp, &timer);
  }
  stats.last_render_blocks = n_items;
  if (backward) {
    if (tgt_buf >= 0) {
      TGS_CUDA(cudaStreamWaitEvent(comp, ev_tgt_ready, 0));
    } else {
      TGS_CUDA(cudaEventRecord(ev_user, user));
      TGS_CUDA(cudaStreamWaitEvent(comp, ev_user, 0));
    }
    TGS_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(float), comp));
    // the rows the chain rule stores and the optimiser updates
    touched_rows(rl, touched, rows_dev, rows_dev + V_cap_rows, comp, prows_dev, prows_dev + V_cap / 2 + 1);
    timer.begin(StageTimer::LOSS, comp);
    if (cfg.loss == 2)
      photometric_loss_ssim(images, tgt, (int)J, W, H, dl_dimg, loss_dev, ssim_buf, comp);
    else
      photometric_loss(images, tgt, (uint64_t)J * pix * 3, (int)cfg.loss, dl_dimg, loss_dev, comp);
    if (tgt_buf >= 0) {
      TGS_CUDA(cudaEventRecord(ev_tgt_used[tgt_buf], comp));
      tgt_used[tgt_buf] = 1;
    }
    // every step's loss reaches the host asynchronously (tgs_losses)
    TGS_CUDA(cudaMemcpyAsync(loss_ring + loss_enq % LOSS_RING, loss_dev, sizeof(float), cudaMemcpyDeviceToHost,
                             comp));
    loss_norm[loss_enq % LOSS_RING] = (float)((uint64_t)J * pix * 3);
    ++loss_enq;
    timer.end(StageTimer::LOSS, comp);
    std::vector<DevCam> dcs(J);
    std::vector<CamState*> css(J);
    for (uint32_t j = 0; j < J; ++j) {
      dcs[j] = make_devcam(p.cams[j]);
      css[j] = &cams[j];
      timer.begin(StageTimer::BWD, comp);
      render_backward_2d(rl, dcs[j], cfg.bg, cams[j], dl_dimg + (uint64_t)j * pix * 3, comp);
      timer.end(StageTimer::BWD, comp);
    }
    timer.begin(StageTimer::PBWD, comp);
    if (J <= (uint32_t)BatchGrad::MAXJ) {
      render_backward_params_batch(rl, dcs.data(), css.data(), (int)J, grad_local, rows_dev, rows_dev + V_cap_rows,
                                   comp);
    } else {
      for (uint32_t j = 0; j < J; ++j)
        render_backward_params(rl, dcs[j], cams[j], grad_local, j == 0 ? 0 : 1, comp, rows_dev,
                               rows_dev + V_cap_rows);
    }
    timer.end(StageTimer::PBWD, comp);
    timer.begin(StageTimer::ADAM, comp);
    mark_touched_blocks(rl, item_touched, block_step, dirty_dev, comp, abort_dev, cfg.beta1, cfg.beta2, item_bias,
                        readmit_dev, churn_dev);
    adam_render_list(rl, grad_local, rows_dev, rows_dev + V_cap_rows, item_bias, block_step, step_lrs(),
                     cfg.beta1, cfg.beta2, cfg.eps, comp, abort_dev, prows_dev, prows_dev + V_cap / 2 + 1);
    timer.end(StageTimer::ADAM, comp);
    // the next batch's cull (control stream) reads the bounds first
    TGS_CUDA(cudaStreamWaitEvent(comp, ev_ctl, 0));
    timer.begin(StageTimer::BOUNDS, comp);
    block_bounds(rl, item_touched, spheres, comp, abort_dev);
    timer.end(StageTimer::BOUNDS, comp);
    for (uint32_t j = 0; j < n_items; ++j) dirty_host[p.render_slots[j]] = 1;
    stats.resident_block_steps += resident_count;
    stats.steps++;
  }
  TGS_CUDA(cudaEventRecord(ev_comp, comp));
  // the caller's stream (NULL: the legacy default stream) waits for this step
  TGS_CUDA(cudaStreamWaitEvent(user, ev_comp, 0));
  last_cams = p.cams;
  last_render = p.render_blocks;
  last_splus = p.s_plus;
  last_sminus = p.s_minus;
  last_kvis_host = p.kvis_host;
  last_r_host = p.r_host;
}

static bool same_cams(const std::vector<tgs_camera>& a, const tgs_camera* b, uint32_t J) {
  if (a.size() != J) return false;
  return std::memcmp(a.data(), b, J * sizeof(tgs_camera)) == 0;
}

void Table::step(const tgs_camera* cs, uint32_t J, const tgs_camera* next, uint32_t nJ, const float* targets_dev,
                 const float* targets_host, cudaStream_t user, float* loss_out) {
  TGS_CHECK(cs && J >= 1, TGS_ERR_INVALID, "tgs_step: no cameras");
  const auto t_step = std::chrono::steady_clock::now();
  struct StepClock {
    Table& t;
    std::chrono::steady_clock::time_point t0;
    ~StepClock() {
      t.stats.host_step_ms +=
          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
  } step_clock{*this, t_step};
  check_overflow(false);
  if (!(prep.valid && same_cams(prep.cams, cs, J))) {
    // reactive path: select and stream this batch's working set now
    Prepared p;
    prepare_enqueue(cs, J, p, true);
    prepare_finish(p);
    issue_early(p);
    issue_evictions_and_late(p);
    prep = std::move(p);
  }
  Prepared cur = std::move(prep);
  prep = Prepared();
  Prepared nxt;
  for (uint32_t j = 0; j < J; ++j) {
    hist.push_back(cs[j]);
    if (hist.size() > MLP_HIST) hist.pop_front();
  }
  const bool prefetch = cfg.prefetch_mode == 1 && next && nJ >= 1;
  const bool learned = cfg.prefetch_mode == 2 && predictor != nullptr;
  const bool lookahead = cfg.prefetch_mode == 3 && !schedule.empty();
  if (lookahead) sched_pos += J;  // the schedule cursor moves past this batch
  // Algorithm 1 for batch t+1 runs on the control stream while batch t is
  // enqueued; it sees the bounds as of the start of step t
  if (prefetch) prepare_enqueue(next, nJ, nxt, false);
  if (learned) prepare_enqueue_predicted(nxt);
  if (lookahead) prepare_enqueue_lookahead(nxt);
  compute(cur, targets_dev, targets_host, user, true, nullptr);
  if (prefetch || learned || (lookahead && nxt.enqueued)) {
    prepare_finish(nxt);
    issue_early(nxt);
    issue_evictions_and_late(nxt);
    prep = std::move(nxt);
  }
  if (loss_out) {
    TGS_CUDA(cudaMemcpyAsync(loss_host, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, comp));
    TGS_CUDA(cudaStreamSynchronize(comp));
    check_overflow(true);
    const uint32_t Jc = (uint32_t)cur.cams.size();
    *loss_out = loss_host[0] / (float)((uint64_t)Jc * cur.cams[0].width * cur.cams[0].height * 3);
  }
  if (!cfg.overlap) TGS_CUDA(cudaStreamSynchronize(comp));
}

void Table::render(const tgs_camera& cam, float* image_dev, cudaStream_t user) {
  Prepared p;
  prepare_enqueue(&cam, 1, p, true);
  prepare_finish(p);
  issue_early(p);
  issue_evictions_and_late(p);
  compute(p, nullptr, nullptr, user, false, image_dev);
  // a render returns a complete image: after an overflow the buffers grow and
  // the same selection is rendered again
  if (check_overflow(true)) compute(p, nullptr, nullptr, user, false, image_dev);
  prep = Prepared();
}

uint64_t Table::losses(float* out, uint64_t max_count) {
  TGS_CUDA(cudaStreamSynchronize(comp));
  uint64_t first = loss_read;
  if (loss_enq - first > LOSS_RING) first = loss_enq - LOSS_RING;
  uint64_t n = 0;
  for (uint64_t k = first; k < loss_enq && n < max_count; ++k, ++n)
    out[n] = loss_ring[k % LOSS_RING] / loss_norm[k % LOSS_RING];
  loss_read = loss_enq;
  return n;
}

LrSet Table::step_lrs() const {
  LrSet r;
  if (!cfg.lr_schedule) {
    for (float& x : r.g) x = cfg.lr;
    return r;
  }
  for (int i = 0; i < 6; ++i) r.g[i] = cfg.lr_groups[i];
  const double T = cfg.lr_decay_steps > 0 ? (double)cfg.lr_decay_steps : 1.0;
  const double t = std::min<double>((double)stats.steps, T) / T;
  r.g[0] = (float)std::exp(std::log((double)cfg.lr_groups[0]) * (1.0 - t) + std::log((double)cfg.lr_means_final) * t);
  return r;
}

bool Table::check_overflow(bool wait) {
  bool any = false;
  uint64_t need = 0;
  for (auto& cs : cams) {
    if (!cam_state_counts(cs, wait) || !cs.overflow) continue;
    any = true;
    if (cs.pairs_needed > need) need = cs.pairs_needed;
  }
  if (!any) return false;
  for (cudaStream_t st : {comp, h2d, h2d_late, tgtq, d2h, ctl}) TGS_CUDA(cudaStreamSynchronize(st));
  TGS_CUDA(cudaMemcpy(abort_host, abort_dev, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  stats.dropped_steps += abort_host[1];
  stats.pair_overflows += 1;
  for (auto& cs : cams) {
    cam_state_grow_pairs(cs, need, comp);
    TGS_CUDA(cudaMemset(cs.counters + 2, 0, 2 * sizeof(uint32_t)));
    cs.overflow = false;
  }
  TGS_CUDA(cudaMemset(abort_dev, 0, 2 * sizeof(uint32_t)));
  return true;
}

// ---- checkpoint file: "TGSCKPT1", header (u64: n, B, K, rec_floats,
// host_bf16, moments_policy, steps), Morton permutation (u32 x n), host tier
// (K records), block step counters, ages (u32 x K each), bounds and the
// snapshot bounds (float4 x K each).
static const char kCkMagic[8] = {'T', 'G', 'S', 'C', 'K', 'P', 'T', '1'};

void ck_read(std::FILE* f, void* dst, uint64_t bytes) {
  char* d = static_cast<char*>(dst);
  while (bytes) {
    const size_t n = std::fread(d, 1, std::min<uint64_t>(bytes, 1ull << 28), f);
    TGS_CHECK(n > 0, TGS_ERR_INVALID, "checkpoint file is truncated");
    d += n;
    bytes -= n;
  }
}

static void ck_write(std::FILE* f, const void* src, uint64_t bytes) {
  const char* p = static_cast<const char*>(src);
  while (bytes) {
    const size_t n = std::fwrite(p, 1, std::min<uint64_t>(bytes, 1ull << 28), f);
    TGS_CHECK(n > 0, TGS_ERR_INVALID, "checkpoint write failed");
    p += n;
    bytes -= n;
  }
}

void Table::save(const char* path) {
  flush();
  for (cudaStream_t st : {comp, h2d, h2d_late, tgtq, d2h, ctl}) TGS_CUDA(cudaStreamSynchronize(st));
  std::FILE* f = std::fopen(path, "wb");
  TGS_CHECK(f, TGS_ERR_INVALID, std::string("cannot open checkpoint for writing: ") + path);
  try {
    const uint64_t hdr[7] = {N, B, K, rec_floats, cfg.host_bf16 ? 1ull : 0ull, cfg.moments_policy, stats.steps};
    ck_write(f, kCkMagic, sizeof(kCkMagic));
    ck_write(f, hdr, sizeof(hdr));
    ck_write(f, perm.data(), N * sizeof(uint32_t));
    if (!tier.tiered)
      ck_write(f, tier.pinned, K * rec_floats * sizeof(float));
    else
      for (uint64_t k = 0; k < K; ++k) ck_write(f, tier.acquire_read((uint32_t)k), rec_floats * sizeof(float));
    std::vector<uint32_t> u(K);
    TGS_CUDA(cudaMemcpy(u.data(), block_step, K * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    ck_write(f, u.data(), K * sizeof(uint32_t));
    TGS_CUDA(cudaMemcpy(u.data(), ages, K * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    ck_write(f, u.data(), K * sizeof(uint32_t));
    std::vector<float4> sp(K);
    TGS_CUDA(cudaMemcpy(sp.data(), spheres, K * sizeof(float4), cudaMemcpyDeviceToHost));
    ck_write(f, sp.data(), K * sizeof(float4));
    TGS_CUDA(cudaMemcpy(sp.data(), spheres_snap, K * sizeof(float4), cudaMemcpyDeviceToHost));
    ck_write(f, sp.data(), K * sizeof(float4));
  } catch (...) {
    std::fclose(f);
    throw;
  }
  TGS_CHECK(std::fclose(f) == 0, TGS_ERR_INVALID, "checkpoint close failed");
}

void Table::resume(const tgs_config& c, const char* path) {
  std::FILE* f = std::fopen(path, "rb");
  TGS_CHECK(f, TGS_ERR_INVALID, std::string("cannot open checkpoint: ") + path);
  try {
    char magic[8];
    ck_read(f, magic, sizeof(magic));
    TGS_CHECK(std::memcmp(magic, kCkMagic, sizeof(magic)) == 0, TGS_ERR_INVALID, "not a checkpoint file");
    uint64_t hdr[7];
    ck_read(f, hdr, sizeof(hdr));
    TGS_CHECK(hdr[1] == c.block_size && hdr[4] == (c.host_bf16 ? 1ull : 0ull), TGS_ERR_INVALID,
              "checkpoint block size or record form differs from the configuration");
    create(c, hdr[0], nullptr, f);
    TGS_CHECK(hdr[2] == K && hdr[3] == rec_floats, TGS_ERR_INVALID, "checkpoint layout differs");
    stats.steps = hdr[6];
  } catch (...) {
    std::fclose(f);
    throw;
  }
  std::fclose(f);
}

// Consistency barrier: every dirty resident block goes back to the host tier.
void Table::flush() {
  for (cudaStream_t st : {comp, h2d, h2d_late, tgtq, d2h}) TGS_CUDA(cudaStreamSynchronize(st));
  const uint64_t pf = p_floats;
  for (uint64_t s = 0; s < n_slots; ++s) {
    int64_t b = block_of_slot[s];
    if (b < 0 || !dirty_host[s]) continue;
    uint64_t nf = cfg.moments_policy == 1 ? pf : rec_floats;
    TGS_CUDA(cudaMemcpyAsync(tier.acquire_write((uint32_t)b, nf == rec_floats), pool + s * rec_floats,
                             nf * sizeof(float), cudaMemcpyDeviceToHost, d2h));
    tier.record_use((uint32_t)b, d2h);
    dirty_host[s] = 0;
  }
  TGS_CUDA(cudaStreamSynchronize(d2h));
}

}  // namespace tgs
