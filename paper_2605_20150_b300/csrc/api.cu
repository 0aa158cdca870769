// extern "C" boundary of the library (declared in include/tidegs.h).  Every
// entry point converts exceptions into a status and a thread-local message.
#include <cuda_bf16.h>

#include <cstring>
#include <string>
#include <vector>

#include "table.cuh"

namespace tgs {

uint64_t g_launches = 0;
static thread_local std::string g_err;
void set_last_error(const std::string& m) { g_err = m; }

template <class F>
static tgs_status guard(F&& f) {
  try {
    g_err.clear();
    f();
    return TGS_OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return TGS_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return TGS_ERR_INVALID;
  }
}

// Resident rasteriser context: one camera's state over an identity render
// list (block g / B of the caller's array is item g / B).
struct Raster {
  CamState cs;
  uint64_t max_n = 0;
  uint32_t* rl_dev = nullptr;
  uint64_t rl_n = 0;
  uint32_t rl_B = 0;
  uint32_t* rl_items = nullptr;
  uint32_t max_items_alloc = 0;
};

static RenderList resident_list(Raster& r, const float* params, uint64_t n, uint32_t B, cudaStream_t s) {
  TGS_CHECK(B >= 1 && n >= 1 && n <= r.max_n, TGS_ERR_INVALID, "n or block_size out of range for this context");
  uint32_t items = (uint32_t)((n + B - 1) / B);
  TGS_CHECK((uint64_t)items * B <= r.cs.cap_v, TGS_ERR_CAPACITY, "n exceeds the context capacity");
  if (r.rl_n != n || r.rl_B != B) {
    if (items > r.max_items_alloc) {
      if (r.rl_dev) cudaFree(r.rl_dev);
      TGS_CUDA(cudaMalloc(&r.rl_dev, 3ull * items * sizeof(uint32_t)));
      r.max_items_alloc = items;
    }
    std::vector<uint32_t> h(3ull * items);
    for (uint32_t j = 0; j < items; ++j) {
      h[j] = j;
      h[items + j] = (uint32_t)std::min<uint64_t>(B, n - (uint64_t)j * B);
      h[2ull * items + j] = j;
    }
    TGS_CUDA(cudaMemcpyAsync(r.rl_dev, h.data(), h.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    TGS_CUDA(cudaStreamSynchronize(s));
    r.rl_n = n;
    r.rl_B = B;
  }
  RenderList rl;
  rl.base = const_cast<float*>(params);
  rl.slot_stride = (uint64_t)D * B;
  rl.B = B;
  rl.n_items = items;
  rl.item_slot = r.rl_dev;
  rl.item_count = r.rl_dev + items;
  rl.item_block = r.rl_dev + 2ull * items;
  rl.m_off = rl.v_off = 0;
  return rl;
}

}  // namespace tgs

using namespace tgs;

struct tgs_table {
  Table t;
};
struct tgs_raster {
  Raster r;
};
struct tgs_mlp {
  Mlp m;
};

extern "C" {

const char* tgs_last_error(void) { return g_err.c_str(); }

void tgs_default_config(tgs_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->block_size = 4096;
  c->moments_policy = 0;
  c->prefetch_mode = 1;
  c->overlap = 1;
  c->cache_blocks = 0;
  c->spare_slots = 64;
  c->max_batch = 4;
  c->max_width = 1920;
  c->max_height = 1080;
  c->quota = 0xFFFFFFFFu;
  c->lambda = 0.75f;
  c->lr = 1e-3f;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->eps = 1e-15f;
  c->cull_margin_px = 4.0f;
  c->bg[0] = c->bg[1] = c->bg[2] = 0.f;
  c->loss = 0;
  c->host_bf16 = 0;
  c->stochastic_round = 1;
  c->seed = 1234;
  // 3DGS rates: means 1.6e-4 -> 1.6e-6 over 30k steps (scale by the scene
  // extent), log-scales 5e-3, rotation 1e-3, opacity 5e-2, SH DC 2.5e-3,
  // SH rest 2.5e-3 / 20
  c->lr_schedule = 0;
  const float g[6] = {1.6e-4f, 5e-3f, 1e-3f, 5e-2f, 2.5e-3f, 1.25e-4f};
  for (int i = 0; i < 6; ++i) c->lr_groups[i] = g[i];
  c->lr_means_final = 1.6e-6f;
  c->lr_decay_steps = 30000;
  c->differential = 1;
  c->morton = 1;
}

tgs_status tgs_create(const tgs_config* cfg, uint64_t n, const float* params_host, tgs_table** out) {
  return guard([&] {
    TGS_CHECK(cfg && out, TGS_ERR_INVALID, "tgs_create: null config or output");
    *out = nullptr;
    tgs_table* t = new tgs_table();
    try {
      t->t.create(*cfg, n, params_host);
    } catch (...) {
      t->t.destroy();
      delete t;
      throw;
    }
    *out = t;
  });
}

tgs_status tgs_checkpoint(tgs_table* t, const char* path) {
  return guard([&] {
    TGS_CHECK(t && path, TGS_ERR_INVALID, "tgs_checkpoint: null argument");
    t->t.save(path);
  });
}

tgs_status tgs_resume(const tgs_config* cfg, const char* path, tgs_table** out) {
  return guard([&] {
    TGS_CHECK(cfg && path && out, TGS_ERR_INVALID, "tgs_resume: null argument");
    *out = nullptr;
    tgs_table* t = new tgs_table();
    try {
      t->t.resume(*cfg, path);
    } catch (...) {
      t->t.destroy();
      delete t;
      throw;
    }
    *out = t;
  });
}

void tgs_destroy(tgs_table* t) {
  if (!t) return;
  t->t.destroy();
  delete t;
}

tgs_status tgs_step(tgs_table* t, const tgs_camera* cams, uint32_t batch, const tgs_camera* next_cams,
                    uint32_t next_batch, const float* targets_dev, const float* targets_host, void* stream,
                    float* loss_out) {
  return guard([&] {
    TGS_CHECK(t && cams, TGS_ERR_INVALID, "tgs_step: null table or cameras");
    TGS_CHECK(targets_dev || targets_host, TGS_ERR_INVALID, "tgs_step: targets required");
    t->t.step(cams, batch, next_cams, next_batch, targets_dev, targets_host, (cudaStream_t)stream, loss_out);
  });
}

tgs_status tgs_render(tgs_table* t, const tgs_camera* cam, float* image_dev, void* stream) {
  return guard([&] {
    TGS_CHECK(t && cam && image_dev, TGS_ERR_INVALID, "tgs_render: null argument");
    t->t.render(*cam, image_dev, (cudaStream_t)stream);
  });
}

tgs_status tgs_set_prefetch_mode(tgs_table* t, uint32_t mode) {
  return guard([&] {
    TGS_CHECK(t && mode <= 3, TGS_ERR_INVALID, "tgs_set_prefetch_mode: bad argument");
    t->t.cfg.prefetch_mode = mode;
  });
}

tgs_status tgs_losses(tgs_table* t, float* out_host, uint64_t max_count, uint64_t* count) {
  return guard([&] {
    TGS_CHECK(t && out_host && count, TGS_ERR_INVALID, "tgs_losses: null argument");
    *count = t->t.losses(out_host, max_count);
  });
}

tgs_status tgs_set_schedule(tgs_table* t, const tgs_camera* cams, uint64_t n, uint32_t horizon) {
  return guard([&] {
    TGS_CHECK(t && (cams || n == 0), TGS_ERR_INVALID, "tgs_set_schedule: null argument");
    TGS_CHECK(horizon >= 1 && horizon <= Table::MAX_LOOKAHEAD, TGS_ERR_INVALID, "tgs_set_schedule: horizon out of [1, 8]");
    t->t.schedule.assign(cams, cams + n);
    t->t.sched_pos = 0;
    t->t.sched_horizon = horizon;
  });
}

tgs_status tgs_sync(tgs_table* t) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_sync: null table");
    for (cudaStream_t s : {t->t.comp, t->t.h2d, t->t.h2d_late, t->t.tgtq, t->t.d2h, t->t.ctl}) TGS_CUDA(cudaStreamSynchronize(s));
    t->t.collect_stall();
    t->t.check_overflow(true);
  });
}

static void read_state(Table& T, float* params, float* m1, float* m2, bool original_order) {
  T.flush();
  const uint64_t B = T.B, rf = T.rec_floats;
  const bool bf = T.cfg.host_bf16 != 0;
  // moments of resident blocks under cold restart live only in the cache
  std::vector<float> resident;
  std::vector<int64_t> slot_of = T.slot_of;
  if ((m1 || m2) && T.cfg.moments_policy == 1) {
    resident.resize(T.n_slots * rf);
    TGS_CUDA(cudaMemcpy(resident.data(), T.pool, T.n_slots * rf * sizeof(float), cudaMemcpyDeviceToHost));
  }
  auto moment = [&](const float* rec, int q, int f, uint64_t l) -> float {
    const float* base = rec + T.p_floats + (uint64_t)q * T.m_floats;
    if (bf) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[(uint64_t)f * B + l]);
    return base[(uint64_t)f * B + l];
  };
  const float* rec = nullptr;
  uint64_t rec_k = ~0ull;
  for (uint64_t g = 0; g < T.N; ++g) {
    uint64_t k = g / B, l = g % B;
    if (k != rec_k) {
      rec = T.tier.acquire_read((uint32_t)k);
      rec_k = k;
    }
    uint64_t row = original_order ? T.perm[g] : g;
    if (params)
      for (int f = 0; f < D; ++f)
        params[row * D + f] =
            (bf && f >= F_BF16)
                ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(rec + (uint64_t)F_BF16 * B)[(uint64_t)(f - F_BF16) * B + l])
                : rec[(uint64_t)f * B + l];
    const float* mrec = rec;
    if (T.cfg.moments_policy == 1) mrec = slot_of[k] >= 0 ? resident.data() + (uint64_t)slot_of[k] * rf : nullptr;
    for (int q = 0; q < 2; ++q) {
      float* dst = q == 0 ? m1 : m2;
      if (!dst) continue;
      for (int f = 0; f < D; ++f) dst[row * D + f] = mrec ? moment(mrec, q, f, l) : 0.f;
    }
  }
}

// Rows ids[0..count) (block-order ids) of the state after the consistency
// barrier; under cold restart the moments of a resident block come from its
// HBM slot (one record copy per distinct resident block), of others are 0.
static void read_state_rows(Table& T, const int64_t* ids, uint64_t count, float* params, float* m1, float* m2) {
  T.flush();
  const uint64_t B = T.B, rf = T.rec_floats;
  const bool bf = T.cfg.host_bf16 != 0;
  std::vector<float> slotrec;
  int64_t slot_blk = -1;
  auto field = [&](const float* rec, int f, uint64_t l) -> float {
    if (bf && f >= F_BF16)
      return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(rec + (uint64_t)F_BF16 * B)[(uint64_t)(f - F_BF16) * B + l]);
    return rec[(uint64_t)f * B + l];
  };
  auto moment = [&](const float* rec, int q, int f, uint64_t l) -> float {
    const float* base = rec + T.p_floats + (uint64_t)q * T.m_floats;
    if (bf) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(base)[(uint64_t)f * B + l]);
    return base[(uint64_t)f * B + l];
  };
  for (uint64_t r = 0; r < count; ++r) {
    TGS_CHECK(ids[r] >= 0 && (uint64_t)ids[r] < T.N, TGS_ERR_INVALID, "tgs_get_state_rows: id out of range");
    const uint64_t g = (uint64_t)ids[r], k = g / B, l = g % B;
    const float* rec = T.tier.acquire_read((uint32_t)k);
    if (params)
      for (int f = 0; f < D; ++f) params[r * D + f] = field(rec, f, l);
    if (!m1 && !m2) continue;
    const float* mrec = rec;
    if (T.cfg.moments_policy == 1) {
      mrec = nullptr;
      if (T.slot_of[k] >= 0) {
        if (slot_blk != (int64_t)k) {
          slotrec.resize(rf);
          TGS_CUDA(cudaMemcpy(slotrec.data(), T.pool + (uint64_t)T.slot_of[k] * rf, rf * sizeof(float),
                              cudaMemcpyDeviceToHost));
          slot_blk = (int64_t)k;
        }
        mrec = slotrec.data();
      }
    }
    for (int q = 0; q < 2; ++q) {
      float* dst = q == 0 ? m1 : m2;
      if (!dst) continue;
      for (int f = 0; f < D; ++f) dst[r * D + f] = mrec ? moment(mrec, q, f, l) : 0.f;
    }
  }
}

tgs_status tgs_get_state_rows(tgs_table* t, const int64_t* ids, uint64_t count, float* params_host, float* m1_host,
                              float* m2_host) {
  return guard([&] {
    TGS_CHECK(t && (ids || count == 0), TGS_ERR_INVALID, "tgs_get_state_rows: null argument");
    read_state_rows(t->t, ids, count, params_host, m1_host, m2_host);
  });
}

tgs_status tgs_set_params(tgs_table* t, const float* params_host) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_set_params: null table");
    t->t.set_params(params_host);
  });
}

tgs_status tgs_get_params(tgs_table* t, float* out_host) {
  return guard([&] {
    TGS_CHECK(t && out_host, TGS_ERR_INVALID, "tgs_get_params: null argument");
    read_state(t->t, out_host, nullptr, nullptr, true);
  });
}

tgs_status tgs_get_state(tgs_table* t, float* params_host, float* m1_host, float* m2_host, uint32_t* steps_host) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_get_state: null table");
    read_state(t->t, params_host, m1_host, m2_host, false);
    if (steps_host)
      TGS_CUDA(cudaMemcpy(steps_host, t->t.block_step, t->t.K * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  });
}

tgs_status tgs_get_block_order(tgs_table* t, int64_t* perm_host) {
  return guard([&] {
    TGS_CHECK(t && perm_host, TGS_ERR_INVALID, "tgs_get_block_order: null argument");
    for (uint64_t g = 0; g < t->t.N; ++g) perm_host[g] = t->t.perm[g];
  });
}

tgs_status tgs_get_spheres(tgs_table* t, float* spheres_host) {
  return guard([&] {
    TGS_CHECK(t && spheres_host, TGS_ERR_INVALID, "tgs_get_spheres: null argument");
    TGS_CUDA(cudaStreamSynchronize(t->t.comp));
    TGS_CUDA(cudaMemcpy(spheres_host, t->t.spheres, t->t.K * sizeof(float4), cudaMemcpyDeviceToHost));
  });
}

tgs_status tgs_get_sizes(tgs_table* t, uint64_t* n, uint64_t* k, uint64_t* slots) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_get_sizes: null table");
    if (n) *n = t->t.N;
    if (k) *k = t->t.K;
    if (slots) *slots = t->t.n_slots;
  });
}

tgs_status tgs_get_sets(tgs_table* t, uint8_t* k_visible, uint8_t* r_resident, uint8_t* k_per_camera,
                        int64_t* s_plus, uint64_t* n_plus, int64_t* s_minus, uint64_t* n_minus) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_get_sets: null table");
    Table& T = t->t;
    const uint64_t J = T.last_cams.size();
    TGS_CHECK(J > 0, TGS_ERR_STATE, "tgs_get_sets: no step yet");
    for (uint64_t k = 0; k < T.K; ++k) {
      uint8_t u = 0;
      for (uint64_t j = 0; j < J; ++j) {
        uint8_t b = (T.last_kvis_host[j * T.words + (k >> 5)] >> (k & 31)) & 1u;
        if (k_per_camera) k_per_camera[j * T.K + k] = b;
        u |= b;
      }
      if (k_visible) k_visible[k] = u;
      if (r_resident) r_resident[k] = (T.last_r_host[k >> 5] >> (k & 31)) & 1u;
    }
    if (n_plus) *n_plus = T.last_splus.size();
    if (n_minus) *n_minus = T.last_sminus.size();
    if (s_plus)
      for (size_t i = 0; i < T.last_splus.size(); ++i) s_plus[i] = T.last_splus[i];
    if (s_minus)
      for (size_t i = 0; i < T.last_sminus.size(); ++i) s_minus[i] = T.last_sminus[i];
  });
}

static void camera_record(CamState& cs, const std::vector<uint32_t>& blocks, uint64_t B, uint64_t N,
                          const float* image_dev, uint64_t* n_gauss, uint64_t* n_pairs, int64_t* ids, float* splat,
                          int32_t* rect, uint32_t* pair_vals, uint32_t* ranges, float* image, float* t_final,
                          int32_t* n_last, float* grad2d) {
  uint64_t ng = 0;
  for (uint32_t b : blocks) ng += std::min<uint64_t>(B, N - (uint64_t)b * B);
  if (n_gauss) *n_gauss = ng;
  if (n_pairs) *n_pairs = cs.n_pairs;
  const uint64_t pix = (uint64_t)cs.W * cs.H, tiles = (uint64_t)cs.TX * cs.TY;
  if (ids)
    for (uint64_t i = 0; i < ng; ++i) ids[i] = (int64_t)blocks[i / B] * (int64_t)B + (int64_t)(i % B);
  if (splat || rect) {
    std::vector<float2> xy(ng);
    std::vector<float> depth(ng);
    std::vector<float4> co(ng), rgb(ng);
    std::vector<int> rad(ng);
    std::vector<uint32_t> nt(ng);
    std::vector<ushort4> rc(ng);
    if (ng) {
      TGS_CUDA(cudaMemcpy(xy.data(), cs.xy, ng * sizeof(float2), cudaMemcpyDeviceToHost));
      TGS_CUDA(cudaMemcpy(depth.data(), cs.depth, ng * sizeof(float), cudaMemcpyDeviceToHost));
      TGS_CUDA(cudaMemcpy(co.data(), cs.conic_o, ng * sizeof(float4), cudaMemcpyDeviceToHost));
      TGS_CUDA(cudaMemcpy(rgb.data(), cs.rgb, ng * sizeof(float4), cudaMemcpyDeviceToHost));
      TGS_CUDA(cudaMemcpy(rad.data(), cs.radius, ng * sizeof(int), cudaMemcpyDeviceToHost));
      TGS_CUDA(cudaMemcpy(nt.data(), cs.ntiles, ng * sizeof(uint32_t), cudaMemcpyDeviceToHost));
      TGS_CUDA(cudaMemcpy(rc.data(), cs.rect, ng * sizeof(ushort4), cudaMemcpyDeviceToHost));
    }
    for (uint64_t i = 0; i < ng; ++i) {
      bool v = nt[i] != 0;
      if (splat) {
        float* o = splat + 12 * i;
        if (v) {
          o[0] = xy[i].x; o[1] = xy[i].y; o[2] = depth[i];
          o[3] = co[i].x; o[4] = co[i].y; o[5] = co[i].z; o[6] = co[i].w;
          o[7] = rgb[i].x; o[8] = rgb[i].y; o[9] = rgb[i].z; o[10] = (float)rad[i];
        } else {
          for (int q = 0; q < 11; ++q) o[q] = 0.f;
        }
        o[11] = v ? 1.f : 0.f;
      }
      if (rect) {
        int32_t* o = rect + 4 * i;
        o[0] = v ? rc[i].x : 0; o[1] = v ? rc[i].y : 0; o[2] = v ? rc[i].z : 0; o[3] = v ? rc[i].w : 0;
      }
    }
  }
  const uint64_t np = std::min(cs.n_pairs, cs.cap_pairs);
  if (pair_vals && np) TGS_CUDA(cudaMemcpy(pair_vals, cs.pvals, np * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  if (ranges) TGS_CUDA(cudaMemcpy(ranges, cs.ranges, tiles * sizeof(uint2), cudaMemcpyDeviceToHost));
  if (image && image_dev) TGS_CUDA(cudaMemcpy(image, image_dev, pix * 3 * sizeof(float), cudaMemcpyDeviceToHost));
  if (t_final) TGS_CUDA(cudaMemcpy(t_final, cs.t_final, pix * sizeof(float), cudaMemcpyDeviceToHost));
  if (n_last) TGS_CUDA(cudaMemcpy(n_last, cs.n_last, pix * sizeof(int), cudaMemcpyDeviceToHost));
  if (grad2d && ng) {
    const uint64_t st = cs.g2_stride;
    TGS_CHECK(st >= ng, TGS_ERR_STATE, "no backward for this render list");
    std::vector<float> g(9 * st);
    TGS_CUDA(cudaMemcpy(g.data(), cs.g2, 9 * st * sizeof(float), cudaMemcpyDeviceToHost));
    for (uint64_t i = 0; i < ng; ++i)
      for (int q = 0; q < 9; ++q) grad2d[9 * i + q] = g[(uint64_t)q * st + i];
  }
}

tgs_status tgs_get_camera_record(tgs_table* t, uint32_t j, uint64_t* n_gauss, uint64_t* n_pairs, int64_t* ids,
                                 float* splat, int32_t* rect, uint32_t* pair_vals, uint32_t* ranges, float* image,
                                 float* t_final, int32_t* n_last, float* grad2d) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_get_camera_record: null table");
    Table& T = t->t;
    TGS_CHECK(j < T.last_cams.size(), TGS_ERR_INVALID, "camera index out of range of the last batch");
    TGS_CUDA(cudaStreamSynchronize(T.comp));
    cam_state_counts(T.cams[j], true);
    const uint64_t pix = (uint64_t)T.cams[j].W * T.cams[j].H;
    camera_record(T.cams[j], T.last_render, T.B, T.N, T.images + (uint64_t)j * pix * 3, n_gauss, n_pairs, ids,
                  splat, rect, pair_vals, ranges, image, t_final, n_last, grad2d);
  });
}

tgs_status tgs_get_stats(tgs_table* t, tgs_stats* out) {
  return guard([&] {
    TGS_CHECK(t && out, TGS_ERR_INVALID, "tgs_get_stats: null argument");
    t->t.collect_stall();
    t->t.copy_timer.collect();
    t->t.check_overflow(true);
    if (!t->t.last_cams.empty()) {
      CamState& cs = t->t.cams[t->t.last_cams.size() - 1];
      cam_state_counts(cs, true);
      t->t.stats.last_pairs = cs.n_pairs;
      t->t.stats.last_visible = cs.n_vis;
    }
    *out = t->t.stats;
    unsigned long long churn[2];
    TGS_CUDA(cudaStreamSynchronize(t->t.comp));
    if (t->t.predictor) {
      TGS_CUDA(cudaStreamSynchronize(t->t.ctl));
      mlp_check(*t->t.predictor);
    }
    TGS_CUDA(cudaMemcpy(churn, t->t.churn_dev, sizeof(churn), cudaMemcpyDeviceToHost));
    out->block_updates = churn[0];
    out->cold_updates = churn[1];
    out->host_cache_hits = t->t.tier.hits;
    out->host_cache_misses = t->t.tier.misses;
    out->log_bytes_read = t->t.tier.bytes_read;
    out->log_bytes_written = t->t.tier.bytes_written;
    out->kernel_launches = g_launches;
    out->h2d_ms = t->t.copy_timer.ms[0];
    out->d2h_ms = t->t.copy_timer.ms[1];
  });
}

tgs_status tgs_set_stage_timing(tgs_table* t, int enable) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_set_stage_timing: null table");
    t->t.timer.on = enable != 0;
  });
}

tgs_status tgs_get_stage_ms(tgs_table* t, double* ms8, uint64_t* counts8, int reset) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_get_stage_ms: null table");
    t->t.timer.collect();
    for (int i = 0; i < StageTimer::NSTAGE; ++i) {
      if (ms8) ms8[i] = t->t.timer.ms[i];
      if (counts8) counts8[i] = t->t.timer.count[i];
    }
    if (reset) t->t.timer.reset();
  });
}

tgs_status tgs_visible_blocks(tgs_table* t, const tgs_camera* cams, uint32_t J, uint8_t* vis_host) {
  return guard([&] {
    TGS_CHECK(t && cams && vis_host, TGS_ERR_INVALID, "tgs_visible_blocks: null argument");
    t->t.cull_only(cams, J, vis_host);
  });
}

tgs_status tgs_mlp_create(uint64_t max_blocks, uint32_t seed, tgs_mlp** out) {
  return guard([&] {
    TGS_CHECK(out && max_blocks > 0, TGS_ERR_INVALID, "tgs_mlp_create: bad arguments");
    *out = nullptr;
    tgs_mlp* m = new tgs_mlp();
    try {
      mlp_alloc(m->m, max_blocks, seed);
    } catch (...) {
      mlp_free(m->m);
      delete m;
      throw;
    }
    *out = m;
  });
}

void tgs_mlp_destroy(tgs_mlp* m) {
  if (!m) return;
  mlp_free(m->m);
  delete m;
}

uint64_t tgs_mlp_num_params(void) { return MLP_NPARAM; }

tgs_status tgs_mlp_get_params(tgs_mlp* m, float* host) {
  return guard([&] {
    TGS_CHECK(m && host, TGS_ERR_INVALID, "tgs_mlp_get_params: null argument");
    TGS_CUDA(cudaMemcpy(host, m->m.params, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
  });
}

tgs_status tgs_mlp_set_params(tgs_mlp* m, const float* host) {
  return guard([&] {
    TGS_CHECK(m && host, TGS_ERR_INVALID, "tgs_mlp_set_params: null argument");
    TGS_CUDA(cudaMemcpy(m->m.params, host, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    TGS_CUDA(cudaMemset(m->m.m, 0, MLP_NPARAM * sizeof(float)));
    TGS_CUDA(cudaMemset(m->m.v, 0, MLP_NPARAM * sizeof(float)));
    m->m.step = 0;
    mlp_refresh_bf16(m->m, 0);
    TGS_CUDA(cudaDeviceSynchronize());
  });
}

tgs_status tgs_mlp_forward(tgs_mlp* m, const float* spheres_dev, uint64_t K, const tgs_camera* hist,
                           float* logits_dev, void* stream) {
  return guard([&] {
    TGS_CHECK(m && spheres_dev && hist && logits_dev, TGS_ERR_INVALID, "tgs_mlp_forward: null argument");
    mlp_forward(m->m, reinterpret_cast<const float4*>(spheres_dev), K, hist, logits_dev, false,
                (cudaStream_t)stream);
  });
}

tgs_status tgs_mlp_train_step(tgs_mlp* m, const float* spheres_dev, uint64_t K, const tgs_camera* hist,
                              const float* labels_dev, float pos_weight, float lr, float weight_decay, int apply,
                              float* loss_out, float* grads_host, void* stream) {
  return guard([&] {
    TGS_CHECK(m && spheres_dev && hist && labels_dev, TGS_ERR_INVALID, "tgs_mlp_train_step: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    mlp_forward(m->m, reinterpret_cast<const float4*>(spheres_dev), K, hist, nullptr, true, s);
    float l = mlp_train_step(m->m, K, labels_dev, pos_weight, lr, weight_decay, apply != 0, s);
    if (loss_out) *loss_out = l;
    if (grads_host) TGS_CUDA(cudaMemcpy(grads_host, m->m.grads, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
  });
}

tgs_status tgs_set_predictor(tgs_table* t, tgs_mlp* m, float threshold, uint32_t horizon_mask) {
  return guard([&] {
    TGS_CHECK(t, TGS_ERR_INVALID, "tgs_set_predictor: null table");
    TGS_CHECK(!m || m->m.max_rows >= t->t.K, TGS_ERR_CAPACITY, "predictor smaller than the table's block count");
    TGS_CHECK(threshold > 0.f && threshold < 1.f && (horizon_mask & 15u), TGS_ERR_INVALID,
              "threshold must be in (0, 1) and horizon_mask non-empty");
    t->t.predictor = m ? &m->m : nullptr;
    t->t.pred_threshold = threshold;
    t->t.pred_mask = horizon_mask & 15u;
  });
}

tgs_status tgs_raster_create(uint64_t max_gaussians, uint32_t max_width, uint32_t max_height, tgs_raster** out) {
  return guard([&] {
    TGS_CHECK(out && max_gaussians > 0 && max_width > 0 && max_height > 0, TGS_ERR_INVALID,
              "tgs_raster_create: bad sizes");
    *out = nullptr;
    tgs_raster* r = new tgs_raster();
    try {
      // capacity leaves room for the partial last block of any block size
      r->r.max_n = max_gaussians;
      cam_state_alloc(r->r.cs, max_gaussians + 65536, 4 * max_gaussians, (int)max_width, (int)max_height);
    } catch (...) {
      cam_state_free(r->r.cs);
      delete r;
      throw;
    }
    *out = r;
  });
}

void tgs_raster_destroy(tgs_raster* r) {
  if (!r) return;
  cam_state_free(r->r.cs);
  if (r->r.rl_dev) cudaFree(r->r.rl_dev);
  delete r;
}

tgs_status tgs_raster_forward(tgs_raster* r, const float* params_dev, uint64_t n, uint32_t block_size,
                              const tgs_camera* cam, const float* bg3, float* image_dev, void* stream) {
  return guard([&] {
    TGS_CHECK(r && params_dev && cam && image_dev, TGS_ERR_INVALID, "tgs_raster_forward: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    RenderList rl = resident_list(r->r, params_dev, n, block_size, s);
    float bg[3] = {0.f, 0.f, 0.f};
    if (bg3) std::memcpy(bg, bg3, sizeof(bg));
    render_forward(rl, make_devcam(*cam), bg, r->r.cs, image_dev, nullptr, nullptr, s);
    // the image is returned complete: after a pair overflow the buffers grow
    // and the render runs again
    cam_state_counts(r->r.cs, true);
    if (r->r.cs.overflow) {
      cam_state_grow_pairs(r->r.cs, r->r.cs.pairs_needed, s);
      TGS_CUDA(cudaMemset(r->r.cs.counters + 2, 0, 2 * sizeof(uint32_t)));
      r->r.cs.overflow = false;
      render_forward(rl, make_devcam(*cam), bg, r->r.cs, image_dev, nullptr, nullptr, s);
    }
  });
}

tgs_status tgs_raster_backward(tgs_raster* r, const float* params_dev, uint64_t n, uint32_t block_size,
                               const tgs_camera* cam, const float* bg3, const float* dl_dimage_dev, float* grad_dev,
                               uint8_t* touched_dev, void* stream) {
  return guard([&] {
    TGS_CHECK(r && params_dev && cam && dl_dimage_dev && grad_dev, TGS_ERR_INVALID,
              "tgs_raster_backward: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    RenderList rl = resident_list(r->r, params_dev, n, block_size, s);
    float bg[3] = {0.f, 0.f, 0.f};
    if (bg3) std::memcpy(bg, bg3, sizeof(bg));
    DevCam dc = make_devcam(*cam);
    TGS_CHECK(dc.W == r->r.cs.W && dc.H == r->r.cs.H, TGS_ERR_STATE, "backward camera differs from the forward");
    render_backward_2d(rl, dc, bg, r->r.cs, dl_dimage_dev, s);
    // grad_dev shares the parameters' block layout
    render_backward_params(rl, dc, r->r.cs, grad_dev, 2, s);
    if (touched_dev) mark_visible_bytes(rl, r->r.cs, touched_dev, s);
  });
}

tgs_status tgs_adam(float* params_dev, const float* grad_dev, float* m1_dev, float* m2_dev,
                    const uint8_t* touched_dev, uint32_t* step_dev, uint64_t n, uint32_t block_size, float lr,
                    float beta1, float beta2, float eps, void* stream) {
  return guard([&] {
    TGS_CHECK(params_dev && grad_dev && m1_dev && m2_dev && touched_dev && step_dev && n > 0 && block_size > 0,
              TGS_ERR_INVALID, "tgs_adam: null argument or empty size");
    adam_dense(params_dev, grad_dev, m1_dev, m2_dev, touched_dev, step_dev, n, block_size, lr, beta1, beta2, eps,
               (cudaStream_t)stream);
  });
}

}  // extern "C"
