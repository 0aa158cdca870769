// Level-1 visibility and Algorithm 1 on the GPU.
//
// Culling: one thread per (block, camera); a warp covers 32 consecutive
// blocks and turns its 32 decisions into one bitmap word with __ballot_sync.
// Residency: candidates are compacted by a scan, ordered by a stable radix
// sort on the inverted FP32 score bits (score desc, id asc), the per-camera
// quotas and the global fill are prefix counts over that order, and the
// S+/S-/render lists are compacted from bitmaps with warp ballots and popc.
#include <math.h>

#include "sort.cuh"
#include "visibility.cuh"

namespace tgs {

namespace {

__device__ __forceinline__ int ord_of(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float of_ord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__global__ void k_aabb_init(int* box) {
  if (threadIdx.x < 3) {
    box[threadIdx.x] = 0x7FFFFFFF;
    box[3 + threadIdx.x] = (int)0x80000000;
  }
}

__global__ void k_aabb(const float* __restrict__ m, uint64_t n, int* box) {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float v = m[3 * i + a];
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&box[a], ord_of(lo[a]));
      atomicMax(&box[3 + a], ord_of(hi[a]));
    }
  }
}

// 10-bit quantisation per axis (FP32: q = min(1023, floor(((x - lo) / (hi - lo)) * 1024))),
// bits interleaved with x in bit 0 of each triple.
__global__ void k_morton(const float* __restrict__ m, uint64_t n, const int* __restrict__ box,
                         uint32_t* __restrict__ codes, uint32_t* __restrict__ idx) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t code = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float lo = of_ord(box[a]), hi = of_ord(box[3 + a]);
    float ext = __fsub_rn(hi, lo);
    uint32_t q = 0;
    if (ext > 0.f) {
      float f = __fmul_rn(__fdiv_rn(__fsub_rn(m[3 * i + a], lo), ext), 1024.f);
      float fl = floorf(f);
      q = fl < 0.f ? 0u : (fl > 1023.f ? 1023u : (uint32_t)fl);
    }
#pragma unroll
    for (int b = 0; b < 10; ++b) code |= ((q >> b) & 1u) << (3 * b + a);
  }
  codes[i] = code;
  idx[i] = (uint32_t)i;
}

__global__ void k_aabb_out(const int* box, float* out) {
  if (threadIdx.x < 6) out[threadIdx.x] = of_ord(box[threadIdx.x]);
}

__global__ void k_cull(const float4* __restrict__ sph, uint64_t K, const Planes* __restrict__ pl, int J,
                       uint32_t* __restrict__ vis, uint32_t* __restrict__ vis_union, uint64_t words) {
  uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float4 s = k < K ? sph[k] : make_float4(0.f, 0.f, 0.f, -1.f);
  uint32_t uni = 0;
  for (int j = 0; j < J; ++j) {
    bool visible = k < K;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      float4 p = pl[j].p[q];
      float d = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(p.x, s.x), __fmul_rn(p.y, s.y)), __fmul_rn(p.z, s.z)), p.w);
      if (d < -s.w) visible = false;
    }
    uint32_t word = __ballot_sync(0xffffffffu, visible);
    uni |= word;
    if ((threadIdx.x & 31) == 0 && (k >> 5) < words) vis[(uint64_t)j * words + (k >> 5)] = word;
  }
  if ((threadIdx.x & 31) == 0 && (k >> 5) < words) vis_union[k >> 5] = uni;
}

__device__ __forceinline__ bool bit(const uint32_t* w, uint64_t k) { return (w[k >> 5] >> (k & 31)) & 1u; }

// ages, candidate flags and inverted score keys
__global__ void k_res_score(const uint32_t* __restrict__ k_acc, const uint32_t* __restrict__ r_cur,
                            const uint32_t* __restrict__ k_next_union, uint64_t K, uint32_t* __restrict__ ages,
                            float lambda, int age_update, uint32_t* __restrict__ flag, uint32_t* __restrict__ key) {
  uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  uint32_t a = ages[k];
  bool r = bit(r_cur, k), kn = bit(k_next_union, k);
  if (age_update) {
    if (r && bit(k_acc, k)) a = 0;
    else if (a < 126) a += 1;
    ages[k] = a;
  }
  float lam = lambda;
  float oml = __fsub_rn(1.f, lam);
  float t = __fmul_rn(oml, ldexpf(1.f, -(int)a));
  float sc = __fadd_rn(kn ? lam : 0.f, t);
  flag[k] = (r || kn) ? 1u : 0u;
  key[k] = ~__float_as_uint(sc);  // scores are >= 0: inverted bits sort descending
}

__global__ void k_res_compact(uint64_t K, const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos,
                              const uint32_t* __restrict__ key_in, uint32_t* __restrict__ key,
                              uint32_t* __restrict__ blk) {
  uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K || !flag[k]) return;
  key[pos[k]] = key_in[k];
  blk[pos[k]] = (uint32_t)k;
}

// counters: [0] n_plus [1] n_minus [2] n_render [3] n_cand [4] n_quota
__global__ void k_res_camflag(const uint32_t* __restrict__ counters, const uint32_t* __restrict__ blk,
                              const uint32_t* __restrict__ knext_j, uint32_t* __restrict__ f) {
  uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= counters[3]) return;
  f[s] = bit(knext_j, blk[s]) ? 1u : 0u;
}

__global__ void k_res_quota(const uint32_t* __restrict__ counters, const uint32_t* __restrict__ f,
                            const uint32_t* __restrict__ rank, uint64_t quota, uint32_t* __restrict__ sel) {
  uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= counters[3]) return;
  if (f[s] && rank[s] < quota) sel[s] = 1u;
}

__global__ void k_res_unsel(const uint32_t* __restrict__ counters, const uint32_t* __restrict__ sel,
                            uint32_t* __restrict__ f) {
  uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= counters[3]) return;
  f[s] = sel[s] ? 0u : 1u;
}

// fill: unselected candidates in order until the capacity is used; writes r_next bits
__global__ void k_res_fill(const uint32_t* __restrict__ counters, const uint32_t* __restrict__ blk,
                           const uint32_t* __restrict__ sel, const uint32_t* __restrict__ rank_unsel,
                           const uint32_t* __restrict__ n_sel, uint64_t capacity, uint32_t* __restrict__ r_next) {
  uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= counters[3]) return;
  uint64_t q = *n_sel;
  bool take = sel[s] || (q < capacity && rank_unsel[s] < capacity - q);
  if (take) {
    uint32_t b = blk[s];
    atomicOr(&r_next[b >> 5], 1u << (b & 31));
  }
}

// S+ = r_next & ~r_cur, S- = r_cur & ~r_next, render = r_next & k_union:
// per word, popcounts of the three masks (for the scans), then the lists.
__global__ void k_res_wordcount(const uint32_t* __restrict__ r_next, const uint32_t* __restrict__ r_cur,
                                const uint32_t* __restrict__ ku, uint64_t words, uint32_t* __restrict__ c_plus,
                                uint32_t* __restrict__ c_minus, uint32_t* __restrict__ c_rend) {
  uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= words) return;
  uint32_t rn = r_next[w], rc = r_cur[w];
  c_plus[w] = __popc(rn & ~rc);
  c_minus[w] = __popc(rc & ~rn);
  c_rend[w] = __popc(rn & ku[w]);
}

__global__ void k_res_lists(const uint32_t* __restrict__ r_next, const uint32_t* __restrict__ r_cur,
                            const uint32_t* __restrict__ ku, uint64_t words, const uint32_t* __restrict__ o_plus,
                            const uint32_t* __restrict__ o_minus, const uint32_t* __restrict__ o_rend,
                            uint32_t* __restrict__ s_plus, uint32_t* __restrict__ s_minus,
                            uint32_t* __restrict__ render, uint32_t* __restrict__ acc_out) {
  uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= words) return;
  uint32_t rn = r_next[w], rc = r_cur[w];
  uint32_t masks[3] = {rn & ~rc, rc & ~rn, rn & ku[w]};
  acc_out[w] = masks[2];
  uint32_t offs[3] = {o_plus[w], o_minus[w], o_rend[w]};
  uint32_t* outs[3] = {s_plus, s_minus, render};
  for (int q = 0; q < 3; ++q) {
    uint32_t m = masks[q], o = offs[q];
    while (m) {
      int b = __ffs(m) - 1;
      outs[q][o++] = (uint32_t)(w * 32 + b);
      m &= m - 1;
    }
  }
}

}  // namespace

Planes frustum_planes(const tgs_camera& c, float m) {
  const int TX = ((int)c.width + TILE - 1) / TILE, TY = ((int)c.height + TILE - 1) / TILE;
  float n[6][3], w[6];
  n[0][0] = 0.f; n[0][1] = 0.f; n[0][2] = 1.f; w[0] = -c.znear;
  n[1][0] = 0.f; n[1][1] = 0.f; n[1][2] = -1.f; w[1] = c.zfar;
  n[2][0] = c.fx; n[2][1] = 0.f; n[2][2] = c.cx + m;
  n[3][0] = -c.fx; n[3][1] = 0.f; {
    float e = (float)(TILE * TX) + m;
    n[3][2] = e - c.cx;
  }
  n[4][0] = 0.f; n[4][1] = c.fy; n[4][2] = c.cy + m;
  n[5][0] = 0.f; n[5][1] = -c.fy; {
    float e = (float)(TILE * TY) + m;
    n[5][2] = e - c.cy;
  }
  for (int p = 2; p < 6; ++p) {
    w[p] = 0.f;
    float s0 = n[p][0] * n[p][0];
    float s1 = n[p][1] * n[p][1];
    float s2 = n[p][2] * n[p][2];
    float ss = s0 + s1;
    ss = ss + s2;
    float len = sqrtf(ss);
    for (int a = 0; a < 3; ++a) n[p][a] = n[p][a] / len;
  }
  Planes out;
  const float* M = c.world_to_cam;
  for (int p = 0; p < 6; ++p) {
    float nw[3];
    for (int j = 0; j < 3; ++j) {
      float a0 = M[0 * 4 + j] * n[p][0];
      float a1 = M[1 * 4 + j] * n[p][1];
      float a2 = M[2 * 4 + j] * n[p][2];
      float s = a0 + a1;
      nw[j] = s + a2;
    }
    float b0 = M[3] * n[p][0];
    float b1 = M[7] * n[p][1];
    float b2 = M[11] * n[p][2];
    float s = b0 + b1;
    s = s + b2;
    out.p[p] = make_float4(nw[0], nw[1], nw[2], s + w[p]);
  }
  return out;
}

void morton_order(const float* means, uint64_t n, uint32_t* perm, uint32_t* codes, uint32_t* codes_alt,
                  uint32_t* perm_alt, void* scratch, float* aabb_dev, cudaStream_t s) {
  int* box = (int*)aabb_dev + 8;
  k_aabb_init<<<1, 32, 0, s>>>(box);
  TGS_LAUNCHED();
  unsigned g = div_up(n, 256);
  if (g > 8 * NSM) g = 8 * NSM;
  k_aabb<<<g, 256, 0, s>>>(means, n, box);
  TGS_LAUNCHED();
  k_aabb_out<<<1, 32, 0, s>>>(box, aabb_dev);
  TGS_LAUNCHED();
  k_morton<<<div_up(n, 256), 256, 0, s>>>(means, n, box, codes, perm);
  TGS_LAUNCHED();
  radix_sort_pairs(codes, perm, codes_alt, perm_alt, n, 30, scratch, s);
}

void cull_blocks(const float4* spheres, uint64_t K, const Planes* planes_dev, int J, uint32_t* vis,
                 uint32_t* vis_union, cudaStream_t s) {
  uint64_t words = (K + 31) / 32;
  k_cull<<<div_up(words * 32, 256), 256, 0, s>>>(spheres, K, planes_dev, J, vis, vis_union, words);
  TGS_LAUNCHED();
}

size_t residency_scratch_bytes(uint64_t K) {
  size_t a = radix_scratch_bytes(K), b = scan_scratch_bytes(K);
  return a > b ? a : b;
}

void residency(const uint32_t* k_acc, const uint32_t* r_cur, const uint32_t* k_next, const uint32_t* k_next_union,
               int J, uint64_t K, uint32_t* ages, uint64_t capacity, float lambda, uint64_t quota, uint32_t* r_next,
               uint32_t* s_plus, uint32_t* s_minus, uint32_t* render, uint32_t* acc_out, ResidencyBuffers& rb,
               cudaStream_t s, bool age_update) {
  const uint64_t words = (K + 31) / 32;
  const unsigned gk = div_up(K, 256);
  uint32_t* cnt = rb.counters;
  k_res_score<<<gk, 256, 0, s>>>(k_acc, r_cur, k_next_union, K, ages, lambda, age_update ? 1 : 0, rb.flag, rb.tmp);
  TGS_LAUNCHED();
  exclusive_scan_u32(rb.flag, rb.pos, cnt + 3, K, rb.scratch, s);
  // non-candidates keep the largest key and sort after every candidate (the
  // sort is stable and candidates precede them); the candidate count stays on
  // the device and the kernels below read it from counters[3]
  TGS_CUDA(cudaMemsetAsync(rb.key, 0xFF, K * sizeof(uint32_t), s));
  k_res_compact<<<gk, 256, 0, s>>>(K, rb.flag, rb.pos, rb.tmp, rb.key, rb.blk);
  TGS_LAUNCHED();
  TGS_CUDA(cudaMemsetAsync(rb.sel, 0, K * sizeof(uint32_t), s));
  radix_sort_pairs(rb.key, rb.blk, rb.key + K, rb.blk + K, K, 32, rb.scratch, s);
  for (int j = 0; j < J; ++j) {
    k_res_camflag<<<gk, 256, 0, s>>>(cnt, rb.blk, k_next + (uint64_t)j * words, rb.tmp);
    TGS_LAUNCHED();
    exclusive_scan_u32(rb.tmp, rb.tmp2, nullptr, K, rb.scratch, s);
    k_res_quota<<<gk, 256, 0, s>>>(cnt, rb.tmp, rb.tmp2, quota, rb.sel);
    TGS_LAUNCHED();
  }
  exclusive_scan_u32(rb.sel, rb.tmp2, cnt + 4, K, rb.scratch, s);  // n_sel -> counters[4]
  k_res_unsel<<<gk, 256, 0, s>>>(cnt, rb.sel, rb.tmp);
  TGS_LAUNCHED();
  exclusive_scan_u32(rb.tmp, rb.tmp2, nullptr, K, rb.scratch, s);
  TGS_CUDA(cudaMemsetAsync(r_next, 0, words * sizeof(uint32_t), s));
  k_res_fill<<<gk, 256, 0, s>>>(cnt, rb.blk, rb.sel, rb.tmp2, cnt + 4, capacity, r_next);
  TGS_LAUNCHED();
  const unsigned gw = div_up(words, 256);
  uint32_t* cp = rb.flag;           // reuse: per-word counts
  uint32_t* cm = rb.pos;
  uint32_t* cr = rb.tmp;
  k_res_wordcount<<<gw, 256, 0, s>>>(r_next, r_cur, k_next_union, words, cp, cm, cr);
  TGS_LAUNCHED();
  exclusive_scan_u32(cp, cp, cnt + 0, words, rb.scratch, s);
  exclusive_scan_u32(cm, cm, cnt + 1, words, rb.scratch, s);
  exclusive_scan_u32(cr, cr, cnt + 2, words, rb.scratch, s);
  k_res_lists<<<gw, 256, 0, s>>>(r_next, r_cur, k_next_union, words, cp, cm, cr, s_plus, s_minus, render, acc_out);
  TGS_LAUNCHED();
}

}  // namespace tgs
