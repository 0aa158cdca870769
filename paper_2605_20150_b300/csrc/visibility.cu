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


// ---- Algorithm 1 in one CTA (K <= SEL_MAX_K): the same selection as the
// multi-kernel path below, in shared memory, so a selection costs one launch
// (the control stream's kernels otherwise each wait for a free SM slot behind
// the compute stream's raster CTAs).
//
// Scores take at most 254 values (visibility flag x age 0..126): candidates
// are ordered by a stable counting sort on the rank of their FP32 score among
// the distinct score values (descending; equal scores share a rank, so ties
// resolve to the lower block id, as in the stable sort by score bits).
constexpr int SEL_THREADS = 1024;
constexpr int SEL_WARPS = SEL_THREADS / 32;
constexpr int SEL_BUCKETS = 254;  // visibility flag x 127 ages
constexpr int SEL_MAX_K = 65536;

__device__ __forceinline__ float res_score(int kn, uint32_t a, float lam) {
  const float oml = __fsub_rn(1.f, lam);
  const float t = __fmul_rn(oml, ldexpf(1.f, -(int)a));
  return __fadd_rn(kn ? lam : 0.f, t);
}

__device__ __forceinline__ uint32_t block_scan_excl(uint32_t x, uint32_t* sw, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sw[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t v = sw[lane];
    uint32_t vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    sw[lane] = vi - v;
    if (lane == 31) sw[32] = vi;
  }
  __syncthreads();
  const uint32_t r = sw[w] + inc - x;
  if (total) *total = sw[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SEL_THREADS) k_select_small(
    const uint32_t* __restrict__ k_acc, const uint32_t* __restrict__ r_cur, const uint32_t* __restrict__ k_next,
    const uint32_t* __restrict__ k_union, int J, uint32_t K, uint32_t* __restrict__ ages, float lambda,
    int age_update, uint32_t capacity, uint32_t quota, uint32_t* __restrict__ r_next,
    uint32_t* __restrict__ s_plus, uint32_t* __restrict__ s_minus, uint32_t* __restrict__ render,
    uint32_t* __restrict__ acc_out, uint32_t* __restrict__ counters) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t words = (K + 31) / 32;
  uint16_t* ids = reinterpret_cast<uint16_t*>(smem);                           // sorted candidates
  uint32_t* hist = reinterpret_cast<uint32_t*>(smem + 2 * SEL_MAX_K);          // [warps][buckets]
  uint32_t* selb = hist + SEL_WARPS * 256;                                     // selected (sorted index bits)
  uint32_t* rnb = selb + SEL_MAX_K / 32;                                       // r_next bits
  __shared__ uint16_t rank_of[SEL_BUCKETS];
  __shared__ float score_of[SEL_BUCKETS];
  __shared__ uint8_t first_of[SEL_BUCKETS];
  __shared__ uint32_t sw[33];
  __shared__ uint32_t s_nr, s_ncand, s_nsel;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;

  // score of every bucket and its rank among the distinct scores (descending)
  if (tid < SEL_BUCKETS) score_of[tid] = res_score(tid >= 127, (uint32_t)(tid % 127), lambda);
  for (uint32_t e = tid; e < SEL_WARPS * 256; e += SEL_THREADS) hist[e] = 0;
  for (uint32_t e = tid; e < SEL_MAX_K / 32; e += SEL_THREADS) selb[e] = 0;
  for (uint32_t e = tid; e < words; e += SEL_THREADS) rnb[e] = 0;
  __syncthreads();
  // first_of[b]: b is the first bucket with its score value
  if (tid < SEL_BUCKETS) {
    const float sc = score_of[tid];
    bool first = true;
    for (int c = 0; c < tid; ++c)
      if (score_of[c] == sc) first = false;
    first_of[tid] = first ? 1 : 0;
  }
  __syncthreads();
  if (tid < SEL_BUCKETS) {
    const float sc = score_of[tid];
    uint32_t r = 0;
    for (int b = 0; b < SEL_BUCKETS; ++b)
      if (first_of[b] && score_of[b] > sc) ++r;
    rank_of[tid] = (uint16_t)r;
  }
  __syncthreads();

  // ages, candidate flags, per-warp histograms of score ranks (warp w walks the
  // contiguous id range [w * chunk, (w + 1) * chunk) 32 ids at a time)
  const uint32_t chunk = ((K + SEL_WARPS - 1) / SEL_WARPS + 31) / 32 * 32;
  const uint32_t k_lo = wid * chunk, k_hi = min(K, k_lo + chunk);
  for (uint32_t k0 = k_lo; k0 < k_hi; k0 += 32) {
    const uint32_t k = k0 + lane;
    bool cand = false;
    uint32_t bkt = 0;
    if (k < k_hi) {
      uint32_t a = ages[k];
      const bool r = (r_cur[k >> 5] >> (k & 31)) & 1u, kn = (k_union[k >> 5] >> (k & 31)) & 1u;
      if (age_update) {
        if (r && ((k_acc[k >> 5] >> (k & 31)) & 1u)) a = 0;
        else if (a < 126) a += 1;
        ages[k] = a;
      }
      cand = r || kn;
      bkt = (kn ? 127u : 0u) + a;
    }
    if (cand) atomicAdd(&hist[wid * 256 + rank_of[bkt]], 1u);
  }
  __syncthreads();
  // offsets: rank-major, then warp order
  if (tid == 0) {
    uint32_t nr = 0;
    for (int b = 0; b < SEL_BUCKETS; ++b) nr = max(nr, (uint32_t)rank_of[b] + 1u);
    s_nr = nr;
  }
  __syncthreads();
  {
    uint32_t tot = 0;
    if (tid < (int)s_nr)
      for (int w = 0; w < SEL_WARPS; ++w) {
        const uint32_t c = hist[w * 256 + tid];
        hist[w * 256 + tid] = tot;
        tot += c;
      }
    uint32_t n;
    const uint32_t base = block_scan_excl(tid < (int)s_nr ? tot : 0u, sw, &n);
    if (tid < (int)s_nr)
      for (int w = 0; w < SEL_WARPS; ++w) hist[w * 256 + tid] += base;
    if (tid == 0) s_ncand = n;
  }
  __syncthreads();
  // stable placement: within a warp's group of 32 ids, earlier lanes of equal
  // rank first (match_any), the warp's running offset per rank in hist
  for (uint32_t k0 = k_lo; k0 < k_hi; k0 += 32) {
    const uint32_t k = k0 + lane;
    bool cand = false;
    uint32_t rk = 0xFFFFu;
    if (k < k_hi) {
      const uint32_t a = ages[k];  // already updated by this lane
      const bool r = (r_cur[k >> 5] >> (k & 31)) & 1u, kn = (k_union[k >> 5] >> (k & 31)) & 1u;
      cand = r || kn;
      if (cand) rk = rank_of[(kn ? 127u : 0u) + a];
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, rk);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader && cand) {
      base = hist[wid * 256 + rk];
      hist[wid * 256 + rk] = base + __popc(peers);
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    if (cand) ids[base + __popc(peers & lt)] = (uint16_t)k;
    __syncwarp();
  }
  __syncthreads();
  const uint32_t nc = s_ncand;

  // camera-balanced quota: per camera, the first `quota` of its visible
  // candidates in sorted order
  for (int j = 0; j < J; ++j) {
    const uint32_t* kj = k_next + (uint64_t)j * words;
    uint32_t carry = 0;
    for (uint32_t s0 = 0; s0 < nc; s0 += SEL_THREADS) {
      const uint32_t s = s0 + tid;
      const uint32_t f = s < nc ? (kj[ids[s] >> 5] >> (ids[s] & 31)) & 1u : 0u;
      uint32_t tot;
      const uint32_t pre = block_scan_excl(f, sw, &tot) + carry;
      if (f && pre < quota) atomicOr(&selb[s >> 5], 1u << (s & 31));
      carry += tot;
    }
    __syncthreads();
  }
  // global fill in sorted order up to the capacity
  {
    uint32_t nsel = 0;
    for (uint32_t e = tid; e < (nc + 31) / 32; e += SEL_THREADS) nsel += __popc(selb[e]);
    uint32_t tot;
    block_scan_excl(nsel, sw, &tot);
    nsel = tot;
    uint32_t carry = 0;
    for (uint32_t s0 = 0; s0 < nc; s0 += SEL_THREADS) {
      const uint32_t s = s0 + tid;
      const bool sel = s < nc && ((selb[s >> 5] >> (s & 31)) & 1u);
      const uint32_t un = (s < nc && !sel) ? 1u : 0u;
      uint32_t t2;
      const uint32_t pre = block_scan_excl(un, sw, &t2) + carry;
      const bool take = sel || (un && nsel < capacity && pre < capacity - nsel);
      if (take) atomicOr(&rnb[ids[s] >> 5], 1u << (ids[s] & 31));
      carry += t2;
    }
    if (tid == 0) s_nsel = nsel;
  }
  __syncthreads();
  // S+ = r_next & ~r_cur, S- = r_cur & ~r_next, render = r_next & K_union, in
  // ascending block id
  uint32_t off[3] = {0, 0, 0};
  uint32_t* outs[3] = {s_plus, s_minus, render};
  for (uint32_t w0 = 0; w0 < words; w0 += SEL_THREADS) {
    const uint32_t w = w0 + tid;
    uint32_t m[3] = {0, 0, 0};
    if (w < words) {
      const uint32_t rn = rnb[w], rc = r_cur[w];
      m[0] = rn & ~rc;
      m[1] = rc & ~rn;
      m[2] = rn & k_union[w];
      r_next[w] = rn;
      acc_out[w] = m[2];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      uint32_t tot;
      uint32_t o = block_scan_excl(__popc(m[q]), sw, &tot) + off[q];
      uint32_t mm = m[q];
      while (mm) {
        const int b = __ffs(mm) - 1;
        outs[q][o++] = w * 32 + b;
        mm &= mm - 1;
      }
      off[q] += tot;
    }
  }
  if (tid == 0) {
    counters[0] = off[0];
    counters[1] = off[1];
    counters[2] = off[2];
    counters[3] = nc;
    counters[4] = s_nsel;
  }
}

size_t select_small_smem() { return 2 * SEL_MAX_K + (SEL_WARPS * 256 + SEL_MAX_K / 32 + SEL_MAX_K / 32) * 4; }

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
  if (K <= SEL_MAX_K && J <= 8) {
    TGS_CUDA(cudaFuncSetAttribute(k_select_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)select_small_smem()));
    k_select_small<<<1, SEL_THREADS, select_small_smem(), s>>>(
        k_acc, r_cur, k_next, k_next_union, J, (uint32_t)K, ages, lambda, age_update ? 1 : 0, (uint32_t)capacity,
        (uint32_t)quota, r_next, s_plus, s_minus, render, acc_out, rb.counters);
    TGS_LAUNCHED();
    return;
  }
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

namespace {

// The selection's results written into mapped host memory by device stores:
// the counts and the used prefixes of the three lists, the visibility rows and
// the resident bitmap.  A copy-engine read-back would queue behind the bulk
// block copies of the same direction (tens of MB of write-back) and keep the
// host waiting for them.
__global__ void k_publish_sets(const uint32_t* __restrict__ counters, const uint32_t* __restrict__ lists, uint64_t K,
                               const uint32_t* __restrict__ kvis, uint64_t kvis_words,
                               const uint32_t* __restrict__ rbits, uint64_t words, uint32_t* out_lists,
                               uint32_t* out_kvis, uint32_t* out_r) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n[3] = {counters[0], counters[1], counters[2]};
  if (tid < 4) out_lists[tid] = counters[tid];
  for (int q = 0; q < 3; ++q)
    for (uint64_t i = tid; i < n[q] && i < K; i += stride) out_lists[16 + q * K + i] = lists[q * K + i];
  for (uint64_t i = tid; i < kvis_words; i += stride) out_kvis[i] = kvis[i];
  for (uint64_t i = tid; i < words; i += stride) out_r[i] = rbits[i];
}

}  // namespace

void publish_sets(const uint32_t* counters, const uint32_t* lists, uint64_t K, const uint32_t* kvis,
                  uint64_t kvis_words, const uint32_t* rbits, uint64_t words, uint32_t* out_lists, uint32_t* out_kvis,
                  uint32_t* out_r, cudaStream_t s) {
  k_publish_sets<<<8, 256, 0, s>>>(counters, lists, K, kvis, kvis_words, rbits, words, out_lists, out_kvis, out_r);
  TGS_LAUNCHED();
}

}  // namespace tgs
