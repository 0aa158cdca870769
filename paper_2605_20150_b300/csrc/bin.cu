// Binning of the Level-2 render (Sec. 3.3 "Level 2"): visible compaction,
// stable depth sort of the visible Gaussians, pair emission in depth order
// and the stable regrouping of the (tile, Gaussian) pairs by tile -- the same
// order as one stable sort of (tile << 32 | depth bits) keys emitted in id
// order.
//
// Every step is a single pass that finds its output offsets with a decoupled
// look-back (Merrill & Garland 2016, "Single-pass parallel prefix scan with
// decoupled look-back"; for radix sorting, Adinets & Merrill 2022,
// "Onesweep"): a CTA takes the next partition of its input from an atomic
// ticket, publishes its partition's count (or, per radix digit, its 256
// counts) tagged with the launch's epoch, sums its predecessors' published
// counts until it meets an inclusive prefix, publishes its own inclusive
// prefix and writes its output.  A partition waits only on partitions whose
// tickets were drawn earlier, by CTAs that are running, so every wait ends;
// each wait is also bounded (LB_SPIN_MAX polls), after which the kernel sets
// an error word the host reads with the render's counts.
//
// Each radix pass also builds the histogram of the next pass's digit, and
// the compaction and pair emission build the first one, so a pass needs no
// histogram or offsets kernel of its own.  Forward chain per camera: one
// memset of the control words, compaction, four depth passes, pair offsets,
// pair emission (balanced over pairs, not over Gaussians: the nearest
// Gaussians of a street view cover thousands of tiles each), one or two tile
// passes, tile ranges.
#include "raster.cuh"

namespace tgs {

namespace {

constexpr int BT = 256;              // threads of every binning kernel
constexpr int BW = BT / 32;
constexpr int CP_ITEMS = 32;         // compaction: positions per thread
constexpr int CP_PART = BT * CP_ITEMS;
constexpr int EM_ITEMS = 4;          // emission: Gaussians per thread
constexpr int EM_PART = BT * EM_ITEMS;
constexpr uint32_t LB_AGG = 1u, LB_INC = 2u;
constexpr uint32_t LB_MAXV = 0x3FFFFFFFu;
constexpr uint32_t LB_SPIN_MAX = 1u << 20;

// status word: epoch (32 bits) | flag (2) | value (30)
__device__ __forceinline__ uint64_t lb_pack(uint32_t epoch, uint32_t flag, uint32_t v) {
  return ((uint64_t)epoch << 32) | ((uint64_t)flag << 30) | (uint64_t)(v & LB_MAXV);
}
__device__ __forceinline__ void lb_store(uint64_t* p, uint64_t w) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ uint64_t lb_load(const uint64_t* p) {
  uint64_t w;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
  return w;
}
__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) {
  const uint32_t s = a + b;
  return (s < a || s > LB_MAXV) ? LB_MAXV : s;
}

// Decoupled look-back with a window: all partitions of a launch start
// together (one wave), so a partition may find only aggregates behind it as
// far as partition 0; reading LB_WIN predecessors per round (independent
// loads) makes that walk LB_WIN times shorter.

constexpr int LB_WIN = 32;

// One thread, one value per partition at status[q * stride]: the exclusive
// prefix of partition p; then p's inclusive prefix is published.  Sums
// saturate at LB_MAXV (a count that large is an overflow anyway).
__device__ uint32_t lb_lookback(uint64_t* status, uint64_t stride, uint32_t p, uint32_t own, uint32_t epoch,
                                uint32_t* err) {
  uint32_t ex = 0;
  int64_t q = (int64_t)p - 1;  // the newest predecessor not yet summed
  uint32_t spins = 0;
  while (q >= 0) {
    uint64_t w[LB_WIN];
#pragma unroll
    for (int k = 0; k < LB_WIN; ++k)
      w[k] = q - k >= 0 ? lb_load(status + (uint64_t)(q - k) * stride) : lb_pack(epoch, LB_INC, 0);
    int took = 0;
    bool done = false, wait = false;
#pragma unroll
    for (int k = 0; k < LB_WIN; ++k) {
      if (!done && !wait) {
        const uint32_t f = (uint32_t)(w[k] >> 30) & 3u;
        if ((uint32_t)(w[k] >> 32) != epoch || f == 0u) {
          wait = true;
        } else {
          ex = sat_add(ex, (uint32_t)(w[k] & LB_MAXV));
          ++took;
          done = f == LB_INC;
        }
      }
    }
    if (done) break;
    q -= took;
    if (wait) {
      if (++spins > LB_SPIN_MAX) {
        atomicOr(err, 1u);
        break;
      }
      if (spins > 16) __nanosleep(64);
    }
  }
  lb_store(status + (uint64_t)p * stride, lb_pack(epoch, LB_INC, sat_add(ex, own)));
  return ex;
}

// The same for one value per partition at status[q], by the 32 lanes of a
// warp (lane l reads predecessor q - l); every lane returns the prefix.
__device__ uint32_t lb_lookback_warp(uint64_t* status, uint32_t p, uint32_t own, uint32_t epoch, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  uint32_t ex = 0;
  int64_t q = (int64_t)p - 1;
  uint32_t spins = 0;
  while (q >= 0) {
    const int64_t qi = q - lane;
    const uint64_t w = qi >= 0 ? lb_load(status + qi) : lb_pack(epoch, LB_INC, 0);
    const uint32_t f = (uint32_t)(w >> 30) & 3u;
    const bool valid = (uint32_t)(w >> 32) == epoch && f != 0u;
    const uint32_t incm = __ballot_sync(0xffffffffu, valid && f == LB_INC);
    const uint32_t bad = __ballot_sync(0xffffffffu, !valid);
    const int li = incm ? __ffs(incm) - 1 : 31;          // nearest inclusive prefix, else the whole window
    const uint32_t need = li == 31 ? 0xffffffffu : ((2u << li) - 1u);
    if (bad & need) {
      // a predecessor within reach has not published yet: sum the valid
      // ones before it and wait on it
      const int lb = __ffs(bad & need) - 1;
      uint64_t v = lane < lb ? (w & LB_MAXV) : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      ex = sat_add(ex, v > LB_MAXV ? LB_MAXV : (uint32_t)v);
      q -= lb;
      if (++spins > LB_SPIN_MAX) {
        if (lane == 0) atomicOr(err, 1u);
        break;
      }
      if (spins > 16) __nanosleep(64);
      continue;
    }
    uint64_t v = lane <= li ? (w & LB_MAXV) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    ex = sat_add(ex, v > LB_MAXV ? LB_MAXV : (uint32_t)v);
    if (incm) break;
    q -= 32;
  }
  if (lane == 0) lb_store(status + p, lb_pack(epoch, LB_INC, sat_add(ex, own)));
  return ex;
}

__device__ __forceinline__ uint32_t warp_incl(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Exclusive scan of one value per thread over the BT threads; *total gets
// the sum.  Ends with a barrier (sw is reused).
__device__ __forceinline__ uint32_t cta_excl(uint32_t x, uint32_t* sw, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl(x);
  if (lane == 31) sw[w] = inc;
  __syncthreads();
  if (w == 0) {
    const uint32_t v = lane < BW ? sw[lane] : 0u;
    const uint32_t vi = warp_incl(v);
    if (lane < BW) sw[lane] = vi - v;
    if (lane == BW - 1) sw[BW] = vi;
  }
  __syncthreads();
  const uint32_t r = sw[w] + inc - x;
  if (total) *total = sw[BW];
  __syncthreads();
  return r;
}

// ---- visible compaction: positions with a non-empty tile rect, ascending,
// as (depth bits, position) pairs; their count; the histogram of the depth
// keys' lowest byte.  One partition of CP_PART positions per CTA, read as
// CP_ITEMS coalesced runs of BT positions; a position's rank is its warp's
// ballot prefix plus the scanned (run, warp) counts.
__global__ void __launch_bounds__(BT) k_compact_lb(uint64_t V, const uint32_t* __restrict__ ntiles,
                                                  const float* __restrict__ depth, uint32_t* __restrict__ dkeys,
                                                  uint32_t* __restrict__ dvals, uint32_t* __restrict__ nv_dev,
                                                  uint32_t* __restrict__ hist0, uint64_t* status, uint32_t epoch,
                                                  uint32_t* ticket, uint32_t* err) {
  __shared__ uint32_t s_t, s_ex;
  __shared__ uint32_t sw[BW + 1];
  __shared__ uint32_t h[256];
  __shared__ uint32_t cnt[CP_ITEMS * BW];  // (run, warp), in position order
  static_assert(CP_ITEMS * BW == BT, "one (run, warp) count per thread");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1u);
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t p = s_t;
  const uint64_t nparts = (V + CP_PART - 1) / CP_PART;
  if (p >= nparts) return;  // uniform per CTA
  const uint64_t base = (uint64_t)p * CP_PART;
  uint32_t bal[CP_ITEMS];
#pragma unroll
  for (int k = 0; k < CP_ITEMS; ++k) {
    const uint64_t i = base + (uint64_t)k * BT + threadIdx.x;
    const bool v = i < V && ntiles[i] != 0u;
    bal[k] = __ballot_sync(0xffffffffu, v);
    if (lane == 0) cnt[k * BW + w] = __popc(bal[k]);
  }
  __syncthreads();
  uint32_t tot;
  const uint32_t my = cnt[threadIdx.x];
  const uint32_t off = cta_excl(my, sw, &tot);
  cnt[threadIdx.x] = off;
  if (threadIdx.x < 32) {
    if (p > 0 && threadIdx.x == 0) lb_store(status + p, lb_pack(epoch, LB_AGG, tot));
    const uint32_t ex = lb_lookback_warp(status, p, tot, epoch, err);
    if (threadIdx.x == 0) {
      s_ex = ex;
      if (p + 1 == nparts) *nv_dev = ex + tot;
    }
  }
  __syncthreads();
  const uint32_t ex = s_ex;
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < CP_ITEMS; ++k) {
    if (bal[k] >> lane & 1u) {
      const uint64_t i = base + (uint64_t)k * BT + threadIdx.x;
      const uint32_t q = ex + cnt[k * BW + w] + __popc(bal[k] & lt);
      const uint32_t key = __float_as_uint(depth[i]);  // depth > 0: the bits order like the values
      dkeys[q] = key;
      dvals[q] = (uint32_t)i;
      atomicAdd(&h[key & 0xFFu], 1u);
    }
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist0[threadIdx.x], h[threadIdx.x]);
}

// ---- one stable LSD radix pass with decoupled look-back over per-digit
// counts.  hist: global counts of this pass's digit (complete before the
// launch); hist_next (may be null): counts of the next pass's digit,
// accumulated here.  Persistent CTAs draw partitions of 256 x ITEMS keys in
// order; each ranks its keys stably with warp multi-split (match_any),
// stages them in shared memory in digit order and writes each digit run
// contiguously.
template <int ITEMS>
__global__ void __launch_bounds__(BT) k_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                const uint32_t* __restrict__ n_dev, uint64_t cap, int shift,
                                                uint32_t mask, const uint32_t* __restrict__ hist,
                                                uint32_t* __restrict__ hist_next, int nshift, uint32_t nmask,
                                                uint64_t* status, uint32_t epoch, uint32_t* ticket, uint32_t* err) {
  constexpr int PART = BT * ITEMS;
  __shared__ uint32_t cnt[BW][256];
  __shared__ uint32_t gbase[256], dstart[256], excl[256], hn[256];
  __shared__ uint32_t sw[BW + 1];
  __shared__ uint32_t s_t;
  __shared__ uint32_t sk[PART], sv[PART];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t n = *n_dev;
  if (n > cap) n = cap;
  const uint32_t nparts = (uint32_t)((n + PART - 1) / PART);
  gbase[tid] = cta_excl(tid <= (int)mask ? hist[tid] : 0u, sw, nullptr);
  for (;;) {
    if (tid == 0) s_t = atomicAdd(ticket, 1u);
    for (int i = tid; i < BW * 256; i += BT) (&cnt[0][0])[i] = 0;
    hn[tid] = 0;
    __syncthreads();
    const uint32_t p = s_t;
    if (p >= nparts) break;  // uniform per CTA
    const uint64_t p0 = (uint64_t)p * PART;
    const uint64_t p1 = p0 + PART < n ? p0 + PART : n;
    // warp w ranks the run [w * 32 ITEMS, (w + 1) * 32 ITEMS) of the partition in input order
    const uint64_t wb = p0 + (uint64_t)w * (32 * ITEMS);
    uint32_t key[ITEMS], val[ITEMS], rk[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint64_t i = wb + (uint64_t)j * 32 + lane;
      const bool valid = i < p1;
      key[j] = valid ? kin[i] : 0u;
      val[j] = valid ? vin[i] : 0u;
      const uint32_t d = valid ? ((key[j] >> shift) & mask) : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (lane == leader && valid) {
        old = cnt[w][d];
        cnt[w][d] = old + __popc(peers);
      }
      old = __shfl_sync(0xffffffffu, old, leader);
      rk[j] = old + __popc(peers & lt);
      if (hist_next && valid) atomicAdd(&hn[(key[j] >> nshift) & nmask], 1u);
      __syncwarp();
    }
    __syncthreads();
    // per digit (thread tid = digit): warp offsets and the partition's count
    uint32_t tot = 0;
#pragma unroll
    for (int k = 0; k < BW; ++k) {
      const uint32_t c = cnt[k][tid];
      cnt[k][tid] = tot;
      tot += c;
    }
    if (p > 0) lb_store(status + (uint64_t)p * 256 + tid, lb_pack(epoch, LB_AGG, tot));
    dstart[tid] = cta_excl(tot, sw, nullptr);
    __syncthreads();  // every digit's start is read below
    // stage the partition in digit order (local offsets only) before the
    // look-back: the registers are free for its window, and predecessors
    // get the staging time to publish
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint64_t i = wb + (uint64_t)j * 32 + lane;
      if (i < p1) {
        const uint32_t d = (key[j] >> shift) & mask;
        const uint32_t pos = dstart[d] + cnt[w][d] + rk[j];  // < PART: a permutation of the partition
        sk[pos] = key[j];
        sv[pos] = val[j];
      }
    }
    excl[tid] = lb_lookback(status + tid, 256, p, tot, epoch, err);
    __syncthreads();
    const uint32_t pn = (uint32_t)(p1 - p0);
#pragma unroll 4
    for (int e = tid; e < PART; e += BT) {
      if ((uint32_t)e < pn) {
        const uint32_t k = sk[e];
        const uint32_t d = (k >> shift) & mask;
        const uint64_t g = (uint64_t)gbase[d] + excl[d] + (uint32_t)(e - dstart[d]);
        if (g < cap) {  // always true unless a look-back wait ran out (err is then set)
          kout[g] = k;
          vout[g] = sv[e];
        }
      }
    }
    if (hist_next && hn[tid]) atomicAdd(&hist_next[tid], hn[tid]);
    __syncthreads();  // shared buffers are reused by the next partition
  }
}

// largest i < n with a[i] <= x (a non-decreasing, a[0] <= x)
__device__ __forceinline__ uint32_t last_le_s(const uint32_t* a, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// ---- pair offsets in depth order: the tile counts of a partition of
// EM_PART depth-sorted Gaussians, scanned, the partition's start found by
// look-back; off[i] = first pair of sorted Gaussian i, *np_dev = all pairs
// (before the capacity clamp; an overflow raises flag[0], the count needed in
// flag[1], and step_flag).
__global__ void __launch_bounds__(BT) k_pair_offsets_lb(const uint32_t* __restrict__ nv_dev,
                                                       const uint32_t* __restrict__ dvals,
                                                       const uint32_t* __restrict__ ntiles,
                                                       uint32_t* __restrict__ off, uint64_t cap,
                                                       uint32_t* __restrict__ np_dev, uint32_t* flag,
                                                       uint32_t* step_flag, uint64_t* status, uint32_t epoch,
                                                       uint32_t* ticket, uint32_t* err) {
  __shared__ uint32_t sw[BW + 1];
  __shared__ uint32_t s_t, s_ex;
  const uint32_t nv = *nv_dev;
  const uint32_t nparts = (nv + EM_PART - 1) / EM_PART;
  if (threadIdx.x == 0) s_t = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t p = s_t;
  if (p >= nparts) return;  // uniform per CTA
  const uint32_t g0 = p * EM_PART + threadIdx.x * EM_ITEMS;
  uint32_t c[EM_ITEMS], sum = 0;
#pragma unroll
  for (int k = 0; k < EM_ITEMS; ++k) {
    c[k] = g0 + k < nv ? ntiles[dvals[g0 + k]] : 0u;
    sum += c[k];
  }
  uint32_t tot;
  uint32_t o = cta_excl(sum, sw, &tot);
  if (threadIdx.x < 32) {
    if (p > 0 && threadIdx.x == 0) lb_store(status + p, lb_pack(epoch, LB_AGG, tot));
    const uint32_t ex = lb_lookback_warp(status, p, tot, epoch, err);
    if (threadIdx.x == 0) {
      s_ex = ex;
      if (p + 1 == nparts) {
        const uint32_t all = sat_add(ex, tot);
        *np_dev = all;
        if ((uint64_t)all > cap) {
          atomicOr(flag, 1u);
          atomicMax(flag + 1, all);
          if (step_flag) atomicOr(step_flag, 1u);
        }
      }
    }
  }
  __syncthreads();
  o = sat_add(o, s_ex);
#pragma unroll
  for (int k = 0; k < EM_ITEMS; ++k) {
    if (g0 + k < nv) off[g0 + k] = o;
    o = sat_add(o, c[k]);
  }
}

// ---- pair emission balanced over pairs: CTA chunks of EM_CHUNK pairs in
// order (grid-stride).  Every visible Gaussian has at least one pair, so the
// Gaussians covering a chunk are at most EM_CHUNK consecutive entries of off;
// a warp-cooperative search finds the first, they are staged in shared
// memory, and each pair finds its Gaussian there by binary search and its
// tile from its index inside the Gaussian's rect (row-major).  Pairs at or
// beyond cap are not written.  Also the histogram of the lowest tile digit.
constexpr uint32_t EM_CHUNK = 1024;

// largest i < n with a[i] <= x (a non-decreasing, a[0] <= x), 32 lanes
// probing 32 evenly spaced entries per round
__device__ __forceinline__ uint32_t warp_last_le_g(const uint32_t* __restrict__ a, uint32_t n, uint32_t x) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = n;
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t pv = lo + lane * step;
    const uint32_t b = __ballot_sync(0xffffffffu, pv < hi && a[pv] <= x);
    lo += (31 - __clz(b)) * step;  // lane 0 always qualifies (a[lo] <= x)
    hi = min(hi, lo + step);
  }
  const uint32_t b = __ballot_sync(0xffffffffu, lo + lane < hi && a[lo + lane] <= x);
  return lo + (31 - __clz(b));
}

__global__ void __launch_bounds__(BT) k_emit_bal(const uint32_t* __restrict__ nv_dev,
                                                const uint32_t* __restrict__ np_dev,
                                                const uint32_t* __restrict__ dvals,
                                                const uint32_t* __restrict__ off, const ushort4* __restrict__ rect,
                                                int TX, uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals,
                                                uint64_t cap, uint32_t* __restrict__ hist0, uint32_t mask0) {
  __shared__ uint32_t s_off[EM_CHUNK];
  __shared__ uint32_t s_id[EM_CHUNK];
  __shared__ ushort4 s_rect[EM_CHUNK];
  __shared__ uint32_t h[256];
  __shared__ uint32_t s_lo, s_cnt;
  const uint32_t nv = *nv_dev;
  const uint64_t np_all = *np_dev;
  const uint32_t np = (uint32_t)(np_all < cap ? np_all : cap);
  h[threadIdx.x] = 0;
  for (uint32_t p0 = blockIdx.x * EM_CHUNK; p0 < np; p0 += gridDim.x * EM_CHUNK) {
    const uint32_t p1 = min(p0 + EM_CHUNK, np) - 1;
    // warp 0 finds the chunk's first Gaussian, warp 1 its last
    if (threadIdx.x < 64) {
      const uint32_t k = warp_last_le_g(off, nv, threadIdx.x < 32 ? p0 : p1);
      if (threadIdx.x == 0) s_lo = k;
      if (threadIdx.x == 32) s_cnt = k;
    }
    __syncthreads();
    const uint32_t lo = s_lo, cnt = s_cnt - s_lo + 1;
    for (uint32_t e = threadIdx.x; e < cnt; e += BT) {
      const uint32_t id = dvals[lo + e];
      s_off[e] = off[lo + e];
      s_id[e] = id;
      s_rect[e] = rect[id];
    }
    __syncthreads();
    for (uint32_t q = p0 + threadIdx.x; q <= p1; q += BT) {
      const uint32_t k = last_le_s(s_off, cnt, q);
      const ushort4 r = s_rect[k];
      const uint32_t wdt = (uint32_t)(r.z - r.x);
      const uint32_t loc = q - s_off[k];
      const uint32_t dy = loc / wdt;
      const uint32_t tile = (uint32_t)((r.y + dy) * TX + r.x + (loc - dy * wdt));
      pkeys[q] = tile;
      pvals[q] = s_id[k];
      atomicAdd(&h[tile & mask0], 1u);
    }
    __syncthreads();  // the staged chunk is rewritten next
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist0[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_ranges_lb(const uint32_t* __restrict__ np_dev, uint64_t cap, const uint32_t* __restrict__ pkeys,
                            uint2* __restrict__ ranges) {
  uint64_t np = *np_dev;
  if (np > cap) np = cap;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t t = pkeys[p];
    if (p == 0 || pkeys[p - 1] != t) ranges[t].x = (uint32_t)p;
    if (p == np - 1 || pkeys[p + 1] != t) ranges[t].y = (uint32_t)(p + 1);
  }
}

int bits_needed(uint64_t n) {
  int b = 1;
  while ((1ull << b) < n) ++b;
  return b;
}

}  // namespace

uint64_t bin_status_words(uint64_t cap_v, uint64_t cap_pairs) {
  const uint64_t d = (cap_v + BT * 8 - 1) / (BT * 8);
  const uint64_t q = (cap_pairs + BT * 16 - 1) / (BT * 16);
  return 256 * (d > q ? d : q) + 256;
}

uint64_t bin_status1_words(uint64_t cap_v) { return (cap_v + EM_PART - 1) / EM_PART + (cap_v + CP_PART - 1) / CP_PART + 2; }

void bin_and_sort(uint64_t V, int TX, uint64_t tiles, CamState& cs, cudaStream_t s) {
  TGS_CHECK(cs.cap_pairs < LB_MAXV && cs.cap_v < LB_MAXV, TGS_ERR_CAPACITY, "pair or render-list capacity above 2^30");
  uint32_t* ctl = cs.bin_ctl;  // [8][256] digit counts, [16] tickets
  uint32_t* hist = ctl;
  uint32_t* tick = ctl + 8 * 256;
  uint32_t* err = cs.counters + 6;
  uint32_t* nv_dev = cs.counters;
  uint32_t* np_dev = cs.counters + 1;
  TGS_CUDA(cudaMemsetAsync(ctl, 0, BIN_CTL_WORDS * sizeof(uint32_t), s));
  const unsigned g_cp = div_up(V, CP_PART);
  k_compact_lb<<<g_cp, BT, 0, s>>>(V, cs.ntiles, cs.depth, cs.dkeys, cs.dvals, nv_dev, hist, cs.status1, ++cs.epoch,
                                   tick + 0, err);
  TGS_LAUNCHED();
  // depth sort: four 8-bit passes (positive float bits), ping-pong ending in dkeys
  const unsigned g_d = std::min<unsigned>(div_up(V, BT * 8), 2 * NSM);
  uint32_t *ki = cs.dkeys, *vi = cs.dvals, *ko = cs.dkeys + cs.cap_v, *vo = cs.dvals + cs.cap_v;
  for (int pass = 0; pass < 4; ++pass) {
    uint32_t* hn = pass < 3 ? hist + (pass + 1) * 256 : nullptr;
    k_onesweep<8><<<g_d, BT, 0, s>>>(ki, vi, ko, vo, nv_dev, V, 8 * pass, 0xFFu, hist + pass * 256, hn,
                                     hn ? 8 * (pass + 1) : 0, 0xFFu, cs.status, ++cs.epoch, tick + 1 + pass, err);
    TGS_LAUNCHED();
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  // tile sort digits: as even as possible, one pass up to 8 bits
  const int bits = bits_needed(tiles);
  const int passes = (bits + 7) / 8;
  const int w0 = (bits + passes - 1) / passes;
  uint32_t *pk = cs.pkeys, *pv = cs.pvals, *pk2 = cs.pkeys + cs.cap_pairs, *pv2 = cs.pvals + cs.cap_pairs;
  // emission writes the buffer that makes the last pass end in pkeys / pvals
  uint32_t *ek = passes & 1 ? pk2 : pk, *ev = passes & 1 ? pv2 : pv;
  // pair offsets of the depth-sorted Gaussians (into cs.scan), then the
  // emission balanced over pairs
  k_pair_offsets_lb<<<div_up(V, EM_PART), BT, 0, s>>>(nv_dev, vi, cs.ntiles, cs.scan, cs.cap_pairs, np_dev,
                                                      cs.counters + 2, cs.step_flag, cs.status1, ++cs.epoch,
                                                      tick + 5, err);
  TGS_LAUNCHED();
  const unsigned g_e = std::min<unsigned>(div_up(cs.cap_pairs, EM_CHUNK), 4 * NSM);
  k_emit_bal<<<g_e, BT, 0, s>>>(nv_dev, np_dev, vi, cs.scan, cs.rect, TX, ek, ev, cs.cap_pairs, hist + 4 * 256,
                                (1u << w0) - 1u);
  TGS_LAUNCHED();
  const unsigned g_p = std::min<unsigned>(div_up(cs.cap_pairs, BT * 16), 2 * NSM);
  uint32_t *ki2 = ek, *vi2 = ev, *ko2 = passes & 1 ? pk : pk2, *vo2 = passes & 1 ? pv : pv2;
  int shift = 0;
  for (int pass = 0; pass < passes; ++pass) {
    const int wb = std::min(w0, bits - shift);
    const int wn = pass + 1 < passes ? std::min(w0, bits - shift - wb) : 0;
    uint32_t* hn = pass + 1 < passes ? hist + (5 + pass) * 256 : nullptr;
    k_onesweep<16><<<g_p, BT, 0, s>>>(ki2, vi2, ko2, vo2, np_dev, cs.cap_pairs, shift, (1u << wb) - 1u,
                                      hist + (4 + pass) * 256, hn, hn ? shift + wb : 0, wn ? (1u << wn) - 1u : 0u, cs.status,
                                      ++cs.epoch, tick + 6 + pass, err);
    TGS_LAUNCHED();
    std::swap(ki2, ko2);
    std::swap(vi2, vo2);
    shift += wb;
  }
  k_ranges_lb<<<2 * NSM, 256, 0, s>>>(np_dev, cs.cap_pairs, cs.pkeys, cs.ranges);
  TGS_LAUNCHED();
}

}  // namespace tgs
