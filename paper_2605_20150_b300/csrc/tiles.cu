// Tile binning of the Level-2 render (Sec. 3.3 "Level 2"): the (tile,
// Gaussian) pairs of every visible Gaussian, grouped by tile and ordered
// inside each tile front to back.  The order is that of one stable sort of
// (tile << 32 | depth bits) keys emitted in render-list order: inside a tile,
// ascending depth bits, ties by ascending render-list position.
//
// Instead of radix-sorting the pairs, the binning counts, places and sorts
// per tile:
//  - the preprocess adds each visible Gaussian's tile rect to a 2D difference
//    array (+1 / -1 at its four corners, one atomic per distinct corner and
//    warp);
//  - k_tile_scan (one CTA) integrates the difference array into per-tile
//    counts, scans them into the tile ranges, detects a pair overflow,
//    lists the tiles too long for a small sort, and orders the tiles for the
//    raster launches (longest list first, with the backward split units);
//  - k_emit_tiles writes every pair into its tile's range at a slot claimed
//    with an atomic on the tile's fill counter (warps cover 32 render-list
//    positions; Gaussians with more than EM_WARP tiles are listed for
//    k_emit_big, where a warp emits each up to EM_CTA tiles and a whole CTA
//    each above);
//  - k_tile_sort sorts each tile's pairs on (depth bits, position) in shared
//    memory: warps sort runs of 32 with shuffles, then runs are merged
//    pairwise along the merge path; k_tile_sort_big takes the tiles above
//    SORT_SMALL pairs (runs of SORT_BIG, merged in global memory beyond).
// The claim order of the atomics does not matter: the per-tile sort keys are
// unique, so the result is the same for every interleaving.
#include "raster.cuh"

namespace tgs {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TS_THREADS = 1024;
constexpr int EM_THREADS = 256;
constexpr uint32_t EM_WARP = 32;    // tiles above which a Gaussian leaves the 32-position warps
constexpr uint32_t EM_CTA = 1024;   // tiles above which a whole CTA (not one warp) emits a Gaussian
constexpr int EM_UNROLL = 8;        // pairs per lane per round (their slot claims in flight together)
constexpr int SORT_THREADS = 256;
constexpr uint32_t SORT_SMALL = 8 * SORT_THREADS;  // 2048 keys: a small CTA (two 16 KB buffers)
constexpr int SORT_BIG_THREADS = 1024;
constexpr uint32_t SORT_BIG = 8 * SORT_BIG_THREADS;  // 8192 keys in shared memory (two 64 KB buffers)

// CamState counter words of the binning (the others: [0] visible, [1] pairs,
// [2] sticky overflow flag, [3] pairs needed, [5] backward units, [6] binning
// consistency error).
constexpr int C_OVER = 8;    // this render overflowed its pair capacity
constexpr int C_NBIG_G = 9;  // Gaussians emitted by a CTA in k_emit_big
constexpr int C_NBIG_T = 10; // tiles sorted by k_tile_sort_big
constexpr int C_NMID_G = 11; // Gaussians emitted by a warp in k_emit_big

__device__ __forceinline__ uint32_t bucket_of(uint32_t len) {
  const int b = 255 - (int)(16.f * log2f(1.f + (float)len));
  return (uint32_t)(b < 0 ? 0 : b);
}

// Exclusive scan of one 64-bit value per thread over the CTA; the total in
// `total`.  sw: 33 words of shared scratch.
__device__ __forceinline__ unsigned long long cta_excl64(unsigned long long x, unsigned long long* sw,
                                                         unsigned long long& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sw[w] = inc;
  __syncthreads();
  if (w == 0) {
    const unsigned long long v = lane < nw ? sw[lane] : 0ull;
    unsigned long long vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(FULL, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nw) sw[lane] = vi - v;
    if (lane == 31) sw[32] = vi;
  }
  __syncthreads();
  const unsigned long long r = sw[w] + inc - x;
  total = sw[32];
  __syncthreads();
  return r;
}

// One CTA: per-tile counts from the difference array (which it leaves zero
// for the next render), tile ranges, the overflow check and the list of long
// tiles.
__global__ void __launch_bounds__(TS_THREADS) k_tile_scan(int32_t* __restrict__ tdiff, int TX, int TY, uint64_t cap,
                                                         uint32_t* __restrict__ counters, uint32_t* step_flag,
                                                         uint2* __restrict__ ranges, uint32_t* __restrict__ tfill,
                                                         uint32_t* __restrict__ tbig) {
  extern __shared__ int32_t Dm[];  // (TY + 1) x (TX + 1): difference array, then counts
  __shared__ unsigned long long sw[33];
  __shared__ uint32_t s_nbig;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int S = TX + 1;
  const int cells = S * (TY + 1);
  const uint32_t tiles = (uint32_t)TX * (uint32_t)TY;
  for (int e = tid; e < cells; e += TS_THREADS) {
    Dm[e] = tdiff[e];
    tdiff[e] = 0;
  }
  if (tid == 0) s_nbig = 0;
  __syncthreads();
  // integrate along rows (warp per row), then along columns (thread per column)
  for (int y = w; y < TY; y += 32) {
    int carry = 0;
    for (int x0 = 0; x0 < TX; x0 += 32) {
      const int x = x0 + lane;
      int v = x < TX ? Dm[y * S + x] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += u;
      }
      v += carry;
      if (x < TX) Dm[y * S + x] = v;
      carry = __shfl_sync(FULL, v, 31);
    }
  }
  __syncthreads();
  for (int x = tid; x < TX; x += TS_THREADS) {
    int run = 0;
    for (int y = 0; y < TY; ++y) {
      run += Dm[y * S + x];
      Dm[y * S + x] = run;
    }
  }
  __syncthreads();
  // ranges: thread tid scans the tiles [t0, t1) in row-major order
  const uint32_t per = (tiles + TS_THREADS - 1) / TS_THREADS;
  const uint32_t t0 = min(tiles, (uint32_t)tid * per), t1 = min(tiles, t0 + per);
  auto count = [&](uint32_t t) { return (uint32_t)Dm[(t / TX) * S + t % TX]; };
  unsigned long long loc = 0, total = 0;
  for (uint32_t t = t0; t < t1; ++t) loc += count(t);
  const unsigned long long ex = cta_excl64(loc, sw, total);
  const bool over = total > cap;
  if (tid == 0) {
    const uint32_t all = total > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)total;
    counters[1] = all;
    counters[C_OVER] = over ? 1u : 0u;
    counters[C_NBIG_G] = 0;
    counters[C_NMID_G] = 0;
    if (over) {
      atomicOr(&counters[2], 1u);
      atomicMax(&counters[3], all);
      if (step_flag) atomicOr(step_flag, 1u);
    }
  }
  {
    unsigned long long o = ex;
    for (uint32_t t = t0; t < t1; ++t) {
      const uint32_t c = count(t);
      // an overflowing render has no pairs (it is rendered again once the
      // buffers have grown)
      ranges[t] = over ? make_uint2(0u, 0u) : make_uint2((uint32_t)o, (uint32_t)(o + c));
      tfill[t] = 0;
      if (!over && c > SORT_SMALL) tbig[atomicAdd(&s_nbig, 1u)] = t;
      o += c;
    }
  }
  __syncthreads();
  if (tid == 0) counters[C_NBIG_T] = s_nbig;
}

// One CTA, on a stream of its own beside the emission and the sorts: the
// raster tile order from the tile ranges (empty after an overflow).
//
// Tile order: a stable counting sort of the tiles on a logarithmic length
// bucket (255 - 16 log2(1 + length), clamped at 0), so the longest lists
// start first; it is a scheduling heuristic, so ties keep tile order.  Then,
// in that order, split tiles take checkpoint slots (while they fit in ck_cap)
// and the backward units (tile | segment << 24) are listed, their count in
// counters[5].
__global__ void __launch_bounds__(TS_THREADS) k_tile_order(const uint2* __restrict__ ranges, uint32_t tiles,
                                                          uint32_t* __restrict__ counters,
                                                          uint32_t* __restrict__ order, uint32_t* __restrict__ tck,
                                                          uint32_t* __restrict__ units, uint32_t ck_cap) {
  __shared__ uint32_t cnt[32][256];
  __shared__ uint32_t base[256];
  __shared__ unsigned long long sw[33];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int e = tid; e < 32 * 256; e += TS_THREADS) (&cnt[0][0])[e] = 0;
  __syncthreads();
  // warp w owns the tiles [w * tw, (w + 1) * tw)
  const uint32_t tw = ((tiles + 31) / 32 + 31) / 32 * 32;
  const uint32_t w_lo = min(tiles, (uint32_t)w * tw), w_hi = min(tiles, w_lo + tw);
  auto len = [&](uint32_t t) {
    const uint2 r = ranges[t];
    return r.y - r.x;
  };
  for (uint32_t a = w_lo; a < w_hi; a += 32)
    if (a + lane < w_hi) atomicAdd(&cnt[w][bucket_of(len(a + lane))], 1u);
  __syncthreads();
  if (tid < 256) {
    uint32_t run = 0;
    for (int k = 0; k < 32; ++k) {
      const uint32_t c = cnt[k][tid];
      cnt[k][tid] = run;
      run += c;
    }
    base[tid] = run;
  }
  __syncthreads();
  if (w == 0) {
    // exclusive scan of the 256 bucket totals: 8 per lane
    uint32_t v[8], s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[k] = base[8 * lane + k];
      s += v[k];
    }
    uint32_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    uint32_t run = inc - s;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      base[8 * lane + k] = run;
      run += v[k];
    }
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
  for (uint32_t a = w_lo; a < w_hi; a += 32) {
    const uint32_t t = a + lane;
    const bool ok = t < w_hi;
    const uint32_t b = ok ? bucket_of(len(t)) : 256u;
    const uint32_t peers = __match_any_sync(FULL, b);
    const int leader = __ffs(peers) - 1;
    uint32_t o = 0;
    if (lane == leader && ok) {
      o = cnt[w][b];
      cnt[w][b] = o + __popc(peers);
    }
    o = __shfl_sync(FULL, o, leader);
    if (ok) order[base[b] + o + __popc(peers & lt)] = t;
    __syncwarp();
  }
  __syncthreads();  // order[] is read back below by other threads
  unsigned long long ccarry = 0, ucarry = 0;
  for (uint32_t i0 = 0; i0 < tiles; i0 += TS_THREADS) {
    const uint32_t i = i0 + tid;
    uint32_t t = 0, ns = 1;
    if (i < tiles) {
      t = order[i];
      ns = seg_count(len(t));
    }
    // a split tile takes ns slots: ns - 1 boundaries and its final state
    const uint32_t want = ns > 1 ? ns : 0u;
    unsigned long long ctot, utot;
    const unsigned long long cb = ccarry + cta_excl64(want, sw, ctot);
    const bool split = want > 0 && cb + want <= ck_cap;
    const uint32_t nu = i < tiles ? (split ? ns : 1u) : 0u;
    const unsigned long long ub = ucarry + cta_excl64(nu, sw, utot);
    if (i < tiles) {
      tck[t] = split ? (uint32_t)cb : ~0u;
      for (uint32_t g = 0; g < nu; ++g) units[ub + g] = t | (g << 24);
    }
    ccarry += ctot;
    ucarry += utot;
  }
  if (tid == 0) counters[5] = (uint32_t)ucarry;
}

// Claims slots for up to 32 EM_UNROLL pairs of a warp (tile FULL: no pair)
// and writes them: lanes placing a pair in the same tile claim with one
// atomic.  The tile ranges are read and every atomic of the round is issued
// before the first result is used, so their latencies overlap.
// nsub (uniform over the warp): the sub-rounds u < nsub that hold a pair; the
// others are skipped whole.
__device__ __forceinline__ void place_pairs(const uint32_t (&tile)[EM_UNROLL], const uint32_t (&dk)[EM_UNROLL],
                                            const uint32_t (&id)[EM_UNROLL], int nsub,
                                            const uint2* __restrict__ ranges, uint32_t* __restrict__ tfill,
                                            uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals,
                                            uint32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint2 rg[EM_UNROLL];
  uint32_t peers[EM_UNROLL], o[EM_UNROLL];
  int leader[EM_UNROLL];
#pragma unroll
  for (int u = 0; u < EM_UNROLL; ++u) rg[u] = tile[u] != FULL ? ranges[tile[u]] : make_uint2(0u, 0u);
#pragma unroll
  for (int u = 0; u < EM_UNROLL; ++u) {
    peers[u] = 0u;
    leader[u] = 0;
    if (u < nsub) {  // uniform
      peers[u] = __match_any_sync(FULL, tile[u]);
      leader[u] = __ffs(peers[u]) - 1;
    }
  }
#pragma unroll
  for (int u = 0; u < EM_UNROLL; ++u)
    o[u] = tile[u] != FULL && lane == leader[u] ? atomicAdd(&tfill[tile[u]], (uint32_t)__popc(peers[u])) : 0u;
#pragma unroll
  for (int u = 0; u < EM_UNROLL; ++u) o[u] = __shfl_sync(FULL, o[u], leader[u]);
#pragma unroll
  for (int u = 0; u < EM_UNROLL; ++u) {
    if (tile[u] == FULL) continue;
    const uint32_t pos = rg[u].x + o[u] + __popc(peers[u] & lt);
    if (pos < rg[u].y) {
      pkeys[pos] = dk[u];
      pvals[pos] = id[u];
    } else {
      atomicOr(err, 1u);  // a tile received more pairs than it counted
    }
  }
}

// Pair emission: warps cover 32 consecutive render-list positions; the
// warp's pairs are dealt 32 EM_UNROLL at a time, each lane finding its
// Gaussian (the owner lane) by a binary search over the warp's inclusive scan
// of tile counts, and its tile from its index inside the owner's rect
// (row-major).  Gaussians with more than EM_WARP tiles are listed for
// k_emit_big (a warp each up to EM_CTA tiles, a CTA each above), so no warp
// here deals more than 32 EM_WARP pairs.
__global__ void __launch_bounds__(EM_THREADS) k_emit_tiles(uint64_t V, const uint32_t* __restrict__ ntiles,
                                                          const ushort4* __restrict__ rect,
                                                          const float* __restrict__ depth, int TX,
                                                          const uint2* __restrict__ ranges,
                                                          uint32_t* __restrict__ tfill, uint32_t* __restrict__ pkeys,
                                                          uint32_t* __restrict__ pvals, uint32_t* __restrict__ big,
                                                          uint32_t* __restrict__ mid, uint32_t* __restrict__ counters) {
  if (counters[C_OVER]) return;  // uniform
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint64_t nw = ((uint64_t)gridDim.x * EM_THREADS) >> 5;
  for (uint64_t b = (((uint64_t)blockIdx.x * EM_THREADS + threadIdx.x) >> 5) * 32; b < V; b += nw * 32) {
    const uint64_t i = b + lane;
    uint32_t n = i < V ? ntiles[i] : 0u;
    // the listed Gaussians, one append per warp and list
    const uint32_t bb = __ballot_sync(FULL, n > EM_CTA), bm = __ballot_sync(FULL, n > EM_WARP && n <= EM_CTA);
    if (bb | bm) {
      uint32_t ob = 0, om = 0;
      if (lane == 0) {
        if (bb) ob = atomicAdd(&counters[C_NBIG_G], (uint32_t)__popc(bb));
        if (bm) om = atomicAdd(&counters[C_NMID_G], (uint32_t)__popc(bm));
      }
      ob = __shfl_sync(FULL, ob, 0);
      om = __shfl_sync(FULL, om, 0);
      if ((bb >> lane) & 1u) big[ob + __popc(bb & lt)] = (uint32_t)i;
      if ((bm >> lane) & 1u) mid[om + __popc(bm & lt)] = (uint32_t)i;
      if (n > EM_WARP) n = 0;
    }
    uint32_t inc = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t tot = __shfl_sync(FULL, inc, 31);
    if (tot == 0) continue;  // uniform
    uint32_t rxy = 0, rz = 0, dk = 0;
    if (n) {
      const ushort4 r = rect[i];
      rxy = (uint32_t)r.x | ((uint32_t)r.y << 16);
      rz = r.z;
      dk = __float_as_uint(depth[i]);
    }
    const uint32_t ex = inc - n;
    for (uint32_t k0 = 0; k0 < tot; k0 += 32 * EM_UNROLL) {
      uint32_t tile[EM_UNROLL], kd[EM_UNROLL], id[EM_UNROLL];
#pragma unroll
      for (int u = 0; u < EM_UNROLL; ++u) {
        const uint32_t k = k0 + 32 * u + lane;
        // owner: the number of lanes whose inclusive count is <= k
        int j = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
          const uint32_t v = __shfl_sync(FULL, inc, j + s - 1);
          if (v <= k) j += s;
        }
        j = min(j, 31);
        const uint32_t oex = __shfl_sync(FULL, ex, j);
        const uint32_t oxy = __shfl_sync(FULL, rxy, j);
        const uint32_t oz = __shfl_sync(FULL, rz, j);
        kd[u] = __shfl_sync(FULL, dk, j);
        id[u] = (uint32_t)(b + (uint64_t)j);
        const uint32_t x0 = oxy & 0xFFFFu, y0 = oxy >> 16;
        const uint32_t wdt = oz > x0 ? oz - x0 : 1u;
        const uint32_t loc = k - oex, dy = loc / wdt;
        tile[u] = k < tot ? (y0 + dy) * (uint32_t)TX + x0 + (loc - dy * wdt) : FULL;
      }
      place_pairs(tile, kd, id, (int)min((tot - k0 + 31) / 32, (uint32_t)EM_UNROLL), ranges, tfill, pkeys, pvals,
                  &counters[6]);
    }
  }
}

// Pairs of the listed Gaussians: CTA c emits the Gaussians of more than
// EM_CTA tiles c, c + gridDim.x, ..., then each warp those of the middle list
// (EM_WARP < tiles <= EM_CTA) in warp-stride order, EM_UNROLL pairs per
// thread per round.
__global__ void __launch_bounds__(EM_THREADS) k_emit_big(const uint32_t* __restrict__ big,
                                                        const uint32_t* __restrict__ mid,
                                                        const ushort4* __restrict__ rect,
                                                        const float* __restrict__ depth, int TX,
                                                        const uint2* __restrict__ ranges,
                                                        uint32_t* __restrict__ tfill, uint32_t* __restrict__ pkeys,
                                                        uint32_t* __restrict__ pvals,
                                                        uint32_t* __restrict__ counters) {
  if (counters[C_OVER]) return;
  const uint32_t nb = counters[C_NBIG_G], nm = counters[C_NMID_G];
  const int lane = threadIdx.x & 31;
  for (uint32_t q = blockIdx.x; q < nb; q += gridDim.x) {
    const uint32_t i = big[q];
    const ushort4 r = rect[i];
    const uint32_t dk = __float_as_uint(depth[i]);
    const uint32_t wdt = (uint32_t)(r.z - r.x), n = wdt * (uint32_t)(r.w - r.y);
    for (uint32_t k0 = 0; k0 < n; k0 += EM_UNROLL * EM_THREADS) {
      uint32_t tile[EM_UNROLL], kd[EM_UNROLL], id[EM_UNROLL];
#pragma unroll
      for (int u = 0; u < EM_UNROLL; ++u) {
        const uint32_t k = k0 + (uint32_t)u * EM_THREADS + threadIdx.x;
        const uint32_t dy = k / wdt;
        tile[u] = k < n ? (r.y + dy) * (uint32_t)TX + r.x + (k - dy * wdt) : FULL;
        kd[u] = dk;
        id[u] = i;
      }
      place_pairs(tile, kd, id, EM_UNROLL, ranges, tfill, pkeys, pvals, &counters[6]);
    }
  }
  const uint32_t nw = (gridDim.x * EM_THREADS) >> 5;
  for (uint32_t q = (blockIdx.x * EM_THREADS + threadIdx.x) >> 5; q < nm; q += nw) {
    const uint32_t i = mid[q];
    const ushort4 r = rect[i];
    const uint32_t dk = __float_as_uint(depth[i]);
    const uint32_t wdt = (uint32_t)(r.z - r.x), n = wdt * (uint32_t)(r.w - r.y);
    for (uint32_t k0 = 0; k0 < n; k0 += EM_UNROLL * 32) {
      uint32_t tile[EM_UNROLL], kd[EM_UNROLL], id[EM_UNROLL];
#pragma unroll
      for (int u = 0; u < EM_UNROLL; ++u) {
        const uint32_t k = k0 + 32 * u + lane;
        const uint32_t dy = k / wdt;
        tile[u] = k < n ? (r.y + dy) * (uint32_t)TX + r.x + (k - dy * wdt) : FULL;
        kd[u] = dk;
        id[u] = i;
      }
      place_pairs(tile, kd, id, (int)min((n - k0 + 31) / 32, (uint32_t)EM_UNROLL), ranges, tfill, pkeys, pvals,
                  &counters[6]);
    }
  }
}

// Ascending bitonic sort of 32 keys, one per lane, with shuffles.
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned long long o = __shfl_xor_sync(FULL, v, j);
      // the lower lane of an ascending pair (or the upper of a descending one) keeps the minimum
      const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
      v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
    }
  return v;
}

// Sorts the keys (depth bits << 32 | position) of the pairs [p0, p0 + n), n
// <= 8 blockDim.x, in shared memory (two buffers of n keys): each warp sorts
// runs of 32 with shuffles, then runs are merged pairwise, every thread
// producing P = the power of two >= n / blockDim.x outputs of one merge (2 run
// >= 64 >= 8 >= P, so a thread's outputs stay in one merge), starting where
// the merge path crosses its first output.  Stores the positions (and, with
// keys_out, the depth bits) back in order.
__device__ void sort_tile(unsigned long long* buf0, unsigned long long* buf1, uint32_t* __restrict__ pkeys,
                          uint32_t* __restrict__ pvals, uint64_t p0, uint32_t n, bool keys_out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const uint32_t nch = (n + 31) / 32;
  for (uint32_t c = w; c < nch; c += nwarp) {
    const uint32_t e = c * 32 + lane;
    unsigned long long v = e < n ? ((unsigned long long)pkeys[p0 + e] << 32) | pvals[p0 + e] : ~0ull;
    v = warp_sort32(v);  // padding keys sort last
    if (e < n) buf0[e] = v;
  }
  __syncthreads();
  uint32_t P = 1;
  while (P * blockDim.x < n) P <<= 1;
  unsigned long long *src = buf0, *dst = buf1;
  for (uint32_t L = 32; L < n; L <<= 1) {
    const uint32_t d0 = threadIdx.x * P;
    if (d0 < n) {
      const uint32_t a0 = d0 & ~(2 * L - 1);
      const uint32_t la = min(L, n - a0);
      const uint32_t lb = a0 + la < n ? min(L, n - a0 - la) : 0u;
      const unsigned long long* A = src + a0;
      const unsigned long long* Bv = A + la;
      const uint32_t d = d0 - a0;
      uint32_t lo = d > lb ? d - lb : 0u, hi = min(d, la);
      while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (A[m] < Bv[d - m - 1])
          lo = m + 1;
        else
          hi = m;
      }
      uint32_t i = lo, j = d - lo;
      const uint32_t cnt = min(P, n - d0);
      for (uint32_t q = 0; q < cnt; ++q) {
        const bool takeA = j >= lb || (i < la && A[i] < Bv[j]);
        dst[d0 + q] = takeA ? A[i] : Bv[j];
        if (takeA)
          ++i;
        else
          ++j;
      }
    }
    __syncthreads();
    unsigned long long* t = src;
    src = dst;
    dst = t;
  }
  for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
    const unsigned long long v = src[e];
    if (keys_out) pkeys[p0 + e] = (uint32_t)(v >> 32);
    pvals[p0 + e] = (uint32_t)v;
  }
  __syncthreads();  // the buffers are reused
}

__global__ void __launch_bounds__(SORT_THREADS) k_tile_sort(const uint2* __restrict__ ranges,
                                                           uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals) {
  __shared__ unsigned long long key[2][SORT_SMALL];
  const uint2 r = ranges[blockIdx.x];
  const uint32_t n = r.y - r.x;
  if (n <= 1 || n > SORT_SMALL) return;  // uniform
  if (n <= 32) {
    if (threadIdx.x < 32) {
      const uint32_t e = threadIdx.x;
      unsigned long long v = e < n ? ((unsigned long long)pkeys[r.x + e] << 32) | pvals[r.x + e] : ~0ull;
      v = warp_sort32(v);
      if (e < n) pvals[r.x + e] = (uint32_t)v;
    }
    return;
  }
  sort_tile(key[0], key[1], pkeys, pvals, r.x, n, false);
}

__device__ __forceinline__ unsigned long long key_at(const uint32_t* pk, const uint32_t* pv, uint64_t i) {
  return ((unsigned long long)pk[i] << 32) | pv[i];
}

// Merges the sorted runs [a0, a0 + la) and [a0 + la, a0 + la + lb) of the
// (pk, pv) key arrays into (qk, qv) at a0: each thread takes an equal share
// of the output and finds where it starts on the merge path.
__device__ void merge_runs(const uint32_t* pk, const uint32_t* pv, uint32_t* qk, uint32_t* qv, uint64_t a0,
                           uint32_t la, uint32_t lb) {
  const uint64_t b0 = a0 + la;
  const uint32_t L = la + lb;
  const uint32_t share = (L + blockDim.x - 1) / blockDim.x;
  const uint32_t d0 = min(L, threadIdx.x * share), d1 = min(L, d0 + share);
  if (d0 >= d1) return;
  // split: i from A and d0 - i from B, with A[i - 1] < B[d0 - i] and B[d0 - i - 1] < A[i]
  uint32_t lo = d0 > lb ? d0 - lb : 0u, hi = min(d0, la);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (key_at(pk, pv, a0 + mid) < key_at(pk, pv, b0 + (d0 - mid - 1)))
      lo = mid + 1;
    else
      hi = mid;
  }
  uint32_t i = lo, j = d0 - lo;
  for (uint32_t d = d0; d < d1; ++d) {
    bool takeA;
    if (i >= la)
      takeA = false;
    else if (j >= lb)
      takeA = true;
    else
      takeA = key_at(pk, pv, a0 + i) < key_at(pk, pv, b0 + j);
    const uint64_t src = takeA ? a0 + i : b0 + j;
    qk[a0 + d] = pk[src];
    qv[a0 + d] = pv[src];
    if (takeA)
      ++i;
    else
      ++j;
  }
}

// Tiles above SORT_SMALL pairs (listed by k_tile_scan), one per CTA at a
// time: up to SORT_BIG keys in shared memory; longer lists are sorted in
// runs of SORT_BIG and merged pairwise between the pair arrays and their
// second halves (at offset cap), the result landing back in pvals.
__global__ void __launch_bounds__(SORT_BIG_THREADS) k_tile_sort_big(const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ tbig,
                                                                   const uint32_t* __restrict__ counters,
                                                                   uint32_t* __restrict__ pkeys,
                                                                   uint32_t* __restrict__ pvals, uint64_t cap) {
  extern __shared__ unsigned long long bkey[];  // 2 x SORT_BIG
  const uint32_t nt = counters[C_NBIG_T];
  for (uint32_t q = blockIdx.x; q < nt; q += gridDim.x) {
    const uint2 r = ranges[tbig[q]];
    const uint32_t n = r.y - r.x;
    const bool runs = n > SORT_BIG;
    for (uint32_t c0 = 0; c0 < n; c0 += SORT_BIG)
      sort_tile(bkey, bkey + SORT_BIG, pkeys, pvals, (uint64_t)r.x + c0, min(SORT_BIG, n - c0), runs);
    if (!runs) continue;
    uint32_t *pk = pkeys, *pv = pvals, *qk = pkeys + cap, *qv = pvals + cap;
    for (uint32_t run = SORT_BIG; run < n; run *= 2) {
      for (uint32_t a = 0; a < n; a += 2 * run) {
        const uint32_t la = min(run, n - a), lb = a + la < n ? min(run, n - a - la) : 0u;
        merge_runs(pk, pv, qk, qv, (uint64_t)r.x + a, la, lb);
      }
      __syncthreads();  // the merged runs are read by other threads next
      uint32_t* t;
      t = pk; pk = qk; qk = t;
      t = pv; pv = qv; qv = t;
    }
    if (pv != pvals) {
      for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) pvals[(uint64_t)r.x + e] = pv[(uint64_t)r.x + e];
      __syncthreads();
    }
  }
}

}  // namespace

size_t tile_scan_smem_bytes(int TX, int TY) { return (size_t)(TX + 1) * (size_t)(TY + 1) * sizeof(int32_t); }

void bin_tiles(uint64_t V, int TX, int TY, CamState& cs, cudaStream_t s) {
  static bool attrs = false;
  if (!attrs) {
    TGS_CUDA(cudaFuncSetAttribute(k_tile_scan, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)TILE_SCAN_SMEM_MAX));
    TGS_CUDA(cudaFuncSetAttribute(k_tile_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(2 * SORT_BIG * sizeof(unsigned long long))));
    attrs = true;
  }
  const uint64_t tiles = (uint64_t)TX * TY;
  const size_t dsm = tile_scan_smem_bytes(TX, TY);
  TGS_CHECK(dsm <= TILE_SCAN_SMEM_MAX, TGS_ERR_CAPACITY, "image has too many tiles for the tile scan");
  TGS_CHECK(cs.cap_pairs < 0x80000000ull, TGS_ERR_CAPACITY, "pair capacity above 2^31");
  k_tile_scan<<<1, TS_THREADS, dsm, s>>>(cs.tdiff, TX, TY, cs.cap_pairs, cs.counters, cs.step_flag, cs.ranges,
                                         cs.tfill, cs.tbig);
  TGS_LAUNCHED();
  // the raster tile order reads only the ranges: it runs beside the emission
  // and the sorts (one CTA on a high-priority stream), joined before the
  // forward raster
  TGS_CUDA(cudaEventRecord(cs.ev_fork, s));
  TGS_CUDA(cudaStreamWaitEvent(cs.aux, cs.ev_fork, 0));
  k_tile_order<<<1, TS_THREADS, 0, cs.aux>>>(cs.ranges, (uint32_t)tiles, cs.counters, cs.torder, cs.tck, cs.units,
                                             cs.ck_cap);
  TGS_LAUNCHED();
  TGS_CUDA(cudaEventRecord(cs.ev_join, cs.aux));
  const unsigned g_e = std::min<uint64_t>(div_up(V, EM_THREADS), 8 * NSM);
  // the big and middle Gaussian lists live in the two halves of dkeys (2 V words)
  k_emit_tiles<<<g_e, EM_THREADS, 0, s>>>(V, cs.ntiles, cs.rect, cs.depth, TX, cs.ranges, cs.tfill, cs.pkeys,
                                          cs.pvals, cs.dkeys, cs.dkeys + cs.cap_v, cs.counters);
  TGS_LAUNCHED();
  k_emit_big<<<2 * NSM, EM_THREADS, 0, s>>>(cs.dkeys, cs.dkeys + cs.cap_v, cs.rect, cs.depth, TX, cs.ranges, cs.tfill,
                                            cs.pkeys, cs.pvals, cs.counters);
  TGS_LAUNCHED();
  k_tile_sort<<<(unsigned)tiles, SORT_THREADS, 0, s>>>(cs.ranges, cs.pkeys, cs.pvals);
  TGS_LAUNCHED();
  k_tile_sort_big<<<NSM, SORT_BIG_THREADS, 2 * SORT_BIG * sizeof(unsigned long long), s>>>(
      cs.ranges, cs.tbig, cs.counters, cs.pkeys, cs.pvals, cs.cap_pairs);
  TGS_LAUNCHED();
  TGS_CUDA(cudaStreamWaitEvent(s, cs.ev_join, 0));
}

}  // namespace tgs
