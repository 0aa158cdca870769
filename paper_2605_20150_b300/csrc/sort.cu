// Device-wide exclusive scan and stable LSD radix sort: the Morton order of a
// new table, the scans of Algorithm 1 and of the predictor's candidate
// blocks, and, in the fixed-capacity render, the depth sort of the visible
// Gaussians and the stable regrouping of their (tile, Gaussian) pairs by tile.
//
// A radix pass = histogram kernel + scan of the digit-major count table +
// scatter kernel.  The scatter ranks keys stably inside a 4096-key tile with
// warp-level multi-split (match_any + popc per warp, then a cross-warp scan),
// stages the tile in shared memory in digit order and writes each digit run
// contiguously, so global stores are coalesced.
#include "sort.cuh"

namespace tgs {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;  // 4096

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;  // 4096
constexpr int RS_BINS = 256;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Block-wide exclusive scan of one value per thread (NT threads).
template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* smem_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = warp_incl_scan(x);
  if (lane == 31) smem_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t v = lane < NT / 32 ? smem_warp[lane] : 0;
    uint32_t vi = warp_incl_scan(v);
    if (lane < NT / 32) smem_warp[lane] = vi - v;
    if (lane == NT / 32 - 1) smem_warp[NT / 32] = vi;
  }
  __syncthreads();
  uint32_t r = smem_warp[w] + inc - x;
  if (total) *total = smem_warp[NT / 32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const uint32_t* __restrict__ in, uint64_t n,
                                                             uint32_t* __restrict__ partial) {
  __shared__ uint32_t sw[SCAN_THREADS / 32 + 1];
  uint64_t base = (uint64_t)blockIdx.x * SCAN_CHUNK;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    uint64_t p = base + (uint64_t)i * SCAN_THREADS + threadIdx.x;
    if (p < n) s += in[p];
  }
  uint32_t tot;
  block_excl_scan<SCAN_THREADS>(s, sw, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t* __restrict__ partial, uint32_t nc,
                                                        uint32_t* __restrict__ total) {
  __shared__ uint32_t sw[1024 / 32 + 1];
  uint32_t carry = 0;
  for (uint32_t b = 0; b < nc; b += 1024) {
    uint32_t i = b + threadIdx.x;
    uint32_t v = i < nc ? partial[i] : 0;
    uint32_t tot;
    uint32_t e = block_excl_scan<1024>(v, sw, &tot);
    if (i < nc) partial[i] = carry + e;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const uint32_t* __restrict__ in,
                                                            uint32_t* __restrict__ out, uint64_t n,
                                                            const uint32_t* __restrict__ partial) {
  __shared__ uint32_t buf[SCAN_CHUNK + SCAN_CHUNK / 32];
  __shared__ uint32_t sw[SCAN_THREADS / 32 + 1];
  uint64_t base = (uint64_t)blockIdx.x * SCAN_CHUNK;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int q = i * SCAN_THREADS + threadIdx.x;
    uint64_t p = base + q;
    buf[q + (q >> 5)] = p < n ? in[p] : 0;
  }
  __syncthreads();
  uint32_t v[SCAN_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int q = threadIdx.x * SCAN_ITEMS + i;
    v[i] = buf[q + (q >> 5)];
    s += v[i];
  }
  uint32_t e = block_excl_scan<SCAN_THREADS>(s, sw, nullptr) + partial[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int q = threadIdx.x * SCAN_ITEMS + i;
    buf[q + (q >> 5)] = e;
    e += v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    int q = i * SCAN_THREADS + threadIdx.x;
    uint64_t p = base + q;
    if (p < n) out[p] = buf[q + (q >> 5)];
  }
}

// Small scans in one CTA: chunks of SCAN_CHUNK in order, carrying the sum.
constexpr uint64_t SCAN_SINGLE_MAX = 16 * SCAN_CHUNK;
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_single(const uint32_t* __restrict__ in,
                                                             uint32_t* __restrict__ out, uint64_t n,
                                                             uint32_t* __restrict__ total) {
  __shared__ uint32_t buf[SCAN_CHUNK + SCAN_CHUNK / 32];
  __shared__ uint32_t sw[SCAN_THREADS / 32 + 1];
  uint32_t carry = 0;
  for (uint64_t base = 0; base < n; base += SCAN_CHUNK) {
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      int q = i * SCAN_THREADS + threadIdx.x;
      uint64_t p = base + q;
      buf[q + (q >> 5)] = p < n ? in[p] : 0;
    }
    __syncthreads();
    uint32_t v[SCAN_ITEMS];
    uint32_t sm = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      int q = threadIdx.x * SCAN_ITEMS + i;
      v[i] = buf[q + (q >> 5)];
      sm += v[i];
    }
    uint32_t tot;
    uint32_t e = block_excl_scan<SCAN_THREADS>(sm, sw, &tot) + carry;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      int q = threadIdx.x * SCAN_ITEMS + i;
      buf[q + (q >> 5)] = e;
      e += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      int q = i * SCAN_THREADS + threadIdx.x;
      uint64_t p = base + q;
      if (p < n) out[p] = buf[q + (q >> 5)];
    }
    carry += tot;
    __syncthreads();  // buf is refilled next
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint32_t* __restrict__ keys, uint64_t n,
                                                          int shift, uint32_t mask,
                                                          uint32_t* __restrict__ counts, uint32_t nc) {
  __shared__ uint32_t h[RS_WARPS][RS_BINS];
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&h[0][0])[i] = 0;
  __syncthreads();
  uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
  for (int i = 0; i < RS_ITEMS; ++i) {
    uint64_t p = base + (uint64_t)i * RS_THREADS + threadIdx.x;
    if (p < n) atomicAdd(&h[w][(keys[p] >> shift) & mask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < RS_WARPS; ++k) s += h[k][d];
    counts[(uint64_t)d * nc + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin,
                                                             uint32_t* __restrict__ kout,
                                                             uint32_t* __restrict__ vout, uint64_t n, int shift,
                                                             uint32_t mask, const uint32_t* __restrict__ offs,
                                                             uint32_t nc) {
  __shared__ uint32_t cnt[RS_WARPS][RS_BINS];
  __shared__ uint32_t dstart[RS_BINS];
  __shared__ uint32_t goff[RS_BINS];
  __shared__ uint32_t sw[RS_THREADS / 32 + 1];
  __shared__ uint32_t sk[RS_TILE];
  __shared__ uint32_t sv[RS_TILE];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&cnt[0][0])[i] = 0;
  for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) goff[d] = offs[(uint64_t)d * nc + blockIdx.x];
  __syncthreads();
  // warp w owns the contiguous run [w*512, w*512+512) of the tile; iteration j
  // covers 32 consecutive keys, so (w, j, lane) is the input order
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE + (uint64_t)w * (32 * RS_ITEMS);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t key[RS_ITEMS], val[RS_ITEMS], rk[RS_ITEMS];
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    uint64_t p = base + (uint64_t)j * 32 + lane;
    bool valid = p < n;
    key[j] = valid ? kin[p] : 0u;
    val[j] = valid ? vin[p] : 0u;
    uint32_t d = valid ? ((key[j] >> shift) & mask) : (uint32_t)RS_BINS;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && valid) {
      old = cnt[w][d];
      cnt[w][d] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rk[j] = old + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();
  uint32_t tot;
  {
    const int d = threadIdx.x;  // RS_THREADS == RS_BINS
    uint32_t run = 0;
#pragma unroll
    for (int k = 0; k < RS_WARPS; ++k) {
      uint32_t c = cnt[k][d];
      cnt[k][d] = run;
      run += c;
    }
    tot = run;
  }
  uint32_t ds = block_excl_scan<RS_THREADS>(tot, sw, nullptr);
  dstart[threadIdx.x] = ds;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RS_ITEMS; ++j) {
    uint64_t p = base + (uint64_t)j * 32 + lane;
    if (p < n) {
      uint32_t d = (key[j] >> shift) & mask;
      uint32_t pos = dstart[d] + cnt[w][d] + rk[j];
      sk[pos] = key[j];
      sv[pos] = val[j];
    }
  }
  __syncthreads();
  uint64_t tile_n = n - (uint64_t)blockIdx.x * RS_TILE;
  if (tile_n > RS_TILE) tile_n = RS_TILE;
#pragma unroll 4
  for (int i = 0; i < RS_ITEMS; ++i) {
    uint32_t e = i * RS_THREADS + threadIdx.x;
    if (e < tile_n) {
      uint32_t k = sk[e];
      uint32_t d = (k >> shift) & mask;
      uint32_t g = goff[d] + (e - dstart[d]);
      kout[g] = k;
      vout[g] = sv[e];
    }
  }
}


// One CTA: exclusive scan of the digit-major count table counts[d][c] in
// place, which gives the global start of (digit d, chunk c).  Each thread
// scans a contiguous segment (independent loads, cached lines), the segment
// sums are scanned across the block.  Used up to RSO_MAX entries (4 per
// thread): with longer segments the serial loads of one CTA cost more than
// the chunked scan (measured 32 us for 18k-76k entries).
constexpr int RSO_THREADS = 1024;
constexpr uint64_t RSO_MAX = 4ull * RSO_THREADS;
__global__ void __launch_bounds__(RSO_THREADS) k_rsd_offsets(uint32_t* __restrict__ counts, uint32_t G) {
  __shared__ uint32_t sw[RSO_THREADS / 32 + 1];
  const uint32_t E = RS_BINS * G;
  const uint32_t per = (E + RSO_THREADS - 1) / RSO_THREADS;
  const uint32_t a = threadIdx.x * per;
  const uint32_t b = min(a + per, E);
  uint32_t sum = 0;
#pragma unroll 8
  for (uint32_t i = a; i < b; ++i) sum += counts[i];
  uint32_t run = block_excl_scan<RSO_THREADS>(sum, sw, nullptr);
#pragma unroll 8
  for (uint32_t i = a; i < b; ++i) {
    const uint32_t x = counts[i];
    counts[i] = run;
    run += x;
  }
}

}  // namespace

size_t scan_scratch_bytes(uint64_t n) { return (size_t)(div_up(n, SCAN_CHUNK) + 4) * sizeof(uint32_t); }

size_t radix_scratch_bytes(uint64_t n) {
  uint64_t nc = div_up(n, RS_TILE);
  uint64_t m = nc * RS_BINS;
  return (size_t)m * sizeof(uint32_t) + scan_scratch_bytes(m) + 256;
}

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint32_t* total_dev, uint64_t n, void* scratch,
                        cudaStream_t s) {
  if (n == 0) {
    if (total_dev) TGS_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s));
    return;
  }
  if (n <= SCAN_SINGLE_MAX) {
    k_scan_single<<<1, SCAN_THREADS, 0, s>>>(in, out, n, total_dev);
    TGS_LAUNCHED();
    return;
  }
  uint32_t nc = div_up(n, SCAN_CHUNK);
  uint32_t* partial = (uint32_t*)scratch;
  k_scan_reduce<<<nc, SCAN_THREADS, 0, s>>>(in, n, partial);
  TGS_LAUNCHED();
  k_scan_partials<<<1, 1024, 0, s>>>(partial, nc, total_dev);
  TGS_LAUNCHED();
  k_scan_apply<<<nc, SCAN_THREADS, 0, s>>>(in, out, n, partial);
  TGS_LAUNCHED();
}

void radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt, uint64_t n,
                      int bits, void* scratch, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  uint32_t nc = div_up(n, RS_TILE);
  uint32_t* counts = (uint32_t*)scratch;
  void* scan_scr = (void*)(counts + (size_t)nc * RS_BINS);
  uint32_t *ki = keys, *vi = vals, *ko = keys_alt, *vo = vals_alt;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    int nb = bits - shift < 8 ? bits - shift : 8;
    uint32_t mask = (1u << nb) - 1u;
    k_radix_hist<<<nc, RS_THREADS, 0, s>>>(ki, n, shift, mask, counts, nc);
    TGS_LAUNCHED();
    if ((uint64_t)nc * RS_BINS <= RSO_MAX) {
      k_rsd_offsets<<<1, RSO_THREADS, 0, s>>>(counts, nc);  // same digit-major table
      TGS_LAUNCHED();
    } else {
      exclusive_scan_u32(counts, counts, nullptr, (uint64_t)nc * RS_BINS, scan_scr, s);
    }
    k_radix_scatter<<<nc, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n, shift, mask, counts, nc);
    TGS_LAUNCHED();
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
    ++passes;
  }
  if (passes & 1) {
    TGS_CUDA(cudaMemcpyAsync(keys, ki, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    TGS_CUDA(cudaMemcpyAsync(vals, vi, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace tgs
