// Level-2 rendering kernels (Sec. 3.3 "Level 2"): the standard 3DGS
// forward/backward run over the Gaussians of a render list of resident
// blocks, written for sm_103a.
//
//  k_preprocess      one thread per Gaussian: coalesced field-major loads from
//                    the block slot, EWA projection, degree-3 SH colour, tile
//                    rect; exact FP32 key path for centre and depth.
//  binning (tiles.cu): per-tile pair counts from the tile rects, pairs
//  placed in their tile's range and sorted per tile on (depth bits,
//  render-list position), the order of one stable sort of (tile << 32 |
//  depth bits) keys emitted in render-list order.  The fixed-capacity render
//  (render_forward_fixed) reaches the same order by visible compaction, a
//  stable radix sort of the visible Gaussians by depth, pair emission in
//  depth order and a stable radix sort of the pairs by tile.
//  k_raster_fwd      one CTA per 16x16 tile (8 warps of 8 x 4 pixels, one
//                    pixel per thread), 32 splats per warp staged in shared
//                    memory, front-to-back blending with the 0.99 clamp,
//                    the 1/255 skip and the T < 1e-4 stop.
//  k_raster_bwd      reverse traversal from each pixel's last contributor,
//                    recomputing T_i = T_{i+1} / (1 - alpha_i); per-Gaussian
//                    a warp's per-lane 2D gradient sums of three splats are
//                    summed row-wise through shared memory and added with one
//                    atomic per (warp, Gaussian, field).
//  k_preprocess_bwd  chain rule to the 59 parameters.
//  k_adam            masked Adam (App. A.1, Eq. masked_update).
#include <math.h>

#include "raster.cuh"
#include "sort.cuh"

namespace tgs {

namespace {

constexpr int PP_THREADS = 256;

// Parameter field f of one Gaussian: FP32 storage, or (BF16 form) BF16 for
// the SH-rest coefficients f >= 14.
template <bool BF>
__device__ __forceinline__ float ldp(const float* __restrict__ p32, const __nv_bfloat16* __restrict__ p16, uint32_t B,
                                     int f) {
  if (BF && f >= F_BF16) return __bfloat162float(p16[(uint64_t)(f - F_BF16) * B]);
  return p32[(uint64_t)f * B];
}

__device__ __forceinline__ const __nv_bfloat16* sh16(const float* slot_lane0, uint32_t B, uint32_t lane) {
  return reinterpret_cast<const __nv_bfloat16*>(slot_lane0 + (uint64_t)F_BF16 * B) + lane;
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014) as a counter hash.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Rounding draws of Adam's BF16 stores: one SplitMix64 finaliser per
// Gaussian and step gives a 32-bit key; per field, the MurmurHash3 32-bit
// finaliser (Appleby) of key + f * golden gives 32 bits (m draw low 16, v
// draw high 16) and, for a BF16 parameter, a second finaliser 16 more.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint32_t sr_key(uint32_t seed, uint64_t gid, uint32_t step) {
  return (uint32_t)mix64(((uint64_t)seed << 40) ^ (gid * 0x9E3779B97F4A7C15ull) ^ ((uint64_t)step << 20));
}

// i / B for a render-list position (a shift when B is a power of two: the
// branch is uniform)
__device__ __forceinline__ unsigned item_of(uint64_t i, uint32_t B) {
  const uint32_t sh = (uint32_t)__ffs(B) - 1u;
  if (B == 1u << sh) return (unsigned)(i >> sh);
  return (unsigned)(i / B);
}

// FP32 -> BF16: round to nearest even, or stochastically with the 16 random
// bits r (added below the kept mantissa, then truncated; unbiased in
// expectation).
__device__ __forceinline__ __nv_bfloat16 to_bf16(float x, bool sr, uint32_t r) {
  if (!sr) return __float2bfloat16_rn(x);
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) == 0x7F800000u) return __float2bfloat16_rn(x);
  uint32_t v = (u + (r & 0xFFFFu)) & 0xFFFF0000u;
  return __ushort_as_bfloat16((unsigned short)(v >> 16));
}

// Real SH normalisations (sqrt(2) Re/Im of the Condon-Shortley complex
// harmonics, l <= 3), from their closed forms:
constexpr float K00 = 0.28209479177387814f;  // 1/(2 sqrt(pi))
constexpr float K1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float K2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float K2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float K2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float K3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
constexpr float K3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float K3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
constexpr float K3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float K3e = 1.445305721320277f;    // sqrt(105/pi)/4

// Basis values Y[16] at unit direction (x, y, z), ordered l, m = -l..l.
__device__ __forceinline__ void sh_eval(float x, float y, float z, float Y[16]) {
  float xx = x * x, yy = y * y, zz = z * z;
  Y[0] = K00;
  Y[1] = -K1 * y;
  Y[2] = K1 * z;
  Y[3] = -K1 * x;
  Y[4] = K2a * x * y;
  Y[5] = -K2a * y * z;
  Y[6] = K2b * (2.f * zz - xx - yy);
  Y[7] = -K2a * x * z;
  Y[8] = K2c * (xx - yy);
  Y[9] = -K3a * y * (3.f * xx - yy);
  Y[10] = K3b * x * y * z;
  Y[11] = -K3c * y * (4.f * zz - xx - yy);
  Y[12] = K3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -K3c * x * (4.f * zz - xx - yy);
  Y[14] = K3e * z * (xx - yy);
  Y[15] = -K3a * x * (xx - 3.f * yy);
}

// Gradient of the basis w.r.t. the (unnormalised-polynomial) direction.
__device__ __forceinline__ void sh_grad(float x, float y, float z, float G[16][3]) {
  float xx = x * x, yy = y * y, zz = z * z;
  G[0][0] = 0; G[0][1] = 0; G[0][2] = 0;
  G[1][0] = 0; G[1][1] = -K1; G[1][2] = 0;
  G[2][0] = 0; G[2][1] = 0; G[2][2] = K1;
  G[3][0] = -K1; G[3][1] = 0; G[3][2] = 0;
  G[4][0] = K2a * y; G[4][1] = K2a * x; G[4][2] = 0;
  G[5][0] = 0; G[5][1] = -K2a * z; G[5][2] = -K2a * y;
  G[6][0] = -2.f * K2b * x; G[6][1] = -2.f * K2b * y; G[6][2] = 4.f * K2b * z;
  G[7][0] = -K2a * z; G[7][1] = 0; G[7][2] = -K2a * x;
  G[8][0] = 2.f * K2c * x; G[8][1] = -2.f * K2c * y; G[8][2] = 0;
  G[9][0] = -K3a * 6.f * x * y; G[9][1] = -K3a * (3.f * xx - 3.f * yy); G[9][2] = 0;
  G[10][0] = K3b * y * z; G[10][1] = K3b * x * z; G[10][2] = K3b * x * y;
  G[11][0] = K3c * 2.f * x * y; G[11][1] = -K3c * (4.f * zz - xx - 3.f * yy); G[11][2] = -K3c * 8.f * y * z;
  G[12][0] = -K3d * 6.f * x * z; G[12][1] = -K3d * 6.f * y * z; G[12][2] = K3d * (6.f * zz - 3.f * xx - 3.f * yy);
  G[13][0] = -K3c * (4.f * zz - 3.f * xx - yy); G[13][1] = K3c * 2.f * x * y; G[13][2] = -K3c * 8.f * x * z;
  G[14][0] = K3e * 2.f * x * z; G[14][1] = -K3e * 2.f * y * z; G[14][2] = K3e * (xx - yy);
  G[15][0] = -K3a * (3.f * xx - 3.f * yy); G[15][1] = K3a * 6.f * x * y; G[15][2] = 0;
}

// Rotation matrix of the normalised quaternion (w, x, y, z).
__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[3][3]) {
  R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
  R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
  R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
}

struct Geo {
  float Rq[3][3], sc[3], qn, qw, qx, qy, qz;
  float S[6];          // Sigma: xx xy xz yy yz zz
  float T[2][3];       // J Rc
  float a, b, c, det;  // dilated 2D covariance
  bool clx, cly;
  float xc, yc;        // clamped tx/tz, ty/tz
};

// Projection geometry shared by the forward and the backward preprocess.
__device__ __forceinline__ void geometry(const DevCam& c, const float* p, uint32_t B, const KeyPath& k, Geo& g) {
  g.sc[0] = expf(p[3 * B]);
  g.sc[1] = expf(p[4 * B]);
  g.sc[2] = expf(p[5 * B]);
  float qw = p[6 * B], qx = p[7 * B], qy = p[8 * B], qz = p[9 * B];
  g.qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  float inv = 1.f / g.qn;
  g.qw = qw * inv; g.qx = qx * inv; g.qy = qy * inv; g.qz = qz * inv;
  quat_rot(g.qw, g.qx, g.qy, g.qz, g.Rq);
  float M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) M[a][b] = g.Rq[a][b] * g.sc[b];
  g.S[0] = M[0][0] * M[0][0] + M[0][1] * M[0][1] + M[0][2] * M[0][2];
  g.S[1] = M[0][0] * M[1][0] + M[0][1] * M[1][1] + M[0][2] * M[1][2];
  g.S[2] = M[0][0] * M[2][0] + M[0][1] * M[2][1] + M[0][2] * M[2][2];
  g.S[3] = M[1][0] * M[1][0] + M[1][1] * M[1][1] + M[1][2] * M[1][2];
  g.S[4] = M[1][0] * M[2][0] + M[1][1] * M[2][1] + M[1][2] * M[2][2];
  g.S[5] = M[2][0] * M[2][0] + M[2][1] * M[2][1] + M[2][2] * M[2][2];
  float tz = k.tz;
  float xr = k.tx / tz, yr = k.ty / tz;
  g.clx = xr < -c.limx || xr > c.limx;
  g.cly = yr < -c.limy || yr > c.limy;
  g.xc = fminf(fmaxf(xr, -c.limx), c.limx);
  g.yc = fminf(fmaxf(yr, -c.limy), c.limy);
  float J00 = c.fx / tz, J02 = -c.fx * g.xc / tz;
  float J11 = c.fy / tz, J12 = -c.fy * g.yc / tz;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    g.T[0][j] = J00 * c.R[0 + j] + J02 * c.R[6 + j];
    g.T[1][j] = J11 * c.R[3 + j] + J12 * c.R[6 + j];
  }
  float TS[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    TS[a][0] = g.T[a][0] * g.S[0] + g.T[a][1] * g.S[1] + g.T[a][2] * g.S[2];
    TS[a][1] = g.T[a][0] * g.S[1] + g.T[a][1] * g.S[3] + g.T[a][2] * g.S[4];
    TS[a][2] = g.T[a][0] * g.S[2] + g.T[a][1] * g.S[4] + g.T[a][2] * g.S[5];
  }
  g.a = TS[0][0] * g.T[0][0] + TS[0][1] * g.T[0][1] + TS[0][2] * g.T[0][2] + DILATION;
  g.b = TS[0][0] * g.T[1][0] + TS[0][1] * g.T[1][1] + TS[0][2] * g.T[1][2];
  g.c = TS[1][0] * g.T[1][0] + TS[1][1] * g.T[1][1] + TS[1][2] * g.T[1][2] + DILATION;
  g.det = g.a * g.c - g.b * g.b;
}

struct PPOut {
  float2* xy;
  float* depth;
  float4* conic_o;
  float4* rgb;
  ushort4* rect;
  int* radius;
  uint32_t* ntiles;
  uint32_t* vflag;
  int32_t* tdiff = nullptr;  // tile difference array and visible count of the tile binning (may be null)
  uint32_t* nvis = nullptr;
};

// One distinct corner of a warp's tile rects: the lanes naming the same cell
// add their +-1 with one atomic.
__device__ __forceinline__ void corner_add(int32_t* __restrict__ d, int idx, int v) {
  const uint32_t key = idx < 0 ? 0xffffffffu : (uint32_t)idx;
  const uint32_t peers = __match_any_sync(0xffffffffu, key);
  if (idx >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&d[idx], v * __popc(peers));
}

template <bool BF>
__global__ void __launch_bounds__(PP_THREADS) k_preprocess(RenderList rl, DevCam c, PPOut o, uint8_t* touched,
                                                          uint32_t* item_touched, unsigned cpi) {
  const unsigned item = blockIdx.x / cpi;
  const unsigned lane = (blockIdx.x - item * cpi) * PP_THREADS + threadIdx.x;
  const uint32_t B = rl.B;
  const bool inb = lane < B;  // no early return: the corner atomics below are warp-wide
  const uint64_t i = (uint64_t)item * B + lane;
  uint32_t area = 0;
  int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
  if (inb && lane < rl.item_count[item]) {
    const float* slot = rl.base + (uint64_t)rl.item_slot[item] * rl.slot_stride;
    const float* p = slot + lane;
    const __nv_bfloat16* q16 = sh16(slot, B, lane);
    float mx = p[0], my = p[B], mz = p[2 * B];
    KeyPath k = key_path(c, mx, my, mz);
    if (k.tz > c.znear && k.tz <= c.zfar) {
      Geo g;
      geometry(c, p, B, k, g);
      if (g.det > 0.f) {
        float mid = 0.5f * (g.a + g.c);
        float lam1 = mid + sqrtf(fmaxf(0.1f, mid * mid - g.det));
        int r = (int)ceilf(3.f * sqrtf(lam1));
        x0 = min(max(floor_div_tile(k.u, -r), 0), c.TX);
        x1 = min(max(floor_div_tile(k.u, r) + 1, 0), c.TX);
        y0 = min(max(floor_div_tile(k.v, -r), 0), c.TY);
        y1 = min(max(floor_div_tile(k.v, r) + 1, 0), c.TY);
        if (x1 > x0 && y1 > y0) {
          area = (uint32_t)((x1 - x0) * (y1 - y0));
          // colour from the degree-3 SH at the view direction
          float dx = mx - c.campos[0], dy = my - c.campos[1], dz = mz - c.campos[2];
          float il = rsqrtf(dx * dx + dy * dy + dz * dz);
          float Y[16];
          sh_eval(dx * il, dy * il, dz * il, Y);
          float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
          for (int kk = 0; kk < 16; ++kk)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) col[ch] += Y[kk] * ldp<BF>(p, q16, B, 11 + 3 * kk + ch);
          uint32_t clampbits = (col[0] < 0.f ? 1u : 0u) | (col[1] < 0.f ? 2u : 0u) | (col[2] < 0.f ? 4u : 0u);
          float opac = 1.f / (1.f + expf(-p[10 * B]));
          o.xy[i] = make_float2(k.u, k.v);
          o.depth[i] = k.tz;
          o.conic_o[i] = make_float4(g.c / g.det, -g.b / g.det, g.a / g.det, opac);
          o.rgb[i] = make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f),
                                 __uint_as_float(clampbits));
          o.rect[i] = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)x1, (unsigned short)y1);
          o.radius[i] = r;
          if (touched) touched[i] = 1;
          if (item_touched) item_touched[item] = 1;
        }
      }
    }
  }
  if (inb) {
    o.ntiles[i] = area;
    o.vflag[i] = area ? 1u : 0u;
  }
  if (o.tdiff) {
    // the rect [x0, x1) x [y0, y1) into the tile difference array
    // ((TX + 1) x (TY + 1)), and the visible count
    const int S = c.TX + 1;
    const bool v = area != 0;
    const uint32_t vb = __ballot_sync(0xffffffffu, v);
    if (vb) {  // uniform
      corner_add(o.tdiff, v ? y0 * S + x0 : -1, 1);
      corner_add(o.tdiff, v ? y0 * S + x1 : -1, -1);
      corner_add(o.tdiff, v ? y1 * S + x0 : -1, -1);
      corner_add(o.tdiff, v ? y1 * S + x1 : -1, 1);
      if ((threadIdx.x & 31) == 0) atomicAdd(o.nvis, (uint32_t)__popc(vb));
    }
  }
}

__global__ void k_compact_visible(uint64_t V, const uint32_t* __restrict__ ntiles, const uint32_t* __restrict__ pos,
                                  const float* __restrict__ depth, uint32_t* __restrict__ dkeys,
                                  uint32_t* __restrict__ dvals) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V || ntiles[i] == 0) return;
  uint32_t q = pos[i];
  dkeys[q] = __float_as_uint(depth[i]);  // depth > 0: the bits order like the values
  dvals[q] = (uint32_t)i;
}

// The counts below (visible Gaussians nv, pairs np) are read from device
// memory, written by the scans that precede them on the stream.
__global__ void k_gather_counts(const uint32_t* __restrict__ nv_dev, const uint32_t* __restrict__ dvals,
                                const uint32_t* __restrict__ ntiles, uint32_t* __restrict__ cnt) {
  uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < *nv_dev) cnt[s] = ntiles[dvals[s]];
}

// Pair emission balanced over pairs: CTA c writes the pairs [1024 c,
// 1024 c + 1024) in order.  Every visible Gaussian has at least one pair, so
// the Gaussians (depth order) covering a chunk are at most 1024 consecutive
// entries of the offsets; they are staged in shared memory and each pair finds
// its Gaussian there by binary search, then its tile from its index inside
// the Gaussian's tile rect (row-major).  Pairs at or beyond cap are not
// written; they raise the camera's overflow flag (flag[0], sticky until the
// host clears it, the pair count needed in flag[1]) and step_flag.
constexpr int EP_THREADS = 256;
constexpr int EP_CHUNK = 1024;

// Warp-cooperative form of last_le: each round the 32 lanes probe 32 evenly
// spaced entries and the range shrinks to one gap.
__device__ __forceinline__ uint32_t warp_last_le(const uint32_t* __restrict__ a, uint32_t n, uint32_t x) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = n;
  while (hi - lo > 32) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint32_t pv = lo + lane * step;
    const uint32_t b = __ballot_sync(0xffffffffu, pv < hi && a[pv] <= x);
    const uint32_t L = 31 - __clz(b);  // lane 0 always qualifies (a[lo] <= x)
    lo += L * step;
    hi = min(hi, lo + step);
  }
  const uint32_t b = __ballot_sync(0xffffffffu, lo + lane < hi && a[lo + lane] <= x);
  return lo + (31 - __clz(b));
}

__device__ __forceinline__ uint32_t last_le(const uint32_t* __restrict__ a, uint32_t n, uint32_t x) {
  // largest i < n with a[i] <= x (a non-decreasing, a[0] <= x)
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(EP_THREADS) k_emit_pairs(const uint32_t* __restrict__ nv_dev,
                                                          const uint32_t* __restrict__ np_dev,
                                                          const uint32_t* __restrict__ dvals,
                                                          const ushort4* __restrict__ rect,
                                                          const uint32_t* __restrict__ off, int TX,
                                                          uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals,
                                                          uint64_t cap, uint32_t* flag, uint32_t* step_flag) {
  __shared__ uint32_t s_off[EP_CHUNK];
  __shared__ uint32_t s_id[EP_CHUNK];
  __shared__ ushort4 s_rect[EP_CHUNK];
  __shared__ uint32_t s_lo, s_cnt;
  const uint32_t nv = *nv_dev;
  const uint64_t np_all = *np_dev;
  const uint32_t np = (uint32_t)(np_all < cap ? np_all : cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && np_all > cap) {
    atomicOr(flag, 1u);
    atomicMax(flag + 1, (uint32_t)(np_all > 0xFFFFFFFFull ? 0xFFFFFFFFull : np_all));
    if (step_flag) atomicOr(step_flag, 1u);
  }
  for (uint32_t p0 = blockIdx.x * EP_CHUNK; p0 < np; p0 += gridDim.x * EP_CHUNK) {
    const uint32_t p1 = min(p0 + EP_CHUNK, np) - 1;
    // warp 0 finds the chunk's first Gaussian, warp 1 its last
    if (threadIdx.x < 64) {
      const uint32_t k = warp_last_le(off, nv, threadIdx.x < 32 ? p0 : p1);
      if (threadIdx.x == 0) s_lo = k;
      if (threadIdx.x == 32) s_cnt = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_cnt = s_cnt - s_lo + 1;
    __syncthreads();
    const uint32_t lo = s_lo, cnt = s_cnt;
    for (uint32_t e = threadIdx.x; e < cnt; e += EP_THREADS) {
      const uint32_t id = dvals[lo + e];
      s_off[e] = off[lo + e];
      s_id[e] = id;
      s_rect[e] = rect[id];
    }
    __syncthreads();
    for (uint32_t p = p0 + threadIdx.x; p <= p1; p += EP_THREADS) {
      const uint32_t k = last_le(s_off, cnt, p);
      const ushort4 r = s_rect[k];
      const uint32_t w = (uint32_t)(r.z - r.x);
      const uint32_t loc = p - s_off[k];
      const uint32_t dy = loc / w;
      pkeys[p] = (uint32_t)((r.y + dy) * TX + r.x + (loc - dy * w));
      pvals[p] = s_id[k];
    }
    __syncthreads();
  }
}

__global__ void k_ranges(const uint32_t* __restrict__ np_dev, uint64_t cap, const uint32_t* __restrict__ pkeys,
                         uint2* __restrict__ ranges) {
  uint64_t np = *np_dev;
  if (np > cap) np = cap;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t t = pkeys[p];
    if (p == 0 || pkeys[p - 1] != t) ranges[t].x = (uint32_t)p;
    if (p == np - 1 || pkeys[p + 1] != t) ranges[t].y = (uint32_t)(p + 1);
  }
}

// Raster CTA: one 16x16 tile, 128 threads in 4 warps; each warp owns an 8x8
// pixel square and each thread two vertically adjacent pixels of it.  The
// warps are independent: each walks the tile's list 32 splats at a time,
// lane l staging splat l of the batch in the warp's slice of shared memory
// together with the test of its alpha >= 1/255 ellipse against the warp's
// square (splat_hits); a ballot of that test is the warp's work list, taken
// in list order, so results are those of visiting every splat.  Pixels are
// evaluated with predicated, branch-free updates; a warp stops when its
// pixels are saturated (forward) and starts at the largest n_last of its
// pixels (backward), without waiting for the other warps.  A backward CTA
// takes one unit: a whole tile, or one list segment of a split tile.
constexpr int R_PPT = 2;                     // backward: pixels per thread
constexpr int R_THREADS = TILE_PIX / R_PPT;  // 128
constexpr int R_WARPS = R_THREADS / 32;
// Forward: one pixel per thread, 8 warps of 8 x 4 pixels.  The forward's
// time is set by its longest warps (the tiles whose lists saturate last);
// half the pixels per thread halves a warp's work per splat, and the smaller
// square passes fewer splats.  The backward keeps two pixels per thread: its
// per-splat warp reduction is then shared by 64 pixels.
constexpr int F_PPT = 1;
constexpr int F_THREADS = TILE_PIX / F_PPT;  // 256

struct WarpPix {
  int px, py0;     // this thread's column and first row
  int lx, ly0;     // the same inside the tile (checkpoint index (ly0 + k) * TILE + lx)
  float wx0, wy0;  // the warp square's first column and row
  float wh;        // its height - 1 (its width is 8)
};
// Warp w of a tile owns the 8-column square at columns (w & 1) * 8 and rows
// (w >> 1) * 4 PPT .. + 4 PPT - 1; lane l its column l & 7 and rows
// (l >> 3) * PPT .. + PPT - 1.
template <int PPT>
__device__ __forceinline__ WarpPix warp_pixels(int tile, int TX) {
  constexpr int RH = 4 * PPT;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  WarpPix q;
  const int tx0 = (tile % TX) * TILE, ty0 = (tile / TX) * TILE;
  const int sx = (w & 1) * 8, sy = (w >> 1) * RH;
  q.lx = sx + (l & 7);
  q.ly0 = sy + (l >> 3) * PPT;
  q.px = tx0 + q.lx;
  q.py0 = ty0 + q.ly0;
  q.wx0 = (float)(tx0 + sx);
  q.wy0 = (float)(ty0 + sy);
  q.wh = (float)(RH - 1);
  return q;
}

// The region where a splat's alpha reaches 1/255 meets the warp's square:
// alpha >= 1/255 iff qf(d) = A dx^2 + 2 B dx dy + C dy^2 <= 2 ln(255 o), and
// the minimum of that convex quadratic over the square [wx0, wx0 + 7] x
// [wy0, wy0 + 7] (offsets from the centre) is 0 if the centre lies inside,
// else the least of its four edge minima (a clamped 1-D minimum each).  The
// bound is widened (relative 2e-3, absolute 1e-3) so that no pixel the
// compositing would take is ever skipped.
__device__ __forceinline__ float edge_min_x(float a, float lo, float hi, float A, float B, float C) {
  // min over dy in [lo, hi] of A a^2 + 2 B a dy + C dy^2
  const float dy = fminf(fmaxf(-B * a / C, lo), hi);
  return A * a * a + 2.f * B * a * dy + C * dy * dy;
}
__device__ __forceinline__ float edge_min_y(float b, float lo, float hi, float A, float B, float C) {
  const float dx = fminf(fmaxf(-B * b / A, lo), hi);
  return A * dx * dx + 2.f * B * dx * b + C * b * b;
}
__device__ __forceinline__ bool splat_hits(const WarpPix& q, float x, float y, float A, float B, float C, float o) {
  const float L = logf(255.f * o);
  if (!(L > 0.f)) return false;
  const float ax0 = q.wx0 - x, ax1 = ax0 + 7.f, by0 = q.wy0 - y, by1 = by0 + q.wh;
  if (ax0 <= 0.f && ax1 >= 0.f && by0 <= 0.f && by1 >= 0.f) return true;
  float m = edge_min_x(ax0, by0, by1, A, B, C);
  m = fminf(m, edge_min_x(ax1, by0, by1, A, B, C));
  m = fminf(m, edge_min_y(by0, ax0, ax1, A, B, C));
  m = fminf(m, edge_min_y(by1, ax0, ax1, A, B, C));
  return m <= 2.004f * L + 1e-3f;
}

// One splat as staged in shared memory, with the conic folded into the
// power's coefficients in base 2: power2 = power log2(e) = dx (a2 dx + b2 dy)
// + c2 dy^2 with a2 = -A log2(e)/2, b2 = -B log2(e), c2 = -C log2(e)/2,
// evaluated as
//   power2 = fma(dx, fma(b2, dy, a2 dx), c2 (dy dy)),  G = 2^power2
// by the forward and the backward alike, so both take the same alphas (the
// power's sign tests are unchanged by the positive scale).
struct Splat {
  float4 a;  // x, y, a2, b2
  float4 b;  // c2, opacity, r, g
  float c;   // b
  uint32_t id;
};

constexpr float LOG2E = 1.4426950408889634f;
constexpr float LN2 = 0.6931471805599453f;
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// alpha = min(0.99, o G), G = 2^power2 (the base-2 power of the staged splat)
__device__ __forceinline__ float splat_alpha2(float opac, float power2, float& G) {
  G = ex2_approx(power2);
  return fminf(ALPHA_MAX, __fmul_rn(opac, G));
}
__device__ __forceinline__ float splat_power(float a2dx, float b2, float c2, float dx, float dy, float dyy) {
  return __fmaf_rn(dx, __fmaf_rn(b2, dy, a2dx), __fmul_rn(c2, dyy));
}

__device__ __forceinline__ bool stage_splat(const uint32_t* __restrict__ pvals, const float2* __restrict__ xy,
                                            const float4* __restrict__ conic_o, const float4* __restrict__ rgb,
                                            uint32_t pos, const WarpPix& q, Splat* slot) {
  const uint32_t id = pvals[pos];
  const float2 g = xy[id];
  const float4 co = conic_o[id];
  const float4 cc = rgb[id];
  slot->a = make_float4(g.x, g.y, -0.5f * LOG2E * co.x, -LOG2E * co.y);
  slot->b = make_float4(-0.5f * LOG2E * co.z, co.w, cc.x, cc.y);
  slot->c = cc.z;
  slot->id = id;
  return splat_hits(q, g.x, g.y, co.x, co.y, co.z, co.w);
}

template <int PPT>
__global__ void __launch_bounds__(TILE_PIX / PPT) k_raster_fwd(const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ pvals,
                                                         const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_o,
                                                         const float4* __restrict__ rgb, int W, int H, int TX,
                                                         float3 bg, float* __restrict__ img,
                                                         float* __restrict__ t_final, int* __restrict__ n_last,
                                                         const uint32_t* __restrict__ order,
                                                         const uint32_t* __restrict__ tck,
                                                         float4* __restrict__ ck) {
  __shared__ Splat s_sp[TILE_PIX / PPT / 32][32];
  const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
  const WarpPix q = warp_pixels<PPT>(tile, TX);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Splat* sp = s_sp[wid];
  const uint2 r = ranges[tile];
  const int n = (int)(r.y - r.x);
  // checkpoints of a split tile (the backward work split): slot ck0 + i - 1
  // holds the state before list position i R_SEG, slot ck0 + ns - 1 the final
  const uint32_t ck0 = tck ? tck[tile] : ~0u;
  const int ns = (int)seg_count((uint32_t)n);
  const float fpx = (float)q.px;
  float T[PPT], C0[PPT], C1[PPT], C2[PPT];
  int last[PPT];
  bool live[PPT];
  bool act = false;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = 1.f;
    C0[k] = C1[k] = C2[k] = 0.f;
    last[k] = 0;
    live[k] = q.px < W && q.py0 + k < H;
    act |= live[k];
  }
  bool going = __any_sync(0xffffffffu, act);
  int wrote = 0;  // boundary slots written (slot i - 1: the state before position i R_SEG)
  for (int b = 0; b < n && going; b += 32) {
    if (ck0 != ~0u && b > 0 && b % R_SEG == 0 && b / R_SEG < ns) {
      float4* c = ck + (uint64_t)(ck0 + b / R_SEG - 1) * TILE_PIX + q.lx;
#pragma unroll
      for (int k = 0; k < PPT; ++k) c[(q.ly0 + k) * TILE] = make_float4(T[k], C0[k], C1[k], C2[k]);
      wrote = b / R_SEG;
    }
    const bool hit = b + lane < n && stage_splat(pvals, xy, conic_o, rgb, r.x + b + lane, q, &sp[lane]);
    __syncwarp();
    uint32_t bal = __ballot_sync(0xffffffffu, hit);
    while (bal) {
      const int j = __ffs(bal) - 1;
      bal &= bal - 1;
      const float4 a = sp[j].a;
      const float4 bb = sp[j].b;
      const float cb = sp[j].c;
      act = false;
      // the thread's pixels share their column: dx and a2 dx once
      const float dx = __fsub_rn(fpx, a.x);
      const float a2dx = __fmul_rn(a.z, dx);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        const float dy = __fsub_rn((float)(q.py0 + k), a.y);
        const float power = splat_power(a2dx, a.w, bb.x, dx, dy, __fmul_rn(dy, dy));
        float G;
        const float alpha = splat_alpha2(bb.y, power, G);
        const float Tn = __fmul_rn(T[k], __fsub_rn(1.f, alpha));
        const bool ok = live[k] && power <= 0.f && alpha >= ALPHA_MIN;
        const bool stop = ok && Tn < T_STOP;
        const bool take = ok && !stop;
        live[k] = live[k] && !stop;
        const float w = take ? alpha * T[k] : 0.f;
        C0[k] += bb.z * w;
        C1[k] += bb.w * w;
        C2[k] += cb * w;
        T[k] = take ? Tn : T[k];
        last[k] = take ? b + j + 1 : last[k];
        act |= live[k];
      }
      if (!__any_sync(0xffffffffu, act)) {
        going = false;
        break;
      }
    }
    __syncwarp();  // the batch slots are rewritten next
  }
  if (ck0 != ~0u) {
    // a warp that saturated early holds its final state at every boundary it
    // did not reach: the backward's squares need not be this warp's, and a
    // backward warp reads the boundary states of all its pixels
    for (int i = wrote; i < ns; ++i) {
      float4* c = ck + (uint64_t)(ck0 + i) * TILE_PIX + q.lx;
#pragma unroll
      for (int k = 0; k < PPT; ++k) c[(q.ly0 + k) * TILE] = make_float4(T[k], C0[k], C1[k], C2[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int py = q.py0 + k;
    if (q.px < W && py < H) {
      uint64_t pix = (uint64_t)py * W + q.px;
      img[3 * pix + 0] = C0[k] + T[k] * bg.x;
      img[3 * pix + 1] = C1[k] + T[k] * bg.y;
      img[3 * pix + 2] = C2[k] + T[k] * bg.z;
      t_final[pix] = T[k];
      n_last[pix] = last[k];
    }
  }
}

// Backward partials: a warp's per-lane sums for a splat wait in shared
// memory until RB_SLOTS splats are pending; then lane r adds up row r (the 32
// lanes' values of one field of one splat) and adds the field's gradient with
// one atomic.  Rows are padded to RB_ROW floats so that the 16-byte reads of
// eight lanes fall in distinct bank groups.
constexpr int RB_SLOTS = 3;  // 27 rows: one row per lane
constexpr int RB_ROW = 36;

// Sums the rows of nslot pending splats and adds their 2D gradients: fields
// u, v (A sx + B sy and B sx + C sy of the geometric sums), the conic
// (-1/2, -1, -1/2 times the second moments), opacity and colour.
__device__ __forceinline__ void flush_partials(float (*red)[RB_ROW], const float4* rinfo, int nslot, int lane,
                                               float* __restrict__ g2, uint64_t V) {
  __syncwarp();  // every lane's row entries are written
  const bool mine = lane < 9 * nslot;
  float s = 0.f;
  if (mine) {
    const float4* r4 = reinterpret_cast<const float4*>(red[lane]);
    float4 x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = r4[i];
#pragma unroll
    for (int w = 4; w > 0; w >>= 1)
#pragma unroll
      for (int i = 0; i < w; ++i) {
        x[i].x += x[i + w].x;
        x[i].y += x[i + w].y;
        x[i].z += x[i + w].z;
        x[i].w += x[i + w].w;
      }
    s = (x[0].x + x[0].y) + (x[0].z + x[0].w);
  }
  // the position fields combine the two first-moment sums of their splat
  const float up = __shfl_down_sync(0xffffffffu, s, 1);
  const float dn = __shfl_up_sync(0xffffffffu, s, 1);
  if (mine) {
    const int slot = lane / 9, f = lane - 9 * slot;
    const float4 in = rinfo[slot];  // A, B, C, Gaussian id
    float fin;
    if (f == 0)
      fin = in.x * s + in.y * up;
    else if (f == 1)
      fin = in.z * s + in.y * dn;
    else if (f == 3)
      fin = -s;
    else if (f == 2 || f == 4)
      fin = -0.5f * s;
    else
      fin = s;
    if (fin != 0.f) atomicAdd(&g2[(uint64_t)f * V + __float_as_uint(in.w)], fin);
  }
  __syncwarp();  // the rows are rewritten after the flush
}

__global__ void __launch_bounds__(R_THREADS) k_raster_bwd(const uint2* __restrict__ ranges,
                                                         const uint32_t* __restrict__ pvals,
                                                         const float2* __restrict__ xy,
                                                         const float4* __restrict__ conic_o,
                                                         const float4* __restrict__ rgb, int W, int H, int TX,
                                                         float3 bg, const float* __restrict__ t_final,
                                                         const int* __restrict__ n_last,
                                                         const float* __restrict__ dl_dimg, float* __restrict__ g2,
                                                         uint64_t V, const uint32_t* __restrict__ units,
                                                         const uint32_t* __restrict__ n_units,
                                                         const uint32_t* __restrict__ tck,
                                                         const float4* __restrict__ ck) {
  __shared__ Splat s_sp[R_WARPS][32];
  __shared__ __align__(16) float s_red[R_WARPS][9 * RB_SLOTS][RB_ROW];
  __shared__ float4 s_rinfo[R_WARPS][RB_SLOTS];
  // the CTA's unit: one tile, or one list segment [b0, b1) of a split tile
  int tile = (int)blockIdx.x, seg = 0;
  if (units) {
    if (blockIdx.x >= *n_units) return;  // uniform per CTA
    const uint32_t u = units[blockIdx.x];
    tile = (int)(u & 0xFFFFFFu);
    seg = (int)(u >> 24);
  }
  const WarpPix q = warp_pixels<R_PPT>(tile, TX);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Splat* sp = s_sp[wid];
  const uint2 r = ranges[tile];
  const float fpx = (float)q.px;
  const uint32_t ck0 = units ? tck[tile] : ~0u;
  const int ns = (int)seg_count(r.y - r.x);
  int b0 = 0, b1 = 0x7fffffff;
  if (ck0 != ~0u) {
    b0 = seg * R_SEG;
    if (seg + 1 < ns) b1 = (seg + 1) * R_SEG;
  }
  // Qs = sum_c dL/dC_c S_c, S_c the colour composited behind the current
  // splat (only this combination enters dL/dalpha)
  float T[R_PPT], gr[R_PPT], gg[R_PPT], gb[R_PPT], Qs[R_PPT], tfb[R_PPT];
  int last[R_PPT];
  int mylast = 0;
#pragma unroll
  for (int k = 0; k < R_PPT; ++k) {
    const int py = q.py0 + k;
    T[k] = 1.f;
    last[k] = 0;
    gr[k] = gg[k] = gb[k] = 0.f;
    Qs[k] = 0.f;
    if (q.px < W && py < H) {
      const uint64_t pix = (uint64_t)py * W + q.px;
      T[k] = t_final[pix];
      last[k] = n_last[pix];
      gr[k] = dl_dimg[3 * pix + 0];
      gg[k] = dl_dimg[3 * pix + 1];
      gb[k] = dl_dimg[3 * pix + 2];
    }
    tfb[k] = T[k] * (bg.x * gr[k] + bg.y * gg[k] + bg.z * gb[k]);
    mylast = max(mylast, last[k]);
  }
  // list positions >= the warp's largest n_last contribute to none of its pixels
  int wlast = mylast;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wlast = max(wlast, __shfl_xor_sync(0xffffffffu, wlast, o));
  if (wlast <= b0) return;  // nothing of this segment reaches the warp's pixels (no CTA barrier follows)
  if (wlast > b1) {
    // the segment lies below the warp's last contribution: start from the
    // forward's state at b1, T = T(b1) and S_c = (C_c final - C_c(b1)) / T(b1)
    const float4* cf = ck + (uint64_t)(ck0 + ns - 1) * TILE_PIX + q.lx;
    const float4* c1 = ck + (uint64_t)(ck0 + seg) * TILE_PIX + q.lx;
#pragma unroll
    for (int k = 0; k < R_PPT; ++k) {
      const float4 f = cf[(q.ly0 + k) * TILE], a = c1[(q.ly0 + k) * TILE];
      T[k] = a.x;
      Qs[k] = (gr[k] * (f.y - a.y) + gg[k] * (f.z - a.z) + gb[k] * (f.w - a.w)) / a.x;
    }
    wlast = b1;
  }
  // the lane-wise partials of up to RB_SLOTS contributing splats wait in
  // shared memory (row 9 s + f of slot s, field f); a flush sums each row
  // (lane r sums row r) and adds it with one atomic
  float(*red)[RB_ROW] = s_red[wid];
  float4* rinfo = s_rinfo[wid];
  int nslot = 0;
  for (int top = wlast; top > b0; top -= 32) {
    // lane l stages list position top - 1 - l: ascending lanes, descending positions
    const int k0 = top - 1 - lane;
    const bool hit = k0 >= b0 && stage_splat(pvals, xy, conic_o, rgb, r.x + (uint32_t)k0, q, &sp[lane]);
    __syncwarp();
    uint32_t bal = __ballot_sync(0xffffffffu, hit);
    while (bal) {
      const int j = __ffs(bal) - 1;
      bal &= bal - 1;
      const int pos = top - 1 - j;
      const float4 a = sp[j].a;
      const float4 bb = sp[j].b;
      const float cb = sp[j].c;
      // sums over the thread's pixels (one column: dx is shared) of dpw,
      // dpw dy and dpw dy^2 (dpw = dL/dpower), from which the five geometric
      // sums dpw dx, dpw dy, dpw dx^2, dpw dx dy, dpw dy^2 follow (the conic
      // and constant factors are applied after the reduction); v: the
      // dL/dopacity-activation and dL/d(r, g, b) sums
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      bool contrib = false;
      const float dx = __fsub_rn(fpx, a.x);
      const float dxx = __fmul_rn(dx, dx);
      const float a2dx = __fmul_rn(a.z, dx);
#pragma unroll
      for (int k = 0; k < R_PPT; ++k) {
        const float dy = __fsub_rn((float)(q.py0 + k), a.y);
        const float dyy = __fmul_rn(dy, dy);
        const float power = splat_power(a2dx, a.w, bb.x, dx, dy, dyy);
        float G;
        const float alpha = splat_alpha2(bb.y, power, G);
        const bool ok = pos < last[k] && power <= 0.f && alpha >= ALPHA_MIN;
        contrib |= ok;
        const float al = ok ? alpha : 0.f;
        const float oma = 1.f - al;
        const float ioma = __fdividef(1.f, oma);  // no decision depends on T here
        const float Ti = T[k] * ioma;
        const float w = al * Ti;
        v[6] += w * gr[k];
        v[7] += w * gg[k];
        v[8] += w * gb[k];
        const float pc = gr[k] * bb.z + gg[k] * bb.w + gb[k] * cb;
        const float dal = Ti * (pc - Qs[k]) - tfb[k] * ioma;
        Qs[k] = al * pc + oma * Qs[k];
        T[k] = Ti;
        const float dsel = (ok && __fmul_rn(bb.y, G) <= ALPHA_MAX) ? dal : 0.f;
        v[5] += G * dsel;
        const float dpw = al * dsel;
        s0 += dpw;
        s1 += dpw * dy;
        s2 += dpw * dyy;
      }
      if (__ballot_sync(0xffffffffu, contrib)) {
        v[0] = dx * s0;
        v[1] = s1;
        v[2] = dxx * s0;
        v[3] = dx * s1;
        v[4] = s2;
#pragma unroll
        for (int f = 0; f < 9; ++f) red[9 * nslot + f][lane] = v[f];
        // the conic (A, B, C) back from the staged base-2 coefficients
        if (lane == 0)
          rinfo[nslot] = make_float4(-2.f * LN2 * a.z, -LN2 * a.w, -2.f * LN2 * bb.x, __uint_as_float(sp[j].id));
        if (++nslot == RB_SLOTS) {
          flush_partials(red, rinfo, nslot, lane, g2, V);
          nslot = 0;
        }
      }
    }
    __syncwarp();  // the batch slots are rewritten next
  }
  if (nslot) flush_partials(red, rinfo, nslot, lane, g2, V);
}

// Chain rule of the Level-2 preprocess (exact derivative of k_preprocess)
// from the 2D gradients of one Gaussian (u, v, A, B, C, opacity, r, g, b) to
// its 59 parameters, accumulated into g[] (kept in registers when unrolled).
template <bool BF>
__device__ __forceinline__ void chain_rule(const DevCam& c, const float* __restrict__ p,
                                           const __nv_bfloat16* __restrict__ q16, uint32_t B,
                                           const float gv2[9], uint32_t clampbits, float opac, float gr[D]) {
  const float gu = gv2[0], gv = gv2[1], gA = gv2[2], gB = gv2[3], gC = gv2[4];
  const float gop = gv2[5];
  const float gcol[3] = {gv2[6], gv2[7], gv2[8]};
  const float mx = p[0], my = p[B], mz = p[2 * B];
  float dmu[3] = {0.f, 0.f, 0.f};
  // ---- colour ----
  {
    float dx = mx - c.campos[0], dy = my - c.campos[1], dz = mz - c.campos[2];
    float len = sqrtf(dx * dx + dy * dy + dz * dz);
    float il = 1.f / len;
    float d[3] = {dx * il, dy * il, dz * il};
    float Y[16];
    sh_eval(d[0], d[1], d[2], Y);
    float Gs[16][3];
    sh_grad(d[0], d[1], d[2], Gs);
    uint32_t cl = clampbits;
    float gc[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) gc[ch] = (cl >> ch) & 1u ? 0.f : gcol[ch];
    float dd[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        uint64_t f = 11 + 3 * kk + ch;
        gr[f] += Y[kk] * gc[ch];
        float shv = ldp<BF>(p, q16, B, (int)f);
        float w = gc[ch] * shv;
        dd[0] += w * Gs[kk][0];
        dd[1] += w * Gs[kk][1];
        dd[2] += w * Gs[kk][2];
      }
    }
    float dot = dd[0] * d[0] + dd[1] * d[1] + dd[2] * d[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) dmu[a] += (dd[a] - d[a] * dot) * il;
  }
  // ---- opacity ----
  {
    float op = opac;
    gr[10] += gop * op * (1.f - op);
  }
  // ---- geometry ----
  KeyPath k = key_path(c, mx, my, mz);
  Geo g;
  geometry(c, p, B, k, g);
  const float tz = k.tz;
  const float idet = 1.f / g.det;
  const float id2 = idet * idet;
  const float dla = (-g.c * g.c * gA + g.b * g.c * gB - g.b * g.b * gC) * id2;
  const float dlc = (-g.b * g.b * gA + g.a * g.b * gB - g.a * g.a * gC) * id2;
  const float dlb = (2.f * g.b * g.c * gA - (g.a * g.c + g.b * g.b) * gB + 2.f * g.a * g.b * gC) * id2;
  const float Gc[2][2] = {{dla, 0.5f * dlb}, {0.5f * dlb, dlc}};
  float GT[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) GT[a][b] = Gc[a][0] * g.T[0][b] + Gc[a][1] * g.T[1][b];
  // dL/dSigma = T^T Gc T (symmetric)
  float dS[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) dS[a][b] = g.T[0][a] * GT[0][b] + g.T[1][a] * GT[1][b];
  const float Sg[3][3] = {{g.S[0], g.S[1], g.S[2]}, {g.S[1], g.S[3], g.S[4]}, {g.S[2], g.S[4], g.S[5]}};
  // dL/dT = 2 Gc T Sigma, dL/dJ = dL/dT Rc^T
  float dT[2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) dT[a][b] = 2.f * (GT[a][0] * Sg[0][b] + GT[a][1] * Sg[1][b] + GT[a][2] * Sg[2][b]);
  float dJ00 = dT[0][0] * c.R[0] + dT[0][1] * c.R[1] + dT[0][2] * c.R[2];
  float dJ02 = dT[0][0] * c.R[6] + dT[0][1] * c.R[7] + dT[0][2] * c.R[8];
  float dJ11 = dT[1][0] * c.R[3] + dT[1][1] * c.R[4] + dT[1][2] * c.R[5];
  float dJ12 = dT[1][0] * c.R[6] + dT[1][1] * c.R[7] + dT[1][2] * c.R[8];
  float tz2 = tz * tz, tz3 = tz2 * tz;
  float dt[3] = {0.f, 0.f, 0.f};
  dt[2] += -c.fx / tz2 * dJ00 - c.fy / tz2 * dJ11;
  if (!g.clx) {
    dt[0] += -c.fx / tz2 * dJ02;
    dt[2] += 2.f * c.fx * k.tx / tz3 * dJ02;
  } else {
    dt[2] += c.fx * g.xc / tz2 * dJ02;
  }
  if (!g.cly) {
    dt[1] += -c.fy / tz2 * dJ12;
    dt[2] += 2.f * c.fy * k.ty / tz3 * dJ12;
  } else {
    dt[2] += c.fy * g.yc / tz2 * dJ12;
  }
  dt[0] += gu * c.fx / tz;
  dt[1] += gv * c.fy / tz;
  dt[2] += -gu * c.fx * k.tx / tz2 - gv * c.fy * k.ty / tz2;
#pragma unroll
  for (int a = 0; a < 3; ++a) dmu[a] += c.R[a] * dt[0] + c.R[3 + a] * dt[1] + c.R[6 + a] * dt[2];
  gr[0] += dmu[0];
  gr[1] += dmu[1];
  gr[2] += dmu[2];
  // Sigma = M M^T, M = Rq diag(sc)
  float M[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) M[a][b] = g.Rq[a][b] * g.sc[b];
  float dR[3][3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    float dsb = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float dM = 2.f * (dS[a][0] * M[0][b] + dS[a][1] * M[1][b] + dS[a][2] * M[2][b]);
      dsb += dM * g.Rq[a][b];
      dR[a][b] = dM * g.sc[b];
    }
    gr[3 + b] += dsb * g.sc[b];
  }
  const float w = g.qw, x = g.qx, y = g.qy, z = g.qz;
  float gw = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
  float gx = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                    z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
  float gy = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                    w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
  float gz = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                    y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
  float qd = gw * w + gx * x + gy * y + gz * z;
  float iq = 1.f / g.qn;
  gr[6] += (gw - w * qd) * iq;
  gr[7] += (gx - x * qd) * iq;
  gr[8] += (gy - y * qd) * iq;
  gr[9] += (gz - z * qd) * iq;
}

// mode 0: store the gradient of every valid render-list position (zero for
// Gaussians without a tile rect) into a local [59][V] array;
// mode 1: add the gradient of visible Gaussians to that array;
// mode 2: add into a pool with the render list's slot layout.
template <bool BF>
__device__ __forceinline__ void pbwd_row(const RenderList& rl, const DevCam& c, const uint32_t* __restrict__ ntiles,
                                         const float4* __restrict__ rgbv, const float4* __restrict__ conic_o,
                                         const float* __restrict__ g2, uint64_t V, float* __restrict__ grad,
                                         uint64_t Vg, int mode, unsigned item, unsigned lane, uint64_t i,
                                         bool listed) {
  const uint32_t B = rl.B;
  const bool vis = ntiles[i] != 0;
  // mode 0 stores the rows the optimiser reads (the listed rows, touched by
  // the batch), zero where this camera does not see the Gaussian
  if (!vis && (mode != 0 || !listed)) return;
  const uint64_t sbase = (uint64_t)rl.item_slot[item] * rl.slot_stride + lane;
  const float* p = rl.base + sbase;
  const __nv_bfloat16* q16 = sh16(rl.base + (uint64_t)rl.item_slot[item] * rl.slot_stride, B, lane);
  float* out = mode == 2 ? grad + sbase : grad + i;
  const uint64_t ostride = mode == 2 ? B : Vg;
  float g[D];
#pragma unroll
  for (int f = 0; f < D; ++f) g[f] = 0.f;
  if (vis) {
    float gv2[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) gv2[q] = g2[(uint64_t)q * V + i];
    chain_rule<BF>(c, p, q16, B, gv2, __float_as_uint(rgbv[i].w), conic_o[i].w, g);
  }
  if (mode == 0) {
#pragma unroll
    for (int f = 0; f < D; ++f) out[(uint64_t)f * ostride] = g[f];
  } else {
#pragma unroll
    for (int f = 0; f < D; ++f) out[(uint64_t)f * ostride] += g[f];
  }
}

// Every render-list position (rows == null; mode 0 then stores every valid
// row) or the listed rows (grid-stride over *nrows).
template <bool BF>
__global__ void __launch_bounds__(PP_THREADS) k_preprocess_bwd(RenderList rl, DevCam c,
                                                              const uint32_t* __restrict__ ntiles,
                                                              const float4* __restrict__ rgbv,
                                                              const float4* __restrict__ conic_o,
                                                              const float* __restrict__ g2, uint64_t V,
                                                              float* __restrict__ grad, uint64_t Vg, int mode,
                                                              unsigned cpi, const uint32_t* __restrict__ rows,
                                                              const uint32_t* __restrict__ nrows) {
  const uint32_t B = rl.B;
  if (rows) {
    const uint32_t n = *nrows;
    for (uint32_t t = blockIdx.x * PP_THREADS + threadIdx.x; t < n; t += gridDim.x * PP_THREADS) {
      const uint32_t i = rows[t];
      const unsigned item = item_of(i, B), lane = i - item * B;
      pbwd_row<BF>(rl, c, ntiles, rgbv, conic_o, g2, V, grad, Vg, mode, item, lane, i, true);
    }
    return;
  }
  const unsigned item = blockIdx.x / cpi;
  const unsigned lane = (blockIdx.x - item * cpi) * PP_THREADS + threadIdx.x;
  if (lane >= B) return;
  const uint64_t i = (uint64_t)item * B + lane;
  if (lane >= rl.item_count[item]) return;
  pbwd_row<BF>(rl, c, ntiles, rgbv, conic_o, g2, V, grad, Vg, mode, item, lane, i, true);
}

// The chain rule of a whole batch in one pass over the listed rows: each row's
// parameters are read once, the gradients of the cameras that see it are
// summed in registers and stored once.
template <bool BF>
__global__ void __launch_bounds__(PP_THREADS, 2) k_preprocess_bwd_batch(RenderList rl, BatchGrad bg,
                                                                    float* __restrict__ grad, uint64_t Vg,
                                                                    const uint32_t* __restrict__ rows,
                                                                    const uint32_t* __restrict__ nrows) {
  const uint32_t B = rl.B;
  const uint32_t n = *nrows;
  for (uint32_t t = blockIdx.x * PP_THREADS + threadIdx.x; t < n; t += gridDim.x * PP_THREADS) {
    const uint32_t i = rows[t];
    const unsigned item = item_of(i, B), lane = i - item * B;
    const uint64_t sbase = (uint64_t)rl.item_slot[item] * rl.slot_stride + lane;
    const float* p = rl.base + sbase;
    const __nv_bfloat16* q16 = sh16(rl.base + (uint64_t)rl.item_slot[item] * rl.slot_stride, B, lane);
    float g[D];
#pragma unroll
    for (int f = 0; f < D; ++f) g[f] = 0.f;
    for (int j = 0; j < bg.J; ++j) {
      if (bg.ntiles[j][i] == 0) continue;
      float gv2[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) gv2[q] = bg.g2[j][(uint64_t)q * bg.stride[j] + i];
      chain_rule<BF>(bg.cam[j], p, q16, B, gv2, __float_as_uint(bg.rgb[j][i].w), bg.conic[j][i].w, g);
    }
#pragma unroll
    for (int f = 0; f < D; ++f) grad[(uint64_t)f * Vg + i] = g[f];
  }
}

// The render-list positions with touched != 0: one warp per 128 positions
// (4 per lane), a warp scan of the counts and one atomic per warp, so each
// group's rows are written in ascending order (groups in any order).
__global__ void k_touched_rows(const uint8_t* __restrict__ touched, uint64_t V, uint32_t* __restrict__ rows,
                               uint32_t* __restrict__ count, uint32_t* __restrict__ prows,
                               uint32_t* __restrict__ pcount) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t g0 = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 128; g0 < V;
       g0 += warps * 128) {
    const uint64_t p0 = g0 + 4 * (uint64_t)lane;
    uint32_t f = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (p0 + e < V && touched[p0 + e]) f |= 1u << e;
    const uint32_t c = __popc(f);
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    uint32_t base = 0;
    if (lane == 0 && total) base = atomicAdd(count, total);
    base = __shfl_sync(0xffffffffu, base, 0) + inc - c;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (f >> e & 1u) rows[base++] = (uint32_t)(p0 + e);
    if (prows) {
      // pairs (p0, p0 + 1) and (p0 + 2, p0 + 3) with a touched member:
      // position | member mask << 30
      const uint32_t ma = f & 3u, mb = (f >> 2) & 3u;
      const uint32_t pc = (ma ? 1u : 0u) + (mb ? 1u : 0u);
      uint32_t pinc = pc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, pinc, o);
        if (lane >= o) pinc += y;
      }
      const uint32_t ptot = __shfl_sync(0xffffffffu, pinc, 31);
      uint32_t pb = 0;
      if (lane == 0 && ptot) pb = atomicAdd(pcount, ptot);
      pb = __shfl_sync(0xffffffffu, pb, 0) + pinc - pc;
      if (ma) prows[pb++] = (uint32_t)p0 | (ma << 30);
      if (mb) prows[pb++] = (uint32_t)(p0 + 2) | (mb << 30);
    }
  }
}

// sqrt(x) for Adam's denominator from the fast reciprocal square root
// (relative error about 1e-7; x >= 0)
__device__ __forceinline__ float adam_sqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
// The parameter's 16 rounding bits: a second finaliser of the field's 32-bit
// draw h (whose two halves round m and v).
__device__ __forceinline__ uint32_t param_draw(uint32_t h) { return fmix32(h ^ 0x27D4EB2Fu); }

constexpr int ADAM_FG = 4;  // fields per thread
constexpr int ADAM_GROUPS = (D + ADAM_FG - 1) / ADAM_FG;

// One Gaussian's ADAM_FG fields f0.. of Adam: every load of the fields (the
// gradient, both moments and the parameter) is issued before the first
// update, so a thread keeps 4 ADAM_FG independent loads in flight; then the
// updates and stores.  BF16 record: moments and SH-rest parameters are read
// as BF16 and stored rounded (stochastically with one counter hash per
// field: three 16-bit draws for m, v and the parameter).
template <bool BF>
__device__ __forceinline__ void adam_row(const RenderList& rl, const float* __restrict__ grad,
                                         const float2* __restrict__ bias, const uint32_t* __restrict__ block_step,
                                         uint64_t V, const LrSet& lrs, float b1, float b2, float eps, unsigned item,
                                         unsigned lane, uint64_t i, int f0) {
  const uint32_t B = rl.B;
  const float2 bc = bias[item];
  const float ic1 = bc.x, ic2 = bc.y;
  float* __restrict__ slot = rl.base + (uint64_t)rl.item_slot[item] * rl.slot_stride;
  float* __restrict__ p = slot + lane;
  float gf[ADAM_FG], mf[ADAM_FG], vf[ADAM_FG], pf[ADAM_FG];
  if (!BF) {
    float* __restrict__ m = p + rl.m_off;
    float* __restrict__ v = p + rl.v_off;
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o = (uint64_t)f * B;
        gf[q] = __ldg(grad + (uint64_t)f * V + i);
        mf[q] = m[o];
        vf[q] = v[o];
        pf[q] = p[o];
      }
    }
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o = (uint64_t)f * B;
        const float mn = b1 * mf[q] + (1.f - b1) * gf[q];
        const float vn = b2 * vf[q] + (1.f - b2) * gf[q] * gf[q];
        m[o] = mn;
        v[o] = vn;
        p[o] = pf[q] - lrs.g[lr_group(f)] * __fdividef(mn * ic1, adam_sqrt(vn * ic2) + eps);
      }
    }
  } else {
    __nv_bfloat16* __restrict__ q16 = reinterpret_cast<__nv_bfloat16*>(slot + (uint64_t)F_BF16 * B) + lane;
    __nv_bfloat16* __restrict__ m = reinterpret_cast<__nv_bfloat16*>(slot + rl.m_off) + lane;
    __nv_bfloat16* __restrict__ v = reinterpret_cast<__nv_bfloat16*>(slot + rl.v_off) + lane;
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o = (uint64_t)f * B;
        gf[q] = __ldg(grad + (uint64_t)f * V + i);
        mf[q] = __bfloat162float(m[o]);
        vf[q] = __bfloat162float(v[o]);
        pf[q] = f < F_BF16 ? p[o] : __bfloat162float(q16[(uint64_t)(f - F_BF16) * B]);
      }
    }
    const bool sr = rl.sr != 0;
    const uint32_t blk = rl.item_block[item];
    const uint32_t key = sr ? sr_key(rl.seed, (uint64_t)blk * B + lane, block_step[blk]) : 0u;
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o = (uint64_t)f * B;
        const float mn = b1 * mf[q] + (1.f - b1) * gf[q];
        const float vn = b2 * vf[q] + (1.f - b2) * gf[q] * gf[q];
        const float upd = lrs.g[lr_group(f)] * __fdividef(mn * ic1, adam_sqrt(vn * ic2) + eps);
        const uint32_t h = sr ? fmix32(key + (uint32_t)f * 0x9E3779B9u) : 0u;
        m[o] = to_bf16(mn, sr, h);
        v[o] = to_bf16(vn, sr, h >> 16);
        if (f < F_BF16)
          p[o] = pf[q] - upd;
        else
          q16[(uint64_t)(f - F_BF16) * B] = to_bf16(pf[q] - upd, sr, param_draw(h));
      }
    }
  }
}

// Masked Adam on a pair of adjacent Gaussians (lanes l, l + 1 of one block,
// l even; B even so a pair never straddles blocks): 8-byte FP32 / 4-byte
// BF16 accesses for both, the item's slot, bias corrections and step counter
// read once.  A member outside the mask keeps its values (stored back
// unchanged).  Same arithmetic and rounding draws per Gaussian as adam_row.
template <bool BF>
__device__ __forceinline__ void adam_pair(const RenderList& rl, const float* __restrict__ grad,
                                          const float2* __restrict__ bias, const uint32_t* __restrict__ block_step,
                                          uint64_t V, const LrSet& lrs, float b1, float b2, float eps, unsigned item,
                                          unsigned lane, uint64_t i, uint32_t mask, int f0) {
  const uint32_t B = rl.B;
  const float2 bc = bias[item];
  const float ic1 = bc.x, ic2 = bc.y;
  float* __restrict__ slot = rl.base + (uint64_t)rl.item_slot[item] * rl.slot_stride;
  const bool t0 = mask & 1u, t1 = mask & 2u;
  float2 gf[ADAM_FG], mf[ADAM_FG], vf[ADAM_FG], pf[ADAM_FG];
  if (!BF) {
    float* __restrict__ p = slot + lane;
    float* __restrict__ m = p + rl.m_off;
    float* __restrict__ v = p + rl.v_off;
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o = (uint64_t)f * B;
        gf[q] = __ldg(reinterpret_cast<const float2*>(grad + (uint64_t)f * V + i));
        mf[q] = *reinterpret_cast<const float2*>(m + o);
        vf[q] = *reinterpret_cast<const float2*>(v + o);
        pf[q] = *reinterpret_cast<const float2*>(p + o);
      }
    }
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o = (uint64_t)f * B;
        const float lr = lrs.g[lr_group(f)];
        float2 mn, vn, pn;
        mn.x = b1 * mf[q].x + (1.f - b1) * gf[q].x;
        vn.x = b2 * vf[q].x + (1.f - b2) * gf[q].x * gf[q].x;
        pn.x = pf[q].x - lr * __fdividef(mn.x * ic1, adam_sqrt(vn.x * ic2) + eps);
        mn.y = b1 * mf[q].y + (1.f - b1) * gf[q].y;
        vn.y = b2 * vf[q].y + (1.f - b2) * gf[q].y * gf[q].y;
        pn.y = pf[q].y - lr * __fdividef(mn.y * ic1, adam_sqrt(vn.y * ic2) + eps);
        if (!t0) { mn.x = mf[q].x; vn.x = vf[q].x; pn.x = pf[q].x; }
        if (!t1) { mn.y = mf[q].y; vn.y = vf[q].y; pn.y = pf[q].y; }
        *reinterpret_cast<float2*>(m + o) = mn;
        *reinterpret_cast<float2*>(v + o) = vn;
        *reinterpret_cast<float2*>(p + o) = pn;
      }
    }
  } else {
    float* __restrict__ p = slot + lane;
    __nv_bfloat162* __restrict__ q16 =
        reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(slot + (uint64_t)F_BF16 * B) + lane);
    __nv_bfloat162* __restrict__ m =
        reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(slot + rl.m_off) + lane);
    __nv_bfloat162* __restrict__ v =
        reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<__nv_bfloat16*>(slot + rl.v_off) + lane);
    __nv_bfloat162 m16[ADAM_FG], v16[ADAM_FG], p16[ADAM_FG];
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o2 = (uint64_t)f * (B / 2);  // in pairs
        gf[q] = __ldg(reinterpret_cast<const float2*>(grad + (uint64_t)f * V + i));
        m16[q] = m[o2];
        v16[q] = v[o2];
        if (f < F_BF16)
          pf[q] = *reinterpret_cast<const float2*>(p + (uint64_t)f * B);
        else
          p16[q] = q16[(uint64_t)(f - F_BF16) * (B / 2)];
      }
    }
    const bool sr = rl.sr != 0;
    const uint32_t blk = rl.item_block[item];
    const uint32_t step = block_step[blk];
    const uint64_t gid0 = (uint64_t)blk * B + lane;
    const uint32_t key0 = sr ? sr_key(rl.seed, gid0, step) : 0u;
    const uint32_t key1 = sr ? sr_key(rl.seed, gid0 + 1, step) : 0u;
#pragma unroll
    for (int q = 0; q < ADAM_FG; ++q) {
      const int f = f0 + q;
      if (f < D) {
        const uint64_t o2 = (uint64_t)f * (B / 2);
        const float lr = lrs.g[lr_group(f)];
        const float2 mo = __bfloat1622float2(m16[q]), vo = __bfloat1622float2(v16[q]);
        const float2 po = f < F_BF16 ? pf[q] : __bfloat1622float2(p16[q]);
        const float mnx = b1 * mo.x + (1.f - b1) * gf[q].x, mny = b1 * mo.y + (1.f - b1) * gf[q].y;
        const float vnx = b2 * vo.x + (1.f - b2) * gf[q].x * gf[q].x;
        const float vny = b2 * vo.y + (1.f - b2) * gf[q].y * gf[q].y;
        const float ux = lr * __fdividef(mnx * ic1, adam_sqrt(vnx * ic2) + eps);
        const float uy = lr * __fdividef(mny * ic1, adam_sqrt(vny * ic2) + eps);
        const uint32_t h0 = sr ? fmix32(key0 + (uint32_t)f * 0x9E3779B9u) : 0u;
        const uint32_t h1 = sr ? fmix32(key1 + (uint32_t)f * 0x9E3779B9u) : 0u;
        __nv_bfloat162 mw, vw;
        mw.x = t0 ? to_bf16(mnx, sr, h0) : m16[q].x;
        mw.y = t1 ? to_bf16(mny, sr, h1) : m16[q].y;
        vw.x = t0 ? to_bf16(vnx, sr, h0 >> 16) : v16[q].x;
        vw.y = t1 ? to_bf16(vny, sr, h1 >> 16) : v16[q].y;
        m[o2] = mw;
        v[o2] = vw;
        if (f < F_BF16) {
          float2 pn = po;
          if (t0) pn.x = po.x - ux;
          if (t1) pn.y = po.y - uy;
          *reinterpret_cast<float2*>(p + (uint64_t)f * B) = pn;
        } else {
          __nv_bfloat162 pw;
          pw.x = t0 ? to_bf16(po.x - ux, sr, param_draw(h0)) : p16[q].x;
          pw.y = t1 ? to_bf16(po.y - uy, sr, param_draw(h1)) : p16[q].y;
          q16[(uint64_t)(f - F_BF16) * (B / 2)] = pw;
        }
      }
    }
  }
}

// Masked Adam over pairs of adjacent render-list positions with a touched
// member (prows[0..*nprows): position | mask << 30), CTA (pair chunk, field
// group).
template <bool BF>
__global__ void __launch_bounds__(PP_THREADS, 3) k_adam_pairs(RenderList rl, const float* __restrict__ grad,
                                                          const uint32_t* __restrict__ prows,
                                                          const uint32_t* __restrict__ nprows,
                                                          const float2* __restrict__ bias,
                                                          const uint32_t* __restrict__ block_step, uint64_t V,
                                                          LrSet lrs, float b1, float b2, float eps,
                                                          const uint32_t* __restrict__ abort_flag) {
  if (abort_flag && *abort_flag) return;  // a render of this step overflowed its pair capacity
  const uint32_t B = rl.B, n = *nprows;
  const int f0 = blockIdx.y * ADAM_FG;
  for (uint32_t t = blockIdx.x * PP_THREADS + threadIdx.x; t < n; t += gridDim.x * PP_THREADS) {
    const uint32_t e = prows[t];
    const uint32_t i = e & 0x3FFFFFFFu, mask = e >> 30;
    const unsigned item = item_of(i, B), lane = i - item * B;
    adam_pair<BF>(rl, grad, bias, block_step, V, lrs, b1, b2, eps, item, lane, i, mask, f0);
  }
}

// Masked Adam over the touched rows of the render list (rows[0..*nrows)):
// CTA (row chunk, field group), each thread ADAM_FG consecutive fields of one
// Gaussian, so a warp keeps several independent coalesced loads of p, g, m
// and v in flight.  The bias corrections of the item's block come
// precomputed.
template <bool BF>
__global__ void __launch_bounds__(PP_THREADS) k_adam(RenderList rl, const float* __restrict__ grad,
                                                    const uint32_t* __restrict__ rows,
                                                    const uint32_t* __restrict__ nrows,
                                                    const float2* __restrict__ bias,
                                                    const uint32_t* __restrict__ block_step, uint64_t V, LrSet lrs,
                                                    float b1, float b2, float eps,
                                                    const uint32_t* __restrict__ abort_flag) {
  if (abort_flag && *abort_flag) return;  // a render of this step overflowed its pair capacity
  const uint32_t B = rl.B, n = *nrows;
  const int f0 = blockIdx.y * ADAM_FG;
  for (uint32_t t = blockIdx.x * PP_THREADS + threadIdx.x; t < n; t += gridDim.x * PP_THREADS) {
    const uint32_t i = rows[t];
    const unsigned item = item_of(i, B), lane = i - item * B;
    adam_row<BF>(rl, grad, bias, block_step, V, lrs, b1, b2, eps, item, lane, i, f0);
  }
}

__global__ void k_mark_touched(RenderList rl, const uint32_t* __restrict__ item_touched, uint32_t* block_step,
                               uint8_t* dirty, uint32_t* abort_flag, float b1, float b2, float2* __restrict__ bias,
                               uint8_t* readmit, unsigned long long* churn) {
  unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
  if (abort_flag && abort_flag[0]) {
    if (j == 0) abort_flag[1] += 1;  // steps dropped since the overflow
    return;
  }
  if (j >= rl.n_items || !item_touched[j]) return;
  const uint32_t blk = rl.item_block[j];
  const uint32_t st = block_step[blk] + 1;
  block_step[blk] = st;
  if (churn) {
    atomicAdd(churn, 1ull);
    if (readmit && readmit[blk]) {
      atomicAdd(churn + 1, 1ull);
      readmit[blk] = 0;
    }
  }
  if (dirty) dirty[rl.item_slot[j]] = 1;
  if (bias) {
    const float tau = (float)st;
    bias[j] = make_float2(1.f / (1.f - powf(b1, tau)), 1.f / (1.f - powf(b2, tau)));
  }
}

__device__ __forceinline__ float block_reduce(float v, float* sm, bool is_max, bool is_min) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float u = __shfl_xor_sync(0xffffffffu, v, o);
    v = is_max ? fmaxf(v, u) : (is_min ? fminf(v, u) : v + u);
  }
  __syncthreads();
  if (lane == 0) sm[w] = v;
  __syncthreads();
  float r = sm[0];
  for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = is_max ? fmaxf(r, sm[k]) : (is_min ? fminf(r, sm[k]) : r + sm[k]);
  return r;
}

// Bounds refresh: one CTA per touched block.  Each thread loads the means of
// its BD_EPT rows of a chunk in one batch (every load of the chunk in flight
// at once) and then their log-scales; the centre is the midpoint of the box
// of the means and the radius the largest |mean - centre| + 3 exp(max
// log-scale).  A block longer than one chunk reloads its rows for the radius.
constexpr int BD_THREADS = 512;
constexpr int BD_EPT = 8;
constexpr uint32_t BD_CHUNK = (uint32_t)BD_THREADS * BD_EPT;
constexpr int BD_WARPS = BD_THREADS / 32;

__device__ __forceinline__ bool bounds_row(uint32_t c0, int e, uint32_t cnt, uint32_t& l) {
  l = c0 + (uint32_t)(e * BD_THREADS) + threadIdx.x;
  return l < cnt;
}
__device__ __forceinline__ void bounds_means(const float* __restrict__ p, uint32_t B, uint32_t cnt, uint32_t c0,
                                             float (&pos)[BD_EPT][3]) {
#pragma unroll
  for (int e = 0; e < BD_EPT; ++e) {
    uint32_t l;
    if (bounds_row(c0, e, cnt, l))
#pragma unroll
      for (int a = 0; a < 3; ++a) pos[e][a] = p[(uint64_t)a * B + l];
  }
}
__device__ __forceinline__ void bounds_scales(const float* __restrict__ p, uint32_t B, uint32_t cnt, uint32_t c0,
                                              float (&ls)[BD_EPT]) {
#pragma unroll
  for (int e = 0; e < BD_EPT; ++e) {
    uint32_t l;
    if (bounds_row(c0, e, cnt, l))
      ls[e] = fmaxf(fmaxf(p[(uint64_t)3 * B + l], p[(uint64_t)4 * B + l]), p[(uint64_t)5 * B + l]);
  }
}
__device__ __forceinline__ float bounds_reach(const float (&q)[3], float ls, const float (&c)[3]) {
  const float dx = q[0] - c[0], dy = q[1] - c[1], dz = q[2] - c[2];
  return sqrtf(dx * dx + dy * dy + dz * dz) + 3.f * expf(ls);
}

__global__ void __launch_bounds__(BD_THREADS, 2) k_bounds(RenderList rl, const uint32_t* __restrict__ only,
                                                         float4* __restrict__ spheres,
                                                         const uint32_t* __restrict__ abort_flag) {
  __shared__ float s_red[6][BD_WARPS];
  __shared__ float s_c[3];
  const unsigned item = blockIdx.x;
  if ((only && !only[item]) || (abort_flag && *abort_flag)) return;
  const uint32_t B = rl.B, cnt = rl.item_count[item];
  const float* p = rl.base + (uint64_t)rl.item_slot[item] * rl.slot_stride;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  float pos[BD_EPT][3], ls[BD_EPT];
  for (uint32_t c0 = 0; c0 < cnt; c0 += BD_CHUNK) {
    bounds_means(p, B, cnt, c0, pos);
#pragma unroll
    for (int e = 0; e < BD_EPT; ++e) {
      uint32_t l;
      if (bounds_row(c0, e, cnt, l))
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          mn[a] = fminf(mn[a], pos[e][a]);
          mx[a] = fmaxf(mx[a], pos[e][a]);
        }
    }
  }
  const bool one_chunk = cnt <= BD_CHUNK;
  if (one_chunk) bounds_scales(p, B, cnt, 0, ls);  // in flight during the reduction
  // the six extrema of the box: warps, then warp 0 over the warps
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
  if (lane == 0)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s_red[a][w] = mn[a];
      s_red[3 + a][w] = mx[a];
    }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float lo = lane < BD_WARPS ? s_red[a][lane] : INFINITY;
      float hi = lane < BD_WARPS ? s_red[3 + a][lane] : -INFINITY;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      if (lane == 0) s_c[a] = __fmul_rn(__fadd_rn(lo, hi), 0.5f);
    }
  }
  __syncthreads();
  const float c[3] = {s_c[0], s_c[1], s_c[2]};
  float r = 0.f;
  for (uint32_t c0 = 0; c0 < cnt; c0 += BD_CHUNK) {
    if (!one_chunk) {
      bounds_means(p, B, cnt, c0, pos);
      bounds_scales(p, B, cnt, c0, ls);
    }
#pragma unroll
    for (int e = 0; e < BD_EPT; ++e) {
      uint32_t l;
      if (bounds_row(c0, e, cnt, l)) r = fmaxf(r, bounds_reach(pos[e], ls[e], c));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
  if (lane == 0) s_red[0][w] = r;  // warp 0 read the box extrema before the barrier above
  __syncthreads();
  if (w == 0) {
    r = lane < BD_WARPS ? s_red[0][lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) spheres[rl.item_block[item]] = make_float4(c[0], c[1], c[2], r);
  }
}

__global__ void k_loss(const float* __restrict__ img, const float* __restrict__ tgt, uint64_t n, int kind,
                       float* __restrict__ grad, float* __restrict__ loss_sum) {
  __shared__ float sm[8];
  float acc = 0.f;
  const float inv = 1.f / (float)n;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    float d = img[i] - tgt[i];
    if (kind == 0) {
      acc += fabsf(d);
      grad[i] = (d > 0.f ? inv : (d < 0.f ? -inv : 0.f));
    } else {
      acc += d * d;
      grad[i] = 2.f * d * inv;
    }
  }
  float s = block_reduce(acc, sm, false, false);
  if (threadIdx.x == 0) atomicAdd(loss_sum, s);
}

__global__ void k_mark_visible(RenderList rl, const uint32_t* __restrict__ ntiles, uint8_t* __restrict__ touched,
                               unsigned cpi) {
  const unsigned item = blockIdx.x / cpi;
  const unsigned lane = (blockIdx.x - item * cpi) * PP_THREADS + threadIdx.x;
  if (lane >= rl.B || lane >= rl.item_count[item]) return;
  const uint64_t i = (uint64_t)item * rl.B + lane;
  if (ntiles[i]) touched[(uint64_t)rl.item_block[item] * rl.B + lane] = 1;
}

__global__ void k_dense_steps(const uint8_t* __restrict__ touched, uint64_t n, uint32_t B, uint32_t* step) {
  const uint64_t k = blockIdx.x;
  int any = 0;
  for (uint32_t l = threadIdx.x; l < B; l += blockDim.x) {
    uint64_t g = k * B + l;
    if (g < n && touched[g]) any = 1;
  }
  if (__syncthreads_or(any) && threadIdx.x == 0) step[k] += 1;
}

__global__ void k_adam_dense(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                             float* __restrict__ v, const uint8_t* __restrict__ touched,
                             const uint32_t* __restrict__ step, uint64_t n, uint32_t B, float lr, float b1, float b2,
                             float eps) {
  const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n || !touched[g]) return;
  const uint64_t k = g / B, l = g % B;
  const float tau = (float)step[k];
  const float ic1 = 1.f / (1.f - powf(b1, tau)), ic2 = 1.f / (1.f - powf(b2, tau));
  const uint64_t base = k * (uint64_t)D * B + l;
#pragma unroll 4
  for (int f = 0; f < D; ++f) {
    const uint64_t o = base + (uint64_t)f * B;
    float gf = gr[o];
    float mf = b1 * m[o] + (1.f - b1) * gf;
    float vf = b2 * v[o] + (1.f - b2) * gf * gf;
    m[o] = mf;
    v[o] = vf;
    p[o] -= lr * (mf * ic1) / (sqrtf(vf * ic2) + eps);
  }
}

}  // namespace

void mark_visible_bytes(const RenderList& rl, const CamState& cs, uint8_t* touched, cudaStream_t s) {
  if (rl.capacity() == 0) return;
  unsigned cpi = div_up(rl.B, PP_THREADS);
  k_mark_visible<<<rl.n_items * cpi, PP_THREADS, 0, s>>>(rl, cs.ntiles, touched, cpi);
  TGS_LAUNCHED();
}

void adam_dense(float* params, const float* grad, float* m1, float* m2, const uint8_t* touched, uint32_t* step,
                uint64_t n, uint32_t B, float lr, float b1, float b2, float eps, cudaStream_t s) {
  uint64_t K = (n + B - 1) / B;
  k_dense_steps<<<(unsigned)K, 256, 0, s>>>(touched, n, B, step);
  TGS_LAUNCHED();
  k_adam_dense<<<div_up(n, 256), 256, 0, s>>>(params, grad, m1, m2, touched, step, n, B, lr, b1, b2, eps);
  TGS_LAUNCHED();
}

DevCam make_devcam(const tgs_camera& c) {
  DevCam d;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) d.R[3 * a + b] = c.world_to_cam[4 * a + b];
    d.t[a] = c.world_to_cam[4 * a + 3];
  }
  d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy; d.znear = c.znear; d.zfar = c.zfar;
  for (int j = 0; j < 3; ++j) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a) s += (double)c.world_to_cam[4 * a + j] * (double)c.world_to_cam[4 * a + 3];
    d.campos[j] = (float)(-s);
  }
  d.W = (int)c.width;
  d.H = (int)c.height;
  d.limx = (float)(1.3 * (double)c.width / (2.0 * (double)c.fx));
  d.limy = (float)(1.3 * (double)c.height / (2.0 * (double)c.fy));
  d.TX = (d.W + TILE - 1) / TILE;
  d.TY = (d.H + TILE - 1) / TILE;
  return d;
}

static int bits_for(uint64_t n) {
  int b = 1;
  while ((1ull << b) < n) ++b;
  return b;
}

void cam_state_alloc(CamState& cs, uint64_t cap_v, uint64_t cap_pairs, int max_w, int max_h) {
  cs.cap_v = cap_v;
  cs.cap_pix = (uint64_t)max_w * max_h;
  cs.cap_tiles = (uint64_t)((max_w + TILE - 1) / TILE) * ((max_h + TILE - 1) / TILE);
  uint64_t V = cap_v > 0 ? cap_v : 1;
  TGS_CUDA(cudaMalloc(&cs.xy, V * sizeof(float2)));
  TGS_CUDA(cudaMalloc(&cs.depth, V * sizeof(float)));
  TGS_CUDA(cudaMalloc(&cs.conic_o, V * sizeof(float4)));
  TGS_CUDA(cudaMalloc(&cs.rgb, V * sizeof(float4)));
  TGS_CUDA(cudaMalloc(&cs.rect, V * sizeof(ushort4)));
  TGS_CUDA(cudaMalloc(&cs.radius, V * sizeof(int)));
  TGS_CUDA(cudaMalloc(&cs.ntiles, V * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&cs.scan, V * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&cs.dkeys, 2 * V * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&cs.dvals, 2 * V * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&cs.g2, 9 * V * sizeof(float)));
  TGS_CUDA(cudaMalloc(&cs.ranges, cs.cap_tiles * sizeof(uint2)));
  TGS_CUDA(cudaMalloc(&cs.t_final, cs.cap_pix * sizeof(float)));
  TGS_CUDA(cudaMalloc(&cs.n_last, cs.cap_pix * sizeof(int)));
  TGS_CUDA(cudaMalloc(&cs.counters, 16 * sizeof(uint32_t)));
  TGS_CUDA(cudaMallocHost(&cs.counters_host, 8 * sizeof(uint32_t)));
  {
    const int mtx = (max_w + TILE - 1) / TILE, mty = (max_h + TILE - 1) / TILE;
    const size_t tb = tile_scan_smem_bytes(mtx, mty);
    TGS_CHECK(tb <= TILE_SCAN_SMEM_MAX, TGS_ERR_INVALID,
              "image too large for the tile binning (at most 40,960 cells of (tiles_x + 1) x (tiles_y + 1))");
    TGS_CUDA(cudaMalloc(&cs.tdiff, tb));
    TGS_CUDA(cudaMemset(cs.tdiff, 0, tb));
  }
  TGS_CUDA(cudaMalloc(&cs.tfill, cs.cap_tiles * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&cs.tbig, cs.cap_tiles * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&cs.torder, 2 * cs.cap_tiles * sizeof(uint32_t)));
  // backward split: up to 4 checkpoint slots per tile, at most 8192 (32 MB)
  TGS_CHECK(cs.cap_tiles < (1ull << 24), TGS_ERR_INVALID, "image has too many tiles");
  cs.ck_cap = (uint32_t)std::min<uint64_t>(8192, 4 * cs.cap_tiles);
  TGS_CUDA(cudaMalloc(&cs.ck, (uint64_t)cs.ck_cap * TILE_PIX * sizeof(float4)));
  TGS_CUDA(cudaMalloc(&cs.tck, cs.cap_tiles * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&cs.units, (cs.cap_tiles + cs.ck_cap) * sizeof(uint32_t)));
  TGS_CUDA(cudaEventCreateWithFlags(&cs.ev_counts, cudaEventDisableTiming));
  {
    int lo = 0, hi = 0;
    TGS_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    TGS_CUDA(cudaStreamCreateWithPriority(&cs.aux, cudaStreamNonBlocking, hi));
    TGS_CUDA(cudaEventCreateWithFlags(&cs.ev_fork, cudaEventDisableTiming));
    TGS_CUDA(cudaEventCreateWithFlags(&cs.ev_join, cudaEventDisableTiming));
  }
  TGS_CUDA(cudaMemset(cs.counters, 0, 16 * sizeof(uint32_t)));
  cs.cap_pairs = 0;
  cam_state_grow_pairs(cs, cap_pairs > 0 ? cap_pairs : 1024, 0);
}

void cam_state_grow_pairs(CamState& cs, uint64_t need, cudaStream_t s) {
  uint64_t want = need > cs.cap_v ? need : cs.cap_v;
  if (need <= cs.cap_pairs && cs.scratch) return;
  if (need > cs.cap_pairs) {
    if (s) TGS_CUDA(cudaStreamSynchronize(s));
    if (cs.pkeys) TGS_CUDA(cudaFree(cs.pkeys));
    if (cs.pvals) TGS_CUDA(cudaFree(cs.pvals));
    uint64_t cap = need + need / 4 + 1024;
    TGS_CUDA(cudaMalloc(&cs.pkeys, 2 * cap * sizeof(uint32_t)));
    TGS_CUDA(cudaMalloc(&cs.pvals, 2 * cap * sizeof(uint32_t)));
    cs.cap_pairs = cap;
    want = cap > cs.cap_v ? cap : cs.cap_v;
  }
  size_t sb = radix_scratch_bytes(want);
  size_t sc = scan_scratch_bytes(want);
  if (sc > sb) sb = sc;
  if (sb > cs.scratch_bytes) {
    if (s) TGS_CUDA(cudaStreamSynchronize(s));
    if (cs.scratch) TGS_CUDA(cudaFree(cs.scratch));
    TGS_CUDA(cudaMalloc(&cs.scratch, sb));
    cs.scratch_bytes = sb;
  }
}

void cam_state_free(CamState& cs) {
  void* ptrs[] = {cs.xy, cs.depth, cs.conic_o, cs.rgb, cs.rect, cs.radius, cs.ntiles, cs.scan, cs.dkeys,
                  cs.dvals, cs.g2, cs.ranges, cs.t_final, cs.n_last, cs.counters, cs.pkeys, cs.pvals, cs.scratch,
                  cs.torder, cs.ck, cs.tck, cs.units, cs.tdiff, cs.tfill, cs.tbig};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (cs.counters_host) cudaFreeHost(cs.counters_host);
  if (cs.ev_counts) cudaEventDestroy(cs.ev_counts);
  if (cs.ev_fork) cudaEventDestroy(cs.ev_fork);
  if (cs.ev_join) cudaEventDestroy(cs.ev_join);
  if (cs.aux) cudaStreamDestroy(cs.aux);
  cs = CamState();
}


void render_forward(const RenderList& rl, const DevCam& cam, const float bg[3], CamState& cs, float* image,
                    uint8_t* touched, uint32_t* item_touched, cudaStream_t s, StageTimer* tm) {
  StageTimer dummy;
  if (!tm) tm = &dummy;
  const uint64_t V = rl.capacity();
  TGS_CHECK(V <= cs.cap_v, TGS_ERR_CAPACITY, "render list exceeds the per-camera capacity");
  TGS_CHECK((uint64_t)cam.W * cam.H <= cs.cap_pix && (uint64_t)cam.TX * cam.TY <= cs.cap_tiles, TGS_ERR_CAPACITY,
            "image larger than the configured maximum");
  cs.W = cam.W; cs.H = cam.H; cs.TX = cam.TX; cs.TY = cam.TY;
  cam_state_counts(cs, false);  // harvest an earlier render's counts if they arrived (grid hints)
  cs.counts_valid = false;
  const uint64_t tiles = (uint64_t)cam.TX * cam.TY;
  const float3 bg3 = make_float3(bg[0], bg[1], bg[2]);
  uint32_t* nv_dev = cs.counters;      // visible Gaussians
  TGS_CUDA(cudaMemsetAsync(cs.ranges, 0, tiles * sizeof(uint2), s));
  TGS_CUDA(cudaMemsetAsync(cs.counters, 0, 2 * sizeof(uint32_t), s));  // the overflow words stay
  if (V > 0) {
    unsigned cpi = div_up(rl.B, PP_THREADS);
    PPOut o{cs.xy, cs.depth, cs.conic_o, cs.rgb, cs.rect, cs.radius, cs.ntiles, cs.scan, cs.tdiff, nv_dev};
    tm->begin(StageTimer::PRE, s);
    if (rl.bf16)
      k_preprocess<true><<<rl.n_items * cpi, PP_THREADS, 0, s>>>(rl, cam, o, touched, item_touched, cpi);
    else
      k_preprocess<false><<<rl.n_items * cpi, PP_THREADS, 0, s>>>(rl, cam, o, touched, item_touched, cpi);
    TGS_LAUNCHED();
    tm->end(StageTimer::PRE, s);
    tm->begin(StageTimer::SORT, s);
    // the sizes stay on the device: no host round trip inside a render
    bin_tiles(V, cam.TX, cam.TY, cs, s);
    cs.order_valid = true;
    tm->end(StageTimer::SORT, s);
  } else {
    cs.order_valid = false;
  }
  tm->begin(StageTimer::FWD, s);
  k_raster_fwd<F_PPT><<<(unsigned)tiles, F_THREADS, 0, s>>>(cs.ranges, cs.pvals, cs.xy, cs.conic_o, cs.rgb, cam.W, cam.H,
                                                   cam.TX, bg3, image, cs.t_final, cs.n_last,
                                                   cs.order_valid ? cs.torder : nullptr,
                                                   cs.order_valid ? cs.tck : nullptr, cs.ck);
  TGS_LAUNCHED();
  tm->end(StageTimer::FWD, s);
  // the counts reach the host asynchronously (read by cam_state_counts)
  TGS_CUDA(cudaMemcpyAsync(cs.counters_host, cs.counters, 8 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  TGS_CUDA(cudaEventRecord(cs.ev_counts, s));
  cs.counts_pending = true;
}

bool cam_state_counts(CamState& cs, bool wait) {
  if (cs.counts_pending) {
    if (wait) {
      TGS_CUDA(cudaEventSynchronize(cs.ev_counts));
    } else {
      cudaError_t e = cudaEventQuery(cs.ev_counts);
      if (e == cudaErrorNotReady) return false;
      TGS_CUDA(e);
    }
    TGS_CHECK(cs.counters_host[6] == 0, TGS_ERR_STATE,
              "tile binning: a tile received more pairs than its rect count");
    cs.n_vis = cs.counters_host[0];
    cs.n_pairs = cs.counters_host[1];
    cs.overflow = cs.counters_host[2] != 0;
    cs.pairs_needed = cs.counters_host[3];
    cs.hint_nv = cs.n_vis;
    cs.hint_np = cs.n_pairs < cs.cap_pairs ? cs.n_pairs : cs.cap_pairs;
    cs.counts_pending = false;
    cs.counts_valid = true;
  }
  return cs.counts_valid;
}

// The forward of render_forward on caller-provided fixed buffers: nothing is
// (re)allocated; a pair count above cs.cap_pairs is an error.  Counts are read
// back into host stack variables.
void render_forward_fixed(const RenderList& rl, const DevCam& cam, const float bg[3], CamState& cs, float* image,
                          cudaStream_t s) {
  const uint64_t V = rl.capacity();
  TGS_CHECK(V <= cs.cap_v, TGS_ERR_CAPACITY, "render list exceeds the fixed capacity");
  TGS_CHECK((uint64_t)cam.W * cam.H <= cs.cap_pix && (uint64_t)cam.TX * cam.TY <= cs.cap_tiles, TGS_ERR_CAPACITY,
            "image larger than the fixed maximum");
  cs.W = cam.W; cs.H = cam.H; cs.TX = cam.TX; cs.TY = cam.TY;
  const uint64_t tiles = (uint64_t)cam.TX * cam.TY;
  const float3 bg3 = make_float3(bg[0], bg[1], bg[2]);
  cs.n_vis = 0;
  cs.n_pairs = 0;
  uint32_t cnt = 0;
  TGS_CUDA(cudaMemsetAsync(cs.ranges, 0, tiles * sizeof(uint2), s));
  TGS_CUDA(cudaMemsetAsync(cs.counters, 0, 4 * sizeof(uint32_t), s));
  if (V > 0) {
    unsigned cpi = div_up(rl.B, PP_THREADS);
    PPOut o{cs.xy, cs.depth, cs.conic_o, cs.rgb, cs.rect, cs.radius, cs.ntiles, cs.scan};
    k_preprocess<false><<<rl.n_items * cpi, PP_THREADS, 0, s>>>(rl, cam, o, nullptr, nullptr, cpi);
    TGS_LAUNCHED();
    exclusive_scan_u32(cs.scan, cs.scan, cs.counters, V, cs.scratch, s);
    k_compact_visible<<<div_up(V, 256), 256, 0, s>>>(V, cs.ntiles, cs.scan, cs.depth, cs.dkeys, cs.dvals);
    TGS_LAUNCHED();
    TGS_CUDA(cudaMemcpyAsync(&cnt, cs.counters, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TGS_CUDA(cudaStreamSynchronize(s));
    cs.n_vis = cnt;
  }
  const uint64_t nv = cs.n_vis;
  if (nv > 0) {
    radix_sort_pairs(cs.dkeys, cs.dvals, cs.dkeys + cs.cap_v, cs.dvals + cs.cap_v, nv, 32, cs.scratch, s);
    k_gather_counts<<<div_up(nv, 256), 256, 0, s>>>(cs.counters, cs.dvals, cs.ntiles, cs.scan);
    TGS_LAUNCHED();
    exclusive_scan_u32(cs.scan, cs.scan, cs.counters + 1, nv, cs.scratch, s);
    TGS_CUDA(cudaMemcpyAsync(&cnt, cs.counters + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TGS_CUDA(cudaStreamSynchronize(s));
    cs.n_pairs = cnt;
    TGS_CHECK(cs.n_pairs <= cs.cap_pairs, TGS_ERR_CAPACITY, "tile/Gaussian pairs exceed the fixed maximum");
    const uint64_t np = cs.n_pairs;
    if (np > 0) {
      k_emit_pairs<<<4 * NSM, EP_THREADS, 0, s>>>(cs.counters, cs.counters + 1, cs.dvals, cs.rect, cs.scan, cam.TX,
                                                  cs.pkeys, cs.pvals, cs.cap_pairs, cs.counters + 2, nullptr);
      TGS_LAUNCHED();
      radix_sort_pairs(cs.pkeys, cs.pvals, cs.pkeys + cs.cap_pairs, cs.pvals + cs.cap_pairs, np,
                       bits_for(tiles), cs.scratch, s);
      k_ranges<<<div_up(np, 256), 256, 0, s>>>(cs.counters + 1, cs.cap_pairs, cs.pkeys, cs.ranges);
      TGS_LAUNCHED();
    }
  }
  k_raster_fwd<F_PPT><<<(unsigned)tiles, F_THREADS, 0, s>>>(cs.ranges, cs.pvals, cs.xy, cs.conic_o, cs.rgb, cam.W, cam.H,
                                                   cam.TX, bg3, image, cs.t_final, cs.n_last, nullptr, nullptr,
                                                   nullptr);
  cs.order_valid = false;
  TGS_LAUNCHED();
}

void render_backward_2d(const RenderList& rl, const DevCam& cam, const float bg[3], CamState& cs,
                        const float* dl_dimage, cudaStream_t s) {
  const uint64_t V = rl.capacity();
  const uint64_t tiles = (uint64_t)cam.TX * cam.TY;
  if (V == 0) return;
  // the 2D gradients use the render list's size as their stride, so only
  // that much is cleared (not the whole capacity)
  cs.g2_stride = V;
  TGS_CUDA(cudaMemsetAsync(cs.g2, 0, 9 * V * sizeof(float), s));
  const float3 bg3 = make_float3(bg[0], bg[1], bg[2]);
  // with a valid tile order: one CTA per backward unit (longest lists
  // first, long lists split into segments); the unit count stays on the
  // device, so the grid takes its bound and the surplus CTAs return at once
  const bool split = cs.order_valid;
  const uint64_t grid = split ? tiles + cs.ck_cap : tiles;
  k_raster_bwd<<<(unsigned)grid, R_THREADS, 0, s>>>(cs.ranges, cs.pvals, cs.xy, cs.conic_o, cs.rgb, cam.W, cam.H,
                                                  cam.TX, bg3, cs.t_final, cs.n_last, dl_dimage, cs.g2, cs.g2_stride,
                                                  split ? cs.units : nullptr, cs.counters + 5,
                                                  split ? cs.tck : nullptr, cs.ck);
  TGS_LAUNCHED();
}

void render_backward_params_batch(const RenderList& rl, const DevCam* cams, CamState* const* cs, int J, float* grad,
                                  const uint32_t* rows, const uint32_t* nrows, cudaStream_t s) {
  if (rl.capacity() == 0 || J <= 0) return;
  TGS_CHECK(J <= BatchGrad::MAXJ, TGS_ERR_INVALID, "batch larger than the fused chain rule supports");
  BatchGrad bg;
  bg.J = J;
  for (int j = 0; j < J; ++j) {
    bg.cam[j] = cams[j];
    bg.ntiles[j] = cs[j]->ntiles;
    bg.rgb[j] = cs[j]->rgb;
    bg.conic[j] = cs[j]->conic_o;
    bg.g2[j] = cs[j]->g2;
    bg.stride[j] = cs[j]->g2_stride;
  }
  const unsigned grid = std::min<uint64_t>(div_up(rl.capacity(), PP_THREADS), 4 * NSM);
  if (rl.bf16)
    k_preprocess_bwd_batch<true><<<grid, PP_THREADS, 0, s>>>(rl, bg, grad, rl.capacity(), rows, nrows);
  else
    k_preprocess_bwd_batch<false><<<grid, PP_THREADS, 0, s>>>(rl, bg, grad, rl.capacity(), rows, nrows);
  TGS_LAUNCHED();
}

void render_backward_params(const RenderList& rl, const DevCam& cam, const CamState& cs, float* grad, int mode,
                            cudaStream_t s, const uint32_t* rows, const uint32_t* nrows) {
  if (rl.capacity() == 0) return;
  unsigned cpi = div_up(rl.B, PP_THREADS);
  if (rows) {
    const unsigned grid = std::min<uint64_t>(div_up(rl.capacity(), PP_THREADS), 4 * NSM);
    if (rl.bf16)
      k_preprocess_bwd<true><<<grid, PP_THREADS, 0, s>>>(rl, cam, cs.ntiles, cs.rgb, cs.conic_o, cs.g2, cs.g2_stride, grad,
                                                        rl.capacity(), mode, cpi, rows, nrows);
    else
      k_preprocess_bwd<false><<<grid, PP_THREADS, 0, s>>>(rl, cam, cs.ntiles, cs.rgb, cs.conic_o, cs.g2, cs.g2_stride, grad,
                                                         rl.capacity(), mode, cpi, rows, nrows);
    TGS_LAUNCHED();
    return;
  }
  if (rl.bf16)
    k_preprocess_bwd<true><<<rl.n_items * cpi, PP_THREADS, 0, s>>>(rl, cam, cs.ntiles, cs.rgb, cs.conic_o, cs.g2,
                                                                  cs.g2_stride, grad, rl.capacity(), mode, cpi, nullptr, nullptr);
  else
    k_preprocess_bwd<false><<<rl.n_items * cpi, PP_THREADS, 0, s>>>(rl, cam, cs.ntiles, cs.rgb, cs.conic_o, cs.g2,
                                                                   cs.g2_stride, grad, rl.capacity(), mode, cpi, nullptr, nullptr);
  TGS_LAUNCHED();
}

void touched_rows(const RenderList& rl, const uint8_t* touched, uint32_t* rows, uint32_t* nrows, cudaStream_t s,
                  uint32_t* prows, uint32_t* nprows) {
  TGS_CUDA(cudaMemsetAsync(nrows, 0, sizeof(uint32_t), s));
  if (prows) TGS_CUDA(cudaMemsetAsync(nprows, 0, sizeof(uint32_t), s));
  const uint64_t V = rl.capacity();
  if (V == 0) return;
  const unsigned grid = std::min<uint64_t>(div_up(V, 128 * 8), 4 * NSM);
  k_touched_rows<<<grid, 256, 0, s>>>(touched, V, rows, nrows, prows, nprows);
  TGS_LAUNCHED();
}

void adam_render_list(const RenderList& rl, const float* grad, const uint32_t* rows, const uint32_t* nrows,
                      const float2* bias, const uint32_t* block_step, const LrSet& lr, float b1, float b2, float eps,
                      cudaStream_t s, const uint32_t* abort_flag, const uint32_t* prows, const uint32_t* nprows) {
  if (rl.capacity() == 0) return;
  // the pair kernel reads FP32 fields as float2 and BF16 ones as bf16x2:
  // every slot, field and moment array must start on an even float
  const bool pairs_aligned = rl.B % 2 == 0 && rl.slot_stride % 2 == 0 && rl.m_off % 2 == 0 && rl.v_off % 2 == 0 &&
                             (reinterpret_cast<uintptr_t>(rl.base) & 7u) == 0 &&
                             (reinterpret_cast<uintptr_t>(grad) & 7u) == 0;
  if (prows && pairs_aligned) {
    const dim3 grid(std::min<uint64_t>(div_up(rl.capacity() / 2, PP_THREADS), 4 * NSM), ADAM_GROUPS);
    if (rl.bf16)
      k_adam_pairs<true><<<grid, PP_THREADS, 0, s>>>(rl, grad, prows, nprows, bias, block_step, rl.capacity(), lr, b1,
                                                    b2, eps, abort_flag);
    else
      k_adam_pairs<false><<<grid, PP_THREADS, 0, s>>>(rl, grad, prows, nprows, bias, block_step, rl.capacity(), lr,
                                                     b1, b2, eps, abort_flag);
    TGS_LAUNCHED();
    return;
  }
  const dim3 grid(std::min<uint64_t>(div_up(rl.capacity(), PP_THREADS), 4 * NSM), ADAM_GROUPS);
  if (rl.bf16)
    k_adam<true><<<grid, PP_THREADS, 0, s>>>(rl, grad, rows, nrows, bias, block_step, rl.capacity(), lr, b1, b2, eps,
                                            abort_flag);
  else
    k_adam<false><<<grid, PP_THREADS, 0, s>>>(rl, grad, rows, nrows, bias, block_step, rl.capacity(), lr, b1, b2, eps,
                                             abort_flag);
  TGS_LAUNCHED();
}

void mark_touched_blocks(const RenderList& rl, const uint32_t* item_touched, uint32_t* block_step, uint8_t* dirty,
                         cudaStream_t s, uint32_t* abort_flag, float b1, float b2, float2* bias, uint8_t* readmit,
                         unsigned long long* churn) {
  if (rl.n_items == 0) return;
  k_mark_touched<<<div_up(rl.n_items, 256), 256, 0, s>>>(rl, item_touched, block_step, dirty, abort_flag, b1, b2,
                                                         bias, readmit, churn);
  TGS_LAUNCHED();
}

void block_bounds(const RenderList& rl, const uint32_t* only_flag, float4* spheres, cudaStream_t s,
                  const uint32_t* abort_flag) {
  if (rl.n_items == 0) return;
  k_bounds<<<rl.n_items, BD_THREADS, 0, s>>>(rl, only_flag, spheres, abort_flag);
  TGS_LAUNCHED();
}

void photometric_loss(const float* img, const float* target, uint64_t n, int kind, float* grad, float* loss_sum,
                      cudaStream_t s) {
  if (n == 0) return;
  unsigned grid = div_up(n, 256);
  if (grid > 4 * NSM) grid = 4 * NSM;
  k_loss<<<grid, 256, 0, s>>>(img, target, n, kind, grad, loss_sum);
  TGS_LAUNCHED();
}

}  // namespace tgs
