// Learned block-prefetch predictor on the GPU.
//
// Inference (every step of the learned-prefetch mode) is one fused kernel on
// the tcgen05 tensor cores, persistent over 128-row tiles of block rows:
// layer 1 (the pose part is a shared 96 x 256 product computed once per step;
// the per-block part has 6 inputs) in FP32 into a BF16 operand tile in shared
// memory, layer 2 (256 x 256, BF16 operands, FP32 accumulator in tensor
// memory) as 16 tcgen05.mma of M = 128, N = 256, K = 16 issued by one thread,
// and layer 3 (256 x 4) plus biases in the epilogue, one accumulator row
// (tcgen05.ld) per thread.  Training kernels (offline, on logged visibility)
// are FP32 SIMT: BCE gradient, the two 256-wide products of the backward,
// column sums, and AdamW on FP32 master weights.
#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "predictor.cuh"
#include "sort.cuh"

namespace tgs {
namespace {


__global__ void k_mlp_feat(const float4* __restrict__ sph, uint64_t K, uint64_t M, DevCam c, float zf,
                           float* __restrict__ feat) {
  uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  float* o = feat + 8 * k;
  if (k >= K) {
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] = 0.f;
    return;
  }
  float4 s = sph[k];
  float cx = c.R[0] * s.x + c.R[1] * s.y + c.R[2] * s.z + c.t[0];
  float cy = c.R[3] * s.x + c.R[4] * s.y + c.R[5] * s.z + c.t[1];
  float cz = c.R[6] * s.x + c.R[7] * s.y + c.R[8] * s.z + c.t[2];
  float d = sqrtf(cx * cx + cy * cy + cz * cz);
  float iz = 1.f / zf;
  o[0] = cx * iz;
  o[1] = cy * iz;
  o[2] = cz * iz;
  o[3] = s.w * iz;
  o[4] = d * iz;
  o[5] = s.w / fmaxf(d, s.w);
  o[6] = 0.f;
  o[7] = 0.f;
}

struct PoseVec {
  float v[MLP_NPOSE];
};

// pose term of layer 1 (shared by every block of a step); also keeps the pose
// vector on the device for the pose part of the weight gradient
__global__ void k_mlp_pose(const float* __restrict__ P, PoseVec pose, float* __restrict__ pose_out,
                           float* __restrict__ pterm) {
  const int j = threadIdx.x;
  float z = P[MLP_OFF_B1 + j];
  for (int i = 0; i < MLP_NPOSE; ++i) z += pose.v[i] * P[MLP_OFF_W1 + (uint64_t)i * MLP_H + j];
  pterm[j] = z;
  if (j < MLP_NPOSE) pose_out[j] = pose.v[j];
}

// ---- the forward on the 5th-generation tensor cores (tcgen05, sm_100+):
// persistent CTAs of 128 threads, one 128-row tile at a time.  W2^T (BF16,
// 256 x 256) is staged once per CTA in shared memory in the canonical K-major
// layout without swizzle: 8-row x 16-byte core matrices, element (r, k) of an
// R-row operand at (k / 8) * 16 R + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// bytes, so a descriptor's leading-dimension offset (next core matrix along
// K) is 16 R bytes and its stride-dimension offset (next 8 rows) 128 bytes.
// Per tile: layer 1 (FP32, thread t = row t) writes h1 as BF16 in the same
// layout, one thread issues the 16 MMAs (M = 128, N = 256, K = 16 each) into
// a 128 x 256 FP32 accumulator in tensor memory and commits them to an
// mbarrier; after the wait each warp reads its 32 accumulator lanes (rows)
// with tcgen05.ld, and each thread applies bias, ReLU and layer 3 to its row.
constexpr int TC_M = 128;
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_COLS = MLP_H;                         // accumulator columns (FP32)
constexpr uint32_t TC_B_BYTES = (uint32_t)MLP_H * MLP_H * 2;  // 128 KB
constexpr uint32_t TC_A_BYTES = (uint32_t)TC_M * MLP_H * 2;   // 64 KB
constexpr uint32_t TC_F_FLOATS = MLP_NFEAT * MLP_H + MLP_H + MLP_H + MLP_H * MLP_OUT + 4 + TC_M * 8;
constexpr uint32_t TC_SPIN_MAX = 1u << 22;  // try_wait polls before a wait gives up
// instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MLP_H >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t cm_off(uint32_t r, uint32_t k, uint32_t R) {
  return (k >> 3) * (R * 16) + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), descriptor version 1 (bits 46-47), no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accum));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_SPIN_MAX; ++i) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// rows_dev (device, may be null): only the first *rows_dev of the M rows are
// wanted.  err (device): set when a wait for the tensor cores runs out.
__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_fwd_tc(const float* __restrict__ P,
                                                             const __nv_bfloat16* __restrict__ w2t,
                                                             const float* __restrict__ pterm,
                                                             const float* __restrict__ feat, uint64_t M,
                                                             const uint32_t* __restrict__ rows_dev,
                                                             float* __restrict__ z3, __nv_bfloat16* __restrict__ h1g,
                                                             float* __restrict__ h2g, uint32_t* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* sB = tsm;
  unsigned char* sA = tsm + TC_B_BYTES;
  float* w1b = reinterpret_cast<float*>(sA + TC_A_BYTES);  // [6][256]
  float* pt = w1b + MLP_NFEAT * MLP_H;
  float* b2 = pt + MLP_H;
  float* w3 = b2 + MLP_H;  // [256][4]
  float* b3 = w3 + MLP_H * MLP_OUT;
  float* fs = b3 + 4;  // [128][8]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(fs + TC_M * 8);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  uint64_t rows = M;
  if (rows_dev && (uint64_t)*rows_dev < rows) rows = *rows_dev;
  const uint32_t ntiles = (uint32_t)((rows + TC_M - 1) / TC_M);
  if (blockIdx.x >= ntiles) return;  // uniform, before any tensor-memory allocation
  for (uint32_t e = tid; e < MLP_H * (MLP_H / 8); e += TC_THREADS) {
    const uint32_t n = e / (MLP_H / 8), k8 = e % (MLP_H / 8);
    *reinterpret_cast<uint4*>(sB + cm_off(n, 8 * k8, MLP_H)) =
        *reinterpret_cast<const uint4*>(w2t + (uint64_t)n * MLP_H + 8 * k8);
  }
  for (uint32_t e = tid; e < MLP_NFEAT * MLP_H; e += TC_THREADS) w1b[e] = P[MLP_OFF_W1 + (uint64_t)MLP_NPOSE * MLP_H + e];
  for (uint32_t e = tid; e < MLP_H; e += TC_THREADS) {
    pt[e] = pterm[e];
    b2[e] = P[MLP_OFF_B2 + e];
  }
  for (uint32_t e = tid; e < MLP_H * MLP_OUT; e += TC_THREADS) w3[e] = P[MLP_OFF_W3 + e];
  if (tid < 4) b3[tid] = P[MLP_OFF_B3 + tid];
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(tmem_slot)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(sA), b0 = (uint32_t)__cvta_generic_to_shared(sB);
  uint32_t parity = 0;
  bool ok = true;
  for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t r0 = (uint64_t)t * TC_M;
    for (uint32_t e = tid; e < TC_M * 8; e += TC_THREADS) {
      const uint64_t r = r0 + e / 8;
      fs[e] = r < M ? feat[r * 8 + e % 8] : 0.f;
    }
    __syncthreads();
    // layer 1: thread tid computes row r0 + tid
    const uint64_t row = r0 + (uint64_t)tid;
#pragma unroll 1
    for (int k0 = 0; k0 < MLP_H; k0 += 8) {
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float z[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int j = k0 + 2 * q + u;
          float a = pt[j];
#pragma unroll
          for (int i = 0; i < MLP_NFEAT; ++i) a += fs[tid * 8 + i] * w1b[i * MLP_H + j];
          z[u] = fmaxf(a, 0.f);
        }
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(z[0], z[1]);
        pk[q] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      const uint4 v = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      *reinterpret_cast<uint4*>(sA + cm_off((uint32_t)tid, (uint32_t)k0, TC_M)) = v;
      if (h1g && row < M) *reinterpret_cast<uint4*>(h1g + row * MLP_H + k0) = v;
    }
    // the tile's h1 (generic-proxy stores) becomes visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll 1
      for (uint32_t s2 = 0; s2 < MLP_H / 16; ++s2) {
        const uint64_t ad = smem_desc(a0 + 2 * s2 * (TC_M * 16), TC_M * 16, 128);
        const uint64_t bd = smem_desc(b0 + 2 * s2 * (MLP_H * 16), MLP_H * 16, 128);
        tc_mma(tmem, ad, bd, s2 > 0 ? 1u : 0u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mb)
                   : "memory");
    }
    if (!mbar_wait(mb, parity)) {
      ok = false;
      if (tid == 0) atomicOr(err, 1u);
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (ok) {
      // epilogue: warp w reads accumulator lanes 32 w .. 32 w + 31 (row tid)
      float lz[MLP_OUT];
#pragma unroll
      for (int o = 0; o < MLP_OUT; ++o) lz[o] = b3[o];
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < TC_COLS; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float h = fmaxf(v[j] + b2[c0 + j], 0.f);
          v[j] = h;
#pragma unroll
          for (int o = 0; o < MLP_OUT; ++o) lz[o] += h * w3[(c0 + j) * MLP_OUT + o];
        }
        if (h2g && row < M) {
          float4* d = reinterpret_cast<float4*>(h2g + row * MLP_H + c0);
#pragma unroll
          for (int j = 0; j < 8; ++j) d[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
      if (row < M) {
#pragma unroll
        for (int o = 0; o < MLP_OUT; ++o) z3[row * MLP_OUT + o] = lz[o];
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // accumulator, features and the A tile are rewritten next
    if (!__syncthreads_or(!ok)) continue;
    break;
  }
  // after a wait that ran out the tensor cores may still be writing the
  // accumulator: wait for that phase once more (bounded) before the columns
  // are freed
  if (__syncthreads_or(!ok)) mbar_wait(mb, parity ^ 1u);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_COLS) : "memory");
}

constexpr size_t TC_SMEM = TC_B_BYTES + TC_A_BYTES + TC_F_FLOATS * sizeof(float) + 16;

__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(__expf(x)); }

// one CTA per row: dz3 (BCE with pos_weight, mean over K x 4) and dh2
__global__ void k_mlp_dh2(const float* __restrict__ P, const float* __restrict__ z3, const float* __restrict__ labels,
                          const float* __restrict__ h2, uint64_t K, float pw, float inv, float* __restrict__ dz3,
                          float* __restrict__ dh2, float* __restrict__ loss) {
  const uint64_t r = blockIdx.x;
  const int n = threadIdx.x;
  float dz[MLP_OUT];
  float l = 0.f;
#pragma unroll
  for (int h = 0; h < MLP_OUT; ++h) {
    if (r < K) {
      const float z = z3[r * MLP_OUT + h], y = labels[r * MLP_OUT + h];
      const float p = 1.f / (1.f + __expf(-z));
      dz[h] = (p * (pw * y + 1.f - y) - pw * y) * inv;
      l += pw * y * softplus(-z) + (1.f - y) * softplus(z);
    } else {
      dz[h] = 0.f;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int h = 0; h < MLP_OUT; ++h) s += dz[h] * P[MLP_OFF_W3 + (uint64_t)n * MLP_OUT + h];
  dh2[r * MLP_H + n] = h2[r * MLP_H + n] > 0.f ? s : 0.f;
  if (n == 0) {
#pragma unroll
    for (int h = 0; h < MLP_OUT; ++h) dz3[r * MLP_OUT + h] = dz[h];
    if (r < K) atomicAdd(loss, l * inv);
  }
}

template <class TA>
__device__ __forceinline__ float tof(TA x) { return (float)x; }
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

// C[i][j] += sum_r A[r][i] B[r][j] over a chunk of 256 rows; 64 x 64 output tile
template <class TA>
__global__ void __launch_bounds__(256) k_mlp_atb(const TA* __restrict__ A, int lda, int na, const float* __restrict__ B,
                                                int ldb, int nb, uint64_t rows, float* __restrict__ C, int ldc) {
  __shared__ float as[32][65];
  __shared__ float bs[32][65];
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  const uint64_t r0 = (uint64_t)blockIdx.z * 256;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (uint64_t rc = r0; rc < r0 + 256 && rc < rows; rc += 32) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      int rr = e / 64, cc = e % 64;
      uint64_t r = rc + rr;
      as[rr][cc] = (r < rows && i0 + cc < na) ? tof(A[r * lda + i0 + cc]) : 0.f;
      bs[rr][cc] = (r < rows && j0 + cc < nb) ? B[r * ldb + j0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = as[rr][ty * 4 + u];
        b[u] = bs[rr][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < na && j < nb && acc[u][v] != 0.f) atomicAdd(&C[(uint64_t)i * ldc + j], acc[u][v]);
    }
}

// dh1[r][i] = (sum_j dh2[r][j] W2r[i][j]) * [h1[r][i] > 0]; 64 x 64 tiles
__global__ void __launch_bounds__(256) k_mlp_dh1(const float* __restrict__ dh2, const float* __restrict__ w2r,
                                                const __nv_bfloat16* __restrict__ h1, float* __restrict__ dh1) {
  __shared__ float as[64][33];
  __shared__ float bs[64][33];
  const uint64_t r0 = (uint64_t)blockIdx.x * 64;
  const int i0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < MLP_H; k0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      int rr = e / 32, kk = e % 32;
      as[rr][kk] = dh2[(r0 + rr) * MLP_H + k0 + kk];
      bs[rr][kk] = w2r[(uint64_t)(i0 + rr) * MLP_H + k0 + kk];
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = as[ty * 4 + u][kk];
        b[u] = bs[tx * 4 + u][kk];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const uint64_t r = r0 + ty * 4 + u;
      const int i = i0 + tx * 4 + v;
      dh1[r * MLP_H + i] = __bfloat162float(h1[r * MLP_H + i]) > 0.f ? acc[u][v] : 0.f;
    }
}

__global__ void k_mlp_colsum(const float* __restrict__ A, int n, uint64_t rows, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const uint64_t r0 = (uint64_t)blockIdx.y * 1024;
  float s = 0.f;
  for (uint64_t r = r0; r < r0 + 1024 && r < rows; ++r) s += A[r * n + j];
  atomicAdd(&out[j], s);
}

__global__ void k_mlp_pose_grad(const float* __restrict__ pose, float* __restrict__ G) {
  const int j = threadIdx.x;
  const float d = G[MLP_OFF_B1 + j];
  for (int i = 0; i < MLP_NPOSE; ++i) G[MLP_OFF_W1 + (uint64_t)i * MLP_H + j] += pose[i] * d;
}

__global__ void k_adamw(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                        float* __restrict__ v, uint64_t n, float lr, float b1, float b2, float eps, float wd, float ic1,
                        float ic2) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * ((mi * ic1) / (sqrtf(vi * ic2) + eps) + wd * p[i]);
}

__global__ void k_mlp_round_w2(const float* __restrict__ P, __nv_bfloat16* __restrict__ w2t, float* __restrict__ w2r) {
  const int k = blockIdx.x, n = threadIdx.x;  // W2[k][n]
  const __nv_bfloat16 b = __float2bfloat16_rn(P[MLP_OFF_W2 + (uint64_t)k * MLP_H + n]);
  w2t[(uint64_t)n * MLP_H + k] = b;
  w2r[(uint64_t)k * MLP_H + n] = __bfloat162float(b);
}

// Candidates of a prediction: blocks whose sphere comes within lim of the
// current camera centre, lim = the distance of the frustum's far corners plus
// how far the camera can travel over the predicted horizons; the others
// cannot enter the frustum in that time.
__global__ void k_mlp_cand(const float4* __restrict__ sph, uint64_t K, DevCam c, float lim,
                           uint32_t* __restrict__ flag) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const float4 s = sph[k];
  float cx = c.R[0] * s.x + c.R[1] * s.y + c.R[2] * s.z + c.t[0];
  float cy = c.R[3] * s.x + c.R[4] * s.y + c.R[5] * s.z + c.t[1];
  float cz = c.R[6] * s.x + c.R[7] * s.y + c.R[8] * s.z + c.t[2];
  flag[k] = sqrtf(cx * cx + cy * cy + cz * cz) - s.w <= lim ? 1u : 0u;
}

// Features of the candidates, packed in block order at rows pos[k].
__global__ void k_mlp_feat_cand(const float4* __restrict__ sph, uint64_t K, const uint32_t* __restrict__ flag,
                                const uint32_t* __restrict__ pos, DevCam c, float zf, float* __restrict__ feat,
                                uint32_t* __restrict__ cid) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K || !flag[k]) return;
  const uint32_t r = pos[k];
  cid[r] = (uint32_t)k;
  float4 s = sph[k];
  float cx = c.R[0] * s.x + c.R[1] * s.y + c.R[2] * s.z + c.t[0];
  float cy = c.R[3] * s.x + c.R[4] * s.y + c.R[5] * s.z + c.t[1];
  float cz = c.R[6] * s.x + c.R[7] * s.y + c.R[8] * s.z + c.t[2];
  float d = sqrtf(cx * cx + cy * cy + cz * cz);
  float iz = 1.f / zf;
  float* o = feat + 8 * (uint64_t)r;
  o[0] = cx * iz;
  o[1] = cy * iz;
  o[2] = cz * iz;
  o[3] = s.w * iz;
  o[4] = d * iz;
  o[5] = s.w / fmaxf(d, s.w);
  o[6] = 0.f;
  o[7] = 0.f;
}

__global__ void k_mlp_threshold_cand(const float* __restrict__ z3, const uint32_t* __restrict__ count,
                                     const uint32_t* __restrict__ cid, uint32_t mask, float zthr,
                                     uint32_t* __restrict__ bits) {
  const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= *count) return;
  bool vis = false;
#pragma unroll
  for (int h = 0; h < MLP_OUT; ++h)
    if ((mask >> h & 1u) && z3[r * MLP_OUT + h] > zthr) vis = true;
  if (vis) atomicOr(bits + (cid[r] >> 5), 1u << (cid[r] & 31));
}


// persistent CTAs: one per SM at most (each holds 208 KB of shared memory)
unsigned tc_grid(uint64_t M) { return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((M + TC_M - 1) / TC_M, NSM)); }

}  // namespace

void mlp_check(Mlp& m) {
  uint32_t e = 0;
  TGS_CUDA(cudaMemcpy(&e, m.err, sizeof(e), cudaMemcpyDeviceToHost));
  TGS_CHECK(e == 0, TGS_ERR_TIMEOUT, "predictor: a wait for the tensor cores ran out");
}

void mlp_alloc(Mlp& m, uint64_t max_rows, uint32_t seed) {
  m.max_rows = (max_rows + MLP_ROWS_PER_CTA - 1) / MLP_ROWS_PER_CTA * MLP_ROWS_PER_CTA;
  const uint64_t R = m.max_rows;
  TGS_CUDA(cudaMalloc(&m.params, MLP_NPARAM * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.grads, MLP_NPARAM * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.m, MLP_NPARAM * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.v, MLP_NPARAM * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.w2t, (uint64_t)MLP_H * MLP_H * sizeof(__nv_bfloat16)));
  TGS_CUDA(cudaMalloc(&m.w2r, (uint64_t)MLP_H * MLP_H * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.pose, MLP_NPOSE * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.pterm, MLP_H * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.feat, R * 8 * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.h1, R * MLP_H * sizeof(__nv_bfloat16)));
  TGS_CUDA(cudaMalloc(&m.h2, R * MLP_H * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.z3, R * MLP_OUT * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.dh2, R * MLP_H * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.dh1, R * MLP_H * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.dz3, R * MLP_OUT * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.loss, sizeof(float)));
  TGS_CUDA(cudaMallocHost(&m.loss_host, sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.cflag, R * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&m.cpos, R * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&m.cid, R * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&m.ccount, 4 * sizeof(uint32_t)));
  TGS_CUDA(cudaMalloc(&m.cscratch, scan_scratch_bytes(R)));
  // rows past a candidate count are computed and ignored: keep them finite
  TGS_CUDA(cudaMemset(m.feat, 0, R * 8 * sizeof(float)));
  // initial weights: N(0, 1/sqrt(fan_in)), zero biases (seeded)
  std::vector<float> h(MLP_NPARAM, 0.f);
  std::mt19937_64 rng(seed);
  auto fill = [&](uint64_t off, uint64_t n, double sd) {
    std::normal_distribution<double> nd(0.0, sd);
    for (uint64_t i = 0; i < n; ++i) h[off + i] = (float)nd(rng);
  };
  fill(MLP_OFF_W1, (uint64_t)MLP_NIN * MLP_H, 1.0 / std::sqrt((double)MLP_NIN));
  fill(MLP_OFF_W2, (uint64_t)MLP_H * MLP_H, 1.0 / std::sqrt((double)MLP_H));
  fill(MLP_OFF_W3, (uint64_t)MLP_H * MLP_OUT, 1.0 / std::sqrt((double)MLP_H));
  TGS_CUDA(cudaMemcpy(m.params, h.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice));
  TGS_CUDA(cudaMemset(m.m, 0, MLP_NPARAM * sizeof(float)));
  TGS_CUDA(cudaMemset(m.v, 0, MLP_NPARAM * sizeof(float)));
  TGS_CUDA(cudaMalloc(&m.err, sizeof(uint32_t)));
  TGS_CUDA(cudaMemset(m.err, 0, sizeof(uint32_t)));
  TGS_CUDA(cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM));
  mlp_refresh_bf16(m, 0);
  TGS_CUDA(cudaDeviceSynchronize());
}

void mlp_free(Mlp& m) {
  void* p[] = {m.params, m.grads, m.m, m.v, m.w2t, m.w2r, m.pose, m.pterm, m.feat, m.h1, m.h2, m.z3, m.dh2, m.dh1,
               m.dz3, m.loss, m.cflag, m.cpos, m.cid, m.ccount, m.cscratch, m.err};
  for (void* x : p)
    if (x) cudaFree(x);
  if (m.loss_host) cudaFreeHost(m.loss_host);
  m = Mlp();
}

void mlp_refresh_bf16(Mlp& m, cudaStream_t s) {
  k_mlp_round_w2<<<MLP_H, MLP_H, 0, s>>>(m.params, m.w2t, m.w2r);
  TGS_LAUNCHED();
}

void mlp_pose_host(const tgs_camera* hist, float out[MLP_NPOSE]) {
  const tgs_camera& c = hist[MLP_HIST - 1];
  double Rt[3][3], tt[3];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) Rt[a][b] = c.world_to_cam[4 * a + b];
    tt[a] = c.world_to_cam[4 * a + 3];
  }
  const double zf = c.zfar;
  for (int s = 0; s < MLP_HIST; ++s) {
    const tgs_camera& h = hist[s];
    double Rs[3][3], ts[3], Rr[3][3];
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) Rs[a][b] = h.world_to_cam[4 * a + b];
      ts[a] = h.world_to_cam[4 * a + 3];
    }
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Rr[a][b] = Rt[a][0] * Rs[b][0] + Rt[a][1] * Rs[b][1] + Rt[a][2] * Rs[b][2];
    float* o = out + 12 * s;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) o[3 * a + b] = (float)Rr[a][b];
    for (int a = 0; a < 3; ++a)
      o[9 + a] = (float)((tt[a] - (Rr[a][0] * ts[0] + Rr[a][1] * ts[1] + Rr[a][2] * ts[2])) / zf);
  }
}

void mlp_forward(Mlp& m, const float4* spheres, uint64_t K, const tgs_camera* hist, float* logits, bool keep,
                 cudaStream_t s) {
  TGS_CHECK(K >= 1 && K <= m.max_rows, TGS_ERR_CAPACITY, "predictor rows exceed the allocated maximum");
  const uint64_t M = (K + MLP_ROWS_PER_CTA - 1) / MLP_ROWS_PER_CTA * MLP_ROWS_PER_CTA;
  PoseVec pv;
  mlp_pose_host(hist, pv.v);
  const tgs_camera& c = hist[MLP_HIST - 1];
  DevCam dc = make_devcam(c);
  k_mlp_feat<<<div_up(M, 256), 256, 0, s>>>(spheres, K, M, dc, c.zfar, m.feat);
  TGS_LAUNCHED();
  k_mlp_pose<<<1, MLP_H, 0, s>>>(m.params, pv, m.pose, m.pterm);
  TGS_LAUNCHED();
  k_mlp_fwd_tc<<<tc_grid(M), TC_THREADS, TC_SMEM, s>>>(m.params, m.w2t, m.pterm, m.feat, M, nullptr, m.z3,
                                                       keep ? m.h1 : nullptr, keep ? m.h2 : nullptr, m.err);
  TGS_LAUNCHED();
  if (logits && logits != m.z3)
    TGS_CUDA(cudaMemcpyAsync(logits, m.z3, K * MLP_OUT * sizeof(float), cudaMemcpyDeviceToDevice, s));
}

float mlp_train_step(Mlp& m, uint64_t K, const float* labels, float pw, float lr, float wd, bool apply,
                     cudaStream_t s) {
  const uint64_t M = (K + MLP_ROWS_PER_CTA - 1) / MLP_ROWS_PER_CTA * MLP_ROWS_PER_CTA;
  TGS_CUDA(cudaMemsetAsync(m.grads, 0, MLP_NPARAM * sizeof(float), s));
  TGS_CUDA(cudaMemsetAsync(m.loss, 0, sizeof(float), s));
  const float inv = 1.f / (float)(K * MLP_OUT);
  k_mlp_dh2<<<(unsigned)M, MLP_H, 0, s>>>(m.params, m.z3, labels, m.h2, K, pw, inv, m.dz3, m.dh2, m.loss);
  TGS_LAUNCHED();
  const unsigned zc = div_up(M, 256);
  // dW3 = h2^T dz3, dW2 = h1^T dh2
  k_mlp_atb<float><<<dim3(MLP_H / 64, 1, zc), 256, 0, s>>>(m.h2, MLP_H, MLP_H, m.dz3, MLP_OUT, MLP_OUT, M,
                                                          m.grads + MLP_OFF_W3, MLP_OUT);
  TGS_LAUNCHED();
  k_mlp_atb<__nv_bfloat16><<<dim3(MLP_H / 64, MLP_H / 64, zc), 256, 0, s>>>(m.h1, MLP_H, MLP_H, m.dh2, MLP_H, MLP_H,
                                                                           M, m.grads + MLP_OFF_W2, MLP_H);
  TGS_LAUNCHED();
  k_mlp_colsum<<<dim3(1, div_up(M, 1024)), MLP_OUT, 0, s>>>(m.dz3, MLP_OUT, M, m.grads + MLP_OFF_B3);
  TGS_LAUNCHED();
  k_mlp_colsum<<<dim3(1, div_up(M, 1024)), MLP_H, 0, s>>>(m.dh2, MLP_H, M, m.grads + MLP_OFF_B2);
  TGS_LAUNCHED();
  // dh1 = dh2 W2^T masked, dW1 (block part) = feat^T dh1, db1 = colsum, dW1 (pose part) = pose x db1
  k_mlp_dh1<<<dim3((unsigned)(M / 64), MLP_H / 64), 256, 0, s>>>(m.dh2, m.w2r, m.h1, m.dh1);
  TGS_LAUNCHED();
  k_mlp_atb<float><<<dim3(1, MLP_H / 64, zc), 256, 0, s>>>(m.feat, 8, MLP_NFEAT, m.dh1, MLP_H, MLP_H, M,
                                                          m.grads + MLP_OFF_W1 + (uint64_t)MLP_NPOSE * MLP_H, MLP_H);
  TGS_LAUNCHED();
  k_mlp_colsum<<<dim3(1, div_up(M, 1024)), MLP_H, 0, s>>>(m.dh1, MLP_H, M, m.grads + MLP_OFF_B1);
  TGS_LAUNCHED();
  k_mlp_pose_grad<<<1, MLP_H, 0, s>>>(m.pose, m.grads);
  TGS_LAUNCHED();
  if (apply) {
    m.step += 1;
    const float ic1 = 1.f / (1.f - std::pow(0.9f, (float)m.step));
    const float ic2 = 1.f / (1.f - std::pow(0.999f, (float)m.step));
    k_adamw<<<div_up(MLP_NPARAM, 256), 256, 0, s>>>(m.params, m.grads, m.m, m.v, MLP_NPARAM, lr, 0.9f, 0.999f, 1e-8f,
                                                    wd, ic1, ic2);
    TGS_LAUNCHED();
    mlp_refresh_bf16(m, s);
  }
  TGS_CUDA(cudaMemcpyAsync(m.loss_host, m.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  TGS_CUDA(cudaStreamSynchronize(s));
  mlp_check(m);
  return *m.loss_host;
}

void mlp_predict_near(Mlp& m, const float4* spheres, uint64_t K, const tgs_camera* hist, float reach, uint32_t mask,
                      float thr, uint32_t* bits, cudaStream_t s) {
  TGS_CHECK(K >= 1 && K <= m.max_rows, TGS_ERR_CAPACITY, "predictor rows exceed the allocated maximum");
  const uint64_t M = (K + MLP_ROWS_PER_CTA - 1) / MLP_ROWS_PER_CTA * MLP_ROWS_PER_CTA;
  const tgs_camera& c = hist[MLP_HIST - 1];
  DevCam dc = make_devcam(c);
  PoseVec pv;
  mlp_pose_host(hist, pv.v);
  // the frustum lies inside the ball through its far corners
  const double tx = 0.5 * c.width / c.fx, ty = 0.5 * c.height / c.fy;
  const float lim = (float)(c.zfar * std::sqrt(1.0 + tx * tx + ty * ty)) + reach;
  k_mlp_cand<<<div_up(K, 256), 256, 0, s>>>(spheres, K, dc, lim, m.cflag);
  TGS_LAUNCHED();
  exclusive_scan_u32(m.cflag, m.cpos, m.ccount, K, m.cscratch, s);
  k_mlp_feat_cand<<<div_up(K, 256), 256, 0, s>>>(spheres, K, m.cflag, m.cpos, dc, c.zfar, m.feat, m.cid);
  TGS_LAUNCHED();
  k_mlp_pose<<<1, MLP_H, 0, s>>>(m.params, pv, m.pose, m.pterm);
  TGS_LAUNCHED();
  k_mlp_fwd_tc<<<tc_grid(M), TC_THREADS, TC_SMEM, s>>>(m.params, m.w2t, m.pterm, m.feat, M, m.ccount, m.z3, nullptr,
                                                       nullptr, m.err);
  TGS_LAUNCHED();
  const float zthr = std::log(thr / (1.f - thr));
  TGS_CUDA(cudaMemsetAsync(bits, 0, (K + 31) / 32 * sizeof(uint32_t), s));
  k_mlp_threshold_cand<<<div_up(K, 256), 256, 0, s>>>(m.z3, m.ccount, m.cid, mask, zthr, bits);
  TGS_LAUNCHED();
}

}  // namespace tgs
