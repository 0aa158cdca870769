// Learned block-prefetch predictor on the GPU.
//
// Inference (every step of the learned-prefetch mode) is one fused kernel per
// 64 block rows: layer 1 (the pose part is a shared 96 x 256 product computed
// once per step; the per-block part has 6 inputs) in FP32 into a BF16 tile in
// shared memory, layer 2 (256 x 256) on the tensor cores with BF16 mma.sync
// and FP32 accumulation, and layer 3 (256 x 4) plus bias folded into the
// epilogue with quad shuffles.  Training kernels (offline, on logged
// visibility) are FP32 SIMT: BCE gradient, the two 256-wide products of the
// backward, column sums, and AdamW on FP32 master weights.
#include <cmath>
#include <random>
#include <vector>

#include "predictor.cuh"
#include "sort.cuh"

namespace tgs {
namespace {

constexpr int W2S = MLP_H + 8;  // padded shared-memory row (bf16 elements)

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

__device__ __forceinline__ void mma_bf16(float* d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 64 rows per CTA, 4 warps of 16 rows; shared: W2^T bf16 [256][264], h1 bf16
// [64][264], W1 block part [6][256], pose term, b2, W3 [256][4], b3, features.
__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ P, const __nv_bfloat16* __restrict__ w2t,
                                                const float* __restrict__ pterm, const float* __restrict__ feat,
                                                uint64_t M, float* __restrict__ z3, __nv_bfloat16* __restrict__ h1g,
                                                float* __restrict__ h2g, const uint32_t* __restrict__ rows_dev) {
  // rows_dev (device, may be null): only the first *rows_dev rows are wanted
  if (rows_dev && (uint64_t)blockIdx.x * MLP_ROWS_PER_CTA >= *rows_dev) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* w2s = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* h1s = w2s + MLP_H * W2S;
  float* w1b = reinterpret_cast<float*>(h1s + MLP_ROWS_PER_CTA * W2S);
  float* pt = w1b + MLP_NFEAT * MLP_H;
  float* b2 = pt + MLP_H;
  float* w3 = b2 + MLP_H;
  float* b3 = w3 + MLP_H * MLP_OUT;
  float* fs = b3 + 4;
  const int tid = threadIdx.x;
  const uint64_t row0 = (uint64_t)blockIdx.x * MLP_ROWS_PER_CTA;
  // stage weights
  for (int e = tid; e < MLP_H * MLP_H / 8; e += 128) {
    int n = e / (MLP_H / 8), k8 = e % (MLP_H / 8);
    *reinterpret_cast<uint4*>(w2s + n * W2S + 8 * k8) = *reinterpret_cast<const uint4*>(w2t + (uint64_t)n * MLP_H + 8 * k8);
  }
  for (int e = tid; e < MLP_NFEAT * MLP_H; e += 128) w1b[e] = P[MLP_OFF_W1 + (uint64_t)MLP_NPOSE * MLP_H + e];
  for (int e = tid; e < MLP_H; e += 128) {
    pt[e] = pterm[e];
    b2[e] = P[MLP_OFF_B2 + e];
  }
  for (int e = tid; e < MLP_H * MLP_OUT; e += 128) w3[e] = P[MLP_OFF_W3 + e];
  if (tid < 4) b3[tid] = P[MLP_OFF_B3 + tid];
  for (int e = tid; e < MLP_ROWS_PER_CTA * 8; e += 128) fs[e] = feat[row0 * 8 + e];
  __syncthreads();
  // layer 1
  for (int e = tid; e < MLP_ROWS_PER_CTA * MLP_H; e += 128) {
    const int r = e / MLP_H, j = e % MLP_H;
    float z = pt[j];
#pragma unroll
    for (int i = 0; i < MLP_NFEAT; ++i) z += fs[r * 8 + i] * w1b[i * MLP_H + j];
    __nv_bfloat16 h = __float2bfloat16_rn(fmaxf(z, 0.f));
    h1s[r * W2S + j] = h;
    if (h1g) h1g[(row0 + r) * MLP_H + j] = h;
  }
  __syncthreads();
  // layer 2 on the tensor cores
  const int w = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
  float acc[MLP_H / 8][4];
#pragma unroll
  for (int nt = 0; nt < MLP_H / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
  const __nv_bfloat16* ar0 = h1s + (16 * w + g) * W2S;
  const __nv_bfloat16* ar8 = ar0 + 8 * W2S;
#pragma unroll 1
  for (int k0 = 0; k0 < MLP_H; k0 += 16) {
    const uint32_t a0 = *reinterpret_cast<const uint32_t*>(ar0 + k0 + 2 * q);
    const uint32_t a1 = *reinterpret_cast<const uint32_t*>(ar8 + k0 + 2 * q);
    const uint32_t a2 = *reinterpret_cast<const uint32_t*>(ar0 + k0 + 8 + 2 * q);
    const uint32_t a3 = *reinterpret_cast<const uint32_t*>(ar8 + k0 + 8 + 2 * q);
#pragma unroll
    for (int nt = 0; nt < MLP_H / 8; ++nt) {
      const __nv_bfloat16* br = w2s + (8 * nt + g) * W2S + k0;
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(br + 2 * q);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(br + 8 + 2 * q);
      mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
    }
  }
  // epilogue: bias + ReLU, layer 3 folded in
  float lz[2][MLP_OUT] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  const uint64_t ra = row0 + 16 * w + g, rb = ra + 8;
#pragma unroll
  for (int nt = 0; nt < MLP_H / 8; ++nt) {
    const int col = 8 * nt + 2 * q;
    const float h00 = fmaxf(acc[nt][0] + b2[col], 0.f), h01 = fmaxf(acc[nt][1] + b2[col + 1], 0.f);
    const float h10 = fmaxf(acc[nt][2] + b2[col], 0.f), h11 = fmaxf(acc[nt][3] + b2[col + 1], 0.f);
    if (h2g) {
      *reinterpret_cast<float2*>(h2g + ra * MLP_H + col) = make_float2(h00, h01);
      *reinterpret_cast<float2*>(h2g + rb * MLP_H + col) = make_float2(h10, h11);
    }
#pragma unroll
    for (int h = 0; h < MLP_OUT; ++h) {
      lz[0][h] += h00 * w3[col * MLP_OUT + h] + h01 * w3[(col + 1) * MLP_OUT + h];
      lz[1][h] += h10 * w3[col * MLP_OUT + h] + h11 * w3[(col + 1) * MLP_OUT + h];
    }
  }
#pragma unroll
  for (int h = 0; h < MLP_OUT; ++h) {
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
      lz[0][h] += __shfl_xor_sync(0xffffffffu, lz[0][h], o);
      lz[1][h] += __shfl_xor_sync(0xffffffffu, lz[1][h], o);
    }
  }
  if (q == 0) {
#pragma unroll
    for (int h = 0; h < MLP_OUT; ++h) {
      z3[ra * MLP_OUT + h] = lz[0][h] + b3[h];
      z3[rb * MLP_OUT + h] = lz[1][h] + b3[h];
    }
  }
}

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

__global__ void k_mlp_threshold(const float* __restrict__ z3, uint64_t K, uint32_t mask, float zthr,
                                uint32_t* __restrict__ bits, uint64_t words) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool vis = false;
  if (k < K)
#pragma unroll
    for (int h = 0; h < MLP_OUT; ++h)
      if ((mask >> h & 1u) && z3[k * MLP_OUT + h] > zthr) vis = true;
  const uint32_t wd = __ballot_sync(0xffffffffu, vis);
  if ((threadIdx.x & 31) == 0 && (k >> 5) < words) bits[k >> 5] = wd;
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

size_t fwd_smem_bytes() {
  return (size_t)MLP_H * W2S * 2 + (size_t)MLP_ROWS_PER_CTA * W2S * 2 +
         sizeof(float) * (MLP_NFEAT * MLP_H + MLP_H + MLP_H + MLP_H * MLP_OUT + 4 + MLP_ROWS_PER_CTA * 8);
}

}  // namespace

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
  TGS_CUDA(cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem_bytes()));
  mlp_refresh_bf16(m, 0);
  TGS_CUDA(cudaDeviceSynchronize());
}

void mlp_free(Mlp& m) {
  void* p[] = {m.params, m.grads, m.m, m.v, m.w2t, m.w2r, m.pose, m.pterm, m.feat, m.h1, m.h2, m.z3, m.dh2, m.dh1,
               m.dz3, m.loss, m.cflag, m.cpos, m.cid, m.ccount, m.cscratch};
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
  k_mlp_fwd<<<(unsigned)(M / MLP_ROWS_PER_CTA), 128, fwd_smem_bytes(), s>>>(
      m.params, m.w2t, m.pterm, m.feat, M, m.z3, keep ? m.h1 : nullptr, keep ? m.h2 : nullptr, nullptr);
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
  k_mlp_fwd<<<(unsigned)(M / MLP_ROWS_PER_CTA), 128, fwd_smem_bytes(), s>>>(m.params, m.w2t, m.pterm, m.feat, M, m.z3,
                                                                            nullptr, nullptr, m.ccount);
  TGS_LAUNCHED();
  const float zthr = std::log(thr / (1.f - thr));
  TGS_CUDA(cudaMemsetAsync(bits, 0, (K + 31) / 32 * sizeof(uint32_t), s));
  k_mlp_threshold_cand<<<div_up(K, 256), 256, 0, s>>>(m.z3, m.ccount, m.cid, mask, zthr, bits);
  TGS_LAUNCHED();
}

void mlp_threshold(const float* logits, uint64_t K, uint32_t mask, float thr, uint32_t* bits, cudaStream_t s) {
  const float zthr = std::log(thr / (1.f - thr));
  const uint64_t words = (K + 31) / 32;
  k_mlp_threshold<<<div_up(words * 32, 256), 256, 0, s>>>(logits, K, mask, zthr, bits, words);
  TGS_LAUNCHED();
}

}  // namespace tgs
