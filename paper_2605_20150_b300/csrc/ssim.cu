// Photometric loss with the D-SSIM term of the 3DGS recipe the paper trains
// with (Sec. 4; f_i of App. A.1): (1 - lam) L1 + lam (1 - SSIM), lam = 0.2,
// SSIM per colour channel over an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2,
// averaged over every pixel and channel of the batch.
//
// Forward (k_ssim_fwd): a CTA takes a 32 x 48 tile of one channel of one
// image, stages x and y with a 5-pixel halo in shared memory, filters four
// moment maps (x, y, x^2 + y^2, xy: the two second moments enter S only
// through their sum, in B2) along rows and then columns (each thread a run of
// eight outputs, so every staged value is loaded once per run and the
// products once per input), and writes per output pixel the three partials of
// S with respect to the filtered maps m_x, E[x^2] (= the partial with respect
// to E[x^2 + y^2]) and E[xy]:
//   dS/dm_x  = 2 m_y (A2 - A1) / (B1 B2) - 2 m_x S (1/B1 - 1/B2),
//   dS/de_xx = -S / B2,    dS/de_xy = 2 A1 / (B1 B2),
// channel-planar, and adds (1 - lam)|x - y| + lam (1 - S) to the loss sum.
// Backward (k_ssim_bwd): the same tiling filters the three partial maps (the
// window is symmetric, so the adjoint of the zero-padded correlation is
// itself) and
//   dL/dx = (1 - lam) sign(x - y) / N - lam (F dm + 2 x F dxx + y F dxy) / N.
#include <cmath>

#include "raster.cuh"

namespace tgs {

namespace {

constexpr int SS_R = 5;
constexpr int SS_K = 2 * SS_R + 1;
constexpr int SS_TW = 32;               // output tile width
constexpr int SS_TH = 48;               // output tile height
constexpr int SS_HW = SS_TW + 2 * SS_R;  // 42: staged width with the halo
constexpr int SS_HH = SS_TH + 2 * SS_R;  // 58: staged height with the halo
constexpr int SS_P = SS_HW + 1;         // padded row of a staged map
constexpr int SS_Q = SS_TW + 1;         // padded row of a row-filtered map
constexpr int SS_RUN = 8;               // outputs per thread along a pass
constexpr int SS_RW = SS_TW / SS_RUN;   // row runs per staged row
constexpr int SS_THREADS = 256;         // >= SS_HH * SS_RW (row pass) and SS_TW * SS_TH / SS_RUN (column pass)
constexpr int SS_CTAS = 4;              // per SM: 64 registers a thread, about 53 KB of shared memory a CTA
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;
static_assert(SS_THREADS >= SS_HH * SS_RW && SS_THREADS >= SS_TW * SS_TH / SS_RUN, "one run per thread and pass");

struct Window {
  float w[SS_K];
};

Window gaussian_window() {
  Window g;
  double s = 0.0, v[SS_K];
  for (int k = 0; k < SS_K; ++k) {
    const double x = k - SS_R;
    v[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
    s += v[k];
  }
  for (int k = 0; k < SS_K; ++k) g.w[k] = (float)(v[k] / s);
  return g;
}

// Stages NM maps of one channel with the halo, zero outside the image, into
// t[m][SS_HH][SS_P].  Interleaved-RGB maps (stride 3, channel c) or planar.
// A thread's SS_ST elements are loaded in one batch (every load in flight at
// once) and then stored.
constexpr int SS_NST = SS_HH * SS_HW;
constexpr int SS_ST = (SS_NST + SS_THREADS - 1) / SS_THREADS;
template <int NM, bool RGB>
__device__ __forceinline__ void stage(const float* const* maps, int W, int H, int c, uint64_t plane, int x0,
                                      int y0, float* t) {
  float v[SS_ST][NM];
#pragma unroll
  for (int i = 0; i < SS_ST; ++i) {
    const int e = threadIdx.x + i * SS_THREADS;
    const int ly = e / SS_HW, lx = e - ly * SS_HW;
    const int gx = x0 + lx - SS_R, gy = y0 + ly - SS_R;
    const bool in = e < SS_NST && gx >= 0 && gx < W && gy >= 0 && gy < H;
    const uint64_t p = (uint64_t)gy * W + gx;
    const uint64_t o = RGB ? plane * 3 + p * 3 + c : plane + p;
#pragma unroll
    for (int m = 0; m < NM; ++m) v[i][m] = in ? maps[m][o] : 0.f;
  }
#pragma unroll
  for (int i = 0; i < SS_ST; ++i) {
    const int e = threadIdx.x + i * SS_THREADS;
    if (e < SS_NST) {
      const int ly = e / SS_HW, lx = e - ly * SS_HW;
#pragma unroll
      for (int m = 0; m < NM; ++m) t[(m * SS_HH + ly) * SS_P + lx] = v[i][m];
    }
  }
}

// Row pass: thread e < SS_HH * SS_RW filters SS_RUN consecutive columns of
// one staged row of NM maps, given per input column j the NM values
// (val(j, out)).
template <int NM, typename Val>
__device__ __forceinline__ void row_pass(const Window& win, float* h, Val val) {
  const int e = threadIdx.x;
  if (e >= SS_HH * SS_RW) return;
  const int ly = e / SS_RW, c0 = (e % SS_RW) * SS_RUN;
  float acc[NM][SS_RUN];
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) acc[m][i] = 0.f;
#pragma unroll
  for (int j = 0; j < SS_K + SS_RUN - 1; ++j) {
    float u[NM];
    val(ly, c0 + j, u);
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) {
      const int k = j - i;
      if (k >= 0 && k < SS_K) {
        const float wk = win.w[k];
#pragma unroll
        for (int m = 0; m < NM; ++m) acc[m][i] += wk * u[m];
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) h[(m * SS_HH + ly) * SS_Q + c0 + i] = acc[m][i];
}

// Column pass: thread tid < SS_TW * SS_TH / SS_RUN filters SS_RUN consecutive
// rows of one column of the NM row-filtered maps into out[m][i].
template <int NM>
__device__ __forceinline__ bool col_pass(const Window& win, const float* h, int& ox, int& r0,
                                         float (&out)[NM][SS_RUN]) {
  const int tid = threadIdx.x;
  if (tid >= SS_TW * SS_TH / SS_RUN) return false;
  ox = tid % SS_TW;
  r0 = (tid / SS_TW) * SS_RUN;
#pragma unroll
  for (int m = 0; m < NM; ++m)
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) out[m][i] = 0.f;
#pragma unroll
  for (int j = 0; j < SS_K + SS_RUN - 1; ++j) {
    float u[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) u[m] = h[(m * SS_HH + r0 + j) * SS_Q + ox];
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) {
      const int k = j - i;
      if (k >= 0 && k < SS_K) {
        const float wk = win.w[k];
#pragma unroll
        for (int m = 0; m < NM; ++m) out[m][i] += wk * u[m];
      }
    }
  }
  return true;
}

__global__ void __launch_bounds__(SS_THREADS, SS_CTAS) k_ssim_fwd(const float* __restrict__ x, const float* __restrict__ y,
                                                        int W, int H, Window win, float lam,
                                                        float* __restrict__ dm, float* __restrict__ dxx,
                                                        float* __restrict__ dxy, float* __restrict__ loss_sum) {
  extern __shared__ float smem[];
  float* t = smem;                      // 2 x SS_HH x SS_P
  float* h = smem + 2 * SS_HH * SS_P;   // 4 x SS_HH x SS_Q
  __shared__ float red[SS_THREADS / 32];
  const int c = blockIdx.z % 3, img = blockIdx.z / 3;
  const uint64_t hw = (uint64_t)H * W;
  const int x0 = blockIdx.x * SS_TW, y0 = blockIdx.y * SS_TH;
  const float* maps[2] = {x, y};
  stage<2, true>(maps, W, H, c, (uint64_t)img * hw, x0, y0, t);
  __syncthreads();
  // maps: x, y, x^2 + y^2, xy
  row_pass<4>(win, h, [&](int ly, int lx, float (&u)[4]) {
    const float a = t[ly * SS_P + lx], b = t[(SS_HH + ly) * SS_P + lx];
    u[0] = a;
    u[1] = b;
    u[2] = a * a + b * b;
    u[3] = a * b;
  });
  __syncthreads();
  float acc = 0.f;
  int ox, r0;
  float f[4][SS_RUN];
  if (col_pass<4>(win, h, ox, r0, f)) {
    const int gx = x0 + ox;
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) {
      const int oy = r0 + i, gy = y0 + oy;
      if (gx < W && gy < H) {
        const float mx = f[0][i], my = f[1][i];
        const float A1 = 2.f * mx * my + SS_C1, A2 = 2.f * (f[3][i] - mx * my) + SS_C2;
        const float B1 = mx * mx + my * my + SS_C1;
        const float B2 = (f[2][i] - mx * mx - my * my) + SS_C2;
        const float iB1 = 1.f / B1, iB2 = 1.f / B2;
        const float iB12 = iB1 * iB2;
        const float S = A1 * A2 * iB12;
        const uint64_t o = ((uint64_t)img * 3 + c) * hw + (uint64_t)gy * W + gx;
        dm[o] = 2.f * my * (A2 - A1) * iB12 - 2.f * mx * S * (iB1 - iB2);
        dxx[o] = -S * iB2;
        dxy[o] = 2.f * A1 * iB12;
        const float xv = t[(oy + SS_R) * SS_P + ox + SS_R], yv = t[(SS_HH + oy + SS_R) * SS_P + ox + SS_R];
        acc += (1.f - lam) * fabsf(xv - yv) + lam * (1.f - S);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int k = 0; k < SS_THREADS / 32; ++k) s += red[k];
    atomicAdd(loss_sum, s);
  }
}

__global__ void __launch_bounds__(SS_THREADS, SS_CTAS) k_ssim_bwd(const float* __restrict__ x, const float* __restrict__ y,
                                                        int W, int H, Window win, float lam, float inv_n,
                                                        const float* __restrict__ dm,
                                                        const float* __restrict__ dxx,
                                                        const float* __restrict__ dxy, float* __restrict__ grad) {
  extern __shared__ float smem[];
  float* t = smem;                      // 3 x SS_HH x SS_P
  float* h = smem + 3 * SS_HH * SS_P;   // 3 x SS_HH x SS_Q
  const int c = blockIdx.z % 3, img = blockIdx.z / 3;
  const uint64_t hw = (uint64_t)H * W;
  const int x0 = blockIdx.x * SS_TW, y0 = blockIdx.y * SS_TH;
  const float* maps[3] = {dm, dxx, dxy};
  stage<3, false>(maps, W, H, c, ((uint64_t)img * 3 + c) * hw, x0, y0, t);
  __syncthreads();
  row_pass<3>(win, h, [&](int ly, int lx, float (&u)[3]) {
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m] = t[(m * SS_HH + ly) * SS_P + lx];
  });
  __syncthreads();
  int ox, r0;
  float f[3][SS_RUN];
  if (!col_pass<3>(win, h, ox, r0, f)) return;
  const int gx = x0 + ox;
#pragma unroll
  for (int i = 0; i < SS_RUN; ++i) {
    const int gy = y0 + r0 + i;
    if (gx < W && gy < H) {
      const uint64_t o = ((uint64_t)img * hw + (uint64_t)gy * W + gx) * 3 + c;
      const float xv = x[o], yv = y[o], dd = xv - yv;
      const float gl1 = dd > 0.f ? inv_n : (dd < 0.f ? -inv_n : 0.f);
      grad[o] = (1.f - lam) * gl1 - lam * (f[0][i] + 2.f * xv * f[1][i] + yv * f[2][i]) * inv_n;
    }
  }
}

constexpr size_t SS_FWD_SMEM = (2 * SS_HH * SS_P + 4 * SS_HH * SS_Q) * sizeof(float);
constexpr size_t SS_BWD_SMEM = (3 * SS_HH * SS_P + 3 * SS_HH * SS_Q) * sizeof(float);

}  // namespace

void photometric_loss_ssim(const float* img, const float* target, int J, int W, int H, float* grad, float* loss_sum,
                           float* scratch, cudaStream_t s) {
  if (J <= 0 || W <= 0 || H <= 0) return;
  static int attrs_dev = -1;
  int dev = 0;
  TGS_CUDA(cudaGetDevice(&dev));
  if (attrs_dev != dev) {
    TGS_CUDA(cudaFuncSetAttribute(k_ssim_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS_FWD_SMEM));
    TGS_CUDA(cudaFuncSetAttribute(k_ssim_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SS_BWD_SMEM));
    attrs_dev = dev;
  }
  const uint64_t n = (uint64_t)J * W * H * 3;
  const Window win = gaussian_window();
  const float lam = 0.2f;
  const dim3 grid(div_up(W, SS_TW), div_up(H, SS_TH), 3 * J);
  float *dm = scratch, *dxx = scratch + n, *dxy = scratch + 2 * n;
  k_ssim_fwd<<<grid, SS_THREADS, SS_FWD_SMEM, s>>>(img, target, W, H, win, lam, dm, dxx, dxy, loss_sum);
  TGS_LAUNCHED();
  k_ssim_bwd<<<grid, SS_THREADS, SS_BWD_SMEM, s>>>(img, target, W, H, win, lam, 1.f / (float)n, dm, dxx, dxy, grad);
  TGS_LAUNCHED();
}

}  // namespace tgs
