// Photometric loss with the D-SSIM term of the 3DGS recipe the paper trains
// with (Sec. 4; f_i of App. A.1): (1 - lam) L1 + lam (1 - SSIM), lam = 0.2,
// SSIM per colour channel over an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2,
// averaged over every pixel and channel of the batch.
//
// Forward (k_ssim_fwd): a CTA stages an input tile of one channel of one image
// with a 5-pixel halo in shared memory, filters the five moment maps (x, y,
// x^2, y^2, xy) along rows and then columns, and writes per output pixel the
// three partials of S with respect to the filtered maps m_x, E[x^2], E[xy]:
//   dS/dm_x  = 2 m_y (A2 - A1) / (B1 B2) - 2 m_x S (1/B1 - 1/B2),
//   dS/de_xx = -S / B2,    dS/de_xy = 2 A1 / (B1 B2),
// and adds (1 - lam)|x - y| + lam (1 - S) to the loss sum.  Backward
// (k_ssim_bwd): the same tiling filters the three partial maps (the window is
// symmetric, so the adjoint of the zero-padded correlation is itself) and
//   dL/dx = (1 - lam) sign(x - y) / N - lam (F dm + 2 x F dxx + y F dxy) / N.
#include <cmath>

#include "raster.cuh"

namespace tgs {

namespace {

constexpr int SS_R = 5;
constexpr int SS_K = 2 * SS_R + 1;
constexpr int SS_TX = 32, SS_TY = 16;
constexpr int SS_HX = SS_TX + 2 * SS_R, SS_HY = SS_TY + 2 * SS_R;  // 42 x 26
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;

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

// Loads nmap maps of one channel of one image (interleaved RGB) with the halo,
// zero outside the image, into t[m][HY][HX].
template <int NM>
__device__ __forceinline__ void load_tile(const float* const* maps, int W, int H, int c, uint64_t img_off,
                                          int x0, int y0, float (*t)[SS_HY][SS_HX]) {
  for (int e = threadIdx.y * blockDim.x + threadIdx.x; e < SS_HX * SS_HY; e += blockDim.x * blockDim.y) {
    const int ly = e / SS_HX, lx = e - ly * SS_HX;
    const int gx = x0 + lx - SS_R, gy = y0 + ly - SS_R;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const uint64_t o = img_off + ((uint64_t)gy * W + gx) * 3 + c;
#pragma unroll
    for (int m = 0; m < NM; ++m) t[m][ly][lx] = in ? maps[m][o] : 0.f;
  }
}

__global__ void __launch_bounds__(256) k_ssim_fwd(const float* __restrict__ x, const float* __restrict__ y, int W,
                                                  int H, Window win, float lam, float* __restrict__ dm,
                                                  float* __restrict__ dxx, float* __restrict__ dxy,
                                                  float* __restrict__ loss_sum) {
  __shared__ float t[2][SS_HY][SS_HX];
  __shared__ float h[5][SS_HY][SS_TX];
  __shared__ float red[8];
  const int c = blockIdx.z % 3;
  const uint64_t img_off = (uint64_t)(blockIdx.z / 3) * H * W * 3;
  const int x0 = blockIdx.x * SS_TX, y0 = blockIdx.y * SS_TY;
  const float* maps[2] = {x, y};
  load_tile<2>(maps, W, H, c, img_off, x0, y0, t);
  __syncthreads();
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  // rows: the five moment maps filtered along x
  for (int e = tid; e < SS_HY * SS_TX; e += nt) {
    const int ly = e / SS_TX, lx = e - ly * SS_TX;
    float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
    for (int k = 0; k < SS_K; ++k) {
      const float wk = win.w[k], u = t[0][ly][lx + k], v = t[1][ly][lx + k];
      a += wk * u;
      b += wk * v;
      aa += wk * u * u;
      bb += wk * v * v;
      ab += wk * u * v;
    }
    h[0][ly][lx] = a;
    h[1][ly][lx] = b;
    h[2][ly][lx] = aa;
    h[3][ly][lx] = bb;
    h[4][ly][lx] = ab;
  }
  __syncthreads();
  float acc = 0.f;
  for (int e = tid; e < SS_TY * SS_TX; e += nt) {
    const int oy = e / SS_TX, ox = e - oy * SS_TX;
    const int gx = x0 + ox, gy = y0 + oy;
    if (gx >= W || gy >= H) continue;
    float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
    for (int k = 0; k < SS_K; ++k) {
      const float wk = win.w[k];
      mx += wk * h[0][oy + k][ox];
      my += wk * h[1][oy + k][ox];
      exx += wk * h[2][oy + k][ox];
      eyy += wk * h[3][oy + k][ox];
      exy += wk * h[4][oy + k][ox];
    }
    const float A1 = 2.f * mx * my + SS_C1, A2 = 2.f * (exy - mx * my) + SS_C2;
    const float B1 = mx * mx + my * my + SS_C1, B2 = (exx - mx * mx) + (eyy - my * my) + SS_C2;
    const float iB12 = 1.f / (B1 * B2);
    const float S = A1 * A2 * iB12;
    const uint64_t o = img_off + ((uint64_t)gy * W + gx) * 3 + c;
    dm[o] = 2.f * my * (A2 - A1) * iB12 - 2.f * mx * S * (1.f / B1 - 1.f / B2);
    dxx[o] = -S / B2;
    dxy[o] = 2.f * A1 * iB12;
    acc += (1.f - lam) * fabsf(t[0][oy + SS_R][ox + SS_R] - t[1][oy + SS_R][ox + SS_R]) + lam * (1.f - S);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int k = 0; k < nt / 32; ++k) s += red[k];
    atomicAdd(loss_sum, s);
  }
}

__global__ void __launch_bounds__(256) k_ssim_bwd(const float* __restrict__ x, const float* __restrict__ y, int W,
                                                  int H, Window win, float lam, float inv_n,
                                                  const float* __restrict__ dm, const float* __restrict__ dxx,
                                                  const float* __restrict__ dxy, float* __restrict__ grad) {
  __shared__ float t[3][SS_HY][SS_HX];
  __shared__ float h[3][SS_HY][SS_TX];
  const int c = blockIdx.z % 3;
  const uint64_t img_off = (uint64_t)(blockIdx.z / 3) * H * W * 3;
  const int x0 = blockIdx.x * SS_TX, y0 = blockIdx.y * SS_TY;
  const float* maps[3] = {dm, dxx, dxy};
  load_tile<3>(maps, W, H, c, img_off, x0, y0, t);
  __syncthreads();
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int e = tid; e < SS_HY * SS_TX; e += nt) {
    const int ly = e / SS_TX, lx = e - ly * SS_TX;
    float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
    for (int k = 0; k < SS_K; ++k) {
      const float wk = win.w[k];
      a += wk * t[0][ly][lx + k];
      b += wk * t[1][ly][lx + k];
      d += wk * t[2][ly][lx + k];
    }
    h[0][ly][lx] = a;
    h[1][ly][lx] = b;
    h[2][ly][lx] = d;
  }
  __syncthreads();
  for (int e = tid; e < SS_TY * SS_TX; e += nt) {
    const int oy = e / SS_TX, ox = e - oy * SS_TX;
    const int gx = x0 + ox, gy = y0 + oy;
    if (gx >= W || gy >= H) continue;
    float fm = 0.f, fxx = 0.f, fxy = 0.f;
#pragma unroll
    for (int k = 0; k < SS_K; ++k) {
      const float wk = win.w[k];
      fm += wk * h[0][oy + k][ox];
      fxx += wk * h[1][oy + k][ox];
      fxy += wk * h[2][oy + k][ox];
    }
    const uint64_t o = img_off + ((uint64_t)gy * W + gx) * 3 + c;
    const float xv = x[o], yv = y[o], d = xv - yv;
    const float gl1 = d > 0.f ? inv_n : (d < 0.f ? -inv_n : 0.f);
    grad[o] = (1.f - lam) * gl1 - lam * (fm + 2.f * xv * fxx + yv * fxy) * inv_n;
  }
}

}  // namespace

void photometric_loss_ssim(const float* img, const float* target, int J, int W, int H, float* grad, float* loss_sum,
                           float* scratch, cudaStream_t s) {
  if (J <= 0 || W <= 0 || H <= 0) return;
  const uint64_t n = (uint64_t)J * W * H * 3;
  const Window win = gaussian_window();
  const float lam = 0.2f;
  const dim3 grid(div_up(W, SS_TX), div_up(H, SS_TY), 3 * J), block(32, 8);
  float *dm = scratch, *dxx = scratch + n, *dxy = scratch + 2 * n;
  k_ssim_fwd<<<grid, block, 0, s>>>(img, target, W, H, win, lam, dm, dxx, dxy, loss_sum);
  TGS_LAUNCHED();
  k_ssim_bwd<<<grid, block, 0, s>>>(img, target, W, H, win, lam, 1.f / (float)n, dm, dxx, dxy, grad);
  TGS_LAUNCHED();
}

}  // namespace tgs
