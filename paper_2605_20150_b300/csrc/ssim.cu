// Photometric loss with the D-SSIM term of the 3DGS recipe the paper trains
// with (Sec. 4; f_i of App. A.1): (1 - lam) L1 + lam (1 - SSIM), lam = 0.2,
// SSIM per colour channel over an 11 x 11 Gaussian window (sigma 1.5,
// normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2,
// averaged over every pixel and channel of the batch.
//
// Forward (k_ssim_fwd): a CTA takes a 32 x 32 tile of one channel of one
// image, stages x and y with a 5-pixel halo in shared memory, filters the five
// moment maps (x, y, x^2, y^2, xy) along rows and then columns (each thread a
// run of four outputs, so every staged value is loaded once per run and the
// products once per input), and writes per output pixel the three partials
// of S with respect to the filtered maps m_x, E[x^2], E[xy]:
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
constexpr int SS_T = 32;               // output tile side
constexpr int SS_H = SS_T + 2 * SS_R;  // 42: staged side with the halo
constexpr int SS_P = SS_H + 1;         // padded row of a staged map
constexpr int SS_Q = SS_T + 1;         // padded row of a row-filtered map
constexpr int SS_RUN = 4;              // outputs per thread along a pass
constexpr int SS_THREADS = 256;
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

// Stages NM maps of one channel with the halo, zero outside the image, into
// t[m][SS_H][SS_P].  Interleaved-RGB maps (stride 3, channel c) or planar.
template <int NM, bool RGB>
__device__ __forceinline__ void stage(const float* const* maps, int W, int H, int c, uint64_t plane, int x0,
                                      int y0, float* t) {
  for (int e = threadIdx.x; e < SS_H * SS_H; e += SS_THREADS) {
    const int ly = e / SS_H, lx = e - ly * SS_H;
    const int gx = x0 + lx - SS_R, gy = y0 + ly - SS_R;
    const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
    const uint64_t p = (uint64_t)gy * W + gx;
    const uint64_t o = RGB ? plane * 3 + p * 3 + c : plane + p;
#pragma unroll
    for (int m = 0; m < NM; ++m) t[(m * SS_H + ly) * SS_P + lx] = in ? maps[m][o] : 0.f;
  }
}

__global__ void __launch_bounds__(SS_THREADS) k_ssim_fwd(const float* __restrict__ x, const float* __restrict__ y,
                                                        int W, int H, Window win, float lam,
                                                        float* __restrict__ dm, float* __restrict__ dxx,
                                                        float* __restrict__ dxy, float* __restrict__ loss_sum) {
  __shared__ float t[2 * SS_H * SS_P];
  __shared__ float h[5 * SS_H * SS_Q];
  __shared__ float red[SS_THREADS / 32];
  const int c = blockIdx.z % 3, img = blockIdx.z / 3;
  const uint64_t hw = (uint64_t)H * W;
  const int x0 = blockIdx.x * SS_T, y0 = blockIdx.y * SS_T;
  const float* maps[2] = {x, y};
  stage<2, true>(maps, W, H, c, (uint64_t)img * hw, x0, y0, t);
  __syncthreads();
  // rows: a thread filters SS_RUN consecutive columns of one staged row
  for (int e = threadIdx.x; e < SS_H * (SS_T / SS_RUN); e += SS_THREADS) {
    const int ly = e / (SS_T / SS_RUN), c0 = (e % (SS_T / SS_RUN)) * SS_RUN;
    const float* tx = t + ly * SS_P + c0;
    const float* ty = t + (SS_H + ly) * SS_P + c0;
    float a[SS_RUN], b[SS_RUN], aa[SS_RUN], bb[SS_RUN], ab[SS_RUN];
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) a[i] = b[i] = aa[i] = bb[i] = ab[i] = 0.f;
#pragma unroll
    for (int j = 0; j < SS_K + SS_RUN - 1; ++j) {
      const float u = tx[j], v = ty[j];
      const float uu = u * u, vv = v * v, uv = u * v;
#pragma unroll
      for (int i = 0; i < SS_RUN; ++i) {
        const int k = j - i;
        if (k >= 0 && k < SS_K) {
          const float wk = win.w[k];
          a[i] += wk * u;
          b[i] += wk * v;
          aa[i] += wk * uu;
          bb[i] += wk * vv;
          ab[i] += wk * uv;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) {
      h[(0 * SS_H + ly) * SS_Q + c0 + i] = a[i];
      h[(1 * SS_H + ly) * SS_Q + c0 + i] = b[i];
      h[(2 * SS_H + ly) * SS_Q + c0 + i] = aa[i];
      h[(3 * SS_H + ly) * SS_Q + c0 + i] = bb[i];
      h[(4 * SS_H + ly) * SS_Q + c0 + i] = ab[i];
    }
  }
  __syncthreads();
  // columns: a thread filters SS_RUN consecutive rows of one column
  float acc = 0.f;
  {
    const int ox = threadIdx.x % SS_T, r0 = (threadIdx.x / SS_T) * SS_RUN;  // SS_THREADS == SS_T * SS_T / SS_RUN
    float mx[SS_RUN], my[SS_RUN], exx[SS_RUN], eyy[SS_RUN], exy[SS_RUN];
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) mx[i] = my[i] = exx[i] = eyy[i] = exy[i] = 0.f;
#pragma unroll
    for (int j = 0; j < SS_K + SS_RUN - 1; ++j) {
      const int ly = r0 + j;
      const float h0 = h[(0 * SS_H + ly) * SS_Q + ox], h1 = h[(1 * SS_H + ly) * SS_Q + ox];
      const float h2 = h[(2 * SS_H + ly) * SS_Q + ox], h3 = h[(3 * SS_H + ly) * SS_Q + ox];
      const float h4 = h[(4 * SS_H + ly) * SS_Q + ox];
#pragma unroll
      for (int i = 0; i < SS_RUN; ++i) {
        const int k = j - i;
        if (k >= 0 && k < SS_K) {
          const float wk = win.w[k];
          mx[i] += wk * h0;
          my[i] += wk * h1;
          exx[i] += wk * h2;
          eyy[i] += wk * h3;
          exy[i] += wk * h4;
        }
      }
    }
    const int gx = x0 + ox;
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) {
      const int oy = r0 + i, gy = y0 + oy;
      if (gx < W && gy < H) {
        const float A1 = 2.f * mx[i] * my[i] + SS_C1, A2 = 2.f * (exy[i] - mx[i] * my[i]) + SS_C2;
        const float B1 = mx[i] * mx[i] + my[i] * my[i] + SS_C1;
        const float B2 = (exx[i] - mx[i] * mx[i]) + (eyy[i] - my[i] * my[i]) + SS_C2;
        const float iB12 = 1.f / (B1 * B2);
        const float S = A1 * A2 * iB12;
        const uint64_t o = ((uint64_t)img * 3 + c) * hw + (uint64_t)gy * W + gx;
        dm[o] = 2.f * my[i] * (A2 - A1) * iB12 - 2.f * mx[i] * S * (1.f / B1 - 1.f / B2);
        dxx[o] = -S / B2;
        dxy[o] = 2.f * A1 * iB12;
        const float xv = t[(oy + SS_R) * SS_P + ox + SS_R], yv = t[(SS_H + oy + SS_R) * SS_P + ox + SS_R];
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

__global__ void __launch_bounds__(SS_THREADS) k_ssim_bwd(const float* __restrict__ x, const float* __restrict__ y,
                                                        int W, int H, Window win, float lam, float inv_n,
                                                        const float* __restrict__ dm,
                                                        const float* __restrict__ dxx,
                                                        const float* __restrict__ dxy, float* __restrict__ grad) {
  __shared__ float t[3 * SS_H * SS_P];
  __shared__ float h[3 * SS_H * SS_Q];
  const int c = blockIdx.z % 3, img = blockIdx.z / 3;
  const uint64_t hw = (uint64_t)H * W;
  const int x0 = blockIdx.x * SS_T, y0 = blockIdx.y * SS_T;
  const float* maps[3] = {dm, dxx, dxy};
  stage<3, false>(maps, W, H, c, ((uint64_t)img * 3 + c) * hw, x0, y0, t);
  __syncthreads();
  for (int e = threadIdx.x; e < SS_H * (SS_T / SS_RUN); e += SS_THREADS) {
    const int ly = e / (SS_T / SS_RUN), c0 = (e % (SS_T / SS_RUN)) * SS_RUN;
    float a[SS_RUN], b[SS_RUN], d[SS_RUN];
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) a[i] = b[i] = d[i] = 0.f;
#pragma unroll
    for (int j = 0; j < SS_K + SS_RUN - 1; ++j) {
      const float u0 = t[(0 * SS_H + ly) * SS_P + c0 + j], u1 = t[(1 * SS_H + ly) * SS_P + c0 + j];
      const float u2 = t[(2 * SS_H + ly) * SS_P + c0 + j];
#pragma unroll
      for (int i = 0; i < SS_RUN; ++i) {
        const int k = j - i;
        if (k >= 0 && k < SS_K) {
          const float wk = win.w[k];
          a[i] += wk * u0;
          b[i] += wk * u1;
          d[i] += wk * u2;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) {
      h[(0 * SS_H + ly) * SS_Q + c0 + i] = a[i];
      h[(1 * SS_H + ly) * SS_Q + c0 + i] = b[i];
      h[(2 * SS_H + ly) * SS_Q + c0 + i] = d[i];
    }
  }
  __syncthreads();
  const int ox = threadIdx.x % SS_T, r0 = (threadIdx.x / SS_T) * SS_RUN;
  float fm[SS_RUN], fxx[SS_RUN], fxy[SS_RUN];
#pragma unroll
  for (int i = 0; i < SS_RUN; ++i) fm[i] = fxx[i] = fxy[i] = 0.f;
#pragma unroll
  for (int j = 0; j < SS_K + SS_RUN - 1; ++j) {
    const int ly = r0 + j;
    const float h0 = h[(0 * SS_H + ly) * SS_Q + ox], h1 = h[(1 * SS_H + ly) * SS_Q + ox];
    const float h2 = h[(2 * SS_H + ly) * SS_Q + ox];
#pragma unroll
    for (int i = 0; i < SS_RUN; ++i) {
      const int k = j - i;
      if (k >= 0 && k < SS_K) {
        const float wk = win.w[k];
        fm[i] += wk * h0;
        fxx[i] += wk * h1;
        fxy[i] += wk * h2;
      }
    }
  }
  const int gx = x0 + ox;
#pragma unroll
  for (int i = 0; i < SS_RUN; ++i) {
    const int gy = y0 + r0 + i;
    if (gx < W && gy < H) {
      const uint64_t o = ((uint64_t)img * hw + (uint64_t)gy * W + gx) * 3 + c;
      const float xv = x[o], yv = y[o], dd = xv - yv;
      const float gl1 = dd > 0.f ? inv_n : (dd < 0.f ? -inv_n : 0.f);
      grad[o] = (1.f - lam) * gl1 - lam * (fm[i] + 2.f * xv * fxx[i] + yv * fxy[i]) * inv_n;
    }
  }
}

}  // namespace

void photometric_loss_ssim(const float* img, const float* target, int J, int W, int H, float* grad, float* loss_sum,
                           float* scratch, cudaStream_t s) {
  if (J <= 0 || W <= 0 || H <= 0) return;
  const uint64_t n = (uint64_t)J * W * H * 3;
  const Window win = gaussian_window();
  const float lam = 0.2f;
  static_assert(SS_THREADS == SS_T * SS_T / SS_RUN, "one column run per thread");
  const dim3 grid(div_up(W, SS_T), div_up(H, SS_T), 3 * J);
  float *dm = scratch, *dxx = scratch + n, *dxy = scratch + 2 * n;
  k_ssim_fwd<<<grid, SS_THREADS, 0, s>>>(img, target, W, H, win, lam, dm, dxx, dxy, loss_sum);
  TGS_LAUNCHED();
  k_ssim_bwd<<<grid, SS_THREADS, 0, s>>>(img, target, W, H, win, lam, 1.f / (float)n, dm, dxx, dxy, grad);
  TGS_LAUNCHED();
}

}  // namespace tgs
