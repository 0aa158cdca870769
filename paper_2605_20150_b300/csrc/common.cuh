// Common definitions of the sm_103a TideGS library: error handling, the
// device camera, launch bookkeeping and the exact FP32 helpers of the key path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <stdexcept>
#include <string>

#include "tidegs.h"

namespace tgs {

constexpr int D = TGS_D;          // 59 floats per Gaussian row
constexpr int TILE = TGS_TILE;    // 16 x 16 pixel tiles
constexpr int TILE_PIX = TILE * TILE;
constexpr float ALPHA_MIN = 1.0f / 255.0f;
constexpr float ALPHA_MAX = 0.99f;
constexpr float T_STOP = 1e-4f;
constexpr float DILATION = 0.3f;
constexpr int NSM = 148;          // B300 streaming multiprocessors

struct Error : std::runtime_error {
  tgs_status code;
  Error(tgs_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define TGS_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::tgs::Error(e_ == cudaErrorMemoryAllocation ? TGS_ERR_OOM : TGS_ERR_CUDA,     \
                         std::string(#call) + ": " + cudaGetErrorString(e_) + " (" +       \
                             __FILE__ + ":" + std::to_string(__LINE__) + ")");             \
  } while (0)

#define TGS_CHECK(cond, code, msg)                  \
  do {                                              \
    if (!(cond)) throw ::tgs::Error((code), (msg)); \
  } while (0)

// Count of kernels this library launched (reported by the benchmark).
extern uint64_t g_launches;
#define TGS_LAUNCHED()                   \
  do {                                   \
    ++::tgs::g_launches;                 \
    TGS_CUDA(cudaGetLastError());        \
  } while (0)

// Camera as the kernels see it: FP32 values of the ABI camera plus derived
// quantities computed on the host (camera centre, Jacobian clamp limits,
// tile grid).
struct DevCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy, znear, zfar;
  float campos[3];
  float limx, limy;
  int W, H, TX, TY;
};

DevCam make_devcam(const tgs_camera& c);

inline unsigned div_up(uint64_t a, uint64_t b) { return (unsigned)((a + b - 1) / b); }

// floor((x + r) / 16) for a float x and a small integer r, exactly: the sum is
// never rounded; an estimate is corrected with exact integer comparisons.
__device__ __forceinline__ int floor_div_tile(float x, int r) {
  x = fminf(fmaxf(x, -16777216.0f), 16777216.0f);
  int k = (int)floorf((x + (float)r) * (1.0f / TILE));
  // largest k with 16 k - r <= x
  while ((float)(TILE * (k + 1) - r) <= x) ++k;
  while ((float)(TILE * k - r) > x) --k;
  return k;
}

// Camera-space position, projected centre and depth in FP32 with the
// operation order fixed and no contraction:
//   t_a = ((R_a0 mx + R_a1 my) + R_a2 mz) + t_a,  u = fx (tx / tz) + cx.
struct KeyPath {
  float tx, ty, tz, u, v;
};
__device__ __forceinline__ KeyPath key_path(const DevCam& c, float mx, float my, float mz) {
  KeyPath k;
  float t3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float m0 = __fmul_rn(c.R[3 * a + 0], mx);
    float m1 = __fmul_rn(c.R[3 * a + 1], my);
    float m2 = __fmul_rn(c.R[3 * a + 2], mz);
    t3[a] = __fadd_rn(__fadd_rn(__fadd_rn(m0, m1), m2), c.t[a]);
  }
  k.tx = t3[0];
  k.ty = t3[1];
  k.tz = t3[2];
  k.u = __fadd_rn(__fmul_rn(c.fx, __fdiv_rn(k.tx, k.tz)), c.cx);
  k.v = __fadd_rn(__fmul_rn(c.fy, __fdiv_rn(k.ty, k.tz)), c.cy);
  return k;
}


}  // namespace tgs
