// Learned block-prefetch predictor (not in the paper): a 3-layer MLP that
// maps the last 8 camera poses plus per-block centroid/extent features to the
// block's visibility in the next 4 iterations.  The forward's 256 x 256 layer
// runs on the tcgen05 tensor cores (BF16 operands in shared memory, FP32
// accumulator in tensor memory).
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace tgs {

constexpr int MLP_HIST = 8;
constexpr int MLP_NPOSE = 12 * MLP_HIST;  // 96
constexpr int MLP_NFEAT = 6;
constexpr int MLP_NIN = MLP_NPOSE + MLP_NFEAT;  // 102
constexpr int MLP_H = 256;
constexpr int MLP_OUT = 4;
constexpr int MLP_ROWS_PER_CTA = 64;
// flat parameter layout: W1 [102][256], b1 [256], W2 [256][256], b2 [256], W3 [256][4], b3 [4]
constexpr uint64_t MLP_OFF_W1 = 0;
constexpr uint64_t MLP_OFF_B1 = MLP_OFF_W1 + (uint64_t)MLP_NIN * MLP_H;
constexpr uint64_t MLP_OFF_W2 = MLP_OFF_B1 + MLP_H;
constexpr uint64_t MLP_OFF_B2 = MLP_OFF_W2 + (uint64_t)MLP_H * MLP_H;
constexpr uint64_t MLP_OFF_W3 = MLP_OFF_B2 + MLP_H;
constexpr uint64_t MLP_OFF_B3 = MLP_OFF_W3 + (uint64_t)MLP_H * MLP_OUT;
constexpr uint64_t MLP_NPARAM = MLP_OFF_B3 + MLP_OUT;

struct Mlp {
  uint64_t max_rows = 0;  // padded to MLP_ROWS_PER_CTA
  float* params = nullptr;  // FP32 masters (flat)
  float* grads = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* w2t = nullptr;  // [out][in] BF16 copy of W2 for the tensor cores
  float* w2r = nullptr;          // [in][out] FP32 copy of the BF16-rounded W2 (backward)
  float* pose = nullptr;         // 96
  float* pterm = nullptr;        // 256: pose W1[0:96] + b1
  float* feat = nullptr;         // rows x 8
  __nv_bfloat16* h1 = nullptr;   // rows x 256
  float* h2 = nullptr;           // rows x 256
  float* z3 = nullptr;           // rows x 4
  float* dh2 = nullptr;          // rows x 256
  float* dh1 = nullptr;          // rows x 256
  float* dz3 = nullptr;          // rows x 4
  float* loss = nullptr;         // device scalar
  float* loss_host = nullptr;    // pinned
  uint32_t* cflag = nullptr;     // candidate prediction: per-block flag,
  uint32_t* cpos = nullptr;      //   packed row,
  uint32_t* cid = nullptr;       //   block of each row,
  uint32_t* ccount = nullptr;    //   device count
  void* cscratch = nullptr;
  uint32_t* err = nullptr;       // device word: a tensor-core wait ran out
  uint32_t step = 0;
};

void mlp_alloc(Mlp& m, uint64_t max_rows, uint32_t seed);
void mlp_free(Mlp& m);
// Throws TGS_ERR_TIMEOUT if a forward's wait for the tensor cores ran out
// (reads a device word: synchronous).
void mlp_check(Mlp& m);
void mlp_refresh_bf16(Mlp& m, cudaStream_t s);
// pose vector (96) of a camera history (8 cameras, oldest first, last = current)
void mlp_pose_host(const tgs_camera* hist, float out[MLP_NPOSE]);
// logits [rows][4] of K blocks (spheres device K x 4) seen from hist[7];
// keep=true stores h1/h2 for a following backward.
void mlp_forward(Mlp& m, const float4* spheres, uint64_t K, const tgs_camera* hist, float* logits, bool keep,
                 cudaStream_t s);
// backward of the loss of the last forward against labels (device [K][4],
// 0/1 floats) and one AdamW step; returns the loss (host).
float mlp_train_step(Mlp& m, uint64_t K, const float* labels, float pos_weight, float lr, float wd,
                     bool apply, cudaStream_t s);
// Prediction over the candidate blocks only: blocks whose sphere comes within
// reach of the ball through the far corners of the current camera's frustum
// (hist[7]) are packed, run through the
// network and thresholded (probability > thr for a horizon in mask) into
// bits (zeroed here); every other block is predicted invisible.
void mlp_predict_near(Mlp& m, const float4* spheres, uint64_t K, const tgs_camera* hist, float reach, uint32_t mask,
                      float thr, uint32_t* bits, cudaStream_t s);

}  // namespace tgs
