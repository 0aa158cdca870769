// Block virtualisation and Level-1 visibility (Sec. 3.3) and the residency
// selection with set-difference streaming (Sec. 3.5, Algorithm 1).
#pragma once
#include "common.cuh"

namespace tgs {

// 6 planes (nx, ny, nz, w) of one camera; a point is inside when n.x + w >= 0.
struct Planes {
  float4 p[6];
};

// FP32 specification of the planes (op order fixed, no contraction):
// near (0,0,1,-znear), far (0,0,-1,zfar), side normals (fx,0,cx+m),
// (-fx,0,(16TX+m)-cx), (0,fy,cy+m), (0,-fy,(16TY+m)-cy) normalised by
// sqrt((n0^2 + n1^2) + n2^2); world normal ((R0j n0 + R1j n1) + R2j n2),
// offset ((t0 n0 + t1 n1) + t2 n2) + w.
Planes frustum_planes(const tgs_camera& c, float margin_px);

// Morton order of n centres (device, n x 3 float): perm[g] = original index.
// keys/vals/alt buffers: 2n u32 each; scratch: radix_scratch_bytes(n).
void morton_order(const float* means, uint64_t n, uint32_t* perm, uint32_t* codes, uint32_t* codes_alt,
                  uint32_t* perm_alt, void* scratch, float* aabb_dev, cudaStream_t s);

// Per-camera visibility bitmaps: vis[j * words + w] bit b = block 32w+b
// visible from camera j (culled iff some plane has d < -r, with
// d = ((nx cx + ny cy) + nz cz) + w in FP32); vis_union = OR over cameras.
void cull_blocks(const float4* spheres, uint64_t K, const Planes* planes_dev, int J, uint32_t* vis,
                 uint32_t* vis_union, cudaStream_t s);

struct ResidencyBuffers {
  uint32_t* flag;      // K
  uint32_t* pos;       // K
  uint32_t* key;       // 2K
  uint32_t* blk;       // 2K
  uint32_t* sel;       // K (per sorted candidate)
  uint32_t* tmp;       // K
  uint32_t* tmp2;      // K
  uint32_t* counters;  // 16
  void* scratch;
};

// Algorithm 1 on device bitmaps (words = ceil(K/32)):
//   k_acc  = blocks accessed by the last computed batch (R & K of it)
//   r_cur  = current resident set, k_next = per-camera visible sets (J)
// Updates ages (reset on access, else +1 saturating at 126), scores candidates
// C_t = R_t | K_{t+1} with s = lambda [k in K_{t+1}] + (1 - lambda) 2^-age in
// FP32, takes each camera's first `quota` visible candidates in (s desc, id
// asc) order, fills to capacity by the same order, and writes r_next.
// Outputs (device): lists s_plus, s_minus, render (r_next & union k_next),
// ascending, with counts in counters[0..2]; acc_out = render as a bitmap
// (the blocks this batch will access).  age_update = false leaves the ages
// unchanged (a selection for predicted, not accessed, blocks).
void residency(const uint32_t* k_acc, const uint32_t* r_cur, const uint32_t* k_next, const uint32_t* k_next_union,
               int J, uint64_t K, uint32_t* ages, uint64_t capacity, float lambda, uint64_t quota,
               uint32_t* r_next, uint32_t* s_plus, uint32_t* s_minus, uint32_t* render, uint32_t* acc_out,
               ResidencyBuffers& rb, cudaStream_t s, bool age_update = true);

size_t residency_scratch_bytes(uint64_t K);

// Writes the selection's results (counters[0..3], the used prefixes of the
// three lists of K entries, kvis_words visibility words, the resident bitmap)
// into host memory mapped for the device (out_*: device views of mapped
// pinned buffers; out_lists holds 16 + 3K words: counts, then the lists).
void publish_sets(const uint32_t* counters, const uint32_t* lists, uint64_t K, const uint32_t* kvis,
                  uint64_t kvis_words, const uint32_t* rbits, uint64_t words, uint32_t* out_lists, uint32_t* out_kvis,
                  uint32_t* out_r, cudaStream_t s);

}  // namespace tgs
