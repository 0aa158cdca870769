/*
 * tgs_oracle.c -- plain FP64 CPU oracle for the out-of-core 3D Gaussian
 * Splatting training step of TideGS (arXiv 2605.20150).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header or constant table with
 * the CUDA library; both follow the same written specification.
 *
 * What it computes, with the passage each part follows:
 *   - Morton ordering and fixed-size blocking: Sec. 3.3 "SSD-aligned blocks
 *     with spatial locality", Eq. (block_def).
 *   - Block bounding spheres and the 6-plane frustum test (cull if
 *     d < -r_k on any plane), union over the batch: Sec. 3.3 "Level 1",
 *     Eq. (Kt_def).
 *   - Residency selection and set-difference streaming: Sec. 3.5,
 *     "Residency scoring", "Set-difference streaming", Algorithm 1.
 *   - Level-2 projection, tile binning, depth sort, front-to-back
 *     compositing and its analytic backward: Sec. 3.3 "Level 2" (the paper
 *     reuses the standard 3DGS forward/backward; the formulas are the
 *     standard EWA splatting ones, written out here from the mathematics).
 *   - Masked Adam: Appendix A.1, Eq. (masked_update).
 *
 * Precision: everything is FP64 except the quantities that decide an
 * integer and are specified in FP32 (Morton quantisation, the culling
 * distance, and -- in "fp32 key" mode -- the projected centre and depth that
 * decide tile membership and the sort key).  Those are emulated exactly: each
 * FP32 operation is done in double and rounded to float, which equals the
 * correctly rounded FP32 result for +, -, *, / and sqrt (53 >= 2*24+2).
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (closed forms, brute force, finite differences, library routines,
 * invariants).  See the header of each function for its pin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define D_PARAMS 59
#define TILE 16
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_STOP 1e-4
#define DILATION 0.3
#define PI_D 3.14159265358979323846

/* round a double to the nearest float and back: one FP32 operation */
static inline double r32(double x) { return (double)(float)x; }

/* ------------------------------------------------------------------------ */
/* Camera: double[20] = W, H, fx, fy, cx, cy, znear, zfar, R (row-major 3x3), */
/* t (3).  A world point mu maps to camera coordinates t_c = R mu + t; the     */
/* camera looks down +z with y pointing down; pixel (px, py) is sampled at   */
/* its integer coordinates.                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int W, H;
  double fx, fy, cx, cy, znear, zfar;
  double R[3][3];
  double t[3];
} cam_t;

static void cam_load(const double* c, cam_t* k) {
  k->W = (int)c[0];
  k->H = (int)c[1];
  k->fx = c[2]; k->fy = c[3]; k->cx = c[4]; k->cy = c[5];
  k->znear = c[6]; k->zfar = c[7];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) k->R[i][j] = c[8 + 3 * i + j];
  for (int i = 0; i < 3; ++i) k->t[i] = c[17 + i];
}

/* camera centre in world coordinates: -R^T t */
static void cam_center(const cam_t* k, double p[3]) {
  for (int j = 0; j < 3; ++j)
    p[j] = -(k->R[0][j] * k->t[0] + k->R[1][j] * k->t[1] + k->R[2][j] * k->t[2]);
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3.                                   */
/* Convention: for m>0 the basis is sqrt(2)*Re(Y_l^m), for m<0 it is          */
/* sqrt(2)*Im(Y_l^|m|), m=0 is Y_l^0, where Y_l^m are the complex harmonics    */
/* with the Condon-Shortley phase; coefficients are ordered l=0..3,           */
/* m=-l..l.  The polynomials below are those functions written in Cartesian   */
/* form for a unit direction (x, y, z).  Pinned against scipy's sph_harm_y.   */
/* ------------------------------------------------------------------------ */
static void sh_norms(double k[16]) {
  k[0] = 0.5 * sqrt(1.0 / PI_D);
  double k1 = sqrt(3.0 / (4.0 * PI_D));
  k[1] = -k1; k[2] = k1; k[3] = -k1;
  k[4] = 0.5 * sqrt(15.0 / PI_D);
  k[5] = -0.5 * sqrt(15.0 / PI_D);
  k[6] = 0.25 * sqrt(5.0 / PI_D);
  k[7] = -0.5 * sqrt(15.0 / PI_D);
  k[8] = 0.25 * sqrt(15.0 / PI_D);
  k[9] = -0.25 * sqrt(35.0 / (2.0 * PI_D));
  k[10] = 0.5 * sqrt(105.0 / PI_D);
  k[11] = -0.25 * sqrt(21.0 / (2.0 * PI_D));
  k[12] = 0.25 * sqrt(7.0 / PI_D);
  k[13] = -0.25 * sqrt(21.0 / (2.0 * PI_D));
  k[14] = 0.25 * sqrt(105.0 / PI_D);
  k[15] = -0.25 * sqrt(35.0 / (2.0 * PI_D));
}

/* polynomial part P_k(x,y,z) and its gradient; Y_k = norm_k * P_k */
static void sh_poly(double x, double y, double z, double P[16], double G[16][3]) {
  P[0] = 1.0;           G[0][0] = 0; G[0][1] = 0; G[0][2] = 0;
  P[1] = y;             G[1][0] = 0; G[1][1] = 1; G[1][2] = 0;
  P[2] = z;             G[2][0] = 0; G[2][1] = 0; G[2][2] = 1;
  P[3] = x;             G[3][0] = 1; G[3][1] = 0; G[3][2] = 0;
  P[4] = x * y;         G[4][0] = y; G[4][1] = x; G[4][2] = 0;
  P[5] = y * z;         G[5][0] = 0; G[5][1] = z; G[5][2] = y;
  P[6] = 2 * z * z - x * x - y * y;
  G[6][0] = -2 * x; G[6][1] = -2 * y; G[6][2] = 4 * z;
  P[7] = x * z;         G[7][0] = z; G[7][1] = 0; G[7][2] = x;
  P[8] = x * x - y * y; G[8][0] = 2 * x; G[8][1] = -2 * y; G[8][2] = 0;
  P[9] = y * (3 * x * x - y * y);
  G[9][0] = 6 * x * y; G[9][1] = 3 * x * x - 3 * y * y; G[9][2] = 0;
  P[10] = x * y * z;
  G[10][0] = y * z; G[10][1] = x * z; G[10][2] = x * y;
  P[11] = y * (4 * z * z - x * x - y * y);
  G[11][0] = -2 * x * y; G[11][1] = 4 * z * z - x * x - 3 * y * y; G[11][2] = 8 * y * z;
  P[12] = z * (2 * z * z - 3 * x * x - 3 * y * y);
  G[12][0] = -6 * x * z; G[12][1] = -6 * y * z; G[12][2] = 6 * z * z - 3 * x * x - 3 * y * y;
  P[13] = x * (4 * z * z - x * x - y * y);
  G[13][0] = 4 * z * z - 3 * x * x - y * y; G[13][1] = -2 * x * y; G[13][2] = 8 * x * z;
  P[14] = z * (x * x - y * y);
  G[14][0] = 2 * x * z; G[14][1] = -2 * y * z; G[14][2] = x * x - y * y;
  P[15] = x * (x * x - 3 * y * y);
  G[15][0] = 3 * x * x - 3 * y * y; G[15][1] = -6 * x * y; G[15][2] = 0;
}

/* Exported for the pin against scipy: Y_k at n unit directions (n x 16). */
void orc_sh_basis(int64_t n, const double* dirs, double* out) {
  double k[16], P[16], G[16][3];
  sh_norms(k);
  for (int64_t i = 0; i < n; ++i) {
    sh_poly(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], P, G);
    for (int j = 0; j < 16; ++j) out[16 * i + j] = k[j] * P[j];
  }
}

/* ------------------------------------------------------------------------ */
/* Morton ordering and blocking (Sec. 3.3, Eq. block_def).                    */
/* Quantisation (FP32 spec): q = min(1023, floor(((x - lo) / (hi - lo)) *    */
/* 1024)); the 30-bit code interleaves x into bit 0, y into bit 1, z into    */
/* bit 2 of each triple.  Ties keep the original index order (stable).        */
/* Pinned by brute-force bit interleaving and sorting in the tests.           */
/* ------------------------------------------------------------------------ */
void orc_scene_aabb(int64_t n, const float* means, float lo[3], float hi[3]) {
  for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      float v = means[3 * i + a];
      if (v < lo[a]) lo[a] = v;
      if (v > hi[a]) hi[a] = v;
    }
}

static uint32_t morton_q(float x, float lo, float hi) {
  double ext = r32((double)hi - (double)lo);
  if (!(ext > 0.0)) return 0;
  double rel = r32((double)x - (double)lo);
  double f = r32(r32(rel / ext) * 1024.0);
  double q = floor(f);
  if (q < 0) q = 0;
  if (q > 1023) q = 1023;
  return (uint32_t)q;
}

void orc_morton_codes(int64_t n, const float* means, const float lo[3], const float hi[3],
                      uint32_t* codes) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) q[a] = morton_q(means[3 * i + a], lo[a], hi[a]);
    uint32_t c = 0;
    for (int b = 0; b < 10; ++b)
      for (int a = 0; a < 3; ++a) c |= ((q[a] >> b) & 1u) << (3 * b + a);
    codes[i] = c;
  }
}

static const uint32_t* g_sort_codes;
static int cmp_code_idx(const void* pa, const void* pb) {
  int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
  uint32_t ca = g_sort_codes[a], cb = g_sort_codes[b];
  if (ca != cb) return ca < cb ? -1 : 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}

/* perm[g] = original index of the Gaussian with Morton-order id g */
void orc_block_order(int64_t n, const uint32_t* codes, int64_t* perm) {
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  g_sort_codes = codes;
  qsort(perm, (size_t)n, sizeof(int64_t), cmp_code_idx);
}

/* ------------------------------------------------------------------------ */
/* Block bounding spheres (Sec. 3.3 "Level 1"; refreshed as centres move).   */
/* c_k = midpoint of the axis-aligned box of the block's means;              */
/* r_k = max_i (|mu_i - c_k| + 3 * max_axis exp(logscale_i)).                 */
/* P is n x 59 in Morton order; block k holds ids [kB, min(N, (k+1)B)).      */
/* out: K x 4 (cx, cy, cz, r).  Pinned by a brute-force containment test.     */
/* ------------------------------------------------------------------------ */
void orc_block_spheres(int64_t n, const double* P, int64_t B, double* out) {
  int64_t K = (n + B - 1) / B;
  for (int64_t k = 0; k < K; ++k) {
    int64_t a = k * B, b = (k + 1) * B < n ? (k + 1) * B : n;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = a; i < b; ++i)
      for (int d = 0; d < 3; ++d) {
        double v = P[i * D_PARAMS + d];
        if (v < mn[d]) mn[d] = v;
        if (v > mx[d]) mx[d] = v;
      }
    double c[3];
    for (int d = 0; d < 3; ++d) c[d] = 0.5 * (mn[d] + mx[d]);
    double r = 0.0;
    for (int64_t i = a; i < b; ++i) {
      const double* p = P + i * D_PARAMS;
      double dx = p[0] - c[0], dy = p[1] - c[1], dz = p[2] - c[2];
      double ls = p[3];
      if (p[4] > ls) ls = p[4];
      if (p[5] > ls) ls = p[5];
      double e = sqrt(dx * dx + dy * dy + dz * dz) + 3.0 * exp(ls);
      if (e > r) r = e;
    }
    out[4 * k + 0] = c[0]; out[4 * k + 1] = c[1]; out[4 * k + 2] = c[2]; out[4 * k + 3] = r;
  }
}

/* ------------------------------------------------------------------------ */
/* Frustum planes (Sec. 3.3 "Level 1", "standard 6-plane frustum test").      */
/* In camera coordinates a plane keeps points with n.t + w >= 0:              */
/*   near  (0,0,1), w=-znear;  far (0,0,-1), w=zfar;                          */
/*   left  (fx, 0, cx+m), right (-fx, 0, 16*TX+m-cx),                          */
/*   top   (0, fy, cy+m), bottom (0, -fy, 16*TY+m-cy),                         */
/* with TX, TY the tile-grid size and m a pixel margin that covers the        */
/* screen-space dilation and the ceiling of the splat radius.  Side normals   */
/* are normalised; world normal = R^T n, world offset = n.t + w.              */
/* fp32=1 follows the FP32 specification op by op (the library's planes);     */
/* fp32=0 is plain FP64.  out: 6 x 4 (nx, ny, nz, w).                          */
/* ------------------------------------------------------------------------ */
void orc_frustum_planes(const double* camd, double margin, int fp32, double* out) {
  cam_t k;
  cam_load(camd, &k);
  int TX = (k.W + TILE - 1) / TILE, TY = (k.H + TILE - 1) / TILE;
  double n[6][3], w[6];
#define RR(x) (fp32 ? r32(x) : (x))
  double fx = RR(k.fx), fy = RR(k.fy), cx = RR(k.cx), cy = RR(k.cy), m = RR(margin);
  n[0][0] = 0; n[0][1] = 0; n[0][2] = 1;  w[0] = -RR(k.znear);
  n[1][0] = 0; n[1][1] = 0; n[1][2] = -1; w[1] = RR(k.zfar);
  n[2][0] = fx;  n[2][1] = 0; n[2][2] = RR(cx + m);
  n[3][0] = -fx; n[3][1] = 0; n[3][2] = RR(RR((double)(TILE * TX) + m) - cx);
  n[4][0] = 0; n[4][1] = fy;  n[4][2] = RR(cy + m);
  n[5][0] = 0; n[5][1] = -fy; n[5][2] = RR(RR((double)(TILE * TY) + m) - cy);
  for (int p = 2; p < 6; ++p) {
    w[p] = 0.0;
    double len = RR(sqrt(RR(RR(RR(n[p][0] * n[p][0]) + RR(n[p][1] * n[p][1])) + RR(n[p][2] * n[p][2]))));
    for (int a = 0; a < 3; ++a) n[p][a] = RR(n[p][a] / len);
  }
  for (int p = 0; p < 6; ++p) {
    double nw[3], ww;
    for (int j = 0; j < 3; ++j)
      nw[j] = RR(RR(RR(RR(k.R[0][j]) * n[p][0]) + RR(RR(k.R[1][j]) * n[p][1])) + RR(RR(k.R[2][j]) * n[p][2]));
    ww = RR(RR(RR(RR(RR(k.t[0]) * n[p][0]) + RR(RR(k.t[1]) * n[p][1])) + RR(RR(k.t[2]) * n[p][2])) + w[p]);
    out[4 * p + 0] = nw[0]; out[4 * p + 1] = nw[1]; out[4 * p + 2] = nw[2]; out[4 * p + 3] = ww;
  }
#undef RR
}

/* Level-1 cull of K spheres against one camera's planes.
 * Rule (Sec. 3.3): culled iff some plane has d < -r with d = n.c + w.
 * fp32=1 evaluates d = ((nx*cx + ny*cy) + nz*cz) + w in FP32 without fused
 * multiply-add (the library's rule); fp32=0 evaluates it in FP64.
 * vis[k] = 1 if visible.  margin_out[k] = min over planes of (d + r) / max(r, 1)
 * in FP64, the distance to the decision boundary. */
void orc_cull(int64_t K, const double* spheres, const double* planes, int fp32, uint8_t* vis,
              double* margin_out) {
  for (int64_t k = 0; k < K; ++k) {
    const double* s = spheres + 4 * k;
    int visible = 1;
    double mind = INFINITY;
    for (int p = 0; p < 6; ++p) {
      const double* pl = planes + 4 * p;
      double d;
      if (fp32) {
        d = r32(r32(r32(r32(pl[0] * s[0]) + r32(pl[1] * s[1])) + r32(pl[2] * s[2])) + pl[3]);
        if (d < -s[3]) visible = 0;
      } else {
        d = pl[0] * s[0] + pl[1] * s[1] + pl[2] * s[2] + pl[3];
        if (d < -s[3]) visible = 0;
      }
      double e = (pl[0] * s[0] + pl[1] * s[1] + pl[2] * s[2] + pl[3] + s[3]) / (s[3] > 1 ? s[3] : 1);
      if (fabs(e) < mind) mind = fabs(e);
    }
    vis[k] = (uint8_t)visible;
    if (margin_out) margin_out[k] = mind;
  }
}

/* ------------------------------------------------------------------------ */
/* Residency selection and set-difference streaming (Sec. 3.5, Algorithm 1). */
/* Inputs: K blocks; J cameras of the next batch with per-camera visible      */
/* sets knext[j*K + k]; the current visible set kcur (blocks accessed at t   */
/* are kcur AND rcur); the current resident set rcur; per-block age (in/out). */
/* Steps, in the algorithm's order:                                          */
/*   K_{t+1} = union_j K_{t+1}^(j)                                            */
/*   Recency: age <- 0 for k in R_t & K_t, age <- min(age+1, 126) otherwise;  */
/*            Recency(k) = 2^-age                                             */
/*   C_t = R_t | K_{t+1}                                                      */
/*   s(k) = lambda*[k in K_{t+1}] + (1-lambda)*Recency(k), in FP32:           */
/*            s = fl(fl(lambda)*[vis] + fl(fl(1-fl(lambda)) * 2^-age))        */
/*   R_{t+1} = CameraBalancedTopC: the union over cameras of each camera's    */
/*            first `quota` visible blocks in (s desc, id asc) order, then    */
/*            filled to capacity C from the rest of C_t in the same order.    */
/*   Omega = R_t & R_{t+1}, S+ = R_{t+1} \ R_t, S- = R_t \ R_{t+1}.           */
/* Outputs: rnext[k] in {0,1}; splus/sminus ascending id lists with counts.   */
/* Pinned by brute-force set identities and a hand-worked example.            */
/* ------------------------------------------------------------------------ */
static const float* g_score;
static int cmp_score_id(const void* pa, const void* pb) {
  int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
  float sa = g_score[a], sb = g_score[b];
  if (sa != sb) return sa > sb ? -1 : 1;
  return a < b ? -1 : (a > b ? 1 : 0);
}

void orc_residency(int64_t K, int J, const uint8_t* kcur, const uint8_t* knext, const uint8_t* rcur,
                   uint32_t* age, int64_t C, double lambda, int64_t quota, uint8_t* rnext,
                   int64_t* splus, int64_t* n_plus, int64_t* sminus, int64_t* n_minus) {
  uint8_t* kn = (uint8_t*)calloc((size_t)K, 1);
  float* score = (float*)malloc(sizeof(float) * (size_t)K);
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)K);
  for (int j = 0; j < J; ++j)
    for (int64_t k = 0; k < K; ++k)
      if (knext[(int64_t)j * K + k]) kn[k] = 1;
  for (int64_t k = 0; k < K; ++k) {
    if (rcur[k] && kcur[k]) age[k] = 0;
    else if (age[k] < 126) age[k] += 1;
  }
  float lam = (float)lambda;
  float oml = (float)(1.0 - (double)lam);
  for (int64_t k = 0; k < K; ++k) {
    double rec = ldexp(1.0, -(int)age[k]);
    double t = r32((double)oml * rec);
    score[k] = (float)r32((kn[k] ? (double)lam : 0.0) + t);
  }
  for (int64_t k = 0; k < K; ++k) rnext[k] = 0;
  int64_t taken = 0;
  g_score = score;
  /* per-camera quota: each camera's first `quota` visible blocks by (s desc, id asc) */
  for (int j = 0; j < J; ++j) {
    int64_t m = 0;
    for (int64_t k = 0; k < K; ++k)
      if (knext[(int64_t)j * K + k]) order[m++] = k;
    qsort(order, (size_t)m, sizeof(int64_t), cmp_score_id);
    for (int64_t i = 0; i < m && i < quota; ++i)
      if (!rnext[order[i]] && taken < C) { rnext[order[i]] = 1; ++taken; }
  }
  /* global fill over the candidate pool C_t = R_t | K_{t+1} */
  int64_t m = 0;
  for (int64_t k = 0; k < K; ++k)
    if (rcur[k] || kn[k]) order[m++] = k;
  qsort(order, (size_t)m, sizeof(int64_t), cmp_score_id);
  for (int64_t i = 0; i < m && taken < C; ++i)
    if (!rnext[order[i]]) { rnext[order[i]] = 1; ++taken; }
  int64_t np = 0, nm = 0;
  for (int64_t k = 0; k < K; ++k) {
    if (rnext[k] && !rcur[k]) splus[np++] = k;
    if (rcur[k] && !rnext[k]) sminus[nm++] = k;
  }
  *n_plus = np;
  *n_minus = nm;
  free(kn); free(score); free(order);
}

/* ------------------------------------------------------------------------ */
/* Level-2 preprocess of one camera (standard EWA splatting; Sec. 3.3 "Level */
/* 2" reuses it unchanged).  Per Gaussian row p (59 values):                  */
/*   mu = p[0:3]; scale = exp(p[3:6]); q = p[6:10]/|p[6:10]| (w,x,y,z);       */
/*   opacity = sigmoid(p[10]); SH coefficients sh[c][ch] = p[11 + 3c + ch].   */
/*   t = R mu + tc; invisible if t_z <= znear or t_z > zfar.                  */
/*   Sigma = (Rq S)(Rq S)^T.  The Jacobian of the perspective map is taken at */
/*   t_x, t_y clamped to |t_x/t_z| <= 1.3*W/(2 fx), |t_y/t_z| <= 1.3*H/(2 fy):*/
/*     J = [[fx/tz, 0, -fx x'/tz^2], [0, fy/tz, -fy y'/tz^2]].               */
/*   cov = (J Rc) Sigma (J Rc)^T + 0.3 I = [[a, b], [b, c]]; invisible if    */
/*   det = ac - b^2 <= 0; conic (A, B, C) = (c, -b, a)/det.                   */
/*   lambda1 = (a+c)/2 + sqrt(max(0.1, ((a+c)/2)^2 - det)); r = ceil(3       */
/*   sqrt(lambda1)).  Centre u = fx tx/tz + cx, v = fy ty/tz + cy.            */
/*   Tile rect [x0,x1)x[y0,y1): x0 = clamp(floor((u-r)/16), 0, TX),           */
/*   x1 = clamp(floor((u+r)/16)+1, 0, TX) (same for y); invisible if empty.  */
/*   Colour: d = (mu - camera centre)/|.|; rgb = sum_c sh[c] Y_c(d) + 0.5,    */
/*   negative channels clamped to 0 (clamp flags kept for the backward).      */
/* fp32key=1 computes t, u, v and the depth in FP32 (the specification of the */
/* key path: t_i = ((R_i0 mu_x + R_i1 mu_y) + R_i2 mu_z) + tc_i,             */
/* u = fx * (tx / tz) + cx), so tile membership and sort keys are decided in  */
/* FP32; fp32key=0 keeps them FP64 (for finite differences).                  */
/* Border flags: a Gaussian is marked 'border' when a decision that fixes its */
/* tile set lies within the given tolerances (|3 sqrt(lambda1) - integer| <   */
/* tol_r, a rect edge (u+-r)/16 within tol_px/16 of an integer, or t_z within */
/* tol_z*znear of the near plane); several outcomes are then valid.           */
/* Output row (NS = 24 doubles): u v depth A B C opac r g b clr clg clb       */
/*   radius x0 y0 x1 y1 visible border tz_raw tx_raw ty_raw lambda1           */
/* ------------------------------------------------------------------------ */
#define NS 24

void orc_preprocess(int64_t n, const double* P, const double* camd, int fp32key, double tol_r,
                    double tol_px, double tol_z, double* out) {
  cam_t k;
  cam_load(camd, &k);
  int TX = (k.W + TILE - 1) / TILE, TY = (k.H + TILE - 1) / TILE;
  double cc[3];
  cam_center(&k, cc);
  double shk[16];
  sh_norms(shk);
  double limx = 1.3 * (double)k.W / (2.0 * k.fx), limy = 1.3 * (double)k.H / (2.0 * k.fy);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double* p = P + i * D_PARAMS;
    double* o = out + i * NS;
    for (int j = 0; j < NS; ++j) o[j] = 0.0;
    double t[3];
    for (int a = 0; a < 3; ++a)
      t[a] = k.R[a][0] * p[0] + k.R[a][1] * p[1] + k.R[a][2] * p[2] + k.t[a];
    double tk[3];
    if (fp32key) {
      for (int a = 0; a < 3; ++a) {
        double m0 = r32(r32(k.R[a][0]) * r32(p[0]));
        double m1 = r32(r32(k.R[a][1]) * r32(p[1]));
        double m2 = r32(r32(k.R[a][2]) * r32(p[2]));
        tk[a] = r32(r32(r32(m0 + m1) + m2) + r32(k.t[a]));
      }
    } else {
      for (int a = 0; a < 3; ++a) tk[a] = t[a];
    }
    o[20] = t[2]; o[21] = t[0]; o[22] = t[1];
    double tzd = fp32key ? tk[2] : t[2];
    if (fabs(tzd - k.znear) < tol_z * k.znear) o[19] = 1;
    if (!(tzd > k.znear) || tzd > k.zfar) continue;
    /* covariance */
    double sc[3] = {exp(p[3]), exp(p[4]), exp(p[5])};
    double qn = sqrt(p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9]);
    double w = p[6] / qn, x = p[7] / qn, y = p[8] / qn, z = p[9] / qn;
    double Rq[3][3] = {
        {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
        {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
        {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    double M[3][3], S[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) M[a][b] = Rq[a][b] * sc[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) S[a][b] = M[a][0] * M[b][0] + M[a][1] * M[b][1] + M[a][2] * M[b][2];
    double tz = t[2];
    double xr = t[0] / tz, yr = t[1] / tz;
    double xc = xr < -limx ? -limx : (xr > limx ? limx : xr);
    double yc = yr < -limy ? -limy : (yr > limy ? limy : yr);
    double J[2][3] = {{k.fx / tz, 0, -k.fx * xc / tz}, {0, k.fy / tz, -k.fy * yc / tz}};
    double T[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b) T[a][b] = J[a][0] * k.R[0][b] + J[a][1] * k.R[1][b] + J[a][2] * k.R[2][b];
    double TS[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b) TS[a][b] = T[a][0] * S[0][b] + T[a][1] * S[1][b] + T[a][2] * S[2][b];
    double ca = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2] + DILATION;
    double cb = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
    double ccv = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2] + DILATION;
    double det = ca * ccv - cb * cb;
    if (!(det > 0.0)) continue;
    double mid = 0.5 * (ca + ccv);
    double disc = mid * mid - det;
    double lam1 = mid + sqrt(disc > 0.1 ? disc : 0.1);
    double r3 = 3.0 * sqrt(lam1);
    double radius = ceil(r3);
    double u, v;
    if (fp32key) {
      u = r32(r32(r32(k.fx) * r32(tk[0] / tk[2])) + r32(k.cx));
      v = r32(r32(r32(k.fy) * r32(tk[1] / tk[2])) + r32(k.cy));
    } else {
      u = k.fx * t[0] / tz + k.cx;
      v = k.fy * t[1] / tz + k.cy;
    }
    double fx0 = floor((u - radius) / TILE), fx1 = floor((u + radius) / TILE) + 1;
    double fy0 = floor((v - radius) / TILE), fy1 = floor((v + radius) / TILE) + 1;
    int x0 = (int)(fx0 < 0 ? 0 : (fx0 > TX ? TX : fx0));
    int x1 = (int)(fx1 < 0 ? 0 : (fx1 > TX ? TX : fx1));
    int y0 = (int)(fy0 < 0 ? 0 : (fy0 > TY ? TY : fy0));
    int y1 = (int)(fy1 < 0 ? 0 : (fy1 > TY ? TY : fy1));
    /* border: radius ceiling or a rect edge close to a decision boundary */
    double fr = r3 - floor(r3);
    if (fr < tol_r || fr > 1.0 - tol_r) o[19] = 1;
    double edges[4] = {u - radius, u + radius, v - radius, v + radius};
    for (int e = 0; e < 4; ++e) {
      double q = edges[e] / TILE;
      double f = q - floor(q);
      if (f < tol_px / TILE || f > 1.0 - tol_px / TILE) o[19] = 1;
    }
    o[13] = radius; o[14] = x0; o[15] = y0; o[16] = x1; o[17] = y1; o[23] = lam1;
    o[0] = u; o[1] = v;
    o[2] = fp32key ? tk[2] : tz;
    o[3] = ccv / det; o[4] = -cb / det; o[5] = ca / det;
    o[6] = 1.0 / (1.0 + exp(-p[10]));
    if ((x1 - x0) * (y1 - y0) <= 0) continue;
    o[18] = 1;
    /* colour */
    double dv[3] = {p[0] - cc[0], p[1] - cc[1], p[2] - cc[2]};
    double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double Pl[16], G[16][3];
    sh_poly(dv[0] / dn, dv[1] / dn, dv[2] / dn, Pl, G);
    for (int ch = 0; ch < 3; ++ch) {
      double s = 0.0;
      for (int c = 0; c < 16; ++c) s += p[11 + 3 * c + ch] * shk[c] * Pl[c];
      s += 0.5;
      o[10 + ch] = s < 0 ? 1.0 : 0.0;
      o[7 + ch] = s < 0 ? 0.0 : s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Tile binning and the depth sort.                                          */
/* Every visible Gaussian i emits one pair per tile of its rect, in id order */
/* and row-major tile order; key = (tile << 32) | bits(float(depth)).  Pairs */
/* are stably sorted by key, so equal keys keep the lower id first.           */
/* ranges[2*tile] = first pair of the tile, ranges[2*tile+1] = one past last. */
/* Returns the pair count; with keys == NULL only counts.                     */
/* Pinned by the untiled brute-force render (tests).                          */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t val; uint64_t pos; } pair_t;
static int cmp_pair(const void* pa, const void* pb) {
  const pair_t* a = (const pair_t*)pa;
  const pair_t* b = (const pair_t*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->pos < b->pos ? -1 : (a->pos > b->pos ? 1 : 0);
}

static uint32_t float_bits(double d) {
  float f = (float)d;
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

int64_t orc_bin_sort(int64_t n, const double* S, int W, int H, int phantom, uint64_t* keys,
                     uint32_t* vals, uint32_t* ranges) {
  int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double* s = S + i * NS;
    int x0 = (int)s[14], y0 = (int)s[15], x1 = (int)s[16], y1 = (int)s[17];
    if (phantom) {
      if (s[19] == 0) continue;
      x0 = x0 > 0 ? x0 - 1 : 0; y0 = y0 > 0 ? y0 - 1 : 0;
      x1 = x1 < TX ? x1 + 1 : TX; y1 = y1 < TY ? y1 + 1 : TY;
      if (s[13] == 0) continue;
    } else if (s[18] == 0) {
      continue;
    }
    if (x1 > x0 && y1 > y0) cnt += (int64_t)(x1 - x0) * (y1 - y0);
  }
  if (!keys) return cnt;
  pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(cnt > 0 ? cnt : 1));
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double* s = S + i * NS;
    int x0 = (int)s[14], y0 = (int)s[15], x1 = (int)s[16], y1 = (int)s[17];
    if (phantom) {
      if (s[19] == 0 || s[13] == 0) continue;
      x0 = x0 > 0 ? x0 - 1 : 0; y0 = y0 > 0 ? y0 - 1 : 0;
      x1 = x1 < TX ? x1 + 1 : TX; y1 = y1 < TY ? y1 + 1 : TY;
    } else if (s[18] == 0) {
      continue;
    }
    uint32_t db = float_bits(s[2]);
    for (int ty = y0; ty < y1; ++ty)
      for (int tx = x0; tx < x1; ++tx) {
        pr[m].key = ((uint64_t)(ty * TX + tx) << 32) | db;
        pr[m].val = (uint32_t)i;
        pr[m].pos = (uint64_t)m;
        ++m;
      }
  }
  qsort(pr, (size_t)cnt, sizeof(pair_t), cmp_pair);
  for (int64_t j = 0; j < 2LL * TX * TY; ++j) ranges[j] = 0;
  for (int64_t j = 0; j < cnt; ++j) {
    keys[j] = pr[j].key;
    vals[j] = pr[j].val;
    uint32_t tile = (uint32_t)(pr[j].key >> 32);
    if (j == 0 || (uint32_t)(pr[j - 1].key >> 32) != tile) ranges[2 * tile] = (uint32_t)j;
    ranges[2 * tile + 1] = (uint32_t)(j + 1);
  }
  free(pr);
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Front-to-back compositing (forward).                                       */
/* For pixel (px, py) over its tile's sorted list: with d = (px-u, py-v),     */
/* power = -(A dx^2 + C dy^2)/2 - B dx dy; skip if power > 0;                 */
/* alpha = min(0.99, opac * exp(power)); skip if alpha < 1/255;               */
/* T' = T (1 - alpha); stop (this entry excluded) if T' < 1e-4;               */
/* C += rgb alpha T; T = T'.  Finally C += T bg.                               */
/* nlast = 1 + position (within the tile list) of the last included entry.   */
/* img: H x W x 3.  Slack (test support): a bound on how far a result taken   */
/* with any of the valid outcomes of a borderline decision can move the       */
/* pixel.  An FP32 alpha carries a relative error of about e_a = 1e-6 +     */
/* POWER_REL_ERR |power| (the power is a quadratic form of FP32 centre and    */
/* conic values, so its absolute error grows with |power|; 1e-6 for the      */
/* exponential).  Every entry whose alpha test lies within max(tol_a, e_a)   */
/* (relative) of 1/255, or whose Gaussian is 'border', or any phantom entry  */
/* (ph_* lists: border Gaussians over their one-tile-enlarged rect), adds    */
/* 2 * alpha * T * max(rgb, bg).  The stop test compares a product of        */
/* (1 - alpha) factors, each with a relative error of alpha / (1 - alpha) e_a */
/* plus two roundings: it is borderline when T' lies within the summed bound */
/* eT (at least tol_a) of 1e-4, and either outcome there moves the pixel by  */
/* at most T * max(rgb, bg) (the transmittance left), so the slack adds      */
/* 2 * T * max(rgb, bg).                                                      */
/* ------------------------------------------------------------------------ */
#define POWER_REL_ERR 1e-5       /* relative error of an FP32 power (quadratic form) */
#define FACTOR_ROUND 1.2e-7      /* two FP32 roundings per (1 - alpha) factor */

static double eval_alpha(const double* s, int px, int py, double* power_out) {
  double dx = (double)px - s[0], dy = (double)py - s[1];
  double power = -0.5 * (s[3] * dx * dx + s[5] * dy * dy) - s[4] * dx * dy;
  *power_out = power;
  if (power > 0) return -1.0;
  double a = s[6] * exp(power);
  return a > ALPHA_MAX ? ALPHA_MAX : a;
}

void orc_composite_fwd(int64_t n, const double* S, int W, int H, const uint32_t* vals,
                       const uint32_t* ranges, const uint32_t* ph_vals, const uint32_t* ph_ranges,
                       const double* bg, double tol_a, double* img, double* Tfinal, int32_t* nlast,
                       double* slack) {
  int TX = (W + TILE - 1) / TILE;
  double bgmax = fmax(bg[0], fmax(bg[1], bg[2]));
  (void)n;
#pragma omp parallel for schedule(dynamic, 4)
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int tile = (py / TILE) * TX + (px / TILE);
      uint32_t a = ranges[2 * tile], b = ranges[2 * tile + 1];
      uint32_t pa = ph_ranges ? ph_ranges[2 * tile] : 0, pb = ph_ranges ? ph_ranges[2 * tile + 1] : 0;
      double T = 1.0, C[3] = {0, 0, 0}, sl = 0.0, eT = 0.0;
      int32_t last = 0;
      int done = 0;
      uint32_t j = a, q = pa;
      while (!done && (j < b || q < pb)) {
        /* merge the phantom list by (depth, id) so each phantom sees its T */
        int take_ph = 0;
        if (q < pb) {
          if (j >= b) take_ph = 1;
          else {
            const double* sj = S + (int64_t)vals[j] * NS;
            const double* sq = S + (int64_t)ph_vals[q] * NS;
            uint32_t dj = float_bits(sj[2]), dq = float_bits(sq[2]);
            take_ph = (dq < dj) || (dq == dj && ph_vals[q] < vals[j]);
          }
        }
        if (take_ph) {
          const double* s = S + (int64_t)ph_vals[q] * NS;
          double pw;
          double al = eval_alpha(s, px, py, &pw);
          if (al >= ALPHA_MIN * (1.0 - tol_a)) {
            double cm = fmax(fmax(s[7], s[8]), fmax(s[9], bgmax));
            sl += 2.0 * al * T * cm;
          }
          ++q;
          continue;
        }
        const double* s = S + (int64_t)vals[j] * NS;
        double pw;
        double al = eval_alpha(s, px, py, &pw);
        double cm = fmax(fmax(s[7], s[8]), fmax(s[9], bgmax));
        int border = s[19] != 0;
        if (al >= 0) {
          double Tn = T * (1.0 - al);
          double ea = 1e-6 + POWER_REL_ERR * fabs(pw);
          double eTn = eT + FACTOR_ROUND + al / (1.0 - al) * ea;
          if (border && al >= ALPHA_MIN * (1.0 - tol_a)) sl += 2.0 * al * T * cm;
          else if (fabs(al - ALPHA_MIN) < fmax(tol_a, ea) * ALPHA_MIN) sl += 2.0 * al * T * cm;
          else if (al >= ALPHA_MIN && fabs(Tn - T_STOP) < fmax(tol_a, eTn) * T_STOP) sl += 2.0 * T * cm;
          if (al >= ALPHA_MIN) {
            if (Tn < T_STOP) {
              done = 1;
            } else {
              for (int ch = 0; ch < 3; ++ch) C[ch] += s[7 + ch] * al * T;
              T = Tn;
              eT = eTn;
              last = (int32_t)(j - a + 1);
            }
          }
        }
        ++j;
      }
      int64_t pix = (int64_t)py * W + px;
      for (int ch = 0; ch < 3; ++ch) img[3 * pix + ch] = C[ch] + T * bg[ch];
      Tfinal[pix] = T;
      nlast[pix] = last;
      if (slack) slack[pix] = sl;
    }
}

/* ------------------------------------------------------------------------ */
/* Backward of the compositing.                                               */
/* Given dL/dC per pixel (g, H x W x 3), accumulates per Gaussian (G2 row of  */
/* 9 doubles): dL/du, dL/dv, dL/dA, dL/dB, dL/dC, dL/dopac, dL/drgb (3).      */
/* For included entry i with transmittance T_i before it and S_i the colour   */
/* composited behind it (normalised by T_i (1 - alpha_i)):                    */
/*   dC/drgb_i = alpha_i T_i;                                                  */
/*   dC/dalpha_i = T_i (rgb_i - S_i) - T_final bg / (1 - alpha_i);            */
/* alpha = opac * exp(power) unless clamped at 0.99 (then no gradient);       */
/* dpower/du = A dx + B dy, dpower/dv = B dx + C dy (d = pixel - centre),     */
/* dpower/dA = -dx^2/2, dpower/dB = -dx dy, dpower/dC = -dy^2/2.              */
/* mode 0: the reverse recurrence the kernel uses, T_i = T_{i+1}/(1-alpha_i), */
/*         S_{i-1} = alpha_i rgb_i + (1 - alpha_i) S_i, starting at nlast.    */
/* mode 1: re-runs the forward and stores the per-pixel list explicitly.     */
/* The two must agree to rounding; both are pinned by finite differences.   */
/* ------------------------------------------------------------------------ */
#define NG2 9
void orc_composite_bwd(int64_t n, const double* S, int W, int H, const uint32_t* vals,
                       const uint32_t* ranges, const double* bg, const double* Tfinal,
                       const int32_t* nlast, const double* g, int mode, double* G2) {
  int TX = (W + TILE - 1) / TILE;
  for (int64_t i = 0; i < n * NG2; ++i) G2[i] = 0.0;
  /* serial over pixels so the accumulation order is fixed */
  int64_t cap = 0;
  for (int64_t t = 0; t < (int64_t)TX * ((H + TILE - 1) / TILE); ++t) {
    int64_t len = (int64_t)ranges[2 * t + 1] - ranges[2 * t];
    if (len > cap) cap = len;
  }
  uint32_t* lst = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(cap + 1));
  double* lal = (double*)malloc(sizeof(double) * (size_t)(cap + 1));
  double* lT = (double*)malloc(sizeof(double) * (size_t)(cap + 1));
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      int64_t pix = (int64_t)py * W + px;
      const double* gg = g + 3 * pix;
      if (gg[0] == 0 && gg[1] == 0 && gg[2] == 0) continue;
      int tile = (py / TILE) * TX + (px / TILE);
      uint32_t a = ranges[2 * tile];
      int32_t nl = nlast[pix];
      double Tf = Tfinal[pix];
      double bgdot = bg[0] * gg[0] + bg[1] * gg[1] + bg[2] * gg[2];
      if (mode == 0) {
        double T = Tf, Sb[3] = {0, 0, 0};
        for (int32_t jj = nl - 1; jj >= 0; --jj) {
          uint32_t id = vals[a + jj];
          const double* s = S + (int64_t)id * NS;
          double pw;
          double al = eval_alpha(s, px, py, &pw);
          if (al < ALPHA_MIN) continue;
          double Ti = T / (1.0 - al);
          double* o = G2 + (int64_t)id * NG2;
          double dal = 0.0;
          for (int ch = 0; ch < 3; ++ch) {
            o[6 + ch] += al * Ti * gg[ch];
            dal += gg[ch] * Ti * (s[7 + ch] - Sb[ch]);
          }
          dal -= Tf * bgdot / (1.0 - al);
          for (int ch = 0; ch < 3; ++ch) Sb[ch] = al * s[7 + ch] + (1.0 - al) * Sb[ch];
          T = Ti;
          double G = exp(pw);
          if (s[6] * G > ALPHA_MAX) continue;
          double dx = (double)px - s[0], dy = (double)py - s[1];
          o[5] += G * dal;
          double dpw = al * dal;
          o[0] += dpw * (s[3] * dx + s[4] * dy);
          o[1] += dpw * (s[4] * dx + s[5] * dy);
          o[2] += dpw * (-0.5 * dx * dx);
          o[3] += dpw * (-dx * dy);
          o[4] += dpw * (-0.5 * dy * dy);
        }
      } else {
        /* forward pass storing the list of included entries with T_i */
        int m = 0;
        double T = 1.0;
        for (int32_t jj = 0; jj < nl; ++jj) {
          uint32_t id = vals[a + jj];
          const double* s = S + (int64_t)id * NS;
          double pw;
          double al = eval_alpha(s, px, py, &pw);
          if (al < ALPHA_MIN) continue;
          lst[m] = id; lal[m] = al; lT[m] = T; ++m;
          T *= 1.0 - al;
        }
        for (int e = 0; e < m; ++e) {
          const double* s = S + (int64_t)lst[e] * NS;
          double* o = G2 + (int64_t)lst[e] * NG2;
          double al = lal[e], Ti = lT[e];
          /* colour behind e, normalised by T_i (1 - alpha_i) */
          double Sb[3] = {0, 0, 0};
          for (int f = e + 1; f < m; ++f) {
            const double* sf = S + (int64_t)lst[f] * NS;
            for (int ch = 0; ch < 3; ++ch) Sb[ch] += sf[7 + ch] * lal[f] * lT[f];
          }
          double den = Ti * (1.0 - al);
          double dal = 0.0;
          for (int ch = 0; ch < 3; ++ch) {
            o[6 + ch] += al * Ti * gg[ch];
            dal += gg[ch] * Ti * (s[7 + ch] - Sb[ch] / den);
          }
          dal -= Tf * bgdot / (1.0 - al);
          double pw;
          eval_alpha(s, px, py, &pw);
          double G = exp(pw);
          if (s[6] * G > ALPHA_MAX) continue;
          double dx = (double)px - s[0], dy = (double)py - s[1];
          o[5] += G * dal;
          double dpw = al * dal;
          o[0] += dpw * (s[3] * dx + s[4] * dy);
          o[1] += dpw * (s[4] * dx + s[5] * dy);
          o[2] += dpw * (-0.5 * dx * dx);
          o[3] += dpw * (-dx * dy);
          o[4] += dpw * (-0.5 * dy * dy);
        }
      }
    }
  free(lst); free(lal); free(lT);
}

/* ------------------------------------------------------------------------ */
/* Backward of the preprocess: chain rule from the per-Gaussian 2D gradients */
/* (G2: u, v, A, B, C, opac, rgb) to the 59 parameters, exact derivative of  */
/* orc_preprocess (FP64 path):                                                */
/*   conic = inverse of [[a,b],[b,c]]:                                        */
/*     dL/da = (-c^2 gA + b c gB - b^2 gC)/det^2,                             */
/*     dL/dc = (-b^2 gA + a b gB - a^2 gC)/det^2,                             */
/*     dL/db = (2 b c gA - (a c + b^2) gB + 2 a b gC)/det^2;                  */
/*   cov = T Sigma T^T: dL/dSigma = T^T Gc T, dL/dT = 2 Gc T Sigma, with Gc = */
/*     [[dL/da, dL/db/2], [dL/db/2, dL/dc]];                                  */
/*   T = J Rc: dL/dJ = dL/dT Rc^T; J depends on t (clamped components of      */
/*     x' = clamp(tx/tz)*tz contribute through tz only);                      */
/*   u, v: dL/dt from the perspective division;                               */
/*   mu: dL/dmu = Rc^T dL/dt + view-direction term of the SH colour;          */
/*   Sigma = M M^T, M = Rq diag(scale): dL/dM = 2 dL/dSigma M; scale = exp;   */
/*   Rq from the normalised quaternion, then through the normalisation;       */
/*   opacity: sigmoid'; SH: dL/dsh[c][ch] = Y_c(d) dL/drgb_ch (unclamped).     */
/* out: n x 59.  Pinned by central finite differences of the whole forward.   */
/* ------------------------------------------------------------------------ */
void orc_preprocess_bwd(int64_t n, const double* P, const double* camd, const double* S,
                        const double* G2, double* out) {
  cam_t k;
  cam_load(camd, &k);
  double cc[3];
  cam_center(&k, cc);
  double shk[16];
  sh_norms(shk);
  double limx = 1.3 * (double)k.W / (2.0 * k.fx), limy = 1.3 * (double)k.H / (2.0 * k.fy);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const double* p = P + i * D_PARAMS;
    const double* s = S + i * NS;
    const double* g2 = G2 + i * NG2;
    double* o = out + i * D_PARAMS;
    for (int j = 0; j < D_PARAMS; ++j) o[j] = 0.0;
    if (s[18] == 0) continue;
    double dmu[3] = {0, 0, 0};
    /* ---- colour ---- */
    double dv[3] = {p[0] - cc[0], p[1] - cc[1], p[2] - cc[2]};
    double dn = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double dir[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
    double Pl[16], G[16][3];
    sh_poly(dir[0], dir[1], dir[2], Pl, G);
    double ddir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
      if (s[10 + ch] != 0) continue;
      double gc = g2[6 + ch];
      for (int c = 0; c < 16; ++c) {
        o[11 + 3 * c + ch] = shk[c] * Pl[c] * gc;
        for (int a = 0; a < 3; ++a) ddir[a] += gc * p[11 + 3 * c + ch] * shk[c] * G[c][a];
      }
    }
    double dd = ddir[0] * dir[0] + ddir[1] * dir[1] + ddir[2] * dir[2];
    for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - dir[a] * dd) / dn;
    /* ---- opacity ---- */
    double sg = s[6];
    o[10] = g2[5] * sg * (1.0 - sg);
    /* ---- recompute geometry ---- */
    double t[3];
    for (int a = 0; a < 3; ++a)
      t[a] = k.R[a][0] * p[0] + k.R[a][1] * p[1] + k.R[a][2] * p[2] + k.t[a];
    double sc[3] = {exp(p[3]), exp(p[4]), exp(p[5])};
    double qn = sqrt(p[6] * p[6] + p[7] * p[7] + p[8] * p[8] + p[9] * p[9]);
    double w = p[6] / qn, x = p[7] / qn, y = p[8] / qn, z = p[9] / qn;
    double Rq[3][3] = {
        {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
        {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
        {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    double M[3][3], Sg[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) M[a][b] = Rq[a][b] * sc[b];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Sg[a][b] = M[a][0] * M[b][0] + M[a][1] * M[b][1] + M[a][2] * M[b][2];
    double tz = t[2];
    double xr = t[0] / tz, yr = t[1] / tz;
    int clx = xr < -limx || xr > limx, cly = yr < -limy || yr > limy;
    double xc = xr < -limx ? -limx : (xr > limx ? limx : xr);
    double yc = yr < -limy ? -limy : (yr > limy ? limy : yr);
    double J[2][3] = {{k.fx / tz, 0, -k.fx * xc / tz}, {0, k.fy / tz, -k.fy * yc / tz}};
    double T[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b) T[a][b] = J[a][0] * k.R[0][b] + J[a][1] * k.R[1][b] + J[a][2] * k.R[2][b];
    double TS[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b) TS[a][b] = T[a][0] * Sg[0][b] + T[a][1] * Sg[1][b] + T[a][2] * Sg[2][b];
    double ca = TS[0][0] * T[0][0] + TS[0][1] * T[0][1] + TS[0][2] * T[0][2] + DILATION;
    double cb = TS[0][0] * T[1][0] + TS[0][1] * T[1][1] + TS[0][2] * T[1][2];
    double ccv = TS[1][0] * T[1][0] + TS[1][1] * T[1][1] + TS[1][2] * T[1][2] + DILATION;
    double det = ca * ccv - cb * cb;
    double d2 = det * det;
    double gA = g2[2], gB = g2[3], gC = g2[4];
    double dla = (-ccv * ccv * gA + cb * ccv * gB - cb * cb * gC) / d2;
    double dlc = (-cb * cb * gA + ca * cb * gB - ca * ca * gC) / d2;
    double dlb = (2 * cb * ccv * gA - (ca * ccv + cb * cb) * gB + 2 * ca * cb * gC) / d2;
    double Gc[2][2] = {{dla, 0.5 * dlb}, {0.5 * dlb, dlc}};
    /* dL/dSigma = T^T Gc T */
    double GT[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b) GT[a][b] = Gc[a][0] * T[0][b] + Gc[a][1] * T[1][b];
    double dSig[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) dSig[a][b] = T[0][a] * GT[0][b] + T[1][a] * GT[1][b];
    /* dL/dT = 2 Gc T Sigma */
    double dT[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b)
        dT[a][b] = 2.0 * (GT[a][0] * Sg[0][b] + GT[a][1] * Sg[1][b] + GT[a][2] * Sg[2][b]);
    /* dL/dJ = dT Rc^T */
    double dJ[2][3];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 3; ++b)
        dJ[a][b] = dT[a][0] * k.R[b][0] + dT[a][1] * k.R[b][1] + dT[a][2] * k.R[b][2];
    double dt[3] = {0, 0, 0};
    double tz2 = tz * tz, tz3 = tz2 * tz;
    dt[2] += -k.fx / tz2 * dJ[0][0] - k.fy / tz2 * dJ[1][1];
    if (!clx) {
      dt[0] += -k.fx / tz2 * dJ[0][2];
      dt[2] += 2.0 * k.fx * t[0] / tz3 * dJ[0][2];
    } else {
      dt[2] += k.fx * xc / tz2 * dJ[0][2];
    }
    if (!cly) {
      dt[1] += -k.fy / tz2 * dJ[1][2];
      dt[2] += 2.0 * k.fy * t[1] / tz3 * dJ[1][2];
    } else {
      dt[2] += k.fy * yc / tz2 * dJ[1][2];
    }
    /* centre u = fx tx/tz + cx */
    double gu = g2[0], gv = g2[1];
    dt[0] += gu * k.fx / tz;
    dt[1] += gv * k.fy / tz;
    dt[2] += -gu * k.fx * t[0] / tz2 - gv * k.fy * t[1] / tz2;
    for (int a = 0; a < 3; ++a) dmu[a] += k.R[0][a] * dt[0] + k.R[1][a] * dt[1] + k.R[2][a] * dt[2];
    o[0] = dmu[0]; o[1] = dmu[1]; o[2] = dmu[2];
    /* Sigma = M M^T */
    double dM[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        dM[a][b] = 2.0 * (dSig[a][0] * M[0][b] + dSig[a][1] * M[1][b] + dSig[a][2] * M[2][b]);
    double dR[3][3];
    for (int b = 0; b < 3; ++b) {
      double dsb = 0.0;
      for (int a = 0; a < 3; ++a) {
        dsb += dM[a][b] * Rq[a][b];
        dR[a][b] = dM[a][b] * sc[b];
      }
      o[3 + b] = dsb * sc[b];
    }
    double gw = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    double gx = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2] + z * dR[2][0] +
                     w * dR[2][1] - 2 * x * dR[2][2]);
    double gy = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] - w * dR[2][0] +
                     z * dR[2][1] - 2 * y * dR[2][2]);
    double gz = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1] +
                     y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    double qd = gw * w + gx * x + gy * y + gz * z;
    o[6] = (gw - w * qd) / qn;
    o[7] = (gx - x * qd) / qn;
    o[8] = (gy - y * qd) / qn;
    o[9] = (gz - z * qd) / qn;
  }
}

/* ------------------------------------------------------------------------ */
/* Photometric loss (Appendix A.1, f_i): L1 (loss=0) or L2 (loss=1) mean over */
/* all n values; writes dL/dimage.  sign(0) = 0.                              */
/* ------------------------------------------------------------------------ */
double orc_loss(int64_t n, const double* img, const double* target, int loss, double* grad) {
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = img[i] - target[i];
    if (loss == 0) {
      acc += fabs(d);
      grad[i] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)n;
    } else {
      acc += d * d;
      grad[i] = 2.0 * d / (double)n;
    }
  }
  return acc / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Masked Adam (Appendix A.1, Eq. masked_update).  For rows with mask[i]=1:  */
/*   m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;                              */
/*   theta -= lr * (m / (1 - b1^step_i)) / (sqrt(v / (1 - b2^step_i)) + eps)   */
/* where step_i is the (already incremented) step count of the row's block.  */
/* Rows with mask 0 are left untouched.  Pinned by the one-step closed form. */
/* ------------------------------------------------------------------------ */
void orc_adam(int64_t n, double* P, const double* Gr, double* M1, double* M2, const uint8_t* mask,
              const int64_t* step, const double* lr, double b1, double b2, double eps) {
  /* lr: one learning rate per parameter column (59) */
  for (int64_t i = 0; i < n; ++i) {
    if (!mask[i]) continue;
    double c1 = 1.0 - pow(b1, (double)step[i]);
    double c2 = 1.0 - pow(b2, (double)step[i]);
    for (int j = 0; j < D_PARAMS; ++j) {
      int64_t e = i * D_PARAMS + j;
      double g = Gr[e];
      M1[e] = b1 * M1[e] + (1.0 - b1) * g;
      M2[e] = b2 * M2[e] + (1.0 - b2) * g * g;
      P[e] -= lr[j] * (M1[e] / c1) / (sqrt(M2[e] / c2) + eps);
    }
  }
}
