"""FP64 CPU oracle for the TideGS out-of-core 3DGS training step.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py; the product library never imports, links or
runs anything here, and this package never imports the product library.

The arithmetic lives in tgs_oracle.c (plain C, FP64, one function per step of
the method, each citing the passage it follows).  This module compiles it,
marshals numpy arrays through ctypes and composes the steps in the paper's
order:

  create  : Morton codes of the centres -> stable sort -> blocks of B
            (Sec. 3.3, Eq. block_def) -> bounding spheres.
  cull    : 6-plane test of the spheres, union over the batch (Eq. Kt_def).
  residency: Algorithm 1 (scores, camera-balanced Top-C, S+, S-).
  render  : Level-2 projection over the Gaussians of the render set (the
            blocks of R_t & K_t), tile binning, stable depth sort,
            front-to-back compositing.
  step    : render each camera of the batch, loss, analytic backward, masked
            Adam on the touched Gaussians (Appendix A.1, Eq. masked_update).

Parity status: pinned (tests/test_oracle_*.py): Morton/blocking by brute
force; culling by containment and FP32/FP64 agreement; residency by
brute-force set identities and a hand-worked example; projection and
compositing by single-Gaussian closed forms, a hand-placed camera and the
untiled brute-force render; the backward by central finite differences and by
its second (stored-list) form; SH by scipy; Adam by the one-step closed form.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tgs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NS = 24  # splat record width (see orc_preprocess)
NG2 = 9  # 2D gradient record width (see orc_composite_bwd)
D = 59
TILE = 16
CULL_MARGIN_PX = 4.0

# column indices of the splat record
U, V, DEPTH, CA, CB, CC, OPAC, R, G, B = range(10)
RADIUS, X0, Y0, X1, Y1, VISIBLE, BORDER = 13, 14, 15, 16, 17, 18, 19


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no fused multiply-add)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", _LIB, _SRC, "-lm"])
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


I64 = ctypes.c_int64


# ----------------------------------------------------------------------------
# Morton ordering and blocks (Sec. 3.3, Eq. block_def)
# ----------------------------------------------------------------------------
def scene_aabb(means_f32):
    m = np.ascontiguousarray(means_f32, np.float32)
    lo = np.zeros(3, np.float32)
    hi = np.zeros(3, np.float32)
    lib().orc_scene_aabb(I64(m.shape[0]), _p(m), _p(lo), _p(hi))
    return lo, hi


def morton_codes(means_f32, lo=None, hi=None):
    m = np.ascontiguousarray(means_f32, np.float32)
    if lo is None:
        lo, hi = scene_aabb(m)
    codes = np.zeros(m.shape[0], np.uint32)
    lib().orc_morton_codes(I64(m.shape[0]), _p(m), _p(np.asarray(lo, np.float32)),
                           _p(np.asarray(hi, np.float32)), _p(codes))
    return codes


def block_order(codes):
    c = np.ascontiguousarray(codes, np.uint32)
    perm = np.zeros(c.shape[0], np.int64)
    lib().orc_block_order(I64(c.shape[0]), _p(c), _p(perm))
    return perm


def create(params_f32, block_size):
    """Morton permutation of the input rows; returns (perm, params in Morton order).
    perm[g] = original row of the Gaussian with id g; block k = ids [kB, (k+1)B)."""
    codes = morton_codes(params_f32[:, 0:3])
    perm = block_order(codes)
    return perm, np.ascontiguousarray(params_f32[perm])


def block_spheres(P, block_size):
    P = _f64(P)
    n = P.shape[0]
    K = (n + block_size - 1) // block_size
    out = np.zeros((K, 4), np.float64)
    lib().orc_block_spheres(I64(n), _p(P), I64(block_size), _p(out))
    return out


# ----------------------------------------------------------------------------
# Level-1 culling (Sec. 3.3, Eq. Kt_def)
# ----------------------------------------------------------------------------
def frustum_planes(cam_arr, margin=CULL_MARGIN_PX, fp32=False):
    out = np.zeros((6, 4), np.float64)
    lib().orc_frustum_planes(_p(_f64(cam_arr)), ctypes.c_double(margin), ctypes.c_int(int(fp32)), _p(out))
    return out


def cull(spheres, planes, fp32=False):
    s = _f64(spheres)
    K = s.shape[0]
    vis = np.zeros(K, np.uint8)
    marg = np.zeros(K, np.float64)
    lib().orc_cull(I64(K), _p(s), _p(_f64(planes)), ctypes.c_int(int(fp32)), _p(vis), _p(marg))
    return vis, marg


def visible_blocks(spheres, cam_arrs, margin=CULL_MARGIN_PX, fp32=False):
    """Per-camera visibility (J x K) and their union K_t."""
    per = np.stack([cull(spheres, frustum_planes(c, margin, fp32), fp32)[0] for c in cam_arrs])
    return per, per.max(axis=0)


# ----------------------------------------------------------------------------
# Residency selection (Sec. 3.5, Algorithm 1)
# ----------------------------------------------------------------------------
def residency(k_cur, k_next_per_cam, r_cur, age, capacity, lam=0.75, quota=None):
    K = k_cur.shape[0]
    kn = np.ascontiguousarray(k_next_per_cam, np.uint8).reshape(-1, K)
    J = kn.shape[0]
    if quota is None:
        quota = capacity // (2 * J)
    age = np.ascontiguousarray(age, np.uint32).copy()
    rnext = np.zeros(K, np.uint8)
    sp = np.zeros(K, np.int64)
    sm = np.zeros(K, np.int64)
    npl = I64(0)
    nmi = I64(0)
    lib().orc_residency(I64(K), ctypes.c_int(J), _p(np.ascontiguousarray(k_cur, np.uint8)), _p(kn),
                        _p(np.ascontiguousarray(r_cur, np.uint8)), _p(age), I64(capacity),
                        ctypes.c_double(lam), I64(quota), _p(rnext), _p(sp), ctypes.byref(npl), _p(sm),
                        ctypes.byref(nmi))
    return dict(r_next=rnext, s_plus=sp[:npl.value].copy(), s_minus=sm[:nmi.value].copy(), age=age)


# ----------------------------------------------------------------------------
# Level-2 render (projection, binning, sort, compositing)
# ----------------------------------------------------------------------------
def preprocess(P, cam_arr, fp32key=True, tol_r=1e-5, tol_px=1e-3, tol_z=1e-6):
    P = _f64(P)
    n = P.shape[0]
    S = np.zeros((n, NS), np.float64)
    lib().orc_preprocess(I64(n), _p(P), _p(_f64(cam_arr)), ctypes.c_int(int(fp32key)),
                         ctypes.c_double(tol_r), ctypes.c_double(tol_px), ctypes.c_double(tol_z), _p(S))
    return S


def bin_sort(S, W, H, phantom=False):
    S = _f64(S)
    n = S.shape[0]
    TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
    cnt = lib().orc_bin_sort
    cnt.restype = ctypes.c_int64
    m = cnt(I64(n), _p(S), ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(int(phantom)), None, None, None)
    keys = np.zeros(max(m, 1), np.uint64)
    vals = np.zeros(max(m, 1), np.uint32)
    ranges = np.zeros(2 * TX * TY, np.uint32)
    cnt(I64(n), _p(S), ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(int(phantom)), _p(keys), _p(vals),
        _p(ranges))
    return keys[:m], vals[:m], ranges.reshape(TY * TX, 2)


def composite_fwd(S, W, H, vals, ranges, bg=(0.0, 0.0, 0.0), ph_vals=None, ph_ranges=None, tol_a=1e-5):
    S = _f64(S)
    img = np.zeros((H, W, 3), np.float64)
    Tf = np.zeros((H, W), np.float64)
    nl = np.zeros((H, W), np.int32)
    sl = np.zeros((H, W), np.float64)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    phv = None if ph_vals is None else np.ascontiguousarray(ph_vals, np.uint32)
    phr = None if ph_ranges is None else np.ascontiguousarray(ph_ranges, np.uint32)
    lib().orc_composite_fwd(I64(S.shape[0]), _p(S), ctypes.c_int(W), ctypes.c_int(H), _p(vals), _p(ranges),
                            None if phv is None else _p(phv), None if phr is None else _p(phr),
                            _p(_f64(bg)), ctypes.c_double(tol_a), _p(img), _p(Tf), _p(nl), _p(sl))
    return img, Tf, nl, sl


def composite_bwd(S, W, H, vals, ranges, bg, Tf, nl, dimg, mode=0):
    S = _f64(S)
    G2 = np.zeros((S.shape[0], NG2), np.float64)
    lib().orc_composite_bwd(I64(S.shape[0]), _p(S), ctypes.c_int(W), ctypes.c_int(H),
                            _p(np.ascontiguousarray(vals, np.uint32)), _p(np.ascontiguousarray(ranges, np.uint32)),
                            _p(_f64(bg)), _p(_f64(Tf)), _p(np.ascontiguousarray(nl, np.int32)), _p(_f64(dimg)),
                            ctypes.c_int(mode), _p(G2))
    return G2


def preprocess_bwd(P, cam_arr, S, G2):
    P = _f64(P)
    out = np.zeros_like(P)
    lib().orc_preprocess_bwd(I64(P.shape[0]), _p(P), _p(_f64(cam_arr)), _p(_f64(S)), _p(_f64(G2)), _p(out))
    return out


def loss(img, target, kind=0):
    """kind 0: L1 mean, 1: L2 mean, 2: (1 - 0.2) L1 + 0.2 (1 - SSIM) (oracle/ssim.py)."""
    if kind == 2:
        from . import ssim
        return ssim.loss(img, target), ssim.loss_grad(img, target)
    img = _f64(img)
    g = np.zeros_like(img)
    f = lib().orc_loss
    f.restype = ctypes.c_double
    val = f(I64(img.size), _p(img), _p(_f64(target)), ctypes.c_int(kind), _p(g))
    return val, g


# parameter groups of the 59 columns: means, log-scales, quaternion, opacity,
# SH DC, SH rest
LR_GROUP_COLUMNS = ((0, 3), (3, 6), (6, 10), (10, 11), (11, 14), (14, 59))


def group_lr(lr_groups):
    """Per-column learning rates (59) from the six group rates."""
    out = np.zeros(59, np.float64)
    for (a, b), v in zip(LR_GROUP_COLUMNS, lr_groups):
        out[a:b] = v
    return out


def lr_schedule_groups(lr_groups, lr_means_final, decay_steps, step):
    """3DGS schedule: the means' rate decays log-linearly from its initial to
    its final value over decay_steps (constant afterwards); the other groups
    keep their rates.  step counts completed training steps."""
    t = min(max(step, 0), decay_steps) / max(decay_steps, 1)
    g = list(lr_groups)
    g[0] = float(np.exp(np.log(lr_groups[0]) * (1.0 - t) + np.log(lr_means_final) * t))
    return g


def adam(P, Gr, M1, M2, mask, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-15):
    """In place on float64 P, M1, M2 (n x 59); mask (n,) uint8; step (n,)
    int64; lr: one rate, or one per column (59)."""
    lrv = np.ascontiguousarray(np.broadcast_to(np.asarray(lr, np.float64), (59,)), np.float64)
    lib().orc_adam(I64(P.shape[0]), _p(P), _p(_f64(Gr)), _p(M1), _p(M2),
                   _p(np.ascontiguousarray(mask, np.uint8)), _p(np.ascontiguousarray(step, np.int64)),
                   _p(lrv), ctypes.c_double(b1), ctypes.c_double(b2), ctypes.c_double(eps))


def sh_basis(dirs):
    d = _f64(dirs)
    out = np.zeros((d.shape[0], 16), np.float64)
    lib().orc_sh_basis(I64(d.shape[0]), _p(d), _p(out))
    return out


def render(P, cam_arr, bg=(0.0, 0.0, 0.0), fp32key=True, with_slack=False, tol_a=1e-5):
    """Forward render of the rows P (the render set, ascending id order)."""
    W, H = int(cam_arr[0]), int(cam_arr[1])
    S = preprocess(P, cam_arr, fp32key=fp32key)
    keys, vals, ranges = bin_sort(S, W, H)
    phv = phr = None
    if with_slack:
        _, phv, phr = bin_sort(S, W, H, phantom=True)
    img, Tf, nl, sl = composite_fwd(S, W, H, vals, ranges, bg, phv, phr, tol_a=tol_a)
    return dict(S=S, keys=keys, vals=vals, ranges=ranges, img=img, T=Tf, nlast=nl, slack=sl)


def render_grad(P, cam_arr, r, dimg, bg=(0.0, 0.0, 0.0), mode=0):
    """Analytic gradient of <dimg, render(P)> w.r.t. P (n x 59) given a forward record r."""
    W, H = int(cam_arr[0]), int(cam_arr[1])
    G2 = composite_bwd(r["S"], W, H, r["vals"], r["ranges"], bg, r["T"], r["nlast"], dimg, mode)
    return preprocess_bwd(P, cam_arr, r["S"], G2), G2


def train_step(P, M1, M2, step_blocks, block_size, block_ids, cam_arrs, targets, lr=1e-3, loss_kind=0,
               bg=(0.0, 0.0, 0.0), fp32key=True, b1=0.9, b2=0.999, eps=1e-15):
    """One training step on a camera batch over the render set (rows of the
    blocks `block_ids`, ascending).  P, M1, M2: float64 (N x 59) in Morton
    order, updated in place for the touched rows; step_blocks: per-block Adam
    step counters (incremented for blocks with a touched Gaussian).
    Returns dict(loss, images, grad (render-set rows), touched, records)."""
    ids = np.concatenate([np.arange(k * block_size, min((k + 1) * block_size, P.shape[0]))
                          for k in sorted(block_ids)]) if len(block_ids) else np.zeros(0, np.int64)
    Ps = P[ids]
    J = len(cam_arrs)
    recs, imgs = [], []
    for c in cam_arrs:
        r = render(Ps, c, bg, fp32key=fp32key, with_slack=True)
        recs.append(r)
        imgs.append(r["img"])
    imgs = np.stack(imgs)
    lval, dimg = loss(imgs, np.asarray(targets, np.float64).reshape(imgs.shape), loss_kind)
    grad = np.zeros_like(Ps)
    touched = np.zeros(len(ids), np.uint8)
    g2s = []
    for j, c in enumerate(cam_arrs):
        gj, g2 = render_grad(Ps, c, recs[j], dimg[j], bg)
        grad += gj
        g2s.append(g2)
        touched |= (recs[j]["S"][:, VISIBLE] != 0).astype(np.uint8)
    blk = ids // block_size
    for k in np.unique(blk[touched.astype(bool)]):
        step_blocks[k] += 1
    Gfull = np.zeros_like(P)
    Gfull[ids] = grad
    mask = np.zeros(P.shape[0], np.uint8)
    mask[ids] = touched
    steps = step_blocks[np.arange(P.shape[0]) // block_size].astype(np.int64)
    adam(P, Gfull, M1, M2, mask, steps, lr, b1, b2, eps)
    return dict(loss=lval, images=imgs, grad=grad, touched=touched, ids=ids, records=recs, g2=g2s,
                dimg=dimg)
