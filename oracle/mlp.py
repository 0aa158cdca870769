"""FP64 oracle of the learned block-prefetch predictor.

TEST INFRASTRUCTURE ONLY (imported by tests and the benchmark's CPU leg).

The predictor is not in the paper; it follows the specification of the
learned prefetch form: a 3-layer MLP (hidden 256) that maps the last 8
camera poses plus per-block centroid/extent features to the visibility of the
block in the next 4 iterations.

Inputs of block k at step t (camera t, history t-7..t, oldest first):
  pose slot s (camera c_s = cams[max(t-7+s, 0)]): R_rel = R_t R_s^T (9 values,
  row-major) and t_rel = (t_t - R_rel t_s) / zfar_t (3 values) -> 96 values;
  block: c = R_t c_k + t_t, d = |c|; [c / zfar, r_k / zfar, d / zfar,
  r_k / max(d, r_k)] -> 6 values.
Network: z1 = x W1 + b1 (W1: 102 x 256), h1 = relu(z1) rounded to BF16;
z2 = h1 W2 + b2 with W2 rounded to BF16, h2 = relu(z2); z3 = h2 W3 + b3
(W3: 256 x 4), p = sigmoid(z3).  Loss: mean over rows and horizons of
-(w y log p + (1 - y) log(1 - p)) with pos_weight w.  AdamW with decoupled
weight decay.  `bf16=False` disables the two roundings (for finite
differences).

Pinned by tests/test_oracle_mlp.py: central finite differences of the loss
and torch float64 autograd of the same network.
"""
from __future__ import annotations

import numpy as np

HIST = 8
NPOSE = 12 * HIST
NFEAT = 6
NIN = NPOSE + NFEAT
HORIZON = 4


def bf16(x):
    """Round-to-nearest-even to BF16 (float64 in, float64 out)."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def pose_vector(cams_hist):
    """cams_hist: list of 8 camera dicts (R, t, zfar), oldest first; the last is current."""
    Rt = np.asarray(cams_hist[-1]["R"], np.float64)
    tt = np.asarray(cams_hist[-1]["t"], np.float64)
    zf = float(cams_hist[-1]["zfar"])
    out = []
    for c in cams_hist:
        Rs = np.asarray(c["R"], np.float64)
        ts = np.asarray(c["t"], np.float64)
        Rr = Rt @ Rs.T
        tr = (tt - Rr @ ts) / zf
        out.append(np.concatenate([Rr.reshape(9), tr]))
    return np.concatenate(out)


def block_features(spheres, cam):
    R = np.asarray(cam["R"], np.float64)
    t = np.asarray(cam["t"], np.float64)
    zf = float(cam["zfar"])
    c = spheres[:, :3] @ R.T + t
    r = spheres[:, 3]
    d = np.linalg.norm(c, axis=1)
    return np.stack([c[:, 0] / zf, c[:, 1] / zf, c[:, 2] / zf, r / zf, d / zf, r / np.maximum(d, r)], 1)


def init(hidden=256, seed=0):
    rng = np.random.default_rng(seed)
    return dict(W1=rng.normal(0, 1 / np.sqrt(NIN), (NIN, hidden)), b1=np.zeros(hidden),
                W2=rng.normal(0, 1 / np.sqrt(hidden), (hidden, hidden)), b2=np.zeros(hidden),
                W3=rng.normal(0, 1 / np.sqrt(hidden), (hidden, HORIZON)), b3=np.zeros(HORIZON))


def forward(P, X, bf16_round=True):
    z1 = X @ P["W1"] + P["b1"]
    h1 = np.maximum(z1, 0.0)
    if bf16_round:
        h1 = bf16(h1)
    W2 = bf16(P["W2"]) if bf16_round else P["W2"]
    z2 = h1 @ W2 + P["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ P["W3"] + P["b3"]
    return dict(X=X, z1=z1, h1=h1, W2=W2, z2=z2, h2=h2, z3=z3)


def loss(z3, Y, pos_weight):
    p = 1.0 / (1.0 + np.exp(-z3))
    l = -(pos_weight * Y * np.log(p) + (1 - Y) * np.log1p(-p))
    return float(l.mean())


def backward(P, f, Y, pos_weight):
    """Gradient of loss() w.r.t. every parameter (exact derivative of forward,
    the BF16 roundings treated as the identity)."""
    M = Y.size
    p = 1.0 / (1.0 + np.exp(-f["z3"]))
    dz3 = (p * (pos_weight * Y + 1 - Y) - pos_weight * Y) / M
    g = {}
    g["W3"] = f["h2"].T @ dz3
    g["b3"] = dz3.sum(0)
    dh2 = (dz3 @ P["W3"].T) * (f["z2"] > 0)
    g["W2"] = f["h1"].T @ dh2
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ f["W2"].T) * (f["z1"] > 0)
    g["W1"] = f["X"].T @ dh1
    g["b1"] = dh1.sum(0)
    return g


def adamw(P, G, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in P:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * G[k]
        v[...] = b2 * v + (1 - b2) * G[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] -= lr * (mh / (np.sqrt(vh) + eps) + wd * P[k])
