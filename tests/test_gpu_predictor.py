"""Learned prefetch predictor on the GPU against the FP64 oracle: logits
(tensor-core layer 2, BF16 weights/activations) rel-L2 1e-3, gradients of
the BCE loss rel-L2 1e-3 per parameter group, and training lowers the loss."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

GROUPS = {"W1": (0, 102 * 256), "b1": (102 * 256, 102 * 256 + 256)}


def _layout():
    from oracle import mlp
    off, lay = 0, {}
    for k, shape in (("W1", (mlp.NIN, 256)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)),
                     ("W3", (256, 4)), ("b3", (4,))):
        n = int(np.prod(shape))
        lay[k] = (off, shape)
        off += n
    return lay, off


def _flat(P):
    lay, n = _layout()
    out = np.zeros(n, np.float32)
    for k, (o, shape) in lay.items():
        out[o:o + int(np.prod(shape))] = P[k].reshape(-1)
    return out


def _unflat(v):
    lay, _ = _layout()
    return {k: v[o:o + int(np.prod(shape))].reshape(shape).astype(np.float64) for k, (o, shape) in lay.items()}


def _problem(K=1000, seed=0):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    sph = np.concatenate([rng.uniform(-40, 40, (K, 3)), rng.uniform(0.5, 6.0, (K, 1))], 1).astype(np.float32)
    hist = []
    for s in range(8):
        R, t = scenes.look_at([-20.0 + 2.5 * s, 1.0, -30.0 + 0.5 * s], [0.0, 0.0, 0.0])
        hist.append(scenes.pinhole(64, 48, 70.0, R, t, zfar=100.0))
    P = mlp.init(256, seed=seed + 1)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(0, 0.05, P[k].shape)
    # round the master weights to float32 as the GPU holds them
    P = {k: v.astype(np.float32).astype(np.float64) for k, v in P.items()}
    Y = (rng.random((K, 4)) < 0.2).astype(np.float64)
    X = np.concatenate([np.tile(mlp.pose_vector(hist), (K, 1)), mlp.block_features(sph.astype(np.float64), hist[-1])],
                       1)
    # the GPU computes features in FP32 from FP32 spheres and poses
    return sph, hist, P, Y, X


def test_predictor_forward_and_gradients_match_oracle(tgs):
    import torch
    from oracle import mlp
    sph, hist, P, Y, X = _problem()
    K = sph.shape[0]
    pr = tgs.Predictor(K, seed=0)
    pr.set_params(_flat(P))
    sd = torch.tensor(sph, device="cuda")
    logits = torch.zeros(K, 4, device="cuda")
    pr.forward(sd, hist, logits)
    torch.cuda.synchronize()
    f = mlp.forward(P, X, bf16_round=True)
    z = logits.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(z - f["z3"]) / np.linalg.norm(f["z3"]) < 1e-3
    lab = torch.tensor(Y.astype(np.float32), device="cuda")
    loss, g = pr.train_step(sd, hist, lab, pos_weight=4.0, apply=False, want_grads=True)
    lo = mlp.loss(f["z3"], Y, 4.0)
    assert abs(loss - lo) <= 1e-4 * lo
    Go = mlp.backward(P, f, Y, 4.0)
    Gg = _unflat(g)
    for k in Go:
        rel = np.linalg.norm(Gg[k] - Go[k]) / np.linalg.norm(Go[k])
        assert rel < 1e-3, (k, rel)
    # pose part and block part of W1 separately
    for a, b in ((0, 96), (96, 102)):
        rel = np.linalg.norm(Gg["W1"][a:b] - Go["W1"][a:b]) / np.linalg.norm(Go["W1"][a:b])
        assert rel < 1e-3, (a, b, rel)
    pr.close()


def test_predictor_adamw_step_and_training(tgs):
    import torch
    from oracle import mlp
    sph, hist, P, Y, X = _problem(K=700, seed=3)
    pr = tgs.Predictor(700, seed=0)
    pr.set_params(_flat(P))
    sd = torch.tensor(sph, device="cuda")
    # labels that depend on the features: visible if in front and near the view axis
    f = mlp.block_features(sph.astype(np.float64), hist[-1])
    lab_np = np.stack([(f[:, 2] > 0) & (np.abs(f[:, 0]) < 0.5 * f[:, 2] + 0.02 * h) for h in range(4)], 1)
    lab = torch.tensor(lab_np.astype(np.float32), device="cuda")
    l0, g = pr.train_step(sd, hist, lab, pos_weight=2.0, lr=1e-3, wd=1e-4, apply=True, want_grads=True)
    # one AdamW step from zero moments moves each weight by about -lr sign(g) - lr wd p
    P1 = _unflat(pr.params())
    G = _unflat(g)
    for k in P:
        exp = P[k] - 1e-3 * (G[k] / (np.abs(G[k]) + 1e-8) + 1e-4 * P[k])
        np.testing.assert_allclose(P1[k], exp, rtol=0, atol=2e-6)
    losses = [pr.train_step(sd, hist, lab, pos_weight=2.0, lr=1e-3) for _ in range(150)]
    assert losses[-1] < 0.5 * l0
    pr.close()
