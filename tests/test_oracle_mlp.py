"""Pins of the predictor oracle (CPU): finite differences of the loss and
torch float64 autograd of the same network."""
import numpy as np

import scenes


def _data(rng, M=37, hidden=8):
    from oracle import mlp
    X = rng.normal(size=(M, mlp.NIN))
    Y = (rng.random((M, mlp.HORIZON)) < 0.3).astype(np.float64)
    P = mlp.init(hidden, seed=3)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.normal(0, 0.1, P[k].shape)
    return X, Y, P


def test_mlp_backward_matches_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    X, Y, P = _data(rng)
    f = mlp.forward(P, X, bf16_round=False)
    G = mlp.backward(P, f, Y, 3.0)
    checked = 0
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
            h = 1e-6
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(P, X, False)["z3"], Y, 3.0)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(P, X, False)["z3"], Y, 3.0)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(G[k].reshape(-1)[idx] - fd) <= 1e-7 + 1e-5 * abs(fd), (k, idx)
            checked += 1
    assert checked >= 50


def test_mlp_matches_torch_autograd():
    import torch
    from oracle import mlp
    rng = np.random.default_rng(1)
    X, Y, P = _data(rng, M=53, hidden=16)
    T = {k: torch.tensor(v, requires_grad=True) for k, v in P.items()}
    x = torch.tensor(X)
    z1 = x @ T["W1"] + T["b1"]
    z2 = torch.relu(z1) @ T["W2"] + T["b2"]
    z3 = torch.relu(z2) @ T["W3"] + T["b3"]
    lt = torch.nn.functional.binary_cross_entropy_with_logits(z3, torch.tensor(Y), pos_weight=torch.tensor(3.0))
    lt.backward()
    f = mlp.forward(P, X, bf16_round=False)
    assert abs(mlp.loss(f["z3"], Y, 3.0) - lt.item()) < 1e-12
    G = mlp.backward(P, f, Y, 3.0)
    for k in P:
        np.testing.assert_allclose(G[k], T[k].grad.numpy(), rtol=1e-10, atol=1e-14)


def test_mlp_adamw_matches_torch():
    import torch
    from oracle import mlp
    rng = np.random.default_rng(2)
    P = {"w": rng.normal(size=(5, 3))}
    t = torch.tensor(P["w"].copy(), requires_grad=True)
    opt = torch.optim.AdamW([t], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-4)
    st = {}
    for _ in range(4):
        g = rng.normal(size=(5, 3))
        t.grad = torch.tensor(g)
        opt.step()
        mlp.adamw(P, {"w": g}, st, lr=1e-3, wd=1e-4)
    # torch applies the decay before the Adam step (p *= 1 - lr wd); ours adds
    # lr wd p to the step: they agree to first order in lr wd
    np.testing.assert_allclose(P["w"], t.detach().numpy(), rtol=0, atol=1e-9)


def test_pose_vector_identity_and_features():
    from oracle import mlp
    R, t = scenes.look_at([1.0, 2.0, 3.0], [0.0, 0.0, 0.0])
    cam = scenes.pinhole(64, 48, 60.0, R, t, zfar=50.0)
    pv = mlp.pose_vector([cam] * 8)
    for s in range(8):
        np.testing.assert_allclose(pv[12 * s:12 * s + 9], np.eye(3).reshape(9), atol=1e-12)
        np.testing.assert_allclose(pv[12 * s + 9:12 * s + 12], 0.0, atol=1e-12)
    sph = np.array([[0.0, 0.0, 0.0, 0.5]])
    f = mlp.block_features(sph, cam)
    d = np.linalg.norm([1.0, 2.0, 3.0])
    np.testing.assert_allclose(f[0], [0, 0, d / 50, 0.5 / 50, d / 50, 0.5 / d], atol=1e-12)
