"""Pins of the oracle's residency selection (Algorithm 1) and masked Adam (CPU only)."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _load_examples():
    with open(os.path.join(HERE, "golden", "residency_examples.json")) as f:
        return json.load(f)["examples"]


def _bits(ids, K):
    b = np.zeros(K, np.uint8)
    b[list(ids)] = 1
    return b


@pytest.mark.parametrize("ex", _load_examples(), ids=lambda e: e["name"])
def test_residency_hand_worked(orc, ex):
    K = ex["K"]
    out = orc.residency(_bits(ex["K_t"], K), np.stack([_bits(s, K) for s in ex["K_next_per_camera"]]),
                        _bits(ex["R_t"], K), np.array(ex["age_before"], np.uint32), ex["C"],
                        ex["lambda"], ex["quota"])
    assert sorted(np.nonzero(out["r_next"])[0].tolist()) == ex["R_next"]
    assert out["s_plus"].tolist() == ex["S_plus"]
    assert out["s_minus"].tolist() == ex["S_minus"]
    assert out["age"].tolist() == ex["age_after"]


def test_residency_identities_random(orc):
    rng = np.random.default_rng(0)
    for trial in range(200):
        K = int(rng.integers(1, 60))
        J = int(rng.integers(1, 5))
        C = int(rng.integers(1, K + 3))
        kn = (rng.random((J, K)) < rng.random()).astype(np.uint8)
        r = np.zeros(K, np.uint8)
        r[rng.permutation(K)[:min(C, K)]] = rng.random(min(C, K)) < 0.8
        kc = (rng.random(K) < 0.4).astype(np.uint8)
        age = rng.integers(0, 130, K).astype(np.uint32)
        lam = float(rng.choice([0.0, 0.3, 0.75, 1.0]))
        quota = int(rng.integers(0, 3))
        out = orc.residency(kc, kn, r, age, C, lam, quota)
        R1 = set(np.nonzero(out["r_next"])[0].tolist())
        R0 = set(np.nonzero(r)[0].tolist())
        Kn = set(np.nonzero(kn.max(0))[0].tolist())
        Sp, Sm = set(out["s_plus"].tolist()), set(out["s_minus"].tolist())
        Om = R0 & R1
        assert R1 == Om | Sp and R0 == Om | Sm and not (Sp & Sm)
        assert len(R1) <= C
        assert R1 <= (R0 | Kn)                       # chosen from the candidate pool
        assert len(R1) == min(C, len(R0 | Kn))       # capacity is used
        if lam > 0.5 and len(Kn) <= C:
            assert Kn <= R1                          # next working set fits -> all resident
        for j in range(J):                           # per-camera quota is honoured
            vis_j = set(np.nonzero(kn[j])[0].tolist())
            if quota * J <= C:
                assert len(vis_j & R1) >= min(quota, len(vis_j))
        # ages: reset on access, aged otherwise (saturating at 126)
        acc = (r & kc).astype(bool)
        exp_age = np.where(acc, 0, np.minimum(age.astype(np.int64) + 1, np.maximum(age, 126)))
        exp_age = np.where(acc, 0, np.where(age < 126, age.astype(np.int64) + 1, age))
        assert np.array_equal(out["age"], exp_age)


def test_residency_pure_recency_is_lru(orc):
    """lambda = 0 and no quota: R_{t+1} = the C most recently used candidates."""
    K, C = 20, 6
    rng = np.random.default_rng(1)
    age = rng.permutation(20).astype(np.uint32)  # distinct ages
    r = np.zeros(K, np.uint8); r[:8] = 1
    kc = np.zeros(K, np.uint8)
    kn = np.zeros((1, K), np.uint8); kn[0, 10:14] = 1
    out = orc.residency(kc, kn, r, age, C, 0.0, 0)
    cand = list(range(8)) + list(range(10, 14))
    lru = sorted(cand, key=lambda k: (int(age[k]) + 1, k))[:C]
    assert sorted(np.nonzero(out["r_next"])[0].tolist()) == sorted(lru)


def test_adam_one_step_closed_form(orc):
    """From zero moments one step moves theta by -lr g / (|g| + eps); rows with
    mask 0 are bit-identical (Eq. masked_update)."""
    rng = np.random.default_rng(0)
    n = 50
    P = rng.normal(size=(n, 59))
    P0 = P.copy()
    G = rng.normal(size=(n, 59)) * 10.0 ** rng.integers(-8, 2, (n, 59))
    M1, M2 = np.zeros_like(P), np.zeros_like(P)
    mask = (rng.random(n) < 0.6).astype(np.uint8)
    step = np.ones(n, np.int64)
    orc.adam(P, G, M1, M2, mask, step, lr=1e-3, eps=1e-15)
    exp = P0 - 1e-3 * G / (np.abs(G) + 1e-15)
    m = mask.astype(bool)
    np.testing.assert_allclose(P[m], exp[m], rtol=0, atol=1e-15)
    assert np.array_equal(P[~m], P0[~m])
    assert not M1[~m].any() and not M2[~m].any()


def test_adam_matches_torch_many_steps(orc):
    """Several steps agree with torch.optim.Adam (float64, same constants)."""
    import torch
    rng = np.random.default_rng(3)
    n = 8
    P = rng.normal(size=(n, 59))
    th = torch.tensor(P.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([th], lr=1e-3, betas=(0.9, 0.999), eps=1e-15)
    M1, M2 = np.zeros_like(P), np.zeros_like(P)
    for s in range(1, 6):
        G = rng.normal(size=(n, 59))
        th.grad = torch.tensor(G)
        opt.step()
        orc.adam(P, G, M1, M2, np.ones(n, np.uint8), np.full(n, s, np.int64), lr=1e-3)
    np.testing.assert_allclose(P, th.detach().numpy(), rtol=0, atol=1e-13)


def test_adam_group_rates_match_torch_param_groups(orc):
    """Per-group learning rates (means, log-scales, rotation, opacity, SH DC,
    SH rest) agree with torch.optim.Adam over six parameter groups, and the
    means' rate follows the log-linear 3DGS decay (closed form at both ends and
    midway the geometric mean)."""
    import torch
    rng = np.random.default_rng(4)
    n = 6
    rates = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3, 1.25e-4]
    P = rng.normal(size=(n, 59))
    cols = orc.LR_GROUP_COLUMNS
    ts = [torch.tensor(P[:, a:b].copy(), requires_grad=True) for a, b in cols]
    opt = torch.optim.Adam([{"params": [t], "lr": r} for t, r in zip(ts, rates)], betas=(0.9, 0.999), eps=1e-15)
    M1, M2 = np.zeros_like(P), np.zeros_like(P)
    for s in range(1, 5):
        G = rng.normal(size=(n, 59))
        for t, (a, b) in zip(ts, cols):
            t.grad = torch.tensor(G[:, a:b])
        opt.step()
        orc.adam(P, G, M1, M2, np.ones(n, np.uint8), np.full(n, s, np.int64), lr=orc.group_lr(rates))
    got = np.concatenate([t.detach().numpy() for t in ts], 1)
    np.testing.assert_allclose(P, got, rtol=0, atol=1e-13)
    assert orc.lr_schedule_groups(rates, 1.6e-6, 100, 0)[0] == rates[0]
    assert abs(orc.lr_schedule_groups(rates, 1.6e-6, 100, 100)[0] - 1.6e-6) < 1e-18
    assert abs(orc.lr_schedule_groups(rates, 1.6e-6, 100, 50)[0] - np.sqrt(1.6e-4 * 1.6e-6)) < 1e-15
    assert orc.lr_schedule_groups(rates, 1.6e-6, 100, 50)[1:] == rates[1:]
