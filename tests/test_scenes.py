"""Pins of the seeded input generators (CPU): SplitMix64 against its published
test vector, the counter-based streams' independence of the requested range,
the torch streams (used for scenes of 10^8 Gaussians) against the numpy ones,
the moments of the uniform and Box-Muller normal draws, and the street
scene's neighbourhood rows against the same rows of the full table (the
full-size parity tests run the oracle on such neighbourhoods)."""
import numpy as np

import scenes


def test_splitmix64_published_sequence():
    # the first five outputs of SplitMix64 seeded with 1234567, the test
    # vector that accompanies the generator's public reference code
    want = np.array([6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
                     16408922859458223821], np.uint64)
    with np.errstate(over="ignore"):
        got = scenes._mix64(np.uint64(1234567) + np.arange(1, 6, dtype=np.uint64) * scenes.GAMMA)
    assert np.array_equal(got, want)


def test_streams_are_counter_based():
    full = scenes.u64(7, 3, 0, 1000)
    assert np.array_equal(scenes.u64(7, 3, 400, 100), full[400:500])
    assert not np.any(scenes.u64(7, 4, 0, 1000) == full)
    assert not np.any(scenes.u64(8, 3, 0, 1000) == full)
    z = scenes.normal(7, 3, 500)
    assert np.array_equal(scenes.normal(7, 3, 100, start=200), z[200:300])
    u = scenes.uniform(7, 3, 500, -2.0, 3.0)
    assert np.array_equal(scenes.uniform(7, 3, 50, -2.0, 3.0, start=450), u[450:])


def test_torch_streams_match_numpy():
    import torch
    a = scenes.u64(11, 5, 123, 4096).view(np.int64)
    b = scenes.t_u64(11, 5, 123, 4096, "cpu").numpy()
    assert np.array_equal(a, b)
    idx = torch.tensor([0, 1, 17, 4095, 10 ** 9], dtype=torch.int64)
    at = scenes.t_u64_at(11, 5, idx).numpy()
    ref = np.concatenate([scenes.u64(11, 5, int(i), 1) for i in idx]).view(np.int64)
    assert np.array_equal(at, ref)
    assert np.array_equal(scenes.t_uniform(11, 5, 4096, -1.0, 2.0, device="cpu").numpy(),
                          scenes.uniform(11, 5, 4096, -1.0, 2.0))
    np.testing.assert_allclose(scenes.t_normal(11, 5, 4096, 0.5, 2.0, device="cpu").numpy(),
                               scenes.normal(11, 5, 4096, 0.5, 2.0), rtol=0, atol=1e-13)


def test_uniform_and_normal_moments():
    m = 1_000_000
    u = scenes.uniform(1, 2, m)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * (1 / 12) ** 0.5 / m ** 0.5
    assert abs(u.var() - 1 / 12) < 1e-3
    z = scenes.normal(1, 2, m)
    assert abs(z.mean()) < 5 / m ** 0.5
    assert abs(z.std() - 1.0) < 5e-3
    assert abs(np.mean(z ** 4) - 3.0) < 0.05  # Gaussian kurtosis
    assert abs(np.mean(np.abs(z) < 1.0) - 0.682689492) < 3e-3


def test_street_neighbourhood_rows_equal_the_full_table():
    import torch
    n = 200_000
    full, sp = scenes.street_scene(n, device="cpu", chunk=1 << 16)
    c = np.array([10.0, -40.0, 1.5])
    r = 400.0
    rows, idx, sp2 = scenes.street_scene(n, device="cpu", chunk=50_000, near=(c, r))
    assert sp == sp2
    sel = ((full[:, :3].double() - torch.tensor(c)) ** 2).sum(1) < r * r
    want = torch.nonzero(sel).squeeze(1)
    assert len(want) > 1000
    assert torch.equal(idx, want)
    assert torch.equal(rows, full[want])
    # quaternions unit, opacity logits and log-scales finite
    q = full[:, 6:10].double()
    assert torch.allclose(q.norm(dim=1), torch.ones(n, dtype=torch.float64), atol=1e-6)
    assert torch.isfinite(full).all()
