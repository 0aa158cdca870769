"""Parity of the mixed-city configuration's step: a batch of four 1920x1080
cameras (two aerial lawnmower frames at 150 m, pitch 45 degrees, and two
street-drive frames at 1.5 m) on the mixed aerial + street city scene, SH-rest
coefficients and Adam moments BF16 in the host tier and the cache, an HBM
cache of half the scene's blocks (the batch's working set streams in), the
benchmark's L1 + D-SSIM loss.  The scene has 2M Gaussians (the benchmark runs
the same generator at the largest N the host holds), so the FP64 oracle can
run the whole batch on the BF16-rounded table:
  - the batch's visible block set is the oracle's Level-1 set;
  - each camera's image matches to max-abs 1e-4 (plus the oracle's slack for
    borderline FP32 decisions) and the batch loss to 1e-4 relative;
  - each camera's 2D gradients match to rel-L2 1e-3 (the L1 sign decided on
    the GPU's images on both sides);
  - the first Adam moments of the touched rows are BF16 neighbours of 0.1 g,
    g the oracle's gradient summed over the four cameras; the FP32 fields
    moved by one Adam step of g and the untouched rows kept their values."""
import numpy as np
import pytest

import scenes
from parity_util import image_within, rel_l2, report
from test_gpu_bf16 import bf16_round, bf16_ulp

pytestmark = pytest.mark.gpu

N = 2_000_000
B = 4096


def test_city_batch4_bf16_step_matches_oracle(orc, tgs):
    import torch
    from oracle import ssim as ossim
    dev = torch.device("cuda", 0)
    host = np.empty((N, 59), np.float32)
    scenes.street_scene(N, device=dev, roof_frac=0.3, chunk=1 << 22, out_host=host)
    allc = scenes.city_cameras(2000)
    cams = [allc[0], allc[1], allc[1000], allc[1001]]
    J = len(cams)
    W, H = cams[0]["width"], cams[0]["height"]
    K = (N + B - 1) // B
    perm, Pm = orc.create(host, B)
    Pb = Pm.astype(np.float64)
    Pb[:, 14:] = bf16_round(Pm[:, 14:])
    cas = [scenes.camera_array(c) for c in cams]
    # targets: the oracle's renders of the table with its SH DC perturbed
    Pt = Pb.copy()
    Pt[:, 11:14] += np.random.default_rng(5).normal(0.0, 0.1, (N, 3))
    tgt = np.stack([orc.render(Pt, ca)["img"] for ca in cas]).astype(np.float32)
    del Pt
    table = tgs.TideTable(host, block_size=B, max_batch=J, max_width=W, max_height=H, cache_blocks=K // 2,
                          spare_slots=64, prefetch_mode=0, loss=2, host_bf16=1, stochastic_round=1)
    lval = table.step(cams, tgt)
    sets = table.sets(J)
    recs = [table.camera_record(j, W, H) for j in range(J)]
    p_g, m1, _, steps_g = table.state()
    table.close()
    del host

    sph = orc.block_spheres(Pb, B)
    _, vis = orc.visible_blocks(sph, cas)
    assert np.array_equal(sets["k_visible"], vis)
    render_blocks = np.nonzero(vis & sets["r_resident"])[0]
    assert 0 < len(render_blocks) <= K // 2
    ids = np.concatenate([np.arange(k * B, min((k + 1) * B, N)) for k in render_blocks])
    Ps = Pb[ids]
    orecs = [orc.render(Ps, ca, with_slack=True) for ca in cas]
    imgs_o = np.stack([r["img"] for r in orecs])
    tg = tgt.astype(np.float64)
    lo, _ = orc.loss(imgs_o, tg, 2)
    assert abs(lval - lo) <= 1e-4 * lo
    # dL/dimage with the L1 sign taken on the GPU's images
    sg = np.sign(np.stack([r["image"] for r in recs]).astype(np.float64) - tg)
    dimg = 0.8 * sg / tg.size - 0.2 * ossim.ssim_grad(imgs_o, tg)
    g_ref = np.zeros_like(Ps)
    touched = np.zeros(len(ids), bool)
    for j in range(J):
        rec, orj = recs[j], orecs[j]
        assert np.array_equal(rec["ids"], ids)
        err, frac = image_within(rec["image"], orj)
        assert err <= 1e-4 and frac < 0.05, (j, err, frac)
        gj, g2 = orc.render_grad(Ps, cas[j], orj, dimg[j])
        g_ref += gj
        vg = rec["splat"][:, 11] != 0
        vo = orj["S"][:, orc.VISIBLE] != 0
        touched |= vo
        both = vg & vo
        assert both.sum() > 1000, j
        r2 = [rel_l2(rec["grad2d"][both, q], g2[both, q]) for q in range(9)]
        for q in range(9):
            assert r2[q] < 1e-3, (j, q)
        report(f"c4 city-2M batch 4 1920x1080 camera {j}", "bf16", image_maxabs=err, slack_frac=frac,
               grad2d_rel_l2=max(r2))
    # step counters: blocks with a touched row
    want_steps = np.zeros(K, np.uint32)
    want_steps[np.unique(ids[touched] // B)] = 1
    assert np.array_equal(steps_g, want_steps)
    # first moments: m = 0.1 g stored as BF16 (one of the two neighbours)
    mo = 0.1 * g_ref[touched]
    mg = m1[ids][touched].astype(np.float64)
    ok = np.abs(mg - mo) <= bf16_ulp(mo) * 1.01 + 1e-3 * np.abs(mo).max(0)
    assert ok.mean() > 0.999
    # FP32 fields: one Adam step of the reference gradient (zero moments, step 1)
    P1 = Ps.copy()
    orc.adam(P1, g_ref, np.zeros_like(P1), np.zeros_like(P1), touched.astype(np.uint8),
             np.ones(len(ids), np.int64), lr=1e-3)
    d_g = p_g[ids][touched][:, :14].astype(np.float64) - Ps[touched][:, :14]
    d_o = P1[touched][:, :14] - Ps[touched][:, :14]
    gt = np.abs(g_ref[touched][:, :14])
    amb = gt < 1e-4 * gt.max(0)
    assert (np.abs(d_g - d_o) <= 1e-6 + 2.4e-7 * np.abs(Ps[touched][:, :14]) + 2.1e-3 * amb).all()
    # untouched rows keep their (BF16-rounded) values
    moved = np.zeros(N, bool)
    moved[ids[touched]] = True
    assert np.array_equal(p_g[~moved].astype(np.float64), Pb[~moved])
