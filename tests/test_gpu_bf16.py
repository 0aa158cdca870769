"""BF16 host tier and cache (SH-rest coefficients and Adam moments stored as
BF16, all arithmetic FP32) against the FP64 oracle run on the same
BF16-rounded parameters: images max-abs 1e-4 (+ slack), 2D gradients rel-L2
1e-3, every stored BF16 value one of the two BF16 neighbours of the exact
update (stochastic rounding), and the rounding unbiased on average."""
import numpy as np
import pytest

import scenes
from parity_util import c1_inputs, image_within, rel_l2, report

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """Round-to-nearest-even to BF16, returned as float64 (test-side helper)."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_ulp(x):
    x = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(x, 1e-30)))
    return 2.0 ** (e - 7)


# 1250: the BF16 record's slots start on odd floats (Adam per Gaussian);
# 1000: even slot, moment and field offsets (Adam on pairs of Gaussians)
@pytest.mark.parametrize("B", [1250, 1000])
def test_bf16_step_matches_oracle(orc, tgs, B):
    c, perm, Pm, tp = c1_inputs(orc, block_size=B)
    cams = [scenes.camera_array(x) for x in c["cams"]]
    _, Pt = orc.create(tp, B)
    target = orc.render(Pt.astype(np.float64), cams[0])["img"].astype(np.float32)
    table = tgs.TideTable(c["params"], block_size=B, max_batch=1, max_width=256, max_height=256, loss=1,
                          host_bf16=1, stochastic_round=1)
    table.step([c["cams"][0]], target[None])
    # oracle on the BF16-rounded table
    Pb = Pm.astype(np.float64).copy()
    Pb[:, 14:] = bf16_round(Pm[:, 14:])
    P0 = Pb.copy()
    M1, M2 = np.zeros_like(Pb), np.zeros_like(Pb)
    steps = np.zeros((Pm.shape[0] + B - 1) // B, np.int64)
    sph = orc.block_spheres(Pm.astype(np.float64), B)
    _, vis = orc.visible_blocks(sph, [cams[0]])
    o = orc.train_step(Pb, M1, M2, steps, B, np.nonzero(vis)[0], [cams[0]], target[None], lr=1e-3,
                       loss_kind=1)
    rec = table.camera_record(0, 256, 256)
    err, frac = image_within(rec["image"], o["records"][0])
    assert err <= 1e-4 and frac < 0.05
    vg = rec["splat"][:, 11] != 0
    vo = o["records"][0]["S"][:, orc.VISIBLE] != 0
    for q in range(9):
        assert rel_l2(rec["grad2d"][vg & vo, q], o["g2"][0][vg & vo, q]) < 1e-3, q
    # the same image and 2D gradients against the oracle on the unrounded
    # FP32 table: the error the BF16 record itself adds
    o32 = orc.render(Pm.astype(np.float64)[o["ids"]], cams[0], with_slack=True)
    err32 = float(np.abs(rec["image"].astype(np.float64) - o32["img"]).max())
    report(f"c1 cube-20k 256x256 B={B}", "bf16", image_maxabs=err, slack_frac=frac,
           grad2d_rel_l2=max(rel_l2(rec["grad2d"][vg & vo, q], o["g2"][0][vg & vo, q]) for q in range(9)),
           image_maxabs_vs_fp32_table=err32)
    p_g, m1, m2, st = table.state()
    ids, touched = o["ids"], o["touched"].astype(bool)
    # first moments: m = 0.1 g, stored as BF16 (one of the two neighbours)
    mo = 0.1 * o["grad"][touched]
    mg = m1[ids][touched].astype(np.float64)
    scale = np.abs(mo).max(0)
    ok = np.abs(mg - mo) <= bf16_ulp(mo) * 1.01 + 1e-3 * scale
    assert ok.mean() > 0.999
    # FP32 fields move like the oracle; BF16 fields land on a neighbour of the exact update
    d32 = np.abs(p_g[ids][touched][:, :14].astype(np.float64) - Pb[ids][touched][:, :14])
    amb = np.abs(o["grad"][touched][:, :14]) < 1e-4 * np.abs(o["grad"][touched][:, :14]).max(0)
    assert (d32 <= 1e-6 + 2.1e-3 * amb).all()
    exact = Pb[ids][touched][:, 14:]
    got = p_g[ids][touched][:, 14:].astype(np.float64)
    assert (np.abs(got - exact) <= bf16_ulp(exact) * 1.01 + 1e-9).mean() > 0.999
    # unbiased on average: mean rounding error well below one ulp
    rel = (got - exact) / bf16_ulp(exact)
    moved = np.abs(P0[ids][touched][:, 14:] - exact) > 0
    assert abs(rel[moved].mean()) < 0.05
    # untouched rows keep their BF16 values
    untouched = np.setdiff1d(np.arange(len(p_g)), ids[touched])
    assert np.array_equal(p_g[untouched].astype(np.float64), P0[untouched])
    table.close()


def test_bf16_record_halves_link_bytes(orc, tgs):
    c, perm, Pm, tp = c1_inputs(orc)
    tgt = np.zeros((1, 256, 256, 3), np.float32)
    out = {}
    for bf in (0, 1):
        t = tgs.TideTable(c["params"], block_size=1250, max_batch=1, max_width=256, max_height=256, host_bf16=bf)
        t.step([c["cams"][0]], tgt)
        out[bf] = t.stats()["bytes_h2d"]
        t.close()
    assert out[0] == 16 * 1250 * 708 and out[1] == 16 * 1250 * 382
