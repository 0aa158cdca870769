"""Comparison helpers shared by the GPU parity tests (test infrastructure)."""
import json
import os

import numpy as np

import scenes


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def image_within(gpu_img, orc_rec, tol=1e-4):
    """Max-abs image error with the oracle's per-pixel slack for borderline
    decisions (alpha near 1/255, the T stop, border Gaussians): every pixel
    must be within tol + slack; returns (max error on slack-free pixels,
    fraction of pixels with slack)."""
    err = np.abs(np.asarray(gpu_img, np.float64) - orc_rec["img"]).max(axis=2)
    sl = orc_rec["slack"]
    bad = err > tol + sl
    assert not bad.any(), f"{bad.sum()} pixels beyond tolerance; worst {err[bad].max()} at {np.argwhere(bad)[:5]}"
    clean = sl == 0
    return float(err[clean].max()) if clean.any() else 0.0, float((~clean).mean())


def c1_inputs(orc, block_size=1250, n=20000, size=256):
    cfg = scenes.small_cube_config(n=n, size=size)
    perm, Pm = orc.create(cfg["params"], block_size)
    target_p = scenes.perturb(cfg["params"], seed=77)
    return cfg, perm, Pm, target_p


def report(config, form, **errors):
    """Appends one record of measured errors against the FP64 oracle (image
    max-abs on slack-free pixels, gradient rel-L2, ...) to the JSON-lines
    file named by TGS_PARITY_REPORT, when set; the tests assert their bounds
    either way."""
    path = os.environ.get("TGS_PARITY_REPORT")
    if not path:
        return
    rec = {"config": config, "form": form}
    rec.update({k: float(v) for k, v in errors.items()})
    with open(path, "a") as f:
        f.write(json.dumps(rec) + "\n")
