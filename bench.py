"""Benchmark of the TideGS training step on B300 (train iterations per second).

Workload (default): the fully resident FP32 aerial configuration -- 2,000,000
Gaussians over a synthetic 1 km x 1 km block scene (jittered ground grid plus
box buildings), 100 cameras on a circular orbit at 150 m altitude, 1920x1080,
batch 1, one training step = cull + residency + Level-2 forward + L1 loss +
backward + masked Adam + bound refresh, cameras taken in orbit order with the
next camera prefetched.  Targets are renders of the unperturbed scene; training
starts from a perturbed copy.  The per-step state (1.4 GB of parameters and
moments) exceeds the 126 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "train iters/s, learned+BF16 vs plain FP32 path at <=0.1 dB PSNR gap; link GB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--cams", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def build_workload(args):
    cfg = scenes.aerial_config(n=args.n, n_cams=args.cams)
    gt = cfg["params"]
    train = scenes.perturb(gt, seed=2001, mean_std=0.02 * cfg["spacing"])
    return cfg, gt, train


def run_ours(args, rank, world, local):
    import torch
    import paper_2605_20150_b300 as tgs
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, gt, train = build_workload(args)
    cams = cfg["cams"]
    W, H = cams[0]["width"], cams[0]["height"]
    J = 1
    tcfg = dict(block_size=4096, max_batch=J, max_width=W, max_height=H, cache_blocks=0, prefetch_mode=1, loss=0)
    # targets: renders of the unperturbed scene by the same library
    ref = tgs.TideTable(gt, **tcfg)
    targets = torch.empty(len(cams), H, W, 3, device=dev, dtype=torch.float32)
    for i, c in enumerate(cams):
        ref.render(c, targets[i])
    torch.cuda.synchronize()
    ref.close()
    del ref
    table = tgs.TideTable(train, **tcfg)
    nc = len(cams)

    def one(t, want_loss=False):
        return table.step([cams[t % nc]], targets[t % nc:t % nc + 1], next_cams=[cams[(t + 1) % nc]],
                          want_loss=want_loss)

    for t in range(args.warmup):
        one(t)
    table.sync()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = table.stats()["kernel_launches"]
    table.stage_timing(True)
    table.stage_ms(reset=True)
    clk = ClockSampler(local)
    clk.start()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for t in range(args.warmup, args.warmup + args.steps):
        one(t)
    e1.record(s)
    table.sync()
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    stages = table.stage_ms(reset=True)
    table.stage_timing(False)
    st = table.stats()
    launches = st["kernel_launches"] - launches0
    rec = table.camera_record(0, W, H)
    if world > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    # ---- end to end through the C ABI with host buffers: targets from pinned
    # host memory copied inside every step, the loss read back every step
    host_t = torch.empty(len(cams), H, W, 3, dtype=torch.float32, pin_memory=True)
    host_t.copy_(targets.cpu())
    host_np = host_t.numpy()
    n_e2e = max(5, args.steps // 2)
    for t in range(2):
        table.step([cams[t % nc]], host_np[t % nc:t % nc + 1], next_cams=[cams[(t + 1) % nc]], want_loss=True)
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(s)
    t0 = time.perf_counter()
    for t in range(n_e2e):
        table.step([cams[t % nc]], host_np[t % nc:t % nc + 1], next_cams=[cams[(t + 1) % nc]], want_loss=True)
    e3.record(s)
    torch.cuda.synchronize()
    wall_e2e = time.perf_counter() - t0
    e2e_ms = max(e2.elapsed_time(e3), 1e3 * wall_e2e) / n_e2e
    return dict(ms=ms, stages=stages, stats=st, launches=launches, clocks=clocks, rec=rec, table=table,
                cfg=cfg, W=W, H=H, e2e_ms=e2e_ms, bytes_in=J * H * W * 3 * 4, train=train)


def roofline(res, steps):
    """Roofline of the dominant stage.  Adam: HBM-bound, 1,652 B per touched
    Gaussian (read p, g, m, v; write p, m, v; FP32 x 59).  Raster: plain FP32
    ALU + MUFU exp, reported as evaluated (pixel, Gaussian) pairs per second."""
    hbm, src = measured_peaks()
    stages = res["stages"]
    name = max(stages, key=lambda k: stages[k][0])
    ms_per = stages[name][0] / max(1, stages[name][1])
    out = {"stage": name, "ms_per_launch": round(ms_per, 4)}
    st = res["stats"]
    if name == "adam":
        touched = st["last_visible"]
        traffic = 1652.0 * touched
        gbs = traffic / (ms_per * 1e-3) / 1e9
        out.update(bound="hbm", achieved=round(gbs, 1), peak=hbm, unit="GB/s", frac=round(gbs / hbm, 4),
                   traffic=None, peak_source=src)
    elif name in ("raster_fwd", "raster_bwd"):
        nl = res["rec"]["n_last"].astype(np.float64)
        evals = float(nl.sum())
        # peak: one exp per evaluation on the MUFU units: 148 SMs x 16 /clk x 2.032 GHz
        peak = 148 * 16 * 2.032e9 / 1e12
        ach = evals / (ms_per * 1e-3) / 1e12
        out.update(bound="alu", achieved=round(ach, 4), peak=round(peak, 3), unit="Teval/s",
                   frac=round(ach / peak, 4), traffic=None, peak_source="derived: MUFU ex2 16/clk/SM")
    else:
        vis = st["last_visible"]
        bytes_ = 236.0 * vis + 48 * vis
        gbs = bytes_ / (ms_per * 1e-3) / 1e9
        out.update(bound="hbm", achieved=round(gbs, 1), peak=hbm, unit="GB/s", frac=round(gbs / hbm, 4),
                   traffic=None, peak_source=src)
    return out


def cpu_baseline(res, budget_s=20.0):
    """The FP64 oracle (as it stands) on a bounded sample of one step: the
    blocks nearest the image centre of camera 0 rendered at full resolution
    with backward and Adam; iters/s scaled by the fraction of the render set
    the sample covers."""
    import oracle
    oracle.build()
    cfg, train = res["cfg"], res["train"]
    cam = scenes.camera_array(cfg["cams"][0])
    B = 4096
    perm, P = oracle.create(train, B)
    P = P.astype(np.float64)
    sph = oracle.block_spheres(P, B)
    _, vis = oracle.visible_blocks(sph, [cam])
    blocks = np.nonzero(vis)[0]
    target = np.zeros((1, int(cam[1]), int(cam[0]), 3))

    def run(n_sample):
        pick = blocks[np.linspace(0, len(blocks) - 1, n_sample).astype(int)]
        M1, M2 = np.zeros_like(P), np.zeros_like(P)
        steps = np.zeros(len(sph), np.int64)
        t0 = time.perf_counter()
        oracle.train_step(P.copy(), M1, M2, steps, B, pick, [cam], target, lr=1e-3, loss_kind=0)
        return time.perf_counter() - t0

    n_sample = max(1, min(len(blocks), 4))
    dt = run(n_sample)
    if dt < budget_s / 4 and n_sample < len(blocks):
        n_sample = int(min(len(blocks), max(n_sample + 1, n_sample * budget_s / max(dt, 1e-3))))
        dt = run(n_sample)
    frac = n_sample / max(1, len(blocks))
    its = frac / dt
    return {"value": round(its, 6), "unit": "train iters/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n_sample} of {len(blocks)} visible 4096-Gaussian blocks of camera 0 at 1920x1080, "
                      f"forward+backward+Adam in FP64, {dt:.1f} s, scaled by the block fraction"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        if rank != 0:
            return
        cfg, gt, train = build_workload(args)
        res = {"cfg": cfg, "train": train}
        times = []
        for _ in range(args.warmup):
            pass
        cb = None
        for _ in range(max(1, min(args.steps, 3))):
            cb = cpu_baseline(res)
            times.append(1.0 / cb["value"])
        v = 1.0 / statistics.median(times)
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "train iters/s",
                "n_gpus": args.gpus, "steps": len(times), "warmup": args.warmup,
                "ms_per_step": round(1e3 / v, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": "aerial-2M-1080p-resident-fp32", "global_batch": 1, "n_gaussians": args.n},
                "cpu_baseline": cb,
                "e2e": {"value": round(v, 6), "unit": "train iters/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    res = run_ours(args, rank, world, local)
    ms_step = res["ms"] / args.steps
    value = world * 1e3 / ms_step
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "train iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "aerial-2M-1080p-resident-fp32", "n_gaussians": args.n, "block_size": 4096,
                   "image": f"{res['W']}x{res['H']}", "global_batch": world, "cameras": args.cams,
                   "parallelism": f"replicas{world}", "l2": "per-step state 1.4 GB > 126 MB L2, no flush"},
        "e2e": {"value": round(world * 1e3 / res["e2e_ms"], 3), "unit": "train iters/s",
                "h2d_bytes_per_step": res["bytes_in"], "d2h_bytes_per_step": 4},
        "gpu_launches": int(res["launches"]),
        "roofline": roofline(res, args.steps),
        "clocks": res["clocks"],
        "stages_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in res["stages"].items()},
        "visible": res["stats"]["last_visible"], "pairs": res["stats"]["last_pairs"],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(res)
    res["table"].close()
    if rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
