"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module only draws random numbers and builds camera poses; it holds none
of the method's arithmetic (no projection, culling, compositing or
optimiser).  Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): value i of stream `key` is mix64(key + (i + 1) * GAMMA), so any
index range can be produced independently of the others.

Parameter rows are float32 [n, 59] in the paper's logical layout (Sec. 2,
D = 59): mean (3), log-scale (3), quaternion w,x,y,z (4), opacity logit (1),
SH DC rgb (3), SH rest 15 x rgb (45, coefficient-major, l = 1..3, m = -l..l).

Cameras are dicts with width, height, fx, fy, cx, cy, znear, zfar and R, t of
the world-to-camera map x_c = R x_w + t (camera looks down +z, y down, x
right); pixels are sampled at integer coordinates, so the principal point of a
centred camera is (W/2 - 0.5, H/2 - 0.5).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
D = 59


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF],
                     dtype=np.uint64)
        return _mix64(s)[0]


def u64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(key + idx * GAMMA)


def uniform(seed: int, stream: int, count: int, lo=0.0, hi=1.0, start: int = 0) -> np.ndarray:
    """Uniform doubles in [lo, hi): top 53 bits of each draw."""
    x = (u64(seed, stream, start, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * x


def normal(seed: int, stream: int, count: int, mean=0.0, std=1.0, start: int = 0) -> np.ndarray:
    """Box-Muller normals from pairs of uniforms of the same stream."""
    u = (u64(seed, stream, 2 * start, 2 * count) >> np.uint64(11)).astype(np.float64)
    u *= 1.0 / 9007199254740992.0
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return mean + std * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------
def look_at(pos, target, up=(0.0, 1.0, 0.0)):
    """World-to-camera R, t for a camera at `pos` looking at `target`."""
    pos = np.asarray(pos, np.float64)
    z = np.asarray(target, np.float64) - pos
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ pos
    return R, t


def pinhole(width, height, fov_x_deg, R, t, znear=0.2, zfar=100.0):
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return dict(width=int(width), height=int(height), fx=fx, fy=fx,
                cx=width / 2.0 - 0.5, cy=height / 2.0 - 0.5,
                znear=float(znear), zfar=float(zfar),
                R=np.asarray(R, np.float64), t=np.asarray(t, np.float64))


def rot_y(deg):
    a = math.radians(deg)
    return np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])


# ----------------------------------------------------------------------------
# Gaussian tables
# ----------------------------------------------------------------------------
def _assemble(means, logs, quats, opac, sh):
    n = means.shape[0]
    p = np.empty((n, D), np.float32)
    p[:, 0:3] = means
    p[:, 3:6] = logs
    p[:, 6:10] = quats
    p[:, 10] = opac
    p[:, 11:59] = sh.reshape(n, 48)
    return p


def random_quats(seed, stream, n):
    q = normal(seed, stream, 4 * n).reshape(n, 4)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def cube_scene(n=20000, seed=1000, log_scale_mean=-4.0, log_scale_std=0.5, sh_std=0.2, extent=1.0):
    """Means uniform in [-extent, extent]^3, log-scales N(mean, std), random unit
    quaternions, opacity logit N(0, 1), 48 SH coefficients N(0, sh_std)."""
    means = uniform(seed, 1, 3 * n, -extent, extent).reshape(n, 3)
    logs = normal(seed, 2, 3 * n, log_scale_mean, log_scale_std).reshape(n, 3)
    quats = random_quats(seed, 3, n)
    opac = normal(seed, 4, n)
    sh = normal(seed, 5, 48 * n, 0.0, sh_std).reshape(n, 16, 3)
    return _assemble(means, logs, quats, opac, sh)


def perturb(params, seed, mean_std=0.02, logscale_std=0.1, opacity_std=0.5, sh_std=0.05):
    """Training start (or target source): Gaussian noise on means, log-scales,
    opacity logits and SH coefficients; quaternions are left unchanged."""
    n = params.shape[0]
    p = params.astype(np.float64).copy()
    p[:, 0:3] += normal(seed, 11, 3 * n, 0.0, mean_std).reshape(n, 3)
    p[:, 3:6] += normal(seed, 12, 3 * n, 0.0, logscale_std).reshape(n, 3)
    p[:, 10] += normal(seed, 13, n, 0.0, opacity_std)
    p[:, 11:59] += normal(seed, 14, 48 * n, 0.0, sh_std).reshape(n, 48)
    return p.astype(np.float32)


def small_cube_config(seed=1000, n=20000, size=256):
    """20,000 Gaussians in [-1,1]^3 (log-scale N(-4, 0.5), opacity logit N(0,1),
    SH N(0, 0.2)), grouped in 16 blocks of 1,250; a 256x256 camera with a 60
    degree field of view at distance 3 looking at the origin, and a second
    camera rotated 20 degrees about the world y axis."""
    params = cube_scene(n, seed)
    p1 = np.array([0.0, 0.0, -3.0])
    R1, t1 = look_at(p1, [0, 0, 0])
    p2 = rot_y(20.0) @ p1
    R2, t2 = look_at(p2, [0, 0, 0])
    cams = [pinhole(size, size, 60.0, R1, t1), pinhole(size, size, 60.0, R2, t2)]
    return dict(params=params, cams=cams, block_size=(n + 15) // 16)


def aerial_block_scene(n=2_000_000, seed=1001, side=1000.0, n_boxes=150, ground_frac=0.8):
    """Aerial block scene (world z up): a jittered ground grid at z=0 plus box
    buildings (footprint U[10,40] m, height U[10,80] m) whose walls and roofs
    carry the remaining Gaussians (area-weighted).  Log-scales log(0.5 *
    spacing) + N(0, 0.3); SH DC from a smooth colour field, the rest N(0,
    0.05); opacity logit N(2, 0.5)."""
    n_ground = int(n * ground_frac)
    g = int(math.ceil(math.sqrt(n_ground)))
    spacing = side / g
    ii = np.arange(n_ground)
    gx = (ii % g + 0.5) * spacing - side / 2
    gy = (ii // g + 0.5) * spacing - side / 2
    jit = uniform(seed, 21, 2 * n_ground, -0.4 * spacing, 0.4 * spacing).reshape(n_ground, 2)
    ground = np.stack([gx + jit[:, 0], gy + jit[:, 1], np.zeros(n_ground)], 1)
    nb = n - n_ground
    # boxes
    cxy = uniform(seed, 22, 2 * n_boxes, -side / 2 + 40, side / 2 - 40).reshape(n_boxes, 2)
    fw = uniform(seed, 23, 2 * n_boxes, 10.0, 40.0).reshape(n_boxes, 2)
    hh = uniform(seed, 24, n_boxes, 10.0, 80.0)
    # faces: 4 walls + roof, areas
    areas = np.stack([fw[:, 0] * hh, fw[:, 0] * hh, fw[:, 1] * hh, fw[:, 1] * hh, fw[:, 0] * fw[:, 1]], 1)
    flat = areas.reshape(-1)
    cdf = np.cumsum(flat) / flat.sum()
    pick = np.searchsorted(cdf, uniform(seed, 25, nb), side="right")
    pick = np.minimum(pick, flat.size - 1)
    box = pick // 5
    face = pick % 5
    a = uniform(seed, 26, nb)
    b = uniform(seed, 27, nb)
    wx, wy, h = fw[box, 0], fw[box, 1], hh[box]
    x0, y0 = cxy[box, 0] - wx / 2, cxy[box, 1] - wy / 2
    pts = np.empty((nb, 3))
    # face 0: y = y0 wall, 1: y = y0 + wy, 2: x = x0, 3: x = x0 + wx, 4: roof
    m = face == 0; pts[m] = np.stack([x0[m] + a[m] * wx[m], y0[m], b[m] * h[m]], 1)
    m = face == 1; pts[m] = np.stack([x0[m] + a[m] * wx[m], y0[m] + wy[m], b[m] * h[m]], 1)
    m = face == 2; pts[m] = np.stack([x0[m], y0[m] + a[m] * wy[m], b[m] * h[m]], 1)
    m = face == 3; pts[m] = np.stack([x0[m] + wx[m], y0[m] + a[m] * wy[m], b[m] * h[m]], 1)
    m = face == 4; pts[m] = np.stack([x0[m] + a[m] * wx[m], y0[m] + b[m] * wy[m], h[m]], 1)
    means = np.concatenate([ground, pts], 0)
    logs = (math.log(0.5 * spacing) + normal(seed, 28, 3 * n, 0.0, 0.3)).reshape(n, 3)
    quats = random_quats(seed, 29, n)
    opac = normal(seed, 30, n, 2.0, 0.5)
    col = np.stack([0.5 + 0.3 * np.sin(means[:, 0] / 37.0 + 0.3 * c) * np.cos(means[:, 1] / 53.0 - 0.7 * c)
                    + 0.1 * np.sin(means[:, 2] / 11.0 + c) for c in range(3)], 1)
    sh = normal(seed, 31, 48 * n, 0.0, 0.05).reshape(n, 16, 3)
    sh[:, 0, :] = (col - 0.5) * 3.5  # smooth DC field, roughly +-1
    return _assemble(means, logs, quats, opac, sh), spacing


def orbit_cameras(n_cams=100, radius=500.0, altitude=150.0, width=1920, height=1080, fov_x=60.0,
                  znear=0.2, zfar=2000.0, phase=0.0):
    """Cameras on a circle around the origin at `altitude`, looking at the centre (world z up)."""
    cams = []
    for i in range(n_cams):
        a = phase + 2 * math.pi * i / n_cams
        pos = [radius * math.cos(a), radius * math.sin(a), altitude]
        R, t = look_at(pos, [0.0, 0.0, 0.0], up=(0.0, 0.0, 1.0))
        cams.append(pinhole(width, height, fov_x, R, t, znear, zfar))
    return cams


def aerial_config(n=2_000_000, seed=1001, n_cams=100, width=1920, height=1080, block_size=4096):
    params, spacing = aerial_block_scene(n, seed)
    cams = orbit_cameras(n_cams, width=width, height=height)
    return dict(params=params, cams=cams, block_size=block_size, spacing=spacing)


def camera_array(cam) -> np.ndarray:
    """The oracle's camera layout: W, H, fx, fy, cx, cy, znear, zfar, R (9), t (3)."""
    return np.concatenate([[cam["width"], cam["height"], cam["fx"], cam["fy"], cam["cx"], cam["cy"],
                            cam["znear"], cam["zfar"]], np.asarray(cam["R"]).reshape(9),
                           np.asarray(cam["t"]).reshape(3)]).astype(np.float64)


# ----------------------------------------------------------------------------
# torch backend of the same streams (for scenes of 10^8 Gaussians, generated
# on the GPU); bit-identical to the numpy functions above
# ----------------------------------------------------------------------------
def _t_lsr(z, k):
    import torch
    return (z >> k) & ((1 << (64 - k)) - 1)


def _t_mix64(z):
    m1 = int(np.int64(np.uint64(0xBF58476D1CE4E5B9).astype(np.int64)))
    m2 = int(np.int64(np.uint64(0x94D049BB133111EB).astype(np.int64)))
    z = (z ^ _t_lsr(z, 30)) * m1
    z = (z ^ _t_lsr(z, 27)) * m2
    return z ^ _t_lsr(z, 31)


def t_u64_at(seed, stream, idx):
    """int64 tensor holding the bits of draws idx (an int64 tensor) of a stream."""
    key = int(np.int64(stream_key(seed, stream).astype(np.int64)))
    gamma = int(np.int64(GAMMA.astype(np.int64)))
    return _t_mix64((idx + 1) * gamma + key)


def t_u64(seed, stream, start, count, device):
    """int64 tensor holding the bits of draws [start, start+count) of a stream."""
    import torch
    return t_u64_at(seed, stream, torch.arange(start, start + count, dtype=torch.int64, device=device))


def _t_unit(bits):
    import torch
    return _t_lsr(bits, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def t_uniform_at(seed, stream, idx, lo=0.0, hi=1.0):
    return lo + (hi - lo) * _t_unit(t_u64_at(seed, stream, idx))


def t_normal_at(seed, stream, idx, mean=0.0, std=1.0):
    """Box-Muller normal of element idx: draws 2 idx and 2 idx + 1."""
    u1 = 1.0 - _t_unit(t_u64_at(seed, stream, 2 * idx))
    u2 = _t_unit(t_u64_at(seed, stream, 2 * idx + 1))
    return mean + std * torch_sqrt_log_cos(u1, u2)


def torch_sqrt_log_cos(u1, u2):
    import torch
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


def t_uniform(seed, stream, count, lo=0.0, hi=1.0, start=0, device="cuda"):
    return lo + (hi - lo) * _t_unit(t_u64(seed, stream, start, count, device))


def t_normal(seed, stream, count, mean=0.0, std=1.0, start=0, device="cuda"):
    u = _t_unit(t_u64(seed, stream, 2 * start, 2 * count, device))
    return mean + std * torch_sqrt_log_cos(1.0 - u[0::2], u[1::2])


def _cols_at(seed, stream, rows, ncol, fn, **kw):
    """[len(rows), ncol] draws of elements ncol * row + c of a stream."""
    import torch
    e = rows[:, None] * ncol + torch.arange(ncol, dtype=torch.int64, device=rows.device)[None, :]
    return fn(seed, stream, e.reshape(-1), **kw).reshape(len(rows), ncol)


def street_scene(n=100_000_000, seed=1003, side=4000.0, road_every=100.0, road_width=20.0, ground_frac=0.5,
                 device="cuda", chunk=1 << 24, near=None, roof_frac=0.0, out_host=None):
    """Synthetic street grid (world z up) of n Gaussians as a float32 torch
    tensor [n, 59] on `device`: roads every 100 m over a side x side square,
    a ground layer (ground_frac of the Gaussians, uniform over the square) and
    building facades set back from the roads (heights U[10, 60] m per city
    block, Gaussians uniform over the facade area).  Log-scales log(spacing/2)
    + N(0, 0.3) with spacing the mean distance between neighbours; opacity
    logit N(2, 0.5); SH DC from a smooth field plus a per-block tint, SH rest
    N(0, 0.05).  roof_frac > 0 (the mixed aerial + street city): that
    fraction of the facade Gaussians lies on the roofs instead (uniform over
    the block interior at the block's height).  Generated in chunks of
    `chunk` rows; every value is a function of its row index only.

    near=(centre xyz, radius): return only the rows whose mean lies within
    the radius of the centre (bit-identical to those rows of the full table),
    as (rows [m, 59], row indices [m] int64, spacing).  out_host (a float32
    numpy array [n, 59]): the rows are generated on `device` chunk by chunk
    and copied into it; returns (out_host, spacing)."""
    import torch
    nb = int(side // road_every)
    heights = t_uniform(seed, 40, nb * nb, 10.0, 60.0, device=device)
    tint = t_uniform(seed, 41, 3 * nb * nb, -0.15, 0.15, device=device).reshape(nb * nb, 3)
    inner = road_every - road_width
    facade_area = (4 * inner * heights).sum().item()
    ground_area = side * side
    n_ground = int(n * ground_frac)
    spacing = math.sqrt((ground_area + facade_area) / n)
    if out_host is not None:
        out = None
    else:
        out = torch.empty((n, D), dtype=torch.float32, device=device) if near is None else []
    kept = []
    # facade sampling: block by cumulative facade area
    cdf = torch.cumsum(4 * inner * heights, 0)
    cdf = cdf / cdf[-1]
    for a in range(0, n, chunk):
        m = min(chunk, n - a)
        i = torch.arange(a, a + m, device=device)
        u1 = t_uniform_at(seed, 42, i)
        u2 = t_uniform_at(seed, 43, i)
        u3 = t_uniform_at(seed, 44, i)
        u4 = t_uniform_at(seed, 45, i)
        pos = torch.empty((m, 3), dtype=torch.float64, device=device)
        g = i < n_ground
        pos[g, 0] = u1[g] * side - side / 2
        pos[g, 1] = u2[g] * side - side / 2
        pos[g, 2] = 0.0
        f = ~g
        blk = torch.searchsorted(cdf, u3[f].contiguous()).clamp_(max=nb * nb - 1)
        bx = (blk // nb).to(torch.float64)
        by = (blk % nb).to(torch.float64)
        h = heights[blk]
        side_id = (u4[f] * 4).floor().clamp_(max=3)
        t = u1[f] * inner
        x0 = bx * road_every - side / 2 + road_width / 2
        y0 = by * road_every - side / 2 + road_width / 2
        fx = torch.where(side_id == 0, x0 + t, torch.where(side_id == 1, x0 + t, torch.where(side_id == 2, x0, x0 + inner)))
        fy = torch.where(side_id == 0, y0, torch.where(side_id == 1, y0 + inner, torch.where(side_id == 2, y0 + t, y0 + t)))
        fz = u2[f] * h
        if roof_frac > 0.0:
            # a draw of its own picks the roof share of the facade rows
            roof = t_uniform_at(seed, 50, i[f]) < roof_frac
            rx = x0 + u1[f] * inner
            ry = y0 + u2[f] * inner
            fx = torch.where(roof, rx, fx)
            fy = torch.where(roof, ry, fy)
            fz = torch.where(roof, h, fz)
        pos[f, 0] = fx
        pos[f, 1] = fy
        pos[f, 2] = fz
        if near is not None:
            c = torch.tensor(np.asarray(near[0], np.float64), device=device)
            sel = ((pos.to(torch.float32).to(torch.float64) - c) ** 2).sum(1) < float(near[1]) ** 2
            i, pos = i[sel], pos[sel]
            m = len(i)
            if m == 0:
                continue
        row = torch.empty((m, D), dtype=torch.float32, device=device)
        row[:, 0:3] = pos.to(torch.float32)
        row[:, 3:6] = (math.log(0.5 * spacing) + _cols_at(seed, 46, i, 3, t_normal_at, std=0.3)).to(torch.float32)
        q = _cols_at(seed, 47, i, 4, t_normal_at)
        row[:, 6:10] = (q / q.norm(dim=1, keepdim=True)).to(torch.float32)
        row[:, 10] = t_normal_at(seed, 48, i, 2.0, 0.5).to(torch.float32)
        rest = _cols_at(seed, 49, i, 48, t_normal_at, std=0.05).reshape(m, 16, 3)
        cell = ((pos[:, 0] + side / 2) // road_every).clamp(0, nb - 1).long() * nb + \
            ((pos[:, 1] + side / 2) // road_every).clamp(0, nb - 1).long()
        col = torch.stack([0.5 + 0.25 * torch.sin(pos[:, 0] / 23.0 + 0.4 * c) * torch.cos(pos[:, 1] / 31.0 - 0.6 * c)
                           + 0.1 * torch.sin(pos[:, 2] / 7.0 + c) for c in range(3)], 1) + tint[cell]
        rest[:, 0, :] = (col - 0.5) * 3.5
        row[:, 11:59] = rest.reshape(m, 48).to(torch.float32)
        if out_host is not None:
            out_host[a:a + m] = row.cpu().numpy()
        elif near is None:
            out[a:a + m] = row
        else:
            out.append(row)
            kept.append(i)
        del pos, rest, col, q, row
    if out_host is not None:
        return out_host, spacing
    if near is None:
        return out, spacing
    if not out:
        return torch.zeros((0, D), dtype=torch.float32, device=device), torch.zeros(0, dtype=torch.int64), spacing
    return torch.cat(out), torch.cat(kept), spacing


def street_drive_cameras(n_cams=500, seed=1003, side=4000.0, road_every=100.0, height=1.5, step=2.0,
                         width=1600, height_px=900, fov_x=90.0, znear=0.2, zfar=200.0, turn_every=400.0,
                         start=(3, 3), heading=(1.0, 0.0)):
    """A connected drive along the road centre lines: 2 m per frame at 1.5 m
    height, starting at intersection `start` (road indices) with `heading`,
    turning left or right at an intersection every `turn_every` metres (turn
    direction from the seeded stream), looking along the road."""
    u = uniform(seed, 60, n_cams + 8)
    pos = np.array([road_every * start[0] - side / 2, road_every * start[1] - side / 2])
    d = np.array(heading, np.float64)
    travelled = 0.0
    cams = []
    k = 0
    for i in range(n_cams):
        p3 = np.array([pos[0], pos[1], height])
        tgt = p3 + np.array([d[0], d[1], 0.0])
        R, t = look_at(p3, tgt, up=(0.0, 0.0, 1.0))
        cams.append(pinhole(width, height_px, fov_x, R, t, znear, zfar))
        pos = pos + step * d
        travelled += step
        if travelled >= turn_every:
            travelled = 0.0
            left = u[k] < 0.5
            k += 1
            d = np.array([-d[1], d[0]]) if left else np.array([d[1], -d[0]])
            nxt = pos + turn_every * d
            if np.any(np.abs(nxt) > side / 2 - road_every):
                d = -d
    return cams


def lawnmower_cameras(n_cams=1000, side=4000.0, altitude=150.0, pitch_deg=45.0, spacing=400.0, step=8.0,
                      width=1920, height_px=1080, fov_x=60.0, znear=0.5, zfar=600.0):
    """An aerial lawnmower path over the square: parallel passes `spacing`
    apart at `altitude`, `step` metres per frame, the camera looking ahead and
    down at `pitch_deg`; the passes alternate direction."""
    cams = []
    half = side / 2 - spacing / 2
    y = -half
    direction = 1.0
    x = -half
    t = math.tan(math.radians(pitch_deg))
    for _ in range(n_cams):
        p3 = np.array([x, y, altitude])
        tgt = p3 + np.array([direction, 0.0, -t])
        R, tv = look_at(p3, tgt, up=(0.0, 0.0, 1.0))
        cams.append(pinhole(width, height_px, fov_x, R, tv, znear, zfar))
        x += direction * step
        if abs(x) > half:
            x = direction * half
            direction = -direction
            y += spacing
            if y > half:
                y = -half
    return cams


def city_cameras(n_cams=2000, side=4000.0, seed=1004):
    """The mixed city trajectory: half aerial lawnmower frames at 1920x1080,
    half street-drive frames at 1920x1080 (two drives), in that order."""
    na = n_cams // 2
    aerial = lawnmower_cameras(na, side=side)
    nb = n_cams - na
    d1 = street_drive_cameras(nb // 2, seed=seed, side=side, width=1920, height_px=1080)
    d2 = street_drive_cameras(nb - nb // 2, seed=seed + 1, side=side, width=1920, height_px=1080, start=(25, 30),
                              heading=(0.0, -1.0))
    return aerial + d1 + d2


def t_perturb_(rows, seed, row0, mean_std=0.02, logscale_std=0.1, opacity_std=0.5, sh_std=0.05):
    """In-place torch version of perturb() on rows [row0, row0 + len(rows)) of a
    table (same streams and indices, so chunks compose to the whole table)."""
    m = rows.shape[0]
    dev = rows.device
    rows[:, 0:3] += t_normal(seed, 11, 3 * m, 0.0, mean_std, start=3 * row0, device=dev).reshape(m, 3).to(rows.dtype)
    rows[:, 3:6] += t_normal(seed, 12, 3 * m, 0.0, logscale_std, start=3 * row0, device=dev).reshape(m, 3).to(rows.dtype)
    rows[:, 10] += t_normal(seed, 13, m, 0.0, opacity_std, start=row0, device=dev).to(rows.dtype)
    rows[:, 11:59] += t_normal(seed, 14, 48 * m, 0.0, sh_std, start=48 * row0, device=dev).reshape(m, 48).to(rows.dtype)
    return rows
