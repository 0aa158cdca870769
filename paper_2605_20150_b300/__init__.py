"""Python binding of the sm_103a TideGS library (include/tidegs.h).

Argument marshalling only: every step of the training path runs in the CUDA
kernels of libtidegs.so.  The functions below keep the C names (tgs_*); torch
tensors are passed as raw device pointers plus the current CUDA stream.
Loading fails loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtidegs.so")
D = 59
TILE = 16

TGS_OK = 0
STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "CAPACITY", 5: "TIMEOUT", 6: "STATE"}


class TgsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tgs error {STATUS.get(code, code)}: {msg}")
        self.code = code


class tgs_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("znear", ctypes.c_float),
                ("zfar", ctypes.c_float), ("world_to_cam", ctypes.c_float * 12)]


class tgs_config(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_uint32), ("moments_policy", ctypes.c_uint32),
                ("prefetch_mode", ctypes.c_uint32), ("overlap", ctypes.c_uint32), ("cache_blocks", ctypes.c_uint64),
                ("spare_slots", ctypes.c_uint32), ("max_batch", ctypes.c_uint32), ("max_width", ctypes.c_uint32),
                ("max_height", ctypes.c_uint32), ("quota", ctypes.c_uint32), ("lambda_", ctypes.c_float),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("cull_margin_px", ctypes.c_float), ("bg", ctypes.c_float * 3), ("loss", ctypes.c_uint32),
                ("host_bf16", ctypes.c_uint32), ("stochastic_round", ctypes.c_uint32), ("seed", ctypes.c_uint32),
                ("pair_capacity", ctypes.c_uint64), ("max_render_blocks", ctypes.c_uint64),
                ("lr_schedule", ctypes.c_uint32), ("lr_groups", ctypes.c_float * 6), ("lr_means_final", ctypes.c_float),
                ("lr_decay_steps", ctypes.c_uint32), ("differential", ctypes.c_uint32), ("morton", ctypes.c_uint32),
                ("host_cache_blocks", ctypes.c_uint64), ("backing_path", ctypes.c_char_p)]


class tgs_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("bytes_h2d", ctypes.c_uint64), ("bytes_d2h", ctypes.c_uint64),
                ("blocks_in", ctypes.c_uint64), ("blocks_out", ctypes.c_uint64), ("writebacks", ctypes.c_uint64),
                ("readmissions", ctypes.c_uint64), ("cold_restarts", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("stall_ms", ctypes.c_double), ("h2d_ms", ctypes.c_double),
                ("d2h_ms", ctypes.c_double), ("demand_blocks", ctypes.c_uint64), ("demand_hits", ctypes.c_uint64),
                ("predicted_blocks", ctypes.c_uint64), ("last_pairs", ctypes.c_uint64),
                ("last_visible", ctypes.c_uint64), ("last_render_blocks", ctypes.c_uint64),
                ("pair_overflows", ctypes.c_uint64), ("dropped_steps", ctypes.c_uint64),
                ("host_step_ms", ctypes.c_double), ("host_wait_ms", ctypes.c_double),
                ("resident_block_steps", ctypes.c_uint64), ("block_updates", ctypes.c_uint64),
                ("cold_updates", ctypes.c_uint64), ("streaks", ctypes.c_uint64), ("streak_steps", ctypes.c_uint64),
                ("host_cache_hits", ctypes.c_uint64), ("host_cache_misses", ctypes.c_uint64),
                ("log_bytes_read", ctypes.c_uint64), ("log_bytes_written", ctypes.c_uint64)]


_VP = ctypes.c_void_p
_U32, _U64, _F = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float
_SIGS = {
    "tgs_last_error": (ctypes.c_char_p, []),
    "tgs_default_config": (None, [ctypes.POINTER(tgs_config)]),
    "tgs_create": (ctypes.c_int32, [ctypes.POINTER(tgs_config), _U64, _VP, ctypes.POINTER(_VP)]),
    "tgs_destroy": (None, [_VP]),
    "tgs_step": (ctypes.c_int32, [_VP, ctypes.POINTER(tgs_camera), _U32, ctypes.POINTER(tgs_camera), _U32, _VP, _VP,
                                  _VP, ctypes.POINTER(_F)]),
    "tgs_render": (ctypes.c_int32, [_VP, ctypes.POINTER(tgs_camera), _VP, _VP]),
    "tgs_sync": (ctypes.c_int32, [_VP]),
    "tgs_losses": (ctypes.c_int32, [_VP, _VP, ctypes.c_uint64, _VP]),
    "tgs_checkpoint": (ctypes.c_int32, [_VP, ctypes.c_char_p]),
    "tgs_set_schedule": (ctypes.c_int32, [_VP, _VP, ctypes.c_uint64, ctypes.c_uint32]),
    "tgs_resume": (ctypes.c_int32, [ctypes.POINTER(tgs_config), ctypes.c_char_p, ctypes.POINTER(_VP)]),
    "tgs_set_prefetch_mode": (ctypes.c_int32, [_VP, _U32]),
    "tgs_get_params": (ctypes.c_int32, [_VP, _VP]),
    "tgs_set_params": (ctypes.c_int32, [_VP, _VP]),
    "tgs_get_state": (ctypes.c_int32, [_VP, _VP, _VP, _VP, _VP]),
    "tgs_get_state_rows": (ctypes.c_int32, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "tgs_get_block_order": (ctypes.c_int32, [_VP, _VP]),
    "tgs_get_spheres": (ctypes.c_int32, [_VP, _VP]),
    "tgs_get_sizes": (ctypes.c_int32, [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    "tgs_get_sets": (ctypes.c_int32, [_VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_U64), _VP, ctypes.POINTER(_U64)]),
    "tgs_get_camera_record": (ctypes.c_int32, [_VP, _U32, ctypes.POINTER(_U64), ctypes.POINTER(_U64), _VP, _VP, _VP,
                                               _VP, _VP, _VP, _VP, _VP, _VP]),
    "tgs_get_stats": (ctypes.c_int32, [_VP, ctypes.POINTER(tgs_stats)]),
    "tgs_set_stage_timing": (ctypes.c_int32, [_VP, ctypes.c_int]),
    "tgs_get_stage_ms": (ctypes.c_int32, [_VP, _VP, _VP, ctypes.c_int]),
    "tgs_visible_blocks": (ctypes.c_int32, [_VP, ctypes.POINTER(tgs_camera), _U32, _VP]),
    "tgs_mlp_create": (ctypes.c_int32, [_U64, _U32, ctypes.POINTER(_VP)]),
    "tgs_mlp_destroy": (None, [_VP]),
    "tgs_mlp_num_params": (_U64, []),
    "tgs_mlp_get_params": (ctypes.c_int32, [_VP, _VP]),
    "tgs_mlp_set_params": (ctypes.c_int32, [_VP, _VP]),
    "tgs_mlp_forward": (ctypes.c_int32, [_VP, _VP, _U64, ctypes.POINTER(tgs_camera), _VP, _VP]),
    "tgs_mlp_train_step": (ctypes.c_int32, [_VP, _VP, _U64, ctypes.POINTER(tgs_camera), _VP, _F, _F, _F, ctypes.c_int,
                                            ctypes.POINTER(_F), _VP, _VP]),
    "tgs_set_predictor": (ctypes.c_int32, [_VP, _VP, _F, _U32]),
    "tgs_raster_create": (ctypes.c_int32, [_U64, _U32, _U32, ctypes.POINTER(_VP)]),
    "tgs_raster_destroy": (None, [_VP]),
    "tgs_raster_forward": (ctypes.c_int32, [_VP, _VP, _U64, _U32, ctypes.POINTER(tgs_camera), _VP, _VP, _VP]),
    "tgs_raster_backward": (ctypes.c_int32, [_VP, _VP, _U64, _U32, ctypes.POINTER(tgs_camera), _VP, _VP, _VP, _VP,
                                             _VP]),
    "tgs_raster_forward_noalloc": (ctypes.c_int32, [_VP, _U64, _U32, ctypes.POINTER(tgs_camera), _VP, _VP, _VP]),
    "tgs_adam": (ctypes.c_int32, [_VP, _VP, _VP, _VP, _VP, _VP, _U64, _U32, _F, _F, _F, _F, _VP]),
}

_lib = None


def load():
    """Loads libtidegs.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        from . import build as _build
        if not os.path.exists(LIB_PATH) or _build.stale():
            _build.build()
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(code):
    if code != TGS_OK:
        raise TgsError(code, load().tgs_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())  # torch tensor


def _stream(torch_stream=None):
    import torch
    s = torch_stream if torch_stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_camera(cam) -> tgs_camera:
    """ABI camera from a dict with width, height, fx, fy, cx, cy, znear, zfar, R, t."""
    c = tgs_camera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    c.znear, c.zfar = cam["znear"], cam["zfar"]
    M = np.concatenate([np.asarray(cam["R"], np.float64), np.asarray(cam["t"], np.float64).reshape(3, 1)], 1)
    for i, v in enumerate(M.reshape(12)):
        c.world_to_cam[i] = float(v)
    return c


def camera_array(cams):
    arr = (tgs_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = c if isinstance(c, tgs_camera) else make_camera(c)
    return arr


def default_config(**kw) -> tgs_config:
    c = tgs_config()
    load().tgs_default_config(ctypes.byref(c))
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                c.bg[i] = v[i]
        elif k == "lr_groups":
            for i in range(6):
                c.lr_groups[i] = v[i]
        elif k == "lam":
            c.lambda_ = v
        elif k == "backing_path":
            c.backing_path = None if v is None else os.fsencode(v)
        else:
            setattr(c, k, v)
    return c


class TideTable:
    """A block-virtualised table of N Gaussians (tgs_create ... tgs_destroy)."""

    def __init__(self, params: np.ndarray, _resume=None, **cfg):
        self.cfg = default_config(**cfg)
        h = ctypes.c_void_p()
        if _resume is not None:
            _check(load().tgs_resume(ctypes.byref(self.cfg), str(_resume).encode(), ctypes.byref(h)))
        else:
            params = np.ascontiguousarray(params, np.float32)
            assert params.ndim == 2 and params.shape[1] == D
            _check(load().tgs_create(ctypes.byref(self.cfg), params.shape[0], _ptr(params), ctypes.byref(h)))
        self.h = h
        n, k, s = _U64(), _U64(), _U64()
        _check(load().tgs_get_sizes(self.h, ctypes.byref(n), ctypes.byref(k), ctypes.byref(s)))
        self.n, self.K, self.slots = n.value, k.value, s.value

    @classmethod
    def resume(cls, path, **cfg):
        """A table from a checkpoint file (tgs_resume)."""
        return cls(None, _resume=path, **cfg)

    def checkpoint(self, path):
        """Writes the training state to a file (tgs_checkpoint)."""
        _check(load().tgs_checkpoint(self.h, str(path).encode()))

    def close(self):
        if getattr(self, "h", None):
            load().tgs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, cams, targets, next_cams=None, want_loss=True, stream=None):
        """targets: torch CUDA tensor (J, H, W, 3) or numpy host array."""
        ca = camera_array(cams)
        na = camera_array(next_cams) if next_cams else None
        loss = _F()
        if isinstance(targets, np.ndarray):
            t_dev, t_host = None, _ptr(np.ascontiguousarray(targets, np.float32))
            st = None
        else:
            t_dev, t_host = _ptr(targets), None
            st = _stream(stream)
        _check(load().tgs_step(self.h, ca, len(cams), na, len(next_cams) if next_cams else 0, t_dev, t_host, st,
                               ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def render(self, cam, image, stream=None):
        _check(load().tgs_render(self.h, ctypes.byref(make_camera(cam)), _ptr(image), _stream(stream)))

    def sync(self):
        _check(load().tgs_sync(self.h))

    def losses(self, max_count=4096):
        """Per-step losses since the previous call (tgs_losses)."""
        out = np.zeros(max_count, np.float32)
        n = _U64()
        _check(load().tgs_losses(self.h, _ptr(out), max_count, ctypes.byref(n)))
        return out[:n.value].copy()

    def set_schedule(self, cams, horizon=2):
        """Known trajectory for the exact lookahead prefetch (mode 3)."""
        ca = camera_array(cams)
        _check(load().tgs_set_schedule(self.h, ca, len(cams), horizon))

    def set_prefetch_mode(self, mode):
        _check(load().tgs_set_prefetch_mode(self.h, mode))

    def set_params(self, params):
        """params: host numpy [n, 59] (original row order) or a CUDA tensor (copied to host)."""
        if not isinstance(params, np.ndarray):
            params = params.detach().cpu().numpy()
        _check(load().tgs_set_params(self.h, _ptr(np.ascontiguousarray(params, np.float32))))

    def params(self):
        out = np.zeros((self.n, D), np.float32)
        _check(load().tgs_get_params(self.h, _ptr(out)))
        return out

    def state(self):
        p, m, v = (np.zeros((self.n, D), np.float32) for _ in range(3))
        st = np.zeros(self.K, np.uint32)
        _check(load().tgs_get_state(self.h, _ptr(p), _ptr(m), _ptr(v), _ptr(st)))
        return p, m, v, st

    def state_rows(self, ids):
        """(params, m1, m2) rows of the given block-order ids (tgs_get_state_rows)."""
        ids = np.ascontiguousarray(ids, np.int64)
        p, m, v = (np.zeros((len(ids), D), np.float32) for _ in range(3))
        _check(load().tgs_get_state_rows(self.h, _ptr(ids), len(ids), _ptr(p), _ptr(m), _ptr(v)))
        return p, m, v

    def block_order(self):
        out = np.zeros(self.n, np.int64)
        _check(load().tgs_get_block_order(self.h, _ptr(out)))
        return out

    def spheres(self):
        out = np.zeros((self.K, 4), np.float32)
        _check(load().tgs_get_spheres(self.h, _ptr(out)))
        return out

    def sets(self, batch):
        kv = np.zeros(self.K, np.uint8)
        rr = np.zeros(self.K, np.uint8)
        kp = np.zeros((batch, self.K), np.uint8)
        sp = np.zeros(self.K, np.int64)
        sm = np.zeros(self.K, np.int64)
        npl, nmi = _U64(), _U64()
        _check(load().tgs_get_sets(self.h, _ptr(kv), _ptr(rr), _ptr(kp), _ptr(sp), ctypes.byref(npl), _ptr(sm),
                                   ctypes.byref(nmi)))
        return dict(k_visible=kv, r_resident=rr, k_per_camera=kp, s_plus=sp[:npl.value].copy(),
                    s_minus=sm[:nmi.value].copy())

    def camera_record(self, j, W, H):
        ng, npairs = _U64(), _U64()
        lib = load()
        _check(lib.tgs_get_camera_record(self.h, j, ctypes.byref(ng), ctypes.byref(npairs), *([None] * 9)))
        n, m = ng.value, npairs.value
        TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
        r = dict(ids=np.zeros(n, np.int64), splat=np.zeros((n, 12), np.float32), rect=np.zeros((n, 4), np.int32),
                 pair_vals=np.zeros(max(m, 1), np.uint32), ranges=np.zeros((TX * TY, 2), np.uint32),
                 image=np.zeros((H, W, 3), np.float32), t_final=np.zeros((H, W), np.float32),
                 n_last=np.zeros((H, W), np.int32), grad2d=np.zeros((n, 9), np.float32))
        _check(lib.tgs_get_camera_record(self.h, j, ctypes.byref(ng), ctypes.byref(npairs), _ptr(r["ids"]),
                                         _ptr(r["splat"]), _ptr(r["rect"]), _ptr(r["pair_vals"]), _ptr(r["ranges"]),
                                         _ptr(r["image"]), _ptr(r["t_final"]), _ptr(r["n_last"]),
                                         _ptr(r["grad2d"])))
        r["pair_vals"] = r["pair_vals"][:m]
        return r

    STAGES = ("preprocess", "sort", "raster_fwd", "loss", "raster_bwd", "preprocess_bwd", "adam", "bounds")

    def stage_timing(self, on=True):
        _check(load().tgs_set_stage_timing(self.h, int(on)))

    def stage_ms(self, reset=False):
        ms = np.zeros(8, np.float64)
        cnt = np.zeros(8, np.uint64)
        _check(load().tgs_get_stage_ms(self.h, _ptr(ms), _ptr(cnt), int(reset)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.STAGES)}

    def visible_blocks(self, cams):
        out = np.zeros((len(cams), self.K), np.uint8)
        _check(load().tgs_visible_blocks(self.h, camera_array(cams), len(cams), _ptr(out)))
        return out

    def set_predictor(self, mlp, threshold=0.5, horizon_mask=1):
        _check(load().tgs_set_predictor(self.h, mlp.h if mlp is not None else None, threshold, horizon_mask))
        self._predictor = mlp  # keep alive

    def stats(self):
        s = tgs_stats()
        _check(load().tgs_get_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}


class Predictor:
    """Learned block-prefetch MLP (tgs_mlp_*)."""

    def __init__(self, max_blocks, seed=0):
        h = ctypes.c_void_p()
        _check(load().tgs_mlp_create(max_blocks, seed, ctypes.byref(h)))
        self.h = h
        self.n_params = load().tgs_mlp_num_params()

    def close(self):
        if getattr(self, "h", None):
            load().tgs_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        _check(load().tgs_mlp_get_params(self.h, _ptr(out)))
        return out

    def set_params(self, flat):
        _check(load().tgs_mlp_set_params(self.h, _ptr(np.ascontiguousarray(flat, np.float32))))

    def forward(self, spheres_dev, hist, logits_dev):
        _check(load().tgs_mlp_forward(self.h, _ptr(spheres_dev), spheres_dev.shape[0], camera_array(hist),
                                      _ptr(logits_dev), _stream()))

    def train_step(self, spheres_dev, hist, labels_dev, pos_weight, lr=1e-3, wd=1e-4, apply=True, want_grads=False):
        loss = _F()
        g = np.zeros(self.n_params, np.float32) if want_grads else None
        _check(load().tgs_mlp_train_step(self.h, _ptr(spheres_dev), spheres_dev.shape[0], camera_array(hist),
                                         _ptr(labels_dev), pos_weight, lr, wd, int(apply), ctypes.byref(loss),
                                         _ptr(g), _stream()))
        return (loss.value, g) if want_grads else loss.value


# ---------------------------------------------------------------------------
# resident rasteriser (autograd form)
# ---------------------------------------------------------------------------
def to_block_layout(params_rows, block_size):
    """[n, 59] rows -> [ceil(n/B), 59, B] block layout (zero-padded)."""
    import torch
    n = params_rows.shape[0]
    K = (n + block_size - 1) // block_size
    pad = K * block_size - n
    x = params_rows
    if pad:
        x = torch.cat([x, x.new_zeros(pad, D)], 0)
    return x.reshape(K, block_size, D).transpose(1, 2).contiguous()


def from_block_layout(blocks, n):
    K, _, B = blocks.shape
    return blocks.transpose(1, 2).reshape(K * B, D)[:n]


class Rasterizer:
    """Owns a tgs_raster context (per-camera state kept between forward and backward)."""

    def __init__(self, max_gaussians, max_width, max_height):
        h = ctypes.c_void_p()
        _check(load().tgs_raster_create(max_gaussians, max_width, max_height, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().tgs_raster_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, blocks, n, cam, bg, image):
        bgc = (ctypes.c_float * 3)(*bg)
        _check(load().tgs_raster_forward(self.h, _ptr(blocks), n, blocks.shape[2], ctypes.byref(make_camera(cam)),
                                         bgc, _ptr(image), _stream()))

    def backward(self, blocks, n, cam, bg, dl_dimage, grad, touched=None):
        bgc = (ctypes.c_float * 3)(*bg)
        _check(load().tgs_raster_backward(self.h, _ptr(blocks), n, blocks.shape[2], ctypes.byref(make_camera(cam)),
                                          bgc, _ptr(dl_dimage), _ptr(grad), _ptr(touched), _stream()))


def _autograd_fn():
    import torch

    class GaussianRasterize(torch.autograd.Function):
        """image = render(blocks) with the hand-written backward (reverse
        transmittance recomputation).  blocks: [K, 59, B] float32 CUDA."""

        @staticmethod
        def forward(ctx, blocks, n, cam, bg, rasterizer):
            H, W = int(cam["height"]), int(cam["width"])
            img = torch.empty(H, W, 3, device=blocks.device, dtype=torch.float32)
            rasterizer.forward(blocks, n, cam, bg, img)
            ctx.save_for_backward(blocks)
            ctx.n, ctx.cam, ctx.bg, ctx.r = n, cam, bg, rasterizer
            return img

        @staticmethod
        def backward(ctx, grad_img):
            (blocks,) = ctx.saved_tensors
            g = torch.zeros_like(blocks)
            ctx.r.backward(blocks, ctx.n, ctx.cam, ctx.bg, grad_img.contiguous(), g)
            return g, None, None, None, None

    return GaussianRasterize


_GR = None


def rasterize(blocks, n, cam, bg, rasterizer):
    global _GR
    if _GR is None:
        _GR = _autograd_fn()
    return _GR.apply(blocks, n, cam, tuple(bg), rasterizer)


def raster_forward_noalloc(blocks, n, cam, bg, image):
    """tgs_raster_forward_noalloc: the forward render without any device
    allocation (fixed 16 MiB static scratch; see include/tidegs.h for limits)."""
    bgc = (ctypes.c_float * 3)(*bg)
    _check(load().tgs_raster_forward_noalloc(_ptr(blocks), n, blocks.shape[2], ctypes.byref(make_camera(cam)), bgc,
                                             _ptr(image), _stream()))


def adam(blocks, grad, m1, m2, touched, steps, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-15):
    _check(load().tgs_adam(_ptr(blocks), _ptr(grad), _ptr(m1), _ptr(m2), _ptr(touched), _ptr(steps), n,
                           blocks.shape[2], lr, b1, b2, eps, _stream()))
