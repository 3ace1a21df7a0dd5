"""ctypes binding of libmvgs (include/mvgs.h) with the same call names.

Argument marshalling only: torch tensors are passed as raw device pointers
and the current CUDA stream; every step of the computation runs in the
library's kernels.  Importing this module raises if the library has not been
built -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

OK, EINVAL, ENOSPACE, EOVERFLOW, ECUDA, EDEVICE = 0, 1, 2, 3, 4, 5
GRAD_STRIDE = 12


class MemoryBudgetError(RuntimeError):
    """A batch needs more device memory than the rasterizer may hold."""

    def __init__(self, need_bytes, budget_bytes):
        super().__init__(f"batch needs {need_bytes} bytes of state + workspace, budget {budget_bytes}")
        self.need_bytes, self.budget_bytes = need_bytes, budget_bytes


class MvgsError(RuntimeError):
    def __init__(self, status, msg, needed=None):
        super().__init__(f"mvgs status {status}: {msg}")
        self.status = status
        self.needed = needed


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("viewmat", ctypes.c_float * 12), ("campos", ctypes.c_float * 3), ("near_z", ctypes.c_float)]


class Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class Config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("bg", ctypes.c_float * 3),
                ("flags", ctypes.c_uint32), ("pixels_per_thread", ctypes.c_int32), ("smem_batch", ctypes.c_int32)]


class Samples(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_void_p), ("pixels", ctypes.c_void_p)]


class Sampling(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int32), ("cell_w", ctypes.c_int32), ("cell_h", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


FLAG_MASKED_PARTIAL = 1
FLAG_DEPTH = 2
FLAG_CAPTURABLE = 4
FLAG_PIXEL_STATS = 8


class DensifyParams(ctypes.Structure):
    _fields_ = [("split_threshold", ctypes.c_double), ("clone_threshold", ctypes.c_double),
                ("prune_logit", ctypes.c_double), ("log_dense_extent", ctypes.c_double)]


class Capacity(ctypes.Structure):
    _fields_ = [("records", ctypes.c_int64), ("keys", ctypes.c_int64)]


_LAYOUT_FIELDS = ["state_bytes", "workspace_bytes", "off_counts", "off_rec_offsets", "off_rec_gauss", "off_rec_view",
                  "off_rec_xy", "off_rec_conic_opacity", "off_rec_rgb", "off_rec_clamp", "off_rec_depth",
                  "off_rec_rect", "off_sorted_records", "off_tile_ranges", "off_tile_order", "off_final_T",
                  "off_n_contrib", "off_pixel_stats", "off_pixel_depth"]


class Layout(ctypes.Structure):
    _fields_ = [(f, ctypes.c_size_t) for f in _LAYOUT_FIELDS] + [("tiles", ctypes.c_int64),
                                                                 ("pixels", ctypes.c_int64)]


# every symbol declared in include/mvgs.h
EXPORTS = ["mvgs_render_layout", "mvgs_render_views", "mvgs_render_views_backward", "mvgs_dssim_workspace_size",
           "mvgs_dssim_loss", "mvgs_adc_accumulate", "mvgs_profile_enable", "mvgs_profile_read", "mvgs_stage_name",
           "mvgs_launch_count", "mvgs_dssim_loss_noalloc", "mvgs_last_error",
           "mvgs_partial_samples_workspace_size", "mvgs_partial_samples", "mvgs_render_views_sampled",
           "mvgs_render_views_sampled_backward", "mvgs_merge_workspace_size", "mvgs_merge_views",
           "mvgs_split_merged_grad", "mvgs_dssim3d_workspace_size", "mvgs_dssim3d_loss",
           "mvgs_densify_workspace_size", "mvgs_densify", "mvgs_densify_carry", "mvgs_adam_step",
           "mvgs_count_workspace_size", "mvgs_count_views"]


def load_library(path: str | None = None):
    path = path or _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libmvgs is not built ({path}); run paper_2506_12727_gb300.build.build() -- "
                          "there is no CPU fallback")
    lib = ctypes.CDLL(path)
    P, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.mvgs_render_layout.argtypes = [I64, P, I32, P, P, P]
    lib.mvgs_render_views.argtypes = [P, P, I32, P, P, P, P, SZ, P, SZ, P, P]
    lib.mvgs_render_views_backward.argtypes = [P, P, I32, P, P, P, P, SZ, P, SZ, P, P, P, P, P, P, P, P]
    lib.mvgs_render_views_sampled.argtypes = [P, P, I32, P, P, P, P, P, SZ, P, SZ, P, P]
    lib.mvgs_render_views_sampled_backward.argtypes = [P, P, I32, P, P, P, P, P, SZ, P, SZ, P, P, P, P, P, P, P,
                                                       P]
    lib.mvgs_partial_samples_workspace_size.argtypes = [P, I32, P]
    lib.mvgs_partial_samples_workspace_size.restype = SZ
    lib.mvgs_partial_samples.argtypes = [P, I32, P, P, P, P, P, SZ, P]
    lib.mvgs_merge_workspace_size.argtypes = [I32]
    lib.mvgs_merge_workspace_size.restype = SZ
    lib.mvgs_merge_views.argtypes = [P, I32, P, ctypes.c_float, P, P, P, P, P, P, P, P, P, SZ, P]
    lib.mvgs_split_merged_grad.argtypes = [P, I32, P, P, P, P, SZ, P]
    lib.mvgs_dssim3d_workspace_size.argtypes = [P, I32]
    lib.mvgs_dssim3d_workspace_size.restype = SZ
    lib.mvgs_dssim3d_loss.argtypes = [P, P, P, P, P, I32, ctypes.c_float, P, P, P, SZ, P]
    lib.mvgs_count_workspace_size.argtypes = [I64, I32]
    lib.mvgs_count_workspace_size.restype = SZ
    lib.mvgs_count_views.argtypes = [P, P, I32, P, P, P, SZ, P]
    lib.mvgs_count_views.restype = ctypes.c_int
    lib.mvgs_densify_workspace_size.argtypes = [I64]
    lib.mvgs_densify_workspace_size.restype = SZ
    lib.mvgs_densify.argtypes = [P, P, P, P, P, P, I64, P, P, P, P, P, P, P, P, P, SZ, P]
    lib.mvgs_densify_carry.argtypes = [I64, P, P, I32, P, P, P]
    lib.mvgs_adam_step.argtypes = [I64, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   I32, P]
    lib.mvgs_dssim_workspace_size.argtypes = [P, I32]
    lib.mvgs_dssim_workspace_size.restype = SZ
    lib.mvgs_dssim_loss.argtypes = [P, P, P, I32, ctypes.c_float, P, P, P, SZ, P]
    lib.mvgs_adc_accumulate.argtypes = [P, I64, P, P, P, P, P, P]
    lib.mvgs_dssim_loss_noalloc.argtypes = [P, P, P, I32, ctypes.c_float, P, P, P]
    lib.mvgs_dssim_loss_noalloc.restype = ctypes.c_int
    lib.mvgs_last_error.restype = ctypes.c_char_p
    lib.mvgs_profile_enable.argtypes = [I32]
    lib.mvgs_profile_enable.restype = ctypes.c_int
    lib.mvgs_profile_read.argtypes = [P, P, I32]
    lib.mvgs_profile_read.restype = I32
    lib.mvgs_stage_name.argtypes = [I32]
    lib.mvgs_stage_name.restype = ctypes.c_char_p
    lib.mvgs_launch_count.argtypes = []
    lib.mvgs_launch_count.restype = I64
    for f in ("mvgs_render_layout", "mvgs_render_views", "mvgs_render_views_backward", "mvgs_dssim_loss",
              "mvgs_adc_accumulate", "mvgs_render_views_sampled", "mvgs_render_views_sampled_backward",
              "mvgs_partial_samples", "mvgs_merge_views", "mvgs_split_merged_grad", "mvgs_dssim3d_loss",
              "mvgs_densify", "mvgs_densify_carry", "mvgs_adam_step"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


_lib = load_library()


def last_error() -> str:
    return _lib.mvgs_last_error().decode()


def _check(status, needed=None):
    if status != OK:
        raise MvgsError(status, last_error(), needed)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "tensors passed to libmvgs must be contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_cameras(cams) -> ctypes.Array:
    """Packs a synth.Cameras (numpy arrays) into an array of mvgs_camera."""
    V = cams.V
    arr = (Camera * V)()
    for v in range(V):
        c = arr[v]
        c.width, c.height = int(cams.width[v]), int(cams.height[v])
        c.fx, c.fy, c.cx, c.cy = float(cams.fx[v]), float(cams.fy[v]), float(cams.cx[v]), float(cams.cy[v])
        c.viewmat[:] = [float(x) for x in np.asarray(cams.viewmat[v], np.float32).reshape(12)]
        c.campos[:] = [float(x) for x in cams.campos[v]]
        c.near_z = float(cams.near[v])
    return arr


def make_config(tile=(16, 16), bg=(0.0, 0.0, 0.0), pixels_per_thread=0, smem_batch=0) -> Config:
    cfg = Config()
    cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
    cfg.bg[:] = [float(b) for b in bg]
    cfg.flags = 0
    cfg.pixels_per_thread = int(pixels_per_thread)
    cfg.smem_batch = int(smem_batch)
    return cfg


def make_scene(params: dict, sh_degree: int) -> Scene:
    """`params`: dict of contiguous float32 CUDA tensors means, log_scales,
    quats, opacity_logits, sh."""
    sc = Scene()
    sc.n = int(params["means"].shape[0])
    sc.sh_degree = int(sh_degree)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        t = params[k]
        assert t.dtype == torch.float32
        setattr(sc, k, _ptr(t))
    return sc


# ---------------------------------------------------------------------------
# the C calls, one to one
# ---------------------------------------------------------------------------
def render_layout(n, cams_c, cfg, cap) -> Layout:
    L = Layout()
    _check(_lib.mvgs_render_layout(n, cams_c, len(cams_c), ctypes.byref(cfg), ctypes.byref(cap), ctypes.byref(L)))
    return L


def render_views(scene_c, cams_c, cfg, cap, images, state, workspace, stream=None):
    """Returns the needed Capacity; raises MvgsError (with .needed) on failure."""
    needed = Capacity()
    st = _lib.mvgs_render_views(ctypes.byref(scene_c), cams_c, len(cams_c), ctypes.byref(cfg), ctypes.byref(cap),
                                _ptr(images), _ptr(state), state.numel(), _ptr(workspace), workspace.numel(),
                                ctypes.byref(needed), _stream(stream))
    _check(st, needed)
    return needed


def render_views_backward(scene_c, cams_c, cfg, cap, dL_dimages, state, workspace, grads: dict, g_mean2d=None,
                          e1=None, stream=None):
    st = _lib.mvgs_render_views_backward(ctypes.byref(scene_c), cams_c, len(cams_c), ctypes.byref(cfg),
                                         ctypes.byref(cap), _ptr(dL_dimages), _ptr(state), state.numel(),
                                         _ptr(workspace), workspace.numel(), _ptr(grads["means"]),
                                         _ptr(grads["log_scales"]), _ptr(grads["quats"]),
                                         _ptr(grads["opacity_logits"]), _ptr(grads["sh"]), _ptr(g_mean2d), _ptr(e1),
                                         _stream(stream))
    _check(st)


class SampleSet:
    """Device arrays of a sample set (mvgs_samples): offsets int64 [tiles + 1]
    and pixel indices inside the tile (uint16 data held in an int16 tensor)."""

    def __init__(self, offsets: torch.Tensor, pixels: torch.Tensor):
        self.offsets, self.pixels = offsets, pixels
        self.c = Samples(_ptr(offsets), _ptr(pixels))

    def pixel_index(self) -> torch.Tensor:
        """The pixel indices as int64 (0 .. tile_w * tile_h - 1)."""
        n = int(self.offsets[-1])
        return self.pixels[:n].to(torch.int64) & 0xFFFF


def count_views(scene_c, cams_c, cfg, device="cuda", stream=None) -> Capacity:
    """mvgs_count_views: the exact records and keys a render of these views needs."""
    ws = torch.empty(int(_lib.mvgs_count_workspace_size(scene_c.n, len(cams_c))), dtype=torch.uint8, device=device)
    needed = Capacity()
    _check(_lib.mvgs_count_views(ctypes.byref(scene_c), cams_c, len(cams_c), ctypes.byref(cfg), ctypes.byref(needed),
                                 _ptr(ws), ws.numel(), _stream(stream)))
    return needed


def sampling(group: int, seed: int, cell=(1, 1)) -> Sampling:
    return Sampling(int(group), int(cell[0]), int(cell[1]), int(seed))


def partial_samples(cams_c, cfg, group: int, seed: int, device="cuda", stream=None, cell=(1, 1)) -> SampleSet:
    """mvgs_partial_samples: view v takes the cells whose hash slot is v mod group."""
    L = render_layout(0, cams_c, cfg, Capacity(0, 0))
    offsets = torch.empty(int(L.tiles) + 1, dtype=torch.int64, device=device)
    pixels = torch.empty(max(int(L.pixels), 1), dtype=torch.int16, device=device)
    nbytes = int(_lib.mvgs_partial_samples_workspace_size(cams_c, len(cams_c), ctypes.byref(cfg)))
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)
    sp = sampling(group, seed, cell)
    _check(_lib.mvgs_partial_samples(cams_c, len(cams_c), ctypes.byref(cfg), ctypes.byref(sp), _ptr(offsets),
                                     _ptr(pixels), _ptr(ws), ws.numel(), _stream(stream)))
    return SampleSet(offsets, pixels)


def render_views_sampled(scene_c, cams_c, cfg, cap, samples: SampleSet, images, state, workspace, stream=None):
    needed = Capacity()
    st = _lib.mvgs_render_views_sampled(ctypes.byref(scene_c), cams_c, len(cams_c), ctypes.byref(cfg),
                                        ctypes.byref(cap), ctypes.byref(samples.c), _ptr(images), _ptr(state),
                                        state.numel(), _ptr(workspace), workspace.numel(), ctypes.byref(needed),
                                        _stream(stream))
    _check(st, needed)
    return needed


def render_views_sampled_backward(scene_c, cams_c, cfg, cap, samples: SampleSet, dL_dimages, state, workspace,
                                  grads: dict, g_mean2d=None, e1=None, stream=None):
    st = _lib.mvgs_render_views_sampled_backward(ctypes.byref(scene_c), cams_c, len(cams_c), ctypes.byref(cfg),
                                                 ctypes.byref(cap), ctypes.byref(samples.c), _ptr(dL_dimages),
                                                 _ptr(state), state.numel(), _ptr(workspace), workspace.numel(),
                                                 _ptr(grads["means"]), _ptr(grads["log_scales"]),
                                                 _ptr(grads["quats"]), _ptr(grads["opacity_logits"]),
                                                 _ptr(grads["sh"]), _ptr(g_mean2d), _ptr(e1), _stream(stream))
    _check(st)


def merge_views(cams_c, group, seed, images=None, targets=None, depth_acc=None, final_T=None, merged_img=None,
                merged_tgt=None, points=None, sigma=None, sigma_px=1.5, stream=None, cell=(1, 1)):
    """mvgs_merge_views (outputs are caller tensors; None skips)."""
    ws = torch.empty(int(_lib.mvgs_merge_workspace_size(len(cams_c))), dtype=torch.uint8, device="cuda")
    sp = sampling(group, seed, cell)
    _check(_lib.mvgs_merge_views(cams_c, len(cams_c), ctypes.byref(sp), ctypes.c_float(sigma_px),
                                 _ptr(images), _ptr(targets), _ptr(depth_acc), _ptr(final_T), _ptr(merged_img),
                                 _ptr(merged_tgt), _ptr(points), _ptr(sigma), _ptr(ws), ws.numel(), _stream(stream)))


def split_merged_grad(cams_c, group, seed, dL_dmerged, dL_dimages, stream=None, cell=(1, 1)):
    ws = torch.empty(int(_lib.mvgs_merge_workspace_size(len(cams_c))), dtype=torch.uint8, device="cuda")
    sp = sampling(group, seed, cell)
    _check(_lib.mvgs_split_merged_grad(cams_c, len(cams_c), ctypes.byref(sp), _ptr(dL_dmerged),
                                       _ptr(dL_dimages), _ptr(ws), ws.numel(), _stream(stream)))


def dssim3d_workspace_size(hw: np.ndarray) -> int:
    hw = np.ascontiguousarray(hw, dtype=np.int32)
    return int(_lib.mvgs_dssim3d_workspace_size(hw.ctypes.data_as(ctypes.c_void_p), hw.shape[0]))


def dssim3d_loss(img, target, points, sigma, hw, lam, loss_per_image, dL_dimg, workspace, stream=None):
    hw = np.ascontiguousarray(hw, dtype=np.int32)
    _check(_lib.mvgs_dssim3d_loss(_ptr(img), _ptr(target), _ptr(points), _ptr(sigma),
                                  hw.ctypes.data_as(ctypes.c_void_p), hw.shape[0], ctypes.c_float(lam),
                                  _ptr(loss_per_image), _ptr(dL_dimg), _ptr(workspace), workspace.numel(),
                                  _stream(stream)))


def densify(params: dict, sh_degree: int, accum_e1, accum_e2, denom, normals, split_threshold, clone_threshold,
            prune_logit, log_dense_extent, carry=(), stream=None):
    """mvgs_densify (+ mvgs_densify_carry for each tensor in `carry`, e.g. Adam
    moments shaped like a parameter).  Returns (new params, src, kind, carried)."""
    n = int(params["means"].shape[0])
    sc = make_scene(params, sh_degree)
    prm = DensifyParams(float(split_threshold), float(clone_threshold), float(prune_logit), float(log_dense_extent))
    ws = torch.empty(max(int(_lib.mvgs_densify_workspace_size(n)), 1), dtype=torch.uint8, device="cuda")
    cap = 2 * n
    out = {k: torch.empty((cap,) + tuple(v.shape[1:]), dtype=torch.float32, device="cuda") for k, v in params.items()}
    src = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    kind = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    n_out = ctypes.c_int64(0)
    _check(_lib.mvgs_densify(ctypes.byref(sc), _ptr(accum_e1), _ptr(accum_e2), _ptr(denom), _ptr(normals),
                             ctypes.byref(prm), cap, _ptr(out["means"]), _ptr(out["log_scales"]), _ptr(out["quats"]),
                             _ptr(out["opacity_logits"]), _ptr(out["sh"]), _ptr(src), _ptr(kind),
                             ctypes.byref(n_out), _ptr(ws), ws.numel(), _stream(stream)))
    m = int(n_out.value)
    new = {k: v[:m].contiguous() for k, v in out.items()}
    carried = []
    for t in carry:
        width = int(t[0].numel()) if t.shape[0] else 1
        o = torch.empty((m,) + tuple(t.shape[1:]), dtype=torch.float32, device="cuda")
        _check(_lib.mvgs_densify_carry(m, _ptr(src), _ptr(kind), width, _ptr(t.contiguous()), _ptr(o),
                                       _stream(stream)))
        carried.append(o)
    return new, src[:m], kind[:m], carried


def adam_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """mvgs_adam_step on one parameter tensor (in place)."""
    _check(_lib.mvgs_adam_step(param.numel(), _ptr(param), _ptr(grad), _ptr(m), _ptr(v), ctypes.c_float(lr),
                               ctypes.c_float(beta1), ctypes.c_float(beta2), ctypes.c_float(eps), int(step),
                               _stream(stream)))


def dssim_workspace_size(hw: np.ndarray) -> int:
    hw = np.ascontiguousarray(hw, dtype=np.int32)
    return int(_lib.mvgs_dssim_workspace_size(hw.ctypes.data_as(ctypes.c_void_p), hw.shape[0]))


def dssim_loss(img, target, hw, lam, loss_per_view, dL_dimg, workspace, stream=None):
    hw = np.ascontiguousarray(hw, dtype=np.int32)
    st = _lib.mvgs_dssim_loss(_ptr(img), _ptr(target), hw.ctypes.data_as(ctypes.c_void_p), hw.shape[0],
                              ctypes.c_float(lam), _ptr(loss_per_view), _ptr(dL_dimg), _ptr(workspace),
                              workspace.numel(), _stream(stream))
    _check(st)


def dssim_loss_noalloc(img, target, hw, lam, loss_per_view, dL_dimg, stream=None):
    """mvgs_dssim_loss with the library's static scratch (no workspace)."""
    hw = np.ascontiguousarray(hw, dtype=np.int32)
    st = _lib.mvgs_dssim_loss_noalloc(_ptr(img), _ptr(target), hw.ctypes.data_as(ctypes.c_void_p), hw.shape[0],
                                      ctypes.c_float(lam), _ptr(loss_per_view), _ptr(dL_dimg), _stream(stream))
    _check(st)


def adc_accumulate(state, n, g_mean2d, e1, accum_e1, accum_e2, denom, stream=None):
    _check(_lib.mvgs_adc_accumulate(_ptr(state), n, _ptr(g_mean2d), _ptr(e1), _ptr(accum_e1), _ptr(accum_e2),
                                    _ptr(denom), _stream(stream)))


def launch_count() -> int:
    return int(_lib.mvgs_launch_count())


def profile_enable(on: bool):
    _check(_lib.mvgs_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """{stage name: (total ms, launches)} since the last read (waits for the events)."""
    n = 32
    ms = (ctypes.c_float * n)()
    cnt = (ctypes.c_int64 * n)()
    k = _lib.mvgs_profile_read(ms, cnt, n)
    return {_lib.mvgs_stage_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(k)}


# ---------------------------------------------------------------------------
# buffer management around the calls
# ---------------------------------------------------------------------------
class Rasterizer:
    """Keeps the caller-owned state and workspace buffers of one scene size
    and camera set, growing them (with headroom) when a batch needs more
    records or keys than the current capacity."""

    def __init__(self, cams, tile=(16, 16), bg=(0.0, 0.0, 0.0), device="cuda", headroom=1.15, pixels_per_thread=0,
                 max_bytes=None, capturable=False, smem_batch=0):
        self.max_bytes = max_bytes  # cap on state + workspace bytes (None: unlimited)
        # capturable: no count read-backs (CUDA-graph capture); call reserve()
        # first and check counts() after a step
        self.capturable = capturable
        self.cams_np = cams
        self.cams_c = make_cameras(cams)
        self.cfg = make_config(tile, bg, pixels_per_thread, smem_batch)
        self.device = device
        self.headroom = headroom
        self.cap = Capacity(0, 0)
        self.state = None
        self.workspace = None
        self.layout = None
        self.n = None
        self.pixels = int(sum(int(w) * int(h) for w, h in zip(cams.width, cams.height)))
        self.needed = Capacity(0, 0)
        # forwards run so far: a backward that needs one forward's state can
        # check that no later forward has overwritten it
        self.generation = 0

    def _ensure(self, n, records, keys):
        grow = self.state is None or n != self.n or records > self.cap.records or keys > self.cap.keys
        if not grow:
            return
        cap = Capacity(max(int(records * self.headroom) + 1024, self.cap.records if n == self.n else 0),
                       max(int(keys * self.headroom) + 4096, self.cap.keys if n == self.n else 0))
        L = render_layout(n, self.cams_c, self.cfg, cap)
        if self.max_bytes is not None and L.state_bytes + L.workspace_bytes > self.max_bytes:
            # try without headroom before giving up
            cap = Capacity(max(records, 1), max(keys, 1))
            L = render_layout(n, self.cams_c, self.cfg, cap)
            if L.state_bytes + L.workspace_bytes > self.max_bytes:
                raise MemoryBudgetError(L.state_bytes + L.workspace_bytes, self.max_bytes)
        self.state = None
        self.workspace = None
        self.state = torch.empty(L.state_bytes, dtype=torch.uint8, device=self.device)
        self.workspace = torch.empty(L.workspace_bytes, dtype=torch.uint8, device=self.device)
        self.cap, self.layout, self.n = cap, L, n

    def reserve(self, n, records, keys):
        self._ensure(n, records, keys)

    def reserve_for(self, scene_c, extra=1.0, stream=None) -> Capacity:
        """Sizes the buffers for this scene from the exact pre-count (times
        `extra` on top of the rasterizer's headroom, for parameters that will
        move, e.g. a captured training step); returns the counts."""
        need = count_views(scene_c, self.cams_c, self.cfg, self.device, stream)
        self.reserve(scene_c.n, int(need.records * extra), int(need.keys * extra))
        return need

    def held_bytes(self) -> int:
        return 0 if self.state is None else self.state.numel() + self.workspace.numel()

    def set_cameras(self, cams):
        """Re-targets the rasterizer to another camera batch, keeping its
        buffers when they are large enough for the current capacities."""
        self.cams_np = cams
        self.cams_c = make_cameras(cams)
        self.pixels = int(sum(int(w) * int(h) for w, h in zip(cams.width, cams.height)))
        if self.state is None:
            return
        L = render_layout(self.n, self.cams_c, self.cfg, self.cap)
        if L.state_bytes <= self.state.numel() and L.workspace_bytes <= self.workspace.numel():
            self.layout = L
        else:
            self.state = self.workspace = self.layout = None

    def _cfg(self, masked=False, depth=False, stats=False):
        if not masked and not depth and not stats and not self.capturable:
            return self.cfg
        cfg = Config.from_buffer_copy(self.cfg)
        cfg.flags = (FLAG_MASKED_PARTIAL if masked else 0) | (FLAG_DEPTH if depth else 0) | \
            (FLAG_CAPTURABLE if self.capturable else 0) | (FLAG_PIXEL_STATS if stats else 0)
        return cfg

    def sample_set(self, group: int, seed: int, stream=None, cell=(1, 1)) -> SampleSet:
        """Seeded partial-render samples for these cameras and this tile size
        (cell="strip": cells of one warp's strip)."""
        if cell == "strip":
            cell = self.strip_cell()
        return partial_samples(self.cams_c, self.cfg, group, seed, self.device, stream, cell)

    def strip_cell(self):
        """(columns, rows) of a warp's strip for this tile size and pixels per
        lane (strips are 8 columns wide)."""
        tw, th = self.cfg.tile_w, self.cfg.tile_h
        sw = min(tw, 8)
        ppt = self.cfg.pixels_per_thread
        if ppt == 0:
            ppt = next(p for p in (4, 2, 1) if th % ((32 // sw) * p) == 0)
        return (sw, (32 // sw) * ppt)

    def forward(self, scene_c, images=None, stream=None, samples: SampleSet | None = None, masked=False,
                depth=False, stats=False):
        """Full render, or with `samples` only the sampled pixels (Alg. 3; with
        masked=True through the full strips with idle lanes, Fig. 3b).  With
        depth=True the expected depth of each rendered pixel is written too
        (records()["depth_acc"]); with stats=True the per-pixel statistics
        (records()["pixel_stats"]: where the pixel stopped, Gaussians blended)."""
        n = scene_c.n
        if images is None:
            images = torch.empty(3 * self.pixels, dtype=torch.float32, device=self.device)
        self.generation += 1
        if self.capturable:
            # no read-backs, no growing: the caller reserved the capacity and
            # checks fits() after the step
            if self.state is None or n != self.n:
                raise MvgsError(EINVAL, "a capturable rasterizer needs reserve(n, records, keys) first")
            if samples is None:
                render_views(scene_c, self.cams_c, self._cfg(False, depth, stats), self.cap, images, self.state,
                             self.workspace, stream)
            else:
                render_views_sampled(scene_c, self.cams_c, self._cfg(masked, depth, stats), self.cap, samples,
                                     images, self.state, self.workspace, stream)
            self.needed = Capacity(self.cap.records, self.cap.keys)
            return images
        self._ensure(n, max(self.cap.records, 1), max(self.cap.keys, 1))
        for _ in range(4):
            try:
                if samples is None:
                    self.needed = render_views(scene_c, self.cams_c, self._cfg(False, depth, stats), self.cap,
                                               images, self.state, self.workspace, stream)
                else:
                    self.needed = render_views_sampled(scene_c, self.cams_c, self._cfg(masked, depth, stats),
                                                       self.cap, samples, images, self.state, self.workspace,
                                                       stream)
                return images
            except MvgsError as e:
                if e.status != ENOSPACE or e.needed is None:
                    raise
                self._ensure(n, max(e.needed.records, self.cap.records),
                             max(e.needed.keys, self.cap.keys))
        raise MvgsError(ENOSPACE, "could not size the buffers")

    def backward(self, scene_c, dL_dimages, grads, g_mean2d=None, e1=None, stream=None,
                 samples: SampleSet | None = None, masked=False):
        if samples is None:
            render_views_backward(scene_c, self.cams_c, self.cfg, self.cap, dL_dimages, self.state,
                                  self.workspace, grads, g_mean2d, e1, stream)
        else:
            render_views_sampled_backward(scene_c, self.cams_c, self._cfg(masked), self.cap, samples, dL_dimages,
                                          self.state, self.workspace, grads, g_mean2d, e1, stream)

    # views into the state (intermediate results)
    def _view(self, off, count, dtype, width=1):
        nbytes = count * width * torch.tensor([], dtype=dtype).element_size()
        t = self.state[off:off + nbytes].view(dtype)
        return t.view(count, width) if width > 1 else t

    def records(self) -> dict:
        L = self.layout
        R, K = int(self.needed.records), int(self.needed.keys)
        return dict(
            rec_off=self._view(L.off_rec_offsets, self.n + 1, torch.int64),
            g=self._view(L.off_rec_gauss, R, torch.int32), v=self._view(L.off_rec_view, R, torch.int32),
            xy=self._view(L.off_rec_xy, R, torch.float32, 2),
            conic_o=self._view(L.off_rec_conic_opacity, R, torch.float32, 4),
            rgb_r=self._view(L.off_rec_rgb, R, torch.float32, 4),
            clamp=self._view(L.off_rec_clamp, R, torch.int32),
            depth=self._view(L.off_rec_depth, R, torch.float32),
            rect=self._view(L.off_rec_rect, R, torch.int16, 4),
            sorted=self._view(L.off_sorted_records, K, torch.int32),
            ranges=self._view(L.off_tile_ranges, int(L.tiles), torch.int64, 2),
            tile_order=self._view(L.off_tile_order, int(L.tiles), torch.int32),
            final_T=self._view(L.off_final_T, int(L.pixels), torch.float32),
            n_contrib=self._view(L.off_n_contrib, int(L.pixels), torch.int32),
            pixel_stats=self._view(L.off_pixel_stats, int(L.pixels), torch.int32, 2),
            depth_acc=self._view(L.off_pixel_depth, int(L.pixels), torch.float32),
            counts=self._view(L.off_counts, 6, torch.int64))

    def counts(self) -> dict:
        """The counts block after the last forward (synchronises): records and
        keys held, and needed (larger after a capturable call ran out of room)."""
        c = self._view(self.layout.off_counts, 6, torch.int64).cpu().tolist()
        return dict(records=c[0], keys=c[1], tiles=c[2], pixels=c[3], records_needed=c[4], keys_needed=c[5])

    def fits(self) -> bool:
        c = self.counts()
        return c["records_needed"] <= self.cap.records and c["keys_needed"] <= self.cap.keys
