"""Python binding of libdarb.so (include/darb.h): argument marshalling only.

Every function here has the name of the C entry point it calls, takes torch CUDA tensors
(PyTorch provides device memory and the current stream) and performs no arithmetic of the
method itself.  If libdarb.so is missing the import of the library raises: there is no
CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np
import torch

from . import build as _build

c_f32 = ctypes.c_float
c_i32 = ctypes.c_int32
c_vp = ctypes.c_void_p

KERNEL_NAMES = ["gaussian", "half_cosine", "raised_cosine", "mod_sinc", "inv_quadric", "inv_multiquadric", "parabola"]
STATUS_NAMES = {0: "DARB_OK", 1: "DARB_ERR_INVALID_ARG", 2: "DARB_ERR_WORKSPACE", 3: "DARB_ERR_CAPACITY",
                4: "DARB_ERR_CUDA", 5: "DARB_ERR_TIMEOUT", 6: "DARB_ERR_ADMISSION", 7: "DARB_ERR_NOT_FOUND"}


class darb_kernel_params(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("psi", c_f32), ("q_max", c_f32), ("q_max_strict", c_i32), ("base", c_i32),
                ("xi", c_f32), ("beta", c_f32), ("lobes", c_i32)]


class darb_camera(ctypes.Structure):
    _fields_ = [("viewmat", c_f32 * 16), ("fx", c_f32), ("fy", c_f32), ("cx", c_f32), ("cy", c_f32),
                ("near_plane", c_f32), ("width", c_i32), ("height", c_i32), ("bg", c_f32 * 3)]


class darb_splats(ctypes.Structure):
    _fields_ = [("means", c_vp), ("scales", c_vp), ("quats", c_vp), ("opacities", c_vp), ("sh", c_vp),
                ("n", c_i32), ("sh_degree", c_i32)]


class darb_projected(ctypes.Structure):
    _fields_ = [("depth", c_vp), ("radius", c_vp), ("tile_rect", c_vp), ("mean2d", c_vp), ("conic_o", c_vp),
                ("rgb", c_vp), ("clamped", c_vp), ("tiles_touched", c_vp), ("tile_runs", c_vp)]


class darb_binning(ctypes.Structure):
    _fields_ = [("keys", c_vp), ("values", c_vp), ("ranges", c_vp), ("num_instances", c_vp), ("status", c_vp)]


class darb_image(ctypes.Structure):
    _fields_ = [("image", c_vp), ("t_final", c_vp), ("last", c_vp), ("n_contrib", c_vp)]


class darb_splat_grads(ctypes.Structure):
    _fields_ = [("dmeans", c_vp), ("dscales", c_vp), ("dquats", c_vp), ("dopacities", c_vp), ("dsh", c_vp)]


class darb_train_params(ctypes.Structure):
    _fields_ = [("means", c_vp), ("log_scales", c_vp), ("quats", c_vp), ("opacity_logits", c_vp), ("sh", c_vp),
                ("scales", c_vp), ("opacities", c_vp), ("n", c_i32), ("sh_degree", c_i32)]


class darb_adam_state(ctypes.Structure):
    _fields_ = [(f, c_vp) for f in ("m_means", "v_means", "m_scales", "v_scales", "m_quats", "v_quats",
                                    "m_opac", "v_opac", "m_sh", "v_sh")]


class darb_adam_config(ctypes.Structure):
    _fields_ = [("lr_means", c_f32), ("lr_scales", c_f32), ("lr_quats", c_f32), ("lr_opacities", c_f32),
                ("lr_sh_dc", c_f32), ("lr_sh_rest", c_f32), ("beta1", c_f32), ("beta2", c_f32), ("eps", c_f32),
                ("step", c_i32)]


class darb_batch_params(ctypes.Structure):
    _fields_ = [("n_views", c_i32), ("tile", c_i32), ("depth", c_i32), ("max_ctas", c_i32),
                ("capacity", ctypes.c_uint64)]


DARB_MAX_BATCH_VIEWS = 4096


class darb_densify_cfg(ctypes.Structure):
    _fields_ = [("grad_threshold", c_f32), ("dense_scale", c_f32), ("min_opacity", c_f32),
                ("max_screen_radius", c_f32), ("max_world_scale", c_f32), ("split_scale_div", c_f32)]


class darb_serve_cfg(ctypes.Structure):
    _fields_ = [("scene_bytes", ctypes.c_uint64), ("workspace_bytes", ctypes.c_uint64), ("tile", c_i32),
                ("max_batch", c_i32), ("depth", c_i32), ("capacity_per_pixel", c_f32),
                ("capacity_margin", c_f32), ("capacity_min", ctypes.c_uint64), ("slots", c_i32)]


class darb_request(ctypes.Structure):
    _fields_ = [("scene_id", c_i32), ("kernel", c_i32), ("cam", darb_camera), ("image", c_vp)]


class darb_result(ctypes.Structure):
    _fields_ = [("status", c_i32), ("num_instances", ctypes.c_uint32), ("attempts", ctypes.c_uint32),
                ("batch_size", ctypes.c_uint32), ("queue_us", ctypes.c_double), ("latency_us", ctypes.c_double),
                ("batch_id", ctypes.c_uint64), ("gpu_begin_us", ctypes.c_double), ("gpu_end_us", ctypes.c_double)]


# Every entry point declared in include/darb.h, with its ctypes signature.
_P = ctypes.POINTER
SIGNATURES = {
    "darb_status_string": (ctypes.c_char_p, [c_i32]),
    "darb_kernel_defaults": (c_i32, [c_i32, _P(darb_kernel_params)]),
    "darb_kernel_generic": (c_i32, [c_i32, c_f32, c_f32, c_i32, _P(darb_kernel_params)]),
    "darb_kernel_psi": (c_i32, [_P(darb_kernel_params), c_vp, _P(ctypes.c_double), c_vp]),
    "darb_tile_grid": (c_i32, [_P(darb_camera), c_i32, _P(c_i32), _P(c_i32)]),
    "darb_preprocess": (c_i32, [_P(darb_splats), _P(darb_camera), _P(darb_kernel_params), c_i32,
                                _P(darb_projected), c_vp]),
    "darb_bin_sort_workspace_size": (c_i32, [c_i32, c_i32, _P(darb_camera), ctypes.c_uint64, c_i32,
                                             _P(ctypes.c_size_t)]),
    "darb_bin_sort": (c_i32, [_P(darb_projected), c_i32, c_i32, _P(darb_camera), _P(darb_kernel_params), c_vp,
                              ctypes.c_size_t,
                              ctypes.c_uint64, c_i32, _P(darb_binning), _P(ctypes.c_uint64), c_vp]),
    "darb_bin_sort_noalloc": (c_i32, [_P(darb_projected), c_i32, c_i32, _P(darb_camera), _P(darb_kernel_params),
                                      ctypes.c_uint64,
                                      _P(darb_binning), _P(ctypes.c_uint64), c_vp]),
    "darb_render_fwd": (c_i32, [_P(darb_projected), _P(darb_binning), _P(darb_camera), _P(darb_kernel_params),
                                c_i32, _P(darb_image), c_vp]),
    "darb_render_fwd_l1": (c_i32, [_P(darb_projected), _P(darb_binning), _P(darb_camera), _P(darb_kernel_params),
                                   c_i32, _P(darb_image), c_vp, c_vp, c_vp, c_vp]),
    "darb_render_bwd": (c_i32, [_P(darb_projected), c_i32, _P(darb_binning), _P(darb_camera),
                                _P(darb_kernel_params), c_i32, _P(darb_image), c_vp, c_vp, c_vp]),
    "darb_preprocess_bwd": (c_i32, [_P(darb_splats), _P(darb_camera), _P(darb_kernel_params), _P(darb_projected),
                                    c_vp, _P(darb_splat_grads), c_vp]),
    "darb_l1_loss": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp]),
    "darb_l1_dssim_workspace_size": (c_i32, [c_i32, c_i32, _P(ctypes.c_size_t)]),
    "darb_l1_dssim_loss": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_f32, c_vp, ctypes.c_size_t, c_vp, c_vp, c_vp]),
    "darb_adam_step": (c_i32, [_P(darb_train_params), _P(darb_splat_grads), _P(darb_adam_state),
                               _P(darb_adam_config), c_vp]),
    "darb_preprocess_bwd_adam": (c_i32, [_P(darb_train_params), _P(darb_camera), _P(darb_kernel_params),
                                         _P(darb_projected), c_vp, _P(darb_adam_state), _P(darb_adam_config),
                                         c_vp]),
    "darb_render_batch_workspace_size": (c_i32, [c_i32, _P(darb_camera), _P(darb_batch_params),
                                                 _P(ctypes.c_size_t)]),
    "darb_render_batch": (c_i32, [_P(darb_splats), _P(darb_camera), _P(darb_kernel_params), _P(darb_batch_params),
                                  c_vp, ctypes.c_size_t, _P(darb_image), c_vp, c_vp, c_vp]),
    "darb_densify_stats": (c_i32, [c_vp, c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "darb_densify_workspace_size": (c_i32, [c_i32, _P(ctypes.c_size_t)]),
    "darb_densify": (c_i32, [_P(darb_train_params), _P(darb_adam_state), c_vp, c_vp, c_vp, c_vp,
                             _P(darb_densify_cfg), c_vp, ctypes.c_size_t, c_i32, _P(darb_train_params),
                             _P(darb_adam_state), c_vp, c_vp]),
    "darb_reset_opacity": (c_i32, [_P(darb_train_params), c_f32, c_vp]),
    "darb_serve_create": (c_i32, [_P(darb_serve_cfg), _P(c_vp)]),
    "darb_serve_add_scene": (c_i32, [c_vp, _P(darb_splats), _P(c_i32)]),
    "darb_serve_submit": (c_i32, [c_vp, _P(darb_request), _P(ctypes.c_uint64)]),
    "darb_serve_submit_many": (c_i32, [c_vp, _P(darb_request), c_i32, _P(ctypes.c_uint64), _P(c_i32)]),
    "darb_serve_poll": (c_i32, [c_vp, ctypes.c_uint64, c_i32, _P(darb_result)]),
    "darb_serve_destroy": (None, [c_vp]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def lib() -> ctypes.CDLL:
    """Load libdarb.so (built in-tree by paper_2501_12369_gb300.build).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libdarb.so not found at {path}; build it with paper_2501_12369_gb300.build.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


class DarbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


def _check(status: int, where: str):
    if status != 0:
        raise DarbError(status, where)


def _p(t):
    return None if t is None else c_vp(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return c_vp(s.cuda_stream)


# ---------------------------------------------------------------------------
# Host structs

def kernel_index(kernel) -> int:
    return KERNEL_NAMES.index(kernel) if isinstance(kernel, str) else int(kernel)


def darb_kernel_defaults(kernel) -> darb_kernel_params:
    """Parameters of a fixed kernel (name or enum); a darb_kernel_params is returned as a copy."""
    if isinstance(kernel, darb_kernel_params):
        return darb_kernel_params.from_buffer_copy(kernel)
    kp = darb_kernel_params()
    _check(lib().darb_kernel_defaults(kernel_index(kernel), ctypes.byref(kp)), "darb_kernel_defaults")
    return kp


DARB_GENERIC = 7
GENERIC_BASES = ("gaussian", "half_cosine", "raised_cosine", "mod_sinc", "inv_multiquadric", "parabola")


def darb_kernel_generic(base, xi, beta, lobes=1, psi="device", device="cuda") -> darb_kernel_params:
    """A member of Table 1's modified family; psi="device" computes it with darb_kernel_psi,
    a number sets it, None leaves 1."""
    b = GENERIC_BASES.index(base) if isinstance(base, str) else int(base)
    kp = darb_kernel_params()
    _check(lib().darb_kernel_generic(b, float(xi), float(beta), int(lobes), ctypes.byref(kp)), "darb_kernel_generic")
    if psi == "device":
        kp.psi = darb_kernel_psi(kp, device=device)
    elif psi is not None:
        kp.psi = float(psi)
    return kp


def darb_kernel_psi(kp: darb_kernel_params, device="cuda", stream=None) -> float:
    """psi of any kernel by the moment integral on the device (synchronises)."""
    scratch = torch.empty(2, dtype=torch.float64, device=device)
    out = ctypes.c_double(0.0)
    _check(lib().darb_kernel_psi(ctypes.byref(kp), _p(scratch), ctypes.byref(out), _stream(stream)),
           "darb_kernel_psi")
    return float(out.value)


def camera(cam) -> darb_camera:
    """darb_camera from any object with viewmat, fx, fy, cx, cy, near, width, height, bg."""
    c = darb_camera()
    c.viewmat[:] = [float(v) for v in np.asarray(cam.viewmat, np.float32).reshape(16)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane = float(cam.near)
    c.width, c.height = int(cam.width), int(cam.height)
    c.bg[:] = [float(b) for b in cam.bg]
    return c


def darb_tile_grid(cam, tile):
    tx, ty = c_i32(), c_i32()
    _check(lib().darb_tile_grid(ctypes.byref(camera(cam)), int(tile), ctypes.byref(tx), ctypes.byref(ty)),
           "darb_tile_grid")
    return tx.value, ty.value


@dataclasses.dataclass
class SplatTensors:
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    opacities: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def n(self):
        return int(self.means.shape[0])

    def struct(self) -> darb_splats:
        for t in (self.means, self.scales, self.quats, self.opacities, self.sh):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        return darb_splats(_p(self.means), _p(self.scales), _p(self.quats), _p(self.opacities), _p(self.sh),
                           self.n, int(self.sh_degree))


def splats_to_device(s, device="cuda") -> SplatTensors:
    """Copy a synth.Splats (numpy) to the device."""
    t = [torch.from_numpy(np.ascontiguousarray(a)).to(device) for a in (s.means, s.scales, s.quats, s.opacities, s.sh)]
    return SplatTensors(*t, s.sh_degree)


@dataclasses.dataclass
class Projected:
    depth: torch.Tensor
    radius: torch.Tensor
    tile_rect: torch.Tensor
    mean2d: torch.Tensor
    conic_o: torch.Tensor
    rgb: torch.Tensor
    clamped: torch.Tensor
    tiles_touched: torch.Tensor
    tile_runs: torch.Tensor

    @staticmethod
    def empty(n, device="cuda"):
        f = dict(device=device)
        return Projected(torch.empty(n, dtype=torch.float32, **f), torch.empty(n, dtype=torch.int32, **f),
                         torch.empty(n, 4, dtype=torch.int32, **f), torch.empty(n, 2, dtype=torch.float32, **f),
                         torch.empty(n, 4, dtype=torch.float32, **f), torch.empty(n, 3, dtype=torch.float32, **f),
                         torch.empty(n, dtype=torch.uint8, **f), torch.empty(n, dtype=torch.int32, **f),
                         torch.empty(n, dtype=torch.int64, **f))

    def struct(self) -> darb_projected:
        return darb_projected(*(_p(getattr(self, f.name)) for f in dataclasses.fields(self)))


@dataclasses.dataclass
class Binning:
    keys: torch.Tensor
    values: torch.Tensor
    ranges: torch.Tensor
    num_instances: torch.Tensor
    status: torch.Tensor
    M: int | None = None

    @staticmethod
    def empty(capacity, n_tiles, device="cuda", keys=True):
        """keys=False leaves out the 64-bit keys (only the DARB_SORT_KEYS64 strategy needs them)."""
        f = dict(device=device)
        cap = max(int(capacity), 1)
        return Binning(torch.empty(cap, dtype=torch.int64, **f) if keys else None,
                       torch.empty(cap, dtype=torch.int32, **f),
                       torch.empty(n_tiles, 2, dtype=torch.int32, **f), torch.zeros(1, dtype=torch.int32, **f),
                       torch.zeros(1, dtype=torch.int32, **f))

    def struct(self) -> darb_binning:
        return darb_binning(_p(self.keys), _p(self.values), _p(self.ranges), _p(self.num_instances), _p(self.status))


@dataclasses.dataclass
class ImageOut:
    image: torch.Tensor
    t_final: torch.Tensor
    last: torch.Tensor
    n_contrib: torch.Tensor

    @staticmethod
    def empty(width, height, device="cuda"):
        f = dict(device=device)
        return ImageOut(torch.empty(3, height, width, dtype=torch.float32, **f),
                        torch.empty(height, width, dtype=torch.float32, **f),
                        torch.empty(height, width, dtype=torch.int32, **f),
                        torch.empty(height, width, dtype=torch.int32, **f))

    def struct(self) -> darb_image:
        return darb_image(_p(self.image), _p(self.t_final), _p(self.last), _p(self.n_contrib))


# ---------------------------------------------------------------------------
# Entry points

def darb_preprocess(splats: SplatTensors, cam, kparams, tile=16, out: Projected | None = None, stream=None):
    """The projected records; they remember `kparams` (the sort needs its q_max)."""
    out = Projected.empty(splats.n, splats.means.device) if out is None else out
    sp, c, o = splats.struct(), camera(cam), out.struct()
    _check(lib().darb_preprocess(ctypes.byref(sp), ctypes.byref(c), ctypes.byref(kparams), int(tile), ctypes.byref(o),
                                 _stream(stream)), "darb_preprocess")
    out.kparams = kparams
    return out


DARB_SORT_DEPTH_THEN_TILE = 0
DARB_SORT_KEYS64 = 1


def darb_bin_sort_workspace_size(n, tile, cam, capacity, strategy=DARB_SORT_DEPTH_THEN_TILE) -> int:
    b = ctypes.c_size_t()
    _check(lib().darb_bin_sort_workspace_size(int(n), int(tile), ctypes.byref(camera(cam)), int(capacity),
                                              int(strategy), ctypes.byref(b)), "darb_bin_sort_workspace_size")
    return int(b.value)


def darb_bin_sort(proj: Projected, n, tile, cam, workspace: torch.Tensor, capacity, out: Binning | None = None,
                  sync=True, stream=None, strategy=DARB_SORT_DEPTH_THEN_TILE, kparams=None):
    """sync=True reads M back (one stream synchronisation) and sizes the sort by it.  kparams:
    the kernel the records were projected with (default: the one darb_preprocess recorded)."""
    tx, ty = darb_tile_grid(cam, tile)
    out = Binning.empty(capacity, tx * ty, workspace.device) if out is None else out
    pr, c, b = proj.struct(), camera(cam), out.struct()
    kp = proj.kparams if kparams is None else kparams
    m = ctypes.c_uint64(0)
    st = lib().darb_bin_sort(ctypes.byref(pr), int(n), int(tile), ctypes.byref(c), ctypes.byref(kp), _p(workspace),
                             workspace.numel() * workspace.element_size(), int(capacity), int(strategy),
                             ctypes.byref(b), ctypes.byref(m) if sync else None, _stream(stream))
    out.M = int(m.value) if sync else None
    if st != 0:
        err = DarbError(st, "darb_bin_sort")
        err.M = out.M  # on DARB_ERR_CAPACITY: the instance count the lists need
        raise err
    return out


def darb_bin_sort_noalloc(proj: Projected, n, tile, cam, capacity, out: Binning | None = None, sync=True,
                          stream=None, kparams=None):
    """darb_bin_sort with the library's static device scratch instead of a caller workspace."""
    tx, ty = darb_tile_grid(cam, tile)
    out = Binning.empty(capacity, tx * ty, proj.depth.device) if out is None else out
    pr, c, b = proj.struct(), camera(cam), out.struct()
    kp = proj.kparams if kparams is None else kparams
    m = ctypes.c_uint64(0)
    st = lib().darb_bin_sort_noalloc(ctypes.byref(pr), int(n), int(tile), ctypes.byref(c), ctypes.byref(kp),
                                     int(capacity),
                                     ctypes.byref(b), ctypes.byref(m) if sync else None, _stream(stream))
    out.M = int(m.value) if sync else None
    _check(st, "darb_bin_sort_noalloc")
    return out


def darb_render_fwd(proj: Projected, bins: Binning, cam, kparams, tile=16, out: ImageOut | None = None, stream=None):
    out = ImageOut.empty(cam.width, cam.height, proj.depth.device) if out is None else out
    pr, b, c, o = proj.struct(), bins.struct(), camera(cam), out.struct()
    _check(lib().darb_render_fwd(ctypes.byref(pr), ctypes.byref(b), ctypes.byref(c), ctypes.byref(kparams), int(tile),
                                 ctypes.byref(o), _stream(stream)), "darb_render_fwd")
    return out


def darb_render_fwd_l1(proj: Projected, bins: Binning, cam, kparams, tile, target, out: ImageOut | None = None,
                       dL_dimage=None, loss=None, stream=None):
    """Forward with the L1 loss in its epilogue; returns (image outputs, dL_dimage, loss[1]).
    out.image and out.n_contrib may be None (not written)."""
    out = ImageOut.empty(cam.width, cam.height, proj.depth.device) if out is None else out
    dL_dimage = torch.empty_like(target) if dL_dimage is None else dL_dimage
    loss = torch.empty(1, dtype=torch.float32, device=target.device) if loss is None else loss
    assert target.is_contiguous() and target.dtype == torch.float32
    assert tuple(target.shape) == (3, cam.height, cam.width)
    pr, b, c, o = proj.struct(), bins.struct(), camera(cam), out.struct()
    _check(lib().darb_render_fwd_l1(ctypes.byref(pr), ctypes.byref(b), ctypes.byref(c), ctypes.byref(kparams),
                                    int(tile), ctypes.byref(o), _p(target), _p(dL_dimage), _p(loss), _stream(stream)),
           "darb_render_fwd_l1")
    return out, dL_dimage, loss


def darb_render_bwd(proj: Projected, n, bins: Binning, cam, kparams, tile, fwd: ImageOut, dL_dimage: torch.Tensor,
                    grad2d: torch.Tensor | None = None, stream=None):
    grad2d = torch.empty(n, 12, dtype=torch.float32, device=proj.depth.device) if grad2d is None else grad2d
    assert dL_dimage.is_contiguous() and dL_dimage.dtype == torch.float32
    pr, b, c, f = proj.struct(), bins.struct(), camera(cam), fwd.struct()
    _check(lib().darb_render_bwd(ctypes.byref(pr), int(n), ctypes.byref(b), ctypes.byref(c), ctypes.byref(kparams),
                                 int(tile), ctypes.byref(f), _p(dL_dimage), _p(grad2d), _stream(stream)),
           "darb_render_bwd")
    return grad2d


@dataclasses.dataclass
class SplatGrads:
    dmeans: torch.Tensor
    dscales: torch.Tensor
    dquats: torch.Tensor
    dopacities: torch.Tensor
    dsh: torch.Tensor

    @staticmethod
    def empty_like(s: SplatTensors):
        return SplatGrads(*(torch.empty_like(t) for t in (s.means, s.scales, s.quats, s.opacities, s.sh)))

    @staticmethod
    def empty_flat(n, sh_degree, device="cuda", dtype=torch.float32):
        """Gradients as views into one contiguous buffer (`.flat`), so a data-parallel step can
        reduce them with a single collective.  Every view starts on a 16-byte boundary."""
        k = (sh_degree + 1) ** 2
        shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, k, 3)]
        sizes = [int(np.prod(sh)) for sh in shapes]
        padded = [(z + 3) // 4 * 4 for z in sizes]
        flat = torch.empty(sum(padded), dtype=dtype, device=device)
        views, off = [], 0
        for sh, z, pz in zip(shapes, sizes, padded):
            views.append(flat[off:off + z].view(sh))
            off += pz
        g = SplatGrads(*views)
        g.flat = flat
        return g

    def struct(self) -> darb_splat_grads:
        return darb_splat_grads(_p(self.dmeans), _p(self.dscales), _p(self.dquats), _p(self.dopacities), _p(self.dsh))


def darb_preprocess_bwd(splats: SplatTensors, cam, kparams, proj: Projected, grad2d: torch.Tensor,
                        out: SplatGrads | None = None, stream=None):
    out = SplatGrads.empty_like(splats) if out is None else out
    sp, c, pr, g = splats.struct(), camera(cam), proj.struct(), out.struct()
    _check(lib().darb_preprocess_bwd(ctypes.byref(sp), ctypes.byref(c), ctypes.byref(kparams), ctypes.byref(pr),
                                     _p(grad2d), ctypes.byref(g), _stream(stream)), "darb_preprocess_bwd")
    return out


def darb_l1_loss(image, target, dL_dimage=None, loss=None, stream=None):
    H, W = image.shape[-2:]
    dL_dimage = torch.empty_like(image) if dL_dimage is None else dL_dimage
    loss = torch.empty(1, dtype=torch.float32, device=image.device) if loss is None else loss
    _check(lib().darb_l1_loss(_p(image), _p(target), int(W), int(H), _p(dL_dimage), _p(loss), _stream(stream)),
           "darb_l1_loss")
    return dL_dimage, loss


def train_params(params) -> darb_train_params:
    """params: an object exposing the darb_train_params fields as tensors (plus sh_degree)."""
    return darb_train_params(_p(params.means), _p(params.log_scales), _p(params.quats), _p(params.opacity_logits),
                             _p(params.sh), _p(params.scales), _p(params.opacities), int(params.means.shape[0]),
                             int(params.sh_degree))


def adam_state(state) -> darb_adam_state:
    """state: an object exposing the darb_adam_state fields as tensors."""
    return darb_adam_state(*(_p(getattr(state, f)) for f, _ in darb_adam_state._fields_))


def darb_preprocess_bwd_adam(params, cam, kparams, proj: Projected, grad2d: torch.Tensor, state,
                             cfg: darb_adam_config, stream=None):
    """Preprocess backward and the Adam step in one pass; params and state are updated in place."""
    p, s, c, pr = train_params(params), adam_state(state), camera(cam), proj.struct()
    _check(lib().darb_preprocess_bwd_adam(ctypes.byref(p), ctypes.byref(c), ctypes.byref(kparams), ctypes.byref(pr),
                                          _p(grad2d), ctypes.byref(s), ctypes.byref(cfg), _stream(stream)),
           "darb_preprocess_bwd_adam")


def darb_l1_dssim_workspace_size(width, height) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().darb_l1_dssim_workspace_size(int(width), int(height), ctypes.byref(n)),
           "darb_l1_dssim_workspace_size")
    return int(n.value)


def darb_l1_dssim_loss(image, target, lam=0.2, workspace=None, dL_dimage=None, loss=None, stream=None):
    """(1 - lam) L1 + lam (1 - SSIM) of [3, H, W] images; returns (dL_dimage, loss[2] = (L, mean SSIM))."""
    H, W = image.shape[-2:]
    if workspace is None:
        workspace = torch.empty(darb_l1_dssim_workspace_size(W, H), dtype=torch.uint8, device=image.device)
    dL_dimage = torch.empty_like(image) if dL_dimage is None else dL_dimage
    loss = torch.empty(2, dtype=torch.float32, device=image.device) if loss is None else loss
    _check(lib().darb_l1_dssim_loss(_p(image), _p(target), int(W), int(H), float(lam), _p(workspace),
                                    workspace.numel() * workspace.element_size(), _p(dL_dimage), _p(loss),
                                    _stream(stream)), "darb_l1_dssim_loss")
    return dL_dimage, loss


def darb_adam_step(params, grads: SplatGrads, state, cfg: darb_adam_config, stream=None):
    """params / state: objects exposing the darb_train_params / darb_adam_state fields as tensors."""
    p, s = train_params(params), adam_state(state)
    g = grads.struct()
    _check(lib().darb_adam_step(ctypes.byref(p), ctypes.byref(g), ctypes.byref(s), ctypes.byref(cfg), _stream(stream)),
           "darb_adam_step")


# ---------------------------------------------------------------------------
# A reusable forward/backward pipeline and its autograd wrapper.

class Rasterizer:
    """Holds the per-view buffers of one camera configuration and runs the four steps.

    The sort workspace is scratch of a single call and is reused by every forward.  The lists a
    forward returns are reused too unless `forward(..., owned=True)` is asked for: then they are
    freshly allocated and belong to the caller, so several forwards can be pending a backward.
    Calls are ordered on the current stream.  With sync=True (the default) forward synchronises
    once to read the instance count and, if the lists did not fit, grows the capacity and sorts
    again.  With sync=False nothing synchronises: the sort runs in its asynchronous capacity mode
    (a view that does not fit renders as background and flags DARB_ERR_CAPACITY on the device),
    and `check()` later reads every pending forward's status at once and raises on an overflow.
    Each pending forward keeps an 8-byte device tensor until the next check(), so a long run
    should call check() now and then (once per step or per batch of views).
    """

    def __init__(self, cam, kernel="half_cosine", tile=16, capacity=None, device="cuda", psi=None,
                 strategy=DARB_SORT_DEPTH_THEN_TILE, sync=True):
        self.cam = cam
        self.sync = bool(sync)
        self._pending = []  # asynchronous mode: (status, M) of every forward since the last check
        self.strategy = int(strategy)
        self.tile = int(tile)
        self.kparams = darb_kernel_defaults(kernel)
        if psi is not None:
            self.kparams.psi = float(psi)
        self.device = device
        self.tiles_x, self.tiles_y = darb_tile_grid(cam, tile)
        self.capacity = int(capacity) if capacity else 0
        self._ws = None
        self._bins = None
        self._n = -1

    def _ensure(self, n, capacity):
        if capacity > self.capacity or self._ws is None or n != self._n:
            self.capacity = max(capacity, self.capacity)
            nbytes = darb_bin_sort_workspace_size(n, self.tile, self.cam, self.capacity, self.strategy)
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self._bins = Binning.empty(self.capacity, self.tiles_x * self.tiles_y, self.device)
            self._n = n

    def _sort(self, proj, n, owned):
        tx, ty = darb_tile_grid(self.cam, self.tile)
        if (tx, ty) != (self.tiles_x, self.tiles_y):  # the camera was changed to another resolution
            self.tiles_x, self.tiles_y = tx, ty
            self._ws = None
        self._ensure(n, self.capacity)
        out = (Binning.empty(self.capacity, tx * ty, self.device, keys=self.strategy == DARB_SORT_KEYS64)
               if owned else self._bins)
        return darb_bin_sort(proj, n, self.tile, self.cam, self._ws, self.capacity, out, sync=self.sync,
                             strategy=self.strategy)

    def forward(self, splats: SplatTensors, owned=False):
        proj = darb_preprocess(splats, self.cam, self.kparams, self.tile)
        if self.capacity == 0:
            self.capacity = max(1024, 8 * splats.n)
        if not self.sync:
            bins = self._sort(proj, splats.n, owned)
            # a device-side copy of this call's status word and instance count (the shared
            # lists of a later forward overwrite bins.status)
            self._pending.append(torch.cat([bins.status[:1], bins.num_instances[:1]]))
            img = darb_render_fwd(proj, bins, self.cam, self.kparams, self.tile)
            return proj, bins, img
        try:
            bins = self._sort(proj, splats.n, owned)
        except DarbError as e:
            if e.status != 3:
                raise
            self._ensure(splats.n, int(e.M * 1.25) + 1)
            bins = self._sort(proj, splats.n, owned)
        img = darb_render_fwd(proj, bins, self.cam, self.kparams, self.tile)
        return proj, bins, img

    def check(self):
        """Asynchronous mode: one synchronisation for every forward since the last check.  Raises
        DarbError (with .M, the largest instance count asked for) if any of them overflowed its
        capacity; those images are background only.  The pending list is cleared either way."""
        pending, self._pending = self._pending, []
        if not pending:
            return
        sm = torch.stack(pending).cpu().numpy().astype(np.int64)
        sm[:, 1] &= 0xFFFFFFFF  # the count is a u32 in an int32 tensor
        bad = sm[:, 0] != 0
        if bad.any():
            err = DarbError(int(sm[bad][0, 0]), "Rasterizer.check")
            err.M = int(sm[bad][:, 1].max())
            raise err

    def backward(self, splats, proj, bins, img, dL_dimage, cam=None):
        cam = self.cam if cam is None else cam
        g2 = darb_render_bwd(proj, splats.n, bins, cam, self.kparams, self.tile, img, dL_dimage.contiguous())
        return darb_preprocess_bwd(splats, cam, self.kparams, proj, g2), g2


class DarbRasterize(torch.autograd.Function):
    """image = DarbRasterize.apply(means, scales, quats, opacities, sh, sh_degree, rasterizer).

    The inputs are the activated splat attributes (scales and opacities after exp / sigmoid,
    quaternions raw: the library normalises them and differentiates through the normalisation);
    the output is the [3, H, W] image of `rasterizer.cam`.  Every call keeps its own projected
    records, lists, image buffers and a snapshot of the camera, so a rasterizer can render several
    views (or the same view twice) before one backward.  The backward is the hand-written one of
    Sec. 4.2: compositing replayed back to front, then the chain through the conic, psi, the EWA
    projection, the quaternion normalisation and the SH basis.
    """

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, sh_degree, rasterizer):
        s = SplatTensors(means.detach().contiguous(), scales.detach().contiguous(), quats.detach().contiguous(),
                         opacities.detach().contiguous(), sh.detach().contiguous(), int(sh_degree))
        proj, bins, img = rasterizer.forward(s, owned=True)
        ctx.state = (s, proj, bins, img, rasterizer, rasterizer.cam)
        return img.image

    @staticmethod
    def backward(ctx, dimage):
        s, proj, bins, img, r, cam = ctx.state
        g, _ = r.backward(s, proj, bins, img, dimage.float().contiguous(), cam=cam)
        return g.dmeans, g.dscales, g.dquats, g.dopacities, g.dsh, None, None


def autotune_tile(splats: SplatTensors, cams, kernel="half_cosine", candidates=(8, 16, 32), reps=5,
                  strategy=DARB_SORT_DEPTH_THEN_TILE):
    """Tile size with the fastest forward (preprocess, bin/sort, compositing) over `cams`.

    Each candidate is warmed once per camera (which also sizes its instance capacity), then
    timed with CUDA events over `reps` passes of the camera list.  Returns
    (best_tile, {tile: ms per view}).  All cameras must share one resolution.
    """
    times = {}
    for t in candidates:
        rast = Rasterizer(cams[0], kernel, t, strategy=strategy)
        for cam in cams:  # warm-up and capacity sizing
            rast.cam = cam
            rast.forward(splats)
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        for _ in range(reps):
            for cam in cams:
                rast.cam = cam
                rast.forward(splats)
        end.record()
        torch.cuda.synchronize()
        times[t] = start.elapsed_time(end) / (reps * len(cams))
    return min(times, key=times.get), times


# ---------------------------------------------------------------------------
# Batched multi-view rendering

def darb_render_batch_workspace_size(n, cams, params: darb_batch_params) -> int:
    arr = (darb_camera * len(cams))(*[camera(c) for c in cams])
    nbytes = ctypes.c_size_t(0)
    _check(lib().darb_render_batch_workspace_size(int(n), arr, ctypes.byref(params), ctypes.byref(nbytes)),
           "darb_render_batch_workspace_size")
    return int(nbytes.value)


def darb_render_batch(splats: SplatTensors, cams, kparams, params: darb_batch_params, workspace: torch.Tensor,
                      outs, num_instances=None, status=None, stream=None):
    """outs: one ImageOut per camera (t_final / last / n_contrib may be None)."""
    arr = (darb_camera * len(cams))(*[camera(c) for c in cams])
    imgs = (darb_image * len(outs))(*[darb_image(_p(o.image), _p(o.t_final), _p(o.last), _p(o.n_contrib))
                                      for o in outs])
    sp = splats.struct()
    _check(lib().darb_render_batch(ctypes.byref(sp), arr, ctypes.byref(kparams), ctypes.byref(params), _p(workspace),
                                   workspace.numel() * workspace.element_size(), imgs, _p(num_instances),
                                   _p(status), _stream(stream)), "darb_render_batch")


class BatchRenderer:
    """Forward renders of many cameras of one splat set: one darb_render_batch call, which can be
    captured once into a CUDA graph and replayed.

    capacity: instances per view; None sizes it from one counting pass per camera (x slack).
    aux: also keep t_final / last / n_contrib per view."""

    def __init__(self, splats: SplatTensors, cams, kernel="half_cosine", tile=16, depth=2, capacity=None,
                 aux=False, max_ctas=0, slack=1.15, device="cuda"):
        self.splats, self.cams = splats, list(cams)
        self.kparams = darb_kernel_defaults(kernel)
        self.tile, self.depth = int(tile), int(depth)
        self.device = device
        self.counts = None
        if capacity is None:
            self.counts = self.count_instances()
            capacity = int(max(self.counts) * slack) + 1024
        self.params = darb_batch_params(len(self.cams), self.tile, self.depth, int(max_ctas), int(capacity))
        nbytes = darb_render_batch_workspace_size(splats.n, self.cams, self.params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        f = dict(device=device)
        self.outs = []
        for c in self.cams:
            if aux:
                self.outs.append(ImageOut.empty(c.width, c.height, device))
            else:
                self.outs.append(ImageOut(torch.empty(3, c.height, c.width, dtype=torch.float32, **f), None, None,
                                          None))
        self.num_instances = torch.zeros(len(self.cams), dtype=torch.int32, **f)
        self.status = torch.zeros(len(self.cams), dtype=torch.int32, **f)
        self.graph = None

    @property
    def capacity(self):
        return int(self.params.capacity)

    def count_instances(self):
        """M of every camera at this tile size (synchronises once per camera)."""
        counts = []
        for c in self.cams:
            proj = darb_preprocess(self.splats, c, self.kparams, self.tile)
            ws = torch.empty(darb_bin_sort_workspace_size(self.splats.n, self.tile, c, 1), dtype=torch.uint8,
                             device=self.device)
            tx, ty = darb_tile_grid(c, self.tile)
            bins = Binning.empty(1, tx * ty, self.device)
            pr, cc, b = proj.struct(), camera(c), bins.struct()
            m = ctypes.c_uint64(0)
            st = lib().darb_bin_sort(ctypes.byref(pr), self.splats.n, self.tile, ctypes.byref(cc),
                                     ctypes.byref(self.kparams), _p(ws),
                                     ws.numel(), 1, DARB_SORT_DEPTH_THEN_TILE, ctypes.byref(b), ctypes.byref(m),
                                     _stream())
            if st not in (0, 3):
                _check(st, "darb_bin_sort")
            counts.append(int(m.value))
        return counts

    def render(self, stream=None):
        darb_render_batch(self.splats, self.cams, self.kparams, self.params, self.workspace, self.outs,
                          self.num_instances, self.status, stream)

    def capture(self):
        """Record one batch into a CUDA graph (after one eager call, which creates the library's
        per-device streams)."""
        self.render()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            g.capture_begin()
            self.render(s)
            g.capture_end()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def check(self):
        """Raises if any view overflowed its capacity or a device wait timed out."""
        st = self.status.cpu().numpy()
        if np.any(st != 0):
            bad = int(np.flatnonzero(st)[0])
            raise DarbError(int(st[bad]), f"view {bad} of the batch (M = {int(self.num_instances[bad])})")


def autotune_batch(splats: SplatTensors, cams, kernel="half_cosine", tiles=(8, 16, 32), depths=(1, 2, 4, 8), reps=5):
    """(tile, depth) with the fastest graph-replayed batch over `cams`, and the ms per batch of
    every pair.  Capacities are sized per tile from counting passes."""
    times = {}
    for t in tiles:
        counts = None
        for d in depths:
            br = BatchRenderer(splats, cams, kernel, t, d,
                               capacity=None if counts is None else int(max(counts) * 1.15) + 1024)
            counts = br.counts if counts is None else counts
            br.capture()
            br.replay()
            torch.cuda.synchronize()
            br.check()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                br.replay()
            e1.record()
            torch.cuda.synchronize()
            times[(t, d)] = e0.elapsed_time(e1) / reps
            del br
    best = min(times, key=times.get)
    return best, times


# ---------------------------------------------------------------------------
# Serving

class Server:
    """A darb_server: resident scenes, submit / poll of render requests (continuous batching in
    the library's worker thread).  Images are caller-owned device tensors [3, H, W]."""

    def __init__(self, scene_bytes, workspace_bytes, tile=32, max_batch=32, depth=2, capacity_per_pixel=16.0,
                 capacity_margin=1.15, capacity_min=1 << 16, slots=2):
        self.cfg = darb_serve_cfg(int(scene_bytes), int(workspace_bytes), int(tile), int(max_batch), int(depth),
                                  float(capacity_per_pixel), float(capacity_margin), int(capacity_min), int(slots))
        self.handle = c_vp()
        _check(lib().darb_serve_create(ctypes.byref(self.cfg), ctypes.byref(self.handle)), "darb_serve_create")
        self._keep = {}  # ticket -> image tensor, alive until collected

    def add_scene(self, splats: SplatTensors) -> int:
        sid = c_i32(0)
        sp = splats.struct()
        _check(lib().darb_serve_add_scene(self.handle, ctypes.byref(sp), ctypes.byref(sid)), "darb_serve_add_scene")
        return int(sid.value)

    def submit(self, scene_id, cam, image: torch.Tensor, kernel="half_cosine") -> int:
        assert image.is_contiguous() and image.dtype == torch.float32 and tuple(image.shape) == (3, cam.height,
                                                                                                 cam.width)
        req = darb_request(int(scene_id), kernel_index(kernel), camera(cam), _p(image))
        t = ctypes.c_uint64(0)
        _check(lib().darb_serve_submit(self.handle, ctypes.byref(req), ctypes.byref(t)), "darb_serve_submit")
        self._keep[int(t.value)] = image
        return int(t.value)

    def submit_many(self, scene_ids, cams, images, kernels="half_cosine"):
        """Queues several requests at once (the worker sees them together); returns their tickets."""
        n = len(cams)
        kernels = [kernels] * n if isinstance(kernels, (str, int)) else list(kernels)
        for cam, image in zip(cams, images):
            assert image.is_contiguous() and image.dtype == torch.float32 and \
                tuple(image.shape) == (3, cam.height, cam.width)
        reqs = (darb_request * n)(*[darb_request(int(sid), kernel_index(k), camera(c), _p(im))
                                    for sid, c, im, k in zip(scene_ids, cams, images, kernels)])
        tickets = (ctypes.c_uint64 * n)()
        done = c_i32(0)
        st = lib().darb_serve_submit_many(self.handle, reqs, n, tickets, ctypes.byref(done))
        for k in range(done.value):
            self._keep[int(tickets[k])] = images[k]
        _check(st, "darb_serve_submit_many")
        return [int(tickets[k]) for k in range(n)]

    def poll(self, ticket, timeout_ms=10_000) -> darb_result:
        r = darb_result()
        _check(lib().darb_serve_poll(self.handle, int(ticket), int(timeout_ms), ctypes.byref(r)), "darb_serve_poll")
        self._keep.pop(int(ticket), None)
        return r

    def close(self):
        if self.handle:
            lib().darb_serve_destroy(self.handle)
            self.handle = c_vp()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Data-parallel training over several views per step

def allreduce_splat_grads(grads: SplatGrads, group=None, average=False):
    """Sums (or averages) the per-splat parameter gradients over the ranks of `group` with one
    all-reduce of the flat buffer (grads from SplatGrads.empty_flat).  Each rank renders its own
    views and runs darb_preprocess_bwd; after this call every rank holds the gradient of the
    summed loss and applies the same darb_adam_step."""
    import torch.distributed as dist
    flat = getattr(grads, "flat", None)
    if flat is None:
        raise ValueError("allreduce_splat_grads needs gradients from SplatGrads.empty_flat")
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    if average:
        flat /= dist.get_world_size(group)
    return grads


# ---------------------------------------------------------------------------
# Adaptive density control

def darb_densify_stats(grad2d, radius, width, height, accum, count, max_radius, stream=None):
    _check(lib().darb_densify_stats(_p(grad2d), _p(radius), int(radius.shape[0]), int(width), int(height), _p(accum),
                                    _p(count), _p(max_radius), _stream(stream)), "darb_densify_stats")


def darb_densify(params, state, accum, count, max_radius, split_normals, cfg: darb_densify_cfg, out_params,
                 out_state, stream=None):
    """One clone / split / prune pass from (params, state) into (out_params, out_state), which
    need 2 n rows; returns the device uint32[3] (rows written, first clone row, first child row)."""
    n = int(params.means.shape[0])
    ws = torch.empty(_ws_size(lib().darb_densify_workspace_size, n), dtype=torch.uint8, device=params.means.device)
    n_out = torch.zeros(3, dtype=torch.int32, device=params.means.device)
    p_in, s_in = train_params(params), adam_state(state)
    p_out, s_out = train_params(out_params), adam_state(out_state)
    p_out.n = int(out_params.means.shape[0])
    _check(lib().darb_densify(ctypes.byref(p_in), ctypes.byref(s_in), _p(accum), _p(count), _p(max_radius),
                              _p(split_normals), ctypes.byref(cfg), _p(ws), ws.numel(), int(out_params.means.shape[0]),
                              ctypes.byref(p_out), ctypes.byref(s_out), _p(n_out), _stream(stream)), "darb_densify")
    return n_out


def _ws_size(fn, *args) -> int:
    n = ctypes.c_size_t(0)
    _check(fn(*args, ctypes.byref(n)), fn.__name__)
    return int(n.value)


def darb_reset_opacity(params, max_opacity=0.01, stream=None):
    p = train_params(params)
    _check(lib().darb_reset_opacity(ctypes.byref(p), float(max_opacity), _stream(stream)), "darb_reset_opacity")

