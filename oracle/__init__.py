"""CPU oracle of the DARB-Splatting rasterizer: ctypes wrapper around darb_oracle.c.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.
It shares no code with the CUDA library and imports nothing from it.

The rasterizer's arithmetic (projection, SH, kernels, tile lists,
compositing, its analytic gradient, psi by quadrature) lives in
darb_oracle.c (see its header for what is computed and where the paper
defines it); the functions wrapping it here only marshal arguments.  The
training-step terms are plain FP64 NumPy in this file: l1_loss, ssim_window,
ssim_map and l1_dssim_loss (the image loss), densify_stats, densify_actions,
densify and reset_opacity (density control), adam_update and
adam_step_splats (the optimiser), and psi_moment's quadrature driver.

Kernel table (Table 1 forms with the xi of Table 2, the psi of the Sec. B
listings, and the main-lobe limits of Sec. A.3 / the listings):

  name               enum  psi    q_max  strict   F(q), q = d_M^2
  gaussian            0    1.0    9.0    no       exp(-q/2)
  half_cosine         1    1.36   9.0    no       cos(pi q / 18)
  raised_cosine       2    0.655  6.25   no       1/2 + 1/2 cos(pi sqrt(q) / 2.5)
  mod_sinc            3    1.18   9.0    no       sin(x)/x, x = pi sqrt(q) / 3
  inv_quadric         4    1.38   9.0    yes      1 / (1 + q)
  inv_multiquadric    5    1.61   9.0    yes      (1 + q)^(-1/2)
  parabola            6    1.3    9.0    no       1 - q/9
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "darb_oracle.c")
_HDR = os.path.join(_HERE, "project_impl.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libdarb_oracle.so")

KERNELS = {
    # name: (enum, psi, q_max, strict)
    "gaussian": (0, 1.0, 9.0, 0),
    "half_cosine": (1, 1.36, 9.0, 0),
    "raised_cosine": (2, 0.655, 6.25, 0),
    "mod_sinc": (3, 1.18, 9.0, 0),
    "inv_quadric": (4, 1.38, 9.0, 1),
    "inv_multiquadric": (5, 1.61, 9.0, 1),
    "parabola": (6, 1.3, 9.0, 0),
}
KERNEL_NAMES = list(KERNELS)

# Default ambiguity margins for the alpha >= 1/255 and T(1-alpha) >= 1e-4 tests:
# |alpha - 1/255| <= EPS_ALPHA (absolute), |T(1-alpha) - 1e-4| <= EPS_T * 1e-4.
EPS_ALPHA = 2e-6
EPS_T = 2e-3


class OrcCamera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("near_plane", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("bg", ctypes.c_float * 3)]


class OrcKernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("psi", ctypes.c_float), ("q_max", ctypes.c_float),
                ("q_max_strict", ctypes.c_int), ("base", ctypes.c_int), ("xi", ctypes.c_float),
                ("beta", ctypes.c_float), ("lobes", ctypes.c_int)]


class OrcOutcome(ctypes.Structure):
    _fields_ = [("pixel", ctypes.c_int), ("count", ctypes.c_int), ("last_id", ctypes.c_int),
                ("primary", ctypes.c_int), ("T", ctypes.c_double), ("C", ctypes.c_double * 3),
                ("sig", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None


def _needs_build() -> bool:
    if not os.path.exists(_LIB_PATH):
        return True
    t = os.path.getmtime(_LIB_PATH)
    return any(os.path.getmtime(p) > t for p in (_SRC, _HDR))


def build(force: bool = False) -> str:
    """Compile darb_oracle.c with gcc (-O2, no FP contraction, OpenMP if available)."""
    if not force and not _needs_build():
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    base = [cc, "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-I", _HERE, _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
            return _LIB_PATH
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
            _lib.orc_build_lists.restype = ctypes.c_longlong
            _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def kernel_params(name_or_kind, psi=None):
    name = KERNEL_NAMES[name_or_kind] if isinstance(name_or_kind, int) else name_or_kind
    kind, p, qmax, strict = KERNELS[name]
    return OrcKernel(kind, float(p if psi is None else psi), float(qmax), int(strict))


# Table 1's "modified" family (kind 7): F = base(u), u = d_M^beta / xi, each base on the
# domain that keeps `lobes` lobes (one lobe: the strictly decaying main lobe).
GENERIC = 7
GENERIC_BASES = ("gaussian", "half_cosine", "raised_cosine", "mod_sinc", "inv_multiquadric", "parabola")


def generic_u_max(base, lobes=1):
    """End of the domain in u (Table 1's limits), inf for the unbounded members."""
    b = GENERIC_BASES.index(base) if isinstance(base, str) else int(base)
    return {0: np.inf, 1: np.pi / 2, 2: lobes * np.pi, 3: (lobes + 1) * np.pi / 2, 4: np.inf, 5: 1.0}[b]


def generic_kernel(base, xi, beta, lobes=1, psi=None):
    """Kernel parameters of a modified member.  q_max = min(9, (xi u_max)^(2/beta)): the tile
    rectangle's radius 3 sqrt(lambda_max) bounds every footprint at q = 9.  psi defaults to the
    moment integral (psi_moment)."""
    b = GENERIC_BASES.index(base) if isinstance(base, str) else int(base)
    xi32, beta32 = float(np.float32(xi)), float(np.float32(beta))  # the parameters as stored
    q_dom = (xi32 * generic_u_max(b, lobes)) ** (2.0 / beta32)
    k = OrcKernel(GENERIC, 1.0, float(min(9.0, q_dom)), 0, b, xi32, beta32, int(lobes))
    k.psi = float(psi_moment(k) if psi is None else psi)
    return k


def psi_moment(kp):
    """psi = per-axis second moment of the truncated 3D kernel with Sigma = I (the quantity the
    Sec. A.2 grid experiment measures): (1/3) int r^4 F(r^2) dr / int r^2 F(r^2) dr over
    r in [0, sqrt(q_max)], by adaptive quadrature (breaks at the lobe ends)."""
    from scipy import integrate
    rmax = float(np.sqrt(kp.q_max))

    def f(r):
        return kernel_eval(kp, np.array([r * r]))[0][0]

    pts = None
    if kp.kind == GENERIC and kp.base in (2, 3):
        ends = [(kp.xi * m * np.pi / 2) ** (1.0 / kp.beta) for m in range(1, 2 * kp.lobes + 2)]
        pts = [e for e in ends if 0 < e < rmax] or None
    num = integrate.quad(lambda r: r ** 4 * f(r), 0.0, rmax, points=pts, limit=400, epsabs=0, epsrel=1e-12)[0]
    den = integrate.quad(lambda r: r ** 2 * f(r), 0.0, rmax, points=pts, limit=400, epsabs=0, epsrel=1e-12)[0]
    return num / (3.0 * den)


def camera_struct(cam) -> OrcCamera:
    c = OrcCamera()
    c.viewmat[:] = [float(v) for v in np.asarray(cam.viewmat, np.float32).reshape(16)]
    c.fx, c.fy, c.cx, c.cy, c.near_plane = cam.fx, cam.fy, cam.cx, cam.cy, cam.near
    c.width, c.height = cam.width, cam.height
    c.bg[:] = [float(b) for b in cam.bg]
    return c


def tiles_xy(cam, tile):
    return (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile


def kernel_eval(kind, q):
    """F(q) and dF/dq: kind is a kernel enum, or kernel parameters (the generic family too)."""
    q = np.ascontiguousarray(q, np.float64)
    F = np.empty_like(q)
    dF = np.empty_like(q)
    if isinstance(kind, OrcKernel):
        lib().orc_kernel_eval_k(ctypes.byref(kind), ctypes.c_int(q.size), _p(q), _p(F), _p(dF))
    else:
        lib().orc_kernel_eval(ctypes.c_int(kind), ctypes.c_int(q.size), _p(q), _p(F), _p(dF))
    return F, dF


def sh_basis(deg, dirs):
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    K = (deg + 1) ** 2
    Y = np.empty((dirs.shape[0], K))
    dY = np.empty((dirs.shape[0], K, 3))
    lib().orc_sh_basis(ctypes.c_int(deg), ctypes.c_int(dirs.shape[0]), _p(dirs), _p(Y), _p(dY))
    return Y, dY


def project(splats, cam, kparams, tile=16, geom32=True):
    """Per-splat preprocessing.  Returns a dict of numpy arrays."""
    n = splats.n
    out = dict(
        culled=np.empty(n, np.int32), radius=np.empty(n, np.int32), rect=np.empty((n, 4), np.int32),
        tiles=np.empty(n, np.int32), depth=np.empty(n, np.float32), clampxy=np.empty((n, 2), np.int32),
        mean2d=np.empty((n, 2)), conic=np.empty((n, 3)), rgb=np.empty((n, 3)), clamped=np.empty(n, np.uint8))
    c = camera_struct(cam)
    r = lib().orc_project(ctypes.c_int(n), _p(splats.means), _p(splats.scales), _p(splats.quats),
                          _p(splats.sh), ctypes.c_int(splats.sh_degree), ctypes.byref(c),
                          ctypes.byref(kparams), ctypes.c_int(tile), ctypes.c_int(int(geom32)),
                          _p(out["culled"]), _p(out["radius"]), _p(out["rect"]), _p(out["tiles"]),
                          _p(out["depth"]), _p(out["clampxy"]), _p(out["mean2d"]), _p(out["conic"]),
                          _p(out["rgb"]), _p(out["clamped"]))
    if r != 0:
        raise ValueError("orc_project rejected its arguments")
    out["geom32"] = bool(geom32)
    out["opac"] = np.ascontiguousarray(splats.opacities, np.float32)
    out["q_max"] = float(kparams.q_max)
    return out


def build_lists(proj, cam, tile=16, tile_mask=None):
    """Sorted (tile, depth, id) instances over every splat's member tiles (the ellipse's row
    spans).  Returns keys u64[M], ids i32[M], ranges i32[tiles,2]."""
    tx, ty = tiles_xy(cam, tile)
    n = proj["culled"].shape[0]
    mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8).reshape(-1)
    L = lib()
    args = (ctypes.c_int(n), _p(proj["culled"]), _p(proj["rect"]), _p(proj["depth"]), _p(proj["mean2d"]),
            _p(proj["conic"]), ctypes.c_float(proj["q_max"]), ctypes.c_int(int(proj["geom32"])), ctypes.c_int(tile),
            ctypes.c_int(cam.width), ctypes.c_int(cam.height), ctypes.c_int(tx), ctypes.c_int(ty), _p(mask))
    M = L.orc_build_lists(*args, None, None, ctypes.c_longlong(0), None)
    keys = np.empty(max(M, 1), np.uint64)
    ids = np.empty(max(M, 1), np.int32)
    ranges = np.zeros((tx * ty, 2), np.int32)
    M2 = L.orc_build_lists(*args, _p(keys), _p(ids), ctypes.c_longlong(M), _p(ranges))
    if M2 != M:
        raise RuntimeError("orc_build_lists failed")
    return dict(keys=keys[:M], ids=ids[:M], ranges=ranges, M=int(M))


def render(proj, cam, kparams, tile=16, mode="tiled", lists=None, tile_mask=None,
           eps_alpha=EPS_ALPHA, eps_T=EPS_T, max_branch=3, alts_cap=1 << 16):
    """Front-to-back composite.  mode: 'tiled' or 'brute'.

    Returns image [3,H,W] (f64), T [H,W], count [H,W], last_id [H,W] (-1 if none),
    amb [H,W] (0 unique, 1 several outcomes enumerated, 2 unverifiable),
    sig [H,W] (hash of the blended id sequence) and alts (list of the other
    outcomes of ambiguous pixels: pixel, count, last_id, T, C).
    """
    W, H = cam.width, cam.height
    mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8).reshape(-1)
    if mode == "tiled" and lists is None:
        lists = build_lists(proj, cam, tile, mask)
    image = np.zeros((3, H, W))
    T = np.ones((H, W))
    count = np.zeros((H, W), np.int32)
    last = np.full((H, W), -1, np.int32)
    amb = np.zeros((H, W), np.int32)
    sig = np.zeros((H, W), np.uint64)
    alts = (OrcOutcome * alts_cap)()
    nalts = ctypes.c_int(0)
    c = camera_struct(cam)
    ids = lists["ids"] if mode == "tiled" else None
    ranges = lists["ranges"] if mode == "tiled" else None
    n = proj["culled"].shape[0]
    r = lib().orc_render(
        ctypes.c_int(n), _p(proj["culled"]), _p(proj["rect"]), _p(proj["depth"]), _p(proj["mean2d"]),
        _p(proj["conic"]), _p(proj["opac"]), _p(proj["rgb"]), ctypes.c_int(int(proj["geom32"])),
        ctypes.byref(c), ctypes.byref(kparams), ctypes.c_int(tile), ctypes.c_int(1 if mode == "tiled" else 0),
        _p(ids), _p(ranges), _p(mask), ctypes.c_double(eps_alpha), ctypes.c_double(eps_T),
        ctypes.c_int(max_branch), _p(image), _p(T), _p(count), _p(last), _p(amb), _p(sig),
        alts, ctypes.c_int(alts_cap), ctypes.byref(nalts))
    if r != 0:
        raise RuntimeError("orc_render failed")
    k = min(nalts.value, alts_cap)
    alt_list = [dict(pixel=alts[i].pixel, count=alts[i].count, last_id=alts[i].last_id, T=alts[i].T,
                     C=tuple(alts[i].C)) for i in range(k)]
    return dict(image=image, T=T, count=count, last_id=last, amb=amb, sig=sig, alts=alt_list,
                alts_overflow=nalts.value > alts_cap, lists=lists)


def render_backward(proj, cam, kparams, lists, dL_dimage, tile=16, tile_mask=None):
    """Gradient of the composite w.r.t. per-splat (mu'x, mu'y, A, B, C, opacity, r, g, b)."""
    n = proj["culled"].shape[0]
    grad2d = np.zeros((n, 9))
    dl = np.ascontiguousarray(dL_dimage, np.float64)
    mask = None if tile_mask is None else np.ascontiguousarray(tile_mask, np.uint8).reshape(-1)
    c = camera_struct(cam)
    r = lib().orc_render_backward(
        ctypes.c_int(n), _p(proj["rect"]), _p(proj["mean2d"]), _p(proj["conic"]), _p(proj["opac"]),
        _p(proj["rgb"]), ctypes.c_int(int(proj["geom32"])), ctypes.byref(c), ctypes.byref(kparams),
        ctypes.c_int(tile), _p(lists["ids"]), _p(lists["ranges"]), ctypes.c_longlong(lists["M"]), _p(mask),
        _p(dl), _p(grad2d))
    if r != 0:
        raise RuntimeError("orc_render_backward failed")
    return grad2d


def project_backward(splats, proj, cam, kparams, grad2d):
    """Chain the per-splat 2D gradients back to means, scales, quats, opacities and SH."""
    n = splats.n
    K = (splats.sh_degree + 1) ** 2
    out = dict(means=np.empty((n, 3)), scales=np.empty((n, 3)), quats=np.empty((n, 4)),
               opacities=np.empty(n), sh=np.empty((n, K, 3)))
    g = np.ascontiguousarray(grad2d, np.float64)
    c = camera_struct(cam)
    lib().orc_project_backward(
        ctypes.c_int(n), _p(splats.means), _p(splats.scales), _p(splats.quats), _p(splats.sh),
        ctypes.c_int(splats.sh_degree), ctypes.byref(c), ctypes.byref(kparams), _p(proj["culled"]),
        _p(proj["clampxy"]), _p(proj["clamped"]), _p(g), _p(out["means"]), _p(out["scales"]),
        _p(out["quats"]), _p(out["opacities"]), _p(out["sh"]))
    return out


def forward(splats, cam, kernel="half_cosine", tile=16, mode="tiled", geom32=True, tile_mask=None, **kw):
    kp = kernel_params(kernel) if isinstance(kernel, (str, int)) else kernel
    proj = project(splats, cam, kp, tile, geom32)
    lists = build_lists(proj, cam, tile, tile_mask) if mode == "tiled" else None
    out = render(proj, cam, kp, tile, mode, lists, tile_mask, **kw)
    out["proj"] = proj
    return out


def gradients(splats, cam, dL_dimage, kernel="half_cosine", tile=16, geom32=True, tile_mask=None):
    """Forward (tiled) + analytic backward.  Returns (forward dict, grad2d, param grads)."""
    kp = kernel_params(kernel) if isinstance(kernel, (str, int)) else kernel
    fwd = forward(splats, cam, kp, tile, "tiled", geom32, tile_mask)
    g2 = render_backward(fwd["proj"], cam, kp, fwd["lists"], dL_dimage, tile, tile_mask)
    gp = project_backward(splats, fwd["proj"], cam, kp, g2)
    return fwd, g2, gp


# ---------------------------------------------------------------------------
# Training-step terms in plain NumPy FP64.

def l1_loss(image, target):
    """L1 term of the loss (Sec. 4.2): mean |image - target| and its gradient sign(.)/count."""
    d = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    return np.abs(d).mean(), np.sign(d) / d.size


# The paper's image loss (Sec. 4.2): L = (1 - lambda) L1 + lambda L_D-SSIM, the two terms of
# the 3DGS work it builds on.  The paper gives neither lambda nor the SSIM window; they are taken
# from that work: lambda = 0.2, D-SSIM = 1 - SSIM, SSIM per channel with an 11 x 11 Gaussian
# window (sigma 1.5, normalised), zero padding outside the image, C1 = 0.01^2, C2 = 0.03^2 for
# intensities in [0, 1], averaged over channels and pixels.
SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2
SSIM_RADIUS = 5
SSIM_SIGMA = 1.5


def ssim_window():
    """The 1-D window g[-5..5] = exp(-k^2 / (2 sigma^2)), normalised to sum 1; the 2-D window is
    its outer product."""
    k = np.arange(-SSIM_RADIUS, SSIM_RADIUS + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * SSIM_SIGMA ** 2))
    return g / g.sum()


def _blur(a):
    """Window-weighted local mean of a [C, H, W] array, zero outside the image: a plain loop over
    the 11 x 11 offsets (the window is symmetric, so this equals its own adjoint)."""
    g = ssim_window()
    C, H, W = a.shape
    R = SSIM_RADIUS
    pad = np.zeros((C, H + 2 * R, W + 2 * R))
    pad[:, R:R + H, R:R + W] = a
    out = np.zeros((C, H, W))
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            out += g[dy + R] * g[dx + R] * pad[:, R + dy:R + dy + H, R + dx:R + dx + W]
    return out


def ssim_map(image, target):
    """SSIM at every channel and pixel (Wang et al. 2004, the form 3DGS trains with)."""
    x = np.asarray(image, np.float64)
    y = np.asarray(target, np.float64)
    mx, my = _blur(x), _blur(y)
    vx = _blur(x * x) - mx * mx
    vy = _blur(y * y) - my * my
    cxy = _blur(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * cxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (vx + vy + SSIM_C2))


def l1_dssim_loss(image, target, lam=0.2):
    """(1 - lam) mean|x - y| + lam (1 - mean SSIM(x, y)) and its gradient w.r.t. x.

    With the local moments m_x = G*x, m_y = G*y, s_xx = G*x^2, s_xy = G*xy and
    A1 = 2 m_x m_y + C1, A2 = 2 (s_xy - m_x m_y) + C2, B1 = m_x^2 + m_y^2 + C1,
    B2 = s_xx - m_x^2 + s_yy - m_y^2 + C2, SSIM = A1 A2 / (B1 B2) has
      dSSIM/dm_x  = 2 m_y (A2 - A1) / (B1 B2) - 2 m_x SSIM (1/B1 - 1/B2)
      dSSIM/ds_xx = -SSIM / B2
      dSSIM/ds_xy = 2 A1 / (B1 B2)
    and, the window being symmetric, d(mean SSIM)/dx = (G*dm + 2 x G*ds_xx + y G*ds_xy) / N."""
    x = np.asarray(image, np.float64)
    y = np.asarray(target, np.float64)
    N = x.size
    mx, my = _blur(x), _blur(y)
    sxx, syy, sxy = _blur(x * x), _blur(y * y), _blur(x * y)
    A1 = 2 * mx * my + SSIM_C1
    A2 = 2 * (sxy - mx * my) + SSIM_C2
    B1 = mx * mx + my * my + SSIM_C1
    B2 = (sxx - mx * mx) + (syy - my * my) + SSIM_C2
    ssim = A1 * A2 / (B1 * B2)
    d_m = 2 * my * (A2 - A1) / (B1 * B2) - 2 * mx * ssim * (1 / B1 - 1 / B2)
    d_sxx = -ssim / B2
    d_sxy = 2 * A1 / (B1 * B2)
    dssim_dx = (_blur(d_m) + 2 * x * _blur(d_sxx) + y * _blur(d_sxy)) / N
    l1, dl1 = l1_loss(x, y)
    loss = (1 - lam) * l1 + lam * (1 - ssim.mean())
    return loss, (1 - lam) * dl1 - lam * dssim_dx, ssim.mean()


# Adaptive density control.  The paper keeps the optimisation pipeline of 3DGS (Sec. 4 block
# diagram), whose density control is restated here: per training step, statistics of every
# visible splat; every few hundred steps, clone, split and prune.  Decisions are taken in float32
# with the same operations as the GPU (the rules require both sides to decide in one precision).

def densify_stats(grad2d, radius, width, height, accum, count, max_radius):
    """One step's statistics: the norm of the view-space mean gradient in normalised device
    units (pixel gradient x (W/2, H/2)) added to accum, 1 added to count, and the largest
    screen radius kept, for every visible splat (radius > 0).  float32, in place."""
    f = np.float32
    vis = np.asarray(radius) > 0
    gx = np.asarray(grad2d[:, 0], f) * f(0.5 * width)
    gy = np.asarray(grad2d[:, 1], f) * f(0.5 * height)
    norm = np.sqrt(gx * gx + gy * gy).astype(f)
    accum[vis] = (accum[vis] + norm[vis]).astype(f)
    count[vis] = (count[vis] + f(1.0)).astype(f)
    max_radius[vis] = np.maximum(max_radius[vis], np.asarray(radius)[vis])


def densify_actions(scales, opacities, accum, count, max_radius, cfg):
    """Per splat: (grow, split, keep) booleans.  avg = accum / count (0 unseen);
    grow = avg >= grad_threshold; clone if grow and max scale <= dense_scale, split if grow and
    max scale > dense_scale; a splat that is split is replaced by its children; any splat is
    pruned (not kept) if opacity < min_opacity, or its max screen radius > max_screen_radius
    (when > 0), or its max scale > max_world_scale (when > 0)."""
    f = np.float32
    cnt = np.asarray(count, f)
    avg = np.where(cnt > 0, np.asarray(accum, f) / np.where(cnt > 0, cnt, f(1)), f(0)).astype(f)
    smax = np.max(np.asarray(scales, f), axis=1)
    grow = avg >= f(cfg["grad_threshold"])
    split = grow & (smax > f(cfg["dense_scale"]))
    clone = grow & ~split
    keep = _survives(np.asarray(opacities, f), smax, np.asarray(max_radius), cfg)
    return clone, split, keep


def _survives(opac, smax, radius, cfg):
    f = np.float32
    ok = opac >= f(cfg["min_opacity"])
    if cfg["max_screen_radius"] > 0:
        ok &= np.asarray(radius, f) <= f(cfg["max_screen_radius"])
    if cfg["max_world_scale"] > 0:
        ok &= smax <= f(cfg["max_world_scale"])
    return ok


def densify(raw, act, state, accum, count, max_radius, normals, cfg):
    """One density-control pass.  raw: dict means, log_scales, quats, opacity_logits, sh;
    act: dict scales, opacities (activated copies); state: dict of Adam moments m_/v_ + the raw
    names; normals: [n, 2, 3] standard normal draws for the split children.
    Output order: surviving originals in index order, then clones in parent order, then split
    children (two per parent, in parent order).  Originals keep their moments; clones and
    children start from zero moments.  A clone carries its parent's statistics for the prune
    test except the screen radius, which starts at 0 (it has not been rendered); so do
    children, whose scales are the parent's / split_scale_div and whose means are
    parent + R(q) (s * z), s the parent's scales, R the rotation of the normalised quaternion.
    Returns (raw', act', state', n_out)."""
    f = np.float32
    n = raw["means"].shape[0]
    clone, split, keep = densify_actions(act["scales"], act["opacities"], accum, count, max_radius, cfg)
    surv = keep & ~split
    smax = np.max(np.asarray(act["scales"], f), axis=1)
    zero_r = np.zeros(n, np.int32)
    opac = np.asarray(act["opacities"], f)
    clone_kept = clone & _survives(opac, smax, zero_r, cfg)
    div = f(cfg["split_scale_div"])
    child_smax = np.max(np.asarray(act["scales"], f) / div, axis=1).astype(f)
    child_kept = split & _survives(opac, child_smax, zero_r, cfg)
    sel_s, sel_c, sel_p = np.flatnonzero(surv), np.flatnonzero(clone_kept), np.flatnonzero(child_kept)
    q = np.asarray(raw["quats"], np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    sc = np.asarray(act["scales"], np.float64)
    out_raw, out_act, out_state = {}, {}, {}
    log_div = f(np.log(np.float64(div)))
    for k, v in raw.items():
        v = np.asarray(v)
        if k == "means":
            kids = []
            for j in range(2):
                off = np.einsum("nab,nb->na", R[sel_p], sc[sel_p] * np.asarray(normals, np.float64)[sel_p, j])
                kids.append(v[sel_p].astype(np.float64) + off)
            children = np.stack(kids, 1).reshape(-1, 3)
        elif k == "log_scales":
            children = np.repeat((v[sel_p].astype(f) - log_div).astype(f), 2, axis=0)
        else:
            children = np.repeat(v[sel_p], 2, axis=0)
        out_raw[k] = np.concatenate([v[sel_s], v[sel_c], children.astype(v.dtype) if k != "means" else children])
    out_act["scales"] = np.exp(np.asarray(out_raw["log_scales"], np.float64))
    out_act["opacities"] = 1.0 / (1.0 + np.exp(-np.asarray(out_raw["opacity_logits"], np.float64)))
    for k, v in state.items():
        v = np.asarray(v)
        new = np.zeros((len(sel_c) + 2 * len(sel_p),) + v.shape[1:], v.dtype)
        out_state[k] = np.concatenate([v[sel_s], new])
    return out_raw, out_act, out_state, len(sel_s) + len(sel_c) + 2 * len(sel_p)


def reset_opacity(opacity_logits, max_opacity=0.01):
    """Opacity reset: every opacity above max_opacity is set to it (logits clamped)."""
    f = np.float32
    cap = f(np.log(np.float64(max_opacity) / (1.0 - np.float64(max_opacity))))
    return np.minimum(np.asarray(opacity_logits, f), cap)


def adam_update(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step (Kingma & Ba, Algorithm 1) on float64 copies; returns (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def adam_step_splats(raw, grads, state, lrs, step, beta1=0.9, beta2=0.999, eps=1e-15):
    """Adam on the raw 3DGS parameters.  raw: dict means, log_scales, quats, opacity_logits, sh;
    grads: dict w.r.t. the activated values (means, scales, quats, opacities, sh); the chain
    through exp (scales) and the sigmoid (opacities) is applied here.  lrs: dict with keys
    means, scales, quats, opacities, sh_dc, sh_rest.  Returns (raw', state')."""
    scales = np.exp(np.asarray(raw["log_scales"], np.float64))
    opac = 1.0 / (1.0 + np.exp(-np.asarray(raw["opacity_logits"], np.float64)))
    g_raw = dict(means=grads["means"], log_scales=np.asarray(grads["scales"]) * scales,
                 quats=grads["quats"], opacity_logits=np.asarray(grads["opacities"]) * opac * (1 - opac),
                 sh=grads["sh"])
    lr_of = dict(means=lrs["means"], log_scales=lrs["scales"], quats=lrs["quats"], opacity_logits=lrs["opacities"])
    out, new_state = {}, {}
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        out[k], m, v = adam_update(raw[k], g_raw[k], state["m_" + k], state["v_" + k], lr_of[k], step, beta1, beta2, eps)
        new_state["m_" + k], new_state["v_" + k] = m, v
    sh = np.asarray(raw["sh"], np.float64)
    lr_sh = np.full(sh.shape, lrs["sh_rest"])
    lr_sh[:, 0, :] = lrs["sh_dc"]
    out["sh"], new_state["m_sh"], new_state["v_sh"] = adam_update(sh, g_raw["sh"], state["m_sh"], state["v_sh"],
                                                                  lr_sh, step, beta1, beta2, eps)
    return out, new_state
