"""CUDA path (through the C ABI) against the CPU oracle, element by element."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2501_12369_gb300 import darb, synth

from gpu_helpers import (ambiguity_masked_grad, check_lists, check_preprocess, check_render, check_tile_runs,
                         gpu_forward, grad_close, to_np)

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

KERNELS = oracle.KERNEL_NAMES


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()
    oracle.build()


def _medium_scene(n=20000, seed=5, deg=3):
    s = synth.cluster_scene(n, seed=seed, sh_degree=deg)
    cam = synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[3]  # ragged: 333x207 is no multiple of any tile
    return s, cam


# --------------------------------------------------------------------------- step 1

@pytest.mark.parametrize("kernel", KERNELS)
def test_preprocess_is_bit_exact_small(kernel):
    s, cam = synth.small_forward_workload()
    r, sd, proj, bins, img = gpu_forward(s, cam, kernel, 16)
    check_preprocess(proj, oracle.project(s, cam, oracle.kernel_params(kernel), 16, True))


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_preprocess_is_bit_exact_clusters(deg):
    s, cam = _medium_scene(deg=deg)
    s.quats *= np.float32(1.7)  # unnormalised quaternions are normalised inside
    for kernel in ("half_cosine", "raised_cosine"):
        r, sd, proj, bins, img = gpu_forward(s, cam, kernel, 16)
        check_preprocess(proj, oracle.project(s, cam, oracle.kernel_params(kernel), 16, True))


# --------------------------------------------------------------------------- steps 2-3

@pytest.mark.parametrize("strategy", [darb.DARB_SORT_DEPTH_THEN_TILE, darb.DARB_SORT_KEYS64])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bin_sort_is_bit_exact(tile, strategy):
    s, cam = _medium_scene()
    s.means[::50] = s.means[7]  # coincident splats: equal keys must keep splat order
    s.means[1::97, 2] = s.means[5, 2]  # equal depths across different tiles
    r = darb.Rasterizer(cam, "half_cosine", tile, strategy=strategy)
    proj, bins, img = r.forward(darb.splats_to_device(s))
    torch.cuda.synchronize()
    ref = oracle.project(s, cam, oracle.kernel_params("half_cosine"), tile, True)
    lists = oracle.build_lists(ref, cam, tile)
    check_lists(bins, lists)
    packed, unpacked = check_tile_runs(proj, ref, lists, (cam.width + tile - 1) // tile)
    assert packed > 0 and (tile > 8 or unpacked > 0)  # both the packed and the warp-wide rows


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_large_elongated_and_border_splats(tile):
    """Rectangles taller than a warp's worth of tile rows (their runs recomputed warp-wide by the
    tile counts and per thread by the duplication), rectangles too large to pack, and elongated
    splats around the image border, whose rectangle may reach into the image while their
    ellipse reaches no tile (culled on both sides)."""
    cam = synth.pinhole((0.0, 0.0, 3.0), 320, 296, 300.0, bg=(0.1, 0.2, 0.3))
    big = synth.uniform_cube_scene(24, seed=11, log_scale=(-1.2, -0.6))
    thin = synth.uniform_cube_scene(600, seed=12, half=1.6, log_scale=(-5.0, -1.5))
    s = synth.Splats(*(np.concatenate([getattr(big, f), getattr(thin, f)])
                       for f in ("means", "scales", "quats", "opacities", "sh")), big.sh_degree)
    r, sd, proj, bins, img = gpu_forward(s, cam, "half_cosine", tile)
    ref = oracle.project(s, cam, oracle.kernel_params("half_cosine"), tile, True)
    check_preprocess(proj, ref)
    lists = oracle.build_lists(ref, cam, tile)
    check_lists(bins, lists)
    packed, unpacked = check_tile_runs(proj, ref, lists, (cam.width + tile - 1) // tile)
    assert packed > 0 and unpacked > 0
    vis = ref["culled"] == 0
    rows = ref["rect"][vis, 3] - ref["rect"][vis, 1] + 1
    if tile == 8:
        assert rows.max() > 32  # a rectangle taller than one warp of tile rows
    check_render(img, bins, oracle.forward(s, cam, "half_cosine", tile=tile), cam, tile)


def test_run_table_overflow_falls_back_to_recomputed_runs():
    """A copy of the library built with a 64-entry run table: the unpacked splats that no
    longer fit are marked and their runs recomputed by the duplication.  The lists must still
    equal the oracle's (the scene and tiles of the elongated-splat test, 8-pixel tiles)."""
    import ctypes
    from paper_2501_12369_gb300 import build
    path = build.build_variant("small_run_table", ["-DDARB_RUN_TABLE_MAX=64"])
    L = ctypes.CDLL(path)
    for name, (res, args) in darb.SIGNATURES.items():
        getattr(L, name).restype, getattr(L, name).argtypes = res, args
    cam = synth.pinhole((0.0, 0.0, 3.0), 320, 296, 300.0, bg=(0.1, 0.2, 0.3))
    big = synth.uniform_cube_scene(24, seed=11, log_scale=(-1.2, -0.6))
    thin = synth.uniform_cube_scene(600, seed=12, half=1.6, log_scale=(-5.0, -1.5))
    s = synth.Splats(*(np.concatenate([getattr(big, f), getattr(thin, f)])
                       for f in ("means", "scales", "quats", "opacities", "sh")), big.sh_degree)
    tile = 8
    saved = darb._lib
    try:
        darb._lib = L
        r, sd, proj, bins, img = gpu_forward(s, cam, "half_cosine", tile)
    finally:
        darb._lib = saved
    ref = oracle.project(s, cam, oracle.kernel_params("half_cosine"), tile, True)
    vis = ref["culled"] == 0
    rows = ref["rect"][vis, 3] - ref["rect"][vis, 1] + 1
    cols = ref["rect"][vis, 2] - ref["rect"][vis, 0] + 1
    assert rows[(rows > 8) | (cols > 15)].sum() > 64  # more unpacked rows than the table holds
    check_lists(bins, oracle.build_lists(ref, cam, tile))
    check_render(img, bins, oracle.forward(s, cam, "half_cosine", tile=tile), cam, tile)


def test_bin_sort_strategies_agree_on_a_large_scene():
    s = synth.cluster_scene(300_000, seed=11)
    cam = synth.fibonacci_cameras(10, 6.0, 1280, 720, 1000.0)[4]
    out = []
    for strategy in (darb.DARB_SORT_DEPTH_THEN_TILE, darb.DARB_SORT_KEYS64):
        r = darb.Rasterizer(cam, "gaussian", 16, strategy=strategy)
        proj, bins, img = r.forward(darb.splats_to_device(s))
        torch.cuda.synchronize()
        M = bins.M
        out.append((M, to_np(bins.keys)[:M].copy(), to_np(bins.values)[:M].copy(), to_np(bins.ranges).copy(),
                    to_np(img.image).copy()))
    a, b = out
    assert a[0] == b[0] and a[0] > 1_000_000
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


def test_bin_sort_async_capacity_mode_matches_sync():
    s, cam = _medium_scene()
    kp = darb.darb_kernel_defaults("half_cosine")
    sd = darb.splats_to_device(s)
    proj = darb.darb_preprocess(sd, cam, kp, 16)
    cap = 400000
    ws = torch.empty(darb.darb_bin_sort_workspace_size(s.n, 16, cam, cap), dtype=torch.uint8, device="cuda")
    a = darb.darb_bin_sort(proj, s.n, 16, cam, ws, cap, sync=True)
    M = a.M
    assert M > 0
    ka, va, ra = to_np(a.keys)[:M].copy(), to_np(a.values)[:M].copy(), to_np(a.ranges).copy()
    b = darb.darb_bin_sort(proj, s.n, 16, cam, ws, cap, sync=False)
    torch.cuda.synchronize()
    assert int(to_np(b.num_instances)[0]) == M and int(to_np(b.status)[0]) == 0
    assert np.array_equal(to_np(b.keys)[:M], ka) and np.array_equal(to_np(b.values)[:M], va)
    assert np.array_equal(to_np(b.ranges), ra)


def test_bin_sort_reports_capacity_overflow():
    s, cam = synth.small_forward_workload()
    kp = darb.darb_kernel_defaults("half_cosine")
    sd = darb.splats_to_device(s)
    proj = darb.darb_preprocess(sd, cam, kp, 16)
    cap = 100
    ws = torch.empty(darb.darb_bin_sort_workspace_size(s.n, 16, cam, cap), dtype=torch.uint8, device="cuda")
    with pytest.raises(darb.DarbError) as e:
        darb.darb_bin_sort(proj, s.n, 16, cam, ws, cap, sync=True)
    assert e.value.status == 3
    b = darb.darb_bin_sort(proj, s.n, 16, cam, ws, cap, sync=False)  # async: flagged on the device
    torch.cuda.synchronize()
    assert int(to_np(b.status)[0]) == 3 and int(to_np(b.num_instances)[0]) > cap
    assert np.all(to_np(b.ranges) == 0)  # nothing to composite after an overflow
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(darb.DarbError) as e:
        darb.darb_bin_sort(proj, s.n, 16, cam, small, cap)
    assert e.value.status == 2


# --------------------------------------------------------------------------- step 4

@pytest.mark.parametrize("kernel", KERNELS)
def test_render_forward_small(kernel):
    s, cam = synth.small_forward_workload()
    r, sd, proj, bins, img = gpu_forward(s, cam, kernel, 16)
    ref = oracle.forward(s, cam, kernel, tile=16, mode="brute")
    n, namb, nunv = check_render(img, bins, ref, cam, 16)
    assert n > 3900


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_render_forward_clusters(kernel, tile):
    s, cam = _medium_scene()
    cam = dataclasses.replace(cam, bg=(0.2, 0.4, 0.6))
    r, sd, proj, bins, img = gpu_forward(s, cam, kernel, tile)
    ref = oracle.forward(s, cam, kernel, tile=tile)
    check_render(img, bins, ref, cam, tile)


# --------------------------------------------------------------------------- backward

def _grads(s, cam, kernel, tile, dl_seed=3):
    r, sd, proj, bins, img = gpu_forward(s, cam, kernel, tile)
    dl = synth.random_image_grad(cam.height, cam.width, seed=dl_seed)
    ref_f = oracle.forward(s, cam, kernel, tile=tile)
    dl = ambiguity_masked_grad(dl, ref_f["amb"])
    dL = torch.from_numpy(dl.astype(np.float32)).cuda()
    g, g2 = r.backward(sd, proj, bins, img, dL)
    torch.cuda.synchronize()
    _, g2_ref, gp_ref = oracle.gradients(s, cam, dl.astype(np.float32).astype(np.float64), kernel, tile=tile)
    return g, g2, g2_ref, gp_ref, sd, proj, r


G2_NAMES = ["dmean_x", "dmean_y", "dA", "dB", "dC", "dopacity", "dr", "dg", "db"]


@pytest.mark.parametrize("kernel", KERNELS)
def test_render_backward_matches_oracle(kernel):
    s, cam = synth.small_forward_workload()
    g, g2, g2_ref, gp_ref, *_ = _grads(s, cam, kernel, 16)
    g2 = to_np(g2)
    assert np.all(g2[:, 9:] == 0)
    for j, name in enumerate(G2_NAMES):
        grad_close(f"{kernel}/{name}", g2[:, j], g2_ref[:, j])


@pytest.mark.parametrize("kernel", KERNELS)
def test_preprocess_backward_matches_oracle(kernel):
    """The per-splat chain alone: the oracle's own grad2d fed to the GPU's preprocess backward."""
    s, cam = _medium_scene(n=5000)
    r, sd, proj, bins, img = gpu_forward(s, cam, kernel, 16)
    ref = oracle.project(s, cam, oracle.kernel_params(kernel), 16, True)
    rng = np.random.default_rng(0)
    g2 = rng.normal(size=(s.n, 9))
    g2[ref["culled"] == 1] = 0.0
    g2_12 = np.zeros((s.n, 12), np.float32)
    g2_12[:, :9] = g2
    out = darb.darb_preprocess_bwd(sd, cam, r.kparams, proj, torch.from_numpy(g2_12).cuda())
    torch.cuda.synchronize()
    gp = oracle.project_backward(s, ref, cam, oracle.kernel_params(kernel), g2_12[:, :9].astype(np.float64))
    for name, got in (("means", out.dmeans), ("scales", out.dscales), ("quats", out.dquats),
                      ("opacities", out.dopacities), ("sh", out.dsh)):
        grad_close(f"{kernel}/{name}", to_np(got), gp[name])


@pytest.mark.parametrize("kernel", KERNELS)
def test_full_gradient_matches_oracle(kernel):
    s, cam = _medium_scene(n=8000)
    g, g2, g2_ref, gp_ref, *_ = _grads(s, cam, kernel, 16)
    for name, got in (("means", g.dmeans), ("scales", g.dscales), ("quats", g.dquats),
                      ("opacities", g.dopacities), ("sh", g.dsh)):
        grad_close(f"{kernel}/{name}", to_np(got), gp_ref[name])


def test_gradients_on_the_256_splat_32x32_subset():
    """The finite-difference subset of the 500k / 720p scene: the 256 splats projecting nearest
    the image centre, seen through a 32x32 crop.  GPU gradient against the oracle's analytic
    gradient (which the CPU suite checks against central differences)."""
    s, cam = synth.scene_500k_720p()
    kp = oracle.kernel_params("half_cosine")
    p = oracle.project(s, cam, kp, 16, True)
    vis = np.flatnonzero(p["culled"] == 0)
    d = np.linalg.norm(p["mean2d"][vis] - [cam.cx, cam.cy], axis=1)
    sub = s.subset(np.sort(vis[np.argsort(d)[:256]]))
    crop = synth.crop_camera(cam, int(cam.cx) - 16, int(cam.cy) - 16, 32, 32)
    for kernel in ("gaussian", "half_cosine"):
        g, g2, g2_ref, gp_ref, *_ = _grads(sub, crop, kernel, 16)
        for name, got in (("means", g.dmeans), ("scales", g.dscales), ("quats", g.dquats),
                          ("opacities", g.dopacities), ("sh", g.dsh)):
            grad_close(f"{kernel}/{name}", to_np(got), gp_ref[name])


# --------------------------------------------------------------------------- edge cases

def test_empty_and_fully_culled_scenes():
    cam = synth.pinhole((0.0, 0.0, 4.0), 48, 40, 50.0, bg=(0.3, 0.2, 0.1))
    s = synth.uniform_cube_scene(500, seed=1)
    s.means[:, 2] += 10.0  # every splat behind the camera
    for scene in (s, s.subset(np.arange(0))):
        r, sd, proj, bins, img = gpu_forward(scene, cam, "half_cosine", 16)
        assert bins.M == 0
        im = to_np(img.image)
        assert np.allclose(im, np.array(cam.bg)[:, None, None]) and np.all(to_np(img.n_contrib) == 0)
        assert np.all(to_np(img.t_final) == 1.0)


@pytest.mark.parametrize("n", [2047, 2048, 2049, 6145])
@pytest.mark.parametrize("pattern", ["all", "last_block", "first_splat", "odd_blocks"])
def test_bin_sort_at_scan_block_boundaries(n, pattern):
    """The sort's scans run over blocks of 2048 splats (visible count and compaction) and of
    2048 depth-ordered positions (instance offsets), each block taking its offset from the blocks
    before it.  Lists against the oracle when the visible splats sit only in the last block, only
    at splat 0, or in every other block (whole blocks contributing nothing), around one and three
    block boundaries."""
    cam = synth.pinhole((0.0, 0.0, 4.0), 64, 48, 60.0)
    s = synth.uniform_cube_scene(n, seed=n % 97)
    behind = np.ones(n, dtype=bool)
    if pattern == "all":
        behind[:] = False
    elif pattern == "last_block":
        behind[(n - 1) // 2048 * 2048:] = False
    elif pattern == "first_splat":
        behind[0] = False
    else:
        for b in range(0, n, 4096):
            behind[b:b + 2048] = False
    s.means[behind, 2] += 10.0  # behind the camera
    r, sd, proj, bins, img = gpu_forward(s, cam, "half_cosine", 16)
    ref = oracle.project(s, cam, oracle.kernel_params("half_cosine"), 16, True)
    assert int((ref["culled"] == 0).sum()) == int((to_np(proj.radius) != 0).sum()) > 0
    lists = oracle.build_lists(ref, cam, 16)
    assert bins.M == int(ref["tiles"][ref["culled"] == 0].sum())
    check_lists(bins, lists)


def test_single_splat_covering_the_image():
    cam = synth.pinhole((0.0, 0.0, 2.0), 100, 60, 80.0, bg=(0.0, 0.0, 0.0))
    s = synth.uniform_cube_scene(1, seed=2, log_scale=(-0.3, -0.2))
    s.means[:] = 0.0
    for kernel in KERNELS:
        r, sd, proj, bins, img = gpu_forward(s, cam, kernel, 16)
        ref_tiles = int(oracle.project(s, cam, oracle.kernel_params(kernel), 16, True)["tiles"].sum())
        assert bins.M == ref_tiles <= 7 * 4  # member tiles within the rectangle clamped to the 7 x 4 grid
        check_render(img, bins, oracle.forward(s, cam, kernel, tile=16), cam, 16)


def test_tiny_and_odd_images():
    s = synth.uniform_cube_scene(300, seed=9)
    for (w, h) in [(1, 1), (7, 3), (17, 33), (129, 65)]:
        cam = synth.pinhole((0.2, 0.1, 3.5), w, h, 0.8 * w + 4)
        for tile in (8, 16, 32):
            r, sd, proj, bins, img = gpu_forward(s, cam, "parabola", tile)
            check_render(img, bins, oracle.forward(s, cam, "parabola", tile=tile), cam, tile)


# --------------------------------------------------------------------------- full sizes

def _tile_pixel_mask(cam, tile, tiles):
    tx = (cam.width + tile - 1) // tile
    m = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        y0, x0 = (t // tx) * tile, (t % tx) * tile
        m[y0:y0 + tile, x0:x0 + tile] = True
    return m


def test_4k_view_with_8_pixel_tiles_on_sampled_tiles():
    """3840 x 2160 with 8-pixel tiles: 129,600 tiles (17 tile bits), so the tile sort takes three
    passes, and the tile counts and their setup run from global memory.  300k clustered splats;
    preprocess for every splat, lists and pixels on 32 sampled occupied tiles."""
    splats = synth.cluster_scene(300_000, seed=4)
    cam = synth.fibonacci_cameras(16, 6.0, 3840, 2160, 3000.0)[5]
    tile, kernel = 8, "half_cosine"
    r, sd, proj, bins, img = gpu_forward(splats, cam, kernel, tile)
    assert int(bins.status.item()) == 0
    kp = oracle.kernel_params(kernel)
    ref_p = oracle.project(splats, cam, kp, tile, True)
    check_preprocess(proj, ref_p)
    ranges = to_np(bins.ranges)
    assert ranges.shape[0] == 480 * 270
    occupied = np.flatnonzero(ranges[:, 1] > ranges[:, 0])
    tiles = np.sort(np.random.default_rng(11).choice(occupied, 32, replace=False))
    mask = np.zeros(ranges.shape[0], np.uint8)
    mask[tiles] = 1
    lists = oracle.build_lists(ref_p, cam, tile, mask)
    check_lists(bins, lists, mask)
    ref_f = oracle.render(ref_p, cam, kp, tile, "tiled", lists, mask)
    check_render(img, bins, ref_f, cam, tile, pixel_mask=_tile_pixel_mask(cam, tile, tiles))


@pytest.mark.parametrize("tile", [32, 8])
def test_full_size_training_view_on_sampled_tiles(tile):
    """3M splats, 1920x1080, half-cosine, default sort: with 32-pixel tiles the configuration the
    benchmark times (its autotuner picks 32), with 8-pixel tiles the sort's global-memory tile
    counts (the 1080p difference array is too large for shared memory).  Preprocess is compared
    for every splat; lists, pixels and gradients on a seeded sample of 24 occupied tiles (the
    upstream gradient is zero elsewhere, so every splat's gradient is exactly the contribution of
    those tiles on both sides)."""
    splats, cams = synth.scene_3m_1080p(num_cameras=100)
    cam, kernel = cams[0], "half_cosine"
    r, sd, proj, bins, img = gpu_forward(splats, cam, kernel, tile)
    kp = oracle.kernel_params(kernel)
    ref_p = oracle.project(splats, cam, kp, tile, True)
    check_preprocess(proj, ref_p)
    ranges = to_np(bins.ranges)
    occupied = np.flatnonzero(ranges[:, 1] > ranges[:, 0])
    rng = np.random.default_rng(7)
    tiles = np.sort(rng.choice(occupied, 24, replace=False))
    mask = np.zeros(ranges.shape[0], np.uint8)
    mask[tiles] = 1
    lists = oracle.build_lists(ref_p, cam, tile, mask)
    check_lists(bins, lists, mask)
    ref_f = oracle.render(ref_p, cam, kp, tile, "tiled", lists, mask)
    pmask = _tile_pixel_mask(cam, tile, tiles)
    check_render(img, bins, ref_f, cam, tile, pixel_mask=pmask)
    dl = synth.random_image_grad(cam.height, cam.width, seed=5)
    dl[:, ~pmask] = 0.0
    dl = ambiguity_masked_grad(dl, ref_f["amb"]).astype(np.float32)
    g, g2 = r.backward(sd, proj, bins, img, torch.from_numpy(dl).cuda())
    torch.cuda.synchronize()
    g2_ref = oracle.render_backward(ref_p, cam, kp, lists, dl.astype(np.float64), tile, mask)
    touched = np.flatnonzero(np.abs(g2_ref).sum(1) > 0)
    assert len(touched) > 100
    g2n = to_np(g2)
    for j, name in enumerate(G2_NAMES):
        grad_close(f"3M/{name}", g2n[:, j], g2_ref[:, j])
    gp_ref = oracle.project_backward(splats, ref_p, cam, kp, g2_ref)
    for name, got in (("means", g.dmeans), ("scales", g.dscales), ("quats", g.dquats),
                      ("opacities", g.dopacities), ("sh", g.dsh)):
        grad_close(f"3M/{name}", to_np(got), gp_ref[name])


def test_full_size_sort_strategies_agree_on_many_views():
    """At the benchmark's size the default sort runs its per-tile counts on a side stream beside
    the depth passes.  Over several views and repeated calls its lists must equal, bit for bit,
    those of the 64-bit-key strategy, which runs on one stream only: a race between the two
    streams (for instance over a buffer both read and write) would show as a difference."""
    splats, cams = synth.scene_3m_1080p(num_cameras=100)
    sd = darb.splats_to_device(splats)
    kp = darb.darb_kernel_defaults("half_cosine")
    tile, cap = 32, 30_000_000
    tx, ty = darb.darb_tile_grid(cams[0], tile)
    ws = {st: torch.empty(darb.darb_bin_sort_workspace_size(splats.n, tile, cams[0], cap, st), dtype=torch.uint8,
                          device="cuda") for st in (darb.DARB_SORT_DEPTH_THEN_TILE, darb.DARB_SORT_KEYS64)}
    a = darb.Binning.empty(cap, tx * ty, "cuda", keys=False)
    b = darb.Binning.empty(cap, tx * ty, "cuda")
    for c in (0, 13, 27, 41, 58, 77, 96):
        proj = darb.darb_preprocess(sd, cams[c], kp, tile)
        darb.darb_bin_sort(proj, splats.n, tile, cams[c], ws[darb.DARB_SORT_KEYS64], cap, b,
                           strategy=darb.DARB_SORT_KEYS64)
        M = b.M
        ref_v, ref_r = b.values[:M].clone(), b.ranges.clone()
        for _ in range(2):
            darb.darb_bin_sort(proj, splats.n, tile, cams[c], ws[darb.DARB_SORT_DEPTH_THEN_TILE], cap, a)
            assert a.M == M
            assert torch.equal(a.values[:M], ref_v), f"camera {c}: values differ"
            assert torch.equal(a.ranges, ref_r), f"camera {c}: ranges differ"


@pytest.mark.parametrize("kernel", ["gaussian", "half_cosine"])
def test_500k_720p_forward_and_backward_full_frame(kernel):
    s, cam = synth.scene_500k_720p()
    g, g2, g2_ref, gp_ref, *_ = _grads(s, cam, kernel, 16)
    for name, got in (("means", g.dmeans), ("scales", g.dscales), ("quats", g.dquats),
                      ("opacities", g.dopacities), ("sh", g.dsh)):
        grad_close(f"500k/{kernel}/{name}", to_np(got), gp_ref[name])
    r, sd, proj, bins, img = gpu_forward(s, cam, kernel, 16)
    check_render(img, bins, oracle.forward(s, cam, kernel, tile=16), cam, 16)
