"""Helpers for the GPU parity tests: run the CUDA path and compare it with the oracle."""
import numpy as np
import torch

import oracle
from paper_2501_12369_gb300 import darb

COLOUR_TOL = 1e-4  # absolute, per channel (FP32 path against the FP64 oracle)
GRAD_RTOL = 1e-3   # relative, per element ...
GRAD_ATOL = 1e-4   # ... plus this fraction of the largest magnitude in the parameter group


def to_np(t):
    return t.detach().cpu().numpy()


def gpu_forward(splats, cam, kernel, tile, capacity=None):
    r = darb.Rasterizer(cam, kernel, tile, capacity=capacity)
    s = darb.splats_to_device(splats)
    proj, bins, img = r.forward(s)
    torch.cuda.synchronize()
    return r, s, proj, bins, img


def f32_bits(a):
    return np.ascontiguousarray(np.asarray(a, np.float32)).view(np.uint32)


def check_preprocess(proj, ref):
    culled = ref["culled"].astype(bool)
    rad = to_np(proj.radius)
    assert np.array_equal(rad == 0, culled), "culling differs"
    vis = ~culled
    assert np.array_equal(rad[vis], ref["radius"][vis]), "radius differs"
    assert np.array_equal(to_np(proj.tile_rect)[vis], ref["rect"][vis]), "tile rectangle differs"
    assert np.array_equal(to_np(proj.tiles_touched)[vis].astype(np.int64), ref["tiles"][vis]), "tiles differ"
    assert np.array_equal(f32_bits(to_np(proj.depth)[vis]), f32_bits(ref["depth"][vis])), "depth bits differ"
    assert np.array_equal(f32_bits(to_np(proj.mean2d)[vis]), f32_bits(ref["mean2d"][vis])), "mean2d bits differ"
    co = to_np(proj.conic_o)
    assert np.array_equal(f32_bits(co[vis, :3]), f32_bits(ref["conic"][vis])), "conic bits differ"
    assert np.array_equal(co[vis, 3], ref["opac"][vis]), "opacity differs"
    rgb = to_np(proj.rgb)
    assert np.abs(rgb[vis] - ref["rgb"][vis]).max(initial=0.0) <= 1e-5, "SH colour differs"
    cl = to_np(proj.clamped)[vis]
    diff = cl != ref["clamped"][vis]
    near0 = (ref["rgb"][vis] < 1e-5).any(axis=1)
    assert not (diff & ~near0).any(), "colour clamp flags differ"


def check_tile_runs(proj, ref, ref_lists, tiles_x):
    """The packed row runs equal, row by row, the oracle's member tiles of every visible splat
    whose rectangle spans at most 8 rows and 15 columns (the bytes past the last row 0x0F);
    all ones for the others."""
    runs = to_np(proj.tile_runs).view(np.uint64)
    ones = np.uint64(0xFFFFFFFFFFFFFFFF)
    rect = ref["rect"]
    vis = ~ref["culled"].astype(bool)
    assert (runs[~vis] == ones).all(), "culled splats must carry all ones"
    tiles = (ref_lists["keys"] >> np.uint64(32)).astype(np.int64)
    ids = ref_lists["ids"].astype(np.int64)
    order = np.argsort(ids, kind="stable")
    ids_s, tiles_s = ids[order], tiles[order]
    starts = np.searchsorted(ids_s, np.arange(len(rect) + 1))
    packed = unpacked = 0
    for i in np.flatnonzero(vis):
        x0, y0, x1, y1 = (int(v) for v in rect[i])
        if y1 - y0 >= 8 or x1 - x0 >= 15:
            assert runs[i] == ones, f"splat {i}: large rectangle must not be packed"
            unpacked += 1
            continue
        packed += 1
        member = tiles_s[starts[i]:starts[i + 1]]
        for k in range(y1 - y0 + 1, 8):
            assert (int(runs[i]) >> (8 * k)) & 0xFF == 0x0F, f"splat {i}: byte {k} past the last row"
        for k in range(y1 - y0 + 1):
            b = (int(runs[i]) >> (8 * k)) & 0xFF
            c0, c1 = x0 + (b & 15), x0 + (b >> 4)
            cols = np.sort(member[member // tiles_x == y0 + k] % tiles_x)
            if cols.size == 0:
                assert c0 > c1, f"splat {i} row {y0 + k}: expected no run"
            else:
                assert (c0, c1) == (int(cols[0]), int(cols[-1])) and cols.size == c1 - c0 + 1, \
                    f"splat {i} row {y0 + k}: run ({c0}, {c1}) != {cols.tolist()}"
    return packed, unpacked


def tile_runs(keys_or_none, values, ranges):
    return [values[a:b] for a, b in ranges]


def check_lists(bins, ref_lists, tile_mask=None):
    """Per-tile runs of the GPU sort equal the oracle's (tile, depth, id) order, bit for bit."""
    ranges = to_np(bins.ranges).astype(np.int64)
    rref = ref_lists["ranges"].astype(np.int64)
    M = int(to_np(bins.num_instances)[0])
    keys = to_np(bins.keys)[:M].view(np.uint64)
    vals = to_np(bins.values)[:M]
    if tile_mask is None:
        assert M == ref_lists["M"], f"instance count {M} != {ref_lists['M']}"
        assert np.array_equal(keys, ref_lists["keys"]), "sorted keys differ"
        assert np.array_equal(vals, ref_lists["ids"]), "sorted values differ"
        assert np.array_equal(ranges, rref), "tile ranges differ"
    else:
        for t in np.flatnonzero(np.asarray(tile_mask).reshape(-1)):
            a, b = ranges[t]
            c, d = rref[t]
            assert b - a == d - c, f"tile {t}: run length {b - a} != {d - c}"
            assert np.array_equal(vals[a:b], ref_lists["ids"][c:d]), f"tile {t}: run differs"
            assert np.array_equal(keys[a:b], ref_lists["keys"][c:d]), f"tile {t}: keys differ"


def last_ids(img, bins, cam, tile):
    """Splat id of each pixel's last contributor from the GPU's run position (-1 if none)."""
    H, W = cam.height, cam.width
    tx = (W + tile - 1) // tile
    last = to_np(img.last).astype(np.int64)
    ranges = to_np(bins.ranges).astype(np.int64)
    vals = to_np(bins.values).astype(np.int64)
    ys, xs = np.mgrid[0:H, 0:W]
    t = (ys // tile) * tx + xs // tile
    start = ranges[t, 0]
    out = np.where(last > 0, vals[np.clip(start + last - 1, 0, len(vals) - 1)], -1)
    return out


def check_render(img, bins, ref, cam, tile, pixel_mask=None, tol=COLOUR_TOL):
    """Counts and last contributors exact where the oracle's decisions are unique; colour and
    transmittance within tol.  Where the oracle enumerated several outcomes the GPU must equal
    one of them.  Returns (#checked, #ambiguous, #unverifiable)."""
    H, W = cam.height, cam.width
    mask = np.ones((H, W), bool) if pixel_mask is None else pixel_mask
    image = to_np(img.image)
    T = to_np(img.t_final)
    count = to_np(img.n_contrib)
    lid = last_ids(img, bins, cam, tile)
    amb = ref["amb"]
    uniq = mask & (amb == 0)
    assert np.array_equal(count[uniq], ref["count"][uniq]), \
        f"contributor counts differ at {np.argwhere(uniq & (count != ref['count']))[:5].tolist()}"
    assert np.array_equal(lid[uniq], ref["last_id"][uniq]), "last contributors differ"
    cerr = np.abs(image - ref["image"])[:, uniq].max(initial=0.0)
    assert cerr <= tol, f"colour error {cerr}"
    terr = np.abs(T - ref["T"])[uniq].max(initial=0.0)
    assert terr <= tol, f"transmittance error {terr}"
    alts = {}
    for a in ref["alts"]:
        alts.setdefault(a["pixel"], []).append(a)
    n_amb = 0
    for y, x in np.argwhere(mask & (amb == 1)):
        pix = y * W + x
        options = [dict(count=ref["count"][y, x], last_id=ref["last_id"][y, x], C=ref["image"][:, y, x])]
        options += [dict(count=a["count"], last_id=a["last_id"], C=np.array(a["C"])) for a in alts.get(pix, [])]
        ok = any(o["count"] == count[y, x] and o["last_id"] == lid[y, x] and
                 np.abs(image[:, y, x] - o["C"]).max() <= tol for o in options)
        assert ok, f"pixel ({x},{y}) matches none of the {len(options)} valid outcomes"
        n_amb += 1
    n_unv = int((mask & (amb == 2)).sum())
    assert n_unv <= max(2, 1e-3 * mask.sum()), f"{n_unv} unverifiable pixels"
    return int(uniq.sum()), n_amb, n_unv


# Per call of grad_close: (name, elements, elements within rtol alone, elements that pass only
# through the atol * max floor).  The session summary (conftest.py) prints the totals.
GRAD_STATS = []
# Per image-level comparison against the FP64-geometry oracle: dicts printed by the summary.
GEOM64_STATS = []


def grad_close(name, got, ref, rtol=GRAD_RTOL, atol=GRAD_ATOL):
    """|got - ref| <= rtol |ref| + atol max|ref| per element.  Records how many elements meet the
    relative bound alone and how many pass only through the absolute floor."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max(initial=0.0)
    err = np.abs(got - ref)
    bound = rtol * np.abs(ref) + atol * scale
    bad = err > bound
    rel_ok = err <= rtol * np.abs(ref)
    nz = ref != 0
    GRAD_STATS.append((name, int(nz.sum()), int((rel_ok & nz).sum()), int((~rel_ok & ~bad & nz).sum())))
    assert not bad.any(), (f"{name}: {bad.sum()} of {bad.size} elements out of tolerance; worst "
                           f"{(err / np.maximum(bound, 1e-300)).max():.3g}x bound, scale {scale:.3g}")


def ambiguity_masked_grad(dL, amb):
    """Zero the upstream gradient at pixels whose forward decisions are not unique."""
    d = np.array(dL, np.float64, copy=True)
    d[:, amb != 0] = 0.0
    return d
