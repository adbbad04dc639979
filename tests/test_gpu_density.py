"""Adaptive density control through the C ABI against the oracle: statistics bit for bit, the
clone / split / prune pass with exact counts, order and copied values, children within float32
rounding, and the opacity reset."""
import types

import numpy as np
import pytest
import torch

import oracle
from paper_2501_12369_gb300 import darb, synth

from gpu_helpers import to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

RAW = ("means", "log_scales", "quats", "opacity_logits", "sh")
STATE_OF = dict(means="means", log_scales="scales", quats="quats", opacity_logits="opac", sh="sh")
CFG = dict(grad_threshold=2e-4, dense_scale=0.05, min_opacity=0.005, max_screen_radius=20.0, max_world_scale=0.5,
           split_scale_div=1.6)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()
    oracle.build()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(n, deg, seed):
    rng = np.random.default_rng(seed)
    s = synth.cluster_scene(n, seed=seed, sh_degree=deg, log_scale=(-4.5, -0.8))
    raw = dict(means=s.means.astype(np.float32), log_scales=np.log(s.scales).astype(np.float32),
               quats=s.quats.astype(np.float32),
               opacity_logits=np.log(s.opacities / (1 - s.opacities)).astype(np.float32), sh=s.sh.astype(np.float32))
    act = dict(scales=np.exp(raw["log_scales"].astype(np.float64)).astype(np.float32),
               opacities=(1 / (1 + np.exp(-raw["opacity_logits"].astype(np.float64)))).astype(np.float32))
    act["opacities"][::13] = 0.002  # prunable
    state = {f"{m}_{k}": rng.normal(size=v.shape).astype(np.float32) for k, v in raw.items() for m in ("m", "v")}
    accum = (rng.exponential(4e-4, n) * rng.integers(0, 6, n)).astype(np.float32)
    count = rng.integers(0, 6, n).astype(np.float32)
    radius = rng.integers(0, 40, n).astype(np.int32)
    normals = rng.normal(size=(n, 2, 3)).astype(np.float32)
    return raw, act, state, accum, count, radius, normals


def _device(raw, act, state, deg, rows=None):
    if rows is None:
        p = types.SimpleNamespace(**{k: _t(v) for k, v in raw.items()}, scales=_t(act["scales"]),
                                  opacities=_t(act["opacities"]), sh_degree=deg)
        st = types.SimpleNamespace(**{f"{m}_{STATE_OF[k]}": _t(state[f"{m}_{k}"]) for k in RAW for m in ("m", "v")})
        return p, st
    z = lambda v: torch.full((rows,) + v.shape[1:], np.nan, dtype=torch.float32, device="cuda")  # noqa: E731
    p = types.SimpleNamespace(**{k: z(v) for k, v in raw.items()}, scales=z(act["scales"]),
                              opacities=z(act["opacities"]), sh_degree=deg)
    st = types.SimpleNamespace(**{f"{m}_{STATE_OF[k]}": z(state[f"{m}_{k}"]) for k in RAW for m in ("m", "v")})
    return p, st


def test_statistics_are_bit_exact():
    rng = np.random.default_rng(1)
    n, W, H = 5003, 333, 207
    accum, count, rmax = np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.int32)
    da, dc, dr = _t(accum), _t(count), _t(rmax)
    for step in range(4):
        g2 = rng.normal(scale=1e-3, size=(n, 12)).astype(np.float32)
        radius = (rng.integers(0, 30, n) * (rng.random(n) < 0.7)).astype(np.int32)
        darb.darb_densify_stats(_t(g2), _t(radius), W, H, da, dc, dr)
        oracle.densify_stats(g2, radius, W, H, accum, count, rmax)
    torch.cuda.synchronize()
    assert np.array_equal(to_np(da), accum) and np.array_equal(to_np(dc), count) and np.array_equal(to_np(dr), rmax)


@pytest.mark.parametrize("deg", [1, 3])
def test_densify_matches_oracle(deg):
    n = 6001
    raw, act, state, accum, count, radius, normals = _case(n, deg, seed=deg)
    ref_raw, ref_act, ref_state, n_ref = oracle.densify(raw, act, state, accum, count, radius, normals, CFG)
    clone, split, keep = oracle.densify_actions(act["scales"], act["opacities"], accum, count, radius, CFG)
    assert clone.sum() > 10 and split.sum() > 10 and (~keep).sum() > 10, "the case should exercise every action"
    p, st = _device(raw, act, state, deg)
    po, so = _device(raw, act, state, deg, rows=2 * n)
    cfg = darb.darb_densify_cfg(**CFG)
    n_out = darb.darb_densify(p, st, _t(accum), _t(count), _t(radius), _t(normals), cfg, po, so)
    torch.cuda.synchronize()
    rows, c0, k0 = (int(x) for x in to_np(n_out))
    assert rows == n_ref
    n_child = 2 * int((split & oracle._survives(act["opacities"], np.max(act["scales"] / np.float32(1.6), axis=1),
                                                np.zeros(n, np.int32), CFG)).sum())
    assert k0 == rows - n_child
    exact = rows - n_child  # survivors and clones are copies
    for k in RAW:
        got = to_np(getattr(po, k))[:rows]
        if k == "means":
            np.testing.assert_array_equal(got[:exact], ref_raw[k][:exact])
            np.testing.assert_allclose(got[exact:], ref_raw[k][exact:], rtol=0, atol=2e-6)
        else:
            np.testing.assert_array_equal(got, ref_raw[k], err_msg=k)
        for m in ("m", "v"):
            np.testing.assert_array_equal(to_np(getattr(so, f"{m}_{STATE_OF[k]}"))[:rows], ref_state[f"{m}_{k}"])
    np.testing.assert_allclose(to_np(po.scales)[:rows], ref_act["scales"], rtol=5e-7)
    np.testing.assert_allclose(to_np(po.opacities)[:rows], ref_act["opacities"], rtol=3e-7, atol=1e-9)


def test_densify_edge_cases():
    raw, act, state, accum, count, radius, normals = _case(100, 0, seed=9)
    p, st = _device(raw, act, state, 0)
    po, so = _device(raw, act, state, 0, rows=200)
    cfg = dict(CFG, min_opacity=2.0)  # every splat pruned, nothing grows either
    n_out = darb.darb_densify(p, st, _t(accum), _t(count), _t(radius), _t(normals), darb.darb_densify_cfg(**cfg),
                              po, so)
    torch.cuda.synchronize()
    assert to_np(n_out).tolist() == [0, 0, 0]
    small, sst = _device(raw, act, state, 0, rows=150)  # capacity below 2 n
    with pytest.raises(darb.DarbError):
        darb.darb_densify(p, st, _t(accum), _t(count), _t(radius), _t(normals), darb.darb_densify_cfg(**CFG), small,
                          sst)
    with pytest.raises(darb.DarbError):  # output overlapping the input
        darb.darb_densify(p, st, _t(accum), _t(count), _t(radius), _t(normals), darb.darb_densify_cfg(**CFG), p, st)


def test_opacity_reset_matches_oracle():
    raw, act, state, *_ = _case(1000, 0, seed=3)
    p, _ = _device(raw, act, state, 0)
    darb.darb_reset_opacity(p, 0.01)
    torch.cuda.synchronize()
    ref = oracle.reset_opacity(raw["opacity_logits"], 0.01)
    np.testing.assert_array_equal(to_np(p.opacity_logits), ref)
    np.testing.assert_allclose(to_np(p.opacities), 1 / (1 + np.exp(-ref.astype(np.float64))), rtol=6e-7)
