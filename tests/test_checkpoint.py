"""Checkpoint and resume (host side): a training state and a splat set written to .npz and read
back are bit for bit what was saved, and mismatched row counts are refused."""
import types

import numpy as np
import pytest
import torch

from paper_2501_12369_gb300 import checkpoint, synth


def _state(n=37, deg=2, seed=3):
    rng = np.random.default_rng(seed)
    k = 3 * (deg + 1) ** 2
    t = lambda *shape: torch.from_numpy(rng.normal(size=shape).astype(np.float32))
    params = types.SimpleNamespace(means=t(n, 3), log_scales=t(n, 3), quats=t(n, 4), opacity_logits=t(n),
                                   sh=t(n, k // 3, 3), scales=t(n, 3), opacities=t(n), sh_degree=deg)
    shapes = dict(means=(n, 3), scales=(n, 3), quats=(n, 4), opac=(n,), sh=(n, k // 3, 3))
    state = types.SimpleNamespace(**{f"{m}_{g}": t(*shape) for g, shape in shapes.items() for m in ("m", "v")})
    return params, state


def test_training_state_round_trip(tmp_path):
    params, state = _state()
    path = tmp_path / "ckpt.npz"
    checkpoint.save_training(path, params, state, step=17)
    p2, s2, step = checkpoint.load_training(path, device="cpu")
    assert step == 17 and p2.sh_degree == params.sh_degree
    for f in checkpoint.PARAM_FIELDS:
        assert torch.equal(getattr(p2, f), getattr(params, f)), f
    for f in checkpoint.STATE_FIELDS:
        assert torch.equal(getattr(s2, f), getattr(state, f)), f


def test_training_state_rejects_wrong_dtype_and_rows(tmp_path):
    params, state = _state()
    bad = types.SimpleNamespace(**vars(params))
    bad.means = bad.means.double()
    with pytest.raises(ValueError):
        checkpoint.save_training(tmp_path / "a.npz", bad, state, step=1)
    params.opacities = params.opacities[:-1].clone()
    checkpoint.save_training(tmp_path / "b.npz", params, state, step=1)
    with pytest.raises(ValueError):
        checkpoint.load_training(tmp_path / "b.npz", device="cpu")


def test_splat_set_round_trip(tmp_path):
    s = synth.cluster_scene(500, seed=2, sh_degree=3)
    checkpoint.save_splats(tmp_path / "s.npz", s)
    t = checkpoint.load_splats(tmp_path / "s.npz")
    assert t.sh_degree == s.sh_degree
    for f in ("means", "scales", "quats", "opacities", "sh"):
        a, b = getattr(s, f), getattr(t, f)
        assert a.dtype == b.dtype and np.array_equal(a, b), f
