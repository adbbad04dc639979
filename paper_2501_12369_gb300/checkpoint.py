"""Checkpoint and resume of a training state, and the splat set alone for reproducible runs.

A training state is what the fused backward + Adam step reads and writes: the raw parameters
(means, log-scales, quaternions, opacity logits, SH), their activated copies (scales,
opacities), both Adam moments of every group, and the step count that sets Adam's bias
corrections.  `save_training` writes host copies of all of them to one .npz file;
`load_training` puts them back on a device as the objects the binding takes (attributes named
as the fields of darb_train_params and darb_adam_state).  Float32 arrays are written as they
are, so a resumed state is bit for bit the saved one.
"""
from __future__ import annotations

import types

import numpy as np
import torch

from . import darb, synth

PARAM_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh", "scales", "opacities")
STATE_FIELDS = tuple(f for f, _ in darb.darb_adam_state._fields_)


def _host(t) -> np.ndarray:
    return t.detach().to("cpu").contiguous().numpy()


def save_training(path, params, state, step: int) -> None:
    """params / state: objects with the darb_train_params / darb_adam_state fields as tensors
    (params also with sh_degree); step: the Adam steps taken so far."""
    arrays = {"param_" + f: _host(getattr(params, f)) for f in PARAM_FIELDS}
    arrays.update({"state_" + f: _host(getattr(state, f)) for f in STATE_FIELDS})
    for k, a in arrays.items():
        if a.dtype != np.float32:
            raise ValueError(f"{k}: expected float32, got {a.dtype}")
    np.savez(path, sh_degree=np.int32(params.sh_degree), step=np.int64(step), **arrays)


def load_training(path, device="cuda"):
    """Returns (params, state, step) as saved, the tensors on `device`."""
    with np.load(path) as z:
        params = types.SimpleNamespace(
            **{f: torch.from_numpy(z["param_" + f].copy()).to(device) for f in PARAM_FIELDS},
            sh_degree=int(z["sh_degree"]))
        state = types.SimpleNamespace(**{f: torch.from_numpy(z["state_" + f].copy()).to(device) for f in STATE_FIELDS})
        step = int(z["step"])
    n = params.means.shape[0]
    for f in PARAM_FIELDS + STATE_FIELDS:
        t = getattr(params, f) if f in PARAM_FIELDS else getattr(state, f)
        if t.shape[0] != n:
            raise ValueError(f"{f}: {t.shape[0]} rows, expected {n}")
    return params, state, step


def save_splats(path, s: synth.Splats) -> None:
    """A splat set (activated scales and opacities, as the forward path takes them)."""
    np.savez(path, means=s.means, scales=s.scales, quats=s.quats, opacities=s.opacities, sh=s.sh,
             sh_degree=np.int32(s.sh_degree))


def load_splats(path) -> synth.Splats:
    with np.load(path) as z:
        return synth.Splats(z["means"].copy(), z["scales"].copy(), z["quats"].copy(), z["opacities"].copy(),
                            z["sh"].copy(), int(z["sh_degree"]))
