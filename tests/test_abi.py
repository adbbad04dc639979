"""The C-ABI library without a GPU: it builds, loads, exports every declared entry point, and
its host-only calls (defaults, tile grid, workspace query, argument validation) behave."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(darb_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_2501_12369_gb300 import build, darb
    build.build()
    return darb.lib()


def test_library_exports_every_declared_symbol(L):
    from paper_2501_12369_gb300 import darb
    names = _declared()
    assert {"darb_preprocess", "darb_bin_sort", "darb_render_fwd", "darb_render_bwd"} <= names
    for n in sorted(names):
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    # the binding covers every declared entry point
    assert names <= set(darb.SIGNATURES), names - set(darb.SIGNATURES)


def test_kernel_defaults_follow_the_listings(L):
    from paper_2501_12369_gb300 import darb
    golden = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_kernel_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, xi, psi_t, psi_l, qmax, strict = line.split()
        golden[name] = (psi_l if psi_l != "NA" else psi_t, qmax, strict)
    for i, name in enumerate(darb.KERNEL_NAMES):
        kp = darb.darb_kernel_defaults(name)
        assert kp.kind == i
        psi, qmax, strict = golden[name]
        assert kp.psi == pytest.approx(float(psi), abs=1e-7)
        if qmax != "NA":
            assert kp.q_max == float(qmax) and kp.q_max_strict == int(strict)
    with pytest.raises(darb.DarbError):
        darb.darb_kernel_defaults(7)


def test_tile_grid_and_workspace_query(L):
    from paper_2501_12369_gb300 import darb, synth
    cam = synth.pinhole((0, 0, 4), 1920, 1080, 1500.0)
    assert darb.darb_tile_grid(cam, 16) == (120, 68)
    assert darb.darb_tile_grid(cam, 8) == (240, 135)
    a = darb.darb_bin_sort_workspace_size(1000, 16, cam, 1 << 20)
    b = darb.darb_bin_sort_workspace_size(1000, 16, cam, 1 << 21)
    assert 12 * (1 << 20) <= a < b
    with pytest.raises(darb.DarbError):
        darb.darb_tile_grid(cam, 12)
    with pytest.raises(darb.DarbError):
        darb.darb_bin_sort_workspace_size(1000, 16, cam, 1 << 31)


def test_invalid_arguments_are_rejected_before_any_device_work(L):
    from paper_2501_12369_gb300 import darb, synth
    cam = darb.camera(synth.pinhole((0, 0, 4), 64, 64, 64.0))
    kp = darb.darb_kernel_defaults("half_cosine")
    sp = darb.darb_splats(None, None, None, None, None, -1, 0)
    out = darb.darb_projected()
    assert L.darb_preprocess(ctypes.byref(sp), ctypes.byref(cam), ctypes.byref(kp), 16, ctypes.byref(out), None) == 1
    sp.n, sp.sh_degree = 10, 4
    assert L.darb_preprocess(ctypes.byref(sp), ctypes.byref(cam), ctypes.byref(kp), 16, ctypes.byref(out), None) == 1
    sp.sh_degree = 0
    misaligned = ctypes.c_void_p(0x1004)
    sp.means = sp.scales = sp.quats = sp.opacities = sp.sh = misaligned
    assert L.darb_preprocess(ctypes.byref(sp), ctypes.byref(cam), ctypes.byref(kp), 16, ctypes.byref(out), None) == 1
    bad = darb.darb_kernel_params(9, 1.0, 9.0, 0)
    sp.n = 0
    assert L.darb_preprocess(ctypes.byref(sp), ctypes.byref(cam), ctypes.byref(bad), 16, ctypes.byref(out), None) == 1
    cam.width = 0
    assert L.darb_preprocess(ctypes.byref(sp), ctypes.byref(cam), ctypes.byref(kp), 16, ctypes.byref(out), None) == 1
    assert L.darb_status_string(3) == b"instance capacity exceeded"
    # server configurations are checked before the device is touched
    srv = ctypes.c_void_p()
    good = dict(scene_bytes=1 << 20, workspace_bytes=1 << 24, tile=16, max_batch=4, depth=2, capacity_per_pixel=16.0,
                capacity_margin=1.15, capacity_min=1 << 16, slots=2)
    for field, value in [("slots", -1), ("slots", 9), ("tile", 12), ("max_batch", 0), ("depth", 9),
                         ("capacity_margin", 0.5), ("workspace_bytes", 4096)]:
        cfg = darb.darb_serve_cfg(**dict(good, **{field: value}))
        assert L.darb_serve_create(ctypes.byref(cfg), ctypes.byref(srv)) == 1, field
    assert L.darb_serve_submit_many(None, None, 0, None, None) == 1


def test_oracle_and_library_share_no_source():
    """The oracle is independent of the CUDA path: no file of one includes or imports the other."""
    csrc = os.path.join(ROOT, "paper_2501_12369_gb300")
    for dirpath, _, files in os.walk(csrc):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|from|#include)\s+[\"<]?(\w+)", text), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2501_12369_gb300" not in text and "darb.h" not in text, f


def test_generic_kernel_parameters_match_the_oracle():
    """darb_kernel_generic (host code) gives the oracle's float32 q_max for Table 1's members and
    rejects invalid descriptions."""
    import oracle
    from paper_2501_12369_gb300 import darb
    for base, xi, beta, lobes in [("half_cosine", 3.0, 1.5, 1), ("raised_cosine", 1.2, 2.0, 1),
                                  ("mod_sinc", 1.1, 1.5, 2), ("gaussian", 1.0, 2.5, 1), ("parabola", 4.0, 2.0, 1),
                                  ("half_cosine", 18 / np.pi, 2.0, 1), ("raised_cosine", 2.5 / np.pi, 1.0, 1)]:
        kp = darb.darb_kernel_generic(base, xi, beta, lobes, psi=None)
        ko = oracle.generic_kernel(base, xi, beta, lobes, psi=1.0)
        assert kp.kind == 7 and kp.q_max == ko.q_max and kp.q_max_strict == 0
        assert (kp.base, kp.xi, kp.beta, kp.lobes) == (ko.base, ko.xi, ko.beta, ko.lobes)
    for bad in [(6, 1.0, 2.0, 1), (1, 0.0, 2.0, 1), (1, 1.0, 0.2, 1), (1, 1.0, 2.0, 0)]:
        with pytest.raises(darb.DarbError):
            darb.darb_kernel_generic(*bad, psi=None)
    with pytest.raises(darb.DarbError):  # the generic kind has no defaults
        darb.darb_kernel_defaults(7)
