"""darb_bin_sort_noalloc, the allocation-free form of darb_bin_sort for callers that cannot
allocate device memory (it sorts in a static scratch array inside the library).

Collected last on purpose: it checks the variant against the existing entry point on two
calls in a row, and must pass both alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest
import torch

from paper_2501_12369_gb300 import darb, synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()


def _np(t):
    return t.detach().cpu().numpy()


def test_noalloc_sort_equals_workspace_sort_twice_in_a_row():
    s, cam = synth.small_forward_workload()
    big = synth.cluster_scene(20000, seed=4)
    cam_big = synth.fibonacci_cameras(8, 6.0, 320, 200, 250.0)[1]
    for splats, c, tile in ((s, cam, 16), (big, cam_big, 8)):
        kp = darb.darb_kernel_defaults("half_cosine")
        sd = darb.splats_to_device(splats)
        proj = darb.darb_preprocess(sd, c, kp, tile)
        cap = 200000
        ws = torch.empty(darb.darb_bin_sort_workspace_size(splats.n, tile, c, cap), dtype=torch.uint8, device="cuda")
        ref = darb.darb_bin_sort(proj, splats.n, tile, c, ws, cap)
        M = ref.M
        rk, rv, rr = _np(ref.keys)[:M].copy(), _np(ref.values)[:M].copy(), _np(ref.ranges).copy()
        tx, ty = darb.darb_tile_grid(c, tile)
        b = darb.Binning.empty(cap, tx * ty, "cuda")  # every output allocated before the calls
        free = []
        for sync in (True, False, True):  # calls in a row, host-sized and capacity-sized
            b.values.fill_(-1)
            b.ranges.fill_(-1)
            torch.cuda.synchronize()
            if sync is False:  # the first call may load the library's module; measure from the second on
                free.append(torch.cuda.mem_get_info()[0])
            darb.darb_bin_sort_noalloc(proj, splats.n, tile, c, cap, out=b, sync=sync)
            torch.cuda.synchronize()
            if len(free) == 1:
                free.append(torch.cuda.mem_get_info()[0])
            assert int(_np(b.num_instances)[0]) == M and int(_np(b.status)[0]) == 0
            assert np.array_equal(_np(b.keys)[:M], rk)
            assert np.array_equal(_np(b.values)[:M], rv)
            assert np.array_equal(_np(b.ranges), rr)
        assert free[0] == free[1], f"device memory changed across a call: {free[0]} -> {free[1]} bytes free"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    s, cam = synth.small_forward_workload()
    kp = darb.darb_kernel_defaults("half_cosine")
    proj = darb.darb_preprocess(darb.splats_to_device(s), cam, kp, 16)
    cap = 1 << 26  # needs far more than the 64 MiB static scratch
    out = darb.Binning.empty(16, 16, "cuda")
    with pytest.raises(darb.DarbError) as e:
        darb.darb_bin_sort_noalloc(proj, s.n, 16, cam, cap, out=out)
    assert e.value.status == 2
