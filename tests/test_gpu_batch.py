"""Batched multi-view rendering through the C ABI: every view of a batch equals the single-view
path bit for bit (and the oracle, on small views), eager or replayed from a CUDA graph."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_12369_gb300 import darb, synth

from gpu_helpers import check_render, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()
    oracle.build()


RESOLUTIONS = ((333, 207), (64, 64), (160, 90), (96, 200), (17, 23))


def _views(n_cams, seed=3):
    return synth.random_pose_cameras(n_cams, 6.0, RESOLUTIONS, 0.8, seed=seed)


def _single(sd, cam, kernel, tile):
    r = darb.Rasterizer(cam, kernel, tile)
    proj, bins, img = r.forward(sd)
    return img, bins


@pytest.mark.parametrize("depth", [1, 3])
@pytest.mark.parametrize("tile", [8, 16, 32])
def test_batch_equals_single_views(tile, depth):
    s = synth.cluster_scene(20000, seed=2)
    sd = darb.splats_to_device(s)
    cams = _views(7)
    br = darb.BatchRenderer(sd, cams, "half_cosine", tile, depth, aux=True)
    br.render()
    torch.cuda.synchronize()
    br.check()
    for v, cam in enumerate(cams):
        img, bins = _single(sd, cam, "half_cosine", tile)
        torch.cuda.synchronize()
        assert int(br.num_instances[v]) == bins.M
        for name in ("image", "t_final", "last", "n_contrib"):
            a, b = to_np(getattr(br.outs[v], name)), to_np(getattr(img, name))
            assert np.array_equal(a, b), f"view {v} {name}"


@pytest.mark.parametrize("kernel", ["gaussian", "raised_cosine", "inv_multiquadric"])
def test_batch_matches_oracle(kernel):
    s, _ = synth.small_forward_workload()
    cams = [synth.pinhole((0.0, 0.0, 4.0), 64, 64, 64.0), synth.pinhole((0.5, 0.3, 3.5), 48, 40, 50.0),
            synth.pinhole((-1.0, 0.2, 3.8), 33, 65, 60.0)]
    sd = darb.splats_to_device(s)
    br = darb.BatchRenderer(sd, cams, kernel, 16, 2, aux=True)
    br.render()
    torch.cuda.synchronize()
    br.check()
    for v, cam in enumerate(cams):
        ref = oracle.forward(s, cam, kernel, tile=16)
        _, bins = _single(sd, cam, kernel, 16)
        check_render(br.outs[v], bins, ref, cam, 16)


def test_batch_graph_replay_equals_eager():
    s = synth.cluster_scene(30000, seed=4)
    sd = darb.splats_to_device(s)
    cams = _views(12, seed=9)
    br = darb.BatchRenderer(sd, cams, "mod_sinc", 16, 4)
    br.render()
    torch.cuda.synchronize()
    eager = [o.image.clone() for o in br.outs]
    for o in br.outs:
        o.image.fill_(-1.0)
    br.capture()
    for o in br.outs:
        o.image.fill_(-1.0)
    for _ in range(3):
        br.replay()
    torch.cuda.synchronize()
    br.check()
    for v in range(len(cams)):
        assert torch.equal(br.outs[v].image, eager[v]), f"view {v}"


def test_single_view_graph_with_forked_sort_equals_eager():
    """Preprocess, the default sort (its per-tile counts forked onto the library's side stream
    and joined back) and compositing captured in one CUDA graph: replays over two cameras
    (the camera is a kernel argument, so each camera gets its own graph) equal the eager calls."""
    s = synth.cluster_scene(200_000, seed=6)
    sd = darb.splats_to_device(s)
    cams = synth.fibonacci_cameras(8, 6.0, 640, 360, 500.0)[2:4]
    kp = darb.darb_kernel_defaults("half_cosine")
    tile, cap = 32, 4_000_000
    tx, ty = darb.darb_tile_grid(cams[0], tile)
    ws = torch.empty(darb.darb_bin_sort_workspace_size(s.n, tile, cams[0], cap), dtype=torch.uint8, device="cuda")
    proj = darb.Projected.empty(s.n)
    bins = darb.Binning.empty(cap, tx * ty, "cuda", keys=False)
    img = darb.ImageOut.empty(cams[0].width, cams[0].height)

    def run(cam):
        darb.darb_preprocess(sd, cam, kp, tile, out=proj)
        darb.darb_bin_sort(proj, s.n, tile, cam, ws, cap, bins, sync=False)
        darb.darb_render_fwd(proj, bins, cam, kp, tile, out=img)

    eager = []
    for cam in cams:  # the first calls also create the sort's side stream
        run(cam)
        torch.cuda.synchronize()
        assert int(bins.status.item()) == 0
        eager.append([t.clone() for t in (img.image, img.n_contrib, bins.ranges)])
    graphs = []
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    for cam in cams:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            run(cam)
        graphs.append(g)
    torch.cuda.synchronize()
    for _ in range(2):
        for g, ref in zip(graphs, eager):
            img.image.fill_(-1.0)
            g.replay()
            torch.cuda.synchronize()
            for got, want in zip((img.image, img.n_contrib, bins.ranges), ref):
                assert torch.equal(got, want)


def test_batch_capacity_overflow_is_per_view():
    """A capacity below one view's M: that view reports DARB_ERR_CAPACITY and shows background;
    the others render normally."""
    s = synth.cluster_scene(20000, seed=2)
    sd = darb.splats_to_device(s)
    cams = _views(4, seed=5)
    probe = darb.BatchRenderer(sd, cams, "half_cosine", 16, 2)
    counts = probe.counts
    big = int(np.argmax(counts))
    cap = sorted(counts)[-2] + 1  # fits every view but the largest
    if cap > counts[big]:
        pytest.skip("two views with equal instance counts")
    br = darb.BatchRenderer(sd, cams, "half_cosine", 16, 2, capacity=cap)
    br.render()
    torch.cuda.synchronize()
    st = to_np(br.status)
    assert st[big] == 3 and np.all(np.delete(st, big) == 0)
    assert int(br.num_instances[big]) == counts[big]
    bg = np.asarray(cams[big].bg, np.float32)[:, None, None]
    assert np.array_equal(to_np(br.outs[big].image), np.broadcast_to(bg, br.outs[big].image.shape))
    for v in range(len(cams)):
        if v != big:
            img, _ = _single(sd, cams[v], "half_cosine", 16)
            assert torch.equal(br.outs[v].image, img.image)


def test_batch_argument_checks():
    s, cam = synth.small_forward_workload()
    sd = darb.splats_to_device(s)
    kp = darb.darb_kernel_defaults("half_cosine")
    for bad in (darb.darb_batch_params(0, 16, 1, 0, 1024), darb.darb_batch_params(1, 12, 1, 0, 1024),
                darb.darb_batch_params(1, 16, 9, 0, 1024), darb.darb_batch_params(1, 16, 1, -1, 1024),
                darb.darb_batch_params(1, 16, 1, 0, 0)):
        with pytest.raises(darb.DarbError):
            darb.darb_render_batch_workspace_size(sd.n, [cam], bad)
    p = darb.darb_batch_params(1, 16, 1, 0, 1024)
    need = darb.darb_render_batch_workspace_size(sd.n, [cam], p)
    ws = torch.empty(need - 300, dtype=torch.uint8, device="cuda")
    out = darb.ImageOut(torch.empty(3, 64, 64, device="cuda"), None, None, None)
    with pytest.raises(darb.DarbError) as e:
        darb.darb_render_batch(sd, [cam], kp, p, ws, [out])
    assert e.value.status == 2
