"""Serving through the C ABI: every request's image equals the single-view render of the same
camera, scene and kernel, whether it ran alone, in a mixed batch, or after a capacity retry."""
import numpy as np
import pytest
import torch

from paper_2501_12369_gb300 import darb, synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

RESOLUTIONS = ((333, 207), (64, 64), (160, 90), (96, 200))
KERNELS = ("half_cosine", "gaussian", "parabola")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def scenes():
    return [darb.splats_to_device(synth.cluster_scene(20000, seed=2)),
            darb.splats_to_device(synth.uniform_cube_scene(1024, seed=0)),
            darb.splats_to_device(synth.cluster_scene(5000, seed=7, sh_degree=1))]


def _single(sd, cam, kernel, tile):
    r = darb.Rasterizer(cam, kernel, tile)
    proj, bins, img = r.forward(sd)
    return img.image


def _requests(n, n_scenes, seed):
    rng = np.random.default_rng(seed)
    cams = synth.random_pose_cameras(n, 4.0, RESOLUTIONS, 0.8, seed=seed)
    return [(int(rng.integers(n_scenes)), cams[i], KERNELS[int(rng.integers(len(KERNELS)))]) for i in range(n)]


@pytest.mark.parametrize("max_batch", [1, 8])
def test_serving_equals_single_views(scenes, max_batch):
    srv = darb.Server(1 << 28, 1 << 30, tile=16, max_batch=max_batch, depth=2)
    try:
        ids = [srv.add_scene(s) for s in scenes]
        reqs = _requests(24, len(scenes), seed=max_batch)
        imgs, tickets = [], []
        for sid, cam, k in reqs:
            imgs.append(torch.full((3, cam.height, cam.width), -1.0, device="cuda"))
            tickets.append(srv.submit(ids[sid], cam, imgs[-1], k))
        results = [srv.poll(t) for t in tickets]
        assert all(r.status == 0 for r in results)
        if max_batch == 1:
            assert all(r.batch_size == 1 for r in results)
        assert all(r.batch_id >= 1 and r.gpu_end_us > r.gpu_begin_us >= 0.0 for r in results)
        for (sid, cam, k), img, r in zip(reqs, imgs, results):
            ref = _single(scenes[sid], cam, k, 16)
            assert torch.equal(img, ref)
            assert r.latency_us >= r.queue_us >= 0.0
    finally:
        srv.close()


@pytest.mark.parametrize("slots", [2, 3])
def test_batches_form_and_overlap_under_load(scenes, slots):
    """48 requests queued at once (one hold of the queue), max_batch 8: the worker must batch
    them, several batches are on the device together (one begins before another has ended, by
    the device clock), and every image still equals its single-view render."""
    big = darb.splats_to_device(synth.cluster_scene(200_000, seed=3))
    srv = darb.Server(1 << 29, 6 << 30, tile=16, max_batch=8, depth=2, slots=slots)
    try:
        ids = [srv.add_scene(s) for s in (big, scenes[0], scenes[2])]
        # views large enough that a batch's device work outlasts the enqueue of the next one
        rng = np.random.default_rng(40 + slots)
        cams = synth.random_pose_cameras(48, 4.0, ((1280, 720), (1920, 1080), (640, 360)), 0.8, seed=40 + slots)
        reqs = [(int(rng.integers(3)), cams[i], KERNELS[int(rng.integers(len(KERNELS)))]) for i in range(48)]
        imgs = [torch.full((3, cam.height, cam.width), -1.0, device="cuda") for _, cam, _ in reqs]
        tickets = srv.submit_many([ids[sid] for sid, _, _ in reqs], [c for _, c, _ in reqs], imgs,
                                  [k for _, _, k in reqs])
        results = [srv.poll(t) for t in tickets]
        assert all(r.status == 0 for r in results)
        sizes = [r.batch_size for r in results]
        assert max(sizes) > 1, "no request was batched with another"
        batches = {}
        for r in results:
            batches.setdefault(r.batch_id, (r.gpu_begin_us, r.gpu_end_us))
        assert len(batches) >= 48 // 8
        spans = sorted(batches.values())
        assert all(b > a for a, b in spans), "every batch has a positive device duration"
        overlapped = sum(1 for (a0, a1), (b0, b1) in zip(spans, spans[1:]) if b0 < a1)
        assert overlapped >= 1, f"no two batches were on the device together: {spans}"
        for (sid, cam, k), img in zip(reqs, imgs):
            ref = _single((big, scenes[0], scenes[2])[sid], cam, k, 16)
            assert torch.equal(img, ref)
    finally:
        srv.close()


def test_capacity_retry(scenes):
    """A first capacity guess far too small: the view is re-queued once with the capacity its
    instance count asks for, and the image is still exact."""
    srv = darb.Server(1 << 28, 1 << 30, tile=8, max_batch=4, capacity_per_pixel=1e-3, capacity_min=16)
    try:
        sid = srv.add_scene(scenes[0])
        cam = synth.random_pose_cameras(1, 4.0, [(333, 207)], 0.8, seed=11)[0]
        img = torch.empty(3, cam.height, cam.width, device="cuda")
        r = srv.poll(srv.submit(sid, cam, img))
        assert r.status == 0 and r.attempts == 2 and r.num_instances > 16
        assert torch.equal(img, _single(scenes[0], cam, "half_cosine", 8))
        # the scene's observed ratio now sizes later requests: no retry
        img2 = torch.empty(3, cam.height, cam.width, device="cuda")
        r2 = srv.poll(srv.submit(sid, cam, img2))
        assert r2.status == 0 and r2.attempts == 1
    finally:
        srv.close()


def test_admission_and_errors(scenes):
    srv = darb.Server(1 << 20, 1 << 24, tile=16, max_batch=4)  # 1 MiB of scenes, 8 MiB per slot
    try:
        with pytest.raises(darb.DarbError) as e:
            srv.add_scene(scenes[0])  # 20k splats at SH degree 3 need more than 1 MiB
        assert e.value.status == 6
        sid = srv.add_scene(scenes[1])
        big = synth.pinhole((0.0, 0.0, 4.0), 4096, 4096, 4096.0)
        with pytest.raises(darb.DarbError) as e:  # its workspace exceeds a slot even alone
            srv.submit(sid, big, torch.empty(3, 4096, 4096, device="cuda"))
        assert e.value.status == 6
        cam = synth.pinhole((0.0, 0.0, 4.0), 64, 64, 64.0)
        with pytest.raises(darb.DarbError) as e:
            srv.submit(sid + 5, cam, torch.empty(3, 64, 64, device="cuda"))
        assert e.value.status == 7
        with pytest.raises(darb.DarbError) as e:
            srv.poll(12345, 0)
        assert e.value.status == 7
        img = torch.empty(3, 64, 64, device="cuda")
        t = srv.submit(sid, cam, img)
        assert srv.poll(t).status == 0
        # a batch submission stops at the first bad request; the ones before it stay queued
        imgs = [torch.empty(3, 64, 64, device="cuda") for _ in range(3)]
        with pytest.raises(darb.DarbError) as e:
            srv.submit_many([sid, sid, sid + 5], [cam, cam, cam], imgs)
        assert e.value.status == 7
        queued = [k for k in srv._keep if k > t]
        assert len(queued) == 2 and all(srv.poll(k).status == 0 for k in queued)
        with pytest.raises(darb.DarbError) as e:  # collected already
            srv.poll(t, 0)
        assert e.value.status == 7
    finally:
        srv.close()


def test_destroy_drains_queue(scenes):
    srv = darb.Server(1 << 28, 1 << 30, tile=16, max_batch=4)
    sid = srv.add_scene(scenes[0])
    cams = synth.random_pose_cameras(12, 4.0, RESOLUTIONS, 0.8, seed=5)
    imgs = [torch.full((3, c.height, c.width), -1.0, device="cuda") for c in cams]
    for c, im in zip(cams, imgs):
        srv.submit(sid, c, im)
    srv.close()  # returns once every queued request has rendered
    torch.cuda.synchronize()
    for c, im in zip(cams, imgs):
        assert torch.equal(im, _single(scenes[0], c, "half_cosine", 16))
