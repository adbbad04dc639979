"""The differentiation form: DarbRasterize (a torch.autograd.Function over the hand-written
backward of Sec. 4.2) driven by loss.backward(), against the oracle's analytic gradient and
against central differences of the CUDA forward itself."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_12369_gb300 import darb, synth

from gpu_helpers import ambiguity_masked_grad, grad_close, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()
    oracle.build()


def _leaves(s):
    """Raw trainable parameters as leaf tensors: means, log-scales, quaternions, opacity logits, SH."""
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda().requires_grad_(True)  # noqa: E731
    o = s.opacities.astype(np.float64)
    return dict(means=t(s.means), log_scales=t(np.log(s.scales)), quats=t(s.quats),
                logits=t(np.log(o / (1.0 - o))), sh=t(s.sh))


def _activated(P, s):
    """The splats exactly as the library sees them (exp and sigmoid taken in FP32 by torch)."""
    with torch.no_grad():
        scales = torch.exp(P["log_scales"]).cpu().numpy()
        opac = torch.sigmoid(P["logits"]).cpu().numpy()
    return synth.Splats(s.means.copy(), scales, s.quats.copy(), opac, s.sh.copy(), s.sh_degree)


def _render(P, sh_degree, rast):
    """Activations in torch (exp, sigmoid); everything after them is the library's."""
    return darb.DarbRasterize.apply(P["means"], torch.exp(P["log_scales"]), P["quats"],
                                    torch.sigmoid(P["logits"]), P["sh"], sh_degree, rast)


def _chain_raw(gp, s):
    """The oracle's gradients w.r.t. activated attributes, chained to the raw leaves."""
    o = s.opacities.astype(np.float64)
    return dict(means=gp["means"], log_scales=gp["scales"] * s.scales.astype(np.float64), quats=gp["quats"],
                logits=gp["opacities"] * o * (1.0 - o), sh=gp["sh"])


@pytest.mark.parametrize("kernel", ["half_cosine", "gaussian"])
def test_two_views_then_one_backward(kernel):
    """Three forwards through one rasterizer (two cameras, the first one twice) before a single
    loss.backward(): every forward keeps its own lists, so the summed gradient equals the sum of
    the oracle's per-view gradients."""
    s = synth.cluster_scene(6000, seed=11, sh_degree=3)
    cams = synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)
    views = [cams[3], cams[9], cams[3]]
    tile = 16
    P = _leaves(s)
    s = _activated(P, s)
    rast = darb.Rasterizer(views[0], kernel, tile)
    imgs, dls = [], []
    total = {k: 0.0 for k in P}
    for i, cam in enumerate(views):
        rast.cam = cam
        imgs.append(_render(P, s.sh_degree, rast))
        ref = oracle.forward(s, cam, kernel, tile=tile)
        dl = ambiguity_masked_grad(synth.random_image_grad(cam.height, cam.width, seed=20 + i), ref["amb"])
        dls.append(torch.from_numpy(dl.astype(np.float32)).cuda())
        _, _, gp = oracle.gradients(s, cam, dl.astype(np.float32).astype(np.float64), kernel, tile=tile)
        for k, v in _chain_raw(gp, s).items():
            total[k] = total[k] + v
    # the images are the plain forward's, bit for bit
    for cam, img in zip(views, imgs):
        _, _, single = darb.Rasterizer(cam, kernel, tile).forward(darb.splats_to_device(s))
        assert torch.equal(img.detach(), single.image)
    loss = sum((img * dl).sum() for img, dl in zip(imgs, dls))
    loss.backward()
    torch.cuda.synchronize()
    for k, leaf in P.items():
        grad_close(f"{kernel}/{k}", to_np(leaf.grad), total[k])


def test_backward_twice_through_retained_graph_and_camera_change():
    """retain_graph: a second backward replays the same saved lists (same gradient up to the
    summation order of the atomics); changing the rasterizer's camera after the forward does not
    change what the backward differentiates."""
    s = synth.cluster_scene(3000, seed=12, sh_degree=1)
    cams = synth.fibonacci_cameras(8, 6.0, 160, 120, 150.0)
    P = _leaves(s)
    s = _activated(P, s)
    rast = darb.Rasterizer(cams[1], "raised_cosine", 8)
    img = _render(P, s.sh_degree, rast)
    rast.cam = cams[5]  # a later camera change must not leak into this view's backward
    dl = torch.from_numpy(synth.random_image_grad(120, 160, seed=3)).cuda()
    (img * dl).sum().backward(retain_graph=True)
    first = {k: v.grad.clone() for k, v in P.items()}
    for v in P.values():
        v.grad = None
    (img * dl).sum().backward()
    for k, v in P.items():  # equal up to the order of the FP32 atomics that sum the gradients
        grad_close(f"second backward/{k}", to_np(v.grad), to_np(first[k]), rtol=1e-4, atol=1e-6)
    ref = oracle.forward(s, cams[1], "raised_cosine", tile=8)
    d = ambiguity_masked_grad(to_np(dl), ref["amb"])
    if (ref["amb"] != 0).any():  # compare on the unique pixels only
        for v in P.values():
            v.grad = None
        img2 = _render(P, s.sh_degree, darb.Rasterizer(cams[1], "raised_cosine", 8))
        (img2 * torch.from_numpy(d.astype(np.float32)).cuda()).sum().backward()
    _, _, gp = oracle.gradients(s, cams[1], d.astype(np.float32).astype(np.float64), "raised_cosine", tile=8)
    for k, v in _chain_raw(gp, s).items():
        grad_close(f"raised_cosine/{k}", to_np(P[k].grad), v)


@pytest.mark.parametrize("kernel", ["half_cosine", "gaussian"])
def test_finite_difference_spot_check(kernel):
    """A gradcheck-style check on the FP32 path alone: 16 splats, 32x32.  Central differences of
    the loss sum(image * dL), rendered by the CUDA forward at theta +- h, against loss.backward().
    Samples where the perturbation flips a discrete decision (a contributor count or a last
    contributor changes: the 1/255 skip, the cutoff, a tile membership) are excluded and counted."""
    s = synth.uniform_cube_scene(16, seed=7, sh_degree=1, half=0.6, log_scale=(-2.6, -1.8))
    cam = synth.pinhole((0.2, -0.1, 3.0), 32, 32, 40.0, bg=(0.1, 0.2, 0.3))
    tile = 16
    P = _leaves(s)
    rast = darb.Rasterizer(cam, kernel, tile)
    dl = torch.from_numpy(synth.random_image_grad(32, 32, seed=5)).cuda()
    img = _render(P, s.sh_degree, rast)
    (img * dl).sum().backward()
    grads = {k: to_np(v.grad).astype(np.float64) for k, v in P.items()}
    dl64 = dl.double()

    def loss_and_decisions(name, idx, h):
        with torch.no_grad():
            Q = {k: v.detach().clone() for k, v in P.items()}
            Q[name].view(-1)[idx] += h
            sp = darb.SplatTensors(Q["means"], torch.exp(Q["log_scales"]), Q["quats"], torch.sigmoid(Q["logits"]),
                                   Q["sh"], s.sh_degree)
            _, _, out = darb.Rasterizer(cam, kernel, tile).forward(sp)
            return float((out.image.double() * dl64).sum()), to_np(out.n_contrib), to_np(out.last)

    _, base_n, base_last = loss_and_decisions("means", 0, 0.0)
    rng = np.random.default_rng(1)
    checked = flipped = 0
    for name in ("means", "log_scales", "quats", "logits", "sh"):
        g = grads[name].reshape(-1)
        scale = np.abs(g).max()
        idxs = rng.choice(g.size, size=min(g.size, 24), replace=False)
        for idx in idxs:
            h = 1e-3
            lp, np_, lastp = loss_and_decisions(name, int(idx), h)
            lm, nm, lastm = loss_and_decisions(name, int(idx), -h)
            if not (np.array_equal(np_, base_n) and np.array_equal(nm, base_n) and
                    np.array_equal(lastp, base_last) and np.array_equal(lastm, base_last)):
                flipped += 1
                continue
            fd = (lp - lm) / (2 * h)
            checked += 1
            assert abs(fd - g[idx]) <= 2e-2 * abs(g[idx]) + 2e-3 * scale, \
                f"{kernel}/{name}[{idx}]: finite difference {fd:.6g} against backward {g[idx]:.6g}"
    assert checked >= 0.8 * (checked + flipped), f"only {checked} of {checked + flipped} samples were smooth"


def test_asynchronous_rasterizer_matches_and_reports_overflow():
    """sync=False: no synchronisation per forward.  With room for the lists, the images, lists and
    the autograd gradients' forward equal the synchronous rasterizer's bit for bit and check()
    passes; with too small a capacity check() raises DARB_ERR_CAPACITY with the instance count
    the view needs, after two forwards (the first one fitting)."""
    s = synth.cluster_scene(20000, seed=5, sh_degree=3)
    cam = synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[3]
    sd = darb.splats_to_device(s)
    r_sync = darb.Rasterizer(cam, "half_cosine", 16)
    proj_a, bins_a, img_a = r_sync.forward(sd, owned=True)
    torch.cuda.synchronize()
    M = bins_a.M
    r_async = darb.Rasterizer(cam, "half_cosine", 16, capacity=r_sync.capacity, sync=False)
    proj_b, bins_b, img_b = r_async.forward(sd, owned=True)
    r_async.check()
    assert bins_b.M is None and int(bins_b.num_instances[0]) == M
    assert torch.equal(bins_a.values[:M], bins_b.values[:M]) and torch.equal(bins_a.ranges, bins_b.ranges)
    assert torch.equal(img_a.image, img_b.image) and torch.equal(img_a.last, img_b.last)
    # too small for the second view: the deferred check names the overflow and the count needed
    small = darb.Rasterizer(cam, "half_cosine", 16, capacity=M - 1, sync=False)
    tiny = darb.splats_to_device(synth.cluster_scene(50, seed=6, sh_degree=3))
    small.forward(tiny)
    small.forward(sd)
    with pytest.raises(darb.DarbError) as e:
        small.check()
    assert e.value.status == 3 and e.value.M == M
    small.check()  # the pending list was cleared
