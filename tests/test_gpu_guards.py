"""Out-of-bounds writes, caught without a memory checker: every buffer the library writes is
carved out of a larger allocation whose bytes before and after it hold a fill pattern, and
every input buffer is compared before and after.  The whole path runs through the C ABI on
ragged sizes (splat counts and image sides that are no multiple of any block or tile size),
for every tile size, both sort strategies, the no-alloc sort, the fused and the separate
backward, both losses and a batch of views; afterwards no guard byte may have changed and
no input may differ."""
import types

import numpy as np
import pytest
import torch

from paper_2501_12369_gb300 import darb, synth

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

GUARD = 4096     # bytes on each side (a multiple of 256 keeps the payload aligned)
PATTERN = 0xA5


class Arena:
    """Device buffers with guard bytes around them."""

    def __init__(self):
        self.bufs = []

    def empty(self, shape, dtype, name, fill=None):
        shape = (shape,) if isinstance(shape, int) else tuple(shape)
        item = torch.empty((), dtype=dtype).element_size()
        nbytes = int(np.prod(shape)) * item
        raw = torch.full((GUARD + nbytes + GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
        t = raw[GUARD:GUARD + nbytes].view(dtype).view(shape)
        if fill is not None:
            t.fill_(fill)
        self.bufs.append((name, raw, nbytes))
        return t

    def like(self, src, name):
        t = self.empty(src.shape, src.dtype, name)
        t.copy_(src)
        return t

    def violations(self):
        torch.cuda.synchronize()
        bad = []
        for name, raw, nbytes in self.bufs:
            head, tail = raw[:GUARD], raw[GUARD + nbytes:]
            if bool((head != PATTERN).any()) or bool((tail != PATTERN).any()):
                bad.append(name)
        return bad


class Inputs:
    """Copies of the inputs, to check afterwards that nothing wrote to them."""

    def __init__(self):
        self.saved = []

    def keep(self, name, t):
        self.saved.append((name, t, t.detach().clone()))
        return t

    def changed(self):
        torch.cuda.synchronize()
        return [name for name, t, c in self.saved if not torch.equal(t, c)]


def _projected(A, n, tag):
    return darb.Projected(A.empty(n, torch.float32, tag + ".depth"), A.empty(n, torch.int32, tag + ".radius"),
                          A.empty((n, 4), torch.int32, tag + ".tile_rect"),
                          A.empty((n, 2), torch.float32, tag + ".mean2d"),
                          A.empty((n, 4), torch.float32, tag + ".conic_o"), A.empty((n, 3), torch.float32, tag + ".rgb"),
                          A.empty(n, torch.uint8, tag + ".clamped"), A.empty(n, torch.int32, tag + ".tiles_touched"),
                          A.empty(n, torch.int64, tag + ".tile_runs"))


def _binning(A, cap, n_tiles, tag):
    return darb.Binning(A.empty(cap, torch.int64, tag + ".keys"), A.empty(cap, torch.int32, tag + ".values"),
                        A.empty((n_tiles, 2), torch.int32, tag + ".ranges"),
                        A.empty(1, torch.int32, tag + ".num", fill=0), A.empty(1, torch.int32, tag + ".status", fill=0))


def _image(A, W, H, tag, image=True, counts=True):
    return darb.ImageOut(A.empty((3, H, W), torch.float32, tag + ".image") if image else None,
                         A.empty((H, W), torch.float32, tag + ".t_final"), A.empty((H, W), torch.int32, tag + ".last"),
                         A.empty((H, W), torch.int32, tag + ".n_contrib") if counts else None)


LRS = dict(means=1.6e-4, scales=5e-3, quats=1e-3, opacities=0.02, sh_dc=2.5e-3, sh_rest=2.5e-3 / 20)


def _adam_cfg(step):
    return darb.darb_adam_config(LRS["means"], LRS["scales"], LRS["quats"], LRS["opacities"], LRS["sh_dc"],
                                 LRS["sh_rest"], 0.9, 0.999, 1e-15, step)


@pytest.mark.parametrize("n,deg,kernel", [(3001, 3, "half_cosine"), (2049, 1, "gaussian"), (777, 0, "raised_cosine")])
def test_no_write_outside_any_buffer(n, deg, kernel):
    A, I = Arena(), Inputs()
    s = synth.cluster_scene(n, seed=n, sh_degree=deg)
    cam = synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[5]
    W, H = cam.width, cam.height
    sd0 = darb.splats_to_device(s)
    sd = darb.SplatTensors(*(I.keep(f, A.like(getattr(sd0, f), f)) for f in ("means", "scales", "quats",
                                                                              "opacities", "sh")), deg)
    kp = darb.darb_kernel_defaults(kernel)
    target = I.keep("target", A.like(torch.rand(3, H, W, device="cuda", generator=torch.Generator("cuda").manual_seed(1)),
                                      "target"))
    for tile in (8, 16, 32):
        tag = f"t{tile}"
        tx, ty = darb.darb_tile_grid(cam, tile)
        proj = darb.darb_preprocess(sd, cam, kp, tile, out=_projected(A, n, tag))
        cap = 64 * n + 4096
        for strategy in (darb.DARB_SORT_DEPTH_THEN_TILE, darb.DARB_SORT_KEYS64):
            st = f"{tag}.s{strategy}"
            ws = A.empty(darb.darb_bin_sort_workspace_size(n, tile, cam, cap, strategy), torch.uint8, st + ".ws")
            bins = darb.darb_bin_sort(proj, n, tile, cam, ws, cap, out=_binning(A, cap, tx * ty, st), sync=True,
                                      strategy=strategy)
            assert 0 < bins.M <= cap
        na = darb.darb_bin_sort_noalloc(proj, n, tile, cam, cap, out=_binning(A, cap, tx * ty, tag + ".noalloc"))
        assert na.M == bins.M
        img = darb.darb_render_fwd(proj, bins, cam, kp, tile, out=_image(A, W, H, tag + ".fwd"))
        dL = A.empty((3, H, W), torch.float32, tag + ".dL")
        loss = A.empty(1, torch.float32, tag + ".loss")
        darb.darb_l1_loss(img.image, target, dL_dimage=dL, loss=loss)
        out_l1, dL2, _ = darb.darb_render_fwd_l1(proj, bins, cam, kp, tile, target,
                                                 out=_image(A, W, H, tag + ".fwdl1", image=False, counts=False),
                                                 dL_dimage=A.empty((3, H, W), torch.float32, tag + ".dL2"),
                                                 loss=A.empty(1, torch.float32, tag + ".loss2"))
        ssim_ws = A.empty(darb.darb_l1_dssim_workspace_size(W, H), torch.uint8, tag + ".ssim_ws")
        darb.darb_l1_dssim_loss(img.image, target, 0.2, workspace=ssim_ws,
                                dL_dimage=A.empty((3, H, W), torch.float32, tag + ".dLs"),
                                loss=A.empty(2, torch.float32, tag + ".loss_s"))
        g2 = darb.darb_render_bwd(proj, n, bins, cam, kp, tile, img, dL,
                                  grad2d=A.empty((n, 12), torch.float32, tag + ".grad2d"))
        k = (deg + 1) ** 2
        grads = darb.SplatGrads(A.empty((n, 3), torch.float32, tag + ".dmeans"),
                                A.empty((n, 3), torch.float32, tag + ".dscales"),
                                A.empty((n, 4), torch.float32, tag + ".dquats"),
                                A.empty(n, torch.float32, tag + ".dopac"),
                                A.empty((n, k, 3), torch.float32, tag + ".dsh"))
        darb.darb_preprocess_bwd(sd, cam, kp, proj, g2, out=grads)
        # the optimiser's in-place buffers: parameters, activated copies and moments
        mk = lambda shape, name, fill: A.empty(shape, torch.float32, f"{tag}.{name}", fill=fill)
        shapes = dict(means=(n, 3), scales=(n, 3), quats=(n, 4), opac=(n,), sh=(n, k, 3))
        for fused in (False, True):
            ft = f"{tag}.f{int(fused)}"
            params = types.SimpleNamespace(
                means=A.like(sd.means, ft + ".means"), log_scales=A.like(torch.log(sd.scales), ft + ".log_scales"),
                quats=A.like(sd.quats, ft + ".quats"),
                opacity_logits=A.like(torch.logit(sd.opacities), ft + ".logits"), sh=A.like(sd.sh, ft + ".sh"),
                scales=A.like(sd.scales, ft + ".scales"), opacities=A.like(sd.opacities, ft + ".opacities"),
                sh_degree=deg)
            state = types.SimpleNamespace(**{f"{m}_{g}": mk(shape, f"f{int(fused)}.{m}_{g}", 0.0)
                                             for g, shape in shapes.items() for m in ("m", "v")})
            if fused:
                darb.darb_preprocess_bwd_adam(params, cam, kp, proj, g2, state, _adam_cfg(1))
            else:
                darb.darb_adam_step(params, grads, state, _adam_cfg(1))
    # a batch of views of ragged sizes
    cams = [synth.pinhole((0.0, 0.0, 6.0 + 0.5 * j), 161 + 40 * j, 97 + 31 * j, 150.0) for j in range(3)]
    bp = darb.darb_batch_params(len(cams), 16, 2, 0, 64 * n + 4096)
    bws = A.empty(darb.darb_render_batch_workspace_size(n, cams, bp), torch.uint8, "batch.ws")
    outs = [_image(A, c.width, c.height, f"batch.v{j}") for j, c in enumerate(cams)]
    num = A.empty(len(cams), torch.int32, "batch.num", fill=0)
    stat = A.empty(len(cams), torch.int32, "batch.status", fill=0)
    darb.darb_render_batch(sd, cams, kp, bp, bws, outs, num_instances=num, status=stat)
    torch.cuda.synchronize()
    assert int(stat.abs().sum()) == 0 and int(num.min()) > 0
    assert A.violations() == []
    assert I.changed() == []
