"""Training-step kernels through the C ABI against the oracle: the L1 term (Sec. 4.2), the Adam
step of the 3DGS optimiser (Sec. 5), and the fused preprocess backward + Adam entry point."""
import types

import numpy as np
import pytest
import torch

import oracle
from paper_2501_12369_gb300 import darb, synth

from gpu_helpers import gpu_forward, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

LRS = dict(means=1.6e-4 * 6.0, scales=5e-3, quats=1e-3, opacities=0.02, sh_dc=2.5e-3, sh_rest=2.5e-3 / 20)
RAW = ("means", "log_scales", "quats", "opacity_logits", "sh")
STATE_OF = dict(means="means", log_scales="scales", quats="quats", opacity_logits="opac", sh="sh")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()
    oracle.build()


def _cfg(step):
    return darb.darb_adam_config(LRS["means"], LRS["scales"], LRS["quats"], LRS["opacities"], LRS["sh_dc"],
                                 LRS["sh_rest"], 0.9, 0.999, 1e-15, step)


def _train_state(s, rng, warm, sigma=None):
    """Raw parameters of splats `s` and Adam moments: zero, or random as after a few steps with
    gradients of size sigma[k] (default 1e-3) for raw group k."""
    raw = dict(means=s.means.astype(np.float32), log_scales=np.log(s.scales).astype(np.float32),
               quats=s.quats.astype(np.float32),
               opacity_logits=np.log(s.opacities / (1 - s.opacities)).astype(np.float32),
               sh=s.sh.astype(np.float32))
    state = {}
    for k in RAW:
        shape = raw[k].shape
        if warm:
            sg = 1e-3 if sigma is None else sigma[k]
            state["m_" + k] = rng.normal(scale=sg, size=shape).astype(np.float32)
            state["v_" + k] = (sg * sg * rng.uniform(0.5, 2.0, size=shape)).astype(np.float32)
        else:
            state["m_" + k] = np.zeros(shape, np.float32)
            state["v_" + k] = np.zeros(shape, np.float32)
    return raw, state


def _to_device(raw, state, sh_degree):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    p = types.SimpleNamespace(**{k: t(v) for k, v in raw.items()}, sh_degree=sh_degree)
    p.scales = torch.exp(p.log_scales)
    p.opacities = torch.sigmoid(p.opacity_logits)
    st = types.SimpleNamespace(**{f"{m}_{STATE_OF[k]}": t(state[f"{m}_{k}"]) for k in RAW for m in ("m", "v")})
    return p, st


def _clone(p, st):
    p2 = types.SimpleNamespace(**{k: (v.clone() if torch.is_tensor(v) else v) for k, v in vars(p).items()})
    st2 = types.SimpleNamespace(**{k: v.clone() for k, v in vars(st).items()})
    return p2, st2


def _f32(x):
    return float(np.float32(x))


def _oracle_adam(p, st, grads, step):
    """Oracle Adam from the device tensors' current values (read back as float64), with the
    hyper-parameters the kernels receive: the float32 values of 0.9, 0.999, 1e-15 and the
    learning rates (1 - float32(0.999) is 1.3e-5 off 0.001, which v shows)."""
    raw = {k: to_np(getattr(p, k)).astype(np.float64) for k in RAW}
    state = {f"{m}_{k}": to_np(getattr(st, f"{m}_{STATE_OF[k]}")).astype(np.float64) for k in RAW for m in ("m", "v")}
    return oracle.adam_step_splats(raw, grads, state, {k: _f32(v) for k, v in LRS.items()}, step,
                                   _f32(0.9), _f32(0.999), _f32(1e-15))


def _lr_of(k, shape):
    if k == "sh":
        lr = np.full(shape, LRS["sh_rest"])
        lr[:, 0, :] = LRS["sh_dc"]
        return lr
    return dict(means=LRS["means"], log_scales=LRS["scales"], quats=LRS["quats"],
                opacity_logits=LRS["opacities"])[k]


def _check_adam(p0, p, st, ref_raw, ref_state, upd_rtol, mom_tol):
    """Updates (p' - p) within upd_rtol of the learning rate, moments within mom_tol (relative,
    and of the group's largest moment), activated copies equal to exp / sigmoid of the new raw
    values."""
    for k in RAW:
        before, after = to_np(getattr(p0, k)).astype(np.float64), to_np(getattr(p, k)).astype(np.float64)
        lr = _lr_of(k, before.shape)
        err = np.abs((after - before) - (ref_raw[k] - before))
        bound = upd_rtol * lr + 2e-7 * np.abs(before)
        assert np.all(err <= bound), f"{k}: worst update error {np.max(err / bound):.3g} x bound"
        for m in ("m", "v"):
            got = to_np(getattr(st, f"{m}_{STATE_OF[k]}")).astype(np.float64)
            ref = ref_state[f"{m}_{k}"]
            scale = np.max(np.abs(ref)) + 1e-30
            np.testing.assert_allclose(got, ref, rtol=mom_tol, atol=mom_tol * scale, err_msg=f"{m}_{k}")
    # expf within 2 ulp; the sigmoid adds the rounding of 1 + e and of the division
    np.testing.assert_allclose(to_np(p.scales), np.exp(to_np(p.log_scales).astype(np.float64)), rtol=5e-7)
    np.testing.assert_allclose(to_np(p.opacities), 1 / (1 + np.exp(-to_np(p.opacity_logits).astype(np.float64))),
                               rtol=6e-7, atol=1e-12)


# --------------------------------------------------------------------------- L1 term

@pytest.mark.parametrize("W,H", [(333, 207), (1, 1), (64, 64)])
def test_l1_loss_matches_oracle(W, H):
    rng = np.random.default_rng(W * 7 + H)
    img = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tgt = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tgt.reshape(-1)[::5] = img.reshape(-1)[::5]  # exact ties: zero gradient
    dL, loss = darb.darb_l1_loss(torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda())
    torch.cuda.synchronize()
    ref_loss, ref_dl = oracle.l1_loss(img, tgt)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * max(ref_loss, 1e-30)
    got = to_np(dL).astype(np.float64)
    assert np.array_equal(np.sign(got), np.sign(ref_dl))
    np.testing.assert_allclose(got, ref_dl, rtol=1e-7)


@pytest.mark.parametrize("kernel,tile", [("half_cosine", 32), ("gaussian", 16), ("parabola", 8)])
def test_forward_with_l1_equals_forward_then_l1(kernel, tile):
    """darb_render_fwd_l1 (the loss taken in the compositing kernel's epilogue) against
    darb_render_fwd followed by darb_l1_loss: every image output and the loss gradient bit for
    bit, the loss up to the order of its FP32 sums; a ragged 333x207 view and a tiny one."""
    for s, cam in ((synth.cluster_scene(20000, seed=5), synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[3]),
                   (synth.uniform_cube_scene(300, seed=9), synth.pinhole((0.2, 0.1, 3.5), 17, 33, 18.0))):
        r, sd, proj, bins, img = gpu_forward(s, cam, kernel, tile)
        target = torch.from_numpy(synth.random_target(cam.height, cam.width, seed=4)).cuda()
        dL, loss = darb.darb_l1_loss(img.image, target)
        out, dL2, loss2 = darb.darb_render_fwd_l1(proj, bins, cam, r.kparams, tile, target)
        torch.cuda.synchronize()
        for a, b in ((img.image, out.image), (img.t_final, out.t_final), (img.last, out.last),
                     (img.n_contrib, out.n_contrib), (dL, dL2)):
            assert torch.equal(a, b)
        assert abs(float(loss2[0]) - float(loss[0])) <= 1e-5 * abs(float(loss[0]))
        ref, _ = oracle.l1_loss(to_np(img.image), to_np(target))
        assert abs(float(loss2[0]) - ref) <= 1e-5 * ref


def test_forward_with_l1_without_image_and_counts():
    """darb_render_fwd_l1 with the image and the contributor counts left out (what a training
    step needs): t_final, last and the loss gradient as with every output, bit for bit."""
    s, cam = synth.cluster_scene(20000, seed=6), synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[5]
    r, sd, proj, bins, img = gpu_forward(s, cam, "half_cosine", 32)
    target = torch.from_numpy(synth.random_target(cam.height, cam.width, seed=5)).cuda()
    full, dL, loss = darb.darb_render_fwd_l1(proj, bins, cam, r.kparams, 32, target)
    lean = darb.ImageOut(None, torch.empty_like(full.t_final), torch.empty_like(full.last), None)
    _, dL2, loss2 = darb.darb_render_fwd_l1(proj, bins, cam, r.kparams, 32, target, out=lean)
    torch.cuda.synchronize()
    assert torch.equal(full.t_final, lean.t_final) and torch.equal(full.last, lean.last)
    assert torch.equal(dL, dL2)
    assert abs(float(loss2[0]) - float(loss[0])) <= 1e-5 * abs(float(loss[0]))


def test_l1_loss_on_buffers_off_a_16_byte_boundary():
    # the float4 lanes need all three buffers aligned; views 4 bytes in take the one-by-one path
    W, H = 97, 31
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tgt = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    n = img.size
    bi, bt, bd = (torch.empty(n + 1, device="cuda") for _ in range(3))
    bi[1:] = torch.from_numpy(img.reshape(-1)).cuda()
    bt[1:] = torch.from_numpy(tgt.reshape(-1)).cuda()
    loss = torch.empty(1, device="cuda")
    dL, loss = darb.darb_l1_loss(bi[1:].view(3, H, W), bt[1:].view(3, H, W), dL_dimage=bd[1:].view(3, H, W),
                                 loss=loss)
    torch.cuda.synchronize()
    ref_loss, ref_dl = oracle.l1_loss(img, tgt)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * ref_loss
    np.testing.assert_allclose(to_np(dL).astype(np.float64), ref_dl, rtol=1e-7)


# --------------------------------------------------------------------------- Adam

@pytest.mark.parametrize("step", [1, 7])
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_adam_step_matches_oracle(deg, step):
    """n = 1003: no multiple of 4 or of a block, so every float4 group has a scalar tail."""
    s = synth.uniform_cube_scene(1003, seed=deg, sh_degree=deg)
    rng = np.random.default_rng(10 + deg)
    raw, state = _train_state(s, rng, warm=step > 1)
    p, st = _to_device(raw, state, deg)
    p0, _ = _clone(p, st)
    grads = dict(means=rng.normal(size=s.means.shape), scales=rng.normal(size=s.scales.shape),
                 quats=rng.normal(size=s.quats.shape), opacities=rng.normal(size=s.opacities.shape),
                 sh=rng.normal(size=s.sh.shape))
    grads = {k: (1e-3 * v).astype(np.float32) for k, v in grads.items()}
    grads["means"][::17] = 0.0  # zero gradients: the moments decay, the step is m-driven
    ref_raw, ref_state = _oracle_adam(p, st, {k: v.astype(np.float64) for k, v in grads.items()}, step)
    g = darb.SplatGrads(*(torch.from_numpy(grads[k]).cuda() for k in ("means", "scales", "quats", "opacities", "sh")))
    darb.darb_adam_step(p, g, st, _cfg(step))
    torch.cuda.synchronize()
    _check_adam(p0, p, st, ref_raw, ref_state, upd_rtol=1e-5, mom_tol=2e-6)


# --------------------------------------------------------------------------- fused backward + Adam

def _fused_case(kernel, deg, n=3001, seed=4):
    s = synth.cluster_scene(n, seed=seed, sh_degree=deg)
    cam = synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[3]
    r, sd, proj, bins, img = gpu_forward(s, cam, kernel, 16)
    rng = np.random.default_rng(seed + deg)
    g2 = np.zeros((n, 12), np.float32)
    g2[:, :9] = rng.normal(size=(n, 9))  # culled splats too: both paths must ignore them
    return s, cam, r, sd, proj, torch.from_numpy(g2).cuda(), rng


@pytest.mark.parametrize("kernel", ["half_cosine", "inv_quadric"])
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_fused_backward_adam_equals_separate(kernel, deg):
    s, cam, r, sd, proj, g2, rng = _fused_case(kernel, deg)
    assert int((proj.radius == 0).sum()) > 0, "the case should hold culled splats"
    raw, state = _train_state(s, rng, warm=True)
    pa, sa = _to_device(raw, state, deg)
    pb, sb = _clone(pa, sa)
    sd_a = darb.SplatTensors(pa.means, pa.scales, pa.quats, pa.opacities, pa.sh, deg)
    grads = darb.darb_preprocess_bwd(sd_a, cam, r.kparams, proj, g2)
    darb.darb_adam_step(pa, grads, sa, _cfg(3))
    darb.darb_preprocess_bwd_adam(pb, cam, r.kparams, proj, g2, sb, _cfg(3))
    torch.cuda.synchronize()
    for k in list(RAW) + ["scales", "opacities"]:
        a, b = to_np(getattr(pa, k)), to_np(getattr(pb, k))
        np.testing.assert_allclose(b, a, rtol=1e-6, atol=1e-7 * (np.max(np.abs(a)) + 1e-30), err_msg=k)
    for k in vars(sa):
        a, b = to_np(getattr(sa, k)), to_np(getattr(sb, k))
        np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-6 * (np.max(np.abs(a)) + 1e-30), err_msg=k)


@pytest.mark.parametrize("kernel", ["half_cosine", "mod_sinc"])
def test_fused_backward_adam_matches_oracle(kernel):
    deg = 3
    s, cam, r, sd, proj, g2, rng = _fused_case(kernel, deg, n=2000, seed=9)
    ref_proj = oracle.project(s, cam, oracle.kernel_params(kernel), 16, True)
    g2_np = to_np(g2)[:, :9].astype(np.float64)
    g2_np[ref_proj["culled"] == 1] = 0.0
    gp = oracle.project_backward(s, ref_proj, cam, oracle.kernel_params(kernel), g2_np)
    o = s.opacities.astype(np.float64)
    chained = dict(means=gp["means"], log_scales=gp["scales"] * s.scales, quats=gp["quats"],
                   opacity_logits=gp["opacities"] * o * (1 - o), sh=gp["sh"])
    # moments of the gradients' own size: the step then depends smoothly on the gradient, so
    # the gradient tolerance (1e-3 relative, 1e-4 of the group maximum) bounds the update error
    raw, state = _train_state(s, rng, warm=True, sigma={k: float(np.max(np.abs(v))) for k, v in chained.items()})
    p, st = _to_device(raw, state, deg)
    p0, _ = _clone(p, st)
    ref_raw, ref_state = _oracle_adam(p, st, gp, 3)
    darb.darb_preprocess_bwd_adam(p, cam, r.kparams, proj, g2, st, _cfg(3))
    torch.cuda.synchronize()
    _check_adam(p0, p, st, ref_raw, ref_state, upd_rtol=1e-3, mom_tol=2e-3)


def test_fused_backward_adam_argument_checks():
    s, cam, r, sd, proj, g2, rng = _fused_case("half_cosine", 1, n=64)
    raw, state = _train_state(s, rng, warm=False)
    p, st = _to_device(raw, state, 1)
    with pytest.raises(darb.DarbError):
        darb.darb_preprocess_bwd_adam(p, cam, r.kparams, proj, g2.reshape(-1)[1:], st, _cfg(1))  # off 16 B
    with pytest.raises(darb.DarbError):
        darb.darb_preprocess_bwd_adam(p, cam, r.kparams, proj, g2, st, _cfg(0))  # steps count from 1
    shifted, _ = _clone(p, st)
    buf = torch.empty(p.means.numel() + 1, device="cuda")
    shifted.means = buf[1:].view_as(p.means)  # 4 B past a 16-byte boundary: the float4 lanes need it
    with pytest.raises(darb.DarbError):
        darb.darb_preprocess_bwd_adam(shifted, cam, r.kparams, proj, g2, st, _cfg(1))


# --------------------------------------------------------------------------- L1 + D-SSIM term

@pytest.mark.parametrize("W,H", [(333, 207), (64, 64), (17, 23), (1, 1)])
def test_l1_dssim_matches_oracle(W, H):
    rng = np.random.default_rng(W + 3 * H)
    img = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tgt = np.clip(img + rng.normal(0, 0.2, img.shape), 0, 1).astype(np.float32)  # correlated, like a render
    tgt.reshape(-1)[::7] = img.reshape(-1)[::7]
    dL, loss = darb.darb_l1_dssim_loss(torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), 0.2)
    torch.cuda.synchronize()
    ref_loss, ref_grad, ref_ssim = oracle.l1_dssim_loss(img, tgt, 0.2)
    got = to_np(loss)
    assert abs(got[0] - ref_loss) <= 2e-6 * max(1.0, abs(ref_loss))
    assert abs(got[1] - ref_ssim) <= 2e-6
    g = to_np(dL).astype(np.float64)
    np.testing.assert_allclose(g, ref_grad, rtol=1e-3, atol=1e-4 * np.abs(ref_grad).max())


def test_l1_dssim_special_cases():
    rng = np.random.default_rng(3)
    img = torch.from_numpy(rng.uniform(0, 1, (3, 40, 50)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(rng.uniform(0, 1, (3, 40, 50)).astype(np.float32)).cuda()
    # lambda = 0 is the L1 term alone
    dL0, loss0 = darb.darb_l1_dssim_loss(img, tgt, 0.0)
    dl1, l1 = darb.darb_l1_loss(img, tgt)
    torch.cuda.synchronize()
    assert torch.equal(dL0, dl1)
    assert float(loss0[0]) == pytest.approx(float(l1[0]), rel=1e-6)
    # an image against itself: D-SSIM 0, SSIM 1, gradient 0
    dLs, losss = darb.darb_l1_dssim_loss(img, img, 1.0)
    torch.cuda.synchronize()
    assert float(losss[1]) == pytest.approx(1.0, abs=1e-6) and abs(float(losss[0])) < 1e-6
    assert float(dLs.abs().max()) < 1e-9
    with pytest.raises(darb.DarbError):
        darb.darb_l1_dssim_loss(img, tgt, 1.5)
    small = torch.empty(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(darb.DarbError) as e:
        darb.darb_l1_dssim_loss(img, tgt, 0.2, workspace=small)
    assert e.value.status == 2


def test_l1_dssim_full_hd_crops():
    """1920 x 1080, the training resolution: gradients of three 96 x 96 windows against the
    oracle on the same window plus a 10-pixel margin (the gradient at a pixel depends on the
    image within 2 x 5 pixels, so the window's inner pixels are exact)."""
    rng = np.random.default_rng(11)
    H, W = 1080, 1920
    img = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tgt = np.clip(img + rng.normal(0, 0.1, img.shape), 0, 1).astype(np.float32)
    dL, loss = darb.darb_l1_dssim_loss(torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), 0.2)
    torch.cuda.synchronize()
    g = to_np(dL).astype(np.float64)
    n_full, m = 3 * H * W, 10
    for (y0, x0) in [(0, 0), (H - 96, W - 96), (500, 900)]:
        ya, xa = max(0, y0 - m), max(0, x0 - m)
        yb, xb = min(H, y0 + 96 + m), min(W, x0 + 96 + m)
        _, ref, _ = oracle.l1_dssim_loss(img[:, ya:yb, xa:xb], tgt[:, ya:yb, xa:xb], 0.2)
        ref = ref * (ref.size / n_full)  # the oracle normalised by the window's size
        sl = (slice(None), slice(y0 - ya, y0 - ya + 96), slice(x0 - xa, x0 - xa + 96))
        got = g[:, y0:y0 + 96, x0:x0 + 96]
        np.testing.assert_allclose(got, ref[sl], rtol=1e-3, atol=1e-4 * np.abs(ref[sl]).max())


def test_resume_from_checkpoint_equals_continuing(tmp_path):
    """One fused step, a checkpoint, then one more step, against the same second step taken
    from the reloaded checkpoint: parameters, activated copies and moments agree bit for bit
    (the fused step is a per-splat computation, so equal inputs give equal outputs)."""
    from paper_2501_12369_gb300 import checkpoint
    deg = 3
    s, cam, r, sd, proj, g2, rng = _fused_case("half_cosine", deg, n=2500, seed=21)
    raw, state = _train_state(s, rng, warm=False)
    p, st = _to_device(raw, state, deg)
    darb.darb_preprocess_bwd_adam(p, cam, r.kparams, proj, g2, st, _cfg(1))
    torch.cuda.synchronize()
    checkpoint.save_training(tmp_path / "ckpt.npz", p, st, step=1)
    darb.darb_preprocess_bwd_adam(p, cam, r.kparams, proj, g2, st, _cfg(2))
    p2, st2, step = checkpoint.load_training(tmp_path / "ckpt.npz", device="cuda")
    assert step == 1
    darb.darb_preprocess_bwd_adam(p2, cam, r.kparams, proj, g2, st2, _cfg(step + 1))
    torch.cuda.synchronize()
    for f in checkpoint.PARAM_FIELDS:
        assert torch.equal(getattr(p2, f), getattr(p, f)), f
    for f in checkpoint.STATE_FIELDS:
        assert torch.equal(getattr(st2, f), getattr(st, f)), f
