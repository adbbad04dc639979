"""Small, self-contained cases for profiling single kernels (for example under ncu).

    python profile_cases.py CASE [N] [TILE] [KERNEL]

CASE is one of
  render     two forward + backward passes (compositing kernels k_render_fwd / k_render_bwd)
  sort       two forward passes (the binning and sorting kernels, then compositing)
  train_tail fused preprocess backward + Adam and the separate pair, 3 warm-up iterations
             each, then 20 timed iterations of each (prints ms per iteration)
  ssim       three L1 + D-SSIM loss evaluations (k_ssim_fwd / k_ssim_bwd) of a seeded image
             against a seeded target, N pixels wide (16:9; default 3840 when N is not given)
  batch      two eager batched renders (k_render_fwd_batch) of 16 cameras of the 1M-splat
             mixed-resolution multi-view scene, 8 streams, TILE-pixel tiles
on N clustered splats (default 1,000,000, SH degree 3) seen by camera 0 of the 1920x1080
Fibonacci-sphere cameras (fx = 1500), with TILE-pixel tiles (default 32) and the kernel KERNEL
(default half_cosine) for the render and sort cases.  Inputs are seeded.
Each case launches a fixed sequence, so `ncu -k <kernel> -s <skip> -c <count>` selects the
same launches every run.
"""
from __future__ import annotations

import sys
import types

import torch

import os

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_2501_12369_gb300 import build, darb, synth  # noqa: E402


KERNEL = "half_cosine"


def _setup(n, tile):
    build.build()
    s = synth.cluster_scene(n, seed=0)
    cam = synth.fibonacci_cameras(100, 6.0, 1920, 1080, 1500.0)[0]
    r = darb.Rasterizer(cam, KERNEL, tile, capacity=40 * n)
    return s, cam, r, darb.splats_to_device(s)


def case_render(n, tile):
    s, cam, r, sd = _setup(n, tile)
    dL = torch.from_numpy(synth.random_image_grad(1080, 1920, seed=3) * 1e-6).cuda()
    for _ in range(2):
        proj, bins, img = r.forward(sd)
        r.backward(sd, proj, bins, img, dL)
    torch.cuda.synchronize()
    print("instances", bins.M)


def case_sort(n, tile):
    s, cam, r, sd = _setup(n, tile)
    for _ in range(2):
        proj, bins, img = r.forward(sd)
    torch.cuda.synchronize()
    print("instances", bins.M, "status", int(bins.status.item()))


def _train_state(sd):
    p = types.SimpleNamespace(means=sd.means.clone(), log_scales=torch.log(sd.scales), quats=sd.quats.clone(),
                              opacity_logits=torch.logit(sd.opacities), sh=sd.sh.clone(), scales=sd.scales.clone(),
                              opacities=sd.opacities.clone(), sh_degree=sd.sh_degree)
    like = dict(m_means="means", v_means="means", m_scales="means", v_scales="means", m_quats="quats",
                v_quats="quats", m_opac="opacities", v_opac="opacities", m_sh="sh", v_sh="sh")
    st = types.SimpleNamespace(**{f: torch.zeros_like(getattr(p, g)) for f, g in like.items()})
    return p, st


def case_train_tail(n, tile):
    s, cam, r, sd = _setup(n, tile)
    dL = torch.from_numpy(synth.random_image_grad(1080, 1920, seed=3) * 1e-6).cuda()
    pa, sa = _train_state(sd)
    pb, sb = _train_state(sd)
    cfg = darb.darb_adam_config(1e-3, 5e-3, 1e-3, 0.02, 2.5e-3, 1.25e-4, 0.9, 0.999, 1e-15, 1)
    proj, bins, img = r.forward(sd)
    g2 = darb.darb_render_bwd(proj, sd.n, bins, cam, r.kparams, tile, img, dL)
    grads = darb.SplatGrads.empty_like(sd)
    sdb = darb.SplatTensors(pb.means, pb.scales, pb.quats, pb.opacities, pb.sh, sd.sh_degree)

    def fused():
        darb.darb_preprocess_bwd_adam(pa, cam, r.kparams, proj, g2, sa, cfg)

    def separate():
        darb.darb_preprocess_bwd(sdb, cam, r.kparams, proj, g2, grads)
        darb.darb_adam_step(pb, grads, sb, cfg)

    for _ in range(3):
        fused()
        separate()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    for _ in range(20):
        fused()
    ev[1].record()
    for _ in range(20):
        separate()
    ev[2].record()
    torch.cuda.synchronize()
    print(f"splats {n}: fused {ev[0].elapsed_time(ev[1]) / 20:.4f} ms, "
          f"separate {ev[1].elapsed_time(ev[2]) / 20:.4f} ms per iteration")


def case_ssim(n, tile):
    build.build()
    W = n if n <= 16384 else 3840
    H = W * 9 // 16
    img = torch.from_numpy(synth.random_target(H, W, seed=1)).cuda()
    tgt = torch.from_numpy(synth.random_target(H, W, seed=2)).cuda()
    ws = torch.empty(darb.darb_l1_dssim_workspace_size(W, H), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        dL, loss = darb.darb_l1_dssim_loss(img, tgt, 0.2, workspace=ws)
    torch.cuda.synchronize()
    print(f"{W}x{H}: loss {float(loss[0]):.6f}, mean SSIM {float(loss[1]):.6f}")


def case_batch(n, tile):
    build.build()
    s, cams = synth.scene_1m_multiview(16)
    sd = darb.splats_to_device(s)
    br = darb.BatchRenderer(sd, cams, "half_cosine", tile, 8)
    for _ in range(2):
        br.render()
    torch.cuda.synchronize()
    br.check()
    print("views", len(cams), "instances", int(br.num_instances.sum()))


CASES = {"render": case_render, "sort": case_sort, "train_tail": case_train_tail, "ssim": case_ssim,
         "batch": case_batch}


def main(argv):
    if not argv or argv[0] not in CASES:
        raise SystemExit(__doc__)
    n = int(argv[1]) if len(argv) > 1 else (3840 if argv[0] == "ssim" else 1_000_000)
    tile = int(argv[2]) if len(argv) > 2 else 32
    global KERNEL
    KERNEL = argv[3] if len(argv) > 3 else KERNEL
    CASES[argv[0]](n, tile)


if __name__ == "__main__":
    main(sys.argv[1:])
