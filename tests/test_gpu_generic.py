"""Table 1's modified DARB members (kind DARB_GENERIC) on the GPU: psi by the device moment
integral against the oracle's quadrature, and forward / backward compositing against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2501_12369_gb300 import darb, synth

from gpu_helpers import ambiguity_masked_grad, check_render, gpu_forward, grad_close, to_np

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

MEMBERS = [("half_cosine", 3.0, 1.5, 1), ("raised_cosine", 1.2, 2.0, 1), ("mod_sinc", 1.1, 1.5, 2),
           ("gaussian", 1.0, 2.5, 1), ("inv_multiquadric", 0.7, 2.0, 1), ("parabola", 4.0, 2.0, 1)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_12369_gb300 import build
    build.build()
    oracle.build()


def _pair(member):
    """The same member for both sides (the oracle's psi, checked equal parameters)."""
    base, xi, beta, lobes = member
    ko = oracle.generic_kernel(base, xi, beta, lobes)
    kg = darb.darb_kernel_generic(base, xi, beta, lobes, psi=ko.psi)
    assert kg.q_max == ko.q_max and kg.psi == ko.psi
    return kg, ko


@pytest.mark.parametrize("member", MEMBERS)
def test_psi_on_device_matches_the_quadrature(member):
    kg, ko = _pair(member)
    assert darb.darb_kernel_psi(kg) == pytest.approx(oracle.psi_moment(ko), rel=2e-6)


@pytest.mark.parametrize("name", oracle.KERNEL_NAMES)
def test_psi_on_device_for_the_fixed_kernels(name):
    kp = darb.darb_kernel_defaults(name)
    ko = oracle.kernel_params(name)
    assert darb.darb_kernel_psi(kp) == pytest.approx(oracle.psi_moment(ko), rel=2e-6)


@pytest.mark.parametrize("member", MEMBERS)
def test_generic_render_forward_matches_oracle(member):
    kg, ko = _pair(member)
    s, cam = synth.small_forward_workload()
    r, sd, proj, bins, img = gpu_forward(s, cam, kg, 16)
    check_render(img, bins, oracle.forward(s, cam, ko, tile=16), cam, 16)
    s = synth.cluster_scene(20000, seed=5)
    cam = synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[3]
    r, sd, proj, bins, img = gpu_forward(s, cam, kg, 32)
    check_render(img, bins, oracle.forward(s, cam, ko, tile=32), cam, 32)


@pytest.mark.parametrize("member", MEMBERS[:4])
def test_generic_gradients_match_oracle(member):
    kg, ko = _pair(member)
    s = synth.cluster_scene(8000, seed=5)
    cam = synth.fibonacci_cameras(16, 6.0, 333, 207, 260.0)[3]
    r, sd, proj, bins, img = gpu_forward(s, cam, kg, 16)
    dl = synth.random_image_grad(cam.height, cam.width, seed=3)
    ref_f = oracle.forward(s, cam, ko, tile=16)
    dl = ambiguity_masked_grad(dl, ref_f["amb"])
    g, g2 = r.backward(sd, proj, bins, img, torch.from_numpy(dl.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    _, g2_ref, gp_ref = oracle.gradients(s, cam, dl.astype(np.float32).astype(np.float64), ko, tile=16)
    for name, got in (("means", g.dmeans), ("scales", g.dscales), ("quats", g.dquats),
                      ("opacities", g.dopacities), ("sh", g.dsh)):
        grad_close(f"{member}/{name}", to_np(got), gp_ref[name])


def test_generic_member_in_a_batch_equals_single_views():
    kg, _ = _pair(MEMBERS[0])
    sd = darb.splats_to_device(synth.cluster_scene(20000, seed=2))
    cams = synth.random_pose_cameras(4, 6.0, ((160, 90), (96, 200)), 0.8, seed=3)
    br = darb.BatchRenderer(sd, cams, kg, 16, 2)
    br.render()
    torch.cuda.synchronize()
    br.check()
    for c, out in zip(cams, br.outs):
        _, _, single = darb.Rasterizer(c, kg, 16).forward(sd)
        assert torch.equal(out.image, single.image)
