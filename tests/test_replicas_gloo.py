"""Multi-rank host logic on CPU with gloo (world size 2): the bench's replica aggregation, and
the gradient exchange of data-parallel training over several views per step, simulated with
the oracle's gradients (one all-reduce of the flat per-splat gradient buffer before Adam)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))


def _aggregation_worker(rank, world, port, out):
    _init(rank, world, port)
    import bench
    w, r, local = bench.dist_env()
    assert (w, r, local) == (world, rank, rank)
    d = bench.dist_init(w, "gloo")
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slowest
        bench.barrier(d)
        ms_max = bench.max_over_ranks(d, ms, "cpu")
        out[rank] = (ms_max, bench.whole_job_rate(w, 40, ms_max))
    finally:
        d.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_aggregation_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ms_max, rate = out[rank]
        assert ms_max == 150.0
        assert rate == pytest.approx(2 * 40 / 0.150)  # units of every rank over the slowest time


def _views():
    from paper_2501_12369_gb300 import synth
    s = synth.uniform_cube_scene(256, seed=3)
    cams = [synth.pinhole((0.0, 0.0, 4.0), 32, 32, 40.0), synth.pinhole((1.5, 0.5, 3.5), 32, 24, 36.0)]
    return s, cams


def _oracle_grads(s, cam, seed):
    import oracle
    from paper_2501_12369_gb300 import synth
    dl = synth.random_image_grad(cam.height, cam.width, seed=seed)
    _, _, gp = oracle.gradients(s, cam, dl, "half_cosine", tile=16)
    return gp


def _exchange_worker(rank, world, port, out):
    _init(rank, world, port)
    import oracle
    from paper_2501_12369_gb300 import darb
    oracle.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, cams = _views()
        gp = _oracle_grads(s, cams[rank], seed=10 + rank)  # this rank's view
        g = darb.SplatGrads.empty_flat(s.n, s.sh_degree, device="cpu", dtype=torch.float64)
        for name, t in (("means", g.dmeans), ("scales", g.dscales), ("quats", g.dquats),
                        ("opacities", g.dopacities), ("sh", g.dsh)):
            t.copy_(torch.from_numpy(np.asarray(gp[name], np.float64).reshape(t.shape)))
        darb.allreduce_splat_grads(g)
        reduced = {k: v.numpy().copy() for k, v in (("means", g.dmeans), ("scales", g.dscales),
                                                     ("quats", g.dquats), ("opacities", g.dopacities),
                                                     ("sh", g.dsh))}
        # the same Adam step on every rank from the reduced gradient
        raw = dict(means=s.means.astype(np.float64), log_scales=np.log(s.scales.astype(np.float64)),
                   quats=s.quats.astype(np.float64),
                   opacity_logits=np.log(s.opacities / (1.0 - s.opacities)).astype(np.float64),
                   sh=s.sh.astype(np.float64))
        state = {f"{m}_{k}": np.zeros_like(raw[k]) for k in raw for m in ("m", "v")}
        lrs = dict(means=1e-3, scales=5e-3, quats=1e-3, opacities=0.02, sh_dc=2.5e-3, sh_rest=1.25e-4)
        new, _ = oracle.adam_step_splats(raw, reduced, state, lrs, 1)
        out[rank] = (reduced, new)
    finally:
        dist.destroy_process_group()


def test_gradient_allreduce_gives_the_summed_loss_gradient():
    import oracle
    oracle.build()
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_exchange_worker, args=(world, port, out), nprocs=world, join=True)
    s, cams = _views()
    expect = {}
    per_view = [_oracle_grads(s, cams[r], seed=10 + r) for r in range(world)]
    for name in ("means", "scales", "quats", "opacities", "sh"):
        expect[name] = sum(np.asarray(g[name], np.float64) for g in per_view)
        assert np.any(expect[name] != 0.0)
    for rank in range(world):
        reduced, new = out[rank]
        for name in expect:
            np.testing.assert_allclose(reduced[name].reshape(expect[name].shape), expect[name], rtol=1e-12,
                                       atol=1e-15, err_msg=f"rank {rank} {name}")
    # every rank applied the identical update
    for k in out[0][1]:
        np.testing.assert_array_equal(out[0][1][k], out[1][1][k])


def test_flat_gradient_views_are_aligned_and_disjoint():
    from paper_2501_12369_gb300 import darb
    for deg in range(4):
        g = darb.SplatGrads.empty_flat(1003, deg, device="cpu")
        views = [g.dmeans, g.dscales, g.dquats, g.dopacities, g.dsh]
        base = g.flat.data_ptr()
        ends = []
        for v in views:
            off = v.data_ptr() - base
            assert off % 16 == 0 and v.is_contiguous()
            ends.append((off, off + v.numel() * 4))
        for (a0, a1), (b0, b1) in zip(ends, ends[1:]):
            assert a1 <= b0
        assert ends[-1][1] <= g.flat.numel() * 4
