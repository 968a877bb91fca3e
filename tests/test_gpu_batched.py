"""Batched draws: one persistent launch over many G-buffer segments (a view
plus ragged tiles) must equal per-segment draws bit for bit, also when the
launch is captured in a CUDA graph and replayed."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mlp as M
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prepared(fab):
    mats = W.frame_materials()
    fab.set_materials(mats)
    dec = W.decoder_init()
    fab.set_params(dec, W.encoder_init())
    z = W.random_latents(len(mats))
    lat = torch.from_numpy(z).cuda()
    return mats, dec, z, lat


def make_segments(sizes, seed=0):
    frame = W.frame_gbuffer()
    rng = np.random.default_rng(seed)
    segs = []
    for n in sizes:
        start = int(rng.integers(0, len(frame["u"]) - n - 1))
        host = W.subset(frame, np.arange(start, start + n))
        g = GBuffer.from_numpy(host)
        segs.append((host, g, torch.full((n, 3), float("nan"), device="cuda"),
                     torch.full((n, 4), float("nan"), device="cuda")))
    return segs


SIZES = [50_000, 1, 127, 128, 129, 0, 300, 4097, 65_536, 256, 999]


def test_plan_with_many_segments(fab, prepared):
    """3000 small segments (empty ones among them): the segment table no
    longer fits the spare shared memory, so the lookup reads it from global
    memory; the draw still equals per-segment draws bit for bit."""
    mats, dec, z, lat = prepared
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.choice(np.array([0, 1, 37, 128, 129, 300]), size=3000)]
    frame = W.frame_gbuffer()
    g_all = GBuffer.from_numpy(W.subset(frame, np.arange(0, sum(sizes))))
    segs, off = [], 0
    for n in sizes:
        g = GBuffer(*(getattr(g_all, k)[off:off + n] for k in ("u", "v", "radius", "wi", "wo", "material")))
        segs.append((g, torch.full((n, 3), float("nan"), device="cuda")))
        off += n
    fab.prepare_neural(lat, "fp16")
    plan = fab.plan([(g, rgb, None) for g, rgb in segs])
    plan.shade("fp16")
    fab.sync_status()
    want, _ = fab.shade_neural_prepared(g_all, "fp16")
    fab.sync_status()
    got = torch.cat([rgb for _, rgb in segs])
    assert torch.equal(got, want)


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp8"])
def test_plan_equals_per_segment_draws(fab, prepared, prec):
    mats, dec, z, lat = prepared
    segs = make_segments(SIZES)
    fab.prepare_neural(lat, prec)
    plan = fab.plan([(g, rgb, comps) for _, g, rgb, comps in segs])
    assert plan.points == sum(SIZES)
    plan.shade(prec)
    fab.sync_status()
    for host, g, rgb, comps in segs:
        if g.n == 0:
            continue
        want_rgb, want_c = fab.shade_neural_prepared(g, prec, comps=True)
        fab.sync_status()
        assert torch.equal(rgb, want_rgb) and torch.equal(comps, want_c)
    # one segment against the FP64 decoder (FP8: against its E4M3 emulation)
    host, g, rgb, comps = segs[0]
    P = M.unpack(dec, M.DEC_SHAPES)
    want_c, _ = M.shade_neural_e4m3(P, z, mats, host) if prec == "fp8" else M.shade_neural(P, z, mats, host)
    d = comps.cpu().numpy() - want_c
    assert np.sqrt((d ** 2).sum() / (want_c ** 2).sum()) < {"fp16": 5e-3, "bf16": 1.2e-2, "fp8": 2e-3}[prec]
    plan.close()


def test_plan_replays_from_cuda_graph(fab, prepared):
    mats, dec, z, lat = prepared
    segs = make_segments([20_000, 77, 5_000, 129], seed=1)
    fab.prepare_neural(lat, "fp16")
    plan = fab.plan([(g, rgb, comps) for _, g, rgb, comps in segs])
    plan.shade("fp16")
    torch.cuda.synchronize()
    first = [(rgb.clone(), comps.clone()) for _, _, rgb, comps in segs]
    for _, _, rgb, comps in segs:
        rgb.fill_(float("nan"))
        comps.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            plan.shade("fp16")
    for _, _, rgb, comps in segs:
        rgb.fill_(float("nan"))
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    fab.sync_status()
    for (want_rgb, want_c), (_, _, rgb, comps) in zip(first, segs):
        assert torch.equal(rgb, want_rgb) and torch.equal(comps, want_c)
    plan.close()


def test_plan_refuses_stale_state_and_takes_unaligned_outputs(fab, prepared):
    mats, dec, z, lat = prepared
    segs = make_segments([1000], seed=2)
    fab.prepare_neural(lat, "fp16")
    plan = fab.plan([(g, rgb, comps) for _, g, rgb, comps in segs])
    with pytest.raises(FabricError):
        plan.shade("bf16")                       # prepared for FP16 only
    fab.set_materials(mats)                      # invalidates the prepared state
    with pytest.raises(FabricError):
        plan.shade("fp16")
    plan.close()
    # components shifted by one float (not 16-byte aligned): accepted, four
    # 4-byte stores per point, bitwise the same values
    _, g, rgb, comps = segs[0]
    fab.prepare_neural(lat, "fp16")
    p1 = fab.plan([(g, rgb, comps)])
    p1.shade("fp16")
    fab.sync_status()
    want = comps.clone()
    p1.close()
    buf = torch.full((comps.numel() + 1,), float("nan"), dtype=torch.float32, device="cuda")
    shifted = buf[1:].view(comps.shape)
    p2 = fab.plan([(g, rgb, shifted)])
    p2.shade("fp16")
    fab.sync_status()
    assert shifted.data_ptr() % 16 != 0 and torch.equal(shifted, want)
    p2.close()
