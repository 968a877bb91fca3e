"""Every launch shape of the tensor-core decoder computes every point the
same way, so all shapes the autotuner may pick must give bit-identical
outputs: tile pipelines per CTA, CTAs per SM, and one or two warpgroups per
tile pipeline (two threads per tile row splitting the encoding and the
epilogue columns), for the single-buffer and the batched (segment table)
kernels, in every operand precision."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2406_17782_gb300 import autotune
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

SHAPES = autotune.DECODER_CANDIDATES


@pytest.fixture(scope="module")
def frame(fab):
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.set_params(W.decoder_init(), W.encoder_init())
    lat = torch.from_numpy(W.random_latents(len(mats))).cuda()
    # ragged: a full tile count plus a tail, several tiles per CTA at 1-4 CTAs/SM
    g = GBuffer.from_numpy(W.subset(W.frame_gbuffer(), np.arange(0, 152 * 4 * 128 * 2 + 77)))
    yield lat, g
    fab.set_launch_config(0, 0, 0, 0)


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp8"])
def test_all_launch_shapes_agree_bitwise(fab, frame, prec):
    lat, g = frame
    fab.prepare_neural(lat, prec)
    fab.set_launch_config(0, 0, 0, 0)
    want_rgb, want_c = fab.shade_neural_prepared(g, prec, comps=True)
    fab.sync_status()
    for wg, ctas, h in SHAPES:
        fab.set_launch_config(ctas, wg, 0, h)
        rgb, comps = fab.shade_neural_prepared(g, prec, comps=True)
        fab.sync_status()
        assert torch.equal(rgb, want_rgb) and torch.equal(comps, want_c), (prec, wg, ctas, h)


@pytest.mark.parametrize("h", [1, 2])
def test_batched_kernel_with_two_warpgroups_per_tile(fab, frame, h):
    lat, _ = frame
    frame_host = W.frame_gbuffer()
    segs = []
    for k, n in enumerate([5000, 1, 129, 0, 4097, 70_000]):
        host = W.subset(frame_host, np.arange(1000 * k, 1000 * k + n))
        segs.append((GBuffer.from_numpy(host), torch.full((n, 3), float("nan"), device="cuda"),
                     torch.full((n, 4), float("nan"), device="cuda")))
    fab.prepare_neural(lat, "fp16")
    fab.set_launch_config(0, 0, 0, h)
    plan = fab.plan(segs)
    plan.shade("fp16")
    fab.sync_status()
    fab.set_launch_config(0, 0, 0, 0)
    for g, rgb, comps in segs:
        if g.n == 0:
            continue
        want_rgb, want_c = fab.shade_neural_prepared(g, "fp16", comps=True)
        fab.sync_status()
        assert torch.equal(rgb, want_rgb) and torch.equal(comps, want_c)
    plan.close()
