"""fabric_shade_neural_noalloc: neural shading for callers that may not
allocate device memory while drawing (e.g. a frame captured into a CUDA
graph, or a host application that forbids plug-in allocations).  Its output
must match fabric_shade_neural within the decoder tests' tolerance, call
after call, although every call reuses the same static scratch array."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from paper_2406_17782_gb300._abi import PREC, FabricError, check
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

TOL = 5e-3    # relative L2, as for the FP16 decoder against the FP64 oracle


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def call_noalloc(fab, g: GBuffer, latents, prec, rgb, comps):
    gs = g.struct()
    return fab.lib.fabric_shade_neural_noalloc(fab.h, ctypes.byref(gs), ctypes.c_void_p(latents.data_ptr()),
                                               PREC[prec], ctypes.c_void_p(rgb.data_ptr()),
                                               ctypes.c_void_p(comps.data_ptr()),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp8"])
def test_noalloc_matches_allocating_call_twice(fab, prec):
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.set_params(W.decoder_init(), W.encoder_init())
    lat = torch.from_numpy(W.random_latents(len(mats))).cuda()
    g = GBuffer.from_numpy(W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 50_000, stream="noalloc")))
    want_rgb, want_c = fab.shade_neural(g, lat, prec, comps=True)
    fab.sync_status()
    for call in range(2):
        rgb = torch.full((g.n, 3), float("nan"), device="cuda")
        comps = torch.full((g.n, 4), float("nan"), device="cuda")
        check(call_noalloc(fab, g, lat, prec, rgb, comps), fab.h)
        fab.sync_status()
        assert rel_l2(rgb.cpu().numpy(), want_rgb.cpu().numpy()) <= TOL, call
        assert rel_l2(comps.cpu().numpy(), want_c.cpu().numpy()) <= TOL, call


def test_noalloc_rejects_what_it_cannot_hold(fab):
    mats = W.frame_materials()
    g = GBuffer.from_numpy(W.subset(W.frame_gbuffer(), np.arange(0, 256)))
    rgb = torch.empty((256, 3), device="cuda")
    comps = torch.empty((256, 4), device="cuda")
    fab.set_materials(np.concatenate([mats] * 12))             # 96 materials: over the decoder's limit
    lat = torch.from_numpy(W.random_latents(96)).cuda()
    assert call_noalloc(fab, g, lat, "fp16", rgb, comps) == 6
    fab.set_materials(mats)
    lat = torch.from_numpy(W.random_latents(len(mats))).cuda()
    assert call_noalloc(fab, g, lat, "fp32", rgb, comps) == 1  # no tensor-core path, no scratch
