"""fabric_shade_neural_noalloc: neural shading for callers that may not
allocate device memory while drawing (e.g. a host application that owns all
device memory and forbids plug-ins to allocate at draw time).  It runs the
same operand packing and tensor-core decoder kernels as fabric_shade_neural,
only with its packed operands in a static array, so its outputs must equal
that call's bit for bit, call after call, although every call reuses and
overwrites the same array."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from paper_2406_17782_gb300._abi import PREC, FabricError, check
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu


def call_noalloc(fab, g: GBuffer, latents, prec, rgb, comps):
    gs = g.struct()
    return fab.lib.fabric_shade_neural_noalloc(fab.h, ctypes.byref(gs), ctypes.c_void_p(latents.data_ptr()),
                                               PREC[prec], ctypes.c_void_p(rgb.data_ptr()),
                                               ctypes.c_void_p(comps.data_ptr()),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_allocating_call_twice(fab):
    """Two calls in a row per precision, in an order that changes the
    array's layout from one precision to the next (E4M3 blobs are smaller
    than 16-bit ones), so stale bytes from an earlier call would show."""
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.set_params(W.decoder_init(), W.encoder_init())
    lat = torch.from_numpy(W.random_latents(len(mats))).cuda()
    g = GBuffer.from_numpy(W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 50_000, stream="noalloc")))
    for prec in ("fp8", "fp16", "bf16", "fp8"):
        want_rgb, want_c = fab.shade_neural(g, lat, prec, comps=True)
        fab.sync_status()
        for call in range(2):
            rgb = torch.full((g.n, 3), float("nan"), device="cuda")
            comps = torch.full((g.n, 4), float("nan"), device="cuda")
            check(call_noalloc(fab, g, lat, prec, rgb, comps), fab.h)
            fab.sync_status()
            assert torch.equal(rgb, want_rgb), (prec, call)
            assert torch.equal(comps, want_c), (prec, call)


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
