"""Output arrays that are float-aligned but not 16-byte aligned: the
[n][4] components take four 4-byte stores instead of one 16-byte store
(the boundary falls back rather than fails), with bitwise the same values
as into an aligned array; an output that is not float-aligned is refused."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu


def unaligned(n, cols):
    """A float32 [n][cols] view whose data starts 4 bytes past a 16-byte boundary."""
    buf = torch.full((n * cols + 4,), float("nan"), dtype=torch.float32, device="cuda")
    base = buf.data_ptr() % 16
    off = ((4 - base) % 16) // 4 if base != 4 else 0
    v = buf[off:off + n * cols].view(n, cols)
    assert v.data_ptr() % 16 == 4
    return v


@pytest.fixture(scope="module")
def scene(fab):
    mats = W.frame_materials()
    fab.set_materials(mats)
    g = W.subset(W.frame_gbuffer(), np.arange(1000, 1000 + 777))
    return mats, GBuffer.from_numpy(g)


def test_reference_components_unaligned(fab, scene):
    _, g = scene
    _, c0 = fab.shade_reference(g, 4, 4, 3, comps=True)
    c1 = unaligned(g.n, 4)
    fab.shade_reference(g, 4, 4, 3, out_comps=c1)
    fab.sync_status()
    assert torch.equal(c0, c1)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16", "fp8"])
def test_neural_components_unaligned(fab, scene, prec):
    mats, g = scene
    fab.set_params(W.decoder_init(), W.encoder_init())
    lat = torch.from_numpy(W.random_latents(len(mats))).cuda()
    _, c0 = fab.shade_neural(g, lat, prec, comps=True)
    c1 = unaligned(g.n, 4)
    fab.shade_neural(g, lat, prec, out_comps=c1)
    fab.sync_status()
    assert torch.equal(c0, c1)


def test_paper_decoder_components_unaligned(fab, scene):
    mats, g = scene
    fab.paper_set_params(64, W.paper_decoder_init(64), W.paper_encoder_init())
    z = torch.from_numpy(W.random_latents(len(mats), dim=64)).cuda()
    _, c0 = fab.paper_shade_neural(g, z, "fp16", comps=True)
    c1 = unaligned(g.n, 4)
    fab.paper_shade_neural(g, z, "fp16", out_comps=c1)
    fab.sync_status()
    assert torch.equal(c0, c1)


def test_output_not_float_aligned_is_refused(fab, scene):
    _, g = scene
    raw = torch.empty(g.n * 16 + 64, dtype=torch.uint8, device="cuda")
    rgb = torch.empty((g.n, 3), dtype=torch.float32, device="cuda")
    from paper_2406_17782_gb300._abi import check
    import ctypes
    gs = g.struct()
    bad = ctypes.c_void_p(raw.data_ptr() + 2)
    with pytest.raises(FabricError):
        check(fab.lib.fabric_shade_reference(fab.h, ctypes.byref(gs), 2, 2, 1, ctypes.c_void_p(rgb.data_ptr()),
                                             bad, None))
