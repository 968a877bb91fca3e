"""NaN inputs stay with their point: a G-buffer where a few points carry a
NaN coordinate, footprint or direction gives, at every other point, bitwise
the outputs of the clean G-buffer (reference kernel, every decoder
precision, the paper's decoder)."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

POISONED = [3, 130, 131, 500]


def buffers():
    g = W.subset(W.frame_gbuffer(), np.arange(20000, 20000 + 777))
    bad = {k: v.copy() if isinstance(v, np.ndarray) else v for k, v in g.items()}
    bad["u"][POISONED[0]] = np.nan
    bad["radius"][POISONED[1]] = np.nan
    bad["wi"][POISONED[2], 1] = np.nan
    bad["wo"][POISONED[3], 2] = np.nan
    keep = np.setdiff1d(np.arange(777), POISONED)
    return GBuffer.from_numpy(g), GBuffer.from_numpy(bad), keep


def same_elsewhere(clean, dirty, keep):
    c, d = clean.cpu().numpy(), dirty.cpu().numpy()
    assert np.array_equal(c[keep], d[keep])


def test_reference_keeps_nan_to_its_point(fab):
    fab.set_materials(W.frame_materials())
    g, bad, keep = buffers()
    r0, c0 = fab.shade_reference(g, 4, 4, 9, comps=True)
    r1, c1 = fab.shade_reference(bad, 4, 4, 9, comps=True)
    fab.sync_status()
    same_elsewhere(c0, c1, keep)
    same_elsewhere(r0, r1, keep)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16", "fp8"])
def test_decoder_keeps_nan_to_its_point(fab, prec):
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.set_params(W.decoder_init(), W.encoder_init())
    lat = torch.from_numpy(W.random_latents(len(mats))).cuda()
    g, bad, keep = buffers()
    r0, c0 = fab.shade_neural(g, lat, prec, comps=True)
    r1, c1 = fab.shade_neural(bad, lat, prec, comps=True)
    fab.sync_status()
    same_elsewhere(c0, c1, keep)
    same_elsewhere(r0, r1, keep)


def test_paper_decoder_keeps_nan_to_its_point(fab):
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.paper_set_params(128, W.paper_decoder_init(128), W.paper_encoder_init())
    z = torch.from_numpy(W.random_latents(len(mats), dim=64)).cuda()
    g, bad, keep = buffers()
    r0, c0 = fab.paper_shade_neural(g, z, "fp16", comps=True)
    r1, c1 = fab.paper_shade_neural(bad, z, "fp16", comps=True)
    fab.sync_status()
    same_elsewhere(c0, c1, keep)
    same_elsewhere(r0, r1, keep)
