"""All twelve built-in weaves (the eight of the 1080p frame plus 4/1 and 7/1
twills, an 8-harness satin and a 5-harness satin with doubled picks) through
the GPU path: the reference integral against the FP64 estimator on the same
sample sequence (1e-4 relative per point), the encoder's latents against
the FP64 encoder, and the FP16 decoder against the FP64 network."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import mlp as M
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weaves():
    rng = W.rng_for(7, "weaves")
    mats = np.concatenate([W.random_materials(rng, range(12)), W.table2_materials(rng, range(12))])
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 3000, stream="weaves"))
    g["material"] = (np.arange(len(g["u"])) % len(mats)).astype(np.uint16)
    return mats, g


def test_reference_all_weaves(fab, weaves):
    mats, g = weaves
    fab.set_materials(mats)
    rgb, comps = fab.shade_reference(GBuffer.from_numpy(g), 4, 4, 0xBEEF, comps=True)
    fab.sync_status()
    want_c, want_rgb = oracle.shade_reference(mats, g, 4, 4, 0xBEEF)
    for got, want in ((comps, want_c), (rgb, want_rgb)):
        got = got.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want) <= 1e-4 * np.abs(want) + 1e-7)


def test_encoder_and_decoder_all_weaves(fab, weaves):
    mats, g = weaves
    fab.set_materials(mats)
    dec, enc = W.decoder_init(), W.encoder_init()
    fab.set_params(dec, enc)
    z = fab.encode_params(mats)
    want_z = M.encoder_forward(M.unpack(enc, M.ENC_SHAPES), M.encoder_features(mats))
    np.testing.assert_allclose(z.cpu().numpy(), want_z, rtol=1e-4, atol=1e-4)
    zz = want_z.astype(np.float32)
    _, comps = fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(zz).cuda(), "fp16", comps=True)
    fab.sync_status()
    want_c, _ = M.shade_neural(M.unpack(dec, M.DEC_SHAPES), zz, mats, g)
    got = comps.cpu().numpy().astype(np.float64)
    assert np.sqrt(((got - want_c) ** 2).sum() / (want_c ** 2).sum()) <= 5e-3


def test_unknown_weave_is_refused(fab):
    bad = W.random_materials(np.random.default_rng(0), [0])
    bad["pattern"] = 12
    with pytest.raises(FabricError):
        fab.set_materials(bad)
