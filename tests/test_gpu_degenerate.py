"""Degenerate and extreme inputs through the GPU path, against the FP64
oracles on the same inputs: zero and very large footprints, grazing,
horizontal and below-horizon directions, opposite directions (zero half
vector), uv far from the origin and negative, and materials at the edges of
their accepted ranges (alpha = 1 and 0.02, beta = 0 and 4, gap 0 and 0.9,
twist and inclination +-89 deg)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import mlp as M
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu


def edge_materials():
    rng = np.random.default_rng(21)
    out = []
    for pid, (a, b, gap, tw, inc) in enumerate([((1.0, 1.0), (0.0, 0.0), 0.2, 0.0, 0.0),
                                                ((0.02, 0.05), (4.0, 4.0), 0.2, 89.0, 89.0),
                                                ((0.3, 0.3), (1.0, 2.0), 0.0, -89.0, -89.0),
                                                ((0.5, 0.1), (0.5, 0.0), 0.9, 30.0, 15.0)]):
        out.append(W.make_material(pattern=[0, 3, 6, 11][pid], twist_deg=tw, incl_deg=inc, alpha=list(a),
                                   beta=list(b), kd=rng.uniform(0.2, 0.8, (2, 3)), ks=rng.uniform(0.2, 0.8, (2, 3)),
                                   gap=gap))
    return np.array(out)


def edge_gbuffer(n_mat):
    rng = np.random.default_rng(22)
    rows = []

    def add(u, v, r, wi, wo):
        for m in range(n_mat):
            rows.append((u, v, r, wi, wo, m))

    up = np.array([0.0, 0.0, 1.0])
    graze = np.array([np.sqrt(1 - 1e-12), 0.0, 1e-6])
    horizon = np.array([0.0, 1.0, 0.0])
    below = np.array([0.6, 0.0, -0.8])
    tilt = np.array([0.48, 0.36, 0.8])
    for r in (0.0, 1e-7, 1e-4, 0.5, 2.5):
        add(0.37, 0.61, r, tilt, up)
    for wi, wo in ((graze, up), (up, graze), (horizon, tilt), (tilt, horizon), (below, tilt), (tilt, -tilt),
                   (graze, graze * np.array([-1, 1, 1]))):
        add(0.2, 0.9, 3e-3, wi, wo)
    for u, v in ((-3.25, -0.125), (1e6 + 0.3, 2e5 + 0.7), (49.999, 0.0)):
        add(u, v, 1e-2, tilt, up)
    for _ in range(40):
        wi, wo = W.hemisphere_uniform(rng, 2)
        add(rng.uniform(0, 50), rng.uniform(0, 50), float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-1)))), wi, wo)
    g = {"u": np.array([x[0] for x in rows], np.float32), "v": np.array([x[1] for x in rows], np.float32),
         "radius": np.array([x[2] for x in rows], np.float32),
         "wi": np.array([x[3] for x in rows], np.float32), "wo": np.array([x[4] for x in rows], np.float32),
         "material": np.array([x[5] for x in rows], np.uint16)}
    return g


def test_reference_on_degenerate_inputs(fab):
    mats = edge_materials()
    fab.set_materials(mats)
    g = edge_gbuffer(len(mats))
    rgb, comps = fab.shade_reference(GBuffer.from_numpy(g), 4, 4, 0xED6E, comps=True)
    fab.sync_status()
    want_c, want_rgb = oracle.shade_reference(mats, g, 4, 4, 0xED6E)
    for got, want in ((comps, want_c), (rgb, want_rgb)):
        got = got.cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all()
        bad = np.abs(got - want) > 1e-4 * np.abs(want) + 1e-7
        assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], want[bad][:5])


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_decoder_on_degenerate_inputs(fab, prec):
    mats = edge_materials()
    fab.set_materials(mats)
    dec = W.decoder_init()
    fab.set_params(dec, W.encoder_init())
    z = W.random_latents(len(mats))
    g = edge_gbuffer(len(mats))
    rgb, comps = fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), prec, comps=True)
    fab.sync_status()
    want_c, _ = M.shade_neural(M.unpack(dec, M.DEC_SHAPES), z, mats, g)
    got = comps.cpu().numpy().astype(np.float64)
    assert np.isfinite(got).all()
    rel = np.sqrt(((got - want_c) ** 2).sum() / (want_c ** 2).sum())
    assert rel <= (2e-5 if prec == "fp32" else 5e-3), rel


@pytest.mark.parametrize("sleep", [False, True])
def test_expired_wait_is_reported_and_context_survives(fab, sleep):
    """A kernel wait that nothing completes gives up after its cycle limit,
    records a timeout in the status word and returns: the next status check
    raises FABRIC_ERR_TIMEOUT, clears the word, and the context keeps
    working (a reference draw afterwards is clean)."""
    fab.sync_status()
    fab.selftest_wait_timeout(sleep)
    with pytest.raises(FabricError) as info:
        fab.sync_status()
    assert info.value.status == 4   # FABRIC_ERR_TIMEOUT
    fab.sync_status()               # cleared
    mats = W.frame_materials()
    fab.set_materials(mats)
    g = W.subset(W.frame_gbuffer(), np.arange(0, 64))
    rgb, _ = fab.shade_reference(GBuffer.from_numpy(g), 2, 2, 1)
    fab.sync_status()
    assert torch.isfinite(rgb).all()
