"""The reference kernel with the proposed inter-yarn visibility model
(fabric_set_visibility) against the FP64 oracle's model on the same sample
sequence: |gpu - oracle| <= 1e-4 |oracle| + 1e-7 per point and component,
except at points where one of the oracle's marches came within 1e-6 repeats
of the surface without a clear occluder (a binary decision that FP32
rounding of the heights could turn); those must stay rare.  The flat weave
(no cross-section, no inclination) gives bitwise the V = 1 result."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-7


def shade(fab, g, sx, sy, seed, vis):
    fab.set_visibility(vis)
    try:
        rgb, comps = fab.shade_reference(GBuffer.from_numpy(g), sx, sy, seed, comps=True)
        fab.sync_status()
    finally:
        fab.set_visibility(False)
    return rgb.cpu().numpy(), comps.cpu().numpy()


def check(got, want, amb, what, max_amb=0.02):
    err = np.abs(np.asarray(got, np.float64) - want) - (RTOL * np.abs(want) + ATOL)
    bad = (err > 0).any(axis=1)
    print(f"{what}: {int(amb.sum())} of {len(amb)} points with a near-tie march; "
          f"{int(bad.sum())} outside the bound, {int((bad & ~amb).sum())} of them elsewhere")
    assert not (bad & ~amb).any()
    assert amb.mean() < max_amb


@pytest.mark.parametrize("frame,stream,spp", [("frame", "vis-frame", 8), ("multiscale", "vis-ms", 8),
                                              ("frame", "vis-frame-256", 16)])
def test_visibility_matches_oracle(fab, frame, stream, spp):
    """Sampled points of the 1080p frame and of the multi-scale frame, at 64
    and 256 samples per point (16 and 32 lanes per point)."""
    mats = W.frame_materials()
    fab.set_materials(mats)
    full = W.frame_gbuffer() if frame == "frame" else W.multiscale_gbuffer()
    g = W.subset(full, W.sample_indices(1920 * 1080, 2048, stream=stream))
    rgb, comps = shade(fab, g, spp, spp, 91, True)
    wc, wr, amb = oracle.shade_reference(mats, g, spp, spp, 91, visibility=True)
    check(comps, wc, amb, f"{frame} comps")
    check(rgb, wr, amb, f"{frame} rgb")
    # the model changes the result (shadowed samples exist), and V = 1 is untouched
    rgb0, comps0 = shade(fab, g, spp, spp, 91, False)
    wc0, _ = oracle.shade_reference(mats, g, spp, spp, 91)
    assert np.abs(wc - wc0).max() > 1e-3
    assert np.all(np.abs(comps0 - wc0) <= RTOL * np.abs(wc0) + ATOL)


def test_flat_weave_equals_unit_visibility(fab):
    mats = W.frame_materials().copy()
    mats["beta"] = 0.0
    mats["incl_deg"] = 0.0
    fab.set_materials(mats)
    try:
        g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 4096, stream="vis-flat-gpu"))
        rgb1, comps1 = shade(fab, g, 8, 8, 5, True)
        rgb0, comps0 = shade(fab, g, 8, 8, 5, False)
        assert np.array_equal(comps1, comps0) and np.array_equal(rgb1, rgb0)
    finally:
        fab.set_materials(W.frame_materials())


def test_visibility_setting_is_checked(fab):
    from paper_2406_17782_gb300._abi import check as abi_check
    with pytest.raises(FabricError):
        abi_check(fab.lib.fabric_set_visibility(fab.h, 2))


def test_visibility_on_degenerate_inputs(fab):
    """The degenerate-input set of the reference (zero to 5-repeat
    footprints; grazing, horizontal, below-horizon and opposite directions;
    uv far out and negative; beta 0 and 4, gap 0 and 0.9, inclination +-89
    degrees, where floats rise by more than a repeat and grazing marches run
    to the 4096-step limit) with the model on."""
    from test_gpu_degenerate import edge_gbuffer, edge_materials
    mats = edge_materials()
    fab.set_materials(mats)
    try:
        g = edge_gbuffer(len(mats))
        rgb, comps = shade(fab, g, 4, 4, 0xED6E, True)
        assert np.isfinite(comps).all() and np.isfinite(rgb).all()
        wc, wr, amb = oracle.shade_reference(mats, g, 4, 4, 0xED6E, visibility=True)
        check(comps, wc, amb, "degenerate comps", max_amb=0.05)
        check(rgb, wr, amb, "degenerate rgb", max_amb=0.05)
    finally:
        fab.set_materials(W.frame_materials())
