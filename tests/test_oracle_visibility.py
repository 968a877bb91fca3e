"""Pins of the oracle's proposed inter-yarn visibility model (V of Eq. 3-5;
the paper's own model is in its missing supplementary): the height field at
hand-worked points, the flat weave (everything visible, so shading equals
V = 1 exactly), straight-up and below-horizon rays, and the float-rise
threshold of a ray leaving the foot of an inclined float along its axis
(occluded below the inclination angle, visible above it)."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def plain_material(beta_w=1.5, beta_f=0.75, incl=30.0, gap=0.25):
    m = W.frame_materials()[:1].copy()
    m["pattern"] = 0          # plain weave, 2 x 2 cells
    m["beta"] = [beta_w, beta_f]
    m["incl_deg"] = incl
    m["gap"] = gap
    m["twist_deg"] = 0.0
    return m


def fixed(x: float) -> int:
    return int(round(x * 2 ** 32)) & 0xFFFFFFFF


def test_height_at_hand_worked_points(O):
    """Plain weave, g = 0.25, beta = (1.5, 0.75), inclination 30 degrees
    (all exact in float32).  Warp on top in cell (0, 0).  Half-width
    w = (1 - 0.25) / (2 * 2) = 0.1875.  Body centre (u, v) = (0.25, 0.25),
    x = 0, middle of a one-cell float:
    1.5 * 0.1875 + (1/2) (-ln cos 30deg) / (2 * pi/6) = 0.28125 + 0.0686790 = 0.3499290.
    Gap at u = 0.025 (s = 0.05 < g/2): the weft under it, across v-local
    0.25, x' = (0.5 - 1) / 0.75 = -2/3: 0.75 * 0.1875 (cos(pi/3) - 1) = -0.0703125."""
    m = O.material_rows(plain_material())[0]
    assert O.height(m, fixed(0.25), fixed(0.25)) == pytest.approx(0.3499290358, abs=1e-9)
    assert O.height(m, fixed(0.025), fixed(0.125)) == pytest.approx(-0.0703125, abs=1e-9)
    # float ends: no rise, and the cross-section's crest alone
    assert O.height(m, fixed(0.25), 0) == pytest.approx(0.28125, abs=1e-9)
    # the largest height: the warp's crest plus the rise of a one-cell float
    assert O.height_max(m) == pytest.approx(0.3499290358, abs=1e-9)


def test_flat_weave_is_fully_visible(O):
    """beta = 0 and no inclination: the surface is flat at height 0 on the
    yarn bodies and in the gaps, so every ray above the horizon is visible
    and shading with the model equals shading with V = 1 exactly."""
    mats = W.frame_materials().copy()
    mats["beta"] = 0.0
    mats["incl_deg"] = 0.0
    rows = O.material_rows(mats)
    rng = np.random.default_rng(5)
    for _ in range(200):
        m = rows[rng.integers(len(rows))]
        pu, pv = int(rng.integers(2 ** 32)), int(rng.integers(2 ** 32))
        assert O.height(m, pu, pv) == 0.0
        w = W.hemisphere_uniform(rng, 1)[0].astype(np.float64)
        assert O.visible(m, pu, pv, w) == (1, False)
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 300, stream="vis-flat"))
    idx = W.sample_indices(1920 * 1080, 300, stream="vis-flat")
    c0, r0 = O.shade_reference(mats, g, 4, 4, 11, pixel_index=idx)
    c1, r1, amb = O.shade_reference(mats, g, 4, 4, 11, pixel_index=idx, visibility=True)
    assert np.array_equal(c0, c1) and np.array_equal(r0, r1)
    # only rays that start almost parallel to the surface come within eps of it
    assert amb.mean() < 0.02


def test_straight_up_and_below_horizon(O):
    rows = O.material_rows(W.frame_materials())
    rng = np.random.default_rng(6)
    for _ in range(100):
        m = rows[rng.integers(len(rows))]
        pu, pv = int(rng.integers(2 ** 32)), int(rng.integers(2 ** 32))
        assert O.visible(m, pu, pv, [0.0, 0.0, 1.0]) == (1, False)
        assert O.visible(m, pu, pv, [0.6, 0.0, -0.8])[0] == 0


@pytest.mark.parametrize("incl", [20.0, 30.0, 45.0])
def test_float_rise_threshold(O, incl):
    """No cross-section (beta = 0): a warp float of the plain weave rises
    along its axis (+v) with slope tan(theta), theta = incl (1 - 2y), which
    is steepest at its foot.  A ray leaving the foot along +v is occluded by
    the rise when its elevation is below the inclination, and clears it (and
    the weft float beyond, lower than the ray there) when above."""
    m = O.material_rows(plain_material(beta_w=0.0, beta_f=0.0, incl=incl))[0]
    pu, pv = fixed(0.25), fixed(0.001)      # warp body centre, at the foot of its float
    for elev, want in ((incl - 5.0, 0), (incl + 5.0, 1)):
        e = math.radians(elev)
        v, amb = O.visible(m, pu, pv, [0.0, math.cos(e), math.sin(e)])
        assert (v, amb) == (want, False), (incl, elev)
    # the opposite direction (-v) crosses the gap beside the foot into the
    # crossing weft's float, whose rise there (its middle) is a step up
    # 1/16 repeat away: occluded below about atan(rise * 16), visible at 70deg
    for elev, want in ((incl - 5.0, 0), (70.0, 1)):
        e = math.radians(elev)
        assert O.visible(m, pu, pv, [0.0, -math.cos(e), math.sin(e)]) == (want, False), (incl, elev)
