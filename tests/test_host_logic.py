"""Host-side logic that needs no GPU: the autotuner's choice and cache, the
G-buffer binding's checks, and the synthetic workloads' shapes and
distributions (the input recipe the benchmarks and tests rely on)."""
import json
import math

import numpy as np
import pytest
import torch

import workloads as W
from paper_2406_17782_gb300 import autotune
from paper_2406_17782_gb300.api import GBuffer


class FakeFab:
    """Stands in for a context: records launch settings; 'times' them from a table."""

    def __init__(self, table):
        self.table = table
        self.calls = []
        self.launch_config = (0, 0, 0)
        self.n_mat = 8
        self.sm_count = 152
        self.device = "cpu"

    def set_launch_config(self, ctas, wg, lanes, h=0):
        self.launch_config = (ctas, wg, lanes)
        self.current = (wg, ctas, h)
        self.calls.append(self.current)

    def shade_neural_prepared(self, g, precision, out_rgb=None):
        pass


def test_autotuner_picks_the_fastest_shape_and_caches_it(tmp_path, monkeypatch):
    table = {c: 1.0 + 0.1 * k for k, c in enumerate(autotune.DECODER_CANDIDATES)}
    best = autotune.DECODER_CANDIDATES[3]
    table[best] = 0.5
    fab = FakeFab(table)
    monkeypatch.setattr(autotune, "_time", lambda fn, reps: fab.table[fab.current])
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d: "fake GPU")
    monkeypatch.setattr(autotune.torch, "empty", lambda *a, **k: None)
    g = GBuffer(*(torch.zeros(1000) for _ in range(6)))
    cache = str(tmp_path / "tune.json")
    e = autotune.tune_decoder(fab, g, "fp16", cache_path=cache)
    assert (e["warpgroups"], e["ctas_per_sm"], e["tile_warpgroups"]) == best
    assert fab.current == best and len(fab.calls) == len(autotune.DECODER_CANDIDATES) + 1
    stored = json.load(open(cache))
    assert len(stored) == 1 and list(stored.values())[0]["ms"] == 0.5
    # a second call reads the cache and times nothing
    fab.calls.clear()
    monkeypatch.setattr(autotune, "_time", lambda fn, reps: pytest.fail("timed again"))
    e2 = autotune.tune_decoder(fab, g, "fp16", cache_path=cache)
    assert e2 == e and fab.calls == [best]


def test_gbuffer_binding_checks_where_its_tensors_live():
    g = GBuffer(*(torch.zeros(10) for _ in range(6)))
    with pytest.raises(ValueError):
        g.struct()                      # a device G-buffer is expected
    s = g.struct(host=True)
    assert s.n == 10
    nc = GBuffer(*(torch.zeros((10, 2))[:, 0] for _ in range(6)))
    with pytest.raises(ValueError):
        nc.struct(host=True)            # not contiguous


def test_frame_gbuffer_recipe():
    g = W.frame_gbuffer()
    n = 1920 * 1080
    assert all(len(g[k]) == n for k in ("u", "v", "radius", "wi", "wo", "material"))
    assert g["u"].min() >= 0 and g["u"].max() < 50 and g["v"].min() >= 0 and g["v"].max() < 50
    lr = np.log(g["radius"].astype(np.float64))
    assert lr.min() >= math.log(1e-4) - 1e-6 and lr.max() <= math.log(1e-1) + 1e-6
    # log-uniform: each decade holds about a third of the points
    dec = np.histogram(lr, bins=[math.log(1e-4), math.log(1e-3), math.log(1e-2), math.log(1e-1)])[0] / n
    assert np.all(np.abs(dec - 1 / 3) < 0.01)
    for d in ("wi", "wo"):
        v = g[d].astype(np.float64)
        assert np.allclose(np.linalg.norm(v, axis=1), 1, atol=1e-6) and v[:, 2].min() >= 0
        # uniform in solid angle: z uniform on [0, 1]
        assert abs(v[:, 2].mean() - 0.5) < 0.01
    # eight vertical bands of 240 pixels
    m = g["material"].reshape(1080, 1920)
    assert np.array_equal(m[0], m[-1]) and np.array_equal(np.unique(m[0] // 1), np.arange(8))
    assert np.all(m[:, :240] == 0) and np.all(m[:, -240:] == 7)


def test_multiscale_gbuffer_recipe():
    f = W.frame_gbuffer()
    g = W.multiscale_gbuffer()
    # everything but the footprint is the 1080p frame's
    for k in ("u", "v", "wi", "wo", "material"):
        assert np.array_equal(f[k], g[k])
    side = 2.0 * g["radius"].astype(np.float64)
    assert side.min() > 0 and side.max() <= 5.0 + 1e-5
    # Table 2: half the sides in (0, 1), half in (1, 5), uniform within each
    small = side < 1.0
    assert abs(small.mean() - 0.5) < 0.01
    assert abs(side[small].mean() - 0.5) < 0.01 and abs(side[~small].mean() - 3.0) < 0.01


def test_batched_4k_recipe():
    segs, n = W.batched_4k()
    assert len(segs) == 1 + 4 * 64
    assert len(segs[0]["u"]) == 3840 * 2160
    sizes = np.array([len(s["u"]) for s in segs[1:]])
    assert sizes.min() >= 256 and sizes.max() <= 65536 and n == sum(len(s["u"]) for s in segs)
    m = segs[0]["material"].reshape(2160, 3840)
    # materials change only at 16 x 16 tile borders, and all eight occur
    assert np.array_equal(m[::16, ::16].repeat(16, 0).repeat(16, 1), m)
    assert set(np.unique(m)) == set(range(8))


def test_training_queries_recipe():
    q = W.training_queries(20000, 256)
    assert q["material"].max() < 256
    half = 10000
    # frame-like half: footprints log-uniform in [1e-4, 1e-1], uv in [0, 50)
    assert q["radius"][:half].min() >= 1e-4 * (1 - 1e-6) and q["radius"][:half].max() <= 1e-1 * (1 + 1e-6)
    # Table 2 half: centre in one repeat, side in (0, 5), directions inside the disc
    assert q["u"][half:].max() < 1 and q["radius"][half:].max() <= 2.5 + 1e-6
    d = q["wi"][half:].astype(np.float64)
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-6) and d[:, 2].min() >= 0


def test_paper_data_generation_recipe():
    """Sec. 5.1: 81 plain, 192 twill and 192 satin materials over seven
    weaves with Table 2's parameter ranges; per material 64 footprint
    centres x 20 sizes (10 in [0, 1], 10 in [1, 5] repeats) x the valid
    direction pairs (about 2500), about 3.2 million queries."""
    m = W.paper_materials()
    assert len(m) == 465
    counts = {w: int((m["pattern"] == w).sum()) for w in W.PAPER_WEAVES}
    assert counts[0] == 81
    assert sum(counts[w] for w in W.PAPER_TWILLS) == 192
    assert sum(counts[w] for w in W.PAPER_WEAVES if w != 0 and w not in W.PAPER_TWILLS) == 192
    assert set(np.unique(m["twist_deg"])) <= {-30.0, 0.0, 30.0}
    assert (m["incl_deg"] >= 15).all() and (m["incl_deg"] <= 45).all()
    assert (m["alpha"] >= 0.1).all() and (m["alpha"] <= 1).all()
    assert (m["beta"] >= 0).all() and (m["beta"] <= 2).all()
    q = W.paper_queries(3)
    n = len(q["u"])
    assert abs(n - 3.2e6) / 3.2e6 < 0.05
    side = 2.0 * q["radius"].astype(np.float64)
    sizes = np.unique(side)
    assert len(sizes) == 64 * 20
    assert ((sizes < 1).sum(), (sizes >= 1).sum()) == (640, 640)
    assert (side <= 5).all()
    centres = np.unique(np.stack([q["u"], q["v"]], 1), axis=0)
    assert len(centres) == 64
    cell = np.floor(centres * 8).astype(int)
    assert len(np.unique(cell[:, 0] * 8 + cell[:, 1])) == 64        # one centre per grid cell
    for w in (q["wi"], q["wo"]):
        assert (w[:, 2] > 0).all()
        np.testing.assert_allclose((w.astype(np.float64) ** 2).sum(1), 1.0, atol=1e-6)
