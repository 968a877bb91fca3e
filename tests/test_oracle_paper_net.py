"""Pins of the FP64 oracle of the paper's decoder structure (Sec. 4.2,
Fig. 3): one-blob encoding, the skip of the angular decoder's residual
block, the backward pass, and the reduction of its operand-rounding
emulation to the network (CPU only)."""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def PN(oracle_mod):
    from oracle import paper_net
    return paper_net


def test_oneblob_shape_and_peak(PN):
    """3 inputs -> 24 channels (Sec. 4.2); a value at a bin centre puts 1 in
    that bin and less everywhere else, the nearest bin always holds the
    largest value."""
    assert PN.spatial_features(np.float32([0.3]), np.float32([0.7]), np.float32([0.01])).shape == (1, 24)
    rng = np.random.default_rng(0)
    s = rng.uniform(0, 1, 500)
    for periodic in (True, False):
        b = PN.oneblob(s, periodic)
        assert np.array_equal(np.argmax(b, 1), np.minimum((s * 8).astype(int), 7))
        centres = (np.arange(8) + 0.5) / 8
        bc = PN.oneblob(centres, periodic)
        np.testing.assert_allclose(np.diag(bc), 1.0, rtol=0, atol=1e-13)
        assert (bc[~np.eye(8, dtype=bool)] < 1.0).all()


def test_oneblob_symmetry_and_shift(PN):
    """Mirror symmetry (s -> 1 - s reverses the bins); the periodic encoding
    is periodic in s and shifting s by one bin width rotates it by one bin."""
    rng = np.random.default_rng(1)
    s = rng.uniform(0, 1, 300)
    for periodic in (True, False):
        np.testing.assert_allclose(PN.oneblob(1.0 - s, periodic), PN.oneblob(s, periodic)[:, ::-1], atol=1e-14)
    b = PN.oneblob(s, True)
    np.testing.assert_allclose(PN.oneblob(s + 3.0, True), b, atol=1e-12)
    np.testing.assert_allclose(PN.oneblob(s + 1.0 / 8, True), np.roll(b, 1, axis=1), atol=1e-12)


def test_periodic_oneblob_sums_to_sqrt_2pi(PN):
    """A Gaussian of standard deviation equal to the bin spacing, summed
    over a periodic lattice of bin centres, is sqrt(2 pi) for every s up to
    2 sqrt(2 pi) exp(-2 pi^2) ~ 1.3e-8 (Poisson summation: the sum is a
    theta function whose first Fourier term has that weight)."""
    s = np.linspace(0, 1, 1001)
    tot = PN.oneblob(s, True).sum(1)
    np.testing.assert_allclose(tot, math.sqrt(2 * math.pi), rtol=0,
                               atol=1.01 * 2 * math.sqrt(2 * math.pi) * math.exp(-2 * math.pi ** 2))
    assert np.ptp(tot) > 0      # the ripple is there, just tiny


def test_size_coordinate_range(PN):
    np.testing.assert_allclose(PN.size_coordinate(np.array([1e-4, 2.5])), [0.0, 1.0], atol=1e-12)
    assert np.isfinite(PN.size_coordinate(np.array([0.0]))).all()


def _zero_dec(PN, w):
    return {k: np.zeros(s) for k, s in PN.dec_shapes(w)}


def test_closed_form_tiny_net_through_the_skip(PN):
    """Hand-set weights: unit 0 of the spatial feature copies latent[5]; the
    angular layer A1 passes it (unit 0) and wi_z (unit 1, with a -1 weight,
    so the leaky slope shows); A2 is zero, so the residual block returns
    lrelu(a3 + k1) through the skip alone; A4 copies, A5 reads out."""
    w = 64
    p = _zero_dec(PN, w)
    p["S1"][0, 5] = 1.0
    p["S2"][0, 0] = 1.0
    p["A1"][0, 0] = 1.0
    p["A1"][1, w + 2] = -1.0             # -wi_z
    p["a3"][:2] = [0.25, 0.0]
    p["A4"][:2, :2] = np.eye(2)
    p["A5"][0, 0] = 2.0
    p["A5"][1, 1] = 1.0
    p["a5"][:] = [0.1, 0.2, 0.3, 0.4]
    z = np.zeros((2, 64))
    z[0, 5] = 0.7
    z[1, 5] = -0.5
    blob = np.zeros((2, 24))
    ang = np.array([[0.0, 0.0, 0.8, 0.3, 0.1], [0.6, 0.0, 0.5, 0.0, 0.0]])
    y = PN.decoder_forward(p, z, blob, ang)
    # point 0: hs0 = 0.7; k1 = (0.7, lrelu(-0.8) = -0.008); k3 = (lrelu(0.25 + 0.7), lrelu(-0.008))
    # = (0.95, -0.00008); k4 = (0.95, lrelu(-0.00008) = -8e-7); y = (2*0.95 + 0.1, -8e-7 + 0.2, 0.3, 0.4)
    # point 1: hs0 = lrelu(lrelu(-0.5)) = -0.00005; k1 = (lrelu(-0.00005) = -5e-7, lrelu(-0.5) = -0.005);
    # k3 = (lrelu(0.25 - 5e-7), lrelu(-0.005)) = (0.2499995, -0.00005); k4 = (0.2499995, -5e-7)
    want = np.array([[1.9 + 0.1, 0.2 - 8e-7, 0.3, 0.4],
                     [2 * 0.2499995 + 0.1, 0.2 - 5e-7, 0.3, 0.4]])
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-15)


def test_backward_finite_differences(PN):
    rng = np.random.default_rng(2)
    for w in PN.WIDTHS:
        p = {k: 0.3 * rng.standard_normal(s) / math.sqrt(s[-1]) * 3 for k, s in PN.dec_shapes(w)}
        n = 5
        z = rng.standard_normal((n, 64))
        blob = PN.spatial_features(rng.uniform(0, 9, n), rng.uniform(0, 9, n), np.exp(rng.uniform(-9, 0.5, n)))
        ang = PN.angular_features(W.hemisphere_uniform(rng, n), W.hemisphere_uniform(rng, n))
        dy = rng.standard_normal((n, 4))
        y, cache = PN.decoder_forward(p, z, blob, ang, keep=True)
        g, dz, dang = PN.decoder_backward(p, cache, dy)
        f = lambda pp, zz, aa: float(np.sum(dy * PN.decoder_forward(pp, zz, blob, aa)))
        h = 1e-6
        for name, shape in PN.dec_shapes(w):
            for _ in range(5):
                idx = tuple(rng.integers(0, s) for s in shape)
                pp = {k: v.copy() for k, v in p.items()}
                pp[name][idx] += h
                fp = f(pp, z, ang)
                pp[name][idx] -= 2 * h
                fm = f(pp, z, ang)
                fd = (fp - fm) / (2 * h)
                assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (w, name, idx, fd, g[name][idx])
        for _ in range(8):
            i, j = rng.integers(0, n), rng.integers(0, 64)
            zz = z.copy()
            zz[i, j] += h
            fp = f(p, zz, ang)
            zz[i, j] -= 2 * h
            assert abs((fp - f(p, zz, ang)) / (2 * h) - dz[i, j]) <= 1e-6 * max(1.0, abs(dz[i, j]))
            j = rng.integers(0, 5)
            aa = ang.copy()
            aa[i, j] += h
            fp = f(p, z, aa)
            aa[i, j] -= 2 * h
            assert abs((fp - f(p, z, aa)) / (2 * h) - dang[i, j]) <= 1e-6 * max(1.0, abs(dang[i, j]))


def test_emulation_without_rounding_is_the_network(PN):
    """The operand-rounding emulation with identity rounding: the latent
    folded into a per-material bias equals the unfolded first layer, and the
    whole path equals shade() to rounding order."""
    rng = np.random.default_rng(3)
    mats = W.frame_materials()
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 500, stream="paper-net-emu"))
    for w in PN.WIDTHS:
        p = {k: rng.standard_normal(s) / math.sqrt(s[-1]) for k, s in PN.dec_shapes(w)}
        z = rng.standard_normal((8, 64))
        c0, r0 = PN.shade(p, z, mats, g)
        c1, r1 = PN.shade_rounded(p, z, mats, g, lambda a: np.asarray(a, np.float64))
        np.testing.assert_allclose(c1, c0, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r1, r0, rtol=1e-12, atol=1e-12)


def test_flop_count(PN):
    # 2 (24*64 + 64*64 + 69*64 + 3*64*64 + 64*4) with the latent folded
    assert PN.flops_per_point(64) == 2 * (24 * 64 + 64 * 64 + 69 * 64 + 3 * 64 * 64 + 64 * 4) == 45_184
    assert PN.flops_per_point(128) == 2 * (24 * 128 + 128 * 128 + 133 * 128 + 3 * 128 * 128 + 128 * 4)


def test_ablation_shapes_and_raw_spatial_inputs(PN):
    """Without the one-blob encoding the spatial channels are the inputs
    themselves; without the spatial fusion the angular decoder's first layer
    takes [z | one-blob | angular] (64 + 24 + 5 = 93 inputs) and the
    decoder keeps the full structure's depth and size."""
    f = PN.spatial_features(np.float32([3.25, -0.75]), np.float32([0.5, 7.125]), np.float32([1e-4, 2.5]),
                            PN.NO_ONEBLOB)
    np.testing.assert_allclose(f, [[0.25, 0.5, 0.0], [0.25, 0.125, 1.0]], atol=1e-7)
    for w in PN.WIDTHS:
        shapes = dict(PN.dec_shapes(w, PN.NO_FUSION))
        assert "S1" not in shapes and shapes["H1"] == (w, 93) and shapes["A1"] == (w, w)
        assert len(shapes) == len(PN.dec_shapes(w))
        n = lambda sh: sum(int(np.prod(d)) for _, d in sh)
        assert n(PN.dec_shapes(w, PN.NO_FUSION)) == n(PN.dec_shapes(w))
        assert dict(PN.dec_shapes(w, PN.NO_ONEBLOB))["S1"] == (w, 67)


def test_no_fusion_closed_form_through_the_skip(PN):
    """No spatial fusion: H1 reads latent[2] (unit 0), wi_z with weight -2
    (unit 1, through the leaky slope) and one-blob channel 3 (unit 2); H2
    and A1 pass units 0..2 on; A2 = 0, so the residual block returns
    lrelu(a3 + k1)."""
    w = 64
    p = {k: np.zeros(s) for k, s in PN.dec_shapes(w, PN.NO_FUSION)}
    p["H1"][0, 2] = 1.0
    p["H1"][1, 64 + 24 + 2] = -2.0       # wi_z
    p["H1"][2, 64 + 3] = 1.0             # one-blob channel 3
    p["H2"][:3, :3] = np.eye(3)
    p["A1"][:3, :3] = np.eye(3)
    p["a3"][:3] = [0.5, 0.0, 0.0]
    p["A4"][:3, :3] = np.eye(3)
    p["A5"][:3, :3] = np.eye(3)
    z = np.zeros((1, 64))
    z[0, 2] = 0.25
    blob = np.zeros((1, 24))
    blob[0, 3] = 0.5
    ang = np.array([[0.0, 0.0, 0.5, 0.0, 0.0]])
    y = PN.decoder_forward(p, z, blob, ang)
    # unit 0: 0.25 through H1, H2, A1 (k1 = 0.25), k3 = lrelu(0.5 + 0.25) = 0.75, y0 = 0.75
    # unit 1: lrelu(-1) = -0.01 -> -1e-4 (H2) -> k1 = -1e-6 -> k3 = -1e-8 -> k4 = -1e-10 = y1
    # unit 2: 0.5 all the way: y2 = 0.5
    np.testing.assert_allclose(y, [[0.75, -1e-10, 0.5, 0.0]], rtol=0, atol=1e-15)


@pytest.mark.parametrize("ablation", [1, 2])
def test_ablation_backward_finite_differences(PN, ablation):
    rng = np.random.default_rng(20 + ablation)
    w = 64
    p = {k: rng.standard_normal(s) / math.sqrt(s[-1]) for k, s in PN.dec_shapes(w, ablation)}
    n = 5
    z = rng.standard_normal((n, 64))
    sp = PN.spatial_features(rng.uniform(0, 9, n), rng.uniform(0, 9, n), np.exp(rng.uniform(-9, 0.5, n)), ablation)
    ang = PN.angular_features(W.hemisphere_uniform(rng, n), W.hemisphere_uniform(rng, n))
    dy = rng.standard_normal((n, 4))
    y, cache = PN.decoder_forward(p, z, sp, ang, keep=True)
    g, dz, dang = PN.decoder_backward(p, cache, dy)
    f = lambda pp, zz, aa: float(np.sum(dy * PN.decoder_forward(pp, zz, sp, aa)))
    h = 1e-6
    for name, shape in PN.dec_shapes(w, ablation):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in shape)
            pp = {k: v.copy() for k, v in p.items()}
            pp[name][idx] += h
            fp = f(pp, z, ang)
            pp[name][idx] -= 2 * h
            fd = (fp - f(pp, z, ang)) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (ablation, name, idx)
    for _ in range(6):
        i, j = rng.integers(0, n), rng.integers(0, 64)
        zz = z.copy()
        zz[i, j] += h
        fp = f(p, zz, ang)
        zz[i, j] -= 2 * h
        assert abs((fp - f(p, zz, ang)) / (2 * h) - dz[i, j]) <= 1e-6 * max(1.0, abs(dz[i, j]))
        j = rng.integers(0, 5)
        aa = ang.copy()
        aa[i, j] += h
        fp = f(p, z, aa)
        aa[i, j] -= 2 * h
        assert abs((fp - f(p, z, aa)) / (2 * h) - dang[i, j]) <= 1e-6 * max(1.0, abs(dang[i, j]))
