"""Parity of the neural decoder kernels with the FP64 network oracle.

* FP32 SIMT: per point and output |dy| <= 1e-5 max(|y*|, 1e-3 rms(y*)) (the
  stated FP32 bound) plus 4 sigma, where sigma is the spread of FP32
  arithmetic itself at that point, estimated by Monte Carlo arithmetic
  (every rounding of an FP32 evaluation replaced by a random relative
  perturbation of up to one unit roundoff; Parker, 1997).  Away from
  cancellation sigma is far below the bound; where the head is a cancelling
  sum no FP32 evaluation can meet the bound alone (about 2 % of the sampled
  outputs, for the GPU and for a sequential FP32 evaluation on the CPU
  alike), and the kernel must then be no noisier than FP32 itself.
* FP16 tensor cores (the default tensor-core precision): relative L2
  <= 5e-3 over the sampled frame against FP64, and <= 5e-4 against the FP16
  operand-rounding emulation of the same network.
* BF16 tensor cores: relative L2 <= 1.2e-2 against FP64 (BF16 operand
  rounding alone costs 8.2e-3 on this network, see the emulation), and
  <= 5e-4 against the BF16 emulation.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import mlp as M
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

TOL_FP64 = {"fp16": 5e-3, "bf16": 1.2e-2}
TOL_EMU = 5e-4


def rel_l2(got, want):
    got = np.asarray(got, np.float64)
    return float(np.sqrt(((got - want) ** 2).sum() / (want ** 2).sum()))


def round_fp16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float64)


ROUND = {"fp16": round_fp16, "bf16": M.round_bf16}


@pytest.fixture(scope="module")
def setup(fab):
    mats = W.frame_materials()
    fab.set_materials(mats)
    dec = W.decoder_init()
    fab.set_params(dec, W.encoder_init())
    z = W.random_latents(len(mats))
    return mats, dec, z


def emulate(prec, dec_flat, z, mats, g):
    """The tensor-core path's operand rounding: rounded query features,
    rounded weights, latent folded into a rounded per-material bias column,
    biases of layers 2-4 rounded (they ride in a constant-one input column),
    rounded activations, FP32 accumulation (FP64 here)."""
    r = ROUND[prec]
    P = M.unpack(dec_flat, M.DEC_SHAPES)
    q = r(M.query_features(g["u"], g["v"], g["radius"], g["wi"], g["wo"]))
    mat = np.asarray(g["material"], np.int64)
    fold = P["b1"][None, :] + z.astype(np.float64) @ P["W1"][:, :32].T
    h = np.maximum(q @ r(P["W1"][:, 32:]).T + r(fold)[mat], 0)
    h = np.maximum(r(h) @ r(P["W2"]).T + r(P["b2"]), 0)
    h = np.maximum(r(h) @ r(P["W3"]).T + r(P["b3"]), 0)
    y = r(h) @ r(P["W4"]).T + r(P["b4"])
    comps = M.head_to_components(y)
    return comps, M.recombine(comps, mats, g["material"])


def fp32_arithmetic_spread(P, x, trials=8, seed=0):
    """Per point and output, the standard deviation of the raw head over
    Monte Carlo arithmetic evaluations of the network: features perturbed by
    a relative U(-2u, 2u) (the kernel computes them with library sin, cos
    and log), every multiply-add result by a relative U(-u, u), u = 2^-24."""
    u = 2.0 ** -24
    rng = np.random.default_rng(seed)
    h = np.repeat(x[None], trials, 0)
    h = h * (1.0 + rng.uniform(-2 * u, 2 * u, h.shape))
    for Wn, bn in (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4")):
        Wm, b = P[Wn], P[bn]
        acc = np.broadcast_to(b, (trials, x.shape[0], len(b))).copy()
        for k in range(Wm.shape[1]):
            acc = (acc + h[:, :, k:k + 1] * Wm[None, None, :, k]) * (1.0 + rng.uniform(-u, u, acc.shape))
        h = np.maximum(acc, 0.0) if Wn != "W4" else acc
    return h.std(0)


def fp32_sequential_forward(P, x):
    """A plain FP32 evaluation on the CPU: features rounded to FP32, each
    output a chain of multiply-adds from its bias in input order."""
    h = x.astype(np.float32)
    for Wn, bn in (("W1", "b1"), ("W2", "b2"), ("W3", "b3"), ("W4", "b4")):
        Wm = P[Wn].astype(np.float32).astype(np.float64)
        acc = np.tile(P[bn].astype(np.float32), (h.shape[0], 1))
        h64 = h.astype(np.float64)
        for k in range(Wm.shape[1]):
            acc = (acc.astype(np.float64) + h64[:, k:k + 1] * Wm[None, :, k]).astype(np.float32)
        h = np.maximum(acc, 0) if Wn != "W4" else acc
    return h.astype(np.float64)


@pytest.mark.parametrize("a_in_tmem", [False, True])
@pytest.mark.parametrize("n,k", [(64, 16), (64, 48), (16, 64), (32, 32), (64, 64)])
def test_tensor_core_product_layout(fab, n, k, a_in_tmem):
    rng = np.random.default_rng(n * 100 + k)
    a = rng.standard_normal((128, k)).astype(np.float32)
    b = rng.standard_normal((n, k)).astype(np.float32)
    d = fab.selftest_mma(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), a_in_tmem).cpu().numpy()
    fab.sync_status()
    want = M.round_bf16(a) @ M.round_bf16(b).T
    np.testing.assert_allclose(d, want, rtol=1e-5, atol=1e-5)


def test_fp32_decoder_per_point(fab, setup):
    mats, dec, z = setup
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 4096, stream="dec-fp32"))
    gd = GBuffer.from_numpy(g)
    zt = torch.from_numpy(z).cuda()
    y_gpu = fab.decoder_forward(gd, zt, torch.from_numpy(dec).cuda()).cpu().numpy().astype(np.float64)
    rgb, comps = fab.shade_neural(gd, zt, "fp32", comps=True)
    fab.sync_status()
    P = M.unpack(dec, M.DEC_SHAPES)
    x = M.decoder_inputs(z, g["material"], g)
    y = M.decoder_forward(P, x)
    tol7 = 1e-5 * np.maximum(np.abs(y), 1e-3 * np.sqrt((y ** 2).mean(0))[None, :])
    sigma = fp32_arithmetic_spread(P, x)
    dy = np.abs(y_gpu - y)
    dy_cpu = np.abs(fp32_sequential_forward(P, x) - y)
    within, within_cpu = np.mean(dy <= tol7), np.mean(dy_cpu <= tol7)
    worst = np.max(dy / (tol7 + 4.0 * sigma))
    print(f"fp32 decoder: outputs within 1e-5 max(|y|, 1e-3 rms): GPU {within:.4f}, CPU FP32 {within_cpu:.4f}; "
          f"worst |dy| / (bound + 4 sigma) {worst:.3f}; rel-L2 {rel_l2(y_gpu, y):.2e}")
    assert worst <= 1.0
    assert within >= within_cpu - 0.01
    assert rel_l2(y_gpu, y) <= 1e-6
    want_c = M.head_to_components(y)
    slope = np.concatenate([np.ones_like(y[:, :2]), np.exp(y[:, 2:]) / M.K_SPEC], axis=1)
    assert np.all(np.abs(comps.cpu().numpy() - want_c) <= (tol7 + 4.0 * sigma) * slope * 1.01 + 1e-12)
    want_rgb = M.recombine(want_c, mats, g["material"])
    np.testing.assert_allclose(rgb.cpu().numpy(), want_rgb, rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tensor_core_decoder_rel_l2(fab, setup, prec):
    mats, dec, z = setup
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 8192, stream="dec-bf16"))
    rgb, comps = fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), prec, comps=True)
    fab.sync_status()
    P = M.unpack(dec, M.DEC_SHAPES)
    want_c, want_rgb = M.shade_neural(P, z, mats, g)
    e_c, e_rgb = rel_l2(comps.cpu().numpy(), want_c), rel_l2(rgb.cpu().numpy(), want_rgb)
    emu_c, _ = emulate(prec, dec, z, mats, g)
    e_emu = rel_l2(comps.cpu().numpy(), emu_c)
    print(f"{prec} rel-L2 vs FP64: comps {e_c:.2e} rgb {e_rgb:.2e}; vs {prec} emulation {e_emu:.2e}")
    assert e_c <= TOL_FP64[prec] and e_rgb <= TOL_FP64[prec]
    assert e_emu <= TOL_EMU


def test_fp16_decoder_multiscale_footprints(fab, setup):
    """Footprints of Table 2's sizes (log-footprint feature beyond the
    1080p frame's range) through the FP16 tensor-core decoder."""
    mats, dec, z = setup
    g = W.subset(W.multiscale_gbuffer(), W.sample_indices(1920 * 1080, 8192, stream="dec-multiscale"))
    rgb, comps = fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), "fp16", comps=True)
    fab.sync_status()
    want_c, want_rgb = M.shade_neural(M.unpack(dec, M.DEC_SHAPES), z, mats, g)
    emu_c, _ = emulate("fp16", dec, z, mats, g)
    e_emu = rel_l2(comps.cpu().numpy(), emu_c)
    print(f"fp16 multi-scale: rel-L2 vs FP64 {rel_l2(comps.cpu().numpy(), want_c):.2e}, vs emulation {e_emu:.2e}")
    assert rel_l2(comps.cpu().numpy(), want_c) <= TOL_FP64["fp16"]
    assert rel_l2(rgb.cpu().numpy(), want_rgb) <= TOL_FP64["fp16"]
    assert e_emu <= TOL_EMU


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000])
def test_fp16_ragged_tiles(fab, setup, n):
    mats, dec, z = setup
    g = W.subset(W.frame_gbuffer(), np.arange(7000, 7000 + n))
    rgb, comps = fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), "fp16", comps=True)
    fab.sync_status()
    want_c, _ = M.shade_neural(M.unpack(dec, M.DEC_SHAPES), z, mats, g)
    emu_c, _ = emulate("fp16", dec, z, mats, g)
    e_emu = rel_l2(comps.cpu().numpy(), emu_c)
    print(f"fp16 ragged n={n}: rel-L2 vs FP64 {rel_l2(comps.cpu().numpy(), want_c):.2e}, vs emulation {e_emu:.2e}")
    assert rel_l2(comps.cpu().numpy(), want_c) <= TOL_FP64["fp16"]
    assert e_emu <= TOL_EMU


def test_fp16_full_frame_sampled(fab, setup):
    """The full 1080p G-buffer in the launch configuration the benchmark
    times (prepared state, one decoder launch); 8192 sampled points
    recomputed by the oracle."""
    mats, dec, z = setup
    g = W.frame_gbuffer()
    gd = GBuffer.from_numpy(g)
    fab.prepare_neural(torch.from_numpy(z).cuda(), "fp16")
    rgb, comps = fab.shade_neural_prepared(gd, "fp16", comps=True)
    fab.sync_status()
    idx = W.sample_indices(len(g["u"]), 8192, stream="dec-full")
    sub = W.subset(g, idx)
    want_c, want_rgb = M.shade_neural(M.unpack(dec, M.DEC_SHAPES), z, mats, sub)
    emu_c, _ = emulate("fp16", dec, z, mats, sub)
    e_emu = rel_l2(comps.cpu().numpy()[idx], emu_c)
    print(f"fp16 full frame: rel-L2 vs FP64 {rel_l2(comps.cpu().numpy()[idx], want_c):.2e}, "
          f"vs emulation {e_emu:.2e}")
    assert rel_l2(comps.cpu().numpy()[idx], want_c) <= TOL_FP64["fp16"]
    assert rel_l2(rgb.cpu().numpy()[idx], want_rgb) <= TOL_FP64["fp16"]
    assert e_emu <= TOL_EMU
    assert np.isfinite(rgb.cpu().numpy()).all()
    # the prepared state is refused once the parameters change
    fab.set_params(dec, W.encoder_init())
    with pytest.raises(FabricError):
        fab.shade_neural_prepared(gd, "fp16")


def test_fp16_material_limit_and_bad_index(fab, setup):
    mats, dec, z = setup
    g = W.subset(W.frame_gbuffer(), np.arange(0, 300))
    g["material"] = g["material"].copy()
    g["material"][17] = 9
    rgb, comps = fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), "fp16", comps=True)
    with pytest.raises(FabricError) as e:
        fab.sync_status()
    assert e.value.status == 7
    c = comps.cpu().numpy()
    assert np.isnan(c[17]).all() and np.isfinite(np.delete(c, 17, 0)).all()
    many = np.concatenate([mats] * 12)          # 96 materials > 89
    fab.set_materials(many)
    with pytest.raises(FabricError) as e:
        fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(W.random_latents(96)).cuda(), "fp16")
    assert e.value.status == 6
    fab.set_materials(mats)


def test_fp16_many_materials_wider_first_layer(fab, setup):
    """40 materials: the one-hot bias columns widen layer 1 to K = 80."""
    mats, dec, z = setup
    many = np.concatenate([mats] * 5)
    fab.set_materials(many)
    zz = W.random_latents(len(many), seed=11)
    g = W.subset(W.frame_gbuffer(), np.arange(0, 2000))
    g["material"] = (np.arange(2000) % len(many)).astype(np.uint16)
    _, comps = fab.shade_neural(GBuffer.from_numpy(g), torch.from_numpy(zz).cuda(), "fp16", comps=True)
    fab.sync_status()
    want_c, _ = M.shade_neural(M.unpack(dec, M.DEC_SHAPES), zz, many, g)
    emu_c, _ = emulate("fp16", dec, zz, many, g)
    fab.set_materials(mats)
    e_emu = rel_l2(comps.cpu().numpy(), emu_c)
    print(f"fp16 40 materials: rel-L2 vs FP64 {rel_l2(comps.cpu().numpy(), want_c):.2e}, vs emulation {e_emu:.2e}")
    assert rel_l2(comps.cpu().numpy(), want_c) <= TOL_FP64["fp16"]
    assert e_emu <= TOL_EMU


def test_error_stats_mixed_magnitudes(fab):
    """Elements outside the range where the reduction forms squares from FP32
    pairs (|x| below 2^-40 or above 2^60) take the FP64 path; sums still
    within 1e-12 of FP64 and the maximum exact, with both kinds mixed."""
    rng = np.random.default_rng(13)
    n = 400_000
    scale = rng.choice(np.array([1e-16, 1e-13, 1.0, 1e3, 1e19, 1e25]), size=n).astype(np.float64)
    a = (rng.standard_normal(n) * scale).astype(np.float32)
    b = (a.astype(np.float64) * (1 + 1e-3 * rng.standard_normal(n))).astype(np.float32)
    out = fab.error_stats(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    d = a.astype(np.float64) - b.astype(np.float64)
    np.testing.assert_allclose(out[0], (d * d).sum(), rtol=1e-12)
    np.testing.assert_allclose(out[1], (b.astype(np.float64) ** 2).sum(), rtol=1e-12)
    assert out[2] == np.abs(d).max()
    # the small-magnitude part alone (its sum is not swamped by the large one)
    small = np.abs(scale) < 1e-12
    out = fab.error_stats(torch.from_numpy(a[small]).cuda(), torch.from_numpy(b[small]).cuda()).cpu().numpy()
    np.testing.assert_allclose(out[0], (d[small] ** 2).sum(), rtol=1e-12)
    assert out[2] == np.abs(d[small]).max()


def test_neural_error_stats_fp64_reduction(fab, setup):
    """The FP64 image-wide error reduction against numpy on the same data."""
    rng = np.random.default_rng(9)
    a = rng.standard_normal(1_000_003).astype(np.float32)
    b = (a + 1e-3 * rng.standard_normal(a.size)).astype(np.float32)
    out = fab.error_stats(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    d = a.astype(np.float64) - b.astype(np.float64)
    np.testing.assert_allclose(out[0], (d * d).sum(), rtol=1e-12)
    np.testing.assert_allclose(out[1], (b.astype(np.float64) ** 2).sum(), rtol=1e-12)
    assert out[2] == np.abs(d).max()
    # one weight per RGB triple, read with a stride (the z of [n][3] directions)
    n = 3 * 100_001
    dirs = rng.uniform(0, 1, (n // 3, 3)).astype(np.float32)
    td = torch.from_numpy(dirs).cuda()
    out = fab.error_stats(torch.from_numpy(a[:n]).cuda(), torch.from_numpy(b[:n]).cuda(), weights=td[:, 2],
                          group=3, weight_stride=3).cpu().numpy()
    w = np.repeat(dirs[:, 2].astype(np.float64), 3)
    np.testing.assert_allclose(out[0], ((d[:n] * w) ** 2).sum(), rtol=1e-12)
    np.testing.assert_allclose(out[1], ((b[:n].astype(np.float64) * w) ** 2).sum(), rtol=1e-12)


def test_error_stats_packed_and_scalar_paths(fab):
    """The reduction takes pairs of elements with packed FP32x2 instructions
    when both arrays are 8-byte aligned and single elements otherwise: both
    forms, odd and even lengths, with and without weights, against numpy."""
    rng = np.random.default_rng(17)
    n = 300_001
    a = (rng.standard_normal(n + 1) * np.exp(rng.uniform(-30, 30, n + 1))).astype(np.float32)
    b = (a.astype(np.float64) * (1 + 1e-3 * rng.standard_normal(n + 1))).astype(np.float32)
    wts = rng.uniform(0.1, 2.0, n + 1).astype(np.float32)
    ta, tb, tw = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), torch.from_numpy(wts).cuda()
    for off_a, off_b, m in ((0, 0, n), (0, 0, n - 1), (1, 1, n), (1, 0, n - 1)):
        for weighted in (False, True):
            x, y = ta[off_a:off_a + m], tb[off_b:off_b + m]
            wv = tw[:m] if weighted else None
            out = fab.error_stats(x, y, weights=wv).cpu().numpy()
            w64 = wts[:m].astype(np.float64) if weighted else 1.0
            d = (a[off_a:off_a + m].astype(np.float64) - b[off_b:off_b + m].astype(np.float64)) * w64
            bb = b[off_b:off_b + m].astype(np.float64) * w64
            np.testing.assert_allclose(out[0], (d * d).sum(), rtol=1e-12)
            np.testing.assert_allclose(out[1], (bb * bb).sum(), rtol=1e-12)
            if weighted:
                np.testing.assert_allclose(out[2], np.abs(d).max(), rtol=1e-13)
            else:
                assert out[2] == np.abs(d).max()
