"""Pins of the FP64 network oracle: encoding values, closed-form tiny nets,
central finite differences, Eq. 9-11 closed forms, Adam's first step and the
BF16 / E4M3 rounding against torch's own casts (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def M(oracle_mod):
    return oracle_mod.mlp


def test_frequency_encoding_values(M):
    # u = 0.125: f_k = 0.125, 0.25, 0.5, 0, 0, ... periods
    s2 = math.sqrt(0.5)
    want = [s2, s2, 1.0, 0.0, 0.0, -1.0] + [0.0, 1.0] * 5
    for u in [0.125, 3.125, 47.125]:
        got = M.freq_encode(np.array([np.float32(u)]))[0]
        np.testing.assert_allclose(got, want, atol=1e-15)
    # every frequency is periodic in one pattern repeat
    u = np.float32(0.3710937500)
    a = M.freq_encode(np.array([u]))
    b = M.freq_encode(np.array([u + np.float32(5.0)]))
    np.testing.assert_array_equal(a, b)


def test_log_footprint_map(M):
    np.testing.assert_allclose(M.log_footprint(np.array([1e-4, 1e-1, math.sqrt(1e-5)])), [-1, 1, 0],
                               atol=1e-12)
    assert np.isfinite(M.log_footprint(np.array([0.0]))).all()


def _zero_dec(M):
    return {k: np.zeros(s) for k, s in M.DEC_SHAPES}


def test_decoder_closed_form_tiny_net(M):
    """Units that copy one input each through the ReLU chain: the head must
    return exactly those inputs (where positive) plus its bias."""
    p = _zero_dec(M)
    # latent[3] -> unit 0, l (index 32+32) -> unit 1, wi_z (index 67) -> unit 2, -wo_x -> unit 3
    p["W1"][0, 3] = 1.0
    p["W1"][1, 64] = 1.0
    p["W1"][2, 67] = 1.0
    p["W1"][3, 68] = -1.0
    for L in ("W2", "W3"):
        p[L][:4, :4] = np.eye(4)
    p["W4"][:, :4] = np.diag([2.0, 1.0, 1.0, 0.5])
    p["b4"][:] = [0.1, 0.2, 0.3, 0.4]
    z = np.zeros((2, 32))
    z[1, 3] = 0.7
    g = dict(u=np.float32([0.1, 0.2]), v=np.float32([0.3, 0.4]), radius=np.float32([1e-1, 1e-4]),
             wi=np.float32([[0, 0, 1], [0.6, 0, 0.8]]), wo=np.float32([[-0.6, 0, 0.8], [0.6, 0, 0.8]]))
    x = M.decoder_inputs(z, np.array([0, 1]), g)
    assert x.shape == (2, 71)
    y = M.decoder_forward(p, x)
    want = np.array([[0.1, 0.2 + 1.0, 0.3 + 1.0, 0.4 + 0.5 * 0.6],
                     [0.1 + 2 * 0.7, 0.2 + 0.0, 0.3 + 0.8, 0.4 + 0.0]])
    np.testing.assert_allclose(y, want, atol=1e-6)


def _rand_dec(M, rng, scale=0.3):
    return {k: scale * rng.standard_normal(s) for k, s in M.DEC_SHAPES}


def _rand_enc(M, rng, scale=0.2):
    return {k: scale * rng.standard_normal(s) for k, s in M.ENC_SHAPES}


def test_decoder_backward_finite_differences(M):
    rng = np.random.default_rng(0)
    p = _rand_dec(M, rng)
    x = rng.standard_normal((6, 71))
    dy = rng.standard_normal((6, 4))
    y, cache = M.decoder_forward(p, x, keep=True)
    g, dx = M.decoder_backward(p, cache, dy)
    f = lambda pp, xx: float(np.sum(dy * M.decoder_forward(pp, xx)))
    h = 1e-6
    for name, shape in M.DEC_SHAPES:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in shape)
            pp = {k: v.copy() for k, v in p.items()}
            pp[name][idx] += h
            fp = f(pp, x)
            pp[name][idx] -= 2 * h
            fm = f(pp, x)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[name][idx])
    for _ in range(10):
        i, j = rng.integers(0, 6), rng.integers(0, 71)
        xx = x.copy()
        xx[i, j] += h
        fp = f(p, xx)
        xx[i, j] -= 2 * h
        fm = f(p, xx)
        assert abs((fp - fm) / (2 * h) - dx[i, j]) <= 1e-6 * max(1.0, abs(dx[i, j]))


def test_encoder_backward_finite_differences(M):
    rng = np.random.default_rng(1)
    p = _rand_enc(M, rng)
    f_in = M.encoder_features(W.table2_materials(rng, range(8)))
    dz = rng.standard_normal((8, 32))
    z, cache = M.encoder_forward(p, f_in, keep=True)
    g = M.encoder_backward(p, cache, dz)
    f = lambda pp: float(np.sum(dz * M.encoder_forward(pp, f_in)))
    h = 1e-6
    for name, shape in M.ENC_SHAPES:
        for _ in range(8):
            idx = tuple(rng.integers(0, s) for s in shape)
            pp = {k: v.copy() for k, v in p.items()}
            pp[name][idx] += h
            fp = f(pp)
            pp[name][idx] -= 2 * h
            fm = f(pp)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)


def test_encoder_features_layout(M):
    m = W.make_material(pattern=5, twist_deg=-30, incl_deg=45, alpha=[0.2, 0.9], beta=[1.5, 0.5],
                        kd=[[0.1] * 3, [0.2] * 3], ks=[[0.3] * 3, [0.4] * 3])
    f = M.encoder_features(m)[0]
    want = np.zeros(22)
    want[5] = 1
    want[16:] = [-1, 1, 0.2, 1.5, 0.9, 0.5]
    np.testing.assert_allclose(f, want, atol=1e-7)


def test_loss_closed_form_and_gradient(M):
    c = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert (M.LAMBDA_S, M.LAMBDA_C, M.K_SPEC) == (c["lambda_S"]["value"], c["lambda_C"]["value"],
                                                  c["k_brdf"]["value"])
    tgt = np.array([[0.2, 0.1, 0.05, 0.0], [0.4, 0.3, 0.0, 0.01]])
    y = np.zeros_like(tgt)
    loss, dy = M.loss_and_grad(y, tgt)
    gS = np.log(100 * tgt[:, 2:] + 1)
    want = 0.4 * (np.mean(gS[:, 0] ** 2) + np.mean(gS[:, 1] ** 2)) + \
        0.1 * (np.mean(tgt[:, 0] ** 2) + np.mean(tgt[:, 1] ** 2))
    assert abs(loss - want) < 1e-15
    # a perfect prediction (y = g(target) for S, y = target for C) has zero loss
    perfect = np.concatenate([tgt[:, :2], gS], 1)
    assert M.loss_and_grad(perfect, tgt)[0] < 1e-30
    rng = np.random.default_rng(2)
    y = rng.standard_normal(tgt.shape)
    _, dy = M.loss_and_grad(y, tgt)
    h = 1e-7
    for i in range(2):
        for j in range(4):
            yp = y.copy(); yp[i, j] += h
            ym = y.copy(); ym[i, j] -= h
            fd = (M.loss_and_grad(yp, tgt)[0] - M.loss_and_grad(ym, tgt)[0]) / (2 * h)
            assert abs(fd - dy[i, j]) < 1e-7


def test_rendered_loss_closed_form_and_gradient(M):
    """The rendered-space loss option: its value on a hand-computed case, zero
    for the prediction that decodes to the target, no weight on light from
    below the surface, and central finite differences of its gradient
    (including past the head clamp, where it is 0)."""
    tgt = np.array([[0.2, 0.1, 0.05, 0.0], [0.4, 0.3, 0.0, 0.01], [1.0, 1.0, 1.0, 1.0]])
    wz = np.array([0.5, 1.0, -0.3])
    y = np.zeros_like(tgt)                       # decodes to C = 0, S = 0
    loss, _ = M.loss_and_grad(y, tgt, "rendered", wz)
    want = ((0.2 ** 2 + 0.1 ** 2 + 0.05 ** 2) * 0.25 + (0.4 ** 2 + 0.3 ** 2 + 0.01 ** 2) * 1.0) / 3
    assert abs(loss - want) < 1e-15
    perfect = np.concatenate([tgt[:, :2], np.log(100 * tgt[:, 2:] + 1)], 1)
    assert M.loss_and_grad(perfect, tgt, "rendered", wz)[0] < 1e-30
    rng = np.random.default_rng(3)
    y = rng.standard_normal(tgt.shape)
    y[0, 3] = 13.0                               # beyond the clamp
    _, dy = M.loss_and_grad(y, tgt, "rendered", wz)
    assert dy[0, 3] == 0.0 and np.all(dy[2] == 0.0)
    h = 1e-4      # the clamped entry makes the loss ~2e5: a larger step keeps rounding below 1e-6
    for i in range(3):
        for j in range(4):
            yp = y.copy(); yp[i, j] += h
            ym = y.copy(); ym[i, j] -= h
            fd = (M.loss_and_grad(yp, tgt, "rendered", wz)[0] - M.loss_and_grad(ym, tgt, "rendered", wz)[0]) / (2 * h)
            assert abs(fd - dy[i, j]) < 1e-6 * max(1.0, abs(dy[i, j]))


def test_head_inverts_specular_mapping(M):
    S = np.array([0.0, 1e-3, 0.05, 2.0])
    y = np.zeros((4, 4))
    y[:, 2] = np.log(100 * S + 1)
    y[:, 0] = [-1, 0, 0.5, 2]
    out = M.head_to_components(y)
    np.testing.assert_allclose(out[:, 2], S, atol=1e-15)
    np.testing.assert_allclose(out[:, 0], [0, 0, 0.5, 2])


def test_adam_first_step_is_sign_step(M):
    rng = np.random.default_rng(3)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = M.adam_step(th, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    np.testing.assert_allclose(new, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_fp64_training_reduces_loss(M):
    rng = np.random.default_rng(4)
    mats = W.training_materials(2)
    g = W.training_queries(256, len(mats), stream="oracle-train")
    target = np.abs(rng.standard_normal((256, 4))) * 0.1
    dec = W.decoder_init().astype(np.float64)
    enc = W.encoder_init().astype(np.float64)
    state = {}
    losses = []
    for _ in range(60):
        loss, dec, enc = M.train_step(dec, enc, state, mats, g["material"], g, target, 1e-3)
        losses.append(loss)
    assert losses[-1] < 0.5 * losses[0]


def test_bf16_rounding_matches_torch(M):
    torch = pytest.importorskip("torch")
    one = 1.0
    ulp = 2.0 ** -7
    # ties go to the even neighbour
    np.testing.assert_array_equal(M.round_bf16([one + ulp / 2, one + 1.5 * ulp, -(one + ulp / 2)]),
                                  [one, one + 2 * ulp, -one])
    x = np.random.default_rng(5).standard_normal(10000) * np.exp(np.random.default_rng(6).uniform(-20, 20, 10000))
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.round_bf16(x), want)


def test_e4m3_rounding_matches_torch(M):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    np.testing.assert_array_equal(M.round_e4m3([448.0, 1000.0, -1000.0, 2.0 ** -9, 2.0 ** -10]),
                                  [448.0, 448.0, -448.0, 2.0 ** -9, 0.0])
    rng = np.random.default_rng(7)
    x = rng.uniform(-440, 440, 20000) * np.exp(rng.uniform(-14, 0, 20000))
    x = x.astype(np.float32).astype(np.float64)
    want = torch.tensor(x, dtype=torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.round_e4m3(x), want)


def test_e4m3_scale_exponent_places_amax_below_the_e4m3_maximum(M):
    rng = np.random.default_rng(11)
    for mag in (1e-6, 3e-3, 0.3, 1.0, 7.5, 300.0):
        w = rng.standard_normal((64, 64)) * mag
        e = M.e4m3_scale_exponent(w)
        top = float(np.float32(np.abs(w).max())) * 2.0 ** e
        assert 128.0 <= top < 256.0
    # exact powers of two land on 128 exactly
    assert M.e4m3_scale_exponent(np.array([[0.5, -0.25]])) == 8
    assert float(0.5 * 2.0 ** 8) == 128.0


def test_e4m3_emulation_reduces_to_the_network_without_rounding(M):
    """With identity rounding the E4M3 emulation (folded latent, scaled
    weights, FP32 bias epilogue) is the FP64 network up to FP32 rounding of
    the intermediate values: a dropped bias, an unreverted scale or a
    transposed operand fails this."""
    import workloads as W
    mats = W.frame_materials()
    P = M.unpack(W.decoder_init(), M.DEC_SHAPES)
    z = W.random_latents(len(mats))
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 2048, stream="e4m3-pin"))
    want, want_rgb = M.shade_neural(P, z, mats, g)
    ident = lambda x: np.asarray(x, np.float64)
    got, got_rgb = M.shade_neural_e4m3(P, z, mats, g, r16=ident, r8=ident)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max())
    np.testing.assert_allclose(got_rgb, want_rgb, rtol=1e-5, atol=1e-6 * np.abs(want_rgb).max())
    # with E4M3 rounding the error is that of a 3-bit mantissa, not a bug's
    q, _ = M.shade_neural_e4m3(P, z, mats, g)
    rel = np.sqrt(((q - want) ** 2).sum() / (want ** 2).sum())
    assert 1e-2 < rel < 0.3


def test_recombine_eq8_hand_values(M):
    """Eq. 8 on hand-set components and albedos, the colours worked out by
    hand: material 0 has every albedo different (a warp / weft or diffuse /
    specular swap changes the result), material 1 only a specular weft
    albedo."""
    mats = np.zeros(2, W.MATERIAL_DTYPE)
    mats[0]["kd"] = [[0.125, 0.25, 0.375], [0.5, 0.0, 0.0]]
    mats[0]["ks"] = [[0.0, 0.25, 0.0], [0.0, 0.0, 1.0]]
    mats[1]["ks"] = [[0.0, 0.0, 0.0], [2.0, 4.0, 8.0]]
    comps = np.array([[1.0, 2.0, 3.0, 4.0],       # C_warp, C_weft, S_warp, S_weft
                      [0.5, 0.0, 0.0, 0.25],
                      [1.0, 2.0, 3.0, 4.0]])
    rgb = M.recombine(comps, mats, np.array([0, 1, 1]))
    # R = 0.125*1 + 0.5*2 + 0*3 + 0*4; G = 0.25*1 + 0*2 + 0.25*3 + 0*4; B = 0.375*1 + 0 + 0 + 1*4
    want = np.array([[1.125, 1.0, 4.375],
                     [0.5, 1.0, 2.0],
                     [8.0, 16.0, 32.0]])
    np.testing.assert_array_equal(rgb, want)


def test_e4m3_rounding_margin(M):
    """The margin is the relative distance to the nearest E4M3 rounding
    midpoint: zero exactly at a midpoint (1.0625 between 1 and 1.125; the
    subnormal midpoint 2^-10 below 2^-9), half a spacing at a representable
    value, and the rounding of values nudged across a midpoint flips."""
    np.testing.assert_allclose(M.e4m3_rounding_margin(np.array([1.0625, 2.0 ** -10, -3.125])), 0.0, atol=1e-15)
    np.testing.assert_allclose(M.e4m3_rounding_margin(np.array([1.0, 1.125, 416.0])),
                               [0.0625, 0.0625 / 1.125, 16.0 / 416.0], rtol=1e-14)
    mid = 1.0625
    assert M.round_e4m3(mid * (1 - 1e-9)) == 1.0 and M.round_e4m3(mid * (1 + 1e-9)) == 1.125
    assert np.isinf(M.e4m3_rounding_margin(np.array([0.0]))).all()
    # FP16 (10 mantissa bits, normals from 2^-14): 1 + 2^-11 is the midpoint
    # between 1 and 1 + 2^-10; 0.75 is representable, half a spacing from both
    # midpoints around it
    np.testing.assert_allclose(M.rounding_midpoint_distance(np.array([1 + 2.0 ** -11, 0.75]), 10, -14),
                               [0.0, 2.0 ** -12], atol=0)
    assert np.float16(1 + 2.0 ** -11 * (1 - 1e-6)) == 1.0 and np.float16(1 + 2.0 ** -11 * (1 + 1e-6)) > 1.0
