"""Latent interpolation and extrapolation (Sec. 6.4): a material edited by
mixing the latents of two encoded parameter values, decoded by the FP16
tensor-core kernel, against the oracle's decoding of the same mixed latent.

The encoder runs on the GPU at both endpoints (roughness alpha 0.2 and 0.8 on
both yarns of the 1080p frame's eight materials) and must match the FP64
encoder there; the mixed latents z(t) = z(0.2) + (t - 0.2) / 0.6 (z(0.8) -
z(0.2)) at t = 0.3, 0.6 (interpolation) and 0.9 (extrapolation) are decoded
over a sampled frame and compared with the FP64 network on the same mixed
latent, at the FP16 gates of the decoder tests (5e-3 relative L2 against
FP64, 5e-4 against the FP16 operand-rounding emulation)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mlp as M
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

TOL_FP64 = 5e-3
TOL_EMU = 5e-4


def rel_l2(got, want):
    got = np.asarray(got, np.float64)
    return float(np.sqrt(((got - want) ** 2).sum() / (want ** 2).sum()))


def emulate_fp16(P, z, mats, g):
    """FP16 operand rounding of the tensor-core path (as in the decoder tests)."""
    r = M.round_fp16
    q = r(M.query_features(g["u"], g["v"], g["radius"], g["wi"], g["wo"]))
    mat = np.asarray(g["material"], np.int64)
    fold = P["b1"][None, :] + np.asarray(z, np.float64) @ P["W1"][:, :32].T
    h = np.maximum(q @ r(P["W1"][:, 32:]).T + r(fold)[mat], 0)
    h = np.maximum(r(h) @ r(P["W2"]).T + r(P["b2"]), 0)
    h = np.maximum(r(h) @ r(P["W3"]).T + r(P["b3"]), 0)
    y = r(h) @ r(P["W4"]).T + r(P["b4"])
    comps = M.head_to_components(y)
    return comps, M.recombine(comps, mats, g["material"])


def with_alpha(base, a):
    m = base.copy()
    m["alpha"][:] = a
    return m


@pytest.mark.parametrize("t", [0.3, 0.6, 0.9])
def test_mixed_latent_decodes_like_the_oracle(fab, t):
    base = W.frame_materials()
    dec, enc = W.decoder_init(), W.encoder_init()
    fab.set_params(dec, enc)
    P, E = M.unpack(dec, M.DEC_SHAPES), M.unpack(enc, M.ENC_SHAPES)
    lo, hi = with_alpha(base, 0.2), with_alpha(base, 0.8)
    z_lo, z_hi = fab.encode_params(lo), fab.encode_params(hi)
    fab.sync_status()
    for m, zg in ((lo, z_lo), (hi, z_hi)):
        np.testing.assert_allclose(zg.cpu().numpy(), M.encoder_forward(E, M.encoder_features(m)),
                                   rtol=1e-5, atol=1e-6)
    z_mix = z_lo + (t - 0.2) / 0.6 * (z_hi - z_lo)
    mats = with_alpha(base, t)          # albedos unchanged; Eq. 8 uses them
    fab.set_materials(mats)
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 8192, stream=f"interp-{t}"))
    rgb, comps = fab.shade_neural(GBuffer.from_numpy(g), z_mix, "fp16", comps=True)
    fab.sync_status()
    zm = z_mix.cpu().numpy().astype(np.float64)
    want_c, want_rgb = M.shade_neural(P, zm, mats, g)
    emu_c, _ = emulate_fp16(P, zm, mats, g)
    c, r = comps.cpu().numpy(), rgb.cpu().numpy()
    e64, e_rgb, e_emu = rel_l2(c, want_c), rel_l2(r, want_rgb), rel_l2(c, emu_c)
    print(f"alpha {t}: mixed latent, rel-L2 vs FP64 comps {e64:.2e} rgb {e_rgb:.2e}, vs FP16 emulation {e_emu:.2e}")
    assert e64 <= TOL_FP64 and e_rgb <= TOL_FP64
    assert e_emu <= TOL_EMU
    # the mixed latent is a different material from either endpoint
    far_c, _ = M.shade_neural(P, z_lo.cpu().numpy().astype(np.float64), mats, g)
    assert rel_l2(c, far_c) > 2 * TOL_FP64
