"""Parity of the tensor-core kernel of the paper's decoder structure (Sec.
4.2, Fig. 3: one-blob spatial encoding, spatial fusion, angular decoder with
a residual skip) with its FP64 oracle.

Against the oracle's operand-rounding emulation of the same path (16-bit
one-blob channels, angular inputs, weights, biases and activations; the
latent folded into a rounded per-material bias; the skip adding the rounded
k1; FP32 accumulation): relative L2 <= 5e-4.  Against the unrounded FP64
network: FP16 <= 5e-3, BF16 <= 1.5e-2 (BF16 operand rounding alone: 3e-3 at width
64, 7e-3 at 128).
Widths 64 and 128."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mlp as M
from oracle import paper_net as PN
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

TOL_EMU = 5e-4
TOL_FP64 = {"fp16": 5e-3, "bf16": 1.5e-2}
ROUND = {"fp16": M.round_fp16, "bf16": M.round_bf16}


def rel_l2(got, want):
    got = np.asarray(got, np.float64)
    return float(np.sqrt(((got - want) ** 2).sum() / (want ** 2).sum()))


@pytest.fixture(scope="module", params=[64, 128])
def net(fab, request):
    w = request.param
    mats = W.frame_materials()
    fab.set_materials(mats)
    dec = W.paper_decoder_init(w)
    fab.paper_set_params(w, dec, W.paper_encoder_init())
    z = W.random_latents(len(mats), seed=31, dim=64)
    return w, mats, dec, z


def run(fab, net, g, prec, z=None, mats=None):
    w, mats0, dec, z0 = net
    z = z0 if z is None else z
    mats = mats0 if mats is None else mats
    rgb, comps = fab.paper_shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), prec, comps=True)
    fab.sync_status()
    P = M.unpack(dec, PN.dec_shapes(w))
    want_c, want_rgb = PN.shade(P, z, mats, g)
    emu_c, emu_rgb = PN.shade_rounded(P, z, mats, g, ROUND[prec])
    c, r = comps.cpu().numpy(), rgb.cpu().numpy()
    return dict(c64=rel_l2(c, want_c), rgb64=rel_l2(r, want_rgb), emu=rel_l2(c, emu_c), emu_rgb=rel_l2(r, emu_rgb),
                finite=bool(np.isfinite(c).all() and np.isfinite(r).all()))


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_paper_decoder_sampled_frame(fab, net, prec):
    g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 8192, stream="paper-dec"))
    e = run(fab, net, g, prec)
    print(f"paper decoder W={net[0]} {prec}: rel-L2 vs FP64 comps {e['c64']:.2e} rgb {e['rgb64']:.2e}; "
          f"vs emulation comps {e['emu']:.2e} rgb {e['emu_rgb']:.2e}")
    assert e["finite"]
    assert e["emu"] <= TOL_EMU and e["emu_rgb"] <= TOL_EMU
    assert e["c64"] <= TOL_FP64[prec] and e["rgb64"] <= TOL_FP64[prec]


def test_paper_decoder_multiscale_footprints(fab, net):
    g = W.subset(W.multiscale_gbuffer(), W.sample_indices(1920 * 1080, 8192, stream="paper-dec-ms"))
    e = run(fab, net, g, "fp16")
    print(f"paper decoder W={net[0]} multi-scale: vs FP64 {e['c64']:.2e}, vs emulation {e['emu']:.2e}")
    assert e["emu"] <= TOL_EMU and e["c64"] <= TOL_FP64["fp16"]


@pytest.mark.parametrize("n", [1, 127, 129, 1000])
def test_paper_decoder_ragged_tiles(fab, net, n):
    g = W.subset(W.frame_gbuffer(), np.arange(5000, 5000 + n))
    e = run(fab, net, g, "fp16")
    print(f"paper decoder W={net[0]} n={n}: vs FP64 {e['c64']:.2e}, vs emulation {e['emu']:.2e}")
    assert e["emu"] <= TOL_EMU and e["c64"] <= TOL_FP64["fp16"]


def test_paper_decoder_full_frame_sampled(fab, net):
    """The whole 1080p G-buffer through the prepared one-launch path (the
    benchmark's launch), 8192 sampled points recomputed by the oracle; the
    prepared state is refused once the parameters change."""
    w, mats, dec, z = net
    g = W.frame_gbuffer()
    gd = GBuffer.from_numpy(g)
    fab.paper_prepare(torch.from_numpy(z).cuda(), "fp16")
    rgb, comps = fab.paper_shade_prepared(gd, "fp16", comps=True)
    fab.sync_status()
    idx = W.sample_indices(len(g["u"]), 8192, stream="paper-dec-full")
    sub = W.subset(g, idx)
    P = M.unpack(dec, PN.dec_shapes(w))
    emu_c, _ = PN.shade_rounded(P, z, mats, sub, M.round_fp16)
    want_c, _ = PN.shade(P, z, mats, sub)
    c = comps.cpu().numpy()
    print(f"paper decoder W={w} full frame: vs FP64 {rel_l2(c[idx], want_c):.2e}, vs emulation "
          f"{rel_l2(c[idx], emu_c):.2e}")
    assert rel_l2(c[idx], emu_c) <= TOL_EMU and rel_l2(c[idx], want_c) <= TOL_FP64["fp16"]
    assert np.isfinite(rgb.cpu().numpy()).all()
    fab.paper_set_params(w, dec, W.paper_encoder_init())
    with pytest.raises(FabricError):
        fab.paper_shade_prepared(gd, "fp16")


def test_paper_decoder_most_materials(fab, net):
    """104 materials: the one-hot bias columns widen the first layer to
    K = 128, its limit; 105 are refused."""
    w, mats, dec, z = net
    many = np.concatenate([mats] * 13)
    fab.set_materials(many)
    try:
        zz = W.random_latents(len(many), seed=32, dim=64)
        g = W.subset(W.frame_gbuffer(), np.arange(0, 3000))
        g["material"] = (np.arange(3000) % len(many)).astype(np.uint16)
        e = run(fab, net, g, "fp16", z=zz, mats=many)
        print(f"paper decoder W={w} 104 materials: vs FP64 {e['c64']:.2e}, vs emulation {e['emu']:.2e}")
        assert e["emu"] <= TOL_EMU and e["c64"] <= TOL_FP64["fp16"]
        fab.set_materials(np.concatenate([many, mats[:1]]))
        with pytest.raises(FabricError) as err:
            fab.paper_shade_neural(GBuffer.from_numpy(g), torch.from_numpy(W.random_latents(105, dim=64)).cuda())
        assert err.value.status == 6
    finally:
        fab.set_materials(mats)


def test_paper_decoder_bad_material_index(fab, net):
    w, mats, dec, z = net
    g = W.subset(W.frame_gbuffer(), np.arange(0, 300))
    g["material"] = g["material"].copy()
    g["material"][40] = 9
    rgb, comps = fab.paper_shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), "fp16", comps=True)
    with pytest.raises(FabricError) as e:
        fab.sync_status()
    assert e.value.status == 7
    c = comps.cpu().numpy()
    assert np.isnan(c[40]).all() and np.isfinite(np.delete(c, 40, 0)).all()
