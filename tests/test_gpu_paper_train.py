"""Training of the paper's decoder structure (fabric_paper_train_step)
against the FP64 oracle: the encoder's latents, the loss and the full
gradient [decoder | encoder] of one step (read back after a step with
lr = 0), at both widths and both losses, for the full structure and its two
ablations (Sec. 6.3); repeatability and learning; the FP32 forward
(fabric_paper_shade_fp32) of every structure."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mlp as M
from oracle import paper_net as PN
from paper_2406_17782_gb300 import FabricError
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


ABL = {"full": PN.FULL, "no_oneblob": PN.NO_ONEBLOB, "no_fusion": PN.NO_FUSION}


def oracle_step(w, mats, g, target, dec, enc, loss_mode, ablation="full"):
    a = ABL[ablation]
    P = M.unpack(dec.astype(np.float64), PN.dec_shapes(w, a))
    E = M.unpack(enc.astype(np.float64), PN.ENC_SHAPES)
    z, ec = M.encoder_forward(E, M.encoder_features(mats), keep=True)
    mat = np.asarray(g["material"], np.int64)
    y, dc = PN.decoder_forward(P, z[mat], PN.spatial_features(g["u"], g["v"], g["radius"], a),
                               PN.angular_features(g["wi"], g["wo"]), keep=True)
    loss, dy = M.loss_and_grad(y, target.astype(np.float64), loss_mode, np.asarray(g["wi"], np.float64)[:, 2])
    gd, dzr, _ = PN.decoder_backward(P, dc, dy)
    dz = np.zeros_like(z)
    np.add.at(dz, mat, dzr)
    ge = M.encoder_backward(E, ec, dz)
    return loss, np.concatenate([M.pack(gd, PN.dec_shapes(w, a)), M.pack(ge, PN.ENC_SHAPES)])


@pytest.mark.parametrize("w", [64, 128])
def test_paper_encoder_matches_oracle(fab, w):
    mats = W.training_materials(4)
    enc = W.paper_encoder_init()
    fab.paper_set_params(w, W.paper_decoder_init(w), enc)
    z = fab.paper_encode_params(mats).cpu().numpy()
    want = M.encoder_forward(M.unpack(enc, PN.ENC_SHAPES), M.encoder_features(mats))
    np.testing.assert_allclose(z, want, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("loss_mode", ["eq11", "rendered"])
@pytest.mark.parametrize("w,n", [(64, 4096), (128, 4096), (64, 1000)])
def test_paper_gradient_matches_oracle(fab, w, n, loss_mode):
    mats = W.training_materials(2)
    g = W.training_queries(n, len(mats), stream=f"paper-grad-{n}")
    target = np.abs(np.random.default_rng(18).standard_normal((n, 4)) * 0.2).astype(np.float32)
    dec, enc = W.paper_decoder_init(w, weight_bound="small"), W.paper_encoder_init(weight_bound="small")
    want_loss, want = oracle_step(w, mats, g, target, dec, enc, loss_mode)
    fab.paper_set_params(w, dec, enc)
    fab.set_train_materials(mats)
    fab.set_train_loss(loss_mode)
    try:
        loss = float(fab.paper_train_step(GBuffer.from_numpy(g), torch.from_numpy(target).cuda(), 0.0).item())
        fab.sync_status()
        got = fab.paper_gradient()
    finally:
        fab.set_train_loss("eq11")
    nd = M.n_params(PN.dec_shapes(w))
    print(f"paper W={w} {loss_mode} n={n}: loss {loss:.7g} vs {want_loss:.7g}; grad rel-L2 decoder "
          f"{rel_l2(got[:nd], want[:nd]):.2e}, encoder {rel_l2(got[nd:], want[nd:]):.2e}")
    assert abs(loss - want_loss) <= 1e-5 * abs(want_loss)
    assert rel_l2(got[:nd], want[:nd]) <= 1e-4 and rel_l2(got[nd:], want[nd:]) <= 1e-4
    # the one step with lr = 0 left the parameters unchanged
    d, e = fab.paper_get_params()
    assert np.array_equal(d, dec) and np.array_equal(e, enc)


@pytest.mark.parametrize("w", [64, 128])
def test_paper_gradient_full_batch(fab, w):
    """The benchmark's step: a batch of 65 536 queries over 256 training
    materials (every weight-gradient chunk and latent-sum segment of the
    launch the bench times), against the oracle."""
    mats = W.training_materials(32)
    g = W.training_queries(65536, len(mats), stream="paper-full-batch")
    target = np.abs(np.random.default_rng(24).standard_normal((65536, 4)) * 0.2).astype(np.float32)
    dec, enc = W.paper_decoder_init(w, weight_bound="small"), W.paper_encoder_init(weight_bound="small")
    want_loss, want = oracle_step(w, mats, g, target, dec, enc, "rendered")
    fab.paper_set_params(w, dec, enc)
    fab.set_train_materials(mats)
    fab.set_train_loss("rendered")
    try:
        loss = float(fab.paper_train_step(GBuffer.from_numpy(g), torch.from_numpy(target).cuda(), 0.0).item())
        fab.sync_status()
        got = fab.paper_gradient()
    finally:
        fab.set_train_loss("eq11")
    nd = M.n_params(PN.dec_shapes(w))
    print(f"paper W={w} full batch: loss {loss:.7g} vs {want_loss:.7g}; grad rel-L2 decoder "
          f"{rel_l2(got[:nd], want[:nd]):.2e}, encoder {rel_l2(got[nd:], want[nd:]):.2e}")
    assert abs(loss - want_loss) <= 1e-5 * abs(want_loss)
    assert rel_l2(got[:nd], want[:nd]) <= 1e-4 and rel_l2(got[nd:], want[nd:]) <= 1e-4


def test_paper_gradient_many_materials(fab):
    """1600 training materials (the limit: per-material latent sums in a
    1600 x 32 shared-memory table) at width 128, against the oracle; 1601
    are refused."""
    w = 128
    mats = W.training_materials(200)
    assert len(mats) == 1600
    g = W.training_queries(8192, len(mats), stream="paper-many")
    target = np.abs(np.random.default_rng(23).standard_normal((8192, 4)) * 0.2).astype(np.float32)
    dec, enc = W.paper_decoder_init(w, weight_bound="small"), W.paper_encoder_init(weight_bound="small")
    want_loss, want = oracle_step(w, mats, g, target, dec, enc, "eq11")
    fab.paper_set_params(w, dec, enc)
    fab.set_train_materials(mats)
    loss = float(fab.paper_train_step(GBuffer.from_numpy(g), torch.from_numpy(target).cuda(), 0.0).item())
    fab.sync_status()
    got = fab.paper_gradient()
    nd = M.n_params(PN.dec_shapes(w))
    print(f"paper W={w} 1600 materials: loss {loss:.7g} vs {want_loss:.7g}; grad rel-L2 decoder "
          f"{rel_l2(got[:nd], want[:nd]):.2e}, encoder {rel_l2(got[nd:], want[nd:]):.2e}")
    assert abs(loss - want_loss) <= 1e-5 * abs(want_loss)
    assert rel_l2(got[:nd], want[:nd]) <= 1e-4 and rel_l2(got[nd:], want[nd:]) <= 1e-4
    fab.set_train_materials(np.concatenate([mats, mats[:1]]))
    try:
        with pytest.raises(FabricError) as err:
            fab.paper_train_step(GBuffer.from_numpy(g), torch.from_numpy(target).cuda(), 0.0)
        assert err.value.status == 6
    finally:
        fab.set_train_materials(mats[:16])


def test_paper_training_is_repeatable_and_learns(fab):
    w = 64
    mats = W.training_materials(2)
    g = W.training_queries(8192, len(mats), stream="paper-learn")
    target = np.abs(np.random.default_rng(19).standard_normal((8192, 4)) * 0.2).astype(np.float32)
    gd, tt = GBuffer.from_numpy(g), torch.from_numpy(target).cuda()
    fab.set_train_materials(mats)
    runs = []
    for _ in range(2):
        fab.paper_set_params(w, W.paper_decoder_init(w, weight_bound="small"),
                             W.paper_encoder_init(weight_bound="small"))
        losses = [float(fab.paper_train_step(gd, tt, 3e-3).item()) for _ in range(100)]
        fab.sync_status()
        runs.append((losses, fab.paper_get_params()))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1][0], runs[1][1][0]) and np.array_equal(runs[0][1][1], runs[1][1][1])
    assert runs[0][0][-1] < 0.5 * runs[0][0][0]


@pytest.mark.parametrize("ablation", ["no_oneblob", "no_fusion"])
@pytest.mark.parametrize("w,n", [(64, 4096), (128, 1000)])
def test_paper_ablation_gradient_matches_oracle(fab, w, n, ablation):
    """The ablated structures' step (S1 over [z | frac u | frac v | t]; no
    S1/S2, A1 over [z | one-blob | angular]) against the oracle's."""
    mats = W.training_materials(2)
    g = W.training_queries(n, len(mats), stream=f"paper-abl-{n}")
    target = np.abs(np.random.default_rng(21).standard_normal((n, 4)) * 0.2).astype(np.float32)
    dec = W.paper_decoder_init(w, weight_bound="small", ablation=ablation)
    enc = W.paper_encoder_init(weight_bound="small")
    want_loss, want = oracle_step(w, mats, g, target, dec, enc, "eq11", ablation)
    fab.paper_set_params(w, dec, enc, ablation=ablation)
    fab.set_train_materials(mats)
    try:
        loss = float(fab.paper_train_step(GBuffer.from_numpy(g), torch.from_numpy(target).cuda(), 0.0).item())
        fab.sync_status()
        got = fab.paper_gradient()
        d, e = fab.paper_get_params()
    finally:
        fab.paper_set_params(w, W.paper_decoder_init(w), W.paper_encoder_init())
    nd = M.n_params(PN.dec_shapes(w, ABL[ablation]))
    assert got.size == want.size and d.size == nd
    print(f"paper {ablation} W={w} n={n}: loss {loss:.7g} vs {want_loss:.7g}; grad rel-L2 decoder "
          f"{rel_l2(got[:nd], want[:nd]):.2e}, encoder {rel_l2(got[nd:], want[nd:]):.2e}")
    assert abs(loss - want_loss) <= 1e-5 * abs(want_loss)
    assert rel_l2(got[:nd], want[:nd]) <= 1e-4 and rel_l2(got[nd:], want[nd:]) <= 1e-4
    assert np.array_equal(d, dec) and np.array_equal(e, enc)


@pytest.mark.parametrize("ablation", ["full", "no_oneblob", "no_fusion"])
@pytest.mark.parametrize("w", [64, 128])
def test_paper_fp32_forward_matches_oracle(fab, w, ablation):
    """fabric_paper_shade_fp32 on sampled frame points (several 64-row
    tiles and a ragged tail) against the FP64 network: relative L2 <= 1e-5
    on components and RGB, per point <= 1e-4 of the components' scale."""
    mats = W.frame_materials()
    fab.set_materials(mats)
    dec = W.paper_decoder_init(w, ablation=ablation)
    fab.paper_set_params(w, dec, W.paper_encoder_init(), ablation=ablation)
    try:
        z = W.random_latents(len(mats), seed=33, dim=64)
        g = W.subset(W.frame_gbuffer(), W.sample_indices(1920 * 1080, 3001, stream="paper-fp32"))
        rgb, comps = fab.paper_shade_fp32(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), comps=True)
        fab.sync_status()
        want_c, want_rgb = PN.shade(M.unpack(dec, PN.dec_shapes(w, ABL[ablation])), z, mats, g, ABL[ablation])
        c, r = comps.cpu().numpy(), rgb.cpu().numpy()
        e_c, e_r = rel_l2(c, want_c), rel_l2(r, want_rgb)
        worst = float(np.abs(c - want_c).max() / np.abs(want_c).max())
        print(f"paper FP32 forward {ablation} W={w}: rel-L2 comps {e_c:.2e} rgb {e_r:.2e}, worst {worst:.2e}")
        assert e_c <= 1e-5 and e_r <= 1e-5 and worst <= 1e-4
        if ablation != "full":
            with pytest.raises(FabricError) as err:
                fab.paper_shade_neural(GBuffer.from_numpy(g), torch.from_numpy(z).cuda(), "fp16")
            assert err.value.status == 6
    finally:
        fab.paper_set_params(w, W.paper_decoder_init(w), W.paper_encoder_init())


def test_paper_fp32_forward_bad_material(fab):
    mats = W.frame_materials()
    fab.set_materials(mats)
    fab.paper_set_params(64, W.paper_decoder_init(64, ablation="no_fusion"), W.paper_encoder_init(),
                         ablation="no_fusion")
    try:
        g = W.subset(W.frame_gbuffer(), np.arange(0, 200))
        g["material"] = g["material"].copy()
        g["material"][17] = len(mats)
        rgb, comps = fab.paper_shade_fp32(GBuffer.from_numpy(g), torch.from_numpy(
            W.random_latents(len(mats), dim=64)).cuda(), comps=True)
        with pytest.raises(FabricError) as e:
            fab.sync_status()
        assert e.value.status == 7
        c = comps.cpu().numpy()
        assert np.isnan(c[17]).all() and np.isfinite(np.delete(c, 17, 0)).all()
    finally:
        fab.paper_set_params(64, W.paper_decoder_init(64), W.paper_encoder_init())


def test_paper_ablation_trains(fab):
    """A few hundred steps of each ablation lower its loss, repeatably."""
    mats = W.training_materials(2)
    g = W.training_queries(8192, len(mats), stream="paper-abl-learn")
    target = np.abs(np.random.default_rng(22).standard_normal((8192, 4)) * 0.2).astype(np.float32)
    gd, tt = GBuffer.from_numpy(g), torch.from_numpy(target).cuda()
    fab.set_train_materials(mats)
    try:
        for ablation in ("no_oneblob", "no_fusion"):
            runs = []
            for _ in range(2):
                fab.paper_set_params(64, W.paper_decoder_init(64, weight_bound="small", ablation=ablation),
                                     W.paper_encoder_init(weight_bound="small"), ablation=ablation)
                runs.append([float(fab.paper_train_step(gd, tt, 3e-3).item()) for _ in range(100)])
                fab.sync_status()
            assert runs[0] == runs[1]
            assert runs[0][-1] < 0.5 * runs[0][0]
    finally:
        fab.paper_set_params(64, W.paper_decoder_init(64), W.paper_encoder_init())
