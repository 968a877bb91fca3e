"""The tensor-core (BF16) training path of fabric_train_step against the
FP64 oracle and the FP32 path.  The gradient of one step is read back from
Adam's first moment (m = (1 - beta1) g after a step with lr = 0, saved in the
checkpoint), so the comparison needs no extra interface.  BF16 operands
(8-bit mantissas) in every product give about 1.5e-3 relative L2 error in
the decoder's gradient and 5-8e-3 in the encoder's (which receives the
latent gradients, sums of BF16 products over every query of a material);
the gates are 5e-3 and 2e-2."""
import os

import numpy as np
import pytest
import torch

import workloads as W
from oracle import mlp as M
from paper_2406_17782_gb300.api import GBuffer

pytestmark = pytest.mark.gpu

ND, NE = M.n_params(M.DEC_SHAPES), M.n_params(M.ENC_SHAPES)
TOL_DEC_BF16 = 5e-3
TOL_ENC_BF16 = 2e-2


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def gradient_from_checkpoint(path):
    raw = open(path, "rb").read()
    n = ND + NE
    adam = np.frombuffer(raw[28 + 4 * n: 28 + 4 * 3 * n], np.float32)
    return adam[:n].astype(np.float64) / (1.0 - M.ADAM_B1)


def one_step_gradient(fab, tmp_path, prec, loss_mode, mats, gd, target, dec, enc):
    fab.set_params(dec, enc)
    fab.set_train_materials(mats)
    fab.set_train_precision(prec)
    fab.set_train_loss(loss_mode)
    try:
        loss = float(fab.train_step(gd, target, 0.0).item())
        fab.sync_status()
        path = str(tmp_path / f"g_{prec}_{loss_mode}.ckpt")
        fab.checkpoint_save(path)
    finally:
        fab.set_train_precision("fp32")
        fab.set_train_loss("eq11")
    return loss, gradient_from_checkpoint(path)


def oracle_gradient(mats, g, target, dec, enc, loss_mode):
    P, E = M.unpack(dec.astype(np.float64), M.DEC_SHAPES), M.unpack(enc.astype(np.float64), M.ENC_SHAPES)
    f = M.encoder_features(mats)
    z, ec = M.encoder_forward(E, f, keep=True)
    x = M.decoder_inputs(z, g["material"], g)
    y, dc = M.decoder_forward(P, x, keep=True)
    loss, dy = M.loss_and_grad(y, target.astype(np.float64), loss_mode, np.asarray(g["wi"], np.float64)[:, 2])
    gd, dx = M.decoder_backward(P, dc, dy)
    dz = np.zeros_like(z)
    np.add.at(dz, np.asarray(g["material"], np.int64), dx[:, :M.LATENT])
    ge = M.encoder_backward(E, ec, dz)
    return loss, np.concatenate([M.pack(gd, M.DEC_SHAPES), M.pack(ge, M.ENC_SHAPES)])


@pytest.mark.parametrize("loss_mode", ["eq11", "rendered"])
@pytest.mark.parametrize("n", [4096, 1000])
def test_tensor_core_gradient_matches_oracle(fab, tmp_path, loss_mode, n):
    mats = W.training_materials(2)
    g = W.training_queries(n, len(mats), stream=f"tc-grad-{n}")
    target = np.abs(np.random.default_rng(8).standard_normal((n, 4)) * 0.2).astype(np.float32)
    gd, tt = GBuffer.from_numpy(g), torch.from_numpy(target).cuda()
    dec, enc = W.decoder_init(weight_bound="small"), W.encoder_init(weight_bound="small")
    want_loss, want = oracle_gradient(mats, g, target, dec, enc, loss_mode)
    loss_bf, g_bf = one_step_gradient(fab, tmp_path, "bf16", loss_mode, mats, gd, tt, dec, enc)
    loss_32, g_32 = one_step_gradient(fab, tmp_path, "fp32", loss_mode, mats, gd, tt, dec, enc)
    print(f"{loss_mode} n={n}: loss bf16 {loss_bf:.6g} fp32 {loss_32:.6g} fp64 {want_loss:.6g}; "
          f"grad rel-L2 bf16 {rel_l2(g_bf, want):.2e} (decoder {rel_l2(g_bf[:ND], want[:ND]):.2e}, "
          f"encoder {rel_l2(g_bf[ND:], want[ND:]):.2e}), fp32 {rel_l2(g_32, want):.2e}")
    assert abs(loss_32 - want_loss) <= 1e-5 * abs(want_loss)
    assert rel_l2(g_32, want) <= 1e-4
    assert abs(loss_bf - want_loss) <= 2e-2 * abs(want_loss)
    assert rel_l2(g_bf[:ND], want[:ND]) <= TOL_DEC_BF16 and rel_l2(g_bf[ND:], want[ND:]) <= TOL_ENC_BF16


def test_tensor_core_gradient_many_materials(fab, tmp_path):
    """1600 materials: too many for the kernel to fold the per-material
    latent-gradient sums into its partials, so the separate per-material
    reduction runs instead; the gradient still matches the oracle."""
    mats = W.training_materials(200)
    n = 4096
    g = W.training_queries(n, len(mats), stream="tc-grad-many")
    target = np.abs(np.random.default_rng(10).standard_normal((n, 4)) * 0.2).astype(np.float32)
    gd, tt = GBuffer.from_numpy(g), torch.from_numpy(target).cuda()
    dec, enc = W.decoder_init(weight_bound="small"), W.encoder_init(weight_bound="small")
    want_loss, want = oracle_gradient(mats, g, target, dec, enc, "eq11")
    loss_bf, g_bf = one_step_gradient(fab, tmp_path, "bf16", "eq11", mats, gd, tt, dec, enc)
    print(f"1600 materials: loss bf16 {loss_bf:.6g} fp64 {want_loss:.6g}; grad rel-L2 decoder "
          f"{rel_l2(g_bf[:ND], want[:ND]):.2e}, encoder {rel_l2(g_bf[ND:], want[ND:]):.2e}")
    assert abs(loss_bf - want_loss) <= 2e-2 * abs(want_loss)
    assert rel_l2(g_bf[:ND], want[:ND]) <= TOL_DEC_BF16 and rel_l2(g_bf[ND:], want[ND:]) <= TOL_ENC_BF16


@pytest.mark.parametrize("n", [65536, 6 * 152 * 128 + 77])
def test_tensor_core_gradient_large_batch(fab, tmp_path, n):
    """Batches whose CTAs take up to five tiles (the latent-gradient rows
    stay in tensor memory until the per-material sums) and more than five
    (the rows go through global memory): both match the oracle."""
    mats = W.training_materials(2)
    g = W.training_queries(n, len(mats), stream=f"tc-grad-large-{n}")
    target = np.abs(np.random.default_rng(12).standard_normal((n, 4)) * 0.2).astype(np.float32)
    gd, tt = GBuffer.from_numpy(g), torch.from_numpy(target).cuda()
    dec, enc = W.decoder_init(weight_bound="small"), W.encoder_init(weight_bound="small")
    want_loss, want = oracle_gradient(mats, g, target, dec, enc, "eq11")
    loss_bf, g_bf = one_step_gradient(fab, tmp_path, "bf16", "eq11", mats, gd, tt, dec, enc)
    print(f"n={n}: loss bf16 {loss_bf:.6g} fp64 {want_loss:.6g}; grad rel-L2 decoder "
          f"{rel_l2(g_bf[:ND], want[:ND]):.2e}, encoder {rel_l2(g_bf[ND:], want[ND:]):.2e}")
    assert abs(loss_bf - want_loss) <= 2e-2 * abs(want_loss)
    assert rel_l2(g_bf[:ND], want[:ND]) <= TOL_DEC_BF16 and rel_l2(g_bf[ND:], want[ND:]) <= TOL_ENC_BF16


def test_tensor_core_training_is_repeatable_and_learns(fab):
    mats = W.training_materials(2)
    g = W.training_queries(8192, len(mats), stream="tc-learn")
    target = np.abs(np.random.default_rng(9).standard_normal((8192, 4)) * 0.2).astype(np.float32)
    gd, tt = GBuffer.from_numpy(g), torch.from_numpy(target).cuda()
    fab.set_train_materials(mats)
    fab.set_train_precision("bf16")
    runs = []
    try:
        for _ in range(2):
            fab.set_params(W.decoder_init(weight_bound="small"), W.encoder_init(weight_bound="small"))
            losses = [float(fab.train_step(gd, tt, 3e-3).item()) for _ in range(100)]
            fab.sync_status()
            runs.append((losses, fab.get_params()))
    finally:
        fab.set_train_precision("fp32")
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1][0], runs[1][1][0]) and np.array_equal(runs[0][1][1], runs[1][1][1])
    assert runs[0][0][-1] < 0.5 * runs[0][0][0]


@pytest.mark.parametrize("n,k", [(64, 16), (64, 64), (16, 32), (32, 48)])
def test_mn_major_operand_layout(fab, n, k):
    """The weight-gradient products read both operands MN-major from shared
    memory; one product in isolation against FP64 on the BF16-rounded inputs."""
    rng = np.random.default_rng(7 * n + k)
    a = rng.standard_normal((128, k)).astype(np.float32)
    b = rng.standard_normal((n, k)).astype(np.float32)
    d = fab.selftest_mma_mn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    fab.sync_status()
    want = M.round_bf16(a).astype(np.float64) @ M.round_bf16(b).astype(np.float64).T
    np.testing.assert_allclose(d, want, rtol=1e-5, atol=1e-5)
