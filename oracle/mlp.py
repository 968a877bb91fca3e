"""FP64 numpy oracle for the neural representation: query encoding, decoder and
encoder forward/backward, the loss of Eq. 9-11, Adam, and BF16 / E4M3 operand
rounding.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written from the paper's
Sec. 4.2 (encoder-decoder, residual block, four-component head of Eq. 7) and
Sec. 4.3 (losses), with the decoder shape of the workload under test:
[z(32) | enc(u)(16) | enc(v)(16) | l(1) | wi(3) | wo(3)] -> 64 -> 64 -> 64 -> 4,
ReLU.  Matrix products are numpy library calls; everything else is spelled
out step by step.

Parameter layout (flat float vectors, shared as an interface with the CUDA
library, each side implementing it on its own):
  decoder: W1[64][71] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[4][64] b4[4]
  encoder: E1[128][22] e1[128] E2[128][128] e2[128] E3[32][128] e3[32]
Weights are [out][in] (row = output unit).
"""
from __future__ import annotations

import math

import numpy as np

LATENT = 32
N_FREQ = 8
N_QFEAT = 2 * 2 * N_FREQ + 1 + 3 + 3      # 39 query features
N_IN = LATENT + N_QFEAT                   # 71
HIDDEN = 64
N_OUT = 4                                 # C_warp, C_weft, S_warp, S_weft (Eq. 7)
N_PATTERN_SLOTS = 16                      # one-hot width of the weave id (ids 0..11 in use)
ENC_IN = N_PATTERN_SLOTS + 6
ENC_HIDDEN = 128

DEC_SHAPES = [("W1", (HIDDEN, N_IN)), ("b1", (HIDDEN,)),
              ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
              ("W3", (HIDDEN, HIDDEN)), ("b3", (HIDDEN,)),
              ("W4", (N_OUT, HIDDEN)), ("b4", (N_OUT,))]
ENC_SHAPES = [("E1", (ENC_HIDDEN, ENC_IN)), ("e1", (ENC_HIDDEN,)),
              ("E2", (ENC_HIDDEN, ENC_HIDDEN)), ("e2", (ENC_HIDDEN,)),
              ("E3", (LATENT, ENC_HIDDEN)), ("e3", (LATENT,))]

# Log-footprint feature: l = (ln max(r, 2^-20) - c0) / c1 maps r in [1e-4, 1e-1]
# onto [-1, 1]; the floor keeps l finite for the r -> 0 queries of data
# generation.  (The workload only says "log footprint"; this affine map and
# the floor are this build's reading.)
LOG_R_C0 = 0.5 * (math.log(1e-4) + math.log(1e-1))
LOG_R_C1 = 0.5 * (math.log(1e-1) - math.log(1e-4))
R_FLOOR = 2.0 ** -20

K_SPEC = 100.0          # g(x) = ln(k x + 1), k = 100 for BRDFs (Eq. 9)
LAMBDA_S = 0.4          # Eq. 11
LAMBDA_C = 0.1
LEAKY = 0.01            # encoder residual block activation slope (reading)


def n_params(shapes) -> int:
    return sum(int(np.prod(s)) for _, s in shapes)


def unpack(flat: np.ndarray, shapes) -> dict:
    out, off = {}, 0
    flat = np.asarray(flat, np.float64)
    for name, s in shapes:
        k = int(np.prod(s))
        out[name] = flat[off:off + k].reshape(s).copy()
        off += k
    assert off == len(flat), (off, len(flat))
    return out


def pack(p: dict, shapes) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in shapes])


# --------------------------------------------------------------------------
# query encoding
# --------------------------------------------------------------------------
def freq_encode(u: np.ndarray) -> np.ndarray:
    """Weave-periodic sin/cos encoding: f_k = frac(2^k frac(u)), k = 0..7,
    features (sin 2 pi f_k, cos 2 pi f_k) interleaved per k.  All steps are
    exact in FP64 for float32 u."""
    u = np.asarray(u, np.float64)
    f0 = u - np.floor(u)
    feats = []
    for k in range(N_FREQ):
        fk = f0 * (2.0 ** k)
        fk = fk - np.floor(fk)
        feats.append(np.sin(2.0 * np.pi * fk))
        feats.append(np.cos(2.0 * np.pi * fk))
    return np.stack(feats, axis=-1)


def log_footprint(r: np.ndarray) -> np.ndarray:
    r = np.maximum(np.asarray(r, np.float64), R_FLOOR)
    return (np.log(r) - LOG_R_C0) / LOG_R_C1


def query_features(u, v, r, wi, wo) -> np.ndarray:
    """The 39 query features: enc(u) | enc(v) | l | wi | wo."""
    return np.concatenate([freq_encode(u), freq_encode(v), log_footprint(r)[:, None],
                           np.asarray(wi, np.float64), np.asarray(wo, np.float64)], axis=1)


def decoder_inputs(z: np.ndarray, material: np.ndarray, gbuf: dict) -> np.ndarray:
    """Full 71-wide decoder input: latent of each point's material, then the
    query features."""
    zq = np.asarray(z, np.float64)[np.asarray(material, np.int64)]
    q = query_features(gbuf["u"], gbuf["v"], gbuf["radius"], gbuf["wi"], gbuf["wo"])
    return np.concatenate([zq, q], axis=1)


# --------------------------------------------------------------------------
# decoder
# --------------------------------------------------------------------------
def relu(x):
    return np.maximum(x, 0.0)


def decoder_forward(p: dict, x: np.ndarray, keep: bool = False):
    """Raw head output y = W4 h3 + b4 (no output activation, as trained)."""
    a1 = x @ p["W1"].T + p["b1"]
    h1 = relu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = relu(a2)
    a3 = h2 @ p["W3"].T + p["b3"]
    h3 = relu(a3)
    y = h3 @ p["W4"].T + p["b4"]
    if keep:
        return y, dict(x=x, a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3)
    return y


def decoder_backward(p: dict, cache: dict, dy: np.ndarray):
    """Gradients of sum(dy * y) w.r.t. every decoder parameter and the input
    (ReLU'(0) = 0)."""
    g = {}
    g["W4"] = dy.T @ cache["h3"]
    g["b4"] = dy.sum(0)
    dh3 = dy @ p["W4"]
    da3 = dh3 * (cache["a3"] > 0)
    g["W3"] = da3.T @ cache["h2"]
    g["b3"] = da3.sum(0)
    dh2 = da3 @ p["W3"]
    da2 = dh2 * (cache["a2"] > 0)
    g["W2"] = da2.T @ cache["h1"]
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (cache["a1"] > 0)
    g["W1"] = da1.T @ cache["x"]
    g["b1"] = da1.sum(0)
    dx = da1 @ p["W1"]
    return g, dx


def head_to_components(y: np.ndarray) -> np.ndarray:
    """Inference head: C = max(0, y), S = max(0, (exp(y) - 1) / k), the
    inverse of Eq. 9's g(x) = ln(k x + 1)."""
    out = np.empty_like(y)
    out[:, 0:2] = np.maximum(y[:, 0:2], 0.0)
    out[:, 2:4] = np.maximum(np.expm1(y[:, 2:4]) / K_SPEC, 0.0)
    return out


def recombine(comps: np.ndarray, materials, material_idx: np.ndarray) -> np.ndarray:
    """Eq. 8: f = kd_warp C_warp + kd_weft C_weft + ks_warp S_warp + ks_weft S_weft."""
    m = np.atleast_1d(materials)
    idx = np.asarray(material_idx, np.int64)
    kd = m["kd"].astype(np.float64)[idx]      # [n, 2, 3]
    ks = m["ks"].astype(np.float64)[idx]
    return (kd[:, 0] * comps[:, 0:1] + kd[:, 1] * comps[:, 1:2]
            + ks[:, 0] * comps[:, 2:3] + ks[:, 1] * comps[:, 3:4])


def shade_neural(dec: dict, z: np.ndarray, materials, gbuf: dict):
    """Per-point neural shading: (components [n,4], rgb [n,3])."""
    x = decoder_inputs(z, gbuf["material"], gbuf)
    comps = head_to_components(decoder_forward(dec, x))
    return comps, recombine(comps, materials, gbuf["material"])


# --------------------------------------------------------------------------
# encoder (parameters -> latent), residual block of Sec. 4.2
# --------------------------------------------------------------------------
def lrelu(x):
    return np.where(x > 0, x, LEAKY * x)


def encoder_features(materials) -> np.ndarray:
    """22 inputs: one-hot weave id (16 slots) | psi / 30 deg | u / 45 deg |
    alpha_warp | beta_warp | alpha_weft | beta_weft.  Albedos are not inputs
    (they enter only through Eq. 8)."""
    m = np.atleast_1d(materials)
    f = np.zeros((len(m), ENC_IN))
    f[np.arange(len(m)), m["pattern"].astype(np.int64)] = 1.0
    b = N_PATTERN_SLOTS
    f[:, b + 0] = m["twist_deg"].astype(np.float64) / 30.0
    f[:, b + 1] = m["incl_deg"].astype(np.float64) / 45.0
    f[:, b + 2] = m["alpha"][:, 0].astype(np.float64)
    f[:, b + 3] = m["beta"][:, 0].astype(np.float64)
    f[:, b + 4] = m["alpha"][:, 1].astype(np.float64)
    f[:, b + 5] = m["beta"][:, 1].astype(np.float64)
    return f


def encoder_forward(p: dict, f: np.ndarray, keep: bool = False):
    a1 = f @ p["E1"].T + p["e1"]
    h1 = lrelu(a1)
    a2 = h1 @ p["E2"].T + p["e2"] + h1          # skip before the last activation
    h2 = lrelu(a2)
    z = h2 @ p["E3"].T + p["e3"]
    if keep:
        return z, dict(f=f, a1=a1, h1=h1, a2=a2, h2=h2)
    return z


def encoder_backward(p: dict, cache: dict, dz: np.ndarray):
    g = {}
    g["E3"] = dz.T @ cache["h2"]
    g["e3"] = dz.sum(0)
    dh2 = dz @ p["E3"]
    da2 = dh2 * np.where(cache["a2"] > 0, 1.0, LEAKY)
    g["E2"] = da2.T @ cache["h1"]
    g["e2"] = da2.sum(0)
    dh1 = da2 @ p["E2"] + da2                     # through the skip
    da1 = dh1 * np.where(cache["a1"] > 0, 1.0, LEAKY)
    g["E1"] = da1.T @ cache["f"]
    g["e1"] = da1.sum(0)
    return g


# --------------------------------------------------------------------------
# loss (Eq. 9-11)
# --------------------------------------------------------------------------
Y_CLAMP = 12.0          # head pre-activation limit of the rendered-space loss


def loss_and_grad(y: np.ndarray, target: np.ndarray, mode: str = "eq11", wz=None):
    """y: raw head [B,4] = (C_warp, C_weft, S'_warp, S'_weft); target: ground
    truth components [B,4].

    mode "eq11" (Eq. 9-11): sum over yarn types of
    lambda_S mean (S' - ln(k S_gt + 1))^2 + lambda_C mean (C - C_gt)^2.

    mode "rendered" (this build's option): the squared error of the
    components as they light the frame, (1/B) sum_p sum_c ((c_hat - c_gt)
    max(wz, 0))^2 with wz = <wi . n_s> per query, c_hat = y for C and
    c_hat = (exp(min(S', 12)) - 1) / k for S (the inverse of Eq. 9 without
    the inference clamp at 0; the gradient is 0 above the limit)."""
    if mode == "rendered":
        return _loss_rendered(np.asarray(y, np.float64), np.asarray(target, np.float64),
                              np.asarray(wz, np.float64))
    if mode != "eq11":
        raise ValueError(mode)
    B = y.shape[0]
    t = np.empty_like(target, dtype=np.float64)
    t[:, 0:2] = target[:, 0:2]
    t[:, 2:4] = np.log(K_SPEC * np.asarray(target[:, 2:4], np.float64) + 1.0)
    d = y - t
    lam = np.array([LAMBDA_C, LAMBDA_C, LAMBDA_S, LAMBDA_S])
    loss = float(np.sum(lam * np.mean(d * d, axis=0)))
    dy = 2.0 * lam * d / B
    return loss, dy


def _loss_rendered(y, target, wz):
    B = y.shape[0]
    w = np.maximum(wz, 0.0)[:, None]
    c = y.copy()
    ys = np.minimum(y[:, 2:4], Y_CLAMP)
    c[:, 2:4] = np.expm1(ys) / K_SPEC
    dc = np.ones_like(y)
    dc[:, 2:4] = np.where(y[:, 2:4] < Y_CLAMP, np.exp(ys) / K_SPEC, 0.0)
    d = (c - target) * w
    loss = float(np.sum(d * d) / B)
    dy = 2.0 * d * w * dc / B
    return loss, dy


# --------------------------------------------------------------------------
# Adam (Kingma and Ba 2015, bias-corrected)
# --------------------------------------------------------------------------
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(theta, grad, m, v, step: int, lr: float):
    """One update at 1-based step `step`; returns new (theta, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * grad * grad
    mh = m / (1.0 - ADAM_B1 ** step)
    vh = v / (1.0 - ADAM_B2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def train_step(dec_flat, enc_flat, state: dict, materials, mat_idx, gbuf, target, lr: float,
               loss_mode: str = "eq11"):
    """One full training step in FP64: encoder over all materials, decoder over
    the batch, the loss (Eq. 11, or the rendered-space option of
    loss_and_grad), backward through both, Adam on the concatenated
    [decoder | encoder] parameter vector.  Returns (loss, new dec, new enc)."""
    dec = unpack(dec_flat, DEC_SHAPES)
    enc = unpack(enc_flat, ENC_SHAPES)
    f = encoder_features(materials)
    z, ecache = encoder_forward(enc, f, keep=True)
    x = decoder_inputs(z, mat_idx, gbuf)
    y, dcache = decoder_forward(dec, x, keep=True)
    loss, dy = loss_and_grad(y, target, loss_mode, np.asarray(gbuf["wi"], np.float64)[:, 2])
    gd, dx = decoder_backward(dec, dcache, dy)
    dz = np.zeros_like(z)
    np.add.at(dz, np.asarray(mat_idx, np.int64), dx[:, :LATENT])
    ge = encoder_backward(enc, ecache, dz)
    theta = np.concatenate([np.asarray(dec_flat, np.float64), np.asarray(enc_flat, np.float64)])
    grad = np.concatenate([pack(gd, DEC_SHAPES), pack(ge, ENC_SHAPES)])
    state["step"] = state.get("step", 0) + 1
    if "m" not in state:
        state["m"] = np.zeros_like(theta)
        state["v"] = np.zeros_like(theta)
    theta, state["m"], state["v"] = adam_step(theta, grad, state["m"], state["v"], state["step"], lr)
    nd = n_params(DEC_SHAPES)
    return loss, theta[:nd], theta[nd:]


# --------------------------------------------------------------------------
# operand rounding (for the quantisation-emulating comparisons)
# --------------------------------------------------------------------------
def round_bf16(x) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even), returned as FP64."""
    f = np.asarray(x, np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


E4M3_MAX = 448.0


def round_e4m3(x) -> np.ndarray:
    """Round to OCP FP8 E4M3 (4 exponent bits, bias 7, 3 mantissa bits,
    subnormal quantum 2^-9, finite maximum 448), ties to even, saturating."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 2.0 ** -6)))
    q = 2.0 ** (e - 3)
    r = np.round(a / q) * q             # np.round is ties-to-even
    r = np.minimum(r, E4M3_MAX)
    return np.sign(x) * r


def round_fp16(x) -> np.ndarray:
    """Round to IEEE binary16 (ties to even) via FP32, returned as FP64."""
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float64)


def e4m3_scale_exponent(w) -> int:
    """Per-layer power-of-two weight scale of the E4M3 operand path: with
    amax = max |w| written as m 2^E (m in [0.5, 1), frexp of the FP32 value),
    the weights are stored as E4M3(w 2^(8 - E)), so the largest lands in
    [128, 256) below the E4M3 maximum of 448 and no weight is rescaled
    inexactly.  Returns 8 - E (the scale is 2^(8 - E))."""
    amax = np.float32(np.max(np.abs(np.asarray(w, np.float32))))
    _, e = np.frexp(amax)
    return 8 - int(e)


def rounding_midpoint_distance(x, mant_bits: int, emin: int) -> np.ndarray:
    """Absolute distance of each value to the nearest rounding boundary (the
    midpoint between two neighbouring representable values) of a binary
    format with `mant_bits` stored mantissa bits and smallest normal
    exponent `emin` (subnormals below 2^emin)."""
    a = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.maximum(a, 2.0 ** emin)))
    q = 2.0 ** (e - mant_bits)
    t = a / q
    return np.abs(t - (np.floor(t) + 0.5)) * q


def e4m3_rounding_margin(x) -> np.ndarray:
    """Relative distance of each value to the nearest E4M3 rounding
    boundary (the midpoint between two neighbouring E4M3 values): where it
    is tiny, two evaluations whose FP32 sums differ in their last bits can
    round the value to different E4M3 neighbours.  inf at exact zeros."""
    a = np.abs(np.asarray(x, np.float64))
    d = rounding_midpoint_distance(a, 3, -6)
    with np.errstate(divide="ignore"):
        return np.where(a > 0, d / a, np.inf)


def shade_neural_e4m3(dec: dict, z: np.ndarray, materials, gbuf: dict,
                      r16=round_fp16, r8=round_e4m3, diag: dict | None = None):
    """Operand-rounding emulation of the E4M3 tensor-core decoder.

    Layer 1 keeps 16-bit operands (r16): its weight block carries the latent
    folded into a per-material bias column (W1 z_m + b1), which E4M3 would
    cut to 3 mantissa bits.  Layers 2-4 take E4M3 operands (r8): the
    activations unscaled (saturating at 448), the weights scaled by the
    per-layer power of two of e4m3_scale_exponent; their biases and the
    undoing of the scale are applied in FP32 to the FP32 product.  Every
    value is rounded to FP32 before it is rounded to an operand type, as in
    the kernel.  With r16 = r8 = identity this is the FP64 network up to
    those FP32 roundings.  Returns (components [n, 4], rgb [n, 3]); when
    `diag` is a dict, the values that the path rounds are stored in it (to
    find where another evaluation whose features or sums differ in their
    last bits may round differently): "features" (FP32 query features
    [n, 39], before FP16 rounding), "w1" (the rounded layer-1 feature
    weights [64, 39]), "fold" (the FP32 folded bias columns [n_mat, 64],
    before FP16 rounding) and "pre" (per E4M3 layer, the ReLU'd FP32 values
    before E4M3 rounding, [n, 64] each)."""
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    q32 = f32(query_features(gbuf["u"], gbuf["v"], gbuf["radius"], gbuf["wi"], gbuf["wo"]))
    q = r16(q32)
    mat = np.asarray(gbuf["material"], np.int64)
    zf = np.asarray(z, np.float64)
    fold = dec["b1"][None, :] + zf @ dec["W1"][:, :LATENT].T            # [n_mat, 64]
    w1 = r16(f32(dec["W1"][:, LATENT:]))
    a = q @ w1.T + r16(f32(fold))[mat]
    pres = [np.maximum(f32(a), 0.0)]
    h = r8(pres[0])
    for wn, bn, last in (("W2", "b2", False), ("W3", "b3", False), ("W4", "b4", True)):
        s = 2.0 ** e4m3_scale_exponent(dec[wn])
        a = f32(f32(h @ r8(f32(dec[wn]) * s).T) / s + f32(dec[bn]))
        if not last:
            pres.append(np.maximum(a, 0.0))
        h = a if last else r8(pres[-1])
    if diag is not None:
        diag.update(features=q32, w1=w1, fold=f32(fold), pre=pres)
    comps = head_to_components(h)
    return comps, recombine(comps, materials, gbuf["material"])
