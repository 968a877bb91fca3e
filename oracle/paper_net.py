"""FP64 numpy oracle for the paper's own decoder structure (Sec. 4.2,
"Decoder"; Fig. 3): one-blob encoding of the footprint's position and size,
a two-layer spatial fusion of the material latent with them, and an angular
decoder of five fully connected layers with one skip connection.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Written from the
paper's description, with this build's readings where it is silent:

* One-blob encoding (Mueller et al., "Neural Importance Sampling", 2019):
  a scalar s in [0, 1] becomes k = 8 bins, bin i holding a Gaussian of
  standard deviation 1/k centred at s, evaluated at the bin centre
  (i + 1/2) / k.  The footprint centre (frac u, frac v) is periodic in the
  weave repeat, so its distance to a bin centre wraps around the unit
  interval (the Gaussian is wrapped: summed over all its periodic
  images); the footprint size enters as
  t = ln(max(r, 2^-20) / 1e-4) / ln(2.5 / 1e-4), which maps the half sides
  1e-4 (the 1080p frame's smallest) and 2.5 (the largest of Table 2, a side
  of five repeats) to 0 and 1.  3 inputs -> 24 channels, as the paper says.
* Latent z in R^64 (the paper's size), from the parameter encoder of the
  workload with 64 outputs.
* Spatial fusion: h = lrelu(S2 lrelu(S1 [z | onehot-blob] + s1) + s2),
  width W.
* Angular decoder on [h | wi (x, y, z) | wo (x, y)] (the paper's angular
  inputs): k1 = lrelu(A1 x + a1); a residual block of two layers whose skip
  joins before the last leaky ReLU, k3 = lrelu(A3 lrelu(A2 k1 + a2) + a3 + k1);
  k4 = lrelu(A4 k3 + a4); y = A5 k4 + a5 (four components, Eq. 7).  Five
  fully connected layers, one skip.
* Leaky ReLU slope 0.01; widths W = 64 or 128 (the paper gives none).

Parameter layout (flat float vectors, weights [out][in]; shared as an
interface with the CUDA library, each side implementing it on its own):
  S1[W][88] s1[W] S2[W][W] s2[W] A1[W][W+5] a1[W] A2[W][W] a2[W]
  A3[W][W] a3[W] A4[W][W] a4[W] A5[4][W] a5[4]
Ablations (Sec. 6.3 varies the one-blob encoding and the spatial fusion):
without the one-blob encoding S1 is [W][67] over [z | frac u, frac v, t];
without the spatial fusion the angular decoder gains two hidden layers in
their place (Sec. 6.3 adds hidden layers for a fair comparison):
H1[W][93] h1[W] H2[W][W] h2[W] over [z | one-blob | wi | wo.xy], then
A1[W][W] a1[W] over their output and A2..a5 as above (same size as the
full structure).
Encoder: E1[128][22] e1[128] E2[128][128] e2[128] E3[64][128] e3[64], the
workload's residual encoder (oracle.mlp) with a 64-wide output.
"""
from __future__ import annotations

import math

import numpy as np

from . import mlp

LATENT = 64
BINS = 8
SIGMA = 1.0 / BINS
N_BLOB = 3 * BINS                         # 24 one-blob channels
N_ANG = 5                                 # wi (x, y, z), wo (x, y)
SLOPE = 0.01
R_LO = 1e-4
R_HI = 2.5
WIDTHS = (64, 128)


# Ablations of the structure (Sec. 6.3 studies the one-blob encoding and the
# spatial fusion): FULL is the structure above; NO_ONEBLOB feeds the three
# spatial inputs (frac u, frac v, size coordinate t) unencoded; NO_FUSION
# queries space and angle together: the section keeps the comparison fair by
# giving the angular decoder more hidden layers when the fusion goes, and
# here the two fusion layers become the angular decoder's first two hidden
# layers H1, H2 over [z | one-blob | angular], then A1 [W][W] over their
# output (same depth and parameter count as FULL).
FULL, NO_ONEBLOB, NO_FUSION = 0, 1, 2
N_RAW = 3


def n_spatial(ablation: int = FULL) -> int:
    return N_RAW if ablation == NO_ONEBLOB else N_BLOB


def dec_shapes(w: int, ablation: int = FULL):
    tail = [("A2", (w, w)), ("a2", (w,)), ("A3", (w, w)), ("a3", (w,)), ("A4", (w, w)), ("a4", (w,)),
            ("A5", (mlp.N_OUT, w)), ("a5", (mlp.N_OUT,))]
    if ablation == NO_FUSION:
        return [("H1", (w, LATENT + N_BLOB + N_ANG)), ("h1", (w,)), ("H2", (w, w)), ("h2", (w,)),
                ("A1", (w, w)), ("a1", (w,))] + tail
    return [("S1", (w, LATENT + n_spatial(ablation))), ("s1", (w,)), ("S2", (w, w)), ("s2", (w,)),
            ("A1", (w, w + N_ANG)), ("a1", (w,))] + tail


def _front(p: dict):
    """Names of the two layers before A1: the spatial fusion (S1, S2), or
    the angular decoder's added hidden layers without it (H1, H2)."""
    return ("S1", "s1", "S2", "s2") if "S1" in p else ("H1", "h1", "H2", "h2")


ENC_SHAPES = [("E1", (mlp.ENC_HIDDEN, mlp.ENC_IN)), ("e1", (mlp.ENC_HIDDEN,)),
              ("E2", (mlp.ENC_HIDDEN, mlp.ENC_HIDDEN)), ("e2", (mlp.ENC_HIDDEN,)),
              ("E3", (LATENT, mlp.ENC_HIDDEN)), ("e3", (LATENT,))]


def lrelu(x):
    return np.where(x > 0, x, SLOPE * x)


def dlrelu(x):
    return np.where(x > 0, 1.0, SLOPE)


# --------------------------------------------------------------------------
# one-blob encoding
# --------------------------------------------------------------------------
def oneblob(s: np.ndarray, periodic: bool) -> np.ndarray:
    """[n] -> [n, 8]: exp(-d^2 / (2 sigma^2)) with d the distance from s to
    bin centre (i + 1/2) / 8.  Periodic: the Gaussian wrapped around the
    unit interval, i.e. summed over the images d + m of every integer m
    (here m = -2..2; farther images weigh below exp(-200))."""
    s = np.asarray(s, np.float64)[:, None]
    c = (np.arange(BINS) + 0.5) / BINS
    d = s - c[None, :]
    if not periodic:
        return np.exp(-d * d / (2.0 * SIGMA * SIGMA))
    d = d - np.round(d)
    return sum(np.exp(-(d + m) ** 2 / (2.0 * SIGMA * SIGMA)) for m in range(-2, 3))


def size_coordinate(r: np.ndarray) -> np.ndarray:
    r = np.maximum(np.asarray(r, np.float64), mlp.R_FLOOR)
    return np.log(r / R_LO) / math.log(R_HI / R_LO)


def spatial_features(u, v, r, ablation: int = FULL) -> np.ndarray:
    """The 24 one-blob channels: frac(u) (8, periodic) | frac(v) (8,
    periodic) | footprint size (8); for NO_ONEBLOB the three inputs
    themselves (frac u, frac v, t)."""
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    fu, fv, t = u - np.floor(u), v - np.floor(v), size_coordinate(r)
    if ablation == NO_ONEBLOB:
        return np.stack([fu, fv, t], axis=1)
    return np.concatenate([oneblob(fu, True), oneblob(fv, True), oneblob(t, False)], axis=1)


def angular_features(wi, wo) -> np.ndarray:
    wi = np.asarray(wi, np.float64)
    wo = np.asarray(wo, np.float64)
    return np.concatenate([wi[:, :3], wo[:, :2]], axis=1)


# --------------------------------------------------------------------------
# decoder
# --------------------------------------------------------------------------
def decoder_forward(p: dict, z: np.ndarray, blob: np.ndarray, ang: np.ndarray, keep: bool = False):
    """Raw head y [n, 4] from per-point latents z [n, 64], spatial channels
    [n, 24] (or [n, 3] without the one-blob encoding) and angular inputs
    [n, 5].  With the spatial fusion the angular inputs join its output at
    A1; without it (H1, H2 in place of S1, S2) they enter the first layer
    with z and the spatial channels."""
    fusion = "S1" in p
    W1, b1, W2, b2 = _front(p)
    z = np.asarray(z, np.float64)
    x0 = np.concatenate([z, blob] if fusion else [z, blob, ang], axis=1)
    c = dict(x0=x0)
    c["g1"] = x0 @ p[W1].T + p[b1]
    c["h1"] = lrelu(c["g1"])
    c["g2"] = c["h1"] @ p[W2].T + p[b2]
    xa = np.concatenate([lrelu(c["g2"]), ang], axis=1) if fusion else lrelu(c["g2"])
    c["xa"] = xa
    c["q1"] = xa @ p["A1"].T + p["a1"]
    c["k1"] = lrelu(c["q1"])
    c["q2"] = c["k1"] @ p["A2"].T + p["a2"]
    c["k2"] = lrelu(c["q2"])
    c["q3"] = c["k2"] @ p["A3"].T + p["a3"] + c["k1"]     # skip joins before the last leaky ReLU
    c["k3"] = lrelu(c["q3"])
    c["q4"] = c["k3"] @ p["A4"].T + p["a4"]
    c["k4"] = lrelu(c["q4"])
    y = c["k4"] @ p["A5"].T + p["a5"]
    return (y, c) if keep else y


def decoder_backward(p: dict, c: dict, dy: np.ndarray):
    """Gradients of sum(dy * y) w.r.t. every parameter, the latents and the
    angular inputs: (grads, dz [n, 64], dang [n, 5])."""
    W1, b1, W2, b2 = _front(p)
    g = {}
    g["A5"] = dy.T @ c["k4"]
    g["a5"] = dy.sum(0)
    dq4 = (dy @ p["A5"]) * dlrelu(c["q4"])
    g["A4"] = dq4.T @ c["k3"]
    g["a4"] = dq4.sum(0)
    dq3 = (dq4 @ p["A4"]) * dlrelu(c["q3"])
    g["A3"] = dq3.T @ c["k2"]
    g["a3"] = dq3.sum(0)
    dq2 = (dq3 @ p["A3"]) * dlrelu(c["q2"])
    g["A2"] = dq2.T @ c["k1"]
    g["a2"] = dq2.sum(0)
    dq1 = (dq2 @ p["A2"] + dq3) * dlrelu(c["q1"])  # through A2 and through the skip
    g["A1"] = dq1.T @ c["xa"]
    g["a1"] = dq1.sum(0)
    dxa = dq1 @ p["A1"]
    n_h = p[W2].shape[0]
    dg2 = dxa[:, :n_h] * dlrelu(c["g2"])
    g[W2] = dg2.T @ c["h1"]
    g[b2] = dg2.sum(0)
    dg1 = (dg2 @ p[W2]) * dlrelu(c["g1"])
    g[W1] = dg1.T @ c["x0"]
    g[b1] = dg1.sum(0)
    dx0 = dg1 @ p[W1]
    dang = dxa[:, n_h:] if "S1" in p else dx0[:, -N_ANG:]
    return g, dx0[:, :LATENT], dang


def shade(p: dict, z_mat: np.ndarray, materials, gbuf: dict, ablation: int = FULL):
    """Per-point shading with the paper's decoder (or one of its
    ablations): (components [n, 4], rgb [n, 3]); z_mat [n_mat, 64] per
    material."""
    mat = np.asarray(gbuf["material"], np.int64)
    y = decoder_forward(p, np.asarray(z_mat, np.float64)[mat],
                        spatial_features(gbuf["u"], gbuf["v"], gbuf["radius"], ablation),
                        angular_features(gbuf["wi"], gbuf["wo"]))
    comps = mlp.head_to_components(y)
    return comps, mlp.recombine(comps, materials, mat)


def shade_rounded(p: dict, z_mat: np.ndarray, materials, gbuf: dict, r):
    """Operand-rounding emulation of the tensor-core path: `r` rounds to the
    16-bit operand type.  The one-blob channels, the angular inputs, every
    weight, every activation after its leaky ReLU and every bias of layers
    2-7 (they ride in a constant-one input column) are rounded; the latent
    enters folded into a rounded per-material bias column
    S1[:, :64] z_m + s1; the skip adds the rounded operand of k1; products
    accumulate in FP32 (FP64 here).  With r = identity this is shade()."""
    mat = np.asarray(gbuf["material"], np.int64)
    blob = r(spatial_features(gbuf["u"], gbuf["v"], gbuf["radius"]))
    ang = r(angular_features(gbuf["wi"], gbuf["wo"]))
    fold = p["s1"][None, :] + np.asarray(z_mat, np.float64) @ p["S1"][:, :LATENT].T
    h1 = r(lrelu(blob @ r(p["S1"][:, LATENT:]).T + r(fold)[mat]))
    hs = r(lrelu(h1 @ r(p["S2"]).T + r(p["s2"])))
    xa = np.concatenate([hs, ang], axis=1)
    k1 = r(lrelu(xa @ r(p["A1"]).T + r(p["a1"])))
    k2 = r(lrelu(k1 @ r(p["A2"]).T + r(p["a2"])))
    k3 = r(lrelu(k2 @ r(p["A3"]).T + r(p["a3"]) + k1))
    k4 = r(lrelu(k3 @ r(p["A4"]).T + r(p["a4"])))
    y = k4 @ r(p["A5"]).T + r(p["a5"])
    comps = mlp.head_to_components(y)
    return comps, mlp.recombine(comps, materials, mat)


def flops_per_point(w: int, folded: bool = True) -> int:
    """Multiply-adds x 2 of one decoder evaluation; with the latent folded
    into a bias, the first layer's K is the 24 one-blob channels."""
    k0 = N_BLOB if folded else LATENT + N_BLOB
    return 2 * (k0 * w + w * w + (w + N_ANG) * w + 3 * w * w + w * mlp.N_OUT)
