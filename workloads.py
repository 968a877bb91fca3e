"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module draws inputs only: material parameters, G-buffers of shading
points and training queries.  It holds none of the shading model's or the
network's arithmetic, so that both implementations can be fed identical inputs
without sharing code.  Everything is numpy with explicit seeds.

Workloads (synthetic stand-ins for the paper's scenes, which are not
available; all at the paper's 1920x1080 resolution, Sec. 6):

* ``plane_scene``: a flat textile plane seen by a pinhole camera and lit by a
  point light (64x64 px, plain weave, 8 repeats across the image).
* ``frame_gbuffer``: a 1920x1080 G-buffer: uv ~ U[0,50)^2, footprint radius
  log-uniform in [1e-4, 1e-1] uv units, wi and wo uniform in solid angle on the
  upper hemisphere, eight materials (one per weave) in eight vertical bands of
  240 px, as in the paper's eight-fabric sofa scene.
* ``multiscale_gbuffer``: the same frame with footprint sides drawn as in the
  paper's Table 2 (half U(0,1), half U(1,5) periods), the regime where a pixel
  covers up to several weave repeats; used only to measure image error.
* ``training_queries``: half frame-like queries, half drawn from the paper's
  Table 2 (footprint centre U(0,1)^2, side U(0,1) or U(1,5) periods, (x, y) of
  both directions U(-1,1)^2 inside the unit disc).
* ``batched_4k``: a 3840x2160 G-buffer with materials interleaved per 16x16
  tile, plus ragged tiles of 256..65536 points from four views.
* ``paper_materials`` / ``paper_queries``: the paper's data-generation set
  (Sec. 5.1, Table 2): 465 materials over its seven weaves, and per material
  an 8x8 grid of footprint centres x 20 footprint sizes x the valid pairs of
  8x8-stratified directions (about 3.2 million queries).
"""
from __future__ import annotations

import math

import numpy as np

# Host material record; the field order and float32 types match the C struct
# `fabric_material` (84 bytes, no padding).
MATERIAL_DTYPE = np.dtype([
    ("pattern", np.int32),
    ("twist_deg", np.float32),
    ("incl_deg", np.float32),
    ("alpha", np.float32, (2,)),       # [warp, weft]
    ("beta", np.float32, (2,)),
    ("kd", np.float32, (2, 3)),        # [yarn][rgb]
    ("ks", np.float32, (2, 3)),
    ("gap", np.float32),
    ("w_blend", np.float32),
])

N_PATTERNS = 8
PATTERN_NAMES = ["plain", "twill 2/1", "twill 3/1", "satin 4/1 (warp-faced)",
                 "satin 5-harness (weft-faced)", "basket 2x2", "herringbone", "warp rib"]

SEED_BASE = 0xFAB00000


def rng_for(config: int, stream: str) -> np.random.Generator:
    """Independent generator per (workload, purpose) pair."""
    tag = sum((i + 1) * b for i, b in enumerate(stream.encode()))
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE + config, tag])))


def make_material(pattern, twist_deg, incl_deg, alpha, beta, kd, ks, gap=0.2, w_blend=0.5):
    m = np.zeros((), MATERIAL_DTYPE)
    m["pattern"] = pattern
    m["twist_deg"] = twist_deg
    m["incl_deg"] = incl_deg
    m["alpha"] = alpha
    m["beta"] = beta
    m["kd"] = kd
    m["ks"] = ks
    m["gap"] = gap
    m["w_blend"] = w_blend
    return m


def random_materials(rng: np.random.Generator, patterns) -> np.ndarray:
    """Frame materials: alpha ~ U[0.1,0.4] and kd, ks ~ U[0.2,0.8]^3 per yarn
    type, twist ~ U[0,30] deg per material; inclination 30 deg, beta 1,
    gap 0.2 (paper Sec. 5.1), blend weight 0.5."""
    patterns = list(patterns)
    out = np.zeros(len(patterns), MATERIAL_DTYPE)
    for k, p in enumerate(patterns):
        out[k] = make_material(
            pattern=p,
            twist_deg=rng.uniform(0.0, 30.0),
            incl_deg=30.0,
            alpha=rng.uniform(0.1, 0.4, 2),
            beta=[1.0, 1.0],
            kd=rng.uniform(0.2, 0.8, (2, 3)),
            ks=rng.uniform(0.2, 0.8, (2, 3)),
        )
    return out


def table2_materials(rng: np.random.Generator, patterns) -> np.ndarray:
    """Materials drawn from the paper's Table 2: twist in {-30, 0, 30} deg,
    inclination U(15,45) deg, alpha U(0.1,1), beta U(0,2) per yarn type;
    albedos U[0.2,0.8]^3 (albedos never enter the network)."""
    patterns = list(patterns)
    out = np.zeros(len(patterns), MATERIAL_DTYPE)
    for k, p in enumerate(patterns):
        out[k] = make_material(
            pattern=p,
            twist_deg=float(rng.choice([-30.0, 0.0, 30.0])),
            incl_deg=rng.uniform(15.0, 45.0),
            alpha=rng.uniform(0.1, 1.0, 2),
            beta=rng.uniform(0.0, 2.0, 2),
            kd=rng.uniform(0.2, 0.8, (2, 3)),
            ks=rng.uniform(0.2, 0.8, (2, 3)),
        )
    return out


def hemisphere_uniform(rng: np.random.Generator, n: int) -> np.ndarray:
    """Directions uniform in solid angle on the upper hemisphere (z ~ U(0,1),
    phi ~ U(0, 2 pi)), float32 [n, 3]."""
    z = rng.uniform(0.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1).astype(np.float32)


def disc_directions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Table 2 directions: (x, y) ~ U(-1,1)^2 restricted to the unit disc,
    z = sqrt(1 - x^2 - y^2)."""
    out = np.empty((0, 2))
    while len(out) < n:
        xy = rng.uniform(-1.0, 1.0, (2 * (n - len(out)) + 16, 2))
        xy = xy[(xy ** 2).sum(1) < 1.0]
        out = np.concatenate([out, xy])[:n]
    z = np.sqrt(np.maximum(0.0, 1.0 - (out ** 2).sum(1)))
    return np.concatenate([out, z[:, None]], axis=1).astype(np.float32)


def frame_materials(config: int = 2) -> np.ndarray:
    return random_materials(rng_for(config, "materials"), range(N_PATTERNS))


def frame_gbuffer(width: int = 1920, height: int = 1080, n_materials: int = N_PATTERNS,
                  config: int = 2, uv_max: float = 50.0) -> dict:
    """1080p G-buffer of shading points, row-major (index = y * width + x);
    material = vertical band of width // n_materials pixels."""
    rng = rng_for(config, "gbuffer")
    n = width * height
    u = rng.uniform(0.0, uv_max, n).astype(np.float32)
    v = rng.uniform(0.0, uv_max, n).astype(np.float32)
    radius = np.exp(rng.uniform(math.log(1e-4), math.log(1e-1), n)).astype(np.float32)
    wi = hemisphere_uniform(rng, n)
    wo = hemisphere_uniform(rng, n)
    x = np.tile(np.arange(width), height)
    band = max(1, width // n_materials)
    material = np.minimum(x // band, n_materials - 1).astype(np.uint16)
    return dict(u=u, v=v, radius=radius, wi=wi, wo=wo, material=material,
                width=width, height=height)


def multiscale_gbuffer(width: int = 1920, height: int = 1080, n_materials: int = N_PATTERNS,
                       config: int = 2) -> dict:
    """``frame_gbuffer`` with the footprint radius replaced: side s drawn as
    in Table 2 (U(0,1) or U(1,5) periods with equal odds), radius = s / 2."""
    g = frame_gbuffer(width, height, n_materials, config)
    rng = rng_for(config, "multiscale-footprint")
    n = width * height
    big = rng.random(n) < 0.5
    side = np.where(big, rng.uniform(1.0, 5.0, n), rng.uniform(0.0, 1.0, n))
    g["radius"] = np.maximum(side / 2.0, 1e-6).astype(np.float32)
    return g


def subset(gbuf: dict, idx: np.ndarray) -> dict:
    """Rows `idx` of a G-buffer (same field layout)."""
    return {k: (gbuf[k][idx] if isinstance(gbuf[k], np.ndarray) else gbuf[k]) for k in gbuf}


def sample_indices(n: int, k: int, config: int = 2, stream: str = "subset") -> np.ndarray:
    rng = rng_for(config, stream)
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def plane_scene(width: int = 64, height: int = 64, config: int = 1) -> tuple[dict, np.ndarray, dict]:
    """Flat textile plane z = 0 seen by a pinhole camera (distance 2, tilted
    45 deg, vertical field of view 40 deg) and lit by a point light.  uv is the
    plane position scaled so that about 8 pattern repeats span the image
    width; the footprint radius is half the geometric mean of the pixel's two
    footprint axes on the plane.  Returns (gbuffer, materials, scene info);
    wi points to the light, wo to the camera (both in the plane's frame)."""
    rng = rng_for(config, "materials")
    mat = random_materials(rng, [0])
    fov = math.radians(40.0)
    dist = 2.0
    tilt = math.radians(45.0)
    cam = np.array([0.0, -dist * math.sin(tilt), dist * math.cos(tilt)])
    fwd = -cam / np.linalg.norm(cam)
    right = np.array([1.0, 0.0, 0.0])
    up = np.cross(right, fwd)
    tan_half = math.tan(fov / 2.0)
    uv_scale = 8.0 / (2.0 * dist * tan_half)
    light = np.array([0.35, -0.25, 1.3])
    ys, xs = np.mgrid[0:height, 0:width]
    sx = ((xs + 0.5) / width * 2.0 - 1.0) * tan_half
    sy = (1.0 - (ys + 0.5) / height * 2.0) * tan_half
    d = fwd[None, None, :] + sx[..., None] * right + sy[..., None] * up
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    t = -cam[2] / d[..., 2]
    p = cam + t[..., None] * d
    wo = cam - p
    wo /= np.linalg.norm(wo, axis=-1, keepdims=True)
    wi = light - p
    light_d2 = (wi ** 2).sum(-1)
    wi /= np.sqrt(light_d2)[..., None]
    pix = 2.0 * tan_half / height
    radius = 0.5 * t * pix / np.sqrt(wo[..., 2]) * uv_scale
    n = width * height
    gbuf = dict(
        u=(p[..., 0] * uv_scale).reshape(n).astype(np.float32) + np.float32(16.0),
        v=(p[..., 1] * uv_scale).reshape(n).astype(np.float32) + np.float32(16.0),
        radius=radius.reshape(n).astype(np.float32),
        wi=wi.reshape(n, 3).astype(np.float32),
        wo=wo.reshape(n, 3).astype(np.float32),
        material=np.zeros(n, np.uint16),
        width=width, height=height)
    info = dict(light_inv_d2=(1.0 / light_d2).reshape(n), uv_scale=uv_scale)
    return gbuf, mat, info


def training_materials(n_sets: int = 32, config: int = 4) -> np.ndarray:
    """n_sets parameter sets x 8 weaves (material index = set * 8 + pattern).
    Set 0 is the 1080p frame's material list; the other sets alternate
    between the frame's distribution and the paper's Table 2."""
    out = [frame_materials()]
    rng = rng_for(config, "materials")
    for s in range(1, n_sets):
        if s % 2:
            out.append(random_materials(rng, range(N_PATTERNS)))
        else:
            out.append(table2_materials(rng, range(N_PATTERNS)))
    return np.concatenate(out)


def training_queries(n: int, n_materials: int, config: int = 4, stream: str = "queries") -> dict:
    """n training queries, material index uniform over n_materials; half
    frame-like, half Table-2-like (see module docstring)."""
    rng = rng_for(config, stream)
    half = n // 2
    material = rng.integers(0, n_materials, n).astype(np.uint16)
    u = np.empty(n, np.float32)
    v = np.empty(n, np.float32)
    r = np.empty(n, np.float32)
    wi = np.empty((n, 3), np.float32)
    wo = np.empty((n, 3), np.float32)
    u[:half] = rng.uniform(0.0, 50.0, half)
    v[:half] = rng.uniform(0.0, 50.0, half)
    r[:half] = np.exp(rng.uniform(math.log(1e-4), math.log(1e-1), half))
    wi[:half] = hemisphere_uniform(rng, half)
    wo[:half] = hemisphere_uniform(rng, half)
    m = n - half
    u[half:] = rng.uniform(0.0, 1.0, m)
    v[half:] = rng.uniform(0.0, 1.0, m)
    big = rng.random(m) < 0.5
    side = np.where(big, rng.uniform(1.0, 5.0, m), rng.uniform(0.0, 1.0, m))
    r[half:] = np.maximum(side / 2.0, 1e-6)
    wi[half:] = disc_directions(rng, m)
    wo[half:] = disc_directions(rng, m)
    return dict(u=u, v=v, radius=r, wi=wi, wo=wo, material=material)


def paper_direction_grid(rng: np.random.Generator, grid: int = 8):
    """The paper's data-generation direction pairs (Sec. 5.1): (x, y) of wi and
    wo stratified on a grid x grid lattice over (-1,1)^2 (one jittered sample
    per cell); pairs with both directions inside the unit disc are valid."""
    cells = (np.arange(grid) + 0.0) / grid * 2.0 - 1.0
    gx, gy = np.meshgrid(cells, cells, indexing="ij")
    jit = rng.uniform(0.0, 2.0 / grid, (grid * grid, 2))
    xy = np.stack([gx.ravel(), gy.ravel()], 1) + jit
    inside = (xy ** 2).sum(1) < 1.0
    return xy, inside


# The paper's seven training weaves (Sec. 5.1) as built-in weave ids: plain,
# twill 3x3 (2/1), twill 5x5 (4/1), twill 8x8 (7/1), satin 5x5 (5-harness,
# weft-faced), satin 8x8 (8-harness, weft-faced), satin 5x10 (5-harness with
# doubled picks).
PAPER_WEAVES = [0, 1, 8, 9, 4, 10, 11]
PAPER_TWILLS = [1, 8, 9]


def paper_materials(config: int = 6) -> np.ndarray:
    """The paper's 465 training materials (Sec. 5.1): per weave, sets of
    (twist, inclination) drawn from Table 2 (9 for plain, 4 for the others),
    each combined with sets of (alpha, beta) per yarn type drawn from Table 2
    (9 for plain, 16 for the others): 81 plain, 192 twill and 192 satin
    materials.  Albedos U[0.2, 0.8]^3 (they never enter the components)."""
    rng = rng_for(config, "paper-materials")
    out = []
    for w in PAPER_WEAVES:
        n_geo, n_app = (9, 9) if w == 0 else (4, 16)
        for _ in range(n_geo):
            psi = float(rng.choice([-30.0, 0.0, 30.0]))
            incl = rng.uniform(15.0, 45.0)
            for _ in range(n_app):
                out.append(make_material(pattern=w, twist_deg=psi, incl_deg=incl,
                                         alpha=rng.uniform(0.1, 1.0, 2), beta=rng.uniform(0.0, 2.0, 2),
                                         kd=rng.uniform(0.2, 0.8, (2, 3)), ks=rng.uniform(0.2, 0.8, (2, 3))))
    m = np.zeros(len(out), MATERIAL_DTYPE)
    for k, r in enumerate(out):
        m[k] = r
    return m


def paper_queries(material: int, config: int = 6, stream: str = "paper-queries", grid: int = 8,
                  sizes: int = 10) -> dict:
    """The paper's query set of one material (Sec. 5.1): footprint centres
    jittered in the cells of a grid x grid partition of one pattern repeat;
    per centre, `sizes` footprint sides in [0, 1] and `sizes` in [1, 5]
    repeats (one jittered sample per equal sub-interval; radius = side / 2);
    per footprint, the (x, y) of wi and of wo each stratified on a grid x grid
    lattice over (-1, 1)^2 (paper_direction_grid), and every pair of valid
    directions (both inside the unit disc, z = sqrt(1 - x^2 - y^2)) becomes a
    query.  Returns a G-buffer dict (material index `material`, footprints
    in centre-major, then size order)."""
    rng = rng_for(config, f"{stream}-{material}")
    cells = (np.arange(grid * grid) % grid, np.arange(grid * grid) // grid)
    cu = (cells[0] + rng.uniform(0.0, 1.0, grid * grid)) / grid
    cv = (cells[1] + rng.uniform(0.0, 1.0, grid * grid)) / grid
    us, vs, rs, wis, wos = [], [], [], [], []
    for c in range(grid * grid):
        side = np.concatenate([(np.arange(sizes) + rng.uniform(0.0, 1.0, sizes)) / sizes,
                               1.0 + 4.0 * (np.arange(sizes) + rng.uniform(0.0, 1.0, sizes)) / sizes])
        for s in side:
            xi, ok_i = paper_direction_grid(rng, grid)
            xo, ok_o = paper_direction_grid(rng, grid)
            xi, xo = xi[ok_i], xo[ok_o]
            wi = np.concatenate([xi, np.sqrt(np.maximum(0.0, 1.0 - (xi ** 2).sum(1)))[:, None]], 1)
            wo = np.concatenate([xo, np.sqrt(np.maximum(0.0, 1.0 - (xo ** 2).sum(1)))[:, None]], 1)
            k = len(wi) * len(wo)
            wis.append(np.repeat(wi, len(wo), 0))
            wos.append(np.tile(wo, (len(wi), 1)))
            us.append(np.full(k, cu[c]))
            vs.append(np.full(k, cv[c]))
            rs.append(np.full(k, s / 2.0))
    n = sum(len(a) for a in us)
    return dict(u=np.concatenate(us).astype(np.float32), v=np.concatenate(vs).astype(np.float32),
                radius=np.concatenate(rs).astype(np.float32), wi=np.concatenate(wis).astype(np.float32),
                wo=np.concatenate(wos).astype(np.float32), material=np.full(n, material, np.uint16))


def batched_4k(config: int = 5, width: int = 3840, height: int = 2160, tile: int = 16,
               n_views: int = 4, ragged_per_view: int = 64, n_materials: int = N_PATTERNS):
    """4K G-buffer whose 16x16-pixel tiles carry interleaved materials, plus
    ragged tiles (sizes floor(exp(U(ln 256, ln 65536)))) from four views.
    Returns (list of G-buffer segments, total points)."""
    rng = rng_for(config, "gbuffer")
    segs = []
    n = width * height
    g = dict(u=rng.uniform(0.0, 50.0, n).astype(np.float32),
             v=rng.uniform(0.0, 50.0, n).astype(np.float32),
             radius=np.exp(rng.uniform(math.log(1e-4), math.log(1e-1), n)).astype(np.float32),
             wi=hemisphere_uniform(rng, n), wo=hemisphere_uniform(rng, n))
    xs = np.tile(np.arange(width), height)
    ys = np.repeat(np.arange(height), width)
    tile_id = (ys // tile) * (width // tile) + xs // tile
    hashed = (tile_id.astype(np.uint64) * np.uint64(0x9E3779B1)) >> np.uint64(7)
    g["material"] = (hashed % np.uint64(n_materials)).astype(np.uint16)
    segs.append(g)
    for _view in range(n_views):
        for _t in range(ragged_per_view):
            k = int(math.floor(math.exp(rng.uniform(math.log(256), math.log(65536)))))
            segs.append(dict(u=rng.uniform(0.0, 50.0, k).astype(np.float32),
                             v=rng.uniform(0.0, 50.0, k).astype(np.float32),
                             radius=np.exp(rng.uniform(math.log(1e-4), math.log(1e-1), k)).astype(np.float32),
                             wi=hemisphere_uniform(rng, k), wo=hemisphere_uniform(rng, k),
                             material=rng.integers(0, n_materials, k).astype(np.uint16)))
    return segs, sum(len(s["u"]) for s in segs)


def init_params(n: int, fan_ins, sizes, seed: int, weight_bound: str = "he") -> np.ndarray:
    """Uniform initialisation: weights U(+-sqrt(6 / fan_in)) ("he") or
    U(+-1/sqrt(fan_in)) ("small", the default of common deep-learning
    libraries' linear layers), biases U(+-1/sqrt(fan_in)); `sizes` lists
    (n_weights, n_bias) per layer in the flat order, `fan_ins` the layer
    fan-ins."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE, seed])))
    out = []
    for (nw, nb), fi in zip(sizes, fan_ins):
        bound = math.sqrt(6.0 / fi) if weight_bound == "he" else 1.0 / math.sqrt(fi)
        out.append(rng.uniform(-bound, bound, nw))
        out.append(rng.uniform(-1.0 / math.sqrt(fi), 1.0 / math.sqrt(fi), nb))
    flat = np.concatenate(out).astype(np.float32)
    assert len(flat) == n
    return flat


DEC_LAYERS = [(64, 71), (64, 64), (64, 64), (4, 64)]       # (out, in)
ENC_LAYERS = [(128, 22), (128, 128), (32, 128)]


def decoder_init(seed: int = 3, weight_bound: str = "he") -> np.ndarray:
    """Random decoder parameters: "he" for the parity tests and the timed
    frame, "small" as the starting point of training."""
    return init_params(sum(o * i + o for o, i in DEC_LAYERS), [i for _, i in DEC_LAYERS],
                       [(o * i, o) for o, i in DEC_LAYERS], seed, weight_bound)


def encoder_init(seed: int = 4, weight_bound: str = "he") -> np.ndarray:
    return init_params(sum(o * i + o for o, i in ENC_LAYERS), [i for _, i in ENC_LAYERS],
                       [(o * i, o) for o, i in ENC_LAYERS], seed, weight_bound)


def random_latents(n_mat: int, seed: int = 5, scale: float = 1.0, dim: int = 32) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_BASE, seed])))
    return (scale * rng.standard_normal((n_mat, dim))).astype(np.float32)


def paper_decoder_layers(width: int, ablation: str = "full"):
    """(out, in) of the paper decoder's layers: S1, S2, A1..A5; without the
    one-blob encoding S1 takes 64 + 3 inputs; without the spatial fusion the
    first layer takes 64 + 24 + 5 and A1 the second's output alone."""
    if ablation == "no_fusion":
        return [(width, 64 + 24 + 5)] + [(width, width)] * 5 + [(4, width)]
    k0 = 64 + (3 if ablation == "no_oneblob" else 24)
    return [(width, k0), (width, width), (width, width + 5), (width, width), (width, width),
            (width, width), (4, width)]


PAPER_ENC_LAYERS = [(128, 22), (128, 128), (64, 128)]


def paper_decoder_init(width: int, seed: int = 13, weight_bound: str = "he", ablation: str = "full") -> np.ndarray:
    layers = paper_decoder_layers(width, ablation)
    return init_params(sum(o * i + o for o, i in layers), [i for _, i in layers], [(o * i, o) for o, i in layers],
                       seed, weight_bound)


def paper_encoder_init(seed: int = 14, weight_bound: str = "he") -> np.ndarray:
    return init_params(sum(o * i + o for o, i in PAPER_ENC_LAYERS), [i for _, i in PAPER_ENC_LAYERS],
                       [(o * i, o) for o, i in PAPER_ENC_LAYERS], seed, weight_bound)
