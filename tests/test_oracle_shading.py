"""Pins of the FP64 shading oracle against what the paper and the mathematics
fix, independently of the oracle's own code paths (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def mat_row(oracle_mod, **kw):
    base = dict(pattern=0, twist_deg=0.0, incl_deg=30.0, alpha=[0.3, 0.3], beta=[1.0, 1.0],
                kd=[[0.5] * 3, [0.5] * 3], ks=[[0.5] * 3, [0.5] * 3], gap=0.2, w_blend=0.5)
    base.update(kw)
    return oracle_mod.material_rows(W.make_material(**base))[0]


def fixed(frac):
    return int(round(frac * 2.0 ** 32)) & 0xFFFFFFFF


def cell_pos(R, C, i, j, au, av):
    """Fixed-point position of local coordinates (au, av) in cell (i, j)."""
    return fixed((j + au) / C), fixed((i + av) / R)


def unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def rand_dir(rng, upper=True):
    while True:
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        if not upper or d[2] > 0.05:
            return d if not upper else d * np.array([1, 1, 1])


# ---------------------------------------------------------------- hashing
def test_mix64_matches_published_splitmix64(oracle_mod):
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    gamma = int(g["golden_gamma"], 16)
    for seq in g["sequences"]:
        state = seq["seed"]
        want = seq.get("outputs") or [int(h, 16) for h in seq["outputs_hex"]]
        for w in want:
            state = (state + gamma) & 0xFFFFFFFFFFFFFFFF
            assert oracle_mod.mix64(state) == w


# ---------------------------------------------------------------- patterns
def test_weave_definitions(oracle_mod):
    P = {pid: oracle_mod.pattern_info(pid)[0].astype(int) for pid in range(12)}
    # plain: alternates along both axes
    assert P[0].shape == (2, 2)
    assert np.all(P[0] != np.roll(P[0], 1, 0)) and np.all(P[0] != np.roll(P[0], 1, 1))
    # twills: each row is the row above shifted by one column (diagonal)
    for pid, (n, over) in {1: (3, 2), 2: (4, 3), 8: (5, 4), 9: (8, 7)}.items():
        assert P[pid].shape == (n, n)
        assert np.all(P[pid].sum(1) == over) and np.all(P[pid].sum(0) == over)
        assert np.array_equal(np.roll(np.roll(P[pid], 1, 0), 1, 1), P[pid])
    # satins: one interlacing per row and column, never in adjacent columns of
    # consecutive rows (no twill line)
    for pid, faced, n in ((3, 0, 5), (4, 1, 5), (10, 1, 8)):
        A = P[pid] if faced == 1 else 1 - P[pid]
        assert A.shape == (n, n)
        assert np.all(A.sum(0) == 1) and np.all(A.sum(1) == 1)
        cols = A.argmax(1)
        steps = (np.roll(cols, -1) - cols) % n
        assert np.all((steps != 1) & (steps != n - 1))
    # satin with doubled picks (10 x 5): every pick repeated, and the
    # undoubled rows form the weft-faced 5-harness satin above
    D = P[11]
    assert D.shape == (10, 5)
    assert np.array_equal(D[0::2], D[1::2]) and np.array_equal(D[0::2], P[4])
    # basket 2x2: constant 2x2 blocks forming a checkerboard
    B = P[5]
    assert np.array_equal(B, np.kron(np.array([[1, 0], [0, 1]]), np.ones((2, 2), int)))
    # herringbone: 2/2 twill whose diagonal reverses at column 4
    H = P[6]
    assert H.shape == (4, 8)
    assert np.array_equal(np.roll(np.roll(H[:, :4], 1, 0), 1, 1), H[:, :4])
    assert np.array_equal(np.roll(np.roll(H[:, 4:], 1, 0), -1, 1), H[:, 4:])
    assert np.all(H.sum(0) == 2)
    # warp rib: warp floats of two rows, alternating columns
    Rb = P[7]
    assert Rb.shape == (4, 2)
    assert np.array_equal(Rb[:, 0], [1, 1, 0, 0]) and np.array_equal(Rb[:, 1], 1 - Rb[:, 0])


def test_float_run_tables_bruteforce(oracle_mod):
    for pid in range(12):
        bits, runlen, runoff = oracle_mod.pattern_info(pid)
        R, C = bits.shape
        for i in range(R):
            for j in range(C):
                warp = bits[i, j] == 1
                line = bits[:, j] == 1 if warp else bits[i, :] == 0
                pos = i if warp else j
                n = len(line)
                if line.all():
                    L, o = n, pos
                else:
                    back = 0
                    while line[(pos - back - 1) % n]:
                        back += 1
                    fwd = 0
                    while line[(pos + fwd + 1) % n]:
                        fwd += 1
                    L, o = back + fwd + 1, back
                assert (runlen[i, j], runoff[i, j]) == (L, o), (pid, i, j)


# ---------------------------------------------------------------- sampler
def test_samples_one_per_stratum(oracle_mod):
    nx, ny = 8, 4
    u, v, r = np.float32(7.3125), np.float32(2.5), np.float32(0.01)
    cu = fixed(float(u) % 1.0)
    cv = fixed(float(v) % 1.0)
    seen = set()
    for k in range(nx * ny):
        pu, pv = oracle_mod.sample_position(u, v, r, 17, k, nx, ny, 99)
        du = ((pu - cu + 2 ** 31) % 2 ** 32 - 2 ** 31) / 2.0 ** 32
        dv = ((pv - cv + 2 ** 31) % 2 ** 32 - 2 ** 31) / 2.0 ** 32
        assert abs(du) <= float(r) and abs(dv) <= float(r)
        sx = int((du / float(r) + 1.0) / 2.0 * nx)
        sy = int((dv / float(r) + 1.0) / 2.0 * ny)
        assert (sx, sy) == (k % nx, k // nx)
        seen.add((sx, sy))
    assert len(seen) == nx * ny
    # the jitter differs between points and between seeds
    assert oracle_mod.sample_position(u, v, r, 18, 0, nx, ny, 99) != oracle_mod.sample_position(u, v, r, 17, 0, nx, ny, 99)
    assert oracle_mod.sample_position(u, v, r, 17, 0, nx, ny, 98) != oracle_mod.sample_position(u, v, r, 17, 0, nx, ny, 99)


# ---------------------------------------------------------------- invariants
def _rand_gbuf(rng, n, n_mat, uv_max=50.0):
    return dict(u=rng.uniform(0, uv_max, n).astype(np.float32),
                v=rng.uniform(0, uv_max, n).astype(np.float32),
                radius=np.exp(rng.uniform(math.log(1e-4), math.log(2.0), n)).astype(np.float32),
                wi=W.hemisphere_uniform(rng, n), wo=W.hemisphere_uniform(rng, n),
                material=rng.integers(0, n_mat, n).astype(np.uint16))


def test_nonnegative_and_finite(oracle_mod):
    rng = np.random.default_rng(1)
    mats = np.concatenate([W.random_materials(rng, range(8)), W.table2_materials(rng, range(8))])
    g = _rand_gbuf(rng, 600, len(mats))
    comps, rgb = oracle_mod.shade_reference(mats, g, 4, 4, 7)
    assert np.all(np.isfinite(comps)) and np.all(comps >= 0.0)
    assert np.all(rgb >= 0.0)
    # a weft-only or warp-only visible footprint leaves the other yarn at zero
    # somewhere, so some components must vanish while others do not
    assert (comps > 0).mean() > 0.5


def test_weave_periodicity_bitwise(oracle_mod):
    rng = np.random.default_rng(2)
    mats = W.random_materials(rng, range(12))
    n = 300
    g = _rand_gbuf(rng, n, 12, uv_max=20.0)
    # uv with at most 16 fractional bits so that +1 / +2 periods are exact
    g["u"] = (np.round(g["u"] * 65536) / 65536).astype(np.float32)
    g["v"] = (np.round(g["v"] * 65536) / 65536).astype(np.float32)
    g2 = dict(g)
    g2["u"] = (g["u"] + np.float32(1.0)).astype(np.float32)
    g2["v"] = (g["v"] + np.float32(2.0)).astype(np.float32)
    c1, _ = oracle_mod.shade_reference(mats, g, 4, 4, 3)
    c2, _ = oracle_mod.shade_reference(mats, g2, 4, 4, 3)
    assert np.array_equal(c1, c2)


# ------------------------------------------------------- closed forms (points)
def _flat_expected(wi, wo, w):
    """alpha = 1, beta = 0, u = 0: n_p = z, D = 1/pi, sigma = 1 (Eq. 1-2)."""
    ci, co = wi[2], wo[2]
    lam = 1.0 / ci + 1.0 / co
    G = (1.0 - math.exp(-2.0 * lam)) / lam
    C = (w * ci / (math.pi * max(ci, 1e-3)) + (1.0 - w) / math.pi) * ci
    S = (1.0 / math.pi) * G / (4.0 * ci * co) * ci
    return C, S


@pytest.mark.parametrize("pid", range(12))
def test_point_closed_form_flat_isotropic(oracle_mod, pid):
    rng = np.random.default_rng(10 + pid)
    m = mat_row(oracle_mod, pattern=pid, alpha=[1.0, 1.0], beta=[0.0, 0.0], incl_deg=0.0,
                twist_deg=17.0, w_blend=0.3)
    bits = oracle_mod.pattern_info(pid)[0]
    R, C = bits.shape
    for _ in range(20):
        i, j = rng.integers(R), rng.integers(C)
        au, av = rng.uniform(0.01, 0.99, 2)
        pu, pv = cell_pos(R, C, i, j, au, av)
        wi, wo = W.hemisphere_uniform(rng, 2).astype(np.float64)
        got = oracle_mod.point_eval(m, pu, pv, wi, wo)
        # which yarn shows: the top one on its body, the other one in its gap
        s_top = au if bits[i, j] else av
        on_body = 0.1 <= s_top <= 0.9
        yarn = (0 if bits[i, j] else 1) if on_body else (1 if bits[i, j] else 0)
        if abs(s_top - 0.1) < 1e-6 or abs(s_top - 0.9) < 1e-6:
            continue
        Cx, Sx = _flat_expected(wi, wo, 0.3)
        want = np.zeros(4)
        want[yarn] = Cx
        want[2 + yarn] = Sx
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def _sggx_matrix(alpha, t):
    """S' = R^T diag(1, 1, alpha^2) R with the third row of R along t."""
    t = unit(t)
    a = unit(np.cross(t, [0.3, 0.5, 0.8]))
    b = np.cross(t, a)
    Rm = np.stack([a, b, t])
    return Rm.T @ np.diag([1.0, 1.0, alpha * alpha]) @ Rm


def _spec_point_expected(alpha, t, n, wi, wo):
    """f_s <wi . n_p> of Eq. 1-2 with a full-matrix SGGX (inverse and
    determinant by numpy), cosines w.r.t. n_p."""
    S = _sggx_matrix(alpha, t)
    ci, co = wi @ n, wo @ n
    if ci <= 0 or co <= 0:
        return 0.0
    h = unit(wi + wo)
    q = h @ np.linalg.inv(S) @ h
    D = 1.0 / (math.pi * math.sqrt(np.linalg.det(S)) * q * q)
    lam = math.sqrt(wi @ S @ wi) / ci + math.sqrt(wo @ S @ wo) / co
    G = (1.0 - math.exp(-2.0 * lam)) / lam
    return D * G / (4.0 * ci * co) * ci


def test_point_fibre_sggx_matches_matrix_form(oracle_mod):
    rng = np.random.default_rng(4)
    for trial in range(30):
        alpha = rng.uniform(0.1, 1.0)
        psi = rng.uniform(-30, 30)
        m = mat_row(oracle_mod, pattern=0, alpha=[alpha, alpha], beta=[0.0, 0.0], incl_deg=0.0,
                    twist_deg=psi)
        alpha, psi = m[3], m[1]        # the float32 values the record holds
        # warp body cell (0, 0) of the plain weave: axis +y, n_p = z
        pu, pv = cell_pos(2, 2, 0, 0, 0.5, rng.uniform(0.05, 0.95))
        wi, wo = (unit(d) for d in W.hemisphere_uniform(rng, 2))
        got = oracle_mod.point_eval(m, pu, pv, wi, wo)
        ps = math.radians(psi)
        t = np.array([-math.sin(ps), math.cos(ps), 0.0])     # axis +y turned by psi about z
        want = _spec_point_expected(alpha, t, np.array([0, 0, 1.0]), wi, wo)
        np.testing.assert_allclose(got[2], want, rtol=1e-10)
        assert got[3] == 0.0


def test_point_tilted_normal_from_height_profile(oracle_mod):
    """beta != 0: the ply normal follows the cross-section height profile
    beta cos(pi x / 2) (slope by central finite differences here), which
    fixes the blended-Lambertian term and, with t_p, the specular term."""
    rng = np.random.default_rng(5)
    g = float(np.float32(0.2))
    for trial in range(30):
        beta = rng.uniform(0.2, 2.0)
        alpha = rng.uniform(0.15, 0.9)
        w = rng.uniform(0.0, 1.0)
        psi = rng.uniform(-30, 30)
        m = mat_row(oracle_mod, pattern=0, alpha=[alpha, 0.5], beta=[beta, 0.0], incl_deg=0.0,
                    twist_deg=psi, w_blend=w)
        alpha, psi, beta, w = m[3], m[1], m[5], m[20]
        s = rng.uniform(0.15, 0.85)
        pu, pv = cell_pos(2, 2, 0, 0, s, rng.uniform(0.05, 0.95))
        s_exact = ((pu * 2) % 2 ** 32) / 2.0 ** 32
        x = (2 * s_exact - 1) / (1 - g)
        hgt = lambda xx: beta * math.cos(math.pi * xx / 2)
        eps = 1e-6
        slope = (hgt(x + eps) - hgt(x - eps)) / (2 * eps)
        n = unit([-slope, 0.0, 1.0])             # across direction of the warp is +x
        t0 = np.array([0.0, 1.0, 0.0])
        ps = math.radians(psi)
        t = math.cos(ps) * t0 + math.sin(ps) * np.cross(n, t0)
        wi, wo = (unit(d) for d in W.hemisphere_uniform(rng, 2))
        got = oracle_mod.point_eval(m, pu, pv, wi, wo)
        ci = max(0.0, wi @ n)
        C = (w * ci / (math.pi * max(wi[2], 1e-3)) + (1 - w) / math.pi) * ci
        if (wo @ n) <= 0:
            C = 0.0
        np.testing.assert_allclose(got[0], C, rtol=1e-7, atol=1e-12)
        np.testing.assert_allclose(got[2], _spec_point_expected(alpha, t, n, wi, wo), rtol=1e-6,
                                   atol=1e-12)


def test_frame_inclination_along_float(oracle_mod):
    """4/1 warp-faced satin: warp floats of four cells.  At the float start
    the yarn axis rises by the inclination angle, at its middle it is level,
    at its end it falls (theta = u (1 - 2y))."""
    bits, runlen, runoff = oracle_mod.pattern_info(3)
    incl = 37.0
    m = mat_row(oracle_mod, pattern=3, incl_deg=incl, twist_deg=0.0, beta=[0.0, 0.0])
    j = 0
    col = bits[:, j]
    start = [i for i in range(5) if col[i] == 1 and col[(i - 1) % 5] == 0][0]
    for frac_y, want_deg in [(1e-9, incl), (0.5 + 1e-9, 0.0), (0.25 + 1e-9, incl / 2)]:
        pos = frac_y * 4            # cells along the float
        o = int(pos)
        i = (start + o) % 5
        pu, pv = cell_pos(5, 5, i, j, 0.5, pos - o)
        yarn, n, t = oracle_mod.frame(m, pu, pv)
        assert yarn == 0
        ang = math.degrees(math.atan2(t[2], t[1]))
        assert abs(ang - want_deg) < 1e-5
        assert abs(n @ t) < 1e-12 and abs(np.linalg.norm(t) - 1) < 1e-12


def test_frame_orthonormal_and_twist_angle(oracle_mod):
    """t_p is a unit vector in the tangent plane of n_p, at the twist angle
    psi from the untwisted yarn axis t0, where t0 is the unique unit vector
    of span(a, z) orthogonal to n_p (a = the visible yarn's axis)."""
    rng = np.random.default_rng(6)
    mats = W.table2_materials(rng, range(8))
    rows = oracle_mod.material_rows(mats)
    for k in range(400):
        m = rows[k % 8]
        pu, pv = int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 2 ** 32))
        yarn, n, t = oracle_mod.frame(m, pu, pv)
        assert abs(np.linalg.norm(n) - 1) < 1e-12 and abs(np.linalg.norm(t) - 1) < 1e-12
        assert abs(n @ t) < 1e-12 and n[2] > 0
        a = np.array([0, 1.0, 0]) if yarn == 0 else np.array([1.0, 0, 0])
        t0 = unit(a - (a @ n) / n[2] * np.array([0, 0, 1.0]))
        assert abs(t0 @ n) < 1e-12
        np.testing.assert_allclose(t @ t0, math.cos(math.radians(m[1])), atol=1e-12)
        # the twist turns t0 towards n_p x t0 for positive psi
        np.testing.assert_allclose(t @ np.cross(n, t0), math.sin(math.radians(m[1])), atol=1e-12)


def test_specular_numerator_reciprocal(oracle_mod):
    """D G / (4 cos cos) is symmetric in (wi, wo) (Eq. 1-2), so the specular
    numerator f_s <wi.n_p> A = D G J / 4 of Eq. 3-4 is too, point by point;
    the diffuse and area terms are not."""
    rng = np.random.default_rng(7)
    rows = oracle_mod.material_rows(W.table2_materials(rng, range(8)))
    for k in range(300):
        m = rows[k % 8]
        pu, pv = int(rng.integers(0, 2 ** 32)), int(rng.integers(0, 2 ** 32))
        wi, wo = W.hemisphere_uniform(rng, 2).astype(np.float64)
        a = oracle_mod.point_contrib(m, pu, pv, wi, wo)
        b = oracle_mod.point_contrib(m, pu, pv, wo, wi)
        np.testing.assert_allclose(a[2:4], b[2:4], rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("alpha", [0.3, 0.6, 1.0])
def test_sggx_area_and_projected_area(oracle_mod, alpha):
    """SGGX identities (Heitz et al. 2015).  D is the normal distribution of
    the ellipsoid with projected area sigma(w) = sqrt(w^T S w), scaled by 1/pi:
    for S = diag(1, 1, alpha^2) that is the prolate spheroid with semi-axes
    (sqrt(alpha), sqrt(alpha), 1/sqrt(alpha)).  So (i) the clamped-cosine
    projection of D along w equals sigma(w), and (ii) the integral of D over
    the sphere equals the spheroid's surface area divided by pi."""
    t = unit([0.3, -0.5, 0.81])
    nt, npf = 500, 1000
    th = (np.arange(nt) + 0.5) / nt * math.pi
    ph = (np.arange(npf) + 0.5) / npf * 2 * math.pi
    T, Pp = np.meshgrid(th, ph, indexing="ij")
    M = np.stack([np.sin(T) * np.cos(Pp), np.sin(T) * np.sin(Pp), np.cos(T)], -1).reshape(-1, 3)
    dA = (np.sin(T) * (math.pi / nt) * (2 * math.pi / npf)).reshape(-1)
    rng = np.random.default_rng(8)
    idx = rng.choice(len(M), 3000, replace=False)
    D_sub = np.array([oracle_mod.sggx_D(alpha, t, M[k]) for k in idx])
    # the oracle's D on a random subset, the rest by interpolation-free reuse:
    # D depends on m only through tau = m.t, so fit the exact tau -> D map
    tau_sub = M[idx] @ t
    q_sub = D_sub * math.pi * alpha
    # q = 1/sqrt(pi alpha D) must be affine in tau^2 (q = 1 + c tau^2)
    qq = 1.0 / np.sqrt(q_sub)
    c = np.polyfit(tau_sub ** 2, qq, 1)
    assert abs(c[1] - 1.0) < 1e-9
    tau = M @ t
    D = 1.0 / (math.pi * alpha * (c[1] + c[0] * tau ** 2) ** 2)
    for w in [unit([0, 0, 1]), unit([0.7, 0.1, 0.2]), t]:
        proj = (D * np.maximum(M @ w, 0.0) * dA).sum()
        assert abs(proj - oracle_mod.sggx_sigma(alpha, t, w)) < 2e-3
    a2, c2 = alpha, 1.0 / alpha                   # squared semi-axes
    if alpha < 1.0:
        e = math.sqrt(1.0 - a2 / c2)
        area = 2 * math.pi * a2 * (1 + math.sqrt(c2) / (math.sqrt(a2) * e) * math.asin(e))
    else:
        area = 4 * math.pi
    assert abs((D * dA).sum() - area / math.pi) < 2e-3 * area


# ------------------------------------------------------- footprint limits
def test_small_footprint_equals_point_evaluation(oracle_mod):
    rng = np.random.default_rng(9)
    mats = W.table2_materials(rng, range(8))
    rows = oracle_mod.material_rows(mats)
    for k in range(40):
        pid = k % 8
        bits = oracle_mod.pattern_info(pid)[0]
        R, C = bits.shape
        i, j = rng.integers(R), rng.integers(C)
        au, av = rng.uniform(0.2, 0.8, 2)
        # stay clear of the gap edges (0.1 / 0.9) and cell borders
        uf = np.float32(3.0 + (j + au) / C)
        vf = np.float32(5.0 + (i + av) / R)
        wi, wo = W.hemisphere_uniform(rng, 2)
        g = dict(u=np.array([uf]), v=np.array([vf]), radius=np.array([2.0 ** -30], np.float32),
                 wi=wi[None], wo=wo[None], material=np.array([pid], np.uint16))
        comps, _ = oracle_mod.shade_reference(mats, g, 4, 4, 11)
        pu = int(np.uint32(np.int64(np.round(np.float64(uf - np.floor(uf)) * 2 ** 32)) & 0xFFFFFFFF))
        pv = int(np.uint32(np.int64(np.round(np.float64(vf - np.floor(vf)) * 2 ** 32)) & 0xFFFFFFFF))
        want = oracle_mod.point_eval(rows[pid], pu, pv, wi.astype(np.float64), wo.astype(np.float64))
        np.testing.assert_allclose(comps[0], want, rtol=1e-6, atol=1e-12)


def _one_period_query(mats, pid, u, v, wi, wo):
    return dict(u=np.array([u], np.float32), v=np.array([v], np.float32),
                radius=np.array([0.5], np.float32), wi=wi[None].astype(np.float32),
                wo=wo[None].astype(np.float32), material=np.array([pid], np.uint16))


def test_whole_period_footprint_equals_period_average(oracle_mod):
    """A footprint of exactly one period (side 2r = 1) averages every weave
    point once, whatever its centre: the estimate converges to the period
    quadrature of Eq. 3-5."""
    rng = np.random.default_rng(12)
    mats = W.table2_materials(rng, range(8))
    rows = oracle_mod.material_rows(mats)
    for pid in [0, 2, 3, 6]:
        wi, wo = W.hemisphere_uniform(rng, 2)
        wi[2] = max(wi[2], 0.3)
        wo[2] = max(wo[2], 0.3)
        wi, wo = wi / np.linalg.norm(wi), wo / np.linalg.norm(wo)
        q = oracle_mod.period_quadrature(rows[pid], wi.astype(np.float64), wo.astype(np.float64), 1024)
        want = q[:4] / q[4]
        for (u, v) in [(0.5, 0.5), (13.3, 7.71)]:
            comps, _ = oracle_mod.shade_reference(mats, _one_period_query(mats, pid, u, v, wi, wo),
                                                  64, 64, 5)
            err = np.abs(comps[0] - want).max() / max(np.abs(want).max(), 1e-12)
            assert err < 2e-2, (pid, u, v, comps[0], want)


def test_estimator_converges_with_sample_count(oracle_mod):
    rng = np.random.default_rng(13)
    mats = W.table2_materials(rng, range(8))
    rows = oracle_mod.material_rows(mats)
    pid = 1
    wi = np.array([0.3, -0.2, 0.93]); wi /= np.linalg.norm(wi)
    wo = np.array([-0.4, 0.1, 0.91]); wo /= np.linalg.norm(wo)
    q = oracle_mod.period_quadrature(rows[pid], wi, wo, 2048)
    want = q[:4] / q[4]
    errs = []
    for n in [2, 4, 8, 16, 32, 64]:
        e = []
        for seed in range(8):
            c, _ = oracle_mod.shade_reference(mats, _one_period_query(mats, pid, 0.37, 0.61, wi, wo), n, n, seed)
            e.append(np.abs(c[0] - want).sum())
        errs.append(np.sqrt(np.mean(np.square(e))))
    slope = np.polyfit(np.log([n * n for n in [2, 4, 8, 16, 32, 64]]), np.log(errs), 1)[0]
    assert slope < -0.5, (errs, slope)
    assert errs[-1] < errs[0] / 20


def test_whole_period_flat_isotropic_coverage_closed_form(oracle_mod):
    """alpha = 1, beta = 0, u = 0: every point shades as the flat closed form,
    so the whole-period value is that form weighted by each yarn's visible
    area fraction, counted exactly from the weave and the fixed-point gap."""
    rng = np.random.default_rng(14)
    for pid in range(12):
        m = mat_row(oracle_mod, pattern=pid, alpha=[1.0, 1.0], beta=[0.0, 0.0], incl_deg=0.0)
        bits = oracle_mod.pattern_info(pid)[0]
        Gf = math.floor(0.5 * float(np.float32(0.2)) * 2 ** 32)
        gap_frac = (2 * Gf) / 2 ** 32
        nw = bits.sum()
        cov_warp = (nw * (1 - gap_frac) + (bits.size - nw) * gap_frac) / bits.size
        wi, wo = W.hemisphere_uniform(rng, 2).astype(np.float64)
        Cx, Sx = _flat_expected(wi, wo, 0.5)
        # 1200 = 10 x lcm(2,3,4,5,8,10): no lattice point lies on a cell or gap edge
        q = oracle_mod.period_quadrature(m, wi, wo, 1200)
        got = q[:4] / q[4]
        want = np.array([cov_warp * Cx, (1 - cov_warp) * Cx, cov_warp * Sx, (1 - cov_warp) * Sx])
        np.testing.assert_allclose(got, want, rtol=1e-7)


# ------------------------------------------------------- data-generation counts
def test_paper_direction_pair_counts():
    g = json.load(open(os.path.join(GOLDEN, "paper_counts.json")))
    rng = np.random.default_rng(15)
    counts = []
    for _ in range(20):
        _, ins_i = W.paper_direction_grid(rng, g["direction_grid"]["value"])
        _, ins_o = W.paper_direction_grid(rng, g["direction_grid"]["value"])
        counts.append(int(ins_i.sum()) * int(ins_o.sum()))
    mean_pairs = float(np.mean(counts))
    assert abs(mean_pairs - g["valid_pairs_about"]["value"]) / g["valid_pairs_about"]["value"] < 0.05
    per_mat = g["footprint_centres"]["value"] * g["footprint_sizes"]["value"] * mean_pairs
    assert abs(per_mat - g["queries_per_material_about"]["value"]) / g["queries_per_material_about"]["value"] < 0.05
    m = g["materials"]
    assert m["plain"] == 9 * 9 and m["twill"] == 3 * 4 * 16 and m["satin"] == 3 * 4 * 16


# ------------------------------------------------------- Eq. 8 recombination
def test_eq8_rgb_from_hand_set_albedos(oracle_mod):
    """Eq. 8 in the estimator's RGB output, on values worked out by hand.

    Flat isotropic yarns (alpha = 1, beta = 0, inclination 0) at a single
    point (r = 2^-30 periods), wi = (0.8, 0, 0.6), wo = (0, 0, 1), w = 0.5:
    Eq. 1-2 give C = 0.6 / pi for the visible yarn and
    S = 0.6 (1 - exp(-16/3)) / (6.4 pi) (D = 1/pi, sigma = 1,
    G = ci co (1 - exp(-2 (ci + co) / (ci co))) / (ci + co), divided by
    4 co); the hidden yarn's components are 0.  Every albedo differs, so a
    warp / weft or diffuse / specular swap in the recombination changes the
    expected colour.  Plain weave: cell (0, 0) shows the warp at its centre
    (u, v) = (0.25, 0.25), cell (0, 1) shows the weft at (0.75, 0.25)."""
    C = 0.6 / math.pi
    S = 0.6 * (1.0 - math.exp(-16.0 / 3.0)) / (6.4 * math.pi)
    mat = W.make_material(pattern=0, twist_deg=0.0, incl_deg=0.0, alpha=[1.0, 1.0], beta=[0.0, 0.0],
                          kd=[[0.2, 0.4, 0.6], [0.9, 0.1, 0.3]],
                          ks=[[1.0, 0.0, 0.5], [0.05, 0.7, 0.25]], gap=0.2, w_blend=0.5)
    g = dict(u=np.array([16.25, 16.75], np.float32), v=np.array([3.25, 3.25], np.float32),
             radius=np.full(2, 2.0 ** -30, np.float32),
             wi=np.array([[0.8, 0.0, 0.6]] * 2, np.float32), wo=np.array([[0.0, 0.0, 1.0]] * 2, np.float32),
             material=np.zeros(2, np.uint16))
    comps, rgb = oracle_mod.shade_reference(np.atleast_1d(mat), g, 4, 4, 5)
    f32 = lambda x: float(np.float32(x))   # albedos are stored as float32
    np.testing.assert_allclose(comps[0], [C, 0.0, S, 0.0], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(comps[1], [0.0, C, 0.0, S], rtol=1e-6, atol=1e-12)
    # warp point: kd_warp C + ks_warp S
    want_warp = [f32(0.2) * C + f32(1.0) * S, f32(0.4) * C + 0.0 * S, f32(0.6) * C + f32(0.5) * S]
    # weft point: kd_weft C + ks_weft S
    want_weft = [f32(0.9) * C + f32(0.05) * S, f32(0.1) * C + f32(0.7) * S, f32(0.3) * C + f32(0.25) * S]
    np.testing.assert_allclose(rgb[0], want_warp, rtol=1e-6)
    np.testing.assert_allclose(rgb[1], want_weft, rtol=1e-6)


def test_eq8_rgb_is_linear_in_each_albedo(oracle_mod):
    """Eq. 8 is linear in each albedo with the matching component as its
    coefficient: with one albedo set to the unit colour and the other three
    to zero, the RGB output is that component in all three channels."""
    rng = np.random.default_rng(21)
    g = _rand_gbuf(rng, 64, 1, uv_max=10.0)
    names = [("kd", 0), ("kd", 1), ("ks", 0), ("ks", 1)]   # C_warp, C_weft, S_warp, S_weft
    for k, (field, yarn) in enumerate(names):
        kd = np.zeros((2, 3))
        ks = np.zeros((2, 3))
        (kd if field == "kd" else ks)[yarn] = 1.0
        mat = W.make_material(pattern=2, twist_deg=12.0, incl_deg=25.0, alpha=[0.3, 0.5], beta=[1.0, 0.6],
                              kd=kd, ks=ks)
        comps, rgb = oracle_mod.shade_reference(np.atleast_1d(mat), g, 4, 4, 9)
        assert (comps[:, k] > 0).any()
        for ch in range(3):
            np.testing.assert_array_equal(rgb[:, ch], comps[:, k])
