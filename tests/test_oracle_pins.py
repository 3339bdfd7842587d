"""Pins of the CPU oracle against values fixed by the paper and by mathematics.

Each test ties one oracle function to something other than the oracle itself:
a published constant, a closed form, an analytic ray/cylinder hit, a series
the closed form must equal, brute force on tiny inputs, or a hand-worked
example.  No GPU is needed.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen

PI = math.pi


def g(beta, x):
    return math.exp(-x * x / (2 * beta * beta)) / (math.sqrt(2 * PI) * beta)


C1_MAT = scenegen.material_absorption(1, 0.3, 0.2)[0].astype(np.float64)
BROWN = scenegen.material_from_melanin(np.array([0.5]), np.array([0.2]))[0].astype(np.float64)
DARK = scenegen.material_from_melanin(np.array([0.9]), np.array([0.1]))[0].astype(np.float64)
LIGHT = scenegen.material_from_melanin(np.array([0.1]), np.array([0.3]))[0].astype(np.float64)


# ---------------------------------------------------------------- random numbers


def test_splitmix64_published_outputs():
    # First three outputs of SplitMix64 seeded with 0 (Steele et al. 2014
    # reference implementation).
    out = [int(x) for x in scenegen.splitmix64(0, [0, 1, 2])]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_camera_jitter_uses_published_stream():
    # orthographic camera with an identity basis: the ray origin gives back the
    # sub-pixel position, which must be the 24-bit SplitMix64 draws.
    W, H, pix = 16, 8, 4.0
    cam = scenegen.Camera(0, W, H, np.zeros(3, np.float32), np.array([1, 0, 0], np.float32),
                          np.array([0, 1, 0], np.float32), np.array([0, 0, -1], np.float32),
                          pix).pack()
    seed, spp = 12345, 3
    for sid in [0, 1, 7, 100, W * H * spp - 1]:
        o, d = oracle.camera_ray(cam, seed, sid, spp)
        pixel = sid // spp
        x, y = pixel % W, pixel // W
        jx = float(int(scenegen.splitmix64(seed, 2 * sid) >> np.uint64(40))) / 2 ** 24
        jy = float(int(scenegen.splitmix64(seed, 2 * sid + 1) >> np.uint64(40))) / 2 ** 24
        assert o[0] == pytest.approx((x + jx - W / 2) / pix, abs=1e-12)
        assert o[1] == pytest.approx((H / 2 - y - jy) / pix, abs=1e-12)
        assert np.allclose(d, [0, 0, -1])


def test_perspective_edge_ray_half_fov():
    # A perspective camera framed with a 40 degree vertical field of view: a
    # ray through the top edge of the image makes 20 degrees with the axis.
    cam = scenegen.frame_camera(np.array([-1, -1, -1.0]), np.array([1, 1, 1.0]), 64, 32,
                                perspective=True, fill=0.5)
    rec = cam.pack().astype(np.float64)
    # find a sample whose jitter is close to (0.5, 0); use the analytic angle of
    # the exact sub-pixel position instead of searching
    sid = 0  # pixel (0, 0)
    o, d = oracle.camera_ray(rec, 9, sid, 1)
    jx = float(int(scenegen.splitmix64(9, 0) >> np.uint64(40))) / 2 ** 24
    jy = float(int(scenegen.splitmix64(9, 1) >> np.uint64(40))) / 2 ** 24
    fwd, up = rec[13:16], rec[10:13]
    # vertical tangent of the ray = (H/2 - jy) / pix, and pix = (H/2) / tan(20 deg)
    tan_v = np.dot(d, up) / np.dot(d, fwd)
    assert tan_v == pytest.approx((16 - jy) / 16 * math.tan(math.radians(20)), rel=1e-6)


# ---------------------------------------------------------------- Morton hierarchy


def test_morton_hand_worked_cube_corners():
    # Roots at the 8 corners of the unit cube: lo = 0, hi = 1, so each
    # coordinate quantises to 0 or 1023 (1024 clamped) and the 30-bit code of
    # corner (x, y, z) is (4x + 2y + z) * 0b001001...001 = (4x+2y+z) * 153391689.
    corners = np.array([[x, y, z] for x in (0, 1) for y in (0, 1) for z in (0, 1)], np.float32)
    perm = np.array([5, 2, 7, 0, 3, 6, 1, 4])
    roots = corners[perm]
    q = oracle.quantize_roots(roots)
    assert set(q.reshape(-1).tolist()) == {0, 1023}
    code = oracle.morton30(q)
    expect = [(4 * int(x) + 2 * int(y) + int(z)) * 153391689 for x, y, z in roots]
    assert code.tolist() == expect
    assert int(oracle.morton30(np.array([[1023, 1023, 1023]]))[0]) == 2 ** 30 - 1
    h = oracle.build_hierarchy(roots, 2)
    # sorted by code: strand ids ordered by 4x+2y+z of their corner
    assert h.order.tolist() == np.argsort(4 * roots[:, 0] + 2 * roots[:, 1] + roots[:, 2]).tolist()
    assert h.cluster_of[h.order].tolist() == [0, 0, 0, 0, 1, 1, 1, 1]


def test_morton_mid_point_and_ties():
    # 0.5 of the extent quantises to 512 = bit 9, i.e. code bits 29/28/27.
    roots = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [0.5, 0.5, 0.5]], np.float32)
    q = oracle.quantize_roots(roots)
    assert q[2].tolist() == [512, 512, 512]
    code = oracle.morton30(q)
    assert int(code[2]) == (1 << 29) | (1 << 28) | (1 << 27)
    h = oracle.build_hierarchy(roots, 1)
    # equal codes keep ascending strand id
    assert h.order.tolist() == [0, 2, 3, 1]


def test_morton_quantises_in_bounding_cube():
    # extents 2 x 1 x 0.5: one scale 1024 / 2 for every axis
    roots = np.array([[0, 0, 0], [2, 1, 0.5], [1, 0.5, 0.25]], np.float32)
    q = oracle.quantize_roots(roots)
    assert q.tolist() == [[0, 0, 0], [1023, 512, 256], [512, 256, 128]]


def _morton_by_strings(q):
    out = []
    for x, y, z in q:
        bx, by, bz = format(int(x), "010b"), format(int(y), "010b"), format(int(z), "010b")
        out.append(int("".join(a + b + c for a, b, c in zip(bx, by, bz)), 2))
    return out


def test_morton_brute_force_random():
    rng = np.random.default_rng(3)
    q = rng.integers(0, 1024, size=(200, 3))
    assert oracle.morton30(q).tolist() == _morton_by_strings(q)


@pytest.mark.parametrize("N,C", [(100, 7), (1000, 16), (777, 13), (64, 4)])
def test_hierarchy_partition_and_nesting(N, C):
    rng = np.random.default_rng(N)
    roots = rng.normal(size=(N, 3)).astype(np.float32)
    h = oracle.build_hierarchy(roots, C)
    sizes = np.bincount(h.cluster_of, minlength=C)
    assert sizes.sum() == N and sizes.max() - sizes.min() <= 1
    assert h.n_levels == oracle.n_eth_levels_for(N, C)
    for k in range(h.n_levels):
        ids = h.eth_of[k] - h.eth_offset[k]
        cnt = np.bincount(ids, minlength=C * 4 ** k)
        assert cnt.min() >= 2  # at least two strands per thick hair
        # member lists agree with the per-strand assignment
        for e in range(h.eth_offset[k], h.eth_offset[k + 1]):
            mem = h.order[h.eth_first_rank[e]: h.eth_first_rank[e] + h.eth_count[e]]
            assert np.all(h.eth_of[k][mem] == e)
        if k + 1 < h.n_levels:
            sub_k = (h.eth_of[k] - h.eth_offset[k]) % 4 ** k
            sub_k1 = (h.eth_of[k + 1] - h.eth_offset[k + 1]) % 4 ** (k + 1)
            assert np.all(sub_k1 // 4 == sub_k)  # level k+1 refines level k


def test_level_count_rule():
    # 10,000 strands in 256 clusters: floor(39/2) = 19 -> 4^2 <= 19 -> 3 levels
    assert oracle.n_eth_levels_for(10000, 256) == 3
    # 100,000 in 4096: floor(24/2) = 12 -> 4^1 <= 12 < 4^2 -> 2 levels
    assert oracle.n_eth_levels_for(100000, 4096) == 2
    assert oracle.n_eth_levels_for(500000, 16384) == 2
    assert oracle.n_eth_levels_for(64, 64) == 0


# ---------------------------------------------------------------- ellipse fit


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cross_section_closed_form(seed):
    # Five parallel strands whose points sit at the centre and at the ends of
    # two known axes: the fit must return that centre, e1 = the longer axis
    # (up to sign) and semi-axes A + r, B + r.
    Rm = _rot(seed)
    A, B, r = 0.3, 0.1, 0.01
    e1, e2, t = Rm[:, 0], Rm[:, 1], Rm[:, 2]
    c = np.array([0.2, -0.4, 1.0])
    pts = np.array([c, c + A * e1, c - A * e1, c + B * e2, c - B * e2])
    tans = np.tile(t, (5, 1))
    cc, tt, f1, f2, a, b = oracle.fit_cross_section(pts, tans, np.full(5, r))
    assert np.allclose(cc, c, atol=1e-14)
    assert np.allclose(tt, t, atol=1e-14)
    assert abs(abs(np.dot(f1, e1)) - 1) < 1e-12
    assert abs(abs(np.dot(f2, e2)) - 1) < 1e-12
    assert a == pytest.approx(A + r, rel=1e-12)
    assert b == pytest.approx(B + r, rel=1e-12)


def test_cross_section_contains_members_and_rotation_invariance():
    rng = np.random.default_rng(7)
    pts = rng.normal(size=(9, 3)) * [0.05, 0.02, 0.001]
    tans = np.tile([0.0, 0.0, 1.0], (9, 1)) + rng.normal(size=(9, 3)) * 1e-3
    tans /= np.linalg.norm(tans, axis=1, keepdims=True)
    radii = np.full(9, 1e-3)
    c, t, e1, e2, a, b = oracle.fit_cross_section(pts, tans, radii)
    u = (pts - c) @ e1
    v = (pts - c) @ e2
    assert np.all((u / a) ** 2 + (v / b) ** 2 <= 1 + 1e-12)
    assert abs(np.dot(e1, t)) < 1e-12 and abs(np.dot(e2, t)) < 1e-12
    Rm = _rot(11)
    c2, t2, f1, f2, a2, b2 = oracle.fit_cross_section(pts @ Rm.T, tans @ Rm.T, radii)
    assert np.allclose(c2, Rm @ c, atol=1e-14)
    assert abs(abs(np.dot(f1, Rm @ e1)) - 1) < 1e-9
    assert a2 == pytest.approx(a, rel=1e-9) and b2 == pytest.approx(b, rel=1e-9)


def test_batched_fit_matches_single_fit():
    w = scenegen.clustered(n=600, S=6, res=32, spp=1, n_clusters=24)
    h = oracle.build_hierarchy(w.scene.verts[:, 0, :3], 24)
    eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h, chunk=17)
    P = w.scene.verts[..., :3].astype(np.float64)
    T = oracle.strand_tangents(P)
    R = w.scene.verts[..., 3].astype(np.float64)
    for e in range(0, h.n_eths, 5):
        mem = h.order[h.eth_first_rank[e]: h.eth_first_rank[e] + h.eth_count[e]]
        for k in range(P.shape[1]):
            c, t, e1, e2, a, b = oracle.fit_cross_section(P[mem, k], T[mem, k], R[mem, 0])
            assert np.allclose(eth.center[e, k], c, atol=1e-13)
            assert abs(abs(np.dot(eth.e1[e, k], e1)) - 1) < 1e-9
            assert eth.a[e, k] == pytest.approx(a, rel=1e-9)
            assert eth.b[e, k] == pytest.approx(b, rel=1e-9)
        assert eth.ntot[e] == len(mem)
        assert np.allclose(eth.mat[e], w.scene.mat[mem].astype(np.float64).mean(0))


# ---------------------------------------------------------------- intersection


def _row(c0, c1, e1, a, b):
    return np.array([*c0, *c1, *e1, a, b, 0, 0, 1, 1e-3], np.float64)


@pytest.mark.parametrize("h", [0.0, 0.3e-3, 0.9e-3, -0.5e-3])
def test_circular_cylinder_perpendicular_hit(h):
    # circular cylinder (a = b = r) along z; ray along -x at height z = 0.5,
    # offset h in y, starting at x = d: t = d - sqrt(r^2 - h^2), chord 2 sqrt(.)
    r, d = 1e-3, 2.0
    row = _row([0, 0, 0], [0, 0, 1], [1, 0, 0], r, r)
    hit, t, ch = oracle.intersect(row, [d, h, 0.5], [-1, 0, 0])
    assert hit
    assert t == pytest.approx(d - math.sqrt(r * r - h * h), abs=1e-15)
    assert ch == pytest.approx(2 * math.sqrt(r * r - h * h), rel=1e-9)


@pytest.mark.parametrize("h", [0.0, 0.2, 0.49])
def test_elliptic_cylinder_axis_aligned_hit(h):
    # ellipse with semi-axis a along x (e1) and b along y: a ray along -x at
    # offset y = h hits at t = d - a sqrt(1 - h^2/b^2)
    a, b, d = 2.0, 0.5, 10.0
    row = _row([0, 0, -1], [0, 0, 1], [1, 0, 0], a, b)
    hit, t, ch = oracle.intersect(row, [d, h, 0.0], [-1, 0, 0])
    assert hit
    assert t == pytest.approx(d - a * math.sqrt(1 - h * h / (b * b)), rel=1e-13)
    # and along -y at offset x = h: t = d - b sqrt(1 - h^2/a^2)
    hit, t, ch = oracle.intersect(row, [h, d, 0.0], [0, -1, 0])
    assert t == pytest.approx(d - b * math.sqrt(1 - h * h / (a * a)), rel=1e-13)


def test_eccentricity_zero_equals_circle():
    rng = np.random.default_rng(5)
    for _ in range(50):
        c0 = rng.normal(size=3)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        c1 = c0 + 0.3 * ax
        e1 = np.cross(ax, rng.normal(size=3))
        e1 /= np.linalg.norm(e1)
        o = c0 + rng.normal(size=3) * 2
        tgt = c0 + 0.15 * ax + rng.normal(size=3) * 0.02
        d = (tgt - o) / np.linalg.norm(tgt - o)
        r = 0.03
        hit, t, ch = oracle.intersect(_row(c0, c1, e1, r, r), o, d)
        # circular cylinder: distance from the axis line equals r at the hit
        if hit:
            p = o + t * d
            q = p - c0
            dist = np.linalg.norm(q - np.dot(q, ax) * ax)
            assert dist == pytest.approx(r, rel=1e-9)
            assert -1e-12 <= np.dot(q, ax) <= 0.3 + 1e-12


def test_intersection_misses_and_open_ends():
    row = _row([0, 0, 0], [0, 0, 1], [1, 0, 0], 0.1, 0.1)
    assert not oracle.intersect(row, [1, 0, 0.5], [0, 0, 1])[0]    # parallel to the axis
    assert not oracle.intersect(row, [1, 0.2, 0.5], [-1, 0, 0])[0]  # passes beside
    assert not oracle.intersect(row, [1, 0, 1.5], [-1, 0, 0])[0]    # beyond the far end
    # a ray down the axis direction enters through an (open) end cap and exits
    # through the side wall: the hit is the exit root
    d = np.array([0.2, 0.0, 1.0])
    d /= np.linalg.norm(d)
    hit, t, ch = oracle.intersect(row, [0, 0, -0.2], d)
    assert hit
    p = np.array([0, 0, -0.2]) + t * d
    assert math.hypot(p[0], p[1]) == pytest.approx(0.1, rel=1e-9)
    assert p[2] == pytest.approx(0.3, rel=1e-9)
    # the chord inside the finite cylinder runs from z = 0 to the exit
    assert ch == pytest.approx(0.3 * math.sqrt(1.04), rel=1e-9)
    # a steeper ray leaves through the far (open) end: no hit
    d = np.array([0.05, 0.0, 1.0])
    assert not oracle.intersect(row, [0, 0, -0.5], d / np.linalg.norm(d))[0]


# ---------------------------------------------------------------- BCSDF


def test_gaussian_definition():
    assert oracle.gauss(0.3, 0.0) == pytest.approx(1 / (math.sqrt(2 * PI) * 0.3), rel=1e-15)
    assert oracle.gauss(0.3, 0.3) == pytest.approx(math.exp(-0.5) / (math.sqrt(2 * PI) * 0.3),
                                                   rel=1e-15)


@pytest.mark.parametrize("beta", [0.04, 0.08, 0.1])
@pytest.mark.parametrize("theta", [0.0, 0.2, 0.35])
def test_longitudinal_integral_closed_form(beta, theta):
    # With theta_o = 2h - theta, IM = 2 int G(beta, h) cos^2(2h - theta) dh.
    # When the Gaussian sits far inside the integration window the window can be
    # dropped, and E[cos(4h - 2 theta)] = cos(2 theta) exp(-8 beta^2) gives
    # IM = 1 + cos(2 theta) exp(-8 beta^2).
    expect = 1 + math.cos(2 * theta) * math.exp(-8 * beta * beta)
    assert oracle.im(theta, beta) == pytest.approx(expect, abs=1e-11)


def test_longitudinal_integral_quadrature_converged():
    for beta in (0.04, 0.2, 0.45, 0.64):
        for th in (0.0, 0.7, 1.5):
            assert oracle.im(th, beta, nq=384) == pytest.approx(oracle.im(th, beta, nq=1200),
                                                                abs=1e-12)


def test_f_single_hand_values():
    # theta_i = theta_o = 0 and phi = pi: every Gaussian at its peak.
    m = BROWN
    f = oracle.f_single(m, 0.0, 0.0, -1.0)
    for c in range(3):
        expect = (m[c] * g(m[9], 0) / (2 * PI) + m[3 + c] * g(m[10], 0) * g(m[11], 0)
                  + m[6 + c] / (2 * PI * PI))
        assert f[c] == pytest.approx(expect, rel=1e-14)
    # theta_h = 0.1, phi = pi/2: TT azimuth at -pi/2
    th_i, th_o = 0.3, -0.1
    f = oracle.f_single(m, th_i, th_o, 0.0)
    for c in range(3):
        expect = (m[c] * g(m[9], 0.1) / (2 * PI) + m[3 + c] * g(m[10], 0.1) * g(m[11], -PI / 2)
                  + m[6 + c] / (2 * PI * PI))
        assert f[c] == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("mat", [C1_MAT, BROWN, DARK, LIGHT])
@pytest.mark.parametrize("theta_d", [0.0, 0.5, 1.3, -2.0, 3.0])
def test_separable_albedo_equals_2d_quadrature(mat, theta_d):
    # a_F / a_B in product form must equal the direct 2-D integral of f_single
    # over the front / back half at incidence |theta_d| / 2.
    aF, aB, s2 = oracle.albedo(mat, theta_d)
    fr, bk = oracle.albedo_2d(mat, abs(theta_d) / 2, nq=300)
    assert np.allclose(aF, fr, rtol=1e-9)
    assert np.allclose(aB, bk, rtol=1e-9)
    assert min(mat[9], mat[10]) ** 2 <= s2 <= max(mat[9], mat[10]) ** 2


def test_albedo_white_furnace_c1_material():
    # the grey C1 fibre loses energy at every incidence: a_F + a_B <= 1
    for th in np.linspace(-3.1, 3.1, 25):
        aF, aB, _ = oracle.albedo(C1_MAT, th)
        assert np.all(aF + aB <= 1.0)
        assert np.all(aF > 0) and np.all(aB > 0)


@pytest.mark.parametrize("aF,aB", [(0.3, 0.1), (0.8, 0.2), (0.95, 0.04), (0.5, 0.5)])
def test_back_lobe_attenuations_equal_their_series(aF, aB):
    A1, A3, _ = oracle.back_atten(aF, aB, 1.0)
    # one backward and 2k forward events, k >= 1
    s1 = sum(aB * aF ** (2 * k) for k in range(1, 4000))
    # three backward events: a_B^3 a_F^2 sum_k C(k+2, 2) a_F^(2k)
    s3 = sum(aB ** 3 * aF ** 2 * math.comb(k + 2, 2) * aF ** (2 * k) for k in range(0, 4000))
    assert A1 == pytest.approx(s1, rel=1e-10)
    assert A3 == pytest.approx(s3, rel=1e-10)
    for n in (1, 2, 5, 17):
        _, _, A1p = oracle.back_atten(aF, aB, float(n))
        series = 0.6 * aB * sum(aF ** (2 * i - 1) for i in range(1, n + 1))
        assert A1p == pytest.approx(series, rel=1e-12)


def _random_angles(rng, n):
    th_i = rng.uniform(-1.4, 1.4, n)
    th_o = rng.uniform(-1.4, 1.4, n)
    cphi = rng.uniform(-1, 1, n)
    return th_i, th_o, cphi


@pytest.mark.parametrize("mat", [BROWN, DARK, LIGHT])
def test_aggregated_reciprocity(mat):
    rng = np.random.default_rng(1)
    for th_i, th_o, cp in zip(*_random_angles(rng, 40)):
        for rho, n in ((0.2, 1.0), (0.5, 3.7), (0.9, 12.0)):
            a = oracle.f_ours(mat, th_i, th_o, cp, rho, n)
            b = oracle.f_ours(mat, th_o, th_i, cp, rho, n)
            assert np.allclose(a, b, rtol=1e-12, atol=0)


@pytest.mark.parametrize("mat", [BROWN, DARK])
def test_aggregated_reduces_to_single_at_n1_front(mat):
    # Section 4: with n = 1 the R^, TT^, D^ lobes are the single-fibre ones;
    # in the front hemisphere B^ and S vanish, so f_ours = f_single.
    rng = np.random.default_rng(2)
    for th_i, th_o, cp in zip(*_random_angles(rng, 30)):
        cp = -abs(cp)
        assert np.allclose(oracle.f_ours(mat, th_i, th_o, cp, 0.3, 1.0),
                           oracle.f_single(mat, th_i, th_o, cp), rtol=1e-12)


def test_back_lobe_uniform_over_back_half():
    # Without S, in the back hemisphere f_ours - f_single is the B^ lobe, whose
    # azimuthal part I_B / pi does not depend on phi.
    m = BROWN
    for th_i, th_o in ((0.2, 0.1), (-0.6, 0.4), (1.0, 1.1)):
        diffs = [oracle.f_ours(m, th_i, th_o, cp, 0.4, 3.0, flags=oracle.FLAG_NO_S)
                 - oracle.f_single(m, th_i, th_o, cp) for cp in (0.05, 0.4, 0.8, 1.0)]
        for d in diffs[1:]:
            assert np.allclose(d, diffs[0], rtol=1e-12)
        assert np.all(diffs[0] > 0)


def test_shadowing_masking_bounds_and_ablation_order():
    # S lies in [0, 1] (Eq. 13), so dropping it brightens (Section 7, S-term
    # ablation); at rho = 1 there is nothing to shadow.
    rng = np.random.default_rng(4)
    for th_i, th_o, cp in zip(*_random_angles(rng, 60)):
        for rho in (0.0, 0.3, 0.8, 1.0):
            with_s = oracle.f_ours(DARK, th_i, th_o, cp, rho, 2.5)
            no_s = oracle.f_ours(DARK, th_i, th_o, cp, rho, 2.5, flags=oracle.FLAG_NO_S)
            assert np.all(with_s <= no_s * (1 + 1e-14))
            assert np.all(with_s >= 0)
            if rho == 1.0 or cp <= 0:
                assert np.allclose(with_s, no_s, rtol=1e-14)


def test_attenuation_with_hair_count():
    # Eq. 6: more hairs crossed in the front hemisphere attenuate R^, TT^, D^ by
    # a_F^(n-1); with the same widened lobes, doubling n-1 squares the factor.
    th_i, th_o, cp = 0.0, 0.0, -1.0
    f1 = oracle.f_ours(BROWN, th_i, th_o, cp, 0.5, 1.0)
    f3 = oracle.f_ours(BROWN, th_i, th_o, cp, 0.5, 3.0)
    assert np.all(f3 < f1)


def test_forward_albedo_stays_below_one_over_parameter_box():
    # the dual-scattering sums of the B lobe need a_F < 1; the input recipe keeps
    # every material of the parameter box well inside
    for mel in (0.1, 0.5, 0.9):
        for rough in (0.1, 0.2, 0.3):
            m = scenegen.material_from_melanin(np.array([mel]), np.array([rough]))[0]
            for th in np.linspace(-3.1, 3.1, 13):
                aF, aB, _ = oracle.albedo(m.astype(np.float64), th)
                assert np.all(aF < 0.7) and np.all(aF + aB < 1.0)


def test_degenerate_cross_section_axis():
    # Two strands offset mostly along the tangent: the separation axis is the
    # one dropped and the kept pair has zero variance; e1 must then point to the
    # member's offset in the normal plane (here along x), and the ellipse must
    # still contain both centres.
    t = np.array([0.0, 0.0, 1.0])
    pts = np.array([[0.01, 0.0, 0.3], [-0.01, 0.0, -0.3]])
    c, tt, e1, e2, a, b = oracle.fit_cross_section(pts, np.tile(t, (2, 1)), np.full(2, 1e-3))
    assert abs(abs(e1[0]) - 1) < 1e-12
    assert a == pytest.approx(0.011, rel=1e-12)
    # the batched fit takes the same branch
    w = scenegen.clustered(n=3000, S=12, res=64, spp=1, n_clusters=64)
    h = oracle.build_hierarchy(w.scene.verts[:, 0, :3], 64)
    eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h)
    P = w.scene.verts[..., :3].astype(np.float64)
    T = oracle.strand_tangents(P)
    R = w.scene.verts[..., 3].astype(np.float64)
    n2 = np.nonzero(h.eth_count == 2)[0][:40]
    for e in n2:
        mem = h.order[h.eth_first_rank[e]: h.eth_first_rank[e] + 2]
        for k in range(P.shape[1]):
            _, _, f1, _, fa, fb = oracle.fit_cross_section(P[mem, k], T[mem, k], R[mem, 0])
            assert abs(abs(np.dot(eth.e1[e, k], f1)) - 1) < 1e-9
            assert eth.a[e, k] == pytest.approx(fa, rel=1e-9)


def _thick_hair_row(c0, c1, e1, a, b, ntot, r):
    return np.array([*c0, *c1, *e1, a, b, 1, 1, ntot, r], np.float64)


def test_composite_front_to_back_with_closed_form_opacity():
    # One circular thick hair (radius R, n_tot members of radius r) in front of
    # an opaque strand.  A ray through the thick hair's axis has chord 2R, so
    # its opacity is alpha = 1 - exp(-2 r (2R) n_tot / (pi R^2)); compositing
    # must give render(thick hair alone) + (1 - alpha) * render(strand alone).
    R, r, ntot = 0.05, 0.002, 20.0
    eth = _thick_hair_row([0, -0.5, 0], [0, 0.5, 0], [1, 0, 0], R, R, ntot, r)
    strand = np.array([0, -0.5, -0.2, 0, 0.5, -0.2, 1, 0, 0, 0.01, 0.01, 0, 0, 1, 0.01],
                      np.float64)
    mats = np.tile(scenegen.material_from_melanin(np.array([0.5]), np.array([0.2]))
                   .astype(np.float64), (2, 1))
    cam = scenegen.Camera(0, 1, 1, np.array([0, 0, 3], np.float32),
                          np.array([1, 0, 0], np.float32), np.array([0, 1, 0], np.float32),
                          np.array([0, 0, -1], np.float32), 1e6).pack()
    lights = scenegen.directional_light((0.3, 0.5, 1.0))

    def render(rows, ids):
        prep = oracle.Prepared(np.ascontiguousarray(rows), np.asarray(ids, np.int64), mats,
                               None, None, None)
        rad, hit = oracle.render_samples(prep, cam, lights, np.array([0]), 1, 4, 1, threads=1)
        return rad[0], hit[0]

    both, hit = render(np.stack([eth, strand]), [5, 9])
    a_only, ha = render(eth[None], [5])
    s_only, hs = render(strand[None], [9])
    alpha = 1 - math.exp(-2 * r * (2 * R) * ntot / (math.pi * R * R))
    assert hit.tolist() == [5, 9, -1, -1] and ha[0] == 5 and hs[0] == 9
    assert np.allclose(both, a_only + (1 - alpha) * s_only, rtol=1e-9)
    # an opaque strand in front hides everything behind it
    front = strand.copy()
    front[[2, 5]] = 0.3
    occl, h2 = render(np.stack([eth, front]), [5, 9])
    f_only, _ = render(front[None], [9])
    assert h2.tolist() == [9, -1, -1, -1] and np.allclose(occl, f_only, rtol=1e-12)


def test_albedo_2d_diffuse_closed_form():
    # A diffuse-only fibre (A_R = A_TT = 0): f = A_D / (2 pi^2) everywhere, so
    # each half's albedo is A_D / (2 pi^2) * int cos^2 = pi / 2 * (azimuth pi)
    # = A_D / 4, at every incidence.
    m = np.zeros(12)
    m[6:9] = (0.2, 0.5, 0.9)
    m[9:12] = (0.1, 0.15, 0.3)
    for th in (0.0, 0.4, 1.2):
        fr, bk = oracle.albedo_2d(m, th, nq=64)
        assert np.allclose(fr, m[6:9] / 4, rtol=1e-12)
        assert np.allclose(bk, m[6:9] / 4, rtol=1e-12)
