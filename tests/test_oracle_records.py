"""Pins of the oracle's primitive records, tangents, active set, k-buffer
and light sum.

Each check compares an oracle function with something fixed outside it: an
orthonormal right-handed basis and the values of Duff et al.'s construction
at the poles; ellipse identities (a b = r^2, b / a = sqrt(1 - e^2)) read off
through the independent ray / cylinder test as hit distances; the tangent of
a circle; a hand-built thick hair whose cylinder must pass through known
surface points; hand-counted active sets; the K nearest hits ordered by hand;
and radiance values worked out from the lights' geometry.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen

PI = math.pi


# ---------------------------------------------------------------- quadrature


def test_gauss_legendre_is_exact_for_polynomials_up_to_degree_2n_minus_1():
    x, w = oracle.gauss_legendre(12)
    for k in range(0, 24):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert np.dot(w, x ** k) == pytest.approx(exact, abs=1e-13)


# ---------------------------------------------------------------- Duff basis


def test_duff_basis_orthonormal_and_right_handed():
    rng = np.random.default_rng(0)
    n = rng.normal(size=(500, 3))
    # include the poles, the equator and near-pole directions
    n = np.concatenate([n, [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, 1, 0], [1e-9, 0, -1],
                            [0, 1e-7, 1]]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    b1, b2 = oracle.duff_basis(n)
    for u in (b1, b2):
        assert np.allclose(np.linalg.norm(u, axis=1), 1, atol=1e-12)
        assert np.allclose(np.sum(u * n, 1), 0, atol=1e-12)
    assert np.allclose(np.sum(b1 * b2, 1), 0, atol=1e-12)
    assert np.allclose(np.cross(b1, b2), n, atol=1e-12)


def test_duff_basis_values_at_the_poles():
    # Duff et al. 2017: sign = copysign(1, n_z), a = -1 / (sign + n_z),
    # b = n_x n_y a; at n = (0, 0, +-1) this gives b1 = (1, 0, 0) and
    # b2 = (0, +-1, 0); at n = (1, 0, 0), b1 = (0, 0, -1) and b2 = (0, 1, 0).
    b1, b2 = oracle.duff_basis(np.array([[0.0, 0, 1], [0, 0, -1], [1, 0, 0]]))
    assert np.allclose(b1, [[1, 0, 0], [1, 0, 0], [0, 0, -1]], atol=0)
    assert np.allclose(b2, [[0, 1, 0], [0, -1, 0], [0, 1, 0]], atol=0)


# ---------------------------------------------------------------- strand records


def _strand_scene(e, psi, r=2e-3, direction=(0, 0, 1), S=2):
    v = np.zeros((1, S + 1, 4), np.float32)
    d = np.asarray(direction, np.float64)
    d /= np.linalg.norm(d)
    v[0, :, :3] = np.arange(S + 1)[:, None] * 0.5 * d[None, :]
    v[0, :, 3] = r
    return v, np.array([[e, psi]], np.float32)


@pytest.mark.parametrize("e", [0.0, 0.6, 0.8, 0.95])
def test_strand_ellipse_area_and_eccentricity(e):
    # a b = r^2 (the area of the area-equivalent circle) and b / a = sqrt(1 - e^2)
    # (the eccentricity's definition), for random orientations
    rng = np.random.default_rng(int(e * 100))
    for _ in range(20):
        d = rng.normal(size=3)
        psi = rng.uniform(0, 2 * PI)
        v, shape = _strand_scene(e, psi, direction=d)
        rows, ids = oracle.strand_prim_rows(v, shape, np.array([0]))
        a, b = rows[:, 9], rows[:, 10]
        r = float(v[0, 0, 3])
        assert np.allclose(a * b, r * r, rtol=1e-6)
        assert np.allclose(b / a, math.sqrt(1 - float(np.float32(e)) ** 2), rtol=1e-6)
        assert np.all(a >= b)


def test_strand_major_axis_orientation():
    # e1 is perpendicular to the segment, of unit length, and makes the angle
    # psi with the first Duff basis vector of the segment direction
    rng = np.random.default_rng(3)
    for _ in range(30):
        d = rng.normal(size=3)
        psi = float(np.float32(rng.uniform(0, 2 * PI)))
        v, shape = _strand_scene(0.8, psi, direction=d)
        rows, _ = oracle.strand_prim_rows(v, shape, np.array([0]))
        t = (rows[0, 3:6] - rows[0, 0:3])
        t /= np.linalg.norm(t)
        e1 = rows[0, 6:9]
        assert abs(np.dot(e1, t)) < 1e-6 and abs(np.linalg.norm(e1) - 1) < 1e-12
        b1, b2 = oracle.duff_basis(t)
        ang = math.atan2(np.dot(e1, b2), np.dot(e1, b1)) % (2 * PI)
        assert min(abs(ang - psi), 2 * PI - abs(ang - psi)) < 1e-6


def test_strand_semi_axes_as_hit_distances():
    # a strand along +z with psi = 0 has its major axis along b1 = (1, 0, 0):
    # a ray along -x at height z = 0.5 meets it at t = d - a, one along -y at
    # t = d - b, with a = r (1 - e^2)^(-1/4), b = r (1 - e^2)^(1/4).  An
    # exponent swap, or psi taken from b2, moves the hits.
    e, r, dist = 0.8, 2e-3, 3.0
    v, shape = _strand_scene(e, 0.0, r=r, direction=(0, 0, 1), S=2)
    rows, ids = oracle.strand_prim_rows(v, shape, np.array([0]))
    a = r * (1 - e * e) ** -0.25
    b = r * (1 - e * e) ** 0.25
    hit, t, _ = oracle.intersect(rows[0], [dist, 0, 0.3], [-1, 0, 0])
    assert hit and t == pytest.approx(dist - a, rel=1e-9)
    hit, t, _ = oracle.intersect(rows[0], [0, dist, 0.3], [0, -1, 0])
    assert hit and t == pytest.approx(dist - b, rel=1e-9)
    # psi = pi / 2: the axes swap
    v, shape = _strand_scene(e, PI / 2, r=r, direction=(0, 0, 1), S=2)
    rows, _ = oracle.strand_prim_rows(v, shape, np.array([0]))
    hit, t, _ = oracle.intersect(rows[0], [dist, 0, 0.3], [-1, 0, 0])
    assert hit and t == pytest.approx(dist - b, rel=1e-6)


def test_strand_record_fields_and_ids():
    v = scenegen.make_strands(5, 4, seed=1)
    shape = np.stack([np.full(5, 0.7), np.linspace(0, 3, 5)], -1).astype(np.float32)
    rows, ids = oracle.strand_prim_rows(v, shape, np.array([3, 1]))
    assert ids.tolist() == [12, 13, 14, 15, 4, 5, 6, 7]        # s * S + k
    assert np.allclose(rows[0, 0:3], v[3, 0, :3]) and np.allclose(rows[0, 3:6], v[3, 1, :3])
    assert np.allclose(rows[7, 0:3], v[1, 3, :3]) and np.allclose(rows[7, 3:6], v[1, 4, :3])
    assert rows[:, 11].tolist() == [0.0] * 8                    # strand kind
    assert rows[:, 12].tolist() == [3.0] * 4 + [1.0] * 4        # material row = strand
    assert np.all(rows[:, 14] == np.float32(1e-3))


# ---------------------------------------------------------------- tangents


def test_strand_tangents_on_a_circle():
    # vertices evenly spaced on a circle: the central difference at vertex k is
    # the circle's tangent there; the one-sided ends are the chord directions
    n = 9
    ang = np.linspace(0.2, 1.8, n)
    P = np.stack([np.cos(ang), np.sin(ang), np.zeros(n)], -1)[None]
    T = oracle.strand_tangents(P)[0]
    tan = np.stack([-np.sin(ang), np.cos(ang), np.zeros(n)], -1)
    assert np.allclose(T[1:-1], tan[1:-1], atol=1e-14)
    mid0, mid1 = 0.5 * (ang[0] + ang[1]), 0.5 * (ang[-2] + ang[-1])
    assert np.allclose(T[0], [-math.sin(mid0), math.cos(mid0), 0], atol=1e-14)
    assert np.allclose(T[-1], [-math.sin(mid1), math.cos(mid1), 0], atol=1e-14)


# ---------------------------------------------------------------- thick-hair records


def _four_strand_bundle(A, B, centres, r=1e-3):
    """Four strands whose k-th vertices sit at c_k +- A_k x and c_k +- B_k y."""
    S1 = len(centres)
    v = np.zeros((4, S1, 4), np.float32)
    for k, c in enumerate(centres):
        c = np.asarray(c, np.float64)
        v[0, k, :3] = c + [A[k], 0, 0]
        v[1, k, :3] = c - [A[k], 0, 0]
        v[2, k, :3] = c + [0, B[k], 0]
        v[3, k, :3] = c - [0, B[k], 0]
    v[..., 3] = r
    mat = scenegen.material_from_melanin(np.full(4, 0.5), np.full(4, 0.2))
    return v, mat


def test_thick_hair_segment_is_the_bundle_cylinder():
    # Four parallel straight strands along z at +-A x and +-B y: one thick hair
    # (4 strands, 1 cluster: one level) whose every segment is the elliptic
    # cylinder of semi-axes A + r and B + r about the z axis.  A ray along -x
    # at height z meets it at t = d - (A + r); along -y at t = d - (B + r).
    A, B, r, d = 0.03, 0.01, 1e-3, 2.0
    zs = [0.0, 0.4, 0.8]
    v, mat = _four_strand_bundle([A] * 3, [B] * 3, [(0, 0, z) for z in zs], r)
    h = oracle.build_hierarchy(v[:, 0, :3], 1)
    assert h.n_levels == 1 and h.n_eths == 1
    eth = oracle.fit_eths(v, mat, h)
    rows, ids = oracle.eth_prim_rows(eth, np.array([0]), 4, 2)
    assert ids.tolist() == [4 * 2 + 0, 4 * 2 + 1]               # N S + e S + k
    assert rows[:, 11].tolist() == [1.0, 1.0]                   # thick-hair kind
    assert rows[:, 12].tolist() == [4.0, 4.0]                   # material row N + e
    assert rows[:, 13].tolist() == [4.0, 4.0]                   # n_tot
    assert np.allclose(rows[:, 14], r)
    for k, zm in enumerate((0.2, 0.6)):
        hit, t, _ = oracle.intersect(rows[k], [d, 0, zm], [-1, 0, 0])
        assert hit and t == pytest.approx(d - (A + r), rel=1e-6)
        hit, t, _ = oracle.intersect(rows[k], [0, d, zm], [0, -1, 0])
        assert hit and t == pytest.approx(d - (B + r), rel=1e-6)
        # the cylinder runs between the two section centres
        assert np.allclose(rows[k, 0:3], [0, 0, zs[k]], atol=1e-7)
        assert np.allclose(rows[k, 3:6], [0, 0, zs[k + 1]], atol=1e-7)


def test_tapered_thick_hair_takes_the_wider_section():
    # Semi-axes that shrink along the hair: each segment keeps the larger
    # ellipse of its two end sections (so it contains both), seen as the hit
    # distance of rays along -x and -y.
    A = [0.04, 0.03, 0.02]
    B = [0.012, 0.015, 0.01]
    r, d = 1e-3, 2.0
    v, mat = _four_strand_bundle(A, B, [(0, 0, 0), (0, 0, 0.4), (0, 0, 0.8)], r)
    h = oracle.build_hierarchy(v[:, 0, :3], 1)
    eth = oracle.fit_eths(v, mat, h)
    rows, _ = oracle.eth_prim_rows(eth, np.array([0]), 4, 2)
    for k in range(2):
        hit, t, _ = oracle.intersect(rows[k], [d, 0, 0.2 + 0.4 * k], [-1, 0, 0])
        assert t == pytest.approx(d - (max(A[k], A[k + 1]) + r), rel=1e-6)
        hit, t, _ = oracle.intersect(rows[k], [0, d, 0.2 + 0.4 * k], [0, -1, 0])
        assert t == pytest.approx(d - (max(B[k], B[k + 1]) + r), rel=1e-6)


def test_bent_thick_hair_segment_frame():
    # A bundle whose axis bends: each segment's major axis is perpendicular to
    # the segment, lies in the plane of the section's axis and the segment, and
    # keeps a consistent sign along the hair.
    cs = [(0, 0, 0), (0, 0, 0.4), (0.1, 0, 0.75), (0.3, 0.05, 1.0)]
    v, mat = _four_strand_bundle([0.03] * 4, [0.01] * 4, cs)
    h = oracle.build_hierarchy(v[:, 0, :3], 1)
    eth = oracle.fit_eths(v, mat, h)
    rows, _ = oracle.eth_prim_rows(eth, np.array([0]), 4, 3)
    for k in range(3):
        t = rows[k, 3:6] - rows[k, 0:3]
        t /= np.linalg.norm(t)
        e1 = rows[k, 6:9]
        assert abs(np.dot(e1, t)) < 1e-12 and abs(np.linalg.norm(e1) - 1) < 1e-12
        # e1 is in span(section e1, t)
        n = np.cross(eth.e1[0, k], t)
        assert abs(np.dot(e1, n)) < 1e-9 * max(1.0, np.linalg.norm(n))
        assert np.dot(e1, eth.e1[0, k]) > 0
    assert np.dot(rows[0, 6:9], rows[1, 6:9]) > 0 and np.dot(rows[1, 6:9], rows[2, 6:9]) > 0


# ---------------------------------------------------------------- active set


def test_active_set_hand_counted():
    # 16 roots in 2 clusters of 8: floor(8 / 2) = 4 >= 4^1, so two thick-hair
    # levels: 1 thick hair per cluster (ids 0, 1) and 4 per cluster (ids 2-9).
    rng = np.random.default_rng(0)
    roots = rng.normal(size=(16, 3)).astype(np.float32)
    h = oracle.build_hierarchy(roots, 2)
    assert h.n_levels == 2 and h.n_eths == 10
    c0 = np.nonzero(h.cluster_of == 0)[0]
    c1 = np.nonzero(h.cluster_of == 1)[0]
    st, eh = oracle.active_set(16, 4, h, np.array([0, 2], np.uint8))
    assert st.tolist() == sorted(c1.tolist()) and eh.tolist() == [0]
    st, eh = oracle.active_set(16, 4, h, np.array([1, 0], np.uint8))
    assert st.tolist() == [] and eh.tolist() == [1, 2, 3, 4, 5]
    st, eh = oracle.active_set(16, 4, h, np.array([2, 2], np.uint8))
    assert st.tolist() == list(range(16)) and eh.tolist() == []
    st, eh = oracle.active_set(16, 4, h, np.array([2, 1], np.uint8))
    assert st.tolist() == sorted(c0.tolist()) and eh.tolist() == [6, 7, 8, 9]
    # prepare() lists exactly those rows and ids
    v = scenegen.make_strands(16, 4, seed=0)
    sc = scenegen.Scene(v, scenegen.material_from_melanin(np.full(16, 0.5), np.full(16, 0.2)),
                        np.zeros((16, 2), np.float32))
    prep = oracle.prepare(sc, 2, lod=np.array([2, 0], np.uint8))
    hs = oracle.build_hierarchy(v[:, 0, :3], 2)
    st, eh = oracle.active_set(16, 4, hs, np.array([2, 0], np.uint8))
    want = sorted([s * 4 + k for s in st for k in range(4)] + [64 + e * 4 + k for e in eh for k in range(4)])
    assert sorted(prep.ids.tolist()) == want
    assert prep.mats.shape[0] == 16 + hs.n_eths


# ---------------------------------------------------------------- k-buffer and light sum


def _ortho_camera(eye, fwd, right, up):
    return scenegen.Camera(0, 1, 1, np.asarray(eye, np.float32), np.asarray(right, np.float32),
                           np.asarray(up, np.float32), np.asarray(fwd, np.float32), 1e6).pack()


def _strand_row(x, z, r, mat, ydir=(0, 1, 0)):
    """Circular strand segment along y through (x, ., z)."""
    return np.array([x, -0.5, z, x, 0.5, z, 1, 0, 0, r, r, 0, mat, 1, r], np.float64)


def _render(rows, ids, mats, cam, lights, K, flags=0):
    prep = oracle.Prepared(np.ascontiguousarray(rows, np.float64), np.asarray(ids, np.int64),
                           np.ascontiguousarray(mats, np.float64), None, None, None)
    rad, hit = oracle.render_samples(prep, cam, lights, np.array([0]), 1, K, 1, flags=flags,
                                     threads=1)
    return rad[0], hit[0]


def test_kbuffer_keeps_the_nearest_in_order_and_breaks_ties_by_id():
    # Four thick hairs (not opaque) on the view ray, at depths 1 (z = 4), 2 and
    # 2 (a tie, z = 3) and 3 (z = 2) from the camera at z = 5: K = 3 keeps the
    # nearest, then the tie in id order; K = 8 keeps all four.
    cam = _ortho_camera([0, 0, 5], [0, 0, -1], [1, 0, 0], [0, 1, 0])
    mats = scenegen.material_from_melanin(np.array([0.5]), np.array([0.2])).astype(np.float64)
    R = 0.05

    def eth(z):
        return np.array([0, -0.5, z, 0, 0.5, z, 1, 0, 0, R, R, 1, 0, 4, 1e-3], np.float64)
    rows = np.stack([eth(2.0), eth(3.0), eth(3.0), eth(4.0)])
    _, hit = _render(rows, [40, 31, 30, 50], mats, cam, scenegen.directional_light((0, 0, 1)), 3)
    assert hit.tolist() == [50, 30, 31]
    _, hit = _render(rows, [40, 31, 30, 50], mats, cam, scenegen.directional_light((0, 0, 1)), 8)
    assert hit.tolist() == [50, 30, 31, 40, -1, -1, -1, -1]


def test_light_sum_point_and_directional_lights():
    # One circular strand along y at the origin, seen head-on by an
    # orthographic ray along -z (theta_o = 0).  Radiance = sum over lights of
    # f_single(theta_i, theta_o, cos phi) * E * cos(theta_i) * rgb with
    #   point light at P: E = 1 / |P - x|^2, omega_i = (P - x) / |P - x|;
    #   directional light: E = 1;
    #   sin(theta) = omega . t, cos(phi) between the projections on the
    #   plane normal to t.
    r = 0.01
    mat = scenegen.material_from_melanin(np.array([0.4]), np.array([0.15])).astype(np.float64)
    cam = _ortho_camera([0, 0, 3], [0, 0, -1], [1, 0, 0], [0, 1, 0])
    o, d = oracle.camera_ray(cam, 1, 0, 1)
    row = _strand_row(0.0, 0.0, r, 0)
    hit, t, _ = oracle.intersect(row, o, d)
    x = o + t * d
    P = np.array([0.0, 0.6, 2.0])
    wd = np.array([0.8, 0.3, 0.5])
    wd /= np.linalg.norm(wd)
    lights = np.zeros((2, 8), np.float32)
    lights[0, 0:3], lights[0, 3], lights[0, 4:7] = P, 1.0, (1.0, 0.5, 0.25)
    lights[1, 0:3], lights[1, 3], lights[1, 4:7] = wd, 0.0, (0.2, 0.4, 0.8)
    rad, h = _render(row[None], [7], mat[None], cam, lights, 1)
    assert h[0] == 7
    tan = np.array([0.0, 1.0, 0.0])
    wo = -d
    th_o = math.asin(np.dot(wo, tan))
    expect = np.zeros(3)
    for L, wi, E in ((lights[0], (P - x) / np.linalg.norm(P - x), 1 / np.dot(P - x, P - x)),
                     (lights[1], wd, 1.0)):
        si = np.dot(wi, tan)
        pi_, po = wi - si * tan, wo - np.dot(wo, tan) * tan
        cphi = np.dot(pi_, po) / (np.linalg.norm(pi_) * np.linalg.norm(po))
        f = oracle.f_single(mat, math.asin(si), th_o, cphi)
        expect += f * E * math.sqrt(1 - si * si) * L[4:7].astype(np.float64)
    assert np.allclose(rad, expect, rtol=1e-12)
    # the point light's geometry by hand: omega_i in the y-z plane, so cos phi = 1,
    # sin(theta_i) = 0.6 / |P - x|, E = 1 / |P - x|^2 with x = (0, 0, r) (to 1e-6)
    dist = math.hypot(0.6, 2.0 - r)
    f0 = oracle.f_single(mat, math.asin(0.6 / dist), 0.0, 1.0)
    alone, _ = _render(row[None], [7], mat[None], cam, lights[:1], 1)
    assert np.allclose(alone, f0 * (2.0 - r) / dist / dist ** 2 * [1.0, 0.5, 0.25], rtol=1e-5)


def test_thick_hair_shading_uses_the_hair_number_of_its_chord():
    # A circular thick hair of radius R with n_tot members of radius r, hit by
    # a ray through its axis (chord 2R): rho = n_tot r^2 / R^2,
    # n = rho 2R sqrt(n_tot / (pi R^2)), alpha = 1 - exp(-2 r (2R) n_tot / (pi R^2)),
    # and the sample's radiance is alpha * f_ours(., rho, n) E cos(theta_i).
    R, r, ntot = 0.05, 0.004, 30.0
    mat = scenegen.material_from_melanin(np.array([0.6]), np.array([0.2])).astype(np.float64)
    row = np.array([0, -0.5, 0, 0, 0.5, 0, 1, 0, 0, R, R, 1, 0, ntot, r], np.float64)
    cam = _ortho_camera([0, 0, 3], [0, 0, -1], [1, 0, 0], [0, 1, 0])
    for wl in ((0.0, 0.4, -1.0), (0.3, 0.2, 1.0)):   # light behind / in front of the hair
        wi = np.asarray(wl) / np.linalg.norm(wl)
        rad, h = _render(row[None], [3], mat[None], cam, scenegen.directional_light(wl), 1)
        rho = ntot * r * r / (R * R)
        n = rho * 2 * R * math.sqrt(ntot / (PI * R * R))
        alpha = 1 - math.exp(-2 * r * 2 * R * ntot / (PI * R * R))
        tan = np.array([0.0, 1.0, 0.0])
        si = np.dot(wi, tan)
        pi_ = wi - si * tan
        cphi = pi_[2] / np.linalg.norm(pi_)          # wo = +z, in the normal plane
        f = oracle.f_ours(mat, math.asin(si), 0.0, cphi, rho, max(1.0, n))
        assert np.allclose(rad, alpha * f * math.sqrt(1 - si * si), rtol=1e-6)
