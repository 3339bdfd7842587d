"""Pins of the oracle's light-path transmittance (dual scattering under shadow
rays, Section 3.2; hairs on the shadow path found by ray shooting, Section 6).

The reading under test: a shadow ray from the shading point toward the light
crosses hairs; a strand segment counts one hair, a thick-hair segment
n = rho l sqrt(n_tot / (pi a b)) hairs for its chord l; each hair multiplies
the transmittance by its forward albedo a_F at incidence |asin(w . t)| and adds
its forward spread variance; T = d_F prod a_F^n with d_F = 0.7 once any hair
is crossed.  The checks below build small scenes whose crossings are known in
closed form (which primitives, which angles, which chords) and compare with
the albedo function, itself pinned in test_oracle_pins.py.
"""
import math

import numpy as np

import oracle
import scenegen

D_F = 0.7


def _mat(melanin, rough):
    return scenegen.material_from_melanin(np.array([melanin]), np.array([rough]))[0].astype(np.float64)


def _row(c0, c1, e1, a, b, kind, mat, ntot=1.0, r=0.01):
    return np.array([*c0, *c1, *e1, a, b, kind, mat, ntot, r], np.float64)


def _seg(x, tilt_deg, mat, r=0.01, L=0.2, kind=0, a=None, b=None, ntot=1.0):
    """A segment centred on (x, 0, 0), axis in the x-y plane at tilt_deg from
    +y toward +x, e1 along +z."""
    t = np.array([math.sin(math.radians(tilt_deg)), math.cos(math.radians(tilt_deg)), 0.0])
    c = np.array([x, 0.0, 0.0])
    return _row(c - 0.5 * L * t, c + 0.5 * L * t, [0.0, 0.0, 1.0], a or r, b or r, kind, mat,
                ntot, r)


def _albedo(mat, theta):
    aF, aB, s2 = oracle.albedo(mat, 2.0 * theta)
    return np.asarray(aF), s2


MATS = np.stack([_mat(0.5, 0.2), _mat(0.2, 0.15), _mat(0.8, 0.3)])
X0 = np.zeros(3)
WX = np.array([1.0, 0.0, 0.0])


def test_single_strand_occluder():
    rows = _seg(1.0, 0.0, 1)[None]
    T, sg2 = oracle.shadow_path(rows, MATS, X0, WX, math.inf, 0)
    aF, s2 = _albedo(MATS[1], 0.0)
    assert np.allclose(T, D_F * aF, rtol=1e-12)
    assert math.isclose(sg2, s2, rel_tol=1e-12)


def test_occluder_behind_the_light_or_the_shading_hair_is_not_counted():
    rows = _seg(1.0, 0.0, 1)[None]
    T, sg2 = oracle.shadow_path(rows, MATS, X0, WX, 0.5, 0)  # point light before it
    assert np.array_equal(T, np.ones(3)) and sg2 == 0.0
    T, sg2 = oracle.shadow_path(rows, MATS, X0, WX, math.inf, 1)  # the shading hair itself
    assert np.array_equal(T, np.ones(3)) and sg2 == 0.0
    T, sg2 = oracle.shadow_path(rows, MATS, X0, -WX, math.inf, 0)  # light on the other side
    assert np.array_equal(T, np.ones(3)) and sg2 == 0.0


def test_two_tilted_occluders_multiply_and_their_spreads_add_in_any_order():
    a, b = _seg(1.0, 0.0, 1), _seg(2.0, 30.0, 2)
    T, sg2 = oracle.shadow_path(np.stack([a, b]), MATS, X0, WX, math.inf, 0)
    T2, sg22 = oracle.shadow_path(np.stack([b, a]), MATS, X0, WX, math.inf, 0)
    aF1, s21 = _albedo(MATS[1], 0.0)
    # the ray along +x meets the axis tilted 30 degrees from +y toward +x:
    # sin(theta) = w . t = sin(30 deg)
    aF2, s22 = _albedo(MATS[2], math.radians(30.0))
    assert np.allclose(T, D_F * aF1 * aF2, rtol=1e-12)
    assert math.isclose(sg2, s21 + s22, rel_tol=1e-12)
    assert np.allclose(T2, T, rtol=1e-14) and math.isclose(sg22, sg2, rel_tol=1e-14)


def test_thick_hair_occluder_counts_its_hair_number_over_the_chord():
    a_, b_, ntot, r = 0.05, 0.03, 40.0, 0.004
    rows = _seg(1.0, 0.0, 2, r=r, kind=1, a=a_, b=b_, ntot=ntot)[None]
    rho = min(1.0, ntot * r * r / (a_ * b_))
    aF, s2 = _albedo(MATS[2], 0.0)
    for h in (0.0, 0.02, 0.04):  # offset along e1 (z): chord 2 b sqrt(1 - h^2 / a^2)
        x = np.array([0.0, 0.0, h])
        chord = 2.0 * b_ * math.sqrt(1.0 - h * h / (a_ * a_))
        n = rho * chord * math.sqrt(ntot / (math.pi * a_ * b_))
        T, sg2 = oracle.shadow_path(rows, MATS, x, WX, math.inf, 0)
        assert np.allclose(T, D_F * aF ** n, rtol=1e-10), (h, T, D_F * aF ** n)
        assert math.isclose(sg2, n * s2, rel_tol=1e-10)
    # starting inside it: only the part of the chord in front of the point
    x = np.array([1.0, 0.0, 0.0])
    n = rho * b_ * math.sqrt(ntot / (math.pi * a_ * b_))
    T, sg2 = oracle.shadow_path(rows, MATS, x, WX, math.inf, 0)
    assert np.allclose(T, D_F * aF ** n, rtol=1e-10)


def test_spread_is_a_wider_lobe():
    """f_single with spread s equals f_single of a material whose lobe
    variances are larger by s."""
    m = MATS[0]
    s = 0.013
    wide = m.copy()
    wide[9:12] = np.sqrt(m[9:12] ** 2 + s)
    for th_i, th_o, cphi in ((0.2, -0.1, 0.3), (-0.6, 0.4, -0.9), (0.05, 0.05, 1.0)):
        assert np.allclose(oracle.f_single_spread(m, th_i, th_o, cphi, s),
                           oracle.f_single(wide, th_i, th_o, cphi), rtol=1e-13)
        assert np.allclose(oracle.f_single_spread(m, th_i, th_o, cphi, 0.0),
                           oracle.f_single(m, th_i, th_o, cphi), rtol=0, atol=0)


def test_unoccluded_scene_renders_the_same_with_shadow_rays():
    """A single strand lit by a directional light has nothing on its light
    path: the shadow-ray render equals the plain one."""
    w = scenegen.tiny_strands()
    one = scenegen.Scene(w.scene.verts[:1], w.scene.mat[:1], w.scene.shape[:1], "one")
    prep = oracle.prepare(one, 0, "all", w.camera.pack())
    sids = np.arange(w.camera.width * w.camera.height * w.spp, dtype=np.int64)
    r0, h0 = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, w.k_depth,
                                   w.sample_seed)
    r1, h1 = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, w.k_depth,
                                   w.sample_seed, flags=oracle.FLAG_SHADOWS)
    assert np.array_equal(h0, h1)
    assert np.array_equal(r0, r1)
    assert r0.max() > 0
