"""Pins of the oracle's LoD selection (Section 5.1 step 5, Section 5.2, Eq. 14)."""
import math

import numpy as np
import pytest

import oracle
import scenegen


def test_init_rule_hand_worked():
    # levels 0..2 are thick hairs, 3 = strands; eps = 2 px
    w = np.array([[5.0, 3.0, 1.5],    # first level below 2 px is level 2
                  [1.0, 0.5, 0.2],    # level 0 already below
                  [9.0, 4.0, 2.0],    # none strictly below -> strands
                  [np.inf, 1.9, 1.0]], np.float32)
    assert oracle.select_lod_init(w, 2.0, 3).tolist() == [2, 0, 3, 1]


def test_deferred_rule_hand_worked():
    w = np.array([[5.0, 3.0, 1.5]] * 4 + [[1.0, 0.5, 0.2]] * 2 + [[2.0, 2.0, 2.0]], np.float32)
    prev = np.array([0, 2, 3, 1, 1, 0, 1], np.uint8)
    out = oracle.select_lod_deferred(w, prev, 2.0, 3)
    # row 0: L=0, w_cur 5 > 2 -> 1
    # row 1: L=2, w_cur 1.5 <= 2 < w_cur- 3 -> stay 2
    # row 2: L=3 (strands), w_cur- = 1.5 <= 2 -> 2
    # row 3: L=1, w_cur 3 > 2 -> 2
    # row 4: L=1, w_cur 0.5, w_cur- 1.0 <= 2 -> 0
    # row 5: L=0, w_cur 1.0 <= 2, w_cur- = +inf -> stay 0
    # row 6: L=1, w_cur 2 is not > 2; w_cur- 2 <= 2 -> 0
    assert out.tolist() == [1, 2, 2, 2, 0, 0, 0]


def test_budget_bias():
    assert oracle.apply_budget(np.array([0, 1, 3, 2], np.uint8), 2).tolist() == [0, 0, 1, 0]


def _single_eth(center, e1, e2, a, b):
    z = lambda v: np.asarray(v, np.float64)[None, None, :]
    return oracle.ETHs(center=z(center), tangent=z(np.cross(e1, e2)), e1=z(e1), e2=z(e2),
                       a=np.array([[a]]), b=np.array([[b]]), seg_e1=None, seg_a=None,
                       seg_b=None, ntot=None, radius=None, mat=None)


def test_width_orthographic_facing_camera():
    # orthographic camera along -z with 100 px per unit: an ellipse facing the
    # camera with a = 0.03 along x and b = 0.01 along y is 2a * 100 = 6 px wide
    cam = scenegen.Camera(0, 64, 64, np.array([0, 0, 5], np.float32),
                          np.array([1, 0, 0], np.float32), np.array([0, 1, 0], np.float32),
                          np.array([0, 0, -1], np.float32), 100.0).pack()
    e = _single_eth([0.1, 0.2, 0.0], [1, 0, 0], [0, 1, 0], 0.03, 0.01)
    w = oracle.cross_section_widths(e, cam)
    assert w[0, 0] == pytest.approx(6.0, rel=1e-6)


def test_width_perspective_depth_scaling_and_near_plane():
    # perspective: the same ellipse at depth z spans 2a * pix / z pixels
    cam = scenegen.Camera(1, 64, 64, np.array([0, 0, 0], np.float32),
                          np.array([1, 0, 0], np.float32), np.array([0, 1, 0], np.float32),
                          np.array([0, 0, -1], np.float32), 500.0).pack()
    for z in (2.0, 4.0, 8.0):
        e = _single_eth([0.0, 0.0, -z], [1, 0, 0], [0, 1, 0], 0.01, 0.004)
        assert oracle.cross_section_widths(e, cam)[0, 0] == pytest.approx(2 * 0.01 * 500 / z,
                                                                          rel=1e-6)
    # edge-on (major axis along the view direction): only b shows
    e = _single_eth([0.0, 0.0, -4.0], [0, 0, 1], [0, 1, 0], 0.01, 0.004)
    wv = oracle.cross_section_widths(e, cam)[0, 0]
    assert wv == pytest.approx(2 * 0.004 * 500 / 4.0, rel=1e-2)
    # behind the camera -> +inf
    e = _single_eth([0.0, 0.0, 1.0], [1, 0, 0], [0, 1, 0], 0.01, 0.004)
    assert np.isinf(oracle.cross_section_widths(e, cam)[0, 0])


def test_coarser_levels_are_wider_on_average():
    w = scenegen.clustered(n=2000, S=8, res=256, spp=1, n_clusters=32)
    h = oracle.build_hierarchy(w.scene.verts[:, 0, :3], 32)
    eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h)
    wcl = oracle.cluster_level_widths(h, eth, w.camera.pack())
    assert h.n_levels == 3
    assert np.all(np.diff(wcl.mean(0)) < 0)


def test_cluster_level_widths_hand_worked():
    # Two clusters with two levels; every thick hair has one cross-section
    # facing an orthographic camera at 100 px per unit, so its width is
    # 2 max(a, b) * 100 px.  w[c, L] is the largest width among cluster c's
    # level-L thick hairs.
    cam = scenegen.Camera(0, 64, 64, np.array([0, 0, 5], np.float32),
                          np.array([1, 0, 0], np.float32), np.array([0, 1, 0], np.float32),
                          np.array([0, 0, -1], np.float32), 100.0).pack()
    a = np.array([0.03, 0.01, 0.005, 0.02, 0.004, 0.007])
    cl = np.array([0, 1, 0, 0, 1, 1])
    lv = np.array([0, 0, 1, 1, 1, 1])
    E = len(a)
    z = np.zeros((E, 1, 3))
    e1 = z + [1.0, 0, 0]
    e2 = z + [0, 1.0, 0]
    eth = oracle.ETHs(center=z.copy(), tangent=z + [0, 0, 1.0], e1=e1, e2=e2, a=a[:, None],
                      b=0.5 * a[:, None], seg_e1=None, seg_a=None, seg_b=None, ntot=None,
                      radius=None, mat=None)
    h = oracle.Hierarchy(0, 2, 2, None, None, None, None, None, None, np.ones(E, np.int64), cl, lv)
    w = oracle.cluster_level_widths(h, eth, cam)
    assert np.allclose(w, [[6.0, 4.0], [2.0, 1.4]], rtol=1e-6)


def test_deferred_rule_with_hysteresis_hand_worked():
    # eps = 2 px: refine above 2.2 px, coarsen at or below 1.8 px
    w = np.array([[5.0, 2.1, 1.0],    # L=1, w_cur 2.1: over eps but inside the band -> stay 1
                  [5.0, 2.3, 1.0],    # L=1, w_cur 2.3 > 2.2 -> 2
                  [5.0, 1.9, 1.0],    # L=2, w_cur- 1.9 > 1.8 -> stay 2
                  [5.0, 1.8, 1.0],    # L=2, w_cur- 1.8 <= 1.8 -> 1
                  [3.0, 1.5, 0.7],    # L=3 (strands), w_cur- 0.7 <= 1.8 -> 2
                  [2.15, 1.0, 0.5]],  # L=0, w_cur 2.15 inside the band, w_cur- = inf -> stay 0
                 np.float32)
    prev = np.array([1, 1, 2, 2, 3, 0], np.uint8)
    out = oracle.select_lod_deferred(w, prev, 2.0, 3, hysteresis=True)
    assert out.tolist() == [1, 2, 2, 1, 2, 0]
    # without the band the first and last rows refine, the third coarsens
    assert oracle.select_lod_deferred(w, prev, 2.0, 3).tolist() == [2, 2, 1, 1, 2, 1]
