"""Pins of the oracle's Marschner R / TT / TRT single fibre and its aggregate
(Section 7, "Extending to Marschner model with TRT term"; Marschner et al.
2003 for the lobes).

With FLAG_TRT the third lobe is TRT instead of D: A_TRT G(2 beta_R, theta_h)
/ 2 pi.  The pins: hand values of the single fibre, the separable albedos
against the direct 2-D integral of the fibre, the furnace bound over the
parameter box, the n = 1 reduction and reciprocity of the aggregate, and the
thick-hair image converging toward the strand image with the TRT fibre.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen

PI = math.pi
TRT = oracle.FLAG_TRT


def g(beta, x):
    return math.exp(-x * x / (2 * beta * beta)) / (math.sqrt(2 * PI) * beta)


DARK = scenegen.material_marschner(np.array([0.9]), np.array([0.1]))[0].astype(np.float64)
BROWN = scenegen.material_marschner(np.array([0.5]), np.array([0.2]))[0].astype(np.float64)
LIGHT = scenegen.material_marschner(np.array([0.1]), np.array([0.3]))[0].astype(np.float64)


def test_trt_single_fibre_hand_values():
    m = BROWN
    bR, bT, gT = m[9], m[10], m[11]
    # theta_i = theta_o = 0, phi = pi: every Gaussian at its peak
    f = oracle.f_single(m, 0.0, 0.0, -1.0, flags=TRT)
    for c in range(3):
        want = (m[c] * g(bR, 0) / (2 * PI) + m[3 + c] * g(bT, 0) * g(gT, 0)
                + m[6 + c] * g(2 * bR, 0) / (2 * PI))
        assert f[c] == pytest.approx(want, rel=1e-14)
    # theta_h = 0.25, phi = pi / 3
    th_i, th_o = 0.6, -0.1
    f = oracle.f_single(m, th_i, th_o, 0.5, flags=TRT)
    for c in range(3):
        want = (m[c] * g(bR, 0.25) / (2 * PI) + m[3 + c] * g(bT, 0.25) * g(gT, PI / 3 - PI)
                + m[6 + c] * g(2 * bR, 0.25) / (2 * PI))
        assert f[c] == pytest.approx(want, rel=1e-12)
    # without the flag the third lobe is the diffuse one
    f0 = oracle.f_single(m, th_i, th_o, 0.5)
    assert not np.allclose(f, f0)


@pytest.mark.parametrize("mat", [DARK, BROWN, LIGHT])
@pytest.mark.parametrize("theta_d", [0.0, 0.7, -1.9, 2.8])
def test_trt_separable_albedo_equals_2d_quadrature(mat, theta_d):
    aF, aB, s2 = oracle.albedo(mat, theta_d, flags=TRT)
    fr, bk = oracle.albedo_2d(mat, abs(theta_d) / 2, nq=300, flags=TRT)
    assert np.allclose(aF, fr, rtol=1e-9)
    assert np.allclose(aB, bk, rtol=1e-9)
    # the forward spread is a mean of beta_R^2, beta_TT^2 and (2 beta_R)^2
    lo = min(mat[9], mat[10]) ** 2
    hi = max(2 * mat[9], mat[10]) ** 2
    assert lo <= s2 <= hi


def test_trt_furnace_over_parameter_box():
    for mel in (0.1, 0.5, 0.9):
        for rough in (0.1, 0.2, 0.3):
            m = scenegen.material_marschner(np.array([mel]), np.array([rough]))[0].astype(np.float64)
            for th in np.linspace(-3.1, 3.1, 13):
                aF, aB, _ = oracle.albedo(m, th, flags=TRT)
                assert np.all(aF + aB < 1.0) and np.all(aF < 0.7) and np.all(aB > 0)


@pytest.mark.parametrize("mat", [DARK, BROWN])
def test_trt_aggregate_reduces_to_single_and_is_reciprocal(mat):
    rng = np.random.default_rng(8)
    for _ in range(30):
        th_i, th_o = rng.uniform(-1.4, 1.4, 2)
        cp = rng.uniform(-1, 1)
        # n = 1 in the front hemisphere: no B lobe, no S, the single fibre
        assert np.allclose(oracle.f_ours(mat, th_i, th_o, -abs(cp), 0.3, 1.0, flags=TRT),
                           oracle.f_single(mat, th_i, th_o, -abs(cp), flags=TRT), rtol=1e-12)
        for rho, n in ((0.2, 1.0), (0.6, 4.5)):
            a = oracle.f_ours(mat, th_i, th_o, cp, rho, n, flags=TRT)
            b = oracle.f_ours(mat, th_o, th_i, cp, rho, n, flags=TRT)
            assert np.allclose(a, b, rtol=1e-12, atol=0)


def test_trt_thick_hair_image_converges_to_the_strand_image():
    w = scenegen.clustered(n=2000, S=8, res=48, spp=4, lod_setting="strands", n_clusters=8)
    N = w.scene.n_strands
    mel = 0.7 + 0.2 * scenegen.Stream(4, 1).uniform(N)
    sc = scenegen.Scene(w.scene.verts, scenegen.material_marschner(mel, np.full(N, 0.15)),
                        w.scene.shape)
    h = oracle.build_hierarchy(sc.verts[:, 0, :3], w.n_clusters)
    sids = np.arange(48 * 48 * 4)
    imgs = []
    for lv in list(range(h.n_levels)) + [h.n_levels]:
        prep = oracle.prepare(sc, w.n_clusters, lod=np.full(w.n_clusters, lv, np.uint8))
        rad, _ = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, 4, 64,
                                       w.sample_seed, flags=TRT)
        imgs.append(rad.reshape(-1, 4, 3).mean(1))
    err = [float(np.linalg.norm(im - imgs[-1]) / np.linalg.norm(imgs[-1])) for im in imgs[:-1]]
    print(f"TRT: rel-RMSE against the strand image per level {[round(e, 3) for e in err]}")
    assert all(b < a for a, b in zip(err, err[1:])), err
