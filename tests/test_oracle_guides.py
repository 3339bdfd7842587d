"""Pins of the oracle's guide hairs, guide-driven hierarchy and skinning
(Section 5.1 steps 1, 2 and 4; Section 5.2).

Against things fixed outside the oracle: D in FP64 and a hand-worked FP32
rounding case that fixes the summation order; k-means on bundles so far apart
that any correct clustering finds them; medoids and nearest guides by FP64
brute force; the triangle-prism weights of hand-placed points and their
invariance under rigid motion of the guides.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


# ---------------------------------------------------------------- distance


def test_strand_distance_against_fp64():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(50, 9, 3)).astype(np.float32)
    B = rng.normal(size=(9, 3)).astype(np.float32)
    want = np.sum((A.astype(np.float64) - B.astype(np.float64)) ** 2, (-1, -2))
    assert np.allclose(oracle.strand_distance(A, B), want, rtol=1e-5)


def test_strand_distance_order_is_sequential():
    # point 0 differs by 4096 along x (2^24), points 1-4 by (0.5, 0.5, 0)
    # (0.5 each).  Summed in vertex order in FP32, every 0.5 is half an ulp of
    # 2^24 and rounds away (ties to even): D = 2^24 exactly, not the 2^24 + 2
    # of the exact sum or of the reverse order.
    A = np.zeros((5, 3), np.float32)
    B = np.zeros((5, 3), np.float32)
    B[0, 0] = 4096.0
    B[1:, 0] = 0.5
    B[1:, 1] = 0.5
    assert float(oracle.strand_distance(A, B)) == 2.0 ** 24


# ---------------------------------------------------------------- k-means and guides


def _bundles(centres, per, S=6, spread=0.01, seed=1):
    """Straight strands along +y in bundles around the given root centres."""
    rng = np.random.default_rng(seed)
    v = []
    for c in centres:
        for _ in range(per):
            root = np.asarray(c, np.float64) + rng.normal(size=3) * spread
            pts = root[None, :] + np.outer(np.arange(S + 1) * 0.1, [0.0, 1.0, 0.0])
            v.append(pts)
    out = np.zeros((len(v), S + 1, 4), np.float32)
    out[..., :3] = np.asarray(v)
    out[..., 3] = 1e-3
    return out


def test_kmeans_two_separated_bundles():
    v = _bundles([(0, 0, 0), (5, 0, 0), (0, 0, 5), (5, 0, 5)], 12)
    a, cent, guides = oracle.guide_kmeans(v, 4, 5)
    truth = np.repeat(np.arange(4), 12)
    # the same partition as the bundles (labels may be permuted)
    for g in range(4):
        assert len(set(truth[a == g])) == 1
    assert len(set(a.tolist())) == 4
    # every guide belongs to its cluster
    for g in range(4):
        assert a[guides[g]] == g


def test_kmeans_assignment_is_nearest_centroid():
    w = scenegen.clustered(n=600, S=8, res=16, spp=1, n_clusters=8)
    a, cent, guides = oracle.guide_kmeans(w.scene.verts, 12, 4)
    P = w.scene.verts[..., :3].astype(np.float64)
    D = np.sum((P[:, None] - cent[None].astype(np.float64)) ** 2, (-1, -2))
    best = D.min(1)
    # FP32 sums: within rounding of the FP64 minimum
    assert np.all(D[np.arange(len(a)), a] <= best * (1 + 1e-5))


def test_medoid_is_the_brute_force_minimiser():
    w = scenegen.clustered(n=400, S=8, res=16, spp=1, n_clusters=8)
    a, cent, guides = oracle.guide_kmeans(w.scene.verts, 6, 3)
    P = w.scene.verts[..., :3].astype(np.float64)
    for g in range(6):
        mem = np.nonzero(a == g)[0]
        if mem.size == 0:
            assert guides[g] == -1
            continue
        D = np.sum((P[mem][:, None] - P[mem][None]) ** 2, (-1, -2))
        s = D.sum(1)
        order = np.argsort(s)
        if mem.size > 1 and s[order[1]] - s[order[0]] < 1e-5 * s[order[0]]:
            continue  # a near tie: FP32 and FP64 may pick either
        assert guides[g] == mem[order[0]]


def test_nearest_guides_brute_force():
    w = scenegen.clustered(n=500, S=8, res=16, spp=1, n_clusters=8)
    P = w.scene.verts[..., :3].astype(np.float64)
    guides = np.array([3, 40, -1, 77, 150, 222, 301, 480])
    tri = oracle.nearest_guides(w.scene.verts, guides)
    valid = np.nonzero(guides >= 0)[0]
    D = np.sum((P[:, None] - P[guides[valid]][None]) ** 2, (-1, -2))
    for i in range(P.shape[0]):
        o = np.argsort(D[i])
        if D[i, o[3]] - D[i, o[2]] < 1e-5 * D[i, o[2]] + 1e-12:
            continue
        assert tri[i].tolist() == sorted(valid[o[:3]].tolist())
    # a guide's nearest guide is itself
    for g in valid:
        assert g in tri[guides[g]]


def test_guided_clusters_share_their_triple():
    w = scenegen.full_head(n=3000, S=12, width=32, height=32, spp=1, n_clusters=64)
    h, guides, tri = oracle.build_guided_hierarchy(w.scene.verts, 24, 4)
    key = (tri[:, 0] << 20) | (tri[:, 1] << 10) | tri[:, 2]
    # strands of one cluster share one triple; triples of clusters differ and rise
    keys_of_cluster = [np.unique(key[h.cluster_of == c]) for c in range(h.n_clusters)]
    assert all(k.size == 1 for k in keys_of_cluster)
    ks = np.array([k[0] for k in keys_of_cluster])
    assert np.all(np.diff(ks) > 0)
    # strands within a cluster in Morton order of their roots
    code = h.code[h.order]
    cl = h.cluster_of[h.order]
    same = cl[1:] == cl[:-1]
    assert np.all(code[1:][same] >= code[:-1][same])
    assert h.n_clusters >= 24


def test_guided_hierarchy_levels_and_empty_buckets():
    w = scenegen.full_head(n=3000, S=8, width=48, height=32, spp=2, n_lights=2, n_clusters=64)
    h, guides, tri = oracle.build_guided_hierarchy(w.scene.verts, 32, 4)
    N = w.scene.n_strands
    sizes = np.bincount(h.cluster_of, minlength=h.n_clusters)
    assert h.n_levels >= 2
    for k in range(h.n_levels):
        sel = h.eth_level == k
        assert h.eth_count[sel].sum() == N
        # empty buckets exactly in clusters smaller than 4^k
        cnt = h.eth_count[sel].reshape(h.n_clusters, 4 ** k)
        assert np.array_equal((cnt == 0).sum(1), np.maximum(0, 4 ** k - sizes))
    # the fit leaves empty thick hairs out, the active set too, and the render
    # stays finite
    eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h)
    empty = h.eth_count == 0
    assert np.all(eth.a[empty] == 0) and np.all(np.isfinite(eth.seg_a))
    lod = np.full(h.n_clusters, h.n_levels - 1, np.uint8)
    st, eh = oracle.active_set(N, 8, h, lod)
    assert np.all(h.eth_count[eh] > 0)
    assert eh.size == int(np.minimum(sizes, 4 ** (h.n_levels - 1)).sum())


# ---------------------------------------------------------------- skinning


def test_prism_weights_affine_in_plane():
    # triangle (0,0,0), (1,0,0), (0,1,0): a point (u, v, z) has w1 = u, w2 = v, h = z
    g0, g1, g2 = np.zeros(3), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    p = np.array([[0.2, 0.3, 0.5], [1.5, -0.25, -0.1], [0.0, 0.0, 0.0]])
    wts = oracle.prism_weights(p, g0, g1, g2)
    assert np.allclose(wts[:, :3], p, atol=1e-15) and np.all(wts[:, 3] == 0)
    # scaled and sheared guides move the in-plane part affinely
    q0, q1, q2 = np.array([1.0, 2, 3]), np.array([3.0, 2, 3]), np.array([2.0, 5, 3])
    s = oracle.skin_points(wts, q0, q1, q2)
    n = np.array([0.0, 0.0, 1.0])
    want = q0 + p[:, :1] * (q1 - q0) + p[:, 1:2] * (q2 - q0) + p[:, 2:3] * n
    assert np.allclose(s, want, atol=1e-14)


def test_prism_weights_rest_pose_and_rigid_motion():
    rng = np.random.default_rng(3)
    g = rng.normal(size=(3, 200, 3))
    p = rng.normal(size=(200, 3))
    wts = oracle.prism_weights(p, g[0], g[1], g[2])
    assert np.allclose(oracle.skin_points(wts, g[0], g[1], g[2]), p, atol=1e-12)
    R, t = _rot(5), np.array([0.3, -1.0, 2.0])
    moved = [gi @ R.T + t for gi in g]
    assert np.allclose(oracle.skin_points(wts, *moved), p @ R.T + t, atol=1e-11)
    # collinear guides: the point keeps its offset from the first guide
    c0, c1, c2 = np.zeros(3), np.array([1.0, 0, 0]), np.array([2.0, 0, 0])
    wd = oracle.prism_weights(np.array([[0.1, 0.2, 0.3]]), c0, c1, c2)
    assert wd[0, 3] == 1
    assert np.allclose(oracle.skin_points(wd, c0 + 1, c1 + 1, c2 + 1), [[1.1, 1.2, 1.3]])
