"""The paper's guide-driven hierarchy and skinning (Section 5.1 steps 1, 2
and 4; Section 5.2) on the GPU against the oracle: guides, clusters and
Morton order bit for bit, the thick-hair fits, renders, and the skinned
strands and thick hairs after the guides move."""
import numpy as np
import pytest

import oracle
import paper_2405_10565_gb300 as hr
import scenegen
from gpu_util import (HIT_AGREE_MIN, KBUF_AGREE_MIN, RMSE_FP32, compare, desc_of, gpu_samples,
                      upload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_10565_gb300.build import build
    build()
    c = hr.hr_create(0)
    yield c
    hr.hr_destroy(c)


def _guided(ctx, w, G, iters):
    a = upload(ctx, w.scene)
    N = w.scene.n_strands
    cl = np.zeros(N, np.uint32)
    order = np.zeros(N, np.uint32)
    hr.hr_build_guided_clusters(ctx, a, G, iters, 0, cl, order)
    return a, cl, order


@pytest.mark.parametrize("n,S,G,iters", [(600, 8, 12, 3), (3000, 12, 32, 6), (20000, 16, 128, 5)])
def test_guided_hierarchy_bit_exact(ctx, n, S, G, iters):
    w = scenegen.full_head(n=n, S=S, width=32, height=32, spp=1, n_lights=2, n_clusters=64,
                           seed=n)
    a, cl, order = _guided(ctx, w, G, iters)
    try:
        h, guides, tri = oracle.build_guided_hierarchy(w.scene.verts, G, iters)
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        assert (C, L, E) == (h.n_clusters, h.n_levels, h.n_eths)
        g_gpu = np.zeros(G, np.int32)
        t_gpu = np.zeros((C, 3), np.uint32)
        hr.hr_guides_export(ctx, a, g_gpu, t_gpu)
        assert np.array_equal(g_gpu.astype(np.int64), guides)
        assert np.array_equal(order.astype(np.int64), h.order)
        assert np.array_equal(cl, h.cluster_of)
        first_of = np.searchsorted(h.cluster_of[h.order], np.arange(C))
        assert np.array_equal(t_gpu.astype(np.int64), tri[h.order[first_of]])
        counts = np.zeros(E, np.uint32)
        hr.hr_eth_export(ctx, a, counts=counts)
        assert np.array_equal(counts.astype(np.int64), h.eth_count)
        print(f"N {n}: {C} clusters from {int((guides >= 0).sum())} guides, {L} levels, "
              f"{int((h.eth_count == 0).sum())} empty thick hairs")
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_guided_fit_and_render(ctx):
    w = scenegen.full_head(n=6000, S=16, width=96, height=64, spp=2, n_lights=4, n_clusters=64,
                           fill=0.25)
    G, iters = 48, 5
    a, cl, order = _guided(ctx, w, G, iters)
    try:
        h, guides, tri = oracle.build_guided_hierarchy(w.scene.verts, G, iters)
        eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h)
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        xs = np.zeros((E, w.scene.n_segments + 1, 12), np.float32)
        hr.hr_eth_export(ctx, a, xsec=xs)
        live = h.eth_count > 0
        assert np.allclose(xs[live][..., 0:3], eth.center[live], atol=2e-7)
        d1 = np.abs(np.sum(xs[live][..., 4:7].astype(np.float64) * eth.e1[live], -1))
        good = d1 > 1 - 1e-5
        assert good.mean() > 0.999
        assert np.all(np.abs(xs[live][..., 3] / eth.a[live] - 1)[good] < 1e-4)
        assert np.all(xs[~live] == 0)
        # renders at the selected LoD and with every cluster on its finest thick hairs
        for lod in (None, np.full(C, L - 1, np.uint8)):
            if lod is None:
                lod = np.zeros(C, np.uint8)
                hr.hr_select_lod(ctx, a, w.camera.pack(), w.eps_w, 0, 0, lod)
            hr.hr_build_bvh(ctx, a, lod)
            prep = _prep_from(w.scene, h, eth, lod)
            sids = np.arange(w.camera.width * w.camera.height * w.spp)
            rg, hg = gpu_samples(ctx, a, desc_of(w), sids)
            ro, ho = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp,
                                           w.k_depth, w.sample_seed)
            frac, full, r, _ = compare(rg, hg, ro, ho)
            print(f"guided render, levels {np.bincount(lod, minlength=L + 1).tolist()}: "
                  f"agreement {frac:.5f} {full:.5f}, rel-RMSE {r:.2e}")
            assert frac >= HIT_AGREE_MIN and full >= KBUF_AGREE_MIN and r <= RMSE_FP32
            assert (ho[:, 0] >= 0).any()
    finally:
        hr.hr_asset_destroy(ctx, a)


def _prep_from(scene, h, eth, lod, verts=None):
    """Oracle rows of the active set of a given hierarchy and thick hairs."""
    N, S = scene.n_strands, scene.n_segments
    v = scene.verts if verts is None else verts
    st, eh = oracle.active_set(N, S, h, lod)
    r1, i1 = oracle.strand_prim_rows(v, scene.shape, st)
    r2, i2 = oracle.eth_prim_rows(eth, eh, N, S)
    return oracle.Prepared(np.ascontiguousarray(np.concatenate([r1, r2])),
                           np.ascontiguousarray(np.concatenate([i1, i2]).astype(np.int64)),
                           np.ascontiguousarray(np.concatenate([scene.mat.astype(np.float64),
                                                                eth.mat])), h, eth, lod)


def _bent(P, amp):
    """A smooth bend of vertex positions growing along the strand, plus a
    rigid turn: a new pose of the guides."""
    P = np.array(P, np.float64)
    s = np.linspace(0, 1, P.shape[-2])[None, :, None]
    P[..., 0:1] += amp * s ** 2
    P[..., 2:3] += 0.5 * amp * np.sin(3 * s)
    c, sn = np.cos(0.1), np.sin(0.1)
    R = np.array([[c, 0, sn], [0, 1, 0], [-sn, 0, c]])
    return P @ R.T


def test_skinning_against_the_oracle(ctx):
    w = scenegen.full_head(n=6000, S=16, width=96, height=64, spp=2, n_lights=4, n_clusters=64,
                           fill=0.25)
    G, iters = 48, 5
    S1 = w.scene.n_segments + 1
    a, cl, order = _guided(ctx, w, G, iters)
    try:
        h, guides, tri = oracle.build_guided_hierarchy(w.scene.verts, G, iters)
        eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h)
        rest = w.scene.verts[..., :3].astype(np.float64)
        valid = guides >= 0
        gv_rest = np.zeros((G, S1, 4), np.float32)
        gv_rest[valid, :, :3] = rest[guides[valid]]
        # the rest pose moves nothing
        hr.hr_asset_skin(ctx, a, gv_rest)
        v = np.zeros_like(w.scene.verts)
        hr.hr_vertex_export(ctx, a, v)
        assert np.allclose(v, w.scene.verts, atol=2e-6)
        # a new pose of the guides
        gnew = _bent(rest[np.maximum(guides, 0)], 0.05)
        gv = np.zeros((G, S1, 4), np.float32)
        gv[:, :, :3] = gnew
        hr.hr_asset_skin(ctx, a, gv)
        hr.hr_vertex_export(ctx, a, v)
        t3 = tri  # per strand
        g = [gnew[t3[:, j]] for j in range(3)]
        grest = [rest[guides[t3[:, j]]] for j in range(3)]
        wts = oracle.prism_weights(rest, grest[0], grest[1], grest[2])
        want = oracle.skin_points(wts, g[0].astype(np.float32), g[1].astype(np.float32),
                                  g[2].astype(np.float32))
        err = np.abs(v[..., :3] - want).max()
        print(f"skinned strand vertices: max abs error {err:.2e}")
        assert err < 2e-5
        assert np.abs(v[..., :3] - rest).max() > 0.02  # they did move
        # thick hairs: centres and corners carried by the cluster's guides
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        xs = np.zeros((E, S1, 12), np.float32)
        hr.hr_eth_export(ctx, a, xsec=xs)
        live = h.eth_count > 0
        ctri = tri[h.order[np.searchsorted(h.cluster_of[h.order], h.eth_cluster)]]
        ae, be = eth.a[..., None] * eth.e1, eth.b[..., None] * eth.e2
        pts = [eth.center, eth.center + ae, eth.center - ae, eth.center + be, eth.center - be]
        gr = [rest[guides[ctri[:, j]]] for j in range(3)]
        gn = [gnew[ctri[:, j]].astype(np.float32) for j in range(3)]
        sk = [oracle.skin_points(oracle.prism_weights(p, gr[0], gr[1], gr[2]), gn[0], gn[1], gn[2])
              for p in pts]
        assert np.abs(xs[live][..., 0:3] - sk[0][live]).max() < 2e-5
        a_new = 0.5 * np.linalg.norm(sk[1] - sk[2], axis=-1)
        b_new = 0.5 * np.linalg.norm(sk[3] - sk[4], axis=-1)
        assert np.allclose(xs[live][..., 3], a_new[live], rtol=1e-4, atol=1e-6)
        assert np.allclose(xs[live][..., 7], b_new[live], rtol=1e-4, atol=1e-6)
        # a frame of the skinned hair (the hierarchy kept) against the oracle's
        # render of the oracle-skinned geometry at the same LoD
        d = desc_of(w, flags=hr.HR_FLAG_KEEP_HIERARCHY)
        img = np.zeros((w.camera.height, w.camera.width, 3), np.float32)
        hr.hr_render_frame(ctx, a, 0, w.eps_w, 0, d, img)
        lod = np.zeros(C, np.uint8)
        hr.hr_select_lod(ctx, a, w.camera.pack(), w.eps_w, 0, 0, lod)
        hr.hr_build_bvh(ctx, a, lod)
        sids = np.arange(w.camera.width * w.camera.height * w.spp)
        rg, hg = gpu_samples(ctx, a, desc_of(w), sids)
        vs = np.array(w.scene.verts)
        vs[..., :3] = want  # the oracle's own skinned strands
        eth_s = _skinned_eths(eth, h, sk)
        prep = _prep_from(w.scene, h, eth_s, lod, verts=vs)
        ro, ho = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, w.k_depth,
                                       w.sample_seed)
        frac, full, r, _ = compare(rg, hg, ro, ho)
        print(f"skinned render: agreement {frac:.5f} {full:.5f}, rel-RMSE {r:.2e}")
        assert frac >= HIT_AGREE_MIN and full >= KBUF_AGREE_MIN and r <= RMSE_FP32
        mean = rg.reshape(-1, w.spp, 3).astype(np.float64).mean(1).reshape(img.shape)
        assert np.allclose(img, mean, rtol=1e-5, atol=1e-7)
    finally:
        hr.hr_asset_destroy(ctx, a)


def _skinned_eths(eth, h, sk):
    """The oracle's thick hairs after skinning: centres, a / e1 and b from the
    skinned centre and corners, the segment frame as in the fit."""
    import copy
    e = copy.deepcopy(eth)
    live = h.eth_count > 0
    c = sk[0]
    u = sk[1] - sk[2]
    a = 0.5 * np.linalg.norm(u, axis=-1)
    with np.errstate(invalid="ignore", divide="ignore"):
        e1 = u / (2 * a[..., None])
    e.center = np.where(live[:, None, None], c, 0)
    e.e1 = np.where(live[:, None, None], e1, 0)
    e.a = np.where(live[:, None], a, 0)
    e.b = np.where(live[:, None], 0.5 * np.linalg.norm(sk[3] - sk[4], axis=-1), 0)
    with np.errstate(invalid="ignore", divide="ignore"):
        ax = e.center[:, 1:] - e.center[:, :-1]
        ax = ax / np.linalg.norm(ax, axis=-1, keepdims=True)
        vv = e.e1[:, :-1] - np.sum(e.e1[:, :-1] * ax, -1, keepdims=True) * ax
        e.seg_e1 = vv / np.linalg.norm(vv, axis=-1, keepdims=True)
    e.seg_e1[~live] = 0
    e.seg_a = np.maximum(e.a[:, :-1], e.a[:, 1:])
    e.seg_b = np.maximum(e.b[:, :-1], e.b[:, 1:])
    return e
