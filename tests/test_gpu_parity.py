"""CUDA path against the oracle, through the C ABI, on seeded inputs.

Integer outputs (Morton order, clusters, LoD levels, active primitive set) are
compared bit-exactly; the FP64 thick-hair fit to FP32 rounding; radiance per
sample within the stated tolerance (relative RMSE 1e-3 in FP32, 5e-3 with
FP16 tables) over samples whose nearest-hit id agrees, which must be at least
99.9% of the samples.
"""
import numpy as np
import pytest

import oracle
import paper_2405_10565_gb300 as hr
import scenegen
from gpu_util import (HIT_AGREE_MIN, KBUF_AGREE_MIN, RMSE_FP16, RMSE_FP32, compare, desc_of,
                      gpu_lod, gpu_samples, hair_pixels, oracle_prepare, upload)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2405_10565_gb300.build import build
    build()
    c = hr.hr_create(0)
    yield c
    hr.hr_destroy(c)


def _oracle_with_lod(w, lod, lod_g):
    """Oracle scene at the GPU's LoD.  When the LoD was selected, the oracle
    selects its own first and must agree bit for bit, except for clusters whose
    width sits within 1e-4 of epsilon_w (FP64-fit rounding may tip those)."""
    if not w.n_clusters:
        return oracle_prepare(w)
    if lod is None and w.lod_setting == "select":
        prep = oracle_prepare(w)
        if np.array_equal(prep.lod, lod_g):
            return prep
        wo = oracle.cluster_level_widths(prep.hier, prep.eth, w.camera.pack())
        near = np.any(np.abs(wo / np.float32(w.eps_w) - 1) < 1e-4, axis=1)
        assert np.array_equal(prep.lod[~near], lod_g[~near])
    return oracle_prepare(w, lod=lod_g)


def _render_check(ctx, w, sids, *, lod=None, precision=None, flags=0, k=None, tol=None):
    a = upload(ctx, w.scene)
    try:
        lod_g = gpu_lod(ctx, a, w, lod)
        prep = _oracle_with_lod(w, lod, lod_g)
        d = desc_of(w, precision=precision, flags=flags, k=k)
        rg, hg = gpu_samples(ctx, a, d, sids)
        ro, ho = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp,
                                       k or w.k_depth, w.sample_seed, flags=flags)
        frac, full, r_agree, r_all = compare(rg, hg, ro, ho)
        prec = w.precision if precision is None else precision
        bound = tol or (RMSE_FP16 if prec == 1 else RMSE_FP32)
        msg = (f"{w.name}: nearest-hit agreement {frac:.5f}, k-buffer agreement {full:.5f}, "
               f"rel-RMSE {r_agree:.2e} (all samples {r_all:.2e})")
        print(msg)
        assert frac >= HIT_AGREE_MIN, msg
        assert full >= KBUF_AGREE_MIN, msg
        assert r_agree <= bound, msg
        assert (hg[:, 0] >= 0).any(), "nothing hit: the test scene is not exercising the path"
        return rg, hg, ro, ho
    finally:
        hr.hr_asset_destroy(ctx, a)


# ---------------------------------------------------------------- hierarchy


@pytest.mark.parametrize("N,C", [(64, 4), (10000, 256), (100000, 4096), (777, 13)])
def test_morton_order_and_clusters_bit_exact(ctx, N, C):
    S = 4
    v = scenegen.make_strands(N, S, seed=N, curl_amp=0.02)
    sc = scenegen.Scene(v, scenegen.material_from_melanin(np.full(N, 0.5), np.full(N, 0.2)),
                        np.zeros((N, 2), np.float32))
    a = upload(ctx, sc)
    try:
        cl = np.zeros(N, np.uint32)
        order = np.zeros(N, np.uint32)
        hr.hr_build_clusters(ctx, a, C, 0, cl, order)
        h = oracle.build_hierarchy(v[:, 0, :3], C)
        assert np.array_equal(order.astype(np.int64), h.order)
        assert np.array_equal(cl, h.cluster_of)
        Cg, L, E = hr.hr_hierarchy_info(ctx, a)
        assert (Cg, L, E) == (C, h.n_levels, h.n_eths)
        if E:
            counts = np.zeros(E, np.uint32)
            hr.hr_eth_export(ctx, a, counts=counts)
            assert np.array_equal(counts.astype(np.int64), h.eth_count)
    finally:
        hr.hr_asset_destroy(ctx, a)


@pytest.mark.parametrize("wl", ["clusters", "full_head_small"])
def test_thick_hair_fit_fp64(ctx, wl):
    if wl == "clusters":
        w = scenegen.clustered(n=3000, S=12, res=64, spp=1, n_clusters=64)
    else:
        w = scenegen.full_head(n=6000, S=16, width=64, height=48, spp=1, n_lights=2,
                               n_clusters=256)
    a = upload(ctx, w.scene)
    try:
        hr.hr_build_clusters(ctx, a, w.n_clusters)
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        S1 = w.scene.n_segments + 1
        xs = np.zeros((E, S1, 12), np.float32)
        mat = np.zeros((E, 12), np.float32)
        hr.hr_eth_export(ctx, a, xsec=xs, mat=mat)
        h = oracle.build_hierarchy(w.scene.verts[:, 0, :3], w.n_clusters)
        eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h)
        assert np.allclose(xs[..., 0:3], eth.center, rtol=0, atol=2e-7)
        assert np.allclose(mat, eth.mat, rtol=1e-6, atol=1e-7)
        d1 = np.abs(np.sum(xs[..., 4:7].astype(np.float64) * eth.e1, -1))
        good = d1 > 1 - 1e-5
        # a cross-section whose two kept eigenvalues (nearly) coincide has no
        # unique major axis: count those apart, they must be rare
        assert good.mean() > 0.999, good.mean()
        # the unit tangents are summed in FP32: on very elongated sections
        # (a/b ~ 100) their ~1e-7 error moves b by ~1e-5
        ra = np.abs(xs[..., 3] / eth.a - 1)[good]
        rb = np.abs(xs[..., 7] / eth.b - 1)[good]
        print(f"{wl}: semi-axis relative error max a {ra.max():.1e}, b {rb.max():.1e}, "
              f"median {np.median(ra):.1e}")
        assert ra.max() < 1e-4 and rb.max() < 1e-4
        same = (xs[..., 3] == eth.a.astype(np.float32)) & (xs[..., 7] == eth.b.astype(np.float32))
        print(f"{wl}: semi-axes bit-identical to the oracle's in {same.mean():.3f} of cross-sections")
    finally:
        hr.hr_asset_destroy(ctx, a)


# ---------------------------------------------------------------- LoD


@pytest.mark.parametrize("fill", [0.15, 0.3, 0.8])
def test_lod_widths_and_selection(ctx, fill):
    w = scenegen.full_head(n=20000, S=16, width=960, height=540, spp=1, n_lights=2,
                           n_clusters=1024, fill=fill)
    a = upload(ctx, w.scene)
    try:
        hr.hr_build_clusters(ctx, a, w.n_clusters)
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        cam = w.camera.pack()
        wg = np.zeros((C, L), np.float32)
        hr.hr_lod_widths(ctx, a, cam, wg)
        h = oracle.build_hierarchy(w.scene.verts[:, 0, :3], w.n_clusters)
        eth = oracle.fit_eths(w.scene.verts, w.scene.mat, h)
        wo = oracle.cluster_level_widths(h, eth, cam)
        exact = wg == wo
        assert np.allclose(wg, wo, rtol=1e-5)
        # integer decisions: identical wherever no width sits within 1e-4 of eps
        eps = np.float32(w.eps_w)
        near = np.any(np.abs(wo / eps - 1) < 1e-4, axis=1)
        lg = np.zeros(C, np.uint8)
        hr.hr_select_lod(ctx, a, cam, w.eps_w, 0, 0, lg)
        lo = oracle.select_lod_init(wo, w.eps_w, L)
        assert np.array_equal(lg[~near], lo[~near])
        # deferred rule (Eq. 14) from a seeded previous selection, and the budget bias
        prev = (np.arange(C) * 7 % (L + 1)).astype(np.uint8)
        ld = prev.copy()
        hr.hr_select_lod(ctx, a, cam, w.eps_w, 1, 0, ld)
        assert np.array_equal(ld[~near], oracle.select_lod_deferred(wo, prev, w.eps_w, L)[~near])
        lb = np.zeros(C, np.uint8)
        hr.hr_select_lod(ctx, a, cam, w.eps_w, 0, 1, lb)
        assert np.array_equal(lb[~near], oracle.apply_budget(lo, 1)[~near])
        # Eq. 14 with the hysteresis band (mode 2): thresholds 1.1 eps and 0.9 eps
        near_h = near | np.any(np.abs(wo / np.float32(1.1 * w.eps_w) - 1) < 1e-4, axis=1) | \
            np.any(np.abs(wo / np.float32(0.9 * w.eps_w) - 1) < 1e-4, axis=1)
        lh = prev.copy()
        hr.hr_select_lod(ctx, a, cam, w.eps_w, 2, 0, lh)
        want_h = oracle.select_lod_deferred(wo, prev, w.eps_w, L, hysteresis=True)
        assert np.array_equal(lh[~near_h], want_h[~near_h])
        print(f"fill {fill}: levels {np.bincount(lg, minlength=L + 1).tolist()}, near {near.sum()}, "
              f"widths bit-identical {exact.mean():.3f}")
    finally:
        hr.hr_asset_destroy(ctx, a)


# ---------------------------------------------------------------- active set / BVH


@pytest.mark.parametrize("setting", ["strands", "half", "eth"])
def test_active_set_bit_exact(ctx, setting):
    w = scenegen.clustered(n=4000, S=8, res=64, spp=1, lod_setting=setting, n_clusters=100)
    a = upload(ctx, w.scene)
    try:
        lod = gpu_lod(ctx, a, w)
        n = hr.hr_bvh_export(ctx, a)
        ids = np.zeros(n, np.uint32)
        hr.hr_bvh_export(ctx, a, ids)
        prep = oracle_prepare(w, lod=lod)
        assert np.array_equal(np.sort(ids.astype(np.int64)), np.sort(prep.ids))
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_active_counts_survive_a_growing_bvh(ctx):
    """The statistics' active and thick-hair primitive counts after a build that
    outgrows the previous BVH's storage (all thick hairs, then half the
    clusters on strands) equal the exported leaves."""
    w = scenegen.clustered(n=4000, S=8, res=32, spp=1, lod_setting="eth", n_clusters=100)
    a = upload(ctx, w.scene)
    try:
        hr.hr_build_clusters(ctx, a, w.n_clusters)
        C, L, _ = hr.hr_hierarchy_info(ctx, a)
        img = np.zeros((32, 32, 3), np.float32)
        d = desc_of(w)
        NS = w.scene.n_strands * w.scene.n_segments
        for setting in ("eth", "half"):
            hr.hr_build_bvh(ctx, a, np.ascontiguousarray(scenegen.lod_preset(setting, C, L)))
            n = hr.hr_bvh_export(ctx, a)
            ids = np.zeros(n, np.uint32)
            hr.hr_bvh_export(ctx, a, ids)
            st = hr.hr_render(ctx, a, d, img, stats=True)
            assert st.n_active_prims == n
            assert st.n_eth_prims == int((ids >= NS).sum()) > 0
            assert st.n_strand_prims == int((ids < NS).sum())
    finally:
        hr.hr_asset_destroy(ctx, a)


# ---------------------------------------------------------------- rendering


def test_tiny_strands_full_image(ctx):
    w = scenegen.tiny_strands()
    n = w.camera.width * w.camera.height * w.spp
    _render_check(ctx, w, np.arange(n))


@pytest.mark.parametrize("setting", ["strands", "half", "eth"])
def test_clustered_settings(ctx, setting):
    w = scenegen.clustered(n=3000, S=12, res=48, spp=4, lod_setting=setting, n_clusters=64)
    n = w.camera.width * w.camera.height * w.spp
    _render_check(ctx, w, np.arange(n))


def test_full_head_small_selected_lod(ctx):
    w = scenegen.full_head(n=8000, S=16, width=96, height=64, spp=2, n_lights=8,
                           n_clusters=320, fill=0.25)
    n = w.camera.width * w.camera.height * w.spp
    _render_check(ctx, w, np.arange(n))


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_kbuffer_depths_on_thick_hairs(ctx, k):
    w = scenegen.clustered(n=3000, S=12, res=40, spp=1, lod_setting="eth", n_clusters=64)
    n = w.camera.width * w.camera.height * w.spp
    _render_check(ctx, w, np.arange(n), k=k)


@pytest.mark.parametrize("flags", [hr.HR_FLAG_NO_S, hr.HR_FLAG_SINGLE_ON_ETH])
def test_ablation_flags(ctx, flags):
    w = scenegen.clustered(n=3000, S=12, res=40, spp=1, lod_setting="half", n_clusters=64)
    n = w.camera.width * w.camera.height * w.spp
    _render_check(ctx, w, np.arange(n), flags=flags)


def test_fp16_tables(ctx):
    w = scenegen.clustered(n=3000, S=12, res=48, spp=2, lod_setting="half", n_clusters=64)
    n = w.camera.width * w.camera.height * w.spp
    _render_check(ctx, w, np.arange(n), precision=1)


def test_ragged_image_odd_spp(ctx):
    # image not a multiple of the 16 x 8 tile, spp 3, K 3
    w = scenegen.clustered(n=2000, S=8, res=37, spp=3, lod_setting="half", n_clusters=50)
    w.camera.height = 23
    w.camera.pix_scale = w.camera.pix_scale * 23 / 37
    n = w.camera.width * w.camera.height * w.spp
    rg, hg, ro, ho = _render_check(ctx, w, np.arange(n), k=3)
    # the frame kernel's pixels are the means of the same per-sample values
    a = upload(ctx, w.scene)
    try:
        gpu_lod(ctx, a, w)
        d = desc_of(w, k=3)
        img = np.zeros((w.camera.height, w.camera.width, 3), np.float32)
        hr.hr_render(ctx, a, d, img)
        mean = rg.reshape(-1, w.spp, 3).astype(np.float64).mean(1).reshape(img.shape)
        assert np.allclose(img, mean, rtol=1e-5, atol=1e-7)
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_degenerate_scenes(ctx):
    # a single one-segment strand (a BVH of one leaf), two strands, and a
    # camera that sees nothing
    for n in (1, 2):
        v = scenegen.make_strands(n, 1, seed=3, head_radius=0.1, length=0.5, radius=0.05)
        sc = scenegen.Scene(v, scenegen.material_absorption(n, 0.3, 0.2),
                            np.zeros((n, 2), np.float32))
        lo, hi = sc.aabb()
        cam = scenegen.frame_camera(lo, hi, 24, 24, perspective=True, fill=0.6)
        w = scenegen.Workload("tiny", sc, cam, scenegen.directional_light((0, 1, 1)), 2, 2, 0)
        _render_check(ctx, w, np.arange(24 * 24 * 2))
    # looking away from the hair: every sample misses
    w = scenegen.tiny_strands()
    w.camera.fwd = -w.camera.fwd
    a = upload(ctx, w.scene)
    try:
        hr.hr_build_bvh(ctx, a, None)
        rg, hg = gpu_samples(ctx, a, desc_of(w), np.arange(128))
        assert np.all(hg == -1) and np.all(rg == 0)
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_device_pointer_inputs_and_outputs(ctx):
    torch = pytest.importorskip("torch")
    w = scenegen.clustered(n=2000, S=8, res=32, spp=2, lod_setting="half", n_clusters=50)
    dev = torch.device("cuda:0")
    v = torch.from_numpy(w.scene.verts).to(dev)
    m = torch.from_numpy(w.scene.mat).to(dev)
    s = torch.from_numpy(w.scene.shape).to(dev)
    a = hr.hr_asset_create(ctx, v, m, s)
    try:
        hr.hr_build_clusters(ctx, a, w.n_clusters)
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        lod = torch.from_numpy(scenegen.lod_preset("half", C, L)).to(dev)
        hr.hr_build_bvh(ctx, a, lod)
        d = desc_of(w)
        img_d = torch.zeros((32, 32, 3), device=dev)
        hr.hr_render(ctx, a, d, img_d)
        torch.cuda.synchronize()
        img_h = np.zeros((32, 32, 3), np.float32)
        hr.hr_render(ctx, a, d, img_h)
        assert np.array_equal(img_d.cpu().numpy(), img_h)
        assert img_h.max() > 0
    finally:
        hr.hr_asset_destroy(ctx, a)


def _full_size_sampled(ctx, w, pix, precision=None, min_hair=2000):
    """Every sample of the listed pixels through the sample kernel against the
    oracle (nearest-hit and k-buffer agreement, radiance bar of the table
    precision), and the frame kernel's pixel values there against the
    oracle's pixel means."""
    W, H, spp = w.camera.width, w.camera.height, w.spp
    prec = w.precision if precision is None else precision
    bar = RMSE_FP16 if prec == 1 else RMSE_FP32
    sids = scenegen.pixel_samples(W, spp, pix)
    a = upload(ctx, w.scene)
    try:
        lod_g = gpu_lod(ctx, a, w)
        prep = _oracle_with_lod(w, None, lod_g)
        L = int(lod_g.max()) if lod_g is not None else 0
        print(f"{w.name}: LoD levels {np.bincount(lod_g, minlength=L + 1).tolist()}, "
              f"active primitives {prep.rows.shape[0]}")
        d = desc_of(w, precision=prec)
        rg, hg = gpu_samples(ctx, a, d, sids)
        ro, ho = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, spp, w.k_depth,
                                       w.sample_seed)
        frac, full, r_agree, r_all = compare(rg, hg, ro, ho)
        on_hair = int((ho[:, 0] >= 0).sum())
        print(f"{w.name} {'fp16' if prec else 'fp32'} sampled: {len(sids)} samples, "
              f"{on_hair} on hair, nearest {frac:.5f} k-buffer {full:.5f} rmse {r_agree:.2e} "
              f"all {r_all:.2e}, eth hits {(ho[:, 0] >= w.scene.n_strands * w.scene.n_segments).mean():.3f}")
        assert frac >= HIT_AGREE_MIN and full >= KBUF_AGREE_MIN and r_agree <= bar
        assert on_hair >= min_hair, "sampled pixels must cover the hair"
        img = np.zeros((H, W, 3), np.float32)
        hr.hr_render(ctx, a, d, img)
        got = img.reshape(-1, 3)[pix]
        want = ro.reshape(-1, spp, 3).mean(1)
        agree_px = (hg.reshape(-1, spp * w.k_depth) == ho.reshape(-1, spp * w.k_depth)).all(1)
        num = np.linalg.norm((got - want)[agree_px])
        assert num <= bar * np.linalg.norm(want[agree_px]) + 1e-12
        return r_agree
    finally:
        hr.hr_asset_destroy(ctx, a)


@pytest.mark.parametrize("precision", [0, 1])
def test_full_head_full_size_sampled(ctx, precision):
    """The bench workload (100k strands x 64 segments, 1920x1080, 8 spp, 8
    lights, LoD selected over 4096 clusters), with FP32 and with FP16 tables,
    on sampled pixels: every sample of 16 seeded pixels anywhere, 48 inside
    the hair's screen box, one 8x8 tile at the centre and 256 pixels that
    contain a projected hair vertex (over 2,000 samples on hair), through the
    sample kernel, and the frame kernel's values at those pixels."""
    w = scenegen.full_head()
    W, H = w.camera.width, w.camera.height
    st = scenegen.Stream(7, 99)
    pix = list((st.u64(16) % np.uint64(W * H)).astype(np.int64))
    half = int(0.09 * H)
    xs = (W // 2 - half + (st.u64(48) % np.uint64(2 * half))).astype(np.int64)
    ys = (H // 2 - half + (st.u64(48) % np.uint64(2 * half))).astype(np.int64)
    pix += list(ys * W + xs)
    x0, y0 = W // 2 - 4, H // 2 - 4
    pix += [(y0 + j) * W + x0 + i for j in range(8) for i in range(8)]
    pix += list(hair_pixels(w, 256, 1 + precision))
    _full_size_sampled(ctx, w, np.unique(np.asarray(pix, np.int64)), precision)


def test_full_head_close_view_sampled(ctx):
    """The full head in the close view (hair 90% of the frame height, every
    cluster on strands: 6.4M active segments), 160 hair pixels x 8 spp."""
    w = scenegen.full_head(fill=0.9)
    _full_size_sampled(ctx, w, hair_pixels(w, 160, 4), min_hair=1000)


def _sampled_pixels(W, H, n_any, n_center, half_frac, seed):
    st = scenegen.Stream(seed, 99)
    pix = list((st.u64(n_any) % np.uint64(W * H)).astype(np.int64))
    half = max(1, int(half_frac * H))
    xs = (W // 2 - half + (st.u64(n_center) % np.uint64(2 * half))).astype(np.int64)
    ys = (H // 2 - half + (st.u64(n_center) % np.uint64(2 * half))).astype(np.int64)
    pix += list(ys * W + xs)
    return np.unique(np.asarray(pix, np.int64))


@pytest.mark.parametrize("setting", ["strands", "half", "eth"])
def test_clustered_full_size_sampled(ctx, setting):
    """The clustered workload at its full size (10,000 strands x 32 segments,
    256 clusters, 512x512, 4 spp, 2 lights, K = 4) in each LoD setting, on
    every sample of 256 seeded pixels."""
    w = scenegen.clustered(lod_setting=setting)
    W, H = w.camera.width, w.camera.height
    pix = _sampled_pixels(W, H, 64, 192, 0.3, 5)
    sids = scenegen.pixel_samples(W, w.spp, pix)
    rg, hg, ro, ho = _render_check(ctx, w, sids)
    assert (ho[:, 0] >= 0).mean() > 0.2


def test_stress_sampled(ctx):
    """The stress workload (500,000 long straight strands x 64 segments,
    16,384 clusters, eccentricity 0.9, 3840x2160, 16 spp, 4 lights, K = 8, FP16
    tables, LoD selected) on every sample of 12 seeded pixels in the centre
    and 128 pixels that contain a projected hair vertex (over 2,000 samples on
    hair): the oracle runs brute force over 28.5M primitives per sample."""
    w = scenegen.stress()
    W, H = w.camera.width, w.camera.height
    pix = np.unique(np.concatenate([_sampled_pixels(W, H, 0, 12, 0.2, 6), hair_pixels(w, 128, 6)]))
    sids = scenegen.pixel_samples(W, w.spp, pix)
    rg, hg, ro, ho = _render_check(ctx, w, sids)
    on_hair = int((ho[:, 0] >= 0).sum())
    print(f"stress: {len(sids)} samples, {on_hair} on hair")
    assert on_hair >= 2000


def test_asset_update_matches_a_fresh_asset(ctx):
    """hr_asset_update (new strand positions, as in animation) followed by a
    full frame gives the frame of an asset created from those positions:
    the hierarchy, thick hairs, LoD and BVH are rebuilt from the new
    vertices, with pageable host, device and page-locked host vertex buffers."""
    torch = pytest.importorskip("torch")
    w0 = scenegen.full_head(n=6000, S=16, width=64, height=48, spp=2, n_lights=2, n_clusters=256)
    w1 = scenegen.full_head(n=6000, S=16, width=64, height=48, spp=2, n_lights=2, n_clusters=256,
                            seed=5)
    d = desc_of(w0)
    a = upload(ctx, w0.scene)
    b = hr.hr_asset_create(ctx, np.ascontiguousarray(w1.scene.verts),
                           np.ascontiguousarray(w0.scene.mat), np.ascontiguousarray(w0.scene.shape))
    try:
        img = np.zeros((48, 64, 3), np.float32)
        hr.hr_render_frame(ctx, a, w0.n_clusters, w0.eps_w, 0, d, img)
        ref = np.zeros_like(img)
        hr.hr_render_frame(ctx, b, w0.n_clusters, w0.eps_w, 0, d, ref)
        assert ref.max() > 0
        hr.hr_asset_update(ctx, a, np.ascontiguousarray(w1.scene.verts))
        hr.hr_render_frame(ctx, a, w0.n_clusters, w0.eps_w, 0, d, img)
        assert np.array_equal(img, ref)
        # device vertices, back to the first positions and forth again
        hr.hr_asset_update(ctx, a, torch.from_numpy(w0.scene.verts).to("cuda:0"))
        hr.hr_render_frame(ctx, a, w0.n_clusters, w0.eps_w, 0, d, img)
        assert not np.array_equal(img, ref)
        hr.hr_asset_update(ctx, a, torch.from_numpy(w1.scene.verts).to("cuda:0"))
        torch.cuda.synchronize()
        hr.hr_render_frame(ctx, a, w0.n_clusters, w0.eps_w, 0, d, img)
        assert np.array_equal(img, ref)
        # page-locked host vertices (read by the update kernel in place)
        hr.hr_asset_update(ctx, a, torch.from_numpy(w0.scene.verts).pin_memory())
        hr.hr_render_frame(ctx, a, w0.n_clusters, w0.eps_w, 0, d, img)
        assert not np.array_equal(img, ref)
        pinned = torch.from_numpy(w1.scene.verts).pin_memory()
        hr.hr_asset_update(ctx, a, pinned)
        hr.hr_render_frame(ctx, a, w0.n_clusters, w0.eps_w, 0, d, img)
        assert np.array_equal(img, ref)
    finally:
        hr.hr_asset_destroy(ctx, a)
        hr.hr_asset_destroy(ctx, b)


def _moved(verts, amp, seed=3, anchored=False):
    """The same strands displaced by a smooth field (radius column kept);
    anchored: the displacement grows from 0 at the root (roots stay on the
    scalp, as attached hair does)."""
    v = np.array(verts, np.float32, copy=True)
    p = v[..., :3].astype(np.float64)
    ph = 1.0 + 0.1 * seed
    g = np.linspace(0.0, 1.0, v.shape[1])[None, :] if anchored else 1.0
    v[..., 0] += (amp * g * np.sin(7.0 * p[..., 1] + ph)).astype(np.float32)
    v[..., 2] += (amp * g * np.cos(5.0 * p[..., 0] - ph)).astype(np.float32)
    return v


def test_frame_refit_matches_rebuild(ctx):
    """HR_FLAG_REFIT after hr_asset_update: with the LoD unchanged the BVH is
    refit (same topology, new bounds and records) and the frame equals a
    rebuilt one; with the LoD changed the frame call rebuilds."""
    w = scenegen.full_head(n=6000, S=16, width=96, height=64, spp=2, n_lights=2, n_clusters=256)
    d = desc_of(w)
    moved = _moved(w.scene.verts, 2e-5, anchored=True)
    a = upload(ctx, w.scene)
    b = hr.hr_asset_create(ctx, moved, np.ascontiguousarray(w.scene.mat),
                           np.ascontiguousarray(w.scene.shape))
    try:
        img = np.zeros((64, 96, 3), np.float32)
        st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, img, stats=True)
        assert st.bvh_refit == 0
        hr.hr_asset_update(ctx, a, moved)
        dr = desc_of(w, flags=hr.HR_FLAG_REFIT)
        st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, dr, img, stats=True)
        ref = np.zeros_like(img)
        hr.hr_render_frame(ctx, b, w.n_clusters, w.eps_w, 0, d, ref)
        assert st.bvh_refit == 1
        assert ref.max() > 0
        assert np.allclose(img, ref, rtol=1e-6, atol=1e-7), np.abs(img - ref).max()
        # another LoD (a larger width threshold): no refit, same frame as a rebuild
        st = hr.hr_render_frame(ctx, a, w.n_clusters, 4.0 * w.eps_w, 0, dr, img, stats=True)
        hr.hr_render_frame(ctx, b, w.n_clusters, 4.0 * w.eps_w, 0, d, ref)
        assert st.bvh_refit == 0
        assert np.array_equal(img, ref)
    finally:
        hr.hr_asset_destroy(ctx, a)
        hr.hr_asset_destroy(ctx, b)


def test_frame_deferred_lod_follows_eq14(ctx):
    """HR_FLAG_DEFERRED_LOD: the second frame's LoD comes from Eq. 14 applied
    to the first frame's selection, as the oracle's deferred rule gives it."""
    w = scenegen.full_head(n=6000, S=16, width=96, height=64, spp=1, n_lights=1, n_clusters=256)
    a = upload(ctx, w.scene)
    try:
        img = np.zeros((64, 96, 3), np.float32)
        d = desc_of(w, flags=hr.HR_FLAG_DEFERRED_LOD)
        st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, img, stats=True)
        assert st.lod_deferred == 0  # no previous selection yet
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        first = np.zeros(C, np.uint8)
        hr.hr_select_lod(ctx, a, w.camera.pack(), w.eps_w, 0, 0, first)
        # a closer camera for the second frame, so Eq. 14 has work to do
        cam2 = scenegen.frame_camera(*w.scene.aabb(), 96, 64, perspective=True, fill=0.3).pack()
        d2 = hr.render_desc(cam2, w.lights, 1, w.k_depth, w.sample_seed, 0,
                            hr.HR_FLAG_DEFERRED_LOD)
        st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d2, img, stats=True)
        assert st.lod_deferred == 1
        prep = oracle_prepare(w)
        wcl = oracle.cluster_level_widths(prep.hier, prep.eth, cam2)
        want = oracle.select_lod_deferred(wcl, first.astype(np.int64), w.eps_w, L)
        n = hr.hr_bvh_export(ctx, a)
        ids = np.zeros(n, np.uint32)
        hr.hr_bvh_export(ctx, a, ids)
        prep2 = oracle_prepare(w, lod=np.asarray(want, np.uint8))
        assert np.array_equal(np.sort(ids.astype(np.int64)), np.sort(prep2.ids))
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_render_profile_records_every_tile(ctx):
    """hr_render_profile: the image of a plain render, one record per warp tile
    (each tile index once), ordered times, and per-lane counts no larger than
    the frame's totals."""
    w = scenegen.full_head(n=3000, S=8, width=64, height=48, spp=4, n_lights=2, n_clusters=64)
    a = upload(ctx, w.scene)
    try:
        gpu_lod(ctx, a, w)
        ref = np.zeros((48, 64, 3), np.float32)
        hr.hr_render(ctx, a, desc_of(w), ref)
        img = np.zeros_like(ref)
        st, rec, n = hr.hr_render_profile(ctx, a, desc_of(w, flags=hr.HR_FLAG_COUNT), img, 1 << 16)
        assert n > 0 and rec.size == n
        assert np.array_equal(np.sort(rec["tile"]), np.arange(n))
        assert np.all(rec["t_end_ns"] >= rec["t_start_ns"])
        assert np.allclose(img, ref, rtol=1e-5, atol=1e-7)
        assert rec["max_prim_tests"].max() <= st.prim_tests
        assert rec["max_node_visits"].max() <= st.node_visits and st.node_visits > 0
        # a short buffer takes the first tiles only
        st2, rec2, n2 = hr.hr_render_profile(ctx, a, desc_of(w), img, 3)
        assert n2 == n and rec2.size == min(3, n)
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_pipelined_frames_equal_single_frames(ctx):
    """Back-to-back hr_render_frame calls (device output, no statistics) build
    each frame's clusters and fit on the side stream while the previous frame
    renders; alternating two views (so LoD and BVH change every frame), every
    image equals a render of the same view without overlap."""
    import torch
    w = scenegen.full_head(n=6000, S=16, width=96, height=64, spp=2, n_lights=2, n_clusters=256)
    cams = [w.camera.pack(),
            scenegen.frame_camera(*w.scene.aabb(), 96, 64, perspective=True, fill=0.3).pack()]
    descs = [hr.render_desc(c, w.lights, w.spp, w.k_depth, w.sample_seed, 0) for c in cams]
    ref = []
    for d in descs:  # a fresh asset per view: its first frame cannot overlap anything
        b = upload(ctx, w.scene)
        try:
            img = np.zeros((64, 96, 3), np.float32)
            hr.hr_render_frame(ctx, b, w.n_clusters, w.eps_w, 0, d, img, stats=True)
            ref.append(img)
        finally:
            hr.hr_asset_destroy(ctx, b)
    a = upload(ctx, w.scene)
    try:
        outs = [torch.zeros((64, 96, 3), dtype=torch.float32, device="cuda") for _ in range(6)]
        for i, o in enumerate(outs):
            hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, descs[i % 2], o)
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            assert np.array_equal(o.cpu().numpy(), ref[i % 2]), i
        frame_ms, fit_ms = hr.hr_frame_times(ctx, 6)
        assert frame_ms.size == 6 and np.all(frame_ms > 0) and np.all(fit_ms > 0)
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_pipelined_updates_equal_single_frames(ctx):
    """hr_asset_update right after hr_render_frame writes the asset's other
    vertex and record set on the side stream while the frame renders; a loop
    of (update, frame) over two poses, device output and no statistics, gives
    every frame the image of a fresh asset in that pose."""
    import torch
    w = scenegen.full_head(n=6000, S=16, width=96, height=64, spp=2, n_lights=2, n_clusters=256)
    poses = [np.ascontiguousarray(w.scene.verts), _moved(w.scene.verts, 2e-3, anchored=True)]
    d = desc_of(w)
    ref = []
    for v in poses:  # a fresh asset per pose: nothing to overlap
        b = hr.hr_asset_create(ctx, v, np.ascontiguousarray(w.scene.mat),
                               np.ascontiguousarray(w.scene.shape))
        try:
            img = np.zeros((64, 96, 3), np.float32)
            hr.hr_render_frame(ctx, b, w.n_clusters, w.eps_w, 0, d, img, stats=True)
            ref.append(img)
        finally:
            hr.hr_asset_destroy(ctx, b)
    a = upload(ctx, w.scene)
    try:
        pinned = [torch.from_numpy(v).pin_memory() for v in poses]
        outs = [torch.zeros((64, 96, 3), dtype=torch.float32, device="cuda") for _ in range(7)]
        hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, outs[0])
        for i in range(1, 7):
            hr.hr_asset_update(ctx, a, pinned[i % 2])
            hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, outs[i])
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            assert np.array_equal(o.cpu().numpy(), ref[i % 2]), i
        # and a plain call afterwards sees the last pose
        img = np.zeros((64, 96, 3), np.float32)
        hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, img, stats=True)
        assert np.array_equal(img, ref[0])
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_frames_changing_the_hierarchy_shape(ctx):
    """Back-to-back frames whose cluster count alternates (the hierarchy's
    shape changes every frame, so no frame may build on the previous one's
    buffers): every image equals a fresh render with that cluster count, and
    the frame-time ring reports a fit for each call."""
    import torch
    w = scenegen.full_head(n=6000, S=16, width=96, height=64, spp=2, n_lights=2, n_clusters=256)
    d = desc_of(w)
    counts = [256, 128]
    ref = []
    for C in counts:
        b = upload(ctx, w.scene)
        try:
            img = np.zeros((64, 96, 3), np.float32)
            hr.hr_render_frame(ctx, b, C, w.eps_w, 0, d, img, stats=True)
            ref.append(img)
        finally:
            hr.hr_asset_destroy(ctx, b)
    a = upload(ctx, w.scene)
    try:
        outs = [torch.zeros((64, 96, 3), dtype=torch.float32, device="cuda") for _ in range(5)]
        for i, o in enumerate(outs):
            hr.hr_render_frame(ctx, a, counts[i % 2], w.eps_w, 0, d, o)
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            assert np.array_equal(o.cpu().numpy(), ref[i % 2]), i
        _, fit_ms, flags = hr.hr_frame_times(ctx, 5, with_flags=True)
        assert np.all(flags & 1) and np.all(fit_ms > 0) and not np.any(flags & 2)
    finally:
        hr.hr_asset_destroy(ctx, a)


# ---------------------------------------------------------------- shadow rays
SHADOW_AGREE_MIN = 0.99  # samples whose radiance agrees to 1e-3 (shadow crossings decided alike)


@pytest.mark.parametrize("wl", ["tiny", "clusters_half", "full_head"])
def test_shadow_rays_against_the_oracle(ctx, wl):
    """HR_FLAG_SHADOWS (dual-scattering light paths): the GPU's transmittance
    and spread along every shadow ray against the oracle's brute force over
    all primitives.  A shadow ray grazing a hair can cross it in FP64 and
    miss it in FP32, which changes that light's term by a_F: such samples are
    counted apart (at most 1%), the rest must agree to the FP32 bar."""
    rng = np.random.default_rng(11)
    if wl == "tiny":
        w = scenegen.tiny_strands()
        sids = np.arange(w.camera.width * w.camera.height * w.spp)
    elif wl == "clusters_half":
        w = scenegen.clustered(n=3000, S=12, res=48, spp=4, lod_setting="half", n_clusters=64)
        sids = rng.choice(w.camera.width * w.camera.height * w.spp, 3000, replace=False)
    else:
        w = scenegen.full_head(n=8000, S=16, width=96, height=64, spp=2, n_lights=4,
                               n_clusters=320, fill=0.25)
        sids = rng.choice(w.camera.width * w.camera.height * w.spp, 1000, replace=False)
    a = upload(ctx, w.scene)
    try:
        lod_g = gpu_lod(ctx, a, w)
        prep = _oracle_with_lod(w, None, lod_g)
        d = desc_of(w, flags=hr.HR_FLAG_SHADOWS)
        rg, hg = gpu_samples(ctx, a, d, sids)
        r0, _ = gpu_samples(ctx, a, desc_of(w), sids)
        ro, ho = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, w.k_depth,
                                       w.sample_seed, flags=oracle.FLAG_SHADOWS)
        frac, full, _, _ = compare(rg, hg, ro, ho)
        same = np.all(np.asarray(hg, np.int64) == ho, axis=1)
        on = np.linalg.norm(ro, axis=1)
        err = np.linalg.norm(rg.astype(np.float64) - ro, axis=1) / np.maximum(on, 1e-3 * on.mean())
        ok = same & (err <= 1e-3)
        agree = ok.sum() / max(1, same.sum())
        rmse = np.linalg.norm(rg[ok].astype(np.float64) - ro[ok]) / np.linalg.norm(ro[ok])
        msg = (f"{w.name}: k-buffer agreement {full:.5f}, shadow agreement {agree:.5f}, "
               f"rel-RMSE {rmse:.2e}, light kept {rg.sum() / r0.sum():.3f}")
        print(msg)
        assert full >= KBUF_AGREE_MIN, msg
        assert agree >= SHADOW_AGREE_MIN, msg
        assert rmse <= RMSE_FP32, msg
        if wl != "tiny":  # hair shadows hair: less light than without shadow rays
            assert rg.sum() < 0.95 * r0.sum(), msg
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_invalid_calls_are_refused_with_a_status(ctx):
    """Argument and state errors come back as status codes (no fault, no
    crash) and leave the context usable."""
    w = scenegen.tiny_strands()

    def status_of(fn, *a, **k):
        with pytest.raises(hr.HairRTError) as e:
            fn(*a, **k)
        return e.value.status

    v = np.ascontiguousarray(w.scene.verts)
    assert status_of(hr.hr_asset_create, ctx, v[:0], w.scene.mat[:0], w.scene.shape[:0]) == hr.HR_EINVAL
    a = upload(ctx, w.scene)
    try:
        img = np.zeros((w.camera.height, w.camera.width, 3), np.float32)
        # no BVH yet
        assert status_of(hr.hr_render, ctx, a, desc_of(w), img) == hr.HR_ESTATE
        assert status_of(hr.hr_build_clusters, ctx, a, w.scene.n_strands + 1) == hr.HR_EINVAL
        hr.hr_build_bvh(ctx, a, None)
        bad = desc_of(w)
        bad.spp = 0
        assert status_of(hr.hr_render, ctx, a, bad, img) == hr.HR_EINVAL
        bad = desc_of(w)
        bad.k_depth = hr.HR_MAX_K + 1
        assert status_of(hr.hr_render, ctx, a, bad, img) == hr.HR_EINVAL
        # the context still renders
        hr.hr_render(ctx, a, desc_of(w), img)
        assert img.max() > 0
    finally:
        hr.hr_asset_destroy(ctx, a)


@pytest.mark.parametrize("n,bits,dups", [(1, 30, False), (2, 30, True), (3071, 21, False),
                                         (3072 * 5 + 17, 21, True), (100_003, 30, False),
                                         (250_000, 32, True)])
def test_radix_sort_is_stable_and_matches_numpy(ctx, n, bits, dups):
    """The library's radix sort (single sweep per digit, decoupled look-back)
    against numpy's stable argsort of the low `bits` key bits, through the
    look-back and through the path where every tile counts the earlier keys
    itself (taken when a wait for an earlier tile runs out)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(n + bits)
    hi = 64 if dups else 2 ** 32
    keys = rng.integers(0, hi, n, dtype=np.uint64).astype(np.uint32)
    if dups:
        keys |= rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32) & ~np.uint32(2 ** bits - 1 if bits < 32 else 0xFFFFFFFF)
    vals = np.arange(n, dtype=np.uint32)[::-1].copy()
    mask = np.uint32(0xFFFFFFFF) if bits == 32 else np.uint32((1 << bits) - 1)
    order = np.argsort(keys & mask, kind="stable")
    for count_earlier in (False, True):
        k = torch.from_numpy(keys.view(np.int32).copy()).to("cuda:0")
        v = torch.from_numpy(vals.view(np.int32).copy()).to("cuda:0")
        torch.cuda.synchronize()
        hr.hr_sort_pairs(ctx, k, v, n, bits, count_earlier)
        kk = k.cpu().numpy().view(np.uint32)
        vv = v.cpu().numpy().view(np.uint32)
        assert np.array_equal(vv, vals[order]), count_earlier
        assert np.array_equal(kk, keys[order]), count_earlier


def test_thick_hair_image_converges_to_the_strand_image(ctx):
    """Section 4 (Eq. 5 against Eq. 1): the GPU's image of the level-L thick
    hairs approaches its strand image of the same clusters as L rises (the
    relative RMSE falls strictly from level to level), and every level's
    samples match the oracle.  A scene whose rays cross few semi-transparent
    thick-hair layers, so a k-buffer of 8 holds them (1,200 strands x 12
    segments in 8 clusters: 1, 4, 16 and 64 thick hairs per cluster)."""
    w = scenegen.clustered(n=1200, S=12, res=48, spp=4, lod_setting="strands", n_clusters=8)
    n = w.camera.width * w.camera.height * w.spp
    sids = np.arange(n)
    a = upload(ctx, w.scene)
    try:
        hr.hr_build_clusters(ctx, a, w.n_clusters)
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        assert L == 4
        imgs = []
        for lv in list(range(L)) + [L]:
            lod = np.full(C, lv, np.uint8)
            hr.hr_build_bvh(ctx, a, lod)
            d = desc_of(w, k=8)
            rg, hg = gpu_samples(ctx, a, d, sids)
            prep = oracle_prepare(w, lod=lod)
            ro, ho = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, 8,
                                           w.sample_seed)
            frac, full, r_agree, _ = compare(rg, hg, ro, ho)
            assert frac >= HIT_AGREE_MIN and full >= KBUF_AGREE_MIN and r_agree <= RMSE_FP32, \
                (lv, frac, full, r_agree)
            imgs.append(rg.astype(np.float64).reshape(-1, w.spp, 3).mean(1))
        ref = imgs[-1]
        err = [float(np.linalg.norm(im - ref) / np.linalg.norm(ref)) for im in imgs[:-1]]
        print(f"GPU rel-RMSE against the strand image per level: {[round(e, 3) for e in err]}")
        assert all(b < a_ for a_, b in zip(err, err[1:])), err
    finally:
        hr.hr_asset_destroy(ctx, a)


def _with_trt_materials(w, seed=4):
    N = w.scene.n_strands
    st = scenegen.Stream(seed, 1)
    mel = 0.1 + 0.8 * st.uniform(N)
    rough = 0.1 + 0.2 * st.uniform(N)
    w.scene = scenegen.Scene(w.scene.verts, scenegen.material_marschner(mel, rough),
                             w.scene.shape, w.scene.name)
    return w


@pytest.mark.parametrize("wl,precision", [("tiny", 0), ("clusters_half", 0), ("clusters_half", 1),
                                          ("clusters_eth", 0), ("full_head_small", 0)])
def test_marschner_trt_lobe(ctx, wl, precision):
    """HR_FLAG_TRT (Section 7: the Marschner R / TT / TRT fibre inside the
    aggregate) on strands, on thick hairs and on a selected LoD, against the
    oracle with the same flag."""
    if wl == "tiny":
        w = scenegen.tiny_strands()
    elif wl == "clusters_half":
        w = scenegen.clustered(n=3000, S=12, res=48, spp=2, lod_setting="half", n_clusters=64)
    elif wl == "clusters_eth":
        w = scenegen.clustered(n=3000, S=12, res=40, spp=1, lod_setting="eth", n_clusters=64)
    else:
        w = scenegen.full_head(n=8000, S=16, width=96, height=64, spp=2, n_lights=8,
                               n_clusters=320, fill=0.25)
    w = _with_trt_materials(w)
    n = w.camera.width * w.camera.height * w.spp
    rg, hg, ro, ho = _render_check(ctx, w, np.arange(n), precision=precision,
                                   flags=hr.HR_FLAG_TRT)
    assert np.linalg.norm(ro) > 0


def test_marschner_trt_with_shadow_rays(ctx):
    w = _with_trt_materials(scenegen.clustered(n=3000, S=12, res=40, spp=2, lod_setting="half",
                                               n_clusters=64))
    a = upload(ctx, w.scene)
    try:
        lod_g = gpu_lod(ctx, a, w)
        prep = _oracle_with_lod(w, None, lod_g)
        flags = hr.HR_FLAG_TRT | hr.HR_FLAG_SHADOWS
        sids = np.random.default_rng(3).choice(w.camera.width * w.camera.height * w.spp, 1500,
                                               replace=False)
        rg, hg = gpu_samples(ctx, a, desc_of(w, flags=flags), sids)
        ro, ho = oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, w.k_depth,
                                       w.sample_seed, flags=oracle.FLAG_SHADOWS | oracle.FLAG_TRT)
        same = np.all(np.asarray(hg, np.int64) == ho, axis=1)
        on = np.linalg.norm(ro, axis=1)
        err = np.linalg.norm(rg.astype(np.float64) - ro, axis=1) / np.maximum(on, 1e-3 * on.mean())
        ok = same & (err <= 1e-3)
        rmse = np.linalg.norm(rg[ok].astype(np.float64) - ro[ok]) / np.linalg.norm(ro[ok])
        print(f"TRT + shadows: k-buffer agreement {same.mean():.5f}, "
              f"shadow agreement {ok.sum() / max(1, same.sum()):.5f}, rel-RMSE {rmse:.2e}")
        assert same.mean() >= KBUF_AGREE_MIN
        assert ok.sum() / max(1, same.sum()) >= SHADOW_AGREE_MIN
        assert rmse <= RMSE_FP32
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_refit_engages_under_small_motion_with_hysteresis(ctx):
    """Animated frames (hr_asset_update with a small displacement every frame,
    roots kept on the scalp) under HR_FLAG_REFIT | HR_FLAG_DEFERRED_LOD |
    HR_FLAG_LOD_HYSTERESIS keep every cluster's strands and level, so every
    frame after the first refits its BVH, and a refit frame equals a rebuilt
    BVH at the same LoD.  Motion that moves the roots reorders the clusters,
    and the frame then rebuilds."""
    w = scenegen.full_head(n=20000, S=32, width=192, height=128, spp=2, n_lights=4,
                           n_clusters=800)
    poses = [np.ascontiguousarray(w.scene.verts), _moved(w.scene.verts, 2e-5, anchored=True)]
    flags = hr.HR_FLAG_REFIT | hr.HR_FLAG_DEFERRED_LOD | hr.HR_FLAG_LOD_HYSTERESIS
    d = desc_of(w, flags=flags)
    a = upload(ctx, w.scene)
    try:
        img = np.zeros((128, 192, 3), np.float32)
        hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, img)
        refits = 0
        for i in range(6):
            hr.hr_asset_update(ctx, a, poses[(i + 1) % 2])
            st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, img, stats=True)
            refits += st.bvh_refit
        assert refits == 6, refits
        ref = np.zeros_like(img)
        hr.hr_build_bvh(ctx, a, None)  # the asset's current selection
        hr.hr_render(ctx, a, desc_of(w), ref)
        assert ref.max() > 0
        assert np.allclose(img, ref, rtol=1e-6, atol=1e-7), np.abs(img - ref).max()
        # roots moved: the Morton clusters change, so no refit
        hr.hr_asset_update(ctx, a, _moved(w.scene.verts, 2e-3))
        st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, img, stats=True)
        assert st.bvh_refit == 0
        # the same loop with page-locked poses and device images: the uploads
        # and clusters overlap the frames, and every frame after the first refits
        import torch
        pinned = [torch.from_numpy(p).pin_memory() for p in poses]
        dimg = torch.zeros((128, 192, 3), dtype=torch.float32, device="cuda")
        hr.hr_asset_update(ctx, a, pinned[0])
        hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, dimg)
        for i in range(6):
            hr.hr_asset_update(ctx, a, pinned[(i + 1) % 2])
            hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, dimg)
        _, _, fl = hr.hr_frame_times(ctx, 6, with_flags=True)
        assert np.all(fl & 2), fl
        hr.hr_build_bvh(ctx, a, None)
        hr.hr_render(ctx, a, desc_of(w), ref)
        assert np.allclose(dimg.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_tile_schedule_keeps_the_image(ctx):
    """The frame kernel traces the previous frame's heaviest warp tiles first,
    a few rays per warp, and composites them from stored lane sums in the
    fixed shuffle order: every frame equals the same frame rendered in the fixed
    tile order (HR_FLAG_FIXED_TILE_ORDER), bit for bit, through a repeated
    view (heavy tiles used), a change of view (tiles of the old grid), a
    change of spp (another tile shape: schedule dropped) and of image size."""
    w = scenegen.full_head(n=6000, S=16, width=128, height=96, spp=8, n_lights=2, n_clusters=256)
    box = w.scene.aabb()
    views = {"near": scenegen.frame_camera(*box, 128, 96, perspective=True, fill=0.6),
             "far": scenegen.frame_camera(*box, 128, 96, perspective=True, fill=0.35),
             "big": scenegen.frame_camera(*box, 160, 120, perspective=True, fill=0.6)}

    def desc(view, spp, flags=0):
        return hr.render_desc(views[view].pack(), w.lights, spp, w.k_depth, w.sample_seed, 0, flags)

    def size(view):
        return (views[view].height, views[view].width, 3)

    seq = [("near", 8), ("near", 8), ("near", 8), ("far", 8), ("near", 8), ("near", 4),
           ("near", 8), ("big", 8), ("big", 8)]
    ref = {}
    a = upload(ctx, w.scene)
    try:
        for view, spp in set(seq):
            img = np.zeros(size(view), np.float32)
            st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0,
                                    desc(view, spp, hr.HR_FLAG_FIXED_TILE_ORDER), img, stats=True)
            assert st.heavy_tiles == 0
            ref[(view, spp)] = img
    finally:
        hr.hr_asset_destroy(ctx, a)
    a = upload(ctx, w.scene)
    try:
        heavy = []
        for view, spp in seq:
            img = np.zeros(size(view), np.float32)
            st = hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, desc(view, spp), img,
                                    stats=True)
            heavy.append(st.heavy_tiles)
            assert np.array_equal(img, ref[(view, spp)]), (view, spp, st.heavy_tiles)
        # the first frame has no previous one; a repeated view has heavy tiles;
        # a frame after an spp change or a resize has none
        assert heavy[0] == 0 and heavy[1] > 0 and heavy[2] > 0, heavy
        assert heavy[5] == 0 and heavy[6] == 0 and heavy[7] == 0 and heavy[8] > 0, heavy
    finally:
        hr.hr_asset_destroy(ctx, a)
