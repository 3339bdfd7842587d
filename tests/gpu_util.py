"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2405_10565_gb300 as hr
import scenegen

# Tolerances (stated for FP32 traversal/intersection against the FP64 oracle).
HIT_AGREE_MIN = 0.999      # fraction of samples with the same nearest-hit id
RMSE_FP32 = 1e-3           # relative RMSE of radiance over agreeing samples
RMSE_FP16 = 5e-3           # same, FP16 lookup tables


def upload(ctx, scene):
    return hr.hr_asset_create(ctx, np.ascontiguousarray(scene.verts),
                              np.ascontiguousarray(scene.mat), np.ascontiguousarray(scene.shape))


def gpu_lod(ctx, asset, w, lod=None):
    """Build the GPU hierarchy and choose the LoD like the oracle's prepare()."""
    if w.n_clusters == 0:
        hr.hr_build_bvh(ctx, asset, None)
        return None
    hr.hr_build_clusters(ctx, asset, w.n_clusters)
    C, L, E = hr.hr_hierarchy_info(ctx, asset)
    if lod is None:
        if w.lod_setting == "select":
            lod = np.zeros(C, np.uint8)
            hr.hr_select_lod(ctx, asset, w.camera.pack(), w.eps_w, 0, 0, lod)
        else:
            lod = scenegen.lod_preset(w.lod_setting, C, L)
    lod = np.ascontiguousarray(lod, np.uint8)
    hr.hr_build_bvh(ctx, asset, lod)
    return lod


def desc_of(w, precision=None, flags=0, k=None, spp=None, seed=None):
    return hr.render_desc(w.camera.pack(), w.lights, spp or w.spp, k or w.k_depth,
                          w.sample_seed if seed is None else seed,
                          w.precision if precision is None else precision, flags)


KBUF_AGREE_MIN = 0.999     # fraction of samples with the same ordered k-buffer ids


def gpu_samples(ctx, asset, desc, sids):
    """Radiance [m, 3] and the K composited hit ids [m, K] of the listed samples."""
    sids = np.ascontiguousarray(sids, np.uint32)
    rad = np.zeros((sids.shape[0], 3), np.float32)
    hit = np.zeros((sids.shape[0], desc.k_depth), np.int32)
    hr.hr_render_samples(ctx, asset, desc, sids, rad, hit)
    return rad, hit


def compare(rad_g, hit_g, rad_o, hit_o):
    """(nearest-hit agreement, whole-k-buffer agreement, rel-RMSE over samples
    whose ordered k-buffer ids agree, rel-RMSE over all samples).

    Two hits at (nearly) equal depth may be ordered differently by FP32 and
    FP64 arithmetic; such a sample composites the same surfaces in another
    order, so its radiance is compared only when the whole ordered list agrees
    (and the fraction of such samples is bounded separately)."""
    hit_g = np.asarray(hit_g, np.int64).reshape(len(hit_g), -1)
    hit_o = np.asarray(hit_o, np.int64).reshape(len(hit_o), -1)
    near = hit_g[:, 0] == hit_o[:, 0]
    full = np.all(hit_g == hit_o, axis=1)
    def rr(mask):
        if not mask.any():
            return 0.0
        num = np.linalg.norm(rad_g[mask].astype(np.float64) - rad_o[mask])
        den = np.linalg.norm(rad_o[mask])
        return float(num / den) if den > 0 else float(num)
    fn = float(near.mean()) if near.size else 1.0
    ff = float(full.mean()) if full.size else 1.0
    return fn, ff, rr(full), rr(np.ones_like(full))


def oracle_prepare(w, lod=None):
    return oracle.prepare(w.scene, w.n_clusters, w.lod_setting, w.camera.pack(), w.eps_w,
                          lod=lod)


def hair_pixels(w, n, seed):
    """Up to n distinct pixels that contain the projection of a seeded hair
    vertex (perspective camera), so that their samples land on hair."""
    v = w.scene.verts[..., :3].reshape(-1, 3).astype(np.float64)
    c = w.camera
    st = scenegen.Stream(seed, 98)
    idx = (st.u64(8 * n) % np.uint64(v.shape[0])).astype(np.int64)
    r = v[idx] - c.eye.astype(np.float64)
    z = r @ c.fwd.astype(np.float64)
    X = (r @ c.right.astype(np.float64)) / z * c.pix_scale + 0.5 * c.width
    Y = 0.5 * c.height - (r @ c.up.astype(np.float64)) / z * c.pix_scale
    ok = (z > 0) & (X >= 0) & (X < c.width) & (Y >= 0) & (Y < c.height)
    pix = np.floor(Y[ok]).astype(np.int64) * c.width + np.floor(X[ok]).astype(np.int64)
    _, first = np.unique(pix, return_index=True)
    return pix[np.sort(first)][:n]
