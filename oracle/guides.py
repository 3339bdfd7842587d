"""Guide hairs, the guide-driven hierarchy and linear skinning (oracle).

TEST INFRASTRUCTURE ONLY, like the rest of this package: plain numpy, sharing
no code with the CUDA library.

Section 5.1 of the paper builds the hierarchy from guide hairs:
  1. k-means over the strands with D(i, j) = sum_k |p^{i,k} - p^{j,k}|^2 over
     corresponding control points; each cluster's guide is the member with the
     smallest average distance to the others (its medoid);
  2. every strand finds its three nearest guides, and strands that share the
     same three form a cluster of the coarsest level L0; finer levels come
     from L0 with about four times less area per level;
  4. three guides form a triangular prism for linear skinning: every control
     point of a strand, and every thick-hair cross-section centre and corner,
     gets interpolation weights that carry it along with the guides.
Section 5.2 moves the hair at run time with those weights.

READINGS (the paper leaves these open):
  * control points are the strand vertices (the synthetic strands are already
    polylines, so no Catmull-Rom refit);
  * D, the centroid sums and the medoid sums are FP32, point by point in
    vertex order, ((dx dx + dy dy) + dz dz) per point, sums over members in
    ascending strand id: the kernels' precision and order, so that the
    integer decisions built on them (cluster ids, medoids, nearest guides)
    compare bit for bit;
  * k-means starts from the strands at Morton ranks floor((2g + 1) N / 2G) of
    the roots (spread over the scalp, deterministic), runs a fixed number of
    update rounds and ends with an assignment; an empty cluster keeps its
    centroid and has no guide; ties go to the lower cluster, guide or strand
    index;
  * a cluster of L0 lists its strands in (Morton code, id) order, and its
    level-k thick hairs split it into 4^k rank buckets as in the Morton
    hierarchy (a cluster with fewer than 4^k strands leaves buckets empty; an
    empty thick hair has no primitives);
  * prism weights: p = g0 + w1 (g1 - g0) + w2 (g2 - g0) + h n with n the unit
    normal of the triangle of the guides' corresponding points; for a
    degenerate triangle the point keeps its offset from g0.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32


def strand_distance(A, B):
    """D(i, j) = sum_k |p^{i,k} - p^{j,k}|^2 (Section 5.1, guide hair selection)
    between polylines A [..., S1, 3] and B [..., S1, 3] (broadcast), in FP32,
    point by point in k order.

    Pinned by test_strand_distance_against_fp64 and
    test_strand_distance_order_is_sequential.
    """
    A = np.asarray(A, F32)
    B = np.asarray(B, F32)
    d = np.zeros(np.broadcast_shapes(A.shape[:-2], B.shape[:-2]), F32)
    for k in range(A.shape[-2]):
        dx = A[..., k, 0] - B[..., k, 0]
        dy = A[..., k, 1] - B[..., k, 1]
        dz = A[..., k, 2] - B[..., k, 2]
        d = d + ((dx * dx + dy * dy) + dz * dz)
    return d


def _morton_order(P):
    from . import morton30, quantize_roots
    N = P.shape[0]
    code = morton30(quantize_roots(P[:, 0]))
    return np.lexsort((np.arange(N), code)).astype(np.int64), code


def guide_kmeans(verts, n_guides: int, iterations: int):
    """k-means of the strands under D (Section 5.1 step 1) and the medoid
    guide of each cluster.  Returns (cluster of every strand [N], centroids
    [G, S1, 3] float32, guide strand of every cluster [G], -1 when empty).

    Pinned by test_kmeans_two_separated_bundles, test_kmeans_assignment_is_nearest_centroid
    and test_medoid_is_the_brute_force_minimiser.
    """
    P = np.asarray(verts, F32)[..., :3]
    N = P.shape[0]
    G = int(n_guides)
    order, _ = _morton_order(P)
    seeds = order[(2 * np.arange(G) + 1) * N // (2 * G)]
    cent = P[seeds].copy()

    def assign():
        D = np.stack([strand_distance(P, cent[g]) for g in range(G)], 1)
        return np.argmin(D, 1)  # first minimum: the lowest cluster on ties

    for _ in range(iterations):
        a = assign()
        for g in range(G):
            mem = np.nonzero(a == g)[0]
            if mem.size == 0:
                continue
            acc = np.zeros(P.shape[1:], F32)
            for i in mem:
                acc = acc + P[i]
            cent[g] = acc / F32(mem.size)
    a = assign()
    guides = np.full(G, -1, np.int64)
    for g in range(G):
        mem = np.nonzero(a == g)[0]
        if mem.size == 0:
            continue
        s = np.zeros(mem.size, F32)
        for j in mem:  # sum over the other members in ascending id, for every candidate
            s = s + strand_distance(P[mem], P[j])
        guides[g] = mem[int(np.argmin(s))]
    return a.astype(np.int64), cent, guides


def nearest_guides(verts, guides):
    """The three guides nearest to every strand under D (Section 5.1 step 2),
    ascending guide index, ties to the lower index.

    Pinned by test_nearest_guides_brute_force.
    """
    P = np.asarray(verts, F32)[..., :3]
    valid = np.nonzero(np.asarray(guides) >= 0)[0]
    D = np.stack([strand_distance(P, P[guides[g]]) for g in valid], 1)
    pick = np.argsort(D, axis=1, kind="stable")[:, :3]
    return np.sort(valid[pick], axis=1)


def build_guided_hierarchy(verts, n_guides: int, iterations: int, max_levels: int = 0):
    """The paper's hierarchy (Section 5.1 steps 1-2): guides by k-means, L0
    clusters of strands sharing their three nearest guides (cluster index in
    ascending order of the guide triple), strands ordered by (triple, Morton
    code of the root, id) and levels split into rank buckets.  Returns the
    Hierarchy, the guide of every k-means cluster and every strand's triple.

    Pinned by test_guided_clusters_share_their_triple and
    test_guided_hierarchy_levels_and_empty_buckets.
    """
    from . import hierarchy_from_clusters
    P = np.asarray(verts, F32)[..., :3]
    N = P.shape[0]
    if n_guides > 1024 or n_guides < 3:
        raise ValueError("3 <= n_guides <= 1024")
    _, _, guides = guide_kmeans(P, n_guides, iterations)
    tri = nearest_guides(P, guides)
    key = (tri[:, 0] << 20) | (tri[:, 1] << 10) | tri[:, 2]
    _, code = _morton_order(P)
    order = np.lexsort((np.arange(N), code, key)).astype(np.int64)
    ks = key[order]
    new = np.ones(N, bool)
    new[1:] = ks[1:] != ks[:-1]
    cl_rank = np.cumsum(new) - 1
    C = int(cl_rank[-1]) + 1
    first = np.append(np.nonzero(new)[0], N).astype(np.int64)
    h = hierarchy_from_clusters(N, C, order, code, first, max_levels)
    return h, guides, tri


# ------------------------------------------------------------------ skinning


def prism_weights(p, g0, g1, g2):
    """Interpolation weights of points p in the triangular prism of three
    guide points g0, g1, g2 (Section 5.1 step 4), FP64: (w1, w2, h, flag) with
    p = g0 + w1 (g1 - g0) + w2 (g2 - g0) + h n, n the unit normal of the
    triangle; flag 1 (a degenerate triangle) stores the offset p - g0 in
    (w1, w2, h) instead.

    Pinned by test_prism_weights_rest_pose_and_rigid_motion and
    test_prism_weights_affine_in_plane.
    """
    p, g0, g1, g2 = (np.asarray(x, np.float64) for x in (p, g0, g1, g2))
    shape = np.broadcast_shapes(p.shape, g0.shape, g1.shape, g2.shape)
    p, g0, g1, g2 = (np.broadcast_to(x, shape) for x in (p, g0, g1, g2))
    e1 = g1 - g0
    e2 = g2 - g0
    n = np.cross(e1, e2)
    nn = np.linalg.norm(n, axis=-1)
    scale = np.linalg.norm(e1, axis=-1) * np.linalg.norm(e2, axis=-1)
    degen = ~(nn > 1e-6 * scale)
    nh = n / np.where(degen, 1.0, nn)[..., None]
    q = p - g0
    h = np.sum(q * nh, -1)
    qp = q - h[..., None] * nh
    den = np.where(degen, 1.0, nn)
    w1 = np.sum(np.cross(qp, e2) * nh, -1) / den
    w2 = np.sum(np.cross(e1, qp) * nh, -1) / den
    out = np.stack([w1, w2, h, np.zeros_like(h)], -1)
    out[degen] = np.concatenate([q[degen], np.ones((int(degen.sum()), 1))], -1)
    return out


def skin_points(wts, g0, g1, g2):
    """Points carried by three moved guide points with prism weights (Section
    5.2: positions at run time from the simulated guides and the weights).

    Pinned by test_prism_weights_rest_pose_and_rigid_motion.
    """
    wts = np.asarray(wts, np.float64)
    g0, g1, g2 = (np.asarray(x, np.float64) for x in (g0, g1, g2))
    e1 = g1 - g0
    e2 = g2 - g0
    n = np.cross(e1, e2)
    nn = np.linalg.norm(n, axis=-1, keepdims=True)
    nh = n / np.where(nn > 0, nn, 1.0)
    p = g0 + wts[..., 0:1] * e1 + wts[..., 1:2] * e2 + wts[..., 2:3] * nh
    off = g0 + wts[..., 0:3]
    return np.where(wts[..., 3:4] > 0.5, off, p)
