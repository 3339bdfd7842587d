"""CPU oracle for the level-of-detail hair renderer (arXiv 2405.10565).

TEST INFRASTRUCTURE ONLY.  This package is imported by the test-suite, by the
smoke check and by the benchmark's CPU-baseline leg, and by nothing in the
product path.  It shares no code with the CUDA library: it re-derives every
step from the paper in plain numpy (hierarchy, ellipse fit, LoD rule, active
primitive list) and in plain C (``trace.c``: brute-force FP64 tracing and the
scattering models).  Where the paper is silent the reading taken is marked
READING and is the same reading the library follows.

Pins (tests/test_oracle_*.py) tie each function to something other than
itself: closed forms, analytic hits, brute force on tiny inputs, the
separable-albedo identity, reciprocity, the n = 1 reduction, hand-worked
Morton, record and light-sum examples, and the convergence of a thick-hair
image toward the strand image of the same clusters.  Every function names its
pins in its docstring.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

FLAG_NO_S = 1
FLAG_SINGLE_ON_ETH = 2
FLAG_SHADOWS = 4
FLAG_TRT = 8
PRIM_STRIDE = 15


def build(force: bool = False) -> str:
    """Compile trace.c into liboracle.so with gcc (no FMA contraction).

    Infrastructure (compiles trace.c; no arithmetic of the method).
    """
    src = os.path.join(_HERE, "trace.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        D = ctypes.c_double
        PD = ctypes.POINTER(ctypes.c_double)
        PI64 = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_render.argtypes = [PD, PI64, ctypes.c_int64, PD, ctypes.c_int64, PD, PD,
                                      ctypes.c_int, PI64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_uint64, ctypes.c_uint, ctypes.c_int,
                                      PD, PD, PD, PI64, ctypes.c_int]
        lib.oracle_render.restype = ctypes.c_int
        lib.oracle_gauss.argtypes = [D, D]
        lib.oracle_gauss.restype = D
        lib.oracle_im.argtypes = [ctypes.c_int, PD, PD, D, D]
        lib.oracle_im.restype = D
        lib.oracle_albedo.argtypes = [PD, ctypes.c_int, PD, PD, D, ctypes.c_uint, PD, PD, PD]
        lib.oracle_albedo_2d.argtypes = [PD, ctypes.c_int, PD, PD, D, ctypes.c_uint, PD, PD]
        lib.oracle_f_single.argtypes = [PD, D, D, D, ctypes.c_uint, PD]
        lib.oracle_f_single_spread.argtypes = [PD, D, D, D, D, PD]
        lib.oracle_shadow_path.argtypes = [PD, ctypes.c_int64, PD, ctypes.c_int64, ctypes.c_int,
                                           PD, PD, PD, PD, D, ctypes.c_int, ctypes.c_uint,
                                           PD, PD]
        lib.oracle_f_ours.argtypes = [PD, ctypes.c_int, PD, PD, D, D, D, D, D, ctypes.c_uint, PD]
        lib.oracle_intersect.argtypes = [PD, PD, PD, PD, PD]
        lib.oracle_intersect.restype = ctypes.c_int
        lib.oracle_back_atten.argtypes = [D, D, D, PD]
        lib.oracle_camera_ray.argtypes = [PD, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, PD, PD]
        _lib = lib
    return _lib


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


# ------------------------------------------------------------------ quadrature

_QUAD = {}


def gauss_legendre(n: int = 384):
    """Gauss-Legendre nodes and weights on [-1, 1] (numpy's leggauss).

    Pinned by test_gauss_legendre_is_exact_for_polynomials_up_to_degree_2n_minus_1.
    """
    if n not in _QUAD:
        x, w = np.polynomial.legendre.leggauss(n)
        _QUAD[n] = (np.ascontiguousarray(x, np.float64), np.ascontiguousarray(w, np.float64))
    return _QUAD[n]


# ------------------------------------------------------------------ BCSDF wrappers


def gauss(beta: float, x: float) -> float:
    """Pinned by test_gaussian_definition (the Gaussian's value at 0 and at one beta)."""
    return _load().oracle_gauss(beta, x)


def im(theta: float, beta: float, nq: int = 384) -> float:
    """Longitudinal albedo factor IM(theta; beta) (see trace.c).

    Pinned by test_longitudinal_integral_closed_form and
    test_longitudinal_integral_quadrature_converged.
    """
    x, w = gauss_legendre(nq)
    return _load().oracle_im(nq, _pd(x), _pd(w), theta, beta)


def albedo(mat12, theta_d: float, nq: int = 384, flags: int = 0):
    """(a_F rgb, a_B rgb, sigma_f^2) of a single fibre at theta_d.

    Pinned by test_separable_albedo_equals_2d_quadrature, test_albedo_white_furnace_c1_material
    and test_forward_albedo_stays_below_one_over_parameter_box.
    """
    m = np.ascontiguousarray(mat12, np.float64)
    x, w = gauss_legendre(nq)
    aF = np.zeros(3)
    aB = np.zeros(3)
    s2 = np.zeros(1)
    _load().oracle_albedo(_pd(m), nq, _pd(x), _pd(w), theta_d, flags, _pd(aF), _pd(aB), _pd(s2))
    return aF, aB, float(s2[0])


def albedo_2d(mat12, theta_i: float, nq: int = 256, flags: int = 0):
    """(front rgb, back rgb) directional albedo of f_single by 2-D quadrature.

    Pinned by test_albedo_2d_diffuse_closed_form (A_D / 4 per half for a diffuse fibre).
    """
    m = np.ascontiguousarray(mat12, np.float64)
    x, w = gauss_legendre(nq)
    f = np.zeros(3)
    b = np.zeros(3)
    _load().oracle_albedo_2d(_pd(m), nq, _pd(x), _pd(w), theta_i, flags, _pd(f), _pd(b))
    return f, b


def f_single(mat12, th_i, th_o, cphi, flags: int = 0):
    """Pinned by test_f_single_hand_values."""
    m = np.ascontiguousarray(mat12, np.float64)
    out = np.zeros(3)
    _load().oracle_f_single(_pd(m), th_i, th_o, cphi, flags, _pd(out))
    return out


def f_single_spread(mat12, th_i, th_o, cphi, sg2):
    """f_single with every lobe's variance grown by sg2 (the spread of the
    light path under shadow rays).

    Pinned by test_spread_is_a_wider_lobe.
    """
    out = np.zeros(3)
    m = np.ascontiguousarray(mat12, np.float64)
    _load().oracle_f_single_spread(_pd(m), th_i, th_o, cphi, sg2, _pd(out))
    return out


def shadow_path(rows, mats, x, wi, t_light, self_mat, nq: int = 384, flags: int = 0):
    """(T [3], sg2): the dual-scattering transmittance and spread variance of
    the light path from x along wi up to t_light, over primitive rows (15
    doubles each) with material rows `mats`, skipping material `self_mat`.

    Pinned by the hand-worked occluder cases of tests/test_oracle_shadows.py.
    """
    r = np.ascontiguousarray(rows, np.float64).reshape(-1, 15)
    mt = np.ascontiguousarray(mats, np.float64).reshape(-1, 12)
    qx, qw = gauss_legendre(nq)
    xx = np.ascontiguousarray(x, np.float64)
    ww = np.ascontiguousarray(wi, np.float64)
    T = np.zeros(3)
    sg2 = np.zeros(1)
    _load().oracle_shadow_path(_pd(r), r.shape[0], _pd(mt), mt.shape[0], nq, _pd(qx), _pd(qw),
                               _pd(xx), _pd(ww), float(t_light), int(self_mat), flags, _pd(T),
                               _pd(sg2))
    return T, float(sg2[0])


def f_ours(mat12, th_i, th_o, cphi, rho, n_view, flags=0, nq: int = 384):
    """Aggregated BCSDF of a thick hair (see trace.c).

    Pinned by test_aggregated_reciprocity, test_aggregated_reduces_to_single_at_n1_front,
    test_back_lobe_uniform_over_back_half, test_shadowing_masking_bounds_and_ablation_order,
    test_attenuation_with_hair_count and the thick-hair / strand convergence of
    tests/test_oracle_convergence.py.
    """
    m = np.ascontiguousarray(mat12, np.float64)
    x, w = gauss_legendre(nq)
    out = np.zeros(3)
    _load().oracle_f_ours(_pd(m), nq, _pd(x), _pd(w), th_i, th_o, cphi, rho, n_view, flags,
                          _pd(out))
    return out


def back_atten(aF: float, aB: float, n: float):
    """(A_1, A_3, A_1+) of one channel (see trace.c).

    Pinned by test_back_lobe_attenuations_equal_their_series.
    """
    out = np.zeros(3)
    _load().oracle_back_atten(aF, aB, n, _pd(out))
    return out


def intersect(row15, o, d):
    """(hit, t, chord) of a ray against one primitive row.

    Pinned by test_circular_cylinder_perpendicular_hit, test_elliptic_cylinder_axis_aligned_hit,
    test_eccentricity_zero_equals_circle and test_intersection_misses_and_open_ends.
    """
    r = np.ascontiguousarray(row15, np.float64)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    t = np.zeros(1)
    c = np.zeros(1)
    hit = _load().oracle_intersect(_pd(r), _pd(o), _pd(d), _pd(t), _pd(c))
    return bool(hit), float(t[0]), float(c[0])


def camera_ray(cam_rec, seed: int, sid: int, spp: int):
    """Pinned by test_camera_jitter_uses_published_stream and test_perspective_edge_ray_half_fov."""
    c = np.ascontiguousarray(cam_rec, np.float64)
    o = np.zeros(3)
    d = np.zeros(3)
    _load().oracle_camera_ray(_pd(c), seed, sid, spp, _pd(o), _pd(d))
    return o, d


# ------------------------------------------------------------------ hierarchy


def morton30(q: np.ndarray) -> np.ndarray:
    """30-bit Morton code of 10-bit integer coordinates: bit i of x, y, z goes
    to bits 3i+2, 3i+1, 3i.

    Pinned by test_morton_hand_worked_cube_corners, test_morton_mid_point_and_ties and
    test_morton_brute_force_random.
    """
    q = np.asarray(q, np.uint64)
    code = np.zeros(q.shape[0], np.uint64)
    for i in range(10):
        for axis, shift in ((0, 2), (1, 1), (2, 0)):
            bit = (q[:, axis] >> np.uint64(i)) & np.uint64(1)
            code |= bit << np.uint64(3 * i + shift)
    return code.astype(np.uint32)


def quantize_roots(roots: np.ndarray) -> np.ndarray:
    """q = min(1023, floor((p - lo) * (1024 / e))) per axis with lo the root
    AABB's low corner and e its largest extent (the bounding cube, so the grid
    is isotropic), each operation rounded to float32 in this order.

    Pinned by test_morton_quantises_in_bounding_cube and test_morton_mid_point_and_ties.
    """
    p = np.asarray(roots, np.float32)
    lo = p.min(0)
    hi = p.max(0)
    ext = np.float32((hi - lo).astype(np.float32).max())
    scale = np.float32(1024.0) / ext if ext > 0 else np.float32(0.0)
    v = ((p - lo).astype(np.float32) * np.float32(scale)).astype(np.float32)
    q = np.floor(v).astype(np.int64)
    return np.clip(q, 0, 1023)


def n_eth_levels_for(n_strands: int, n_clusters: int, max_levels: int = 0) -> int:
    """Number of thick-hair levels: 1 + max k with 4^k <= floor(N/C) / 2
    (READING: each level splits every cluster into 4x as many thick hairs,
    Section 5.1 "approximately four times"; a level must keep >= 2 strands
    per thick hair).  ``max_levels`` > 0 caps it.

    Pinned by test_level_count_rule.
    """
    per = n_strands // n_clusters
    if per < 2:
        return 0
    k = 0
    while 4 ** (k + 1) <= per // 2:
        k += 1
    lv = k + 1
    if max_levels > 0:
        lv = min(lv, max_levels)
    return lv


@dataclasses.dataclass
class Hierarchy:
    n_strands: int
    n_clusters: int
    n_levels: int            # thick-hair levels; level n_levels means strands
    order: np.ndarray        # strand ids sorted by (Morton code, id)
    code: np.ndarray         # Morton code per strand
    cluster_of: np.ndarray   # uint32 [N]
    eth_of: np.ndarray       # int64 [n_levels, N] global thick-hair index
    eth_offset: np.ndarray   # first thick-hair index of each level
    eth_first_rank: np.ndarray  # per thick hair: first rank of its members
    eth_count: np.ndarray       # per thick hair: member count
    eth_cluster: np.ndarray     # per thick hair: cluster
    eth_level: np.ndarray       # per thick hair: level

    @property
    def n_eths(self) -> int:
        return int(self.eth_count.shape[0])


def build_hierarchy(roots: np.ndarray, n_clusters: int, max_levels: int = 0) -> Hierarchy:
    """Deterministic Morton-bucket hierarchy (READING: replaces the paper's
    guide-hair clustering of Section 5.1 step 2 by a rule with a unique
    answer).  Strands are sorted by (30-bit Morton code of the quantised root,
    strand id); the strand of rank r joins cluster floor(r C / N); at level k a
    cluster of m members splits into 4^k thick hairs, rank-in-cluster i going
    to floor(i 4^k / m).

    Pinned by test_morton_hand_worked_cube_corners and test_hierarchy_partition_and_nesting.
    """
    N = roots.shape[0]
    C = n_clusters
    code = morton30(quantize_roots(roots))
    order = np.lexsort((np.arange(N), code)).astype(np.int64)
    first = np.array([-(-c * N // C) for c in range(C + 1)], np.int64)  # ceil(c N / C)
    return hierarchy_from_clusters(N, C, order, code, first, max_levels)


def hierarchy_from_clusters(N: int, C: int, order: np.ndarray, code: np.ndarray,
                            first: np.ndarray, max_levels: int = 0) -> Hierarchy:
    """The levels of a hierarchy whose cluster c holds the strands of ranks
    first[c] .. first[c + 1] - 1 of `order`: at level k cluster c of m
    members splits into 4^k thick hairs, rank-in-cluster i going to
    floor(i 4^k / m) (a bucket with no member is an empty thick hair when
    m < 4^k).  Levels: n_eth_levels_for(N, C).

    Pinned through build_hierarchy's and build_guided_hierarchy's tests.
    """
    rank = np.empty(N, np.int64)
    rank[order] = np.arange(N)
    cl_of_rank = np.searchsorted(first, np.arange(N), side="right") - 1
    cluster = cl_of_rank[rank]
    L = n_eth_levels_for(N, C, max_levels)
    eth_of = np.zeros((L, N), np.int64)
    offs = np.zeros(L + 1, np.int64)
    e_first, e_count, e_cluster, e_level = [], [], [], []
    m = first[1:] - first[:-1]
    for k in range(L):
        offs[k + 1] = offs[k] + C * 4 ** k
        sub_n = 4 ** k
        ric = rank - first[cluster]
        sub = (ric * sub_n) // m[cluster]
        eth_of[k] = offs[k] + cluster * sub_n + sub
        for c in range(C):
            for j in range(sub_n):
                # members of sub-bucket j: rank-in-cluster i with floor(i 4^k / m) == j
                lo = -(-j * m[c] // sub_n)
                hi = -(-(j + 1) * m[c] // sub_n)
                e_first.append(first[c] + lo)
                e_count.append(hi - lo)
                e_cluster.append(c)
                e_level.append(k)
    return Hierarchy(N, C, L, order, code, cluster.astype(np.uint32), eth_of, offs,
                     np.asarray(e_first, np.int64), np.asarray(e_count, np.int64),
                     np.asarray(e_cluster, np.int64), np.asarray(e_level, np.int64))


# ------------------------------------------------------------------ ellipse fit


@dataclasses.dataclass
class ETHs:
    """Thick hairs.  Cross-section arrays are [E, S+1, ...]; segment arrays [E, S, ...]."""
    center: np.ndarray   # f64 [E, S+1, 3]
    tangent: np.ndarray  # f64 [E, S+1, 3]
    e1: np.ndarray       # f64 [E, S+1, 3]
    e2: np.ndarray       # f64 [E, S+1, 3]
    a: np.ndarray        # f64 [E, S+1]
    b: np.ndarray        # f64 [E, S+1]
    seg_e1: np.ndarray   # f64 [E, S, 3]
    seg_a: np.ndarray    # f64 [E, S]
    seg_b: np.ndarray    # f64 [E, S]
    ntot: np.ndarray     # f64 [E]
    radius: np.ndarray   # f64 [E] mean member radius
    mat: np.ndarray      # f64 [E, 12] mean member material


def strand_tangents(P: np.ndarray) -> np.ndarray:
    """Unit tangent at every vertex: central difference inside, one-sided at
    the ends.

    Pinned by test_strand_tangents_on_a_circle.
    """
    d = np.empty_like(P)
    d[:, 1:-1] = P[:, 2:] - P[:, :-2]
    d[:, 0] = P[:, 1] - P[:, 0]
    d[:, -1] = P[:, -1] - P[:, -2]
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def degenerate_axis(q: np.ndarray, t: np.ndarray) -> np.ndarray:
    """READING (the two kept PCA axes have equal variance, e.g. two strands
    whose offset runs along the tangent, so the principal axis is undefined):
    e1 points to the member farthest from the centre in the plane normal to t
    (first such member in rank order), or along the Duff basis vector b1 of t
    when every member projects onto the centre.

    Pinned by test_degenerate_cross_section_axis.
    """
    qp = q - np.outer(q @ t, t)
    d2 = np.sum(qp * qp, 1)
    i = int(np.argmax(d2))
    if d2[i] > 0.0:
        return qp[i] / np.sqrt(d2[i])
    return duff_basis(t)[0]


def fit_cross_section(pts: np.ndarray, tans: np.ndarray, radii: np.ndarray):
    """Ellipse of one cross-section, Section 5.1 step 3 "Cross-section fitting".

    centre = mean of the k-th control points; tangent = normalised mean of the
    members' unit tangents; PCA of the points (covariance / n, numpy eigh);
    drop the eigenvector with the largest |v . t| (ties: lower index in
    ascending-eigenvalue order); e1 = the remaining one with the larger
    eigenvalue, made orthogonal to t; e2 = t x e1.
    READING (semi-axes, the paper's corner-point distance is unstated): a =
    max(|u| + r), b = max(|v| + r) over members, u, v their coordinates along
    e1, e2; both scaled by s = max sqrt((u/a)^2 + (v/b)^2) when s > 1 so the
    ellipse contains every member centre.

    Pinned by test_cross_section_closed_form,
    test_cross_section_contains_members_and_rotation_invariance and
    test_degenerate_cross_section_axis.
    """
    c = pts.mean(0)
    t = tans.sum(0)
    t = t / np.linalg.norm(t)
    q = pts - c
    cov = q.T @ q / pts.shape[0]
    w, V = np.linalg.eigh(cov)
    dots = np.abs(V.T @ t)
    drop = int(np.argmax(dots))
    keep = [i for i in range(3) if i != drop]
    if w[keep[1]] - w[keep[0]] <= 1e-9 * w[2] or w[2] <= 0.0:
        e1 = degenerate_axis(q, t)
    else:
        e1 = V[:, keep[1]]  # larger eigenvalue of the two kept (ascending order)
    e1 = e1 - np.dot(e1, t) * t
    e1 = e1 / np.linalg.norm(e1)
    e2 = np.cross(t, e1)
    u = q @ e1
    v = q @ e2
    a = np.max(np.abs(u) + radii)
    b = np.max(np.abs(v) + radii)
    s = np.max(np.sqrt((u / a) ** 2 + (v / b) ** 2))
    if s > 1.0:
        a *= s
        b *= s
    return c, t, e1, e2, a, b


def fit_eths(verts: np.ndarray, mat: np.ndarray, hier: Hierarchy, chunk: int = 512) -> ETHs:
    """Fit every thick hair of every level (FP64).  The thick hairs are
    processed in batches with members padded and masked; per cross-section the
    arithmetic is that of ``fit_cross_section`` (checked against it by the
    tests).

    Pinned by test_batched_fit_matches_single_fit (cross-sections) and, for the segment frame,
    test_thick_hair_segment_is_the_bundle_cylinder,
    test_tapered_thick_hair_takes_the_wider_section and test_bent_thick_hair_segment_frame.
    """
    P = verts[..., :3].astype(np.float64)
    R = verts[..., 3].astype(np.float64)
    T = strand_tangents(P)
    E = hier.n_eths
    S1 = P.shape[1]
    center = np.zeros((E, S1, 3))
    tangent = np.zeros((E, S1, 3))
    E1 = np.zeros((E, S1, 3))
    E2 = np.zeros((E, S1, 3))
    A = np.zeros((E, S1))
    B = np.zeros((E, S1))
    ntot = hier.eth_count.astype(np.float64)
    radius = np.zeros(E)
    emat = np.zeros((E, mat.shape[1]))
    live = np.nonzero(hier.eth_count > 0)[0]  # an empty thick hair has no fit
    for e0 in range(0, live.size, chunk):
        ee = live[e0:e0 + chunk]
        M = int(hier.eth_count[ee].max())
        idx = hier.eth_first_rank[ee][:, None] + np.arange(M)[None, :]
        mask = np.arange(M)[None, :] < hier.eth_count[ee][:, None]
        mem = hier.order[np.where(mask, idx, hier.eth_first_rank[ee][:, None])]
        n = hier.eth_count[ee].astype(np.float64)
        mk = mask[:, :, None].astype(np.float64)
        radius[ee] = (R[mem, 0] * mask).sum(1) / n
        emat[ee] = (mat[mem].astype(np.float64) * mk).sum(1) / n[:, None]
        pts = P[mem]                      # [b, M, S1, 3]
        tns = T[mem]
        rad = np.broadcast_to(R[mem, 0][:, :, None], R[mem].shape)  # strand radius
        m4 = mask[:, :, None, None]
        c = (pts * m4).sum(1) / n[:, None, None]
        t = (tns * m4).sum(1)
        t = t / np.linalg.norm(t, axis=-1, keepdims=True)
        q = (pts - c[:, None]) * m4
        cov = np.einsum("bmki,bmkj->bkij", q, q) / n[:, None, None, None]
        w, V = np.linalg.eigh(cov)        # ascending eigenvalues, vectors in columns
        dots = np.abs(np.einsum("bkij,bki->bkj", V, t))
        drop = np.argmax(dots, -1)
        keep = np.where(drop == 2, 1, 2)  # larger eigenvalue of the two kept
        keep0 = np.where(drop == 0, 1, 0)
        e1 = np.take_along_axis(V, keep[..., None, None], -1)[..., 0]
        wk1 = np.take_along_axis(w, keep[..., None], -1)[..., 0]
        wk0 = np.take_along_axis(w, keep0[..., None], -1)[..., 0]
        degen = (wk1 - wk0 <= 1e-9 * w[..., 2]) | (w[..., 2] <= 0.0)
        if degen.any():
            # see degenerate_axis(): farthest member in the plane normal to t
            qp = q - np.einsum("bmki,bki->bmk", q, t)[..., None] * t[:, None]
            d2 = np.where(mask[:, :, None], np.sum(qp * qp, -1), -1.0)
            far = np.argmax(d2, 1)                     # [b, S1], first max in rank order
            qf = np.take_along_axis(qp, far[:, None, :, None], 1)[:, 0]
            df = np.take_along_axis(d2, far[:, None, :], 1)[:, 0]
            b1 = duff_basis(t)[0]
            alt = np.where(df[..., None] > 0.0, qf / np.sqrt(np.maximum(df, 1e-300))[..., None], b1)
            e1 = np.where(degen[..., None], alt, e1)
        e1 = e1 - np.sum(e1 * t, -1, keepdims=True) * t
        e1 = e1 / np.linalg.norm(e1, axis=-1, keepdims=True)
        e2 = np.cross(t, e1)
        u = np.einsum("bmki,bki->bmk", q, e1)
        v = np.einsum("bmki,bki->bmk", q, e2)
        neg = np.where(mask[:, :, None], 0.0, -np.inf)
        a = np.max(np.abs(u) + rad + neg, 1)
        b = np.max(np.abs(v) + rad + neg, 1)
        s = np.max(np.sqrt((u / a[:, None]) ** 2 + (v / b[:, None]) ** 2) + neg, 1)
        sc = np.where(s > 1.0, s, 1.0)
        center[ee], tangent[ee], E1[ee], E2[ee] = c, t, e1, e2
        A[ee], B[ee] = a * sc, b * sc
    with np.errstate(invalid="ignore", divide="ignore"):
        ax = center[:, 1:] - center[:, :-1]
        ax = ax / np.linalg.norm(ax, axis=-1, keepdims=True)
        v = E1[:, :-1] - np.sum(E1[:, :-1] * ax, -1, keepdims=True) * ax
        seg_e1 = v / np.linalg.norm(v, axis=-1, keepdims=True)
    seg_e1[hier.eth_count == 0] = 0.0
    seg_a = np.maximum(A[:, :-1], A[:, 1:])
    seg_b = np.maximum(B[:, :-1], B[:, 1:])
    return ETHs(center=center, tangent=tangent, e1=E1, e2=E2, a=A, b=B, seg_e1=seg_e1,
                seg_a=seg_a, seg_b=seg_b, ntot=ntot, radius=radius, mat=emat)


# ------------------------------------------------------------------ LoD selection


def _f32(x):
    return np.asarray(x, np.float32)


def project_px(p: np.ndarray, cam: np.ndarray):
    """Pixel-plane coordinates of points p [.., 3] (float32, fixed order:
    relative position, then ((x*r0 + y*r1) + z*r2) per camera axis, then the
    perspective division and the pixel scale).  Returns (X, Y, depth).

    Pinned by test_width_orthographic_facing_camera and
    test_width_perspective_depth_scaling_and_near_plane.
    """
    p = _f32(p)
    cam = _f32(cam)
    rx = p[..., 0] - cam[4]
    ry = p[..., 1] - cam[5]
    rz = p[..., 2] - cam[6]

    def axis(o):
        return ((rx * cam[o]).astype(np.float32) + (ry * cam[o + 1]).astype(np.float32)
                ).astype(np.float32) + (rz * cam[o + 2]).astype(np.float32)

    xc = _f32(axis(7))
    yc = _f32(axis(10))
    zc = _f32(axis(13))
    if int(cam[0]) == 1:
        with np.errstate(divide="ignore", invalid="ignore"):
            X = _f32(_f32(xc / zc) * cam[3])
            Y = _f32(_f32(yc / zc) * cam[3])
    else:
        X = _f32(xc * cam[3])
        Y = _f32(yc * cam[3])
    return X, Y, zc


def cross_section_widths(eth: ETHs, cam: np.ndarray) -> np.ndarray:
    """Screen width l_w of every cross-section (Section 5.2 "Hair width
    calculation"): the four corner points c +- a e1, c +- b e2 (READING: the
    ends of the fitted axes stand for the corner control points) are projected
    and l_w is the largest pairwise xy distance in pixels.  float32 with a
    fixed operation order; a corner at or behind the near plane gives +inf.

    Pinned by test_width_orthographic_facing_camera and
    test_width_perspective_depth_scaling_and_near_plane.
    """
    c = _f32(eth.center)
    e1 = _f32(eth.e1)
    e2 = _f32(eth.e2)
    a = _f32(eth.a)[..., None]
    b = _f32(eth.b)[..., None]
    ae = _f32(a * e1)
    be = _f32(b * e2)
    corners = [_f32(c + ae), _f32(c - ae), _f32(c + be), _f32(c - be)]
    XY = [project_px(q, cam) for q in corners]
    w = np.zeros(c.shape[:-1], np.float32)
    for i in range(4):
        for j in range(i + 1, 4):
            dx = _f32(XY[i][0] - XY[j][0])
            dy = _f32(XY[i][1] - XY[j][1])
            d = np.sqrt(_f32(_f32(dx * dx) + _f32(dy * dy)))
            w = np.maximum(w, d)
    if int(cam[0]) == 1:
        near = np.float32(cam[16])
        behind = np.zeros(w.shape, bool)
        for q in XY:
            behind |= ~(q[2] > near)
        w = np.where(behind, np.float32(np.inf), w)
    return w.astype(np.float32)


def cluster_level_widths(hier: Hierarchy, eth: ETHs, cam: np.ndarray) -> np.ndarray:
    """w[c, L]: maximum cross-section width over the level-L thick hairs of
    cluster c (the per-cluster maximum the paper records with atomicMax).

    Pinned by test_cluster_level_widths_hand_worked.
    """
    w = cross_section_widths(eth, cam).max(1)
    out = np.zeros((hier.n_clusters, max(1, hier.n_levels)), np.float32)
    for e in range(hier.n_eths):
        if hier.eth_count[e] == 0:  # an empty thick hair has no width
            continue
        c = hier.eth_cluster[e]
        L = hier.eth_level[e]
        out[c, L] = max(out[c, L], w[e])
    return out


def select_lod_init(wcl: np.ndarray, eps: float, n_levels: int) -> np.ndarray:
    """Section 5.1 step 5: coarsest to finest, the first level whose maximum
    width is below eps; the strands (level n_levels) if none is.

    Pinned by test_init_rule_hand_worked.
    """
    eps = np.float32(eps)
    C = wcl.shape[0]
    lod = np.full(C, n_levels, np.uint8)
    for c in range(C):
        for L in range(n_levels):
            if wcl[c, L] < eps:
                lod[c] = L
                break
    return lod


def select_lod_deferred(wcl: np.ndarray, prev: np.ndarray, eps: float, n_levels: int,
                        hysteresis: bool = False) -> np.ndarray:
    """Eq. (14): L+1 if w_cur > eps; L if w_cur <= eps < w_cur-; L-1 if
    w_cur- <= eps; cases tested in that order.  READING: w_cur- is +inf at
    L = 0; at the strand level only the coarsening case applies; L stays in
    [0, n_levels].  READING (hysteresis=True, the paper's "approximately
    correct" deferred selection with a band): refine when w_cur > 1.1 eps and
    coarsen when w_cur- <= 0.9 eps, each threshold one float32 product.

    Pinned by test_deferred_rule_hand_worked and test_deferred_rule_with_hysteresis_hand_worked.
    """
    eps = np.float32(eps)
    refine = np.float32(eps * np.float32(1.1)) if hysteresis else eps
    coarsen = np.float32(eps * np.float32(0.9)) if hysteresis else eps
    out = np.array(prev, np.uint8).copy()
    for c in range(wcl.shape[0]):
        L = min(int(prev[c]), n_levels)
        wcur = wcl[c, L] if L < n_levels else -np.inf
        wminus = wcl[c, L - 1] if L > 0 else np.inf
        if L < n_levels and wcur > refine:
            L += 1
        elif wminus <= coarsen:
            L -= 1
        out[c] = L
    return out


def apply_budget(lod: np.ndarray, bias: int) -> np.ndarray:
    """READING (serving LoD budget): a bias b >= 0 coarsens every cluster by b
    levels, L <- max(0, L - b).

    Pinned by test_budget_bias.
    """
    return np.maximum(lod.astype(np.int64) - int(bias), 0).astype(np.uint8)


# ------------------------------------------------------------------ active primitives


def duff_basis(n: np.ndarray):
    """Orthonormal basis (b1, b2) around unit vectors n (Duff et al. 2017,
    "Building an orthonormal basis, revisited").

    Pinned by test_duff_basis_orthonormal_and_right_handed and test_duff_basis_values_at_the_poles.
    """
    sign = np.copysign(1.0, n[..., 2])
    a = -1.0 / (sign + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    b1 = np.stack([1.0 + sign * n[..., 0] * n[..., 0] * a, sign * b, -sign * n[..., 0]], -1)
    b2 = np.stack([b, sign + n[..., 1] * n[..., 1] * a, -n[..., 1]], -1)
    return b1, b2


def strand_prim_rows(verts: np.ndarray, shape: np.ndarray, strands: np.ndarray):
    """Primitive rows of every segment of the listed strands.

    Segment (s, k) runs from vertex k to k+1.  READING (cross-section of a
    strand): an ellipse of eccentricity e with the area of the circle of the
    area-equivalent radius r, a = r (1 - e^2)^(-1/4), b = r (1 - e^2)^(1/4),
    whose major axis e1 = cos(psi) b1 + sin(psi) b2 in the Duff basis of the
    segment direction.  Global id = s * S + k; material index = s.

    Pinned by test_strand_ellipse_area_and_eccentricity, test_strand_major_axis_orientation,
    test_strand_semi_axes_as_hit_distances and test_strand_record_fields_and_ids.
    """
    S = verts.shape[1] - 1
    strands = np.asarray(strands, np.int64)
    P = verts[strands, :, :3].astype(np.float64)
    r = verts[strands, 0, 3].astype(np.float64)
    e = shape[strands, 0].astype(np.float64)
    psi = shape[strands, 1].astype(np.float64)
    c0 = P[:, :-1]
    c1 = P[:, 1:]
    t = c1 - c0
    t = t / np.linalg.norm(t, axis=-1, keepdims=True)
    b1, b2 = duff_basis(t)
    e1 = np.cos(psi)[:, None, None] * b1 + np.sin(psi)[:, None, None] * b2
    q = (1.0 - e * e) ** 0.25
    a = (r / q)[:, None] * np.ones(S)
    b = (r * q)[:, None] * np.ones(S)
    n = strands.shape[0]
    rows = np.zeros((n, S, PRIM_STRIDE))
    rows[..., 0:3] = c0
    rows[..., 3:6] = c1
    rows[..., 6:9] = e1
    rows[..., 9] = a
    rows[..., 10] = b
    rows[..., 11] = 0.0
    rows[..., 12] = strands[:, None]
    rows[..., 13] = 1.0
    rows[..., 14] = r[:, None]
    ids = strands[:, None] * S + np.arange(S)[None, :]
    return rows.reshape(-1, PRIM_STRIDE), ids.reshape(-1)


def eth_prim_rows(eth: ETHs, eths: np.ndarray, n_strands: int, S: int):
    """Primitive rows of every segment of the listed thick hairs.  Global id =
    N S + e S + k; material index = N + e.

    Pinned by test_thick_hair_segment_is_the_bundle_cylinder,
    test_tapered_thick_hair_takes_the_wider_section and test_bent_thick_hair_segment_frame.
    """
    eths = np.asarray(eths, np.int64)
    n = eths.shape[0]
    rows = np.zeros((n, S, PRIM_STRIDE))
    rows[..., 0:3] = eth.center[eths, :-1]
    rows[..., 3:6] = eth.center[eths, 1:]
    rows[..., 6:9] = eth.seg_e1[eths]
    rows[..., 9] = eth.seg_a[eths]
    rows[..., 10] = eth.seg_b[eths]
    rows[..., 11] = 1.0
    rows[..., 12] = (n_strands + eths)[:, None]
    rows[..., 13] = eth.ntot[eths][:, None]
    rows[..., 14] = eth.radius[eths][:, None]
    ids = n_strands * S + eths[:, None] * S + np.arange(S)[None, :]
    return rows.reshape(-1, PRIM_STRIDE), ids.reshape(-1)


def active_set(n_strands: int, S: int, hier: Optional[Hierarchy], lod: Optional[np.ndarray]):
    """(strand ids, thick-hair ids) rendered at this LoD: every strand of a
    cluster at the strand level, the level-L thick hairs of a cluster at L.

    Pinned by test_active_set_hand_counted.
    """
    if hier is None or lod is None or hier.n_levels == 0:
        return np.arange(n_strands, dtype=np.int64), np.zeros(0, np.int64)
    lod = np.minimum(np.asarray(lod, np.int64), hier.n_levels)
    st = np.nonzero(lod[hier.cluster_of] == hier.n_levels)[0].astype(np.int64)
    eh = np.nonzero((lod[hier.eth_cluster] == hier.eth_level) & (hier.eth_count > 0))[0]
    eh = eh.astype(np.int64)
    return st, eh


# ------------------------------------------------------------------ rendering


@dataclasses.dataclass
class Prepared:
    rows: np.ndarray
    ids: np.ndarray
    mats: np.ndarray
    hier: Optional[Hierarchy]
    eth: Optional[ETHs]
    lod: Optional[np.ndarray]


def prepare(scene, n_clusters: int, lod_setting: str = "select", cam=None, eps_w: float = 2.0,
            lod: Optional[np.ndarray] = None, max_levels: int = 0, budget: int = 0) -> Prepared:
    """Hierarchy, fit, LoD and active primitive rows of a scene.

    Pinned by test_active_set_hand_counted (the rows and ids it lists) and, end to end, by the
    render pins.
    """
    N, S = scene.n_strands, scene.n_segments
    hier = eth = None
    if n_clusters > 0:
        hier = build_hierarchy(scene.verts[:, 0, :3], n_clusters, max_levels)
        if hier.n_levels > 0:
            eth = fit_eths(scene.verts, scene.mat, hier)
        if lod is None:
            if lod_setting == "select" and eth is not None:
                wcl = cluster_level_widths(hier, eth, cam)
                lod = select_lod_init(wcl, eps_w, hier.n_levels)
            else:
                import scenegen
                lod = scenegen.lod_preset(lod_setting, n_clusters, hier.n_levels)
        if lod is not None and budget:
            lod = apply_budget(lod, budget)
    st, eh = active_set(N, S, hier, lod)
    r1, i1 = strand_prim_rows(scene.verts, scene.shape, st)
    rows, ids = [r1], [i1]
    mats = [scene.mat.astype(np.float64)]
    if eth is not None:
        r2, i2 = eth_prim_rows(eth, eh, N, S)
        rows.append(r2)
        ids.append(i2)
        mats.append(eth.mat)
    return Prepared(np.ascontiguousarray(np.concatenate(rows)),
                    np.ascontiguousarray(np.concatenate(ids).astype(np.int64)),
                    np.ascontiguousarray(np.concatenate(mats)), hier, eth, lod)


def render_samples(prep: Prepared, cam: np.ndarray, lights: np.ndarray, samples: np.ndarray,
                   spp: int, K: int, seed: int, flags: int = 0, nq: int = 384,
                   threads: Optional[int] = None):
    """Radiance (f64 [m, 3]) and the global ids of the composited hits
    (int64 [m, K]: the K nearest, nearest first, cut after the first opaque
    strand hit, -1 padded) of the listed samples, by brute force over every
    active primitive.

    Pinned by test_kbuffer_keeps_the_nearest_in_order_and_breaks_ties_by_id,
    test_composite_front_to_back_with_closed_form_opacity,
    test_light_sum_point_and_directional_lights,
    test_thick_hair_shading_uses_the_hair_number_of_its_chord and
    tests/test_oracle_convergence.py.
    """
    samples = np.ascontiguousarray(samples, np.int64)
    m = samples.shape[0]
    rad = np.zeros((m, 3))
    hit = np.full((m, K), -1, np.int64)
    x, w = gauss_legendre(nq)
    camd = np.ascontiguousarray(cam, np.float64)
    L = np.ascontiguousarray(lights, np.float64)
    if threads is None:
        threads = os.cpu_count() or 1
    rc = _load().oracle_render(_pd(prep.rows), _pi64(prep.ids), prep.rows.shape[0],
                               _pd(prep.mats), prep.mats.shape[0], _pd(camd), _pd(L),
                               L.shape[0], _pi64(samples), m, spp, K, seed, flags, nq, _pd(x),
                               _pd(w), _pd(rad), _pi64(hit), threads)
    if rc != 0:
        raise RuntimeError(f"oracle_render failed with {rc}")
    return rad, hit


from .guides import (build_guided_hierarchy, guide_kmeans, nearest_guides,  # noqa: E402,F401
                     prism_weights, skin_points, strand_distance)
