"""ctypes binding of libhairrt.so (include/hairrt.h).

Argument marshalling only: every function here converts Python arguments
(numpy arrays, torch tensors, plain numbers) into the C ABI's pointers and
structs, calls the same-named C entry point and turns a non-OK status into
``HairRTError``.  All computation happens in the library's CUDA kernels.  If
the library is missing, the first call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhairrt.so")

c_float = ctypes.c_float
c_u32 = ctypes.c_uint32
c_i32 = ctypes.c_int32
c_u64 = ctypes.c_uint64
c_int = ctypes.c_int
c_void_p = ctypes.c_void_p

HR_OK, HR_EINVAL, HR_ENOMEM, HR_ECUDA, HR_ENOTREADY, HR_ETIMEOUT, HR_EBUSY, HR_ESTATE = range(8)
STATUS_NAMES = ["HR_OK", "HR_EINVAL", "HR_ENOMEM", "HR_ECUDA", "HR_ENOTREADY", "HR_ETIMEOUT",
                "HR_EBUSY", "HR_ESTATE"]
HR_MAT_FLOATS = 12
HR_MAX_LIGHTS = 16
HR_MAX_K = 8
HR_PREC_FP32 = 0
HR_PREC_FP16 = 1
HR_FLAG_NO_S = 1
HR_FLAG_SINGLE_ON_ETH = 2
HR_FLAG_SHADOWS = 4
HR_FLAG_TRT = 8
HR_FLAG_COUNT = 256
HR_FLAG_REFIT = 512
HR_FLAG_DEFERRED_LOD = 1024
HR_FLAG_LOD_HYSTERESIS = 2048
HR_FLAG_KEEP_HIERARCHY = 4096
HR_FLAG_FIXED_TILE_ORDER = 8192


class HairRTError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class hr_hair_desc(ctypes.Structure):
    _fields_ = [("n_strands", c_u32), ("n_segments", c_u32), ("vertices", c_void_p),
                ("material", c_void_p), ("shape", c_void_p)]


class hr_camera(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("width", c_u32), ("height", c_u32), ("pix_scale", c_float),
                ("eye", c_float * 3), ("right", c_float * 3), ("up", c_float * 3),
                ("fwd", c_float * 3), ("near_plane", c_float)]


class hr_light(ctypes.Structure):
    _fields_ = [("xyz", c_float * 3), ("type", c_float), ("rgb", c_float * 3), ("pad", c_float)]


class hr_render_desc(ctypes.Structure):
    _fields_ = [("camera", hr_camera), ("spp", c_u32), ("k_depth", c_u32), ("seed", c_u64),
                ("n_lights", c_u32), ("lights", hr_light * HR_MAX_LIGHTS), ("precision", c_i32),
                ("flags", c_u32)]


class hr_stats(ctypes.Structure):
    _fields_ = [("render_ms", ctypes.c_double), ("n_samples", c_u64), ("n_active_prims", c_u32),
                ("n_eth_prims", c_u32), ("n_strand_prims", c_u32), ("stack_overflows", c_u32),
                ("node_visits", c_u64), ("prim_tests", c_u64), ("strand_shades", c_u64),
                ("eth_shades", c_u64), ("shaded_hits", c_u64), ("traced_samples", c_u64),
                ("hierarchy_ms", ctypes.c_double), ("fit_ms", ctypes.c_double),
                ("lod_ms", ctypes.c_double), ("bvh_ms", ctypes.c_double),
                ("bvh_refit", c_u32), ("lod_deferred", c_u32),
                ("refined_tests", c_u64), ("refined_entries", c_u64),
                ("heavy_tiles", c_u32), ("reserved", c_u32)]


class hr_tile_record(ctypes.Structure):
    _fields_ = [("t_start_ns", c_u64), ("t_end_ns", c_u64), ("tile", c_u32), ("sm", c_u32),
                ("max_node_visits", c_u32), ("max_prim_tests", c_u32)]


class hr_request(ctypes.Structure):
    _fields_ = [("asset", c_void_p), ("desc", hr_render_desc), ("eps_w_px", c_float),
                ("budget_bias", c_i32), ("rgb_out", c_void_p)]


class hr_result(ctypes.Structure):
    _fields_ = [("status", c_int), ("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double), ("n_samples", c_u64)]


P = c_void_p
_SIGS = {
    "hr_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_u64, c_void_p]),
    "hr_destroy": (c_int, [P]),
    "hr_last_error": (ctypes.c_char_p, [P]),
    "hr_bytes_in_use": (c_u64, [P]),
    "hr_kernel_launches": (c_u64, [P]),
    "hr_asset_create": (c_int, [P, ctypes.POINTER(hr_hair_desc), ctypes.POINTER(c_void_p)]),
    "hr_asset_destroy": (c_int, [P, P]),
    "hr_asset_update": (c_int, [P, P, P]),
    "hr_build_clusters": (c_int, [P, P, c_u32, c_u32, P, P]),
    "hr_hierarchy_info": (c_int, [P, P, ctypes.POINTER(c_u32), ctypes.POINTER(c_u32),
                                  ctypes.POINTER(c_u32)]),
    "hr_eth_export": (c_int, [P, P, P, P, P]),
    "hr_lod_widths": (c_int, [P, P, ctypes.POINTER(hr_camera), P]),
    "hr_select_lod": (c_int, [P, P, ctypes.POINTER(hr_camera), c_float, c_int, c_int, P]),
    "hr_build_bvh": (c_int, [P, P, P]),
    "hr_bvh_export": (c_int, [P, P, P, ctypes.POINTER(c_u32)]),
    "hr_sort_pairs": (c_int, [P, P, P, c_u32, c_u32, c_int]),
    "hr_table_export": (c_int, [P, P, P, ctypes.POINTER(c_u32), ctypes.POINTER(c_u32)]),
    "hr_build_guided_clusters": (c_int, [P, P, c_u32, c_u32, c_u32, P, P]),
    "hr_guides_export": (c_int, [P, P, P, P]),
    "hr_asset_skin": (c_int, [P, P, P]),
    "hr_vertex_export": (c_int, [P, P, P]),
    "hr_im_lookup": (c_int, [P, P, P, c_u32, c_int, P]),
    "hr_render": (c_int, [P, P, ctypes.POINTER(hr_render_desc), P, ctypes.POINTER(hr_stats)]),
    "hr_render_samples": (c_int, [P, P, ctypes.POINTER(hr_render_desc), P, c_u32, P, P]),
    "hr_frame_times": (c_int, [P, c_u32, P, P, P, ctypes.POINTER(c_u32)]),
    "hr_render_profile": (c_int, [P, P, ctypes.POINTER(hr_render_desc), P, ctypes.POINTER(hr_stats),
                                  P, c_u32, ctypes.POINTER(c_u32)]),
    "hr_render_frame": (c_int, [P, P, c_u32, c_float, c_int, ctypes.POINTER(hr_render_desc), P,
                                ctypes.POINTER(hr_stats)]),
    "hr_serve_start": (c_int, [P, c_u32, c_u64]),
    "hr_serve_stop": (c_int, [P]),
    "hr_submit": (c_int, [P, ctypes.POINTER(hr_request), ctypes.POINTER(c_u64)]),
    "hr_poll": (c_int, [P, c_u64, c_int, ctypes.POINTER(hr_result)]),
    "hr_serve_inject": (c_int, [P, c_int, ctypes.c_int64]),
    "hr_morton_clusters_noalloc": (c_int, [P, c_u32, c_u32, c_u32, P, P, P]),
}

_lib = None


def load(path: Optional[str] = None):
    """Load libhairrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_2405_10565_gb300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ptr(x) -> Optional[int]:
    """Address of a numpy array or torch tensor (None passes through)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _check(ctx, st: int, what: str):
    if st != HR_OK:
        msg = ""
        if ctx:
            m = load().hr_last_error(ctx)
            msg = m.decode() if m else ""
        raise HairRTError(st, f"{what}: {msg}")


# ---------------------------------------------------------------- struct builders


def camera(rec) -> hr_camera:
    """hr_camera from a packed float32[20] camera record (scenegen layout)."""
    r = np.asarray(rec, np.float32)
    c = hr_camera()
    c.kind = int(r[0])
    c.width = int(r[1])
    c.height = int(r[2])
    c.pix_scale = float(r[3])
    for i in range(3):
        c.eye[i] = float(r[4 + i])
        c.right[i] = float(r[7 + i])
        c.up[i] = float(r[10 + i])
        c.fwd[i] = float(r[13 + i])
    c.near_plane = float(r[16])
    return c


def render_desc(cam_rec, lights, spp: int, k_depth: int, seed: int, precision: int = 0,
                flags: int = 0) -> hr_render_desc:
    d = hr_render_desc()
    d.camera = camera(cam_rec)
    d.spp = spp
    d.k_depth = k_depth
    d.seed = seed
    L = np.asarray(lights, np.float32).reshape(-1, 8)
    if not 1 <= L.shape[0] <= HR_MAX_LIGHTS:
        raise ValueError("1..16 lights")
    d.n_lights = L.shape[0]
    for i in range(L.shape[0]):
        for j in range(3):
            d.lights[i].xyz[j] = float(L[i, j])
            d.lights[i].rgb[j] = float(L[i, 4 + j])
        d.lights[i].type = float(L[i, 3])
    d.precision = precision
    d.flags = flags
    return d


# ---------------------------------------------------------------- entry points


def hr_create(device: int = 0, hbm_budget: int = 0, stream: Optional[int] = None) -> int:
    h = c_void_p()
    _check(None, load().hr_create(ctypes.byref(h), device, hbm_budget, stream), "hr_create")
    return h.value


def hr_destroy(ctx: int) -> None:
    _check(None, load().hr_destroy(ctx), "hr_destroy")


def hr_last_error(ctx: int) -> str:
    m = load().hr_last_error(ctx)
    return m.decode() if m else ""


def hr_bytes_in_use(ctx: int) -> int:
    return int(load().hr_bytes_in_use(ctx))


def hr_kernel_launches(ctx: int) -> int:
    return int(load().hr_kernel_launches(ctx))


def hr_asset_create(ctx: int, vertices, material, shape) -> int:
    """vertices [N, S+1, 4], material [N, 12], shape [N, 2] float32 (host or device)."""
    n, s1 = int(vertices.shape[0]), int(vertices.shape[1])
    d = hr_hair_desc(n, s1 - 1, ptr(vertices), ptr(material), ptr(shape))
    h = c_void_p()
    _check(ctx, load().hr_asset_create(ctx, ctypes.byref(d), ctypes.byref(h)), "hr_asset_create")
    return h.value


def hr_asset_destroy(ctx: int, asset: int) -> None:
    _check(ctx, load().hr_asset_destroy(ctx, asset), "hr_asset_destroy")


def hr_asset_update(ctx: int, asset: int, vertices) -> None:
    """New vertices [N, S+1, 4] float32 (host or device) in the asset's sizes."""
    _check(ctx, load().hr_asset_update(ctx, asset, ptr(vertices)), "hr_asset_update")


def hr_build_clusters(ctx: int, asset: int, n_clusters: int, max_levels: int = 0,
                      cluster_of_out=None, order_out=None) -> None:
    _check(ctx, load().hr_build_clusters(ctx, asset, n_clusters, max_levels, ptr(cluster_of_out),
                                         ptr(order_out)), "hr_build_clusters")


def hr_hierarchy_info(ctx: int, asset: int):
    c, l, e = c_u32(), c_u32(), c_u32()
    _check(ctx, load().hr_hierarchy_info(ctx, asset, ctypes.byref(c), ctypes.byref(l),
                                         ctypes.byref(e)), "hr_hierarchy_info")
    return c.value, l.value, e.value


def hr_eth_export(ctx: int, asset: int, xsec=None, counts=None, mat=None) -> None:
    _check(ctx, load().hr_eth_export(ctx, asset, ptr(xsec), ptr(counts), ptr(mat)),
           "hr_eth_export")


def hr_lod_widths(ctx: int, asset: int, cam_rec, width_out) -> None:
    c = camera(cam_rec)
    _check(ctx, load().hr_lod_widths(ctx, asset, ctypes.byref(c), ptr(width_out)),
           "hr_lod_widths")


def hr_select_lod(ctx: int, asset: int, cam_rec, eps_w_px: float, mode: int, budget_bias: int,
                  lod_inout) -> None:
    c = camera(cam_rec)
    _check(ctx, load().hr_select_lod(ctx, asset, ctypes.byref(c), eps_w_px, mode, budget_bias,
                                     ptr(lod_inout)), "hr_select_lod")


def hr_build_bvh(ctx: int, asset: int, lod=None) -> None:
    _check(ctx, load().hr_build_bvh(ctx, asset, ptr(lod)), "hr_build_bvh")


def hr_sort_pairs(ctx: int, keys, vals, n: int, bits: int, count_earlier: bool = False) -> None:
    """Stable in-place radix sort of device uint32 (key, value) pairs on the
    low `bits` key bits (test export of the library's sort)."""
    _check(ctx, load().hr_sort_pairs(ctx, ptr(keys), ptr(vals), n, bits, 1 if count_earlier else 0),
           "hr_sort_pairs")


def hr_table_export(ctx: int, im32_out=None, im16_out=None):
    """Copy the baked IM(theta, beta) tables out (test export): FP32 values and
    the FP16 copy's half bit patterns, each [n_beta, n_theta] (host or
    device), either optional.  Returns (n_theta, n_beta)."""
    nt, nb = c_u32(), c_u32()
    _check(ctx, load().hr_table_export(ctx, ptr(im32_out), ptr(im16_out), ctypes.byref(nt),
                                       ctypes.byref(nb)), "hr_table_export")
    return nt.value, nb.value


def hr_im_lookup(ctx: int, theta, beta, out, precision: int = 0) -> None:
    """The shading code's bilinear IM lookup at the points (theta[k], beta[k])
    (test export); float32 arrays, host or device."""
    m = int(theta.shape[0])
    _check(ctx, load().hr_im_lookup(ctx, ptr(theta), ptr(beta), m, precision, ptr(out)),
           "hr_im_lookup")


def hr_build_guided_clusters(ctx: int, asset: int, n_guides: int, iterations: int = 8,
                             max_levels: int = 0, cluster_of_out=None, order_out=None) -> None:
    """Guide k-means, clusters of strands sharing their three nearest guides,
    thick-hair fits and skinning weights (Section 5.1)."""
    _check(ctx, load().hr_build_guided_clusters(ctx, asset, n_guides, iterations, max_levels,
                                                ptr(cluster_of_out), ptr(order_out)),
           "hr_build_guided_clusters")


def hr_guides_export(ctx: int, asset: int, guides_out=None, cluster_guides_out=None) -> None:
    _check(ctx, load().hr_guides_export(ctx, asset, ptr(guides_out), ptr(cluster_guides_out)),
           "hr_guides_export")


def hr_asset_skin(ctx: int, asset: int, guide_vertices) -> None:
    """Move the hair with new guide vertices [n_guides, S+1, 4] (Section 5.2)."""
    _check(ctx, load().hr_asset_skin(ctx, asset, ptr(guide_vertices)), "hr_asset_skin")


def hr_vertex_export(ctx: int, asset: int, verts_out) -> None:
    _check(ctx, load().hr_vertex_export(ctx, asset, ptr(verts_out)), "hr_vertex_export")


def hr_bvh_export(ctx: int, asset: int, leaf_ids=None) -> int:
    n = c_u32()
    _check(ctx, load().hr_bvh_export(ctx, asset, ptr(leaf_ids), ctypes.byref(n)), "hr_bvh_export")
    return n.value


def hr_render(ctx: int, asset: int, desc: hr_render_desc, rgb_out, stats: bool = False):
    st = hr_stats() if stats else None
    _check(ctx, load().hr_render(ctx, asset, ctypes.byref(desc), ptr(rgb_out),
                                 ctypes.byref(st) if st is not None else None), "hr_render")
    return st


def hr_frame_times(ctx: int, n: int, with_flags: bool = False):
    """Frame-kernel and fit times (ms) of the last n hr_render_frame calls,
    oldest first (numpy float32 arrays), and with with_flags their flags
    (bit 0 fitted, bit 1 refit the BVH)."""
    import numpy as np
    f = np.zeros(max(int(n), 1), np.float32)
    g = np.zeros(max(int(n), 1), np.float32)
    fl = np.zeros(max(int(n), 1), np.uint32)
    m = c_u32(0)
    _check(ctx, load().hr_frame_times(ctx, int(n), f.ctypes.data, g.ctypes.data, fl.ctypes.data,
                                      ctypes.byref(m)), "hr_frame_times")
    out = (f[:m.value].copy(), g[:m.value].copy())
    return out + (fl[:m.value].copy(),) if with_flags else out


def hr_render_profile(ctx: int, asset: int, desc: hr_render_desc, rgb_out, capacity: int):
    """Counting render with per-warp-tile records: returns (hr_stats, records as
    a numpy structured array [min(capacity, tiles)], number of tiles)."""
    import numpy as np
    st = hr_stats()
    buf = (hr_tile_record * max(int(capacity), 1))()
    nt = c_u32(0)
    _check(ctx, load().hr_render_profile(ctx, asset, ctypes.byref(desc), ptr(rgb_out),
                                         ctypes.byref(st), ctypes.cast(buf, c_void_p),
                                         int(capacity), ctypes.byref(nt)), "hr_render_profile")
    n = min(int(nt.value), int(capacity))
    dt = np.dtype([("t_start_ns", np.uint64), ("t_end_ns", np.uint64), ("tile", np.uint32),
                   ("sm", np.uint32), ("max_node_visits", np.uint32), ("max_prim_tests", np.uint32)])
    rec = np.frombuffer(buf, dtype=dt, count=max(int(capacity), 1))[:n].copy()
    return st, rec, int(nt.value)


def hr_render_samples(ctx: int, asset: int, desc: hr_render_desc, sample_ids, radiance_out,
                      hit_out) -> None:
    """radiance_out [m, 3] float32, hit_out [m, k_depth] int32 (host or device)."""
    m = int(sample_ids.shape[0])
    _check(ctx, load().hr_render_samples(ctx, asset, ctypes.byref(desc), ptr(sample_ids), m,
                                         ptr(radiance_out), ptr(hit_out)), "hr_render_samples")


def hr_render_frame(ctx: int, asset: int, n_clusters: int, eps_w_px: float, budget_bias: int,
                    desc: hr_render_desc, rgb_out, stats: bool = False):
    st = hr_stats() if stats else None
    _check(ctx, load().hr_render_frame(ctx, asset, n_clusters, eps_w_px, budget_bias,
                                       ctypes.byref(desc), ptr(rgb_out),
                                       ctypes.byref(st) if st is not None else None),
           "hr_render_frame")
    return st


def hr_serve_start(ctx: int, max_slots: int, max_batch_samples: int) -> None:
    _check(ctx, load().hr_serve_start(ctx, max_slots, max_batch_samples), "hr_serve_start")


def hr_serve_stop(ctx: int) -> None:
    _check(ctx, load().hr_serve_stop(ctx), "hr_serve_stop")


def hr_submit(ctx: int, asset: int, desc: hr_render_desc, rgb_out, eps_w_px: float = 2.0,
              budget_bias: int = 0) -> int:
    r = hr_request()
    r.asset = asset
    r.desc = desc
    r.eps_w_px = eps_w_px
    r.budget_bias = budget_bias
    r.rgb_out = ptr(rgb_out)
    t = c_u64()
    _check(ctx, load().hr_submit(ctx, ctypes.byref(r), ctypes.byref(t)), "hr_submit")
    return t.value


def hr_poll(ctx: int, ticket: int, timeout_ms: int = 0):
    """(status, hr_result).  HR_OK, HR_ENOTREADY and HR_ETIMEOUT are returned,
    other statuses raise."""
    res = hr_result()
    st = load().hr_poll(ctx, ticket, timeout_ms, ctypes.byref(res))
    if st not in (HR_OK, HR_ENOTREADY, HR_ETIMEOUT):
        _check(ctx, st, "hr_poll")
    return st, res


def hr_serve_inject(ctx: int, kind: int, arg: int = 0) -> None:
    _check(ctx, load().hr_serve_inject(ctx, kind, arg), "hr_serve_inject")


HR_NOALLOC_MAX_STRANDS = 1048576


def hr_morton_clusters_noalloc(vertices, n_clusters: int, order_out, cluster_of_out,
                               stream: Optional[int] = None) -> None:
    """Allocation-free Morton clustering; every buffer is device memory."""
    n, s1 = int(vertices.shape[0]), int(vertices.shape[1])
    _check(None, load().hr_morton_clusters_noalloc(ptr(vertices), n, s1 - 1, n_clusters,
                                                   ptr(order_out), ptr(cluster_of_out), stream),
           "hr_morton_clusters_noalloc")


def header_functions(header_path: Optional[str] = None) -> Sequence[str]:
    """Names of the functions declared in include/hairrt.h."""
    import re
    hp = header_path or os.path.join(_HERE, "..", "include", "hairrt.h")
    txt = open(hp).read()
    return sorted(set(re.findall(r"^\s*(?:hr_status|const char\*|uint64_t)\s+(hr_\w+)\s*\(",
                                 txt, re.M)))
