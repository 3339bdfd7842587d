"""Seeded synthetic hair scenes, cameras, lights and sample lists.

This module only *makes inputs*.  It holds none of the rendering method's
arithmetic (no clustering, no ellipse fit, no LoD rule, no intersection, no
scattering model), so that the CPU oracle and the CUDA library can both consume
the same arrays while sharing no computation.

Randomness comes from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated as a counter-based
stream, so every array is a pure function of (seed, tag, index) and is the same
on any host.

Workload shapes follow the paper's experimental setup (Section 6: tens of
thousands of strands with 60k-120k typical, 256 clusters, 5-6 LoD levels,
epsilon_w = 2 px, 1024x1024 output) and the parameter ranges it prints for the
single-fibre lobes (Section 6: M_R 0.08-0.15, M_TT 0.12-0.3, N_TT 0.2-0.4 and
the RGB ranges of A_R, A_TT, A_D).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Material record layout shared by every consumer (12 floats per strand):
#   A_R(rgb) A_TT(rgb) A_D(rgb) beta_R beta_TT gamma_TT
MAT_STRIDE = 12


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64).copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, index) -> np.ndarray:
    """Output number ``index`` (0-based) of the SplitMix64 stream started at ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.asarray(index, dtype=np.uint64) + np.uint64(1)
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN)


class Stream:
    """A tagged SplitMix64 stream that hands out consecutive numbers."""

    def __init__(self, seed: int, tag: int):
        self.seed = int(splitmix64(seed ^ (tag * 0x632BE59BD9B4E019), 0))
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, np.arange(self.pos, self.pos + n, dtype=np.uint64))
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        """Standard normals by the Box-Muller transform."""
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------- scene


@dataclasses.dataclass
class Scene:
    """Strand hair input.

    verts : float32 [N, S+1, 4]  vertex xyz and area-equivalent radius r
    mat   : float32 [N, 12]      single-fibre lobe parameters (see MAT_STRIDE)
    shape : float32 [N, 2]       cross-section eccentricity e in [0, 1) and
                                 orientation angle psi (radians)
    """

    verts: np.ndarray
    mat: np.ndarray
    shape: np.ndarray
    name: str = ""

    @property
    def n_strands(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_segments(self) -> int:
        return int(self.verts.shape[1] - 1)

    def aabb(self):
        p = self.verts[..., :3].reshape(-1, 3)
        return p.min(0), p.max(0)


def _normalize(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def make_strands(n: int, S: int, *, seed: int, head_radius: float = 0.5,
                 cap_deg: float = 60.0, length: float = 1.0, jitter: float = 0.002,
                 curl_amp: float = 0.0, curl_turns: float = 3.0, radius: float = 1e-3,
                 droop: float = 1.6, spread: float = 0.35, straight: bool = False,
                 hang: float = 0.0) -> np.ndarray:
    """Polyline strands rooted on a spherical cap of a head sphere at the origin.

    Roots are uniform on the cap (polar angle <= cap_deg around +y).  Each strand
    grows along the scalp normal and droops toward -y; curls are a helix of
    seeded amplitude whose phase varies smoothly over the scalp, so that
    neighbouring strands curl together; every vertex but the root receives
    isotropic Gaussian jitter.
    """
    rs = Stream(seed, 1)
    cos_t = 1.0 - rs.uniform(n) * (1.0 - math.cos(math.radians(cap_deg)))
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = 2.0 * math.pi * rs.uniform(n)
    nrm = np.stack([sin_t * np.cos(phi), cos_t, sin_t * np.sin(phi)], -1)
    root = head_radius * nrm
    # horizontal part of the scalp normal, left unnormalised so that the flow
    # field is smooth over the crown (neighbouring strands stay together)
    horiz = nrm * np.array([1.0, 0.0, 1.0])
    down = np.array([0.0, -1.0, 0.0])

    s = (np.arange(S, dtype=np.float64) + 0.5) / S  # mid-parameter of each step
    if straight:
        d = np.repeat(nrm[:, None, :], S, 1)
    elif hang > 0.0:
        # rise along the scalp normal for a short length `hang`, then hang
        # down with a slight outward tilt (long hair falling in sheets)
        w_n = np.exp(-s / hang)[None, :, None]
        d = w_n * nrm[:, None, :] + (1.0 - w_n) * (spread * horiz[:, None, :] + down)
    else:
        d = (1.0 - s)[None, :, None] * nrm[:, None, :] + \
            (s[None, :, None] * droop) * (spread * horiz[:, None, :] + down)
    d = _normalize(d)
    steps = d * (length / S)
    verts = np.zeros((n, S + 1, 3))
    verts[:, 0] = root
    verts[:, 1:] = root[:, None, :] + np.cumsum(steps, 1)

    if curl_amp > 0.0:
        cs = Stream(seed, 2)
        # amplitude and phase vary smoothly over the scalp (clumps curl alike)
        amp = curl_amp * (1.0 + 0.2 * np.sin(7.0 * root[:, 0] + 5.0 * root[:, 2]))
        # smooth phase field over the scalp: neighbouring roots curl alike
        phase0 = 2.0 * math.pi * (1.5 * root[:, 0] + 1.1 * root[:, 2]) + 0.05 * cs.normal(n)
        u = _normalize(np.cross(nrm, np.array([0.0, 0.0, 1.0])) + np.array([1e-6, 0.0, 0.0]))
        v = _normalize(np.cross(nrm, u))
        sk = np.arange(S + 1, dtype=np.float64) / S
        ang = 2.0 * math.pi * curl_turns * sk[None, :] + phase0[:, None]
        ang0 = phase0[:, None]
        off = (np.cos(ang) - np.cos(ang0))[..., None] * u[:, None, :] + \
              (np.sin(ang) - np.sin(ang0))[..., None] * v[:, None, :]
        # curls grow in from the root
        verts += amp[:, None, None] * np.minimum(1.0, 4.0 * sk)[None, :, None] * off

    if jitter > 0.0:
        js = Stream(seed, 3)
        jit = js.normal(n * S * 3).reshape(n, S, 3) * jitter
        verts[:, 1:] += jit

    out = np.empty((n, S + 1, 4), dtype=np.float32)
    out[..., :3] = verts.astype(np.float32)
    out[..., 3] = np.float32(radius)
    return out


def _lerp(a, b, t):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return a[None, :] + (b - a)[None, :] * t[:, None]


def material_from_melanin(melanin: np.ndarray, roughness: np.ndarray) -> np.ndarray:
    """Map (melanin, roughness) to the 12 single-fibre lobe parameters.

    The paper prints only parameter ranges (Section 6); this input recipe maps
    melanin m in [0.1, 0.9] linearly onto those RGB ranges with t = (m-0.1)/0.8
    and roughness q in [0.1, 0.3] linearly onto the M_R, M_TT and N_TT ranges.
    The printed A ranges are read as lobe energies: a longitudinal Gaussian in
    theta_h has mass 2 over theta_o, so the attenuations A_p of Eq. 1 are half
    of them (otherwise the forward albedo of light hair exceeds 1 and the
    dual-scattering series of the B lobe diverge).
    """
    t = np.clip((np.asarray(melanin, np.float64) - 0.1) / 0.8, 0.0, 1.0)
    q = np.clip((np.asarray(roughness, np.float64) - 0.1) / 0.2, 0.0, 1.0)
    m = np.empty((t.shape[0], MAT_STRIDE))
    m[:, 0:3] = 0.5 * _lerp((0.03, 0.03, 0.03), (0.25, 0.25, 0.25), t)
    m[:, 3:6] = 0.5 * _lerp((0.25, 0.17, 0.07), (0.38, 0.25, 0.18), t)
    m[:, 6:9] = 0.5 * _lerp((0.20, 0.11, 0.10), (0.40, 0.21, 0.08), t)
    m[:, 9] = 0.08 + 0.07 * q
    m[:, 10] = 0.12 + 0.18 * q
    m[:, 11] = 0.20 + 0.20 * q
    return m.astype(np.float32)


def material_marschner(melanin: np.ndarray, roughness: np.ndarray) -> np.ndarray:
    """Lobe parameters for the Marschner R / TT / TRT single fibre (the
    paper's Section 7 extension): R and TT as in material_from_melanin, and the
    third attenuation triple holds A_TRT instead of A_D.  The paper prints no
    TRT range; this recipe maps melanin onto a TRT lobe energy from
    (0.20, 0.14, 0.08) (light) to (0.10, 0.06, 0.03) (dark), halved like the
    other lobe energies, so the fibre's forward plus backward albedo stays
    below 1 over the parameter box.
    """
    m = material_from_melanin(melanin, roughness).astype(np.float64)
    t = np.clip((np.asarray(melanin, np.float64) - 0.1) / 0.8, 0.0, 1.0)
    m[:, 6:9] = 0.5 * _lerp((0.20, 0.14, 0.08), (0.10, 0.06, 0.03), t)
    return m.astype(np.float32)


def material_absorption(n: int, sigma_a: float, beta: float) -> np.ndarray:
    """Grey fibre from an absorption and a longitudinal roughness.

    A_R is the normal-incidence Fresnel reflectance of a fibre of index 1.55,
    A_TT the two-interface transmission times exp(-2 sigma_a), and A_D splits
    the remainder; beta_R = beta, beta_TT = 1.5 beta, gamma_TT = 0.3.
    """
    fr = ((1.55 - 1.0) / (1.55 + 1.0)) ** 2
    att = (1.0 - fr) ** 2 * math.exp(-2.0 * sigma_a)
    ad = (1.0 - fr - att) / 2.0
    row = [fr] * 3 + [att] * 3 + [ad] * 3 + [beta, 1.5 * beta, 0.3]
    return np.tile(np.asarray(row, np.float32), (n, 1))


# --------------------------------------------------------------------------- camera


# camera record (float32[20]):
#   0 kind (0 ortho, 1 perspective)   1 width   2 height   3 pix_scale
#   4..6 eye   7..9 right   10..12 up   13..15 fwd   16 near   17..19 unused
CAM_FLOATS = 20


@dataclasses.dataclass
class Camera:
    kind: int
    width: int
    height: int
    eye: np.ndarray
    right: np.ndarray
    up: np.ndarray
    fwd: np.ndarray
    pix_scale: float  # pixels per unit of image-plane offset (tan-space for perspective)
    near: float = 1e-3

    def pack(self) -> np.ndarray:
        c = np.zeros(CAM_FLOATS, np.float32)
        c[0] = self.kind
        c[1] = self.width
        c[2] = self.height
        c[3] = self.pix_scale
        c[4:7] = self.eye
        c[7:10] = self.right
        c[10:13] = self.up
        c[13:16] = self.fwd
        c[16] = self.near
        return c


def look_at(eye, target, world_up=(0.0, 1.0, 0.0)):
    eye = np.asarray(eye, np.float64)
    fwd = _normalize(np.asarray(target, np.float64) - eye)
    right = _normalize(np.cross(fwd, np.asarray(world_up, np.float64)))
    up = np.cross(right, fwd)
    return fwd, right, up


def frame_camera(lo, hi, width: int, height: int, *, perspective: bool, fill: float,
                 fov_y_deg: float = 40.0) -> Camera:
    """Camera looking along -z at the AABB centre; the AABB height fills ``fill`` of the frame."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    ctr = 0.5 * (lo + hi)
    ext = hi - lo
    half_h = 0.5 * max(ext[1], ext[0] * height / width)
    if perspective:
        tan_h = math.tan(math.radians(0.5 * fov_y_deg))
        dist = half_h / (fill * tan_h) + 0.5 * ext[2]
        eye = ctr + np.array([0.0, 0.0, dist])
        fwd, right, up = look_at(eye, ctr)
        pix = 0.5 * height / tan_h
    else:
        eye = ctr + np.array([0.0, 0.0, 2.0 + ext[2]])
        fwd, right, up = look_at(eye, ctr)
        pix = 0.5 * height / (half_h / fill)
    return Camera(1 if perspective else 0, width, height,
                  eye.astype(np.float32), right.astype(np.float32), up.astype(np.float32),
                  fwd.astype(np.float32), float(np.float32(pix)))


# --------------------------------------------------------------------------- lights


# light record (float32[8]): xyz, type (0 directional: xyz = unit vector toward the
# light; 1 point: xyz = position), rgb intensity, unused
LIGHT_FLOATS = 8


def directional_light(direction, rgb=(1.0, 1.0, 1.0)) -> np.ndarray:
    d = _normalize(np.asarray(direction, np.float64))
    return np.array([[*d, 0.0, *rgb, 0.0]], np.float32)


def point_lights(count: int, center, *, radius: float = 3.0, seed: int = 0,
                 total_intensity: float = 9.0) -> np.ndarray:
    """Seeded point lights on a sphere around ``center`` (upper-front half)."""
    st = Stream(seed, 7)
    u = st.uniform(count)
    v = st.uniform(count)
    th = np.arccos(0.9 - 1.5 * u)  # bias toward the camera side
    ph = 2.0 * math.pi * v
    dirs = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph) * 0.5 + 0.3, np.cos(th)], -1)
    dirs = _normalize(dirs)
    pos = np.asarray(center, np.float64)[None, :] + radius * dirs
    out = np.zeros((count, LIGHT_FLOATS), np.float32)
    out[:, 0:3] = pos
    out[:, 3] = 1.0
    out[:, 4:7] = total_intensity / count
    return out


# --------------------------------------------------------------------------- workloads


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    camera: Camera
    lights: np.ndarray
    spp: int
    k_depth: int
    n_clusters: int          # 0 = no clustering (full strands)
    sample_seed: int = 1
    eps_w: float = 2.0
    lod_setting: str = "select"   # "select", "strands", "half", "eth"
    precision: int = 0            # 0 FP32 tables, 1 FP16 tables
    notes: str = ""


def tiny_strands(seed: int = 0) -> Workload:
    """64 strands x 16 segments on a unit-sphere cap, jitter 0.02, r = 4e-3;
    128x128 orthographic, 1 spp, one directional light, full strands."""
    v = make_strands(64, 16, seed=seed, head_radius=1.0, cap_deg=60.0, length=1.0,
                     jitter=0.02, radius=4e-3)
    n = v.shape[0]
    st = Stream(seed, 11)
    shape = np.stack([np.zeros(n), 2.0 * math.pi * st.uniform(n)], -1).astype(np.float32)
    sc = Scene(v, material_absorption(n, 0.3, 0.2), shape, "tiny")
    lo, hi = sc.aabb()
    cam = frame_camera(lo, hi, 128, 128, perspective=False, fill=0.8)
    return Workload("tiny_strands_64x16_128sq_1spp", sc, cam,
                    directional_light((1.0, 1.0, 1.0)), 1, 1, 0)


def clustered(n: int = 10000, S: int = 32, res: int = 512, spp: int = 4,
              lod_setting: str = "half", seed: int = 0, n_clusters: int = 256) -> Workload:
    """Wavy curls of amplitude ~0.05, eccentricity 0.8 at random orientation,
    256 Morton clusters; 512x512 perspective, 4 spp, two point lights."""
    v = make_strands(n, S, seed=seed, curl_amp=0.05, curl_turns=3.0, jitter=0.002,
                     radius=1e-3)
    st = Stream(seed, 12)
    shape = np.stack([np.full(n, 0.8), 2.0 * math.pi * st.uniform(n)], -1).astype(np.float32)
    mat = material_from_melanin(np.full(n, 0.5), np.full(n, 0.2))
    sc = Scene(v, mat, shape, "clusters")
    lo, hi = sc.aabb()
    cam = frame_camera(lo, hi, res, res, perspective=True, fill=0.8)
    lights = point_lights(2, 0.5 * (lo + hi), seed=seed)
    return Workload(f"clusters_{n}x{S}_{res}sq_{spp}spp_{lod_setting}", sc, cam, lights,
                    spp, 4, n_clusters, lod_setting=lod_setting)


def full_head(n: int = 100000, S: int = 64, width: int = 1920, height: int = 1080,
              spp: int = 8, n_lights: int = 8, n_clusters: int = 4096, seed: int = 0,
              precision: int = 0, fill: float = 0.15, cap_deg: float = 25.0) -> Workload:
    """Scalp patch of 100k strands x 64 segments, per-strand melanin U[0.1,0.9],
    roughness U[0.1,0.3], eccentricity U[0.6,1.0); 1920x1080, 8 spp, 8 point
    lights, LoD chosen per cluster by projected width (epsilon_w = 2 px).
    The default framing (hair 15% of the frame height) is the view at which
    the 2 px rule puts about a third of the clusters on thick hairs; at
    larger framings every cluster stays on strands."""
    v = make_strands(n, S, seed=seed, curl_amp=0.02, curl_turns=2.0, jitter=0.0004,
                     radius=1e-3, cap_deg=cap_deg, hang=0.08, spread=0.3)
    st = Stream(seed, 13)
    mel = 0.1 + 0.8 * st.uniform(n)
    rough = 0.1 + 0.2 * st.uniform(n)
    ecc = np.minimum(0.6 + 0.4 * st.uniform(n), 0.99)
    psi = 2.0 * math.pi * st.uniform(n)
    sc = Scene(v, material_from_melanin(mel, rough), np.stack([ecc, psi], -1).astype(np.float32),
               "full_head")
    lo, hi = sc.aabb()
    cam = frame_camera(lo, hi, width, height, perspective=True, fill=fill)
    lights = point_lights(n_lights, 0.5 * (lo + hi), seed=seed)
    tag = "fp16" if precision else "fp32"
    if fill != 0.15:
        tag += f"_fill{round(100 * fill)}"
    return Workload(f"full_head_{n}x{S}_{width}x{height}_{spp}spp_{tag}", sc, cam, lights,
                    spp, 4, n_clusters, lod_setting="select", precision=precision)


def stress(n: int = 500000, S: int = 64, width: int = 3840, height: int = 2160,
           spp: int = 16, n_clusters: int = 16384, seed: int = 0) -> Workload:
    """500k long straight strands x 64 segments, eccentricity 0.9, 16,384
    clusters; 3840x2160, 16 spp, 4 lights, k-buffer depth 8, FP16 tables."""
    v = make_strands(n, S, seed=seed, length=2.0, jitter=0.0, radius=1e-3, cap_deg=35.0,
                     hang=0.05, spread=0.25)
    st = Stream(seed, 14)
    psi = 2.0 * math.pi * st.uniform(n)
    mel = 0.1 + 0.8 * st.uniform(n)
    rough = 0.1 + 0.2 * st.uniform(n)
    sc = Scene(v, material_from_melanin(mel, rough),
               np.stack([np.full(n, 0.9), psi], -1).astype(np.float32), "stress")
    lo, hi = sc.aabb()
    cam = frame_camera(lo, hi, width, height, perspective=True, fill=0.3)
    lights = point_lights(4, 0.5 * (lo + hi), seed=seed)
    return Workload(f"stress_{n}x{S}_{width}x{height}_{spp}spp", sc, cam, lights, spp, 8,
                    n_clusters, lod_setting="select", precision=1)


def lod_preset(setting: str, n_clusters: int, n_eth_levels: int) -> Optional[np.ndarray]:
    """Fixed LoD settings of the clustered workload: every cluster on strands,
    every even cluster on its coarsest thick hair ("half"), or every cluster on
    its coarsest thick hair.  Returns None for "select" (use the selector)."""
    if setting == "select":
        return None
    lod = np.full(n_clusters, n_eth_levels, np.uint8)
    if setting == "eth":
        lod[:] = 0
    elif setting == "half":
        lod[0::2] = 0
    elif setting != "strands":
        raise ValueError(setting)
    return lod


# --------------------------------------------------------------------------- samples


def sample_subset(width: int, height: int, spp: int, count: int, *, seed: int = 5,
                  tiles: int = 0, tile: int = 16) -> np.ndarray:
    """Seeded sample ids ``pixel * spp + s`` (pixel = y * width + x): ``count``
    uniform picks plus ``tiles`` full tile x tile pixel blocks (all their samples)."""
    total = width * height * spp
    st = Stream(seed, 21)
    ids = [(st.u64(count) % np.uint64(total)).astype(np.int64)] if count else []
    for _ in range(tiles):
        x0 = int(st.u64(1)[0] % np.uint64(max(1, width - tile + 1)))
        y0 = int(st.u64(1)[0] % np.uint64(max(1, height - tile + 1)))
        ys, xs = np.meshgrid(np.arange(y0, min(height, y0 + tile)),
                             np.arange(x0, min(width, x0 + tile)), indexing="ij")
        pix = (ys * width + xs).reshape(-1)
        ids.append((pix[:, None] * spp + np.arange(spp)[None, :]).reshape(-1))
    if not ids:
        return np.zeros(0, np.int64)
    return np.unique(np.concatenate(ids)).astype(np.int64)


def pixel_samples(width: int, spp: int, pixels: np.ndarray) -> np.ndarray:
    """All sample ids of the listed pixel indices (pixel = y * width + x)."""
    pixels = np.asarray(pixels, np.int64)
    return (pixels[:, None] * spp + np.arange(spp)[None, :]).reshape(-1)


def serving_stream(count: int = 256, *, seed: int = 2, rate_hz: float = 50.0,
                   asset_sizes=(10000, 50000, 100000),
                   resolutions=((256, 256), (1280, 720), (1920, 1080)),
                   spp_range=(1, 8), budget_range=(0, 4)) -> List[dict]:
    """Seeded request stream: Poisson arrivals, asset, resolution, LoD budget, spp."""
    st = Stream(seed, 31)
    gaps = -np.log1p(-st.uniform(count)) / rate_hz
    arr = np.cumsum(gaps)
    a = st.u64(count) % np.uint64(len(asset_sizes))
    r = st.u64(count) % np.uint64(len(resolutions))
    sp = spp_range[0] + (st.u64(count) % np.uint64(spp_range[1] - spp_range[0] + 1))
    bd = budget_range[0] + (st.u64(count) % np.uint64(budget_range[1] - budget_range[0] + 1))
    out = []
    for i in range(count):
        out.append(dict(arrival_s=float(arr[i]), asset=int(a[i]),
                        width=int(resolutions[int(r[i])][0]), height=int(resolutions[int(r[i])][1]),
                        spp=int(sp[i]), budget=int(bd[i]), seed=int(1000 + i)))
    return out
