/*
 * hairrt.h — C ABI of the level-of-detail strand-hair ray tracer.
 *
 * Method: "Real-time Level-of-detail Strand-based Hair Rendering"
 * (Huang, Zhou, Lin, Zhu, Yan, Wu; arXiv 2405.10565).  Each pixel sample is
 * traced against a scene that mixes single hair strands and clustered
 * elliptical thick hairs (ETHs); the K nearest hits are found with ray versus
 * elliptic-cylinder-segment tests over a BVH, shaded with the single-fibre
 * BCSDF (Eq. 1) or the aggregated BCSDF (Eq. 5-13) and composited front to
 * back.  Every computation runs in this library's own CUDA kernels on one
 * GPU; there is no CPU fallback.
 *
 * Conventions that hold for every call:
 *  - Every call returns an hr_status; HR_OK is success.  On failure the
 *    library keeps a message readable with hr_last_error(ctx).  No C++
 *    exception crosses the boundary.
 *  - Work is ordered on the context's CUDA stream.  Calls that return data to
 *    the caller (host outputs, hr_stats, hr_poll) synchronise that stream
 *    before returning; calls that write caller device buffers do not, unless
 *    stated.
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes: device (or managed) memory is written on the
 *    stream, anything else is treated as host memory.
 *  - Output buffers are caller-owned.  The library owns the device copies it
 *    makes of inputs and frees them in hr_asset_destroy / hr_destroy.
 *  - Array layouts are dense, C order, little-endian, 32-bit floats unless
 *    stated.
 */
#ifndef HAIRRT_H
#define HAIRRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hr_status {
  HR_OK = 0,
  HR_EINVAL = 1,     /* bad argument (null pointer, size out of range, bad enum) */
  HR_ENOMEM = 2,     /* device allocation failed or the context's HBM budget is exceeded */
  HR_ECUDA = 3,      /* a CUDA runtime call or kernel failed; see hr_last_error */
  HR_ENOTREADY = 4,  /* hr_poll: the request has not finished yet */
  HR_ETIMEOUT = 5,   /* hr_poll: the wait ran out; a kernel's bounded wait gave up */
  HR_EBUSY = 6,      /* the serving queue is full */
  HR_ESTATE = 7      /* call made in the wrong order (e.g. render before hr_build_bvh) */
} hr_status;

typedef struct hr_ctx hr_ctx;
typedef struct hr_asset hr_asset;

/* Material record per strand: 12 floats
 *   A_R(r,g,b) A_TT(r,g,b) A_D(r,g,b) beta_R beta_TT gamma_TT
 * the attenuations and Gaussian widths (standard deviations, radians) of the
 * single-fibre lobes R, TT and D (Eq. 1; M_R, M_TT as G(beta, theta_h),
 * N_TT as G(gamma_TT, phi - pi)). */
#define HR_MAT_FLOATS 12

/* A strand hair model (Section 5.1 "Given a strand-based hair model").
 *   vertices : [n_strands][n_segments + 1][4] = x, y, z, r (r: area-equivalent
 *              fibre radius; only the root vertex's r is read)
 *   material : [n_strands][HR_MAT_FLOATS]
 *   shape    : [n_strands][2] = eccentricity e in [0, 1), orientation psi
 *              (radians) of the elliptical cross-section (a = r (1-e^2)^-1/4,
 *              b = r (1-e^2)^1/4, major axis rotated by psi in the segment's
 *              Duff et al. 2017 orthonormal basis)
 * The three arrays are host or device memory. */
typedef struct hr_hair_desc {
  uint32_t n_strands;
  uint32_t n_segments;
  const float* vertices;
  const float* material;
  const float* shape;
} hr_hair_desc;

/* Camera.  kind 0: orthographic, 1: perspective.  right/up/fwd are an
 * orthonormal basis; pix_scale converts image-plane offsets to pixels
 * (perspective: pixels per unit of tangent, i.e. (height/2)/tan(fov_y/2);
 * orthographic: pixels per world unit).  near_plane: depth below which a
 * corner point gives an infinite LoD width.  A sample of pixel (x, y) at
 * sub-pixel position (jx, jy) looks through image-plane offset
 * ((x + jx - width/2) / pix_scale, (height/2 - y - jy) / pix_scale). */
typedef struct hr_camera {
  int32_t kind;
  uint32_t width, height;
  float pix_scale;
  float eye[3];
  float right[3];
  float up[3];
  float fwd[3];
  float near_plane;
} hr_camera;

/* Light: type 0 directional (xyz = unit vector toward the light, irradiance
 * rgb), type 1 point (xyz = position, intensity rgb, 1/d^2 falloff). */
typedef struct hr_light {
  float xyz[3];
  float type;
  float rgb[3];
  float pad;
} hr_light;

#define HR_MAX_LIGHTS 16
#define HR_MAX_K 8

/* Precision of the scattering lookups (spec precision form): FP32
 * tables and FP32 lobe Gaussians, or FP16 longitudinal-integral and
 * Gaussian-lobe tables accumulated in FP32.  Traversal and intersection are
 * FP32 in both. */
#define HR_PREC_FP32 0
#define HR_PREC_FP16 1

/* Render flags (ablations of Section 7, "S-term" figure). */
#define HR_FLAG_NO_S 1u          /* drop the shadowing-masking term S of Eq. 13 */
#define HR_FLAG_SINGLE_ON_ETH 2u /* shade thick hairs with the single-fibre BCSDF */
/* Dual-scattering light paths (Section 3.2; the hairs on a shadow path found
 * by ray shooting as in Section 6): per hit and light a shadow ray toward the
 * light crosses hairs; T = d_F prod a_F^n over them (d_F = 0.7, a strand
 * counts one hair, a thick hair n = rho l sqrt(n_tot / (pi a b)) for its
 * chord l, a_F at incidence |asin(w . t)|; the shading hair itself is
 * skipped) scales the light, and the hairs' forward spread variances widen
 * every lobe of the shading BCSDF.  Off: primary hits only. */
#define HR_FLAG_SHADOWS 4u
/* Marschner R / TT / TRT single fibre (Section 7, "Extending to Marschner
 * model with TRT term"), in f_single and inside the aggregate f_ours: the
 * material's third attenuation triple is A_TRT and the third lobe is
 * A_TRT G(2 beta_R, theta_h) / 2 pi (width 2 beta_R after Marschner et al.
 * 2003, uniform azimuth as the paper's R lobe) instead of the diffuse
 * A_D / 2 pi^2; it enters a_F, a_B and the forward spread like the other
 * lobes, and the TRT^ lobe of a thick hair is widened and attenuated as R^. */
#define HR_FLAG_TRT 8u
/* Counting build: hr_render also counts node visits, primitive tests and
 * shading evaluations into hr_stats (slower; used to derive the algorithmic
 * FLOP count of a frame). */
#define HR_FLAG_COUNT 256u
/* hr_render_frame options for animated hair (a new frame of the same asset
 * after hr_asset_update):
 *  - HR_FLAG_REFIT: when the hierarchy's shape and the LoD selection equal
 *    those the asset's BVH was built for, refit the BVH's bounds and leaf
 *    records to the current primitives (same topology and leaf order)
 *    instead of rebuilding it.  The hits are the same; traversal may slow
 *    down after large motion.  Otherwise the BVH is rebuilt.
 *  - HR_FLAG_DEFERRED_LOD: choose the LoD with Eq. 14 from the previous
 *    frame's selection when there is one (else the initial rule).
 *  - HR_FLAG_LOD_HYSTERESIS (with HR_FLAG_DEFERRED_LOD): Eq. 14 with a band
 *    around eps_w: refine when w_cur > 1.1 eps_w, coarsen when
 *    w_cur- <= 0.9 eps_w (each threshold one FP32 product).  Eq. 14 as
 *    printed changes a cluster's level whenever its width crosses eps_w; the
 *    paper calls its deferred selection approximately correct, and the band
 *    keeps the levels of clusters whose widths hover at eps_w under small
 *    motion, so that animated frames can refit the BVH. */
#define HR_FLAG_REFIT 512u
#define HR_FLAG_DEFERRED_LOD 1024u
#define HR_FLAG_LOD_HYSTERESIS 2048u
/* hr_render_frame: keep the asset's hierarchy and thick hairs as they are
 * (built by hr_build_clusters or hr_build_guided_clusters, moved by
 * hr_asset_skin); n_clusters is ignored.  Section 5.2: at run time the hair
 * moves by its guides' weights, without a new clustering or fit. */
#define HR_FLAG_KEEP_HIERARCHY 4096u
/* The frame kernel normally carries a schedule from one frame of an asset to
 * the next (no counterpart in the paper): the warp tiles whose slowest lane
 * took the most traversal steps in the previous frame (at most 16, at least
 * half the steps of that frame's slowest) are traced first, four rays per
 * warp, so that the frame is not held up by 32 long rays sharing one warp.
 * Their pixels are composited with the same summation order, so the image
 * does not depend on the schedule.  The schedule lives in the asset and is
 * dropped when the image size or spp changes.  A frame right after an
 * overlapped hr_asset_update (the call before it) uses the fixed order and
 * leaves the schedule as it is, and so does HR_FLAG_FIXED_TILE_ORDER, which
 * traces every tile whole, in raster order.  Counting renders (HR_FLAG_COUNT,
 * hr_render_profile) always use the fixed order. */
#define HR_FLAG_FIXED_TILE_ORDER 8192u

typedef struct hr_render_desc {
  hr_camera camera;
  uint32_t spp;        /* samples per pixel, >= 1 */
  uint32_t k_depth;    /* k-buffer depth K, 1..HR_MAX_K */
  uint64_t seed;       /* sample-position seed (SplitMix64 stream) */
  uint32_t n_lights;   /* 1..HR_MAX_LIGHTS */
  hr_light lights[HR_MAX_LIGHTS];
  int32_t precision;   /* HR_PREC_FP32 or HR_PREC_FP16 */
  uint32_t flags;      /* HR_FLAG_* */
} hr_render_desc;

typedef struct hr_stats {
  double render_ms;      /* trace/shade/composite kernel time (CUDA events) */
  uint64_t n_samples;
  uint32_t n_active_prims;
  uint32_t n_eth_prims;
  uint32_t n_strand_prims;
  uint32_t stack_overflows; /* samples whose traversal stack overflowed (0 expected) */
  /* filled only with HR_FLAG_COUNT */
  uint64_t node_visits;     /* internal BVH nodes whose two child boxes were tested */
  uint64_t prim_tests;      /* ray / elliptic-cylinder tests */
  uint64_t strand_shades;   /* (hit, light) evaluations of f_single */
  uint64_t eth_shades;      /* (hit, light) evaluations of f_ours */
  uint64_t shaded_hits;     /* hits composited */
  uint64_t traced_samples;  /* samples traced (pixels outside the scene's
                               projected bounds are background untraced) */
  /* filled by hr_render_frame (CUDA events on the context stream, ms) */
  double hierarchy_ms;      /* clusters, thick-hair fit, records (K1, K2) */
  double fit_ms;            /* of which the FP64 cross-section fit kernel */
  double lod_ms;            /* LoD widths and rule (K4) */
  double bvh_ms;            /* compaction and LBVH (K5, K6), or the refit */
  uint32_t bvh_refit;       /* 1 when hr_render_frame refit the BVH (HR_FLAG_REFIT) */
  uint32_t lod_deferred;    /* 1 when it chose the LoD with Eq. 14 (HR_FLAG_DEFERRED_LOD) */
  /* filled only with HR_FLAG_COUNT: the precise decision path */
  uint64_t refined_tests;   /* hits decided precisely (near an outline, an end, the
                               search cut or another hit, or a wide FP32 bound) */
  uint64_t refined_entries; /* kept FP32 hits decided precisely afterwards (their
                               order against a precise hit was open) */
  uint32_t heavy_tiles;     /* warp tiles traced a few rays per warp from the previous
                               frame's schedule (see HR_FLAG_FIXED_TILE_ORDER) */
  uint32_t reserved;
} hr_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  hbm_budget: bytes the library may
 * allocate (0 = no limit beyond the device).  cuda_stream: a cudaStream_t to
 * order work on (NULL: the library creates its own non-blocking stream).
 * Also bakes the scattering lookup tables (longitudinal albedo integral over
 * (theta, beta), Gaussian lobe table) on the device. */
hr_status hr_create(hr_ctx** ctx, int device, uint64_t hbm_budget, void* cuda_stream);
hr_status hr_destroy(hr_ctx* ctx);
const char* hr_last_error(hr_ctx* ctx);
/* Bytes currently allocated by the context (assets, BVHs, tables, scratch). */
uint64_t hr_bytes_in_use(hr_ctx* ctx);
/* Number of this library's kernels launched on the context so far
 * (diagnostics: lets a caller count the kernels of a timed region). */
uint64_t hr_kernel_launches(hr_ctx* ctx);

/* ---------------------------------------------------------------- assets */

/* Copy a hair model to the device and precompute every strand segment's
 * elliptic-cylinder record (Section 4 "elliptical cross-section").
 * n_strands >= 1, 1 <= n_segments <= 4096, n_strands * n_segments < 2^30
 * (primitive ids are 30 bits; strand and thick-hair segments together must
 * stay below 2^30, else hr_build_clusters gives HR_EINVAL). */
hr_status hr_asset_create(hr_ctx* ctx, const hr_hair_desc* desc, hr_asset** out);
hr_status hr_asset_destroy(hr_ctx* ctx, hr_asset* asset);

/* New strand positions for an existing asset: the per-frame input of animated
 * hair (Section 6, "Animated hairs": every strand moves each frame, with the
 * same strands, materials and cross-sections).  vertices: host or device,
 * [n_strands][n_segments + 1] float4 (x, y, z, r) in the asset's sizes,
 * copied on the context stream; the strand segment records are rebuilt in
 * place (no allocation).  Device memory and page-locked host memory are read
 * directly by the rebuilding kernel (the transfer overlaps the rebuild);
 * either must stay unchanged until the context stream has passed it (the
 * next call that returns results, e.g. hr_render_frame).  Pageable host
 * memory is copied before the call returns.  Right after hr_render_frame
 * (no other call in between, no serving loop), with device or page-locked
 * source vertices, the new positions and records go to a second set of the
 * asset's buffers on a second stream while that frame renders from the set
 * it was launched with (the first such call allocates the set: the asset's
 * vertex and record memory once more); later calls see the new set.  The
 * hierarchy, thick hairs and BVH of the old positions are stale afterwards:
 * hr_render_frame rebuilds them, or call hr_build_clusters and hr_build_bvh.  The LoD kept for Eq. 14's deferred
 * rule is the previous frame's, as the paper intends.  With serving running,
 * the asset's queued requests end with HR_ESTATE, running ones are waited
 * for, and its cached BVHs are dropped. */
hr_status hr_asset_update(hr_ctx* ctx, hr_asset* asset, const float* vertices);

/* Build the hair hierarchy and fit the thick hairs (Section 5.1 steps 2-3).
 * Clustering rule (deterministic Morton buckets): strands are sorted by
 * (30-bit Morton code of the root quantised to 10 bits per axis in the roots'
 * bounding cube, strand id); rank r joins cluster floor(r * C / N); level k
 * splits each cluster of m members into 4^k thick hairs, rank-in-cluster i
 * going to floor(i * 4^k / m).  Levels: 1 + max k with 4^k <= floor(N/C)/2,
 * capped by max_levels when > 0; the strands are level n_levels.
 * Each thick hair is fitted per cross-section (mean centre, mean tangent,
 * PCA, drop the axis closest to the tangent, semi-axes covering the members):
 * sums, mean and covariance in double-word FP32 (about FP64 accuracy), FP32
 * eigenvectors corrected from a double-word residual, and a full FP64 solve
 * for near-degenerate sections.  n_clusters: 1..min(N, 2^20).
 * cluster_of_out: optional, host or device, [N] uint32 cluster per strand.
 * order_out: optional, host or device, [N] uint32 strand ids in Morton order. */
hr_status hr_build_clusters(hr_ctx* ctx, hr_asset* asset, uint32_t n_clusters,
                            uint32_t max_levels, uint32_t* cluster_of_out, uint32_t* order_out);
/* The paper's own hierarchy (Section 5.1 steps 1, 2 and 4), in place of the
 * Morton rule of hr_build_clusters:
 *  1. guide hairs: k-means over the strands with D(i, j) = sum_k
 *     |p^{i,k} - p^{j,k}|^2 over corresponding vertices (n_guides clusters,
 *     `iterations` update rounds from the strands at Morton ranks
 *     floor((2g + 1) N / 2 n_guides), then a final assignment; ties to the
 *     lower index; an empty cluster keeps its centroid and has no guide);
 *     each cluster's guide is its medoid (least sum of D to its members);
 *  2. clusters of the coarsest level: strands sharing their three nearest
 *     guides (under D), in ascending order of the guide triple, each listing
 *     its strands by (Morton code of the root, id); level k splits a cluster
 *     into 4^k rank buckets as hr_build_clusters does (a cluster of fewer
 *     than 4^k strands leaves buckets empty: such a thick hair has no
 *     primitives); thick hairs fitted as in hr_build_clusters;
 *  4. skinning weights: every strand vertex and every thick-hair
 *     cross-section centre and corner (c +- a e1, c +- b e2) in the
 *     triangular prism of its cluster's three guides' corresponding points
 *     (p = g0 + w1 (g1 - g0) + w2 (g2 - g0) + h n, n the triangle's unit
 *     normal; a degenerate triangle, |e1 x e2| <= 1e-6 |e1| |e2|, keeps the
 *     offset p - g0), for hr_asset_skin.
 * D, the centroid sums and the medoid sums are FP32 in vertex order (and in
 * ascending strand id over members), so the clustering is reproducible.
 * n_guides: 3..min(1024, N); iterations: 0..1000; max_levels as for
 * hr_build_clusters.  The number of clusters C depends on the hair
 * (hr_hierarchy_info).  cluster_of_out, order_out: optional, host or device,
 * [N] uint32.  HR_EINVAL when fewer than three guide clusters are non-empty. */
hr_status hr_build_guided_clusters(hr_ctx* ctx, hr_asset* asset, uint32_t n_guides,
                                   uint32_t iterations, uint32_t max_levels,
                                   uint32_t* cluster_of_out, uint32_t* order_out);
/* The guides of hr_build_guided_clusters: guides_out [n_guides] int32, the
 * guide strand of every k-means cluster (-1 when empty); cluster_guides_out
 * [n_clusters][3] uint32, the three guides (ascending k-means cluster
 * indices) of every cluster.  Both optional, host or device. */
hr_status hr_guides_export(hr_ctx* ctx, hr_asset* asset, int32_t* guides_out,
                           uint32_t* cluster_guides_out);
/* Move the hair with its guides (Section 5.2, "Runtime"): guide_vertices
 * [n_guides][n_segments + 1][4] floats (host or device; xyz of the guide
 * strand of every k-means cluster, w ignored, rows of empty clusters
 * unused) carry every strand vertex and every thick-hair cross-section
 * centre and corner by its weights (FP32; the radius is kept); a
 * cross-section's a and e1 come from its skinned corners c +- a e1, b and e2
 * from c +- b e2; the strand and thick-hair records are rebuilt, the
 * clustering and the fits are not.  Render with HR_FLAG_KEEP_HIERARCHY.
 * HR_ESTATE without a guide-driven hierarchy. */
hr_status hr_asset_skin(hr_ctx* ctx, hr_asset* asset, const float* guide_vertices);
/* The asset's current strand vertices (test export): verts_out [N][S + 1][4]
 * floats, host or device. */
hr_status hr_vertex_export(hr_ctx* ctx, hr_asset* asset, float* verts_out);
/* Number of clusters and thick-hair levels of the built hierarchy. */
hr_status hr_hierarchy_info(hr_ctx* ctx, hr_asset* asset, uint32_t* n_clusters,
                            uint32_t* n_levels, uint32_t* n_eths);
/* Copy thick-hair data out (host or device buffers, each optional):
 *   xsec   : [n_eths][n_segments + 1][12] floats per cross-section:
 *            centre xyz, a, e1 xyz, b, e2 xyz, 0
 *   counts : [n_eths] uint32 member counts
 *   mat    : [n_eths][HR_MAT_FLOATS] mean member material */
hr_status hr_eth_export(hr_ctx* ctx, hr_asset* asset, float* xsec, uint32_t* counts, float* mat);

/* Per-cluster screen width of every thick-hair level (Section 5.2 "Hair width
 * calculation"): the four corner points c +- a e1, c +- b e2 of every
 * cross-section are projected to pixels, l_w is their largest pairwise
 * distance, and the cluster's level-L width is the maximum over its level-L
 * thick hairs (FP32, fixed operation order, no contraction; +inf when a
 * corner is at or behind the near plane).
 * width_out: host or device, [n_clusters][n_levels] floats. */
hr_status hr_lod_widths(hr_ctx* ctx, hr_asset* asset, const hr_camera* camera, float* width_out);

/* Select the LoD of every cluster.
 * mode 0: initial rule (Section 5.1 step 5): the coarsest level whose width is
 *         below eps_w_px, else the strands.
 * mode 1: deferred rule, Eq. (14), from the levels in lod_inout.
 * mode 2: Eq. (14) with the hysteresis band of HR_FLAG_LOD_HYSTERESIS.
 * budget_bias >= 0 then coarsens every cluster: L <- max(0, L - budget_bias).
 * lod_inout: host or device, [n_clusters] uint8 (read in mode 1, written
 * always).  The selection is also kept in the asset for hr_build_bvh. */
hr_status hr_select_lod(hr_ctx* ctx, hr_asset* asset, const hr_camera* camera, float eps_w_px,
                        int mode, int budget_bias, uint8_t* lod_inout);

/* Compact the active primitives of an LoD (strand segments of clusters at the
 * strand level, level-L thick-hair segments otherwise) and build a linear BVH
 * over them (Morton codes of primitive centroids, radix sort, Karras 2012
 * hierarchy, bottom-up bounds).  lod: host or device [n_clusters] uint8, or
 * NULL for the asset's current selection (or all strands when no hierarchy
 * was built).  Global primitive id: strand segment (s, k) -> s * S + k;
 * thick-hair segment (e, k) -> N * S + e * S + k. */
hr_status hr_build_bvh(hr_ctx* ctx, hr_asset* asset, const uint8_t* lod);
/* Primitive ids in BVH leaf order (host or device, [n_active] uint32) and the
 * number of active primitives; both optional. */
hr_status hr_bvh_export(hr_ctx* ctx, hr_asset* asset, uint32_t* leaf_ids, uint32_t* n_active);
/* The library's radix sort (the cluster build's and the BVH build's), for
 * tests: stable ascending sort of (keys[i], vals[i]) on the low `bits` bits of
 * the keys (1..32), in place, n < 2^30; keys and vals are device memory and
 * the call returns when the sort is done.  Each 3,072-pair tile finds where
 * its digits go by reading the counts that earlier tiles publish; with
 * count_earlier != 0 every tile counts the earlier keys itself instead (the
 * path the library takes when a wait for a published count runs out), which
 * must give the same order.  No counterpart in the paper: it checks Section
 * 5.1's Morton ordering step and Karras 2012's sorted-key precondition. */
hr_status hr_sort_pairs(hr_ctx* ctx, uint32_t* keys, uint32_t* vals, uint32_t n, uint32_t bits,
                        int count_earlier);

/* The baked scattering table of the shading code, for tests.  IM(theta,
 * beta) is the integral over theta_o in [-pi/2, pi/2] of G(beta, (theta +
 * theta_o)/2) cos^2(theta_o): the longitudinal factor of a lobe's directional
 * albedo, from which the single-fibre attenuations a_F, a_B and the forward
 * spread of Section 4 (Eq. 6-9) are formed.  The grid is n_theta x n_beta
 * points, theta_i = (pi/2) i / (n_theta - 1), beta_j = 0.04 + 0.64 j /
 * (n_beta - 1), stored row-major [beta][theta].
 * im32_out: optional, host or device, [n_beta][n_theta] floats.
 * im16_out: optional, host or device, the FP16 copy as IEEE half bit patterns.
 * n_theta, n_beta: optional, the grid size (256 x 64). */
hr_status hr_table_export(hr_ctx* ctx, float* im32_out, uint16_t* im16_out, uint32_t* n_theta,
                          uint32_t* n_beta);
/* The shading code's bilinear lookup of IM (see hr_table_export) at m points
 * (theta_k, beta_k), for tests; theta is clamped to [0, pi/2] and beta to
 * [0.04, 0.68].  precision: HR_PREC_FP32 or HR_PREC_FP16 (the table read).
 * theta, beta, out: host or device, [m] floats.  HR_EINVAL for a null
 * pointer or another precision. */
hr_status hr_im_lookup(hr_ctx* ctx, const float* theta, const float* beta, uint32_t m,
                       int precision, float* out);

/* ---------------------------------------------------------------- rendering */

/* Render a frame: per sample a camera ray (sample sid = pixel * spp + s,
 * pixel = y * width + x, sub-pixel position from SplitMix64 outputs 2 sid and
 * 2 sid + 1 of `seed`, top 24 bits each), the K nearest hits by (t, id),
 * shading of each hit with f_single (strands) or f_ours (thick hairs) summed
 * over the lights, front-to-back compositing (strand opacity 1, thick-hair
 * opacity 1 - exp(-2 r l n_tot / (pi a b)) for view chord l), and the mean
 * over the pixel's samples.
 * rgb_out: host or device, [height][width][3] floats.  Requires hr_build_bvh. */
/* One warp tile of a profiled frame (hr_render_profile): the 32 / spp-lane
 * pixels (all their samples) that one warp traces, shades and composites. */
typedef struct hr_tile_record {
  uint64_t t_start_ns;       /* GPU global timer when the warp took the tile */
  uint64_t t_end_ns;         /* and when it had written the tile's pixels */
  uint32_t tile;             /* the tile's index in the frame's hand-out order */
  uint32_t sm;               /* the SM that ran it */
  uint32_t max_node_visits;  /* most BVH node visits of one lane (its rays) */
  uint32_t max_prim_tests;   /* most primitive tests of one lane */
} hr_tile_record;

hr_status hr_render(hr_ctx* ctx, hr_asset* asset, const hr_render_desc* desc, float* rgb_out,
                    hr_stats* stats);
/* hr_render with HR_FLAG_COUNT and, per warp tile of the frame kernel, its
 * start and end times and its largest per-lane counts, for the study of the
 * frame's tail (the kernel lasts as long as its slowest tiles).  No
 * counterpart in the paper.  tiles_out: host or device, capacity records;
 * the first min(capacity, tiles) of the frame's tiles in hand-out order are
 * written.  n_tiles (optional): the frame's number of tiles.  The timing
 * adds two timer reads and a warp reduction per tile to the counting
 * kernel.  HR_EINVAL for a null tiles_out with capacity > 0. */
hr_status hr_render_profile(hr_ctx* ctx, hr_asset* asset, const hr_render_desc* desc,
                            float* rgb_out, hr_stats* stats, hr_tile_record* tiles_out,
                            uint32_t capacity, uint32_t* n_tiles);

/* Render only the listed samples (parity hook): radiance [m][3] and the
 * global ids of the composited hits, [m][k_depth]: the k nearest by (t, id),
 * nearest first, cut after the first opaque (strand) hit, -1 padded (column 0
 * is the nearest hit, -1 for a miss).
 * sample_ids, radiance_out and hit_out are host or device. */
hr_status hr_render_samples(hr_ctx* ctx, hr_asset* asset, const hr_render_desc* desc,
                            const uint32_t* sample_ids, uint32_t m, float* radiance_out,
                            int32_t* hit_out);

/* Whole hot path in one call (Section 5.2, run time): clusters and the
 * thick-hair fit (n_clusters > 0; none with HR_FLAG_KEEP_HIERARCHY), LoD
 * selection (eps_w_px, budget_bias; Eq. 14 with HR_FLAG_DEFERRED_LOD), BVH
 * (or its refit with HR_FLAG_REFIT) and frame.  With device output and no
 * stats the call returns without waiting for the frame.  When the previous
 * call on the context was also hr_render_frame (no other call in between,
 * no serving loop) and the hierarchy keeps its shape, this frame's clusters
 * and fit run on a second stream of the context as soon as the previous
 * frame's BVH is built, overlapping that frame's rendering (they write a
 * second cross-section buffer; the records that frame reads are rewritten
 * after it).  Results are the same as without the overlap.  stats: optional;
 * hierarchy_ms then runs from the start of the clusters, on whichever stream. */
hr_status hr_render_frame(hr_ctx* ctx, hr_asset* asset, uint32_t n_clusters, float eps_w_px,
                          int budget_bias, const hr_render_desc* desc, float* rgb_out,
                          hr_stats* stats);
/* Kernel times of the last n hr_render_frame calls on the context, oldest
 * first, from events every call records (so a loop of frames needs no
 * synchronisation per frame to be timed): frame_ms[i] the frame kernel
 * (with the image clear and scene rectangle), fit_ms[i] the cross-section
 * fit (0 when that call fitted nothing), flags[i] bit 0 the call fitted,
 * bit 1 it refit the BVH instead of rebuilding it.  Waits for those frames.
 * At most the last 256 calls are kept; n_out (optional) receives the number
 * written.  frame_ms, fit_ms, flags: optional host arrays of n elements. */
hr_status hr_frame_times(hr_ctx* ctx, uint32_t n, float* frame_ms, float* fit_ms, uint32_t* flags,
                         uint32_t* n_out);

/* Morton clustering without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that may
 * not let a library allocate device memory, such as a host application that
 * owns every allocation under a fixed budget, or a real-time loop in which
 * cudaMalloc / cudaFree are not allowed because they synchronise the device.
 * It computes the same strand order and cluster ids as hr_build_clusters
 * (order_out and cluster_of_out there) and needs no context.  The root
 * bounds, Morton-code and cluster kernels are those of hr_build_clusters;
 * the stable radix sort is a different one, four kernels per 8-bit digit
 * (digit histogram per 2,048-key tile, scan, scatter), whose scratch fits a
 * fixed array, where hr_build_clusters runs the single-sweep sort.  Both
 * sorts are stable, so the outputs are the same.
 *   vertices       : device, [n_strands][n_segments + 1][4] floats (as in
 *                    hr_hair_desc; only the root vertex of each strand is read)
 *   order_out      : device, [n_strands] uint32, strand ids in Morton order
 *   cluster_of_out : device, [n_strands] uint32, cluster of each strand
 *   cuda_stream    : stream the work is ordered on (NULL: legacy default
 *                    stream); the call returns without synchronising it.
 * Scratch lives in one fixed device array of the library (about 13 MB, held
 * on every device that loads the library until the process exits); hence
 * n_strands <= HR_NOALLOC_MAX_STRANDS, larger inputs are rejected with
 * HR_EINVAL.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call on a device uses the same array:
 * calls whose work overlaps on the GPU (different streams, no ordering
 * between them) race and must not be issued.  Pointers that are not device
 * memory, or sizes out of range, give HR_EINVAL; a CUDA error gives HR_ECUDA. */
#define HR_NOALLOC_MAX_STRANDS 1048576u
hr_status hr_morton_clusters_noalloc(const float* vertices, uint32_t n_strands,
                                     uint32_t n_segments, uint32_t n_clusters,
                                     uint32_t* order_out, uint32_t* cluster_of_out,
                                     void* cuda_stream);

/* ---------------------------------------------------------------- serving */

/* A render request for the serving loop: asset (already clustered), its
 * render description, LoD budget bias and epsilon_w, and a caller-owned
 * output buffer (host or device, [height][width][3]) that must stay valid
 * until hr_poll reports completion. */
typedef struct hr_request {
  hr_asset* asset;
  hr_render_desc desc;
  float eps_w_px;
  int32_t budget_bias;
  float* rgb_out;
} hr_request;

typedef struct hr_result {
  hr_status status;
  double submit_ms;  /* host clock (ms since hr_create) when hr_submit was called */
  double admit_ms;   /* when admitted (slot and memory granted) */
  double done_ms;    /* when its last tile completed on the device */
  uint64_t n_samples;
} hr_result;

/* Start the serving loop: up to max_slots requests resident at once, batches
 * of at most max_batch_samples samples per persistent launch, admission while
 * the context's bytes in use stay under its HBM budget. */
hr_status hr_serve_start(hr_ctx* ctx, uint32_t max_slots, uint64_t max_batch_samples);
hr_status hr_serve_stop(hr_ctx* ctx);
/* Non-blocking submit; *ticket identifies the request.  HR_EBUSY when the
 * queue holds too many pending requests; HR_EINVAL for HR_FLAG_SHADOWS or
 * HR_FLAG_COUNT (served frames are primary hits only). */
hr_status hr_submit(hr_ctx* ctx, const hr_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (0: do not wait) for a request.  HR_OK and *result
 * filled when done; HR_ENOTREADY if timeout_ms == 0 and not done;
 * HR_ETIMEOUT if the wait ran out; HR_EINVAL for an unknown ticket. */
hr_status hr_poll(hr_ctx* ctx, uint64_t ticket, int timeout_ms, hr_result* result);

/* Host-side fault injection for the serving tests (no GPU fault is ever
 * made): kind 1 fails the next admission's allocation with HR_ENOMEM; kind 2
 * delays completion reporting of the next request by `arg` ms. */
hr_status hr_serve_inject(hr_ctx* ctx, int kind, int64_t arg);

#ifdef __cplusplus
}
#endif

#endif /* HAIRRT_H */
