#!/usr/bin/env python
"""Throughput of the level-of-detail hair ray tracer on one GB300.

One step is one pass of the whole hot path over the full-head workload
(100,000 strands x 64 segments, 1920x1080, 8 samples per pixel, 8 point
lights, 4096 clusters, LoD chosen per cluster by projected width with
epsilon_w = 2 px): Morton clusters, thick-hair fit, LoD selection,
active-primitive compaction, LBVH build, and the trace / shade / composite
kernel.  The metric is samples per second of that step (Msamples/s) with the
inputs resident on the device; ms/frame is printed beside it.

Also measured in the same run:
  * e2e    - the same step through the C ABI with host buffers, as an
             animated frame: the strand positions uploaded from pinned
             memory (hr_asset_update) and the image read back, inside the
             timed region;
  * roofline - the kernel that takes more of the step, the trace kernel or
             the cross-section fit, against its ALU peak (FP32 for the trace
             kernel, with algorithmic FLOPs from a counting render; FP32 for
             the fit), and the other kernel beside it;
  * cpu_baseline - the FP64 brute-force CPU oracle on a bounded sample of the
             same workload, on this host's cores;
  * serving - a seeded Poisson request stream through hr_submit / hr_poll
             (p50 / p99 latency, aggregate samples/s).

``--impl reference`` times the CPU oracle alone (the reference arm).
Multi-GPU (torchrun, N > 1): every rank renders its own replica of the frame
(replicas only: the path has no exchange step); the time is the maximum over
ranks and the value counts the samples of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Msamples/s and ms/frame, 100k strands 1080p; p50/p99 served latency at RMSE<=5e-3"

# Algorithmic FP32 operations per counted event of the frame kernel, the
# per-unit figures of the hot path's measurement plan: 24 per internal-node
# visit (two slab tests of 12), 60 per primitive test, 150 per (strand hit,
# light) and 300 per (thick-hair hit, light) shading, 30 per traced sample
# (camera ray and compositing).  The headline roofline uses these.
FLOPS_PER_NODE = 24
FLOPS_PER_TEST = 60
FLOPS_PER_STRAND_SHADE = 150
FLOPS_PER_ETH_SHADE = 300
FLOPS_PER_HIT = 0
FLOPS_PER_SAMPLE = 30
# The same events with operation counts read off the kernel source
# (trace_core.cuh; an FMA counts 2, every other FP32 arithmetic, min/max or
# compare 1, a special-function call 1): a node visit is 12 FMA (24) plus 12
# min/max per child box and the ordering (50); a primitive test 41; a strand
# shade 100; a thick-hair shade 250; a composited hit 40 (tangent, outgoing
# angles, opacity, blend); a traced sample 30.  Reported beside the headline
# as "frac_source_count".
SRC_FLOPS = {"node": 50, "test": 41, "sshade": 100, "eshade": 250, "hit": 40, "sample": 30}
# FP32 operations of the cross-section fit (k_fit_cross_sections), same rules
# (hierarchy.cu).  Per member and section: the exact offsets and their
# double-word first and second moments (3 TwoSum, 3 double-word adds, 6
# double-word product accumulations: 132), the unit tangent (15), and the two
# projection passes for the semi-axes and the coverage scale (22 + 22) = 191.
# Per section: folding the 9 sums (54), 1/n and the mean (34), the double-word
# covariance (240), the mean tangent, trace and FP32 copy (33), two cyclic
# Jacobi sweeps (444: the fewest a section takes, so a lower bound), axis
# choice (48), the double-word residual and first-order correction of the
# kept axis (370), the frame and semi-axis scalars (39) and the centre (63)
# = 1325.  The rare full FP64 solve of near-degenerate sections is not counted.
FIT_FLOPS_PER_MEMBER = 191
FIT_FLOPS_PER_SECTION = 1325


def sources_hash(names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2405_10565_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


TRACE_SOURCES = ["trace_core.cuh", "trace_frame.cuh", "trace_frame.cu", "common.cuh", "dword.cuh"]
FIT_SOURCES = ["hierarchy.cu", "common.cuh", "dword.cuh"]


def traffic_record(name, sources, workload_name):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's
    sources are unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    try:
        pj = json.load(open(path))
    except (OSError, ValueError):
        return None
    if pj.get("sources") == sources_hash(sources) and pj.get("workload") == workload_name:
        return pj.get("dram_bytes_per_launch")
    return None


# ------------------------------------------------------------------ clocks


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"hairrt_clocks_{os.getpid()}.csv")
        self.gpu_id = gpu_id

    def __enter__(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts))
            except ValueError:
                continue
        os.remove(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        smax = max(r[1] for r in rows)
        load = [r for r in rows if r[0] > 0.5 * smax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2][4 + i] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": smax,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workload


def workload(name):
    import scenegen
    if name == "full_head":
        return scenegen.full_head()
    if name == "full_head_fp16":
        return scenegen.full_head(precision=1)
    if name == "small":
        return scenegen.full_head(n=10000, S=32, width=480, height=270, spp=4, n_lights=8,
                                  n_clusters=512)
    raise ValueError(name)


def oracle_baseline(w, seconds: float, seed: int = 11):
    """Samples/s of the FP64 brute-force oracle on a bounded seeded sample."""
    import oracle
    import scenegen
    t0 = time.time()
    prep = oracle.prepare(w.scene, w.n_clusters, w.lod_setting, w.camera.pack(), w.eps_w)
    t_prep = time.time() - t0
    total = w.camera.width * w.camera.height * w.spp
    st = scenegen.Stream(seed, 5)
    probe = (st.u64(32) % np.uint64(total)).astype(np.int64)
    cores = os.cpu_count() or 1
    t0 = time.time()
    oracle.render_samples(prep, w.camera.pack(), w.lights, probe, w.spp, w.k_depth, w.sample_seed,
                          threads=cores)
    per = (time.time() - t0) / probe.shape[0]
    m = int(max(cores, min(65536, seconds / max(per, 1e-9))))
    sids = (st.u64(m) % np.uint64(total)).astype(np.int64)
    t0 = time.time()
    oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, w.k_depth, w.sample_seed,
                          threads=cores)
    dt = time.time() - t0
    P = int(prep.rows.shape[0])
    return {"value": m / dt / 1e6, "unit": "Msamples/s", "cores": cores, "kind": "oracle",
            "sample": f"{m} seeded samples of the {total}-sample frame, brute force over "
                      f"{P} active primitives (FP64); setup {t_prep:.1f}s untimed",
            "seconds": dt,
            "ns_per_sample_primitive": dt * cores / (m * max(P, 1)) * 1e9,
            "full_frame_s_extrapolated": total * dt / m}


def event_flops(st) -> int:
    """Algorithmic FP32 operations of a frame from the event counts of a
    counting render (the measurement plan's per-event figures)."""
    return (FLOPS_PER_NODE * st.node_visits + FLOPS_PER_TEST * st.prim_tests +
            FLOPS_PER_STRAND_SHADE * st.strand_shades + FLOPS_PER_ETH_SHADE * st.eth_shades +
            FLOPS_PER_HIT * st.shaded_hits + FLOPS_PER_SAMPLE * st.traced_samples)


def event_flops_source(st) -> int:
    """The same events weighted by the operation counts of the kernel source."""
    c = SRC_FLOPS
    return (c["node"] * st.node_visits + c["test"] * st.prim_tests + c["sshade"] * st.strand_shades
            + c["eshade"] * st.eth_shades + c["hit"] * st.shaded_hits
            + c["sample"] * st.traced_samples)


def measure_config(hr, ctx, torch, dev, w, steps: int, warmup: int = 2, peak_tflops=None):
    """Step time of another configuration (not the headline line): for a
    fixed LoD setting (all strands, half, all thick hairs) the clusters, BVH
    and frame per step, for a selected LoD the whole hr_render_frame step."""
    import scenegen
    verts = torch.from_numpy(w.scene.verts).to(dev)
    mat = torch.from_numpy(w.scene.mat).to(dev)
    shape = torch.from_numpy(w.scene.shape).to(dev)
    a = hr.hr_asset_create(ctx, verts, mat, shape)
    d = hr.render_desc(w.camera.pack(), w.lights, w.spp, w.k_depth, w.sample_seed, w.precision)
    img = torch.empty((w.camera.height, w.camera.width, 3), device=dev)
    try:
        if w.n_clusters and w.lod_setting != "select":
            hr.hr_build_clusters(ctx, a, w.n_clusters)
            C, L, _ = hr.hr_hierarchy_info(ctx, a)
            lod = torch.from_numpy(scenegen.lod_preset(w.lod_setting, C, L)).to(dev)

            def one():
                hr.hr_build_clusters(ctx, a, w.n_clusters)
                hr.hr_build_bvh(ctx, a, lod)
                hr.hr_render(ctx, a, d, img)
        elif w.n_clusters:
            def one():
                hr.hr_render_frame(ctx, a, w.n_clusters, w.eps_w, 0, d, img)
        else:
            def one():
                hr.hr_build_bvh(ctx, a, None)
                hr.hr_render(ctx, a, d, img)
        for _ in range(warmup):
            one()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps):
            one()
        torch.cuda.synchronize(dev)
        dt = (time.perf_counter() - t0) / steps
        # what the step traced (one counting frame after the timed steps), and
        # the frame kernel alone on the same BVH (CUDA events, median of 5)
        dc = hr.render_desc(w.camera.pack(), w.lights, w.spp, w.k_depth, w.sample_seed, w.precision,
                            hr.HR_FLAG_COUNT)
        st = hr.hr_render(ctx, a, dc, img, stats=True)
        frame_ms = statistics.median(hr.hr_render(ctx, a, d, img, stats=True).render_ms for _ in range(5))
    finally:
        hr.hr_asset_destroy(ctx, a)
    n = w.camera.width * w.camera.height * w.spp
    out = {"workload": w.name, "ms_per_step": dt * 1e3, "Msamples_per_s": n / dt / 1e6,
           "strands": w.scene.n_strands, "segments": w.scene.n_segments,
           "lod": w.lod_setting, "precision": "fp16" if w.precision else "fp32", "k_depth": w.k_depth,
           "active_prims": int(st.n_active_prims), "eth_prims": int(st.n_eth_prims),
           "traced_samples": int(st.traced_samples), "frame_ms": frame_ms,
           "prim_tests": int(st.prim_tests), "refined_tests": int(st.refined_tests),
           "refined_entries": int(st.refined_entries)}
    out["traced_msamples_per_s_frame"] = st.traced_samples / (frame_ms * 1e-3) / 1e6
    if peak_tflops:
        tf = event_flops(st) / (frame_ms * 1e-3) / 1e12
        ts = event_flops_source(st) / (frame_ms * 1e-3) / 1e12
        out["frame_fp32"] = {"achieved_tflops": tf, "frac": tf / peak_tflops,
                             "frac_source_count": ts / peak_tflops}
    return out


def frame_tail(hr, ctx, asset, desc, img, capacity: int = 1 << 20):
    """Per-warp-tile times of one counting frame (hr_render_profile): how long
    the frame kernel's tiles take and how far the slowest ones set its length."""
    st, rec, n = hr.hr_render_profile(ctx, asset, desc, img, capacity)
    if rec.size == 0:
        return {"tiles": n}
    t0 = rec["t_start_ns"].astype(np.int64)
    t1 = rec["t_end_ns"].astype(np.int64)
    dur = (t1 - t0) / 1e3
    span = (t1.max() - t0.min()) / 1e3
    slow = int(np.argmax(dur))
    warps = len(np.unique(rec["sm"])) * 16  # 4 blocks of 4 warps per SM
    visits = int(rec["max_node_visits"][slow])
    return {"tiles": n, "recorded": int(rec.size), "span_us": span,
            "tile_us": {"median": float(np.median(dur)), "p99": float(np.percentile(dur, 99)),
                        "max": float(dur.max())},
            "balanced_span_us": float(dur.sum() / warps),
            "slowest_tile": {"index": int(rec["tile"][slow]), "max_node_visits": visits,
                             "max_prim_tests": int(rec["max_prim_tests"][slow]),
                             "ns_per_node_visit": float(dur[slow] * 1e3 / max(visits, 1))},
            "tiles_running_after_half_span": int(((t1 - t0.min()) / 1e3 > span / 2).sum()),
            "note": "counting kernel (event counters on); tiles in hand-out order"}


def max_over_ranks(x: float, dist, device) -> float:
    """The maximum of a per-rank time over all ranks (x itself on one rank):
    a multi-GPU step lasts as long as its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_msamples_per_s(world: int, samples_per_rank: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank renders its own replica, so the job
    processes world x samples per step in the slowest rank's time."""
    return world * samples_per_rank * steps / seconds / 1e6


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, on this host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    import scenegen
    w = workload(args.workload)
    prep = oracle.prepare(w.scene, w.n_clusters, w.lod_setting, w.camera.pack(), w.eps_w)
    total = w.camera.width * w.camera.height * w.spp
    cores = os.cpu_count() or 1
    m = args.ref_samples
    st = scenegen.Stream(13, 5)
    times = []
    for i in range(args.warmup + args.steps):
        sids = (st.u64(m) % np.uint64(total)).astype(np.int64)
        t0 = time.time()
        oracle.render_samples(prep, w.camera.pack(), w.lights, sids, w.spp, w.k_depth,
                              w.sample_seed, threads=cores)
        if i >= args.warmup:
            times.append(time.time() - t0)
    dt = sum(times)
    value = m * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Msamples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, args),
            "cpu_baseline": {"value": value, "unit": "Msamples/s", "cores": cores, "kind": "oracle",
                             "sample": f"{m} seeded samples per step of the {total}-sample frame"},
            "e2e": {"value": value, "unit": "Msamples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_of(w, args):
    return {"workload": w.name, "strands": w.scene.n_strands, "segments": w.scene.n_segments,
            "clusters": w.n_clusters, "width": w.camera.width, "height": w.camera.height,
            "spp": w.spp, "lights": int(w.lights.shape[0]), "k_depth": w.k_depth,
            "eps_w_px": w.eps_w, "precision": "fp16_tables" if w.precision else "fp32",
            "l2": "inputs larger than L2 (no flush): vertices 104 MB, primitive records "
                  "0.7 GB, BVH per frame",
            "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "single"}


# ------------------------------------------------------------------ serving


def run_serving(hr, ctx, torch, dev, n_requests: int, seed: int = 2):
    """Seeded request stream (three assets of 10k/50k/100k strands x 64
    segments, resolutions 256^2 / 720p / 1080p, 1-8 spp, LoD budget 0-4).

    * plain: the plain FP32 renderer, one request after another through the C
      ABI (LoD selection, BVH, frame) - the baseline of the served form;
    * served, saturated: every request submitted at once to the continuous-
      batching loop with FP16 lookup tables - aggregate throughput;
    * served, Poisson arrivals at 80% of the saturated rate - latency
      (completion minus submission) p50 / p99.
    """
    import scenegen
    assets = []
    for i, n in enumerate((10000, 50000, 100000)):
        wl = scenegen.full_head(n=n, S=64, width=64, height=64, spp=1, n_clusters=max(64, n // 25),
                                seed=10 + i)
        a = hr.hr_asset_create(ctx, torch.from_numpy(wl.scene.verts).to(dev),
                               torch.from_numpy(wl.scene.mat).to(dev),
                               torch.from_numpy(wl.scene.shape).to(dev))
        hr.hr_build_clusters(ctx, a, wl.n_clusters)
        assets.append((a, wl))
    reqs = scenegen.serving_stream(n_requests, seed=seed, rate_hz=1.0)
    jobs = []
    for r in reqs:
        a, wl = assets[r["asset"]]
        lo, hi = wl.scene.aabb()
        cam = scenegen.frame_camera(lo, hi, r["width"], r["height"], perspective=True, fill=0.3)
        jobs.append((a, cam, r))
    outs = [torch.empty((r["height"], r["width"], 3), device=dev) for _, _, r in jobs]
    total_samples = sum(r["width"] * r["height"] * r["spp"] for _, _, r in jobs)

    # plain FP32 renderer, sequential
    lods = {}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for (a, cam, r), o in zip(jobs, outs):
        C, L, E = hr.hr_hierarchy_info(ctx, a)
        lod = lods.setdefault(C, torch.empty(C, dtype=torch.uint8, device=dev))
        hr.hr_select_lod(ctx, a, cam.pack(), 2.0, 0, r["budget"], lod)
        hr.hr_build_bvh(ctx, a, lod)
        d = hr.render_desc(cam.pack(), assets[r["asset"]][1].lights, r["spp"], 4, r["seed"], 0)
        hr.hr_render(ctx, a, d, o)
    torch.cuda.synchronize(dev)
    plain_s = time.perf_counter() - t0

    # the plain renderer with the same BVH reuse as serving: requests grouped by
    # (asset, resolution, LoD budget), one LoD selection and BVH build per group,
    # then one hr_render per request, in FP32 and with FP16 tables (the
    # comparison isolates batching and the table precision)
    groups = {}
    for i, (a, cam, r) in enumerate(jobs):
        groups.setdefault((r["asset"], r["width"], r["height"], r["budget"]), []).append(i)
    grouped_s = {}
    for prec in (0, 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for key, idx in groups.items():
            a, cam, r0 = jobs[idx[0]]
            C, L, E = hr.hr_hierarchy_info(ctx, a)
            lod = lods.setdefault(C, torch.empty(C, dtype=torch.uint8, device=dev))
            hr.hr_select_lod(ctx, a, cam.pack(), 2.0, 0, r0["budget"], lod)
            hr.hr_build_bvh(ctx, a, lod)
            for i in idx:
                _, cam_i, r = jobs[i]
                d = hr.render_desc(cam_i.pack(), assets[r["asset"]][1].lights, r["spp"], 4,
                                   r["seed"], prec)
                hr.hr_render(ctx, a, d, outs[i])
        torch.cuda.synchronize(dev)
        grouped_s[prec] = time.perf_counter() - t0

    descs = [hr.render_desc(cam.pack(), assets[r["asset"]][1].lights, r["spp"], 4, r["seed"], 1)
             for a, cam, r in jobs]
    hr.hr_serve_start(ctx, 16, 8 << 20)
    try:
        # warm the slots
        for (a, cam, r), d, o in list(zip(jobs, descs, outs))[:16]:
            hr.hr_poll(ctx, hr.hr_submit(ctx, a, d, o, 2.0, r["budget"]), 60000)
        # saturated
        t0 = time.perf_counter()
        ts = [hr.hr_submit(ctx, a, d, o, 2.0, r["budget"])
              for (a, cam, r), d, o in zip(jobs, descs, outs)]
        for t in ts:
            st, res = hr.hr_poll(ctx, t, 600000)
            if st != hr.HR_OK or res.status != hr.HR_OK:
                raise RuntimeError(f"request failed: {st} {res.status}")
        sat_s = time.perf_counter() - t0
        sat_rate = total_samples / sat_s
        # Poisson arrivals at 80% of the saturated request rate
        rate = 0.8 * len(jobs) / sat_s
        arr = np.asarray([r["arrival_s"] for _, _, r in jobs]) / rate
        tickets = []
        start = time.perf_counter()
        for (a, cam, r), d, o, at in zip(jobs, descs, outs, arr):
            now = time.perf_counter() - start
            if at > now:
                time.sleep(at - now)
            tickets.append(hr.hr_submit(ctx, a, d, o, 2.0, r["budget"]))
        lat = []
        for t in tickets:
            st, res = hr.hr_poll(ctx, t, 600000)
            if st != hr.HR_OK or res.status != hr.HR_OK:
                raise RuntimeError(f"request failed: {st} {res.status}")
            lat.append(res.done_ms - res.submit_ms)
    finally:
        hr.hr_serve_stop(ctx)
        for a, _ in assets:
            hr.hr_asset_destroy(ctx, a)
    lat = np.asarray(lat)
    return {"requests": n_requests, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "arrival_rate_hz": rate,
            "served_fp16_msamples_per_s": sat_rate / 1e6,
            "plain_fp32_sequential_msamples_per_s": total_samples / plain_s / 1e6,
            "speedup_served_vs_plain": (total_samples / sat_s) / (total_samples / plain_s),
            "bvh_groups": len(groups),
            "plain_fp32_grouped_msamples_per_s": total_samples / grouped_s[0] / 1e6,
            "plain_fp16_grouped_msamples_per_s": total_samples / grouped_s[1] / 1e6,
            "speedup_served_vs_plain_grouped_fp32": grouped_s[0] / sat_s,
            "accuracy": "FP16 tables: rel-RMSE <= 5e-3 vs the FP64 oracle "
                        "(tests/test_serving.py::test_served_full_size_asset_vs_oracle: the "
                        "100k-strand asset served at 1280x720, 4 spp; "
                        "tests/test_gpu_parity.py::test_stress_sampled)"}


# ------------------------------------------------------------------ main arm


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=250)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full_head")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-samples", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2405_10565_gb300 as hr
    from paper_2405_10565_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if rank == 0:
        build()
    if dist:
        dist.barrier()
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = hr.hr_create(local, 0, stream.cuda_stream)
    w = workload(args.workload)
    W, H, spp = w.camera.width, w.camera.height, w.spp
    samples = W * H * spp
    verts = torch.from_numpy(w.scene.verts).to(dev)
    mat = torch.from_numpy(w.scene.mat).to(dev)
    shape = torch.from_numpy(w.scene.shape).to(dev)
    asset = hr.hr_asset_create(ctx, verts, mat, shape)
    desc = hr.render_desc(w.camera.pack(), w.lights, spp, w.k_depth, w.sample_seed, w.precision)
    img = torch.empty((H, W, 3), device=dev)

    def step():
        # no statistics: the call returns without waiting for its frame, so the
        # next step's clusters and fit overlap this frame's rendering
        hr.hr_render_frame(ctx, asset, w.n_clusters, w.eps_w, 0, desc, img)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    # the same frame with FP16 lookup tables (outside the timed region)
    d16 = hr.render_desc(w.camera.pack(), w.lights, spp, w.k_depth, w.sample_seed, 1)
    fp16_ms = statistics.median(hr.hr_render(ctx, asset, d16, img, stats=True).render_ms
                                for _ in range(10))
    fp32_st = [hr.hr_render(ctx, asset, desc, img, stats=True) for _ in range(10)]
    fp32_ms = statistics.median(s.render_ms for s in fp32_st)
    # the same frame in the fixed tile order (HR_FLAG_FIXED_TILE_ORDER: no
    # heavy tiles first; the schedule is left as it is)
    dfix = hr.render_desc(w.camera.pack(), w.lights, spp, w.k_depth, w.sample_seed, w.precision,
                          hr.HR_FLAG_FIXED_TILE_ORDER)
    fixed_ms = statistics.median(hr.hr_render(ctx, asset, dfix, img, stats=True).render_ms
                                 for _ in range(10))
    tile_schedule = {"heavy_tiles": int(fp32_st[-1].heavy_tiles), "frame_ms_warm": fp32_ms,
                     "frame_ms_fixed_order_warm": fixed_ms,
                     "note": "warm frames alone: the previous frame's heaviest warp tiles traced "
                             "first, four rays per warp, against the fixed tile order; the images "
                             "are identical"}
    # the same frame with dual-scattering light paths (a shadow ray per hit and
    # light, HR_FLAG_SHADOWS), outside the timed region
    dsh = hr.render_desc(w.camera.pack(), w.lights, spp, w.k_depth, w.sample_seed, w.precision,
                         hr.HR_FLAG_SHADOWS)
    shadow_ms = statistics.median(hr.hr_render(ctx, asset, dsh, img, stats=True).render_ms
                                  for _ in range(5))
    # counting render (outside the timed region): events of the algorithmic FLOP model
    cdesc = hr.render_desc(w.camera.pack(), w.lights, spp, w.k_depth, w.sample_seed, w.precision,
                           hr.HR_FLAG_COUNT)
    cst = hr.hr_render(ctx, asset, cdesc, img, stats=True)
    tail = frame_tail(hr, ctx, asset, cdesc, img)
    n_levels_info = hr.hr_hierarchy_info(ctx, asset)
    flops = event_flops(cst)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = hr.hr_kernel_launches(ctx)
    render_ms, fit_ms = [], []
    with ClockSampler(uuid) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize(dev)
    launches = hr.hr_kernel_launches(ctx) - launches0
    # the timed steps' frame-kernel and fit times, from the library's per-call events
    frame_t, fit_t = hr.hr_frame_times(ctx, args.steps)
    render_ms, fit_ms = [float(x) for x in frame_t], [float(x) for x in fit_t]
    # phase times from one more step with statistics (outside the timed region;
    # it waits for its frame and does not overlap the previous one)
    st = hr.hr_render_frame(ctx, asset, w.n_clusters, w.eps_w, 0, desc, img, stats=True)
    elapsed = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
    if dist:
        dist.barrier()
    ms_step = 1e3 * elapsed / args.steps
    value = job_msamples_per_s(world, samples, args.steps, elapsed)
    render_avg = statistics.mean(render_ms)
    clocks = clk.summary()

    # e2e: the same step through the C ABI with host buffers, as an animated
    # frame: the strand positions come from pinned host memory every step
    # (hr_asset_update), the image goes back to pinned host memory
    pv = torch.from_numpy(w.scene.verts).pin_memory()
    hout = torch.empty((H, W, 3), dtype=torch.float32).pin_memory()
    h2d = pv.numel() * 4
    d2h = hout.numel() * 4

    img_e = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    # two device images and two pinned host images, alternating; each step's
    # image goes back on its own copy stream
    img_pair = [img_e, torch.empty_like(img_e)]
    hout_pair = [hout, torch.empty_like(hout).pin_memory()]
    copy_stream = torch.cuda.Stream(device=dev)
    frame_done = [torch.cuda.Event(), torch.cuda.Event()]
    copy_done = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_i = [0]

    def e2e_step():
        # upload, whole path, image back to pinned host memory.  The read-back
        # runs on a copy stream without blocking the host, so the next step's
        # upload, clusters and fit overlap this frame (hr_asset_update and
        # hr_render_frame pipelining) and its main-stream work overlaps the
        # read-back; a frame waits only for the copy that last read its image.
        j = e2e_i[0] % 2
        e2e_i[0] += 1
        hr.hr_asset_update(ctx, asset, pv)
        stream.wait_event(copy_done[j])
        hr.hr_render_frame(ctx, asset, w.n_clusters, w.eps_w, 0, desc, img_pair[j])
        frame_done[j].record(stream)
        copy_stream.wait_event(frame_done[j])
        with torch.cuda.stream(copy_stream):
            hout_pair[j].copy_(img_pair[j], non_blocking=True)
            copy_done[j].record(copy_stream)

    e2e = None
    if not args.no_e2e:
        e2e_step()
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.e2e_steps, dist, dev)
        fr_ms, ft_ms = hr.hr_frame_times(ctx, args.e2e_steps)
        e2e = {"value": job_msamples_per_s(world, samples, 1, e2e_s), "unit": "Msamples/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
               "frame_kernel_ms": float(np.mean(fr_ms)), "fit_kernel_ms": float(np.mean(ft_ms))}

    # animated frames: the strands alternate between two poses (a smooth
    # displacement field of amplitude `amp` that grows from 0 at the root, so
    # roots stay on the scalp), uploaded from pinned memory each frame; full
    # BVH rebuild against a refit when the clusters and their levels are
    # unchanged (Eq. 14 deferred selection, with or without the hysteresis
    # band).  "skinned" is the paper's run time (Section 5.2): the guide-driven
    # hierarchy is built once, each frame uploads only the guides' poses, and
    # hr_asset_skin moves strands and thick hairs by their weights (no new
    # clustering or fit) before the LoD, the BVH and the frame.
    animation = None
    if not args.no_e2e:
        p = w.scene.verts[..., :3].astype(np.float64)
        grow = np.linspace(0.0, 1.0, w.scene.verts.shape[1])[None, :]
        animation = {"frames": args.e2e_steps * 4}
        for amp in (2e-5, 2e-3):
            moved = np.array(w.scene.verts, copy=True)
            moved[..., 0] += (amp * grow * np.sin(7.0 * p[..., 1] + 1.3)).astype(np.float32)
            moved[..., 2] += (amp * grow * np.cos(5.0 * p[..., 0] - 1.3)).astype(np.float32)
            poses = [torch.from_numpy(moved).pin_memory(), pv]
            res = {}
            for key, flags in (("rebuild", 0), ("refit", hr.HR_FLAG_REFIT | hr.HR_FLAG_DEFERRED_LOD),
                               ("refit_hysteresis", hr.HR_FLAG_REFIT | hr.HR_FLAG_DEFERRED_LOD |
                                hr.HR_FLAG_LOD_HYSTERESIS)):
                da = hr.render_desc(w.camera.pack(), w.lights, w.spp, w.k_depth, w.sample_seed,
                                    w.precision, flags)
                for i in range(2):  # warm-up
                    hr.hr_asset_update(ctx, asset, poses[i])
                    hr.hr_render_frame(ctx, asset, w.n_clusters, w.eps_w, 0, da, hout)
                torch.cuda.synchronize(dev)
                refits, bvh = 0, []
                t0 = time.perf_counter()
                for i in range(animation["frames"]):
                    hr.hr_asset_update(ctx, asset, poses[i % 2])
                    sa = hr.hr_render_frame(ctx, asset, w.n_clusters, w.eps_w, 0, da, hout,
                                            stats=True)
                    refits += sa.bvh_refit
                    bvh.append(sa.bvh_ms)
                torch.cuda.synchronize(dev)
                dt = (time.perf_counter() - t0) / animation["frames"]
                res[key] = {"ms_per_frame": dt * 1e3, "bvh_ms": statistics.median(bvh),
                            "bvh_refits": refits, "h2d_bytes_per_frame": pv.numel() * 4}
                # the same frames without statistics (device image, copied back
                # asynchronously): each frame's upload, clusters and fit
                # overlap the previous frame
                for i in range(2):
                    hr.hr_asset_update(ctx, asset, poses[i])
                    hr.hr_render_frame(ctx, asset, w.n_clusters, w.eps_w, 0, da, img_e)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                for i in range(animation["frames"]):
                    hr.hr_asset_update(ctx, asset, poses[i % 2])
                    hr.hr_render_frame(ctx, asset, w.n_clusters, w.eps_w, 0, da, img_e)
                    with torch.cuda.stream(stream):
                        hout.copy_(img_e, non_blocking=True)
                torch.cuda.synchronize(dev)
                dto = (time.perf_counter() - t0) / animation["frames"]
                _, _, fl = hr.hr_frame_times(ctx, animation["frames"], with_flags=True)
                res[key]["ms_per_frame_overlapped"] = dto * 1e3
                res[key]["bvh_refits_overlapped"] = int(((fl >> 1) & 1).sum())
            # the guide-driven hierarchy, once, then skinned frames
            G = 256
            hr.hr_asset_update(ctx, asset, pv)
            t0 = time.perf_counter()
            hr.hr_build_guided_clusters(ctx, asset, G, 4)
            torch.cuda.synchronize(dev)
            build_s = time.perf_counter() - t0
            gid = np.zeros(G, np.int32)
            hr.hr_guides_export(ctx, asset, gid)
            gposes = []
            for vv in (moved, w.scene.verts):
                gv = np.zeros((G, w.scene.verts.shape[1], 4), np.float32)
                ok = gid >= 0
                gv[ok] = vv[gid[ok]]
                gposes.append(torch.from_numpy(gv).pin_memory())
            ds = hr.render_desc(w.camera.pack(), w.lights, w.spp, w.k_depth, w.sample_seed,
                                w.precision, hr.HR_FLAG_KEEP_HIERARCHY | hr.HR_FLAG_REFIT |
                                hr.HR_FLAG_DEFERRED_LOD | hr.HR_FLAG_LOD_HYSTERESIS)
            for i in range(2):
                hr.hr_asset_skin(ctx, asset, gposes[i])
                hr.hr_render_frame(ctx, asset, 0, w.eps_w, 0, ds, hout)
            torch.cuda.synchronize(dev)
            refits, bvh = 0, []
            t0 = time.perf_counter()
            for i in range(animation["frames"]):
                hr.hr_asset_skin(ctx, asset, gposes[i % 2])
                sa = hr.hr_render_frame(ctx, asset, 0, w.eps_w, 0, ds, hout, stats=True)
                refits += sa.bvh_refit
                bvh.append(sa.bvh_ms)
            torch.cuda.synchronize(dev)
            dt = (time.perf_counter() - t0) / animation["frames"]
            C_g, L_g, E_g = hr.hr_hierarchy_info(ctx, asset)
            res["skinned"] = {"ms_per_frame": dt * 1e3, "bvh_ms": statistics.median(bvh),
                              "bvh_refits": refits, "h2d_bytes_per_frame": gposes[0].numel() * 4,
                              "guides": G, "clusters": C_g, "levels": L_g,
                              "guided_build_ms": build_s * 1e3}
            animation[f"displacement_{amp:g}"] = res
        hr.hr_asset_update(ctx, asset, pv)

    serving = None
    if not args.no_serve and rank == 0 and world == 1:
        serving = run_serving(hr, ctx, torch, dev, args.serve_requests)

    # the other configurations, one step each (host-timed, synchronous calls)
    other_configs = None
    if not args.no_configs and rank == 0:
        import scenegen
        props0 = torch.cuda.get_device_properties(dev)
        peak0 = props0.multi_processor_count * 128 * 2 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
        other_configs = [measure_config(hr, ctx, torch, dev, cw, 5, peak_tflops=peak0) for cw in (
            scenegen.tiny_strands(),
            scenegen.clustered(lod_setting="strands"), scenegen.clustered(lod_setting="half"),
            scenegen.clustered(lod_setting="eth"),
            scenegen.full_head(precision=1),
            scenegen.full_head(fill=0.45),  # middle view: hair 45% of the frame height
            scenegen.full_head(fill=0.9),  # close view: hair 90% of the frame height, all strands
            scenegen.stress())]

    hr.hr_asset_destroy(ctx, asset)
    hr.hr_destroy(ctx)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(dev)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    sm_load = clocks.get("sm_mhz") or sm_max
    peak_load = props.multi_processor_count * 128 * 2 * sm_load * 1e6 / 1e12
    achieved = flops / (render_avg * 1e-3) / 1e12
    flops_src = event_flops_source(cst)
    roof_frame = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                  "frac": achieved / peak,
                  "frac_source_count": flops_src / (render_avg * 1e-3) / 1e12 / peak,
                  "flops_per_event": {"node": FLOPS_PER_NODE, "test": FLOPS_PER_TEST,
                                      "strand_shade": FLOPS_PER_STRAND_SHADE,
                                      "eth_shade": FLOPS_PER_ETH_SHADE, "hit": FLOPS_PER_HIT,
                                      "traced_sample": FLOPS_PER_SAMPLE},
                  "traffic": traffic_record("k_frame_full_head_traffic.json", TRACE_SOURCES, w.name),
                  "kernel": "k_frame (trace/shade/composite, FP32)", "kernel_ms": render_avg,
                  "flops_per_launch": flops,
                  "peak_basis": f"FP32: {props.multi_processor_count} SMs x 128 lanes x 2 (FMA) x "
                                f"{sm_max:.0f} MHz (derived from unit counts and clock)",
                  "peak_at_load_clock": peak_load, "frac_at_load_clock": achieved / peak_load,
                  "frac_standalone": flops / (fp32_ms * 1e-3) / 1e12 / peak,
                  "kernel_ms_standalone": fp32_ms,
                  "kernel_ms_note": "kernel_ms: the timed steps' frames, each overlapping the next "
                                    "step's clusters and fit; kernel_ms_standalone: the same frame "
                                    "alone (median of 10)",
                  "events": {"node_visits": cst.node_visits, "prim_tests": cst.prim_tests,
                             "strand_shades": cst.strand_shades, "eth_shades": cst.eth_shades,
                             "hits": cst.shaded_hits, "traced_samples": cst.traced_samples,
                             "samples": samples, "refined_tests": cst.refined_tests,
                             "refined_entries": cst.refined_entries}}
    # FP32 work of the cross-section fit: every strand is a member of one thick
    # hair per level, so the members sum to N * levels over S+1 sections
    C_, L_, E_ = n_levels_info
    fit_avg = statistics.mean(fit_ms)
    fit_flops = (w.scene.n_segments + 1) * (FIT_FLOPS_PER_SECTION * E_ +
                                            FIT_FLOPS_PER_MEMBER * w.scene.n_strands * L_)
    fit_ach = fit_flops / (fit_avg * 1e-3) / 1e12 if fit_avg > 0 else 0.0
    roof_fit = {"bound": "alu", "achieved": fit_ach, "peak": peak, "unit": "TFLOP/s",
                "frac": fit_ach / peak,
                "traffic": traffic_record("k_fit_cross_sections_full_head_traffic.json",
                                          FIT_SOURCES, w.name),
                "kernel": "k_fit_cross_sections (thick-hair fit, double-word FP32)",
                "kernel_ms": fit_avg, "flops_per_launch": fit_flops,
                "peak_basis": roof_frame["peak_basis"]}
    dominant_fit = fit_avg >= render_avg
    roof = dict(roof_fit if dominant_fit else roof_frame)
    roof["dominant_by_time_in_step"] = True
    other = roof_frame if dominant_fit else roof_fit
    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_baseline(w, args.cpu_seconds)
    line = {"metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_of(w, args),
            "traced_samples": int(cst.traced_samples),
            "traced_msamples_per_s": job_msamples_per_s(world, int(cst.traced_samples), args.steps,
                                                        elapsed),
            "traced_msamples_per_s_frame": cst.traced_samples / (render_avg * 1e-3) / 1e6,
            "frame_ms": render_avg, "frame_ms_fp32_warm": fp32_ms, "frame_ms_fp16_warm": fp16_ms,
            "frame_ms_shadow_rays": shadow_ms, "frame_tail": tail, "tile_schedule": tile_schedule,
            "active_prims": int(st.n_active_prims),
            "eth_prims": int(st.n_eth_prims), "stack_overflows": int(st.stack_overflows),
            "roofline": roof, "roofline_other": other,
            "phase_ms": {"hierarchy": st.hierarchy_ms, "fit": st.fit_ms, "lod": st.lod_ms,
                         "bvh": st.bvh_ms, "render": st.render_ms,
                         "note": "one step with statistics after the timed region (no overlap)"},
            "step_overlap": "each timed step's clusters and fit run on a second stream while the "
                            "previous step's frame renders (hr_render_frame pipelining)",
            "cpu_baseline": cpu,
            "e2e": e2e, "animation": animation, "other_configs": other_configs,
            "gpu_launches": launches, "clocks": clocks, "serving": serving}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
