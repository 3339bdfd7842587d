"""The allocation-free Morton clustering entry point against hr_build_clusters.

hr_morton_clusters_noalloc exists for callers that may not let a library
allocate device memory (a host application owning every allocation under a
fixed budget, or a loop where cudaMalloc / cudaFree must not run because they
synchronise the device).  It keeps its scratch in one fixed device array that
every call reuses, so this test calls it several times in a row on different
inputs and checks each result against the allocating entry point.  Strand
orders and cluster ids are integers: the comparison is exact.
"""
import numpy as np
import pytest

import paper_2405_10565_gb300 as hr
import scenegen

pytestmark = pytest.mark.gpu


def _reference(ctx, scene, C):
    a = hr.hr_asset_create(ctx, scene.verts, scene.mat, scene.shape)
    try:
        order = np.zeros(scene.n_strands, np.uint32)
        cl = np.zeros(scene.n_strands, np.uint32)
        hr.hr_build_clusters(ctx, a, C, 0, cl, order)
        return order, cl
    finally:
        hr.hr_asset_destroy(ctx, a)


def test_noalloc_clusters_match_allocating_entry_point():
    torch = pytest.importorskip("torch")
    from paper_2405_10565_gb300.build import build
    build()
    dev = torch.device("cuda:0")
    scenes = [(scenegen.full_head(n=60000, S=8, width=8, height=8, spp=1, n_lights=1).scene, 2400),
              (scenegen.clustered(n=7000, S=6, res=8, spp=1).scene, 256)]
    ctx = hr.hr_create(0)
    try:
        refs = [_reference(ctx, sc, C) for sc, C in scenes]
    finally:
        hr.hr_destroy(ctx)
    stream = torch.cuda.Stream(device=dev)
    # two calls in a row on each input, alternating inputs, outputs pre-filled
    # with garbage so a skipped write shows
    for sc, C in (scenes[0], scenes[0], scenes[1], scenes[0]):
        i = 0 if sc is scenes[0][0] else 1
        verts = torch.from_numpy(sc.verts).to(dev)
        order = torch.full((sc.n_strands,), -1, dtype=torch.int32, device=dev)
        cl = torch.full((sc.n_strands,), -1, dtype=torch.int32, device=dev)
        torch.cuda.synchronize(dev)
        hr.hr_morton_clusters_noalloc(verts, C, order, cl, stream.cuda_stream)
        stream.synchronize()
        assert np.array_equal(order.cpu().numpy().view(np.uint32), refs[i][0])
        assert np.array_equal(cl.cpu().numpy().view(np.uint32), refs[i][1])


def test_noalloc_rejects_oversize_and_host_buffers():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    v = torch.zeros((4, 3, 4), device=dev)
    o = torch.zeros(4, dtype=torch.int32, device=dev)
    c = torch.zeros(4, dtype=torch.int32, device=dev)
    lib = hr.load()
    # a strand count beyond the fixed scratch is refused before any work
    st = lib.hr_morton_clusters_noalloc(hr.ptr(v), hr.HR_NOALLOC_MAX_STRANDS + 1, 2, 1,
                                        hr.ptr(o), hr.ptr(c), None)
    assert st == hr.HR_EINVAL
    # host memory is not accepted
    h = np.zeros(4, np.uint32)
    st = lib.hr_morton_clusters_noalloc(hr.ptr(v), 4, 2, 2, h.ctypes.data, hr.ptr(c), None)
    assert st == hr.HR_EINVAL
