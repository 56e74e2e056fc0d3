"""dg_bin_sort_noalloc, the binning entry point for callers that cannot
allocate device memory (a plugin whose host application owns the device's
memory, a loop that must not pay cudaMalloc's synchronisation).  It keeps its
scratch in a static array of the library; this test calls it through the C
ABI twice in a row, on two different inputs, and checks every output against
dg_bin_sort with a caller workspace: the work is integer, so bit for bit.
The file is named to be collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import synth as S



@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from paper_2405_13943_b300 import _lib, dogs
    return _lib, dogs


def project_batch(D, g, cams, blk_off):
    xb = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch(cams, blk_off, 16, 16, keep_keys=True, capacity=1 << 20)
    D.dg_project(xb, vb)
    return xb, vb


def outputs_noalloc(L, vb, capacity):
    dev = vb.rec.device
    vals = torch.full((capacity,), -1, dtype=torch.int32, device=dev)
    keys = torch.full((capacity,), -1, dtype=torch.int64, device=dev)
    ranges = torch.full_like(vb.ranges, -1)
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = L.lib().dg_bin_sort_noalloc(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), capacity,
                                     L.ptr(keys), L.ptr(vals), L.ptr(ranges), L.ptr(count), L.ptr(status),
                                     L.stream_handle())
    assert rc == L.DG_OK
    return vals, keys, ranges, count, status


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_twice(mods):
    """A small problem, a larger one, then the small one again: each call
    equals dg_bin_sort bit for bit, so nothing a larger call left in the
    shared array leaks into a later, smaller one.  The outputs start filled
    with a pattern, so every element compared was written by the call."""
    L, D = mods
    small = (S.cube_scene(4096, 1001), [S.cube_camera()], [0, 4096])
    large = (S.cube_scene(9000, 77, log_scale_mu=-2.4), [S.cube_camera(200, 150, f=160.0),
                                                         S.cube_camera(96, 120, f=90.0)], [0, 9000])
    for g, cams, off in (small, large, small):
        xb, vb = project_batch(D, g, cams, off)
        vb.status.zero_()
        D.dg_bin_sort(vb)
        torch.cuda.synchronize()
        m = int(vb.count.item())
        assert 0 < m <= vb.capacity and int(vb.status.item()) == 0
        vals, keys, ranges, count, status = outputs_noalloc(L, vb, vb.capacity)
        torch.cuda.synchronize()
        assert int(count.item()) == m and int(status.item()) == 0
        assert torch.equal(vals[:m], vb.vals[:m])
        assert torch.equal(keys[:m], vb.keys[:m])
        n = vb.n_tiles
        assert torch.equal(ranges[:2 * n], vb.ranges[:2 * n])
        # the work order: every tile once (its order within a magnitude is unspecified)
        assert torch.equal(torch.sort(ranges[2 * n:3 * n]).values, torch.sort(vb.ranges[2 * n:3 * n]).values)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_limit(mods):
    L, D = mods
    xb, vb = project_batch(D, S.cube_scene(100, 3), [S.cube_camera()], [0, 100])
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = L.lib().dg_bin_sort_noalloc(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan),
                                     L.DG_NOALLOC_MAX_INSTANCES + 1, None, L.ptr(dummy), L.ptr(vb.ranges),
                                     L.ptr(dummy), L.ptr(dummy), L.stream_handle())
    assert rc == L.DG_ERR_TOO_LARGE


def test_noalloc_rejects_bad_arguments_on_the_host():
    """The entry point checks its arguments as dg_bin_sort does, on the host
    and before any launch (no GPU is needed to see it): an unsupported tile
    shape, a misaligned record or rectangle pointer, a capacity beyond 32-bit
    instance numbers."""
    from paper_2405_13943_b300 import _lib as L
    from paper_2405_13943_b300 import build as B
    from paper_2405_13943_b300 import dogs as D
    B.build()
    lib = L.lib()
    arr, plan = D.plan_views([S.cube_camera(32, 32)], [0, 64], 16, 16)
    rec, rect, cams, keys, vals, ranges, cnt, st = 0x10000, 0x20000, 0x30000, 0x40000, 0x50000, 0x60000, 0x70000, \
        0x80000
    launches = lib.dg_launch_count()

    def call(p=plan, r=rec, rc_=rect, k=keys, cap=1024):
        return lib.dg_bin_sort_noalloc(r, rc_, cams, C.byref(p), cap, k, vals, ranges, cnt, st, None)
    assert call(r=rec + 8) == L.DG_ERR_INVALID                 # records are read as float4
    assert call(rc_=rect + 4) == L.DG_ERR_INVALID              # rectangles as uint2
    assert call(k=keys + 4) == L.DG_ERR_INVALID                # keys are 64-bit
    assert call(cap=-1) == L.DG_ERR_INVALID
    assert call(cap=0xFFFFFFFF) == L.DG_ERR_INVALID
    bad = L.DgPlan.from_buffer_copy(plan)
    bad.tile_h = 8                                             # 16x8 is not a supported tile shape
    assert call(p=bad) == L.DG_ERR_INVALID
    assert lib.dg_launch_count() == launches
