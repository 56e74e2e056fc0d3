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

pytestmark = pytest.mark.gpu


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
    vals = torch.zeros(capacity, dtype=torch.int32, device=dev)
    keys = torch.zeros(capacity, dtype=torch.int64, device=dev)
    ranges = torch.zeros_like(vb.ranges)
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    rc = L.lib().dg_bin_sort_noalloc(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan), capacity,
                                     L.ptr(keys), L.ptr(vals), L.ptr(ranges), L.ptr(count), L.ptr(status),
                                     L.stream_handle())
    assert rc == L.DG_OK
    return vals, keys, ranges, count, status


def test_noalloc_matches_workspace_entry_point_twice(mods):
    L, D = mods
    cases = [(S.cube_scene(4096, 1001), [S.cube_camera()], [0, 4096]),
             (S.cube_scene(9000, 77, log_scale_mu=-2.4), [S.cube_camera(200, 150, f=160.0),
                                                          S.cube_camera(96, 120, f=90.0)], [0, 9000])]
    for g, cams, off in cases:
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
        assert torch.equal(ranges, vb.ranges)


def test_noalloc_rejects_sizes_beyond_its_limit(mods):
    L, D = mods
    xb, vb = project_batch(D, S.cube_scene(100, 3), [S.cube_camera()], [0, 100])
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = L.lib().dg_bin_sort_noalloc(L.ptr(vb.rec), L.ptr(vb.rect), L.ptr(vb.dev_cams), C.byref(vb.plan),
                                     L.DG_NOALLOC_MAX_INSTANCES + 1, None, L.ptr(dummy), L.ptr(vb.ranges),
                                     L.ptr(dummy), L.ptr(dummy), L.stream_handle())
    assert rc == L.DG_ERR_TOO_LARGE
