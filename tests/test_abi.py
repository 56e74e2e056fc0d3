"""CPU checks of the C ABI: the library loads without a GPU, exports every
function include/dogs.h declares, the ctypes mirrors have the C layout, and
the host-side batch planning validates its inputs."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2405_13943_b300 import _lib as L
from paper_2405_13943_b300 import build as B
from paper_2405_13943_b300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dogs.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.exported_symbols())


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dogs.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(dg_gaussians), sizeof(dg_camera),'
                   ' sizeof(dg_plan), offsetof(dg_camera, rec_off), offsetof(dg_camera, gauss_end),'
                   ' offsetof(dg_plan, blk_off), offsetof(dg_plan, blk_view_off), offsetof(dg_plan, max_height));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(L.DgGaussians), C.sizeof(L.DgCamera), C.sizeof(L.DgPlan),
            L.DgCamera.rec_off.offset, L.DgCamera.gauss_end.offset, L.DgPlan.blk_off.offset,
            L.DgPlan.blk_view_off.offset, L.DgPlan.max_height.offset]
    assert got == want


def test_plan_numbering(lib):
    from paper_2405_13943_b300 import dogs as D
    cams = [S.cube_camera(40, 35), S.cube_camera(64, 48), S.cube_camera(17, 90)]
    cams[0].block, cams[1].block, cams[2].block = 0, 0, 2
    arr, plan = D.plan_views(cams, [0, 100, 150, 400], 16, 16)
    assert plan.n_views == 3 and plan.n_blocks == 3
    assert [arr[i].rec_off for i in range(3)] == [0, 100, 200]
    assert plan.n_rec == 450
    assert [arr[i].tiles_x for i in range(3)] == [3, 4, 2]
    assert [arr[i].tile_off for i in range(3)] == [0, 9, 21]
    assert plan.n_tiles == 9 + 12 + 12
    assert [arr[i].pix_off for i in range(3)] == [0, 1400, 1400 + 3072]
    assert list(plan.blk_view_off[:4]) == [0, 2, 2, 3]
    assert (arr[2].gauss_begin, arr[2].gauss_end) == (150, 400)
    assert (plan.max_width, plan.max_height) == (64, 90)


def test_plan_rejects_bad_input(lib):
    from paper_2405_13943_b300 import dogs as D
    cams = [S.cube_camera(40, 35), S.cube_camera(64, 48)]
    cams[0].block, cams[1].block = 1, 0           # not grouped by ascending block
    with pytest.raises(L.DogsError):
        D.plan_views(cams, [0, 10, 20], 16, 16)
    cams[0].block, cams[1].block = 0, 0
    with pytest.raises(L.DogsError):
        D.plan_views(cams, [0, 10, 20], 16, 8)     # unsupported tile shape
    with pytest.raises(L.DogsError):
        D.plan_views(cams, [0, 30, 20], 16, 16)    # decreasing block offsets
    bad = [S.cube_camera(0, 35)]
    with pytest.raises(L.DogsError):
        D.plan_views(bad, [0, 10], 16, 16)


def test_pack_unpack_roundtrip():
    from paper_2405_13943_b300 import dogs as D
    g = S.cube_scene(37, 3, sh_degree=3)
    a = D.GaussianBuffer.pack(g)
    h = D.GaussianBuffer.unpack(a, 37, 3, 64)
    for f in ("means", "quats", "log_scales", "opacity_logits", "sh"):
        np.testing.assert_array_equal(getattr(g, f), getattr(h, f))
    assert a.size == (12 + 48) * 64


def test_calls_reject_null_arguments_without_touching_the_gpu(lib):
    """Argument checks happen on the host, before any launch."""
    plan = L.DgPlan()
    g = L.DgGaussians(None, 10, 8, 0, 0)           # ld < n
    assert lib.dg_project(C.byref(g), None, C.byref(plan), None, None, None) == L.DG_ERR_INVALID
    assert lib.dg_gaussian_floats(64, 3) == 60 * 64
    assert lib.dg_gaussian_floats(64, 4) == -1


def test_misaligned_pointers_are_rejected_before_launch(lib):
    """Vector-accessed buffers must carry their alignment; a violation is an
    argument error found on the host, never a device fault."""
    from paper_2405_13943_b300 import dogs as D
    arr, plan = D.plan_views([S.cube_camera(32, 32)], [0, 64], 16, 16)
    g = L.DgGaussians(0x10000, 64, 64, 0, 0)
    assert lib.dg_project(C.byref(g), 0x20000, C.byref(plan), 0x30008, 0x40000, None) == L.DG_ERR_INVALID
    assert lib.dg_project(C.byref(g), 0x20000, C.byref(plan), 0x30000, 0x40004, None) == L.DG_ERR_INVALID
    x = L.DgGaussians(0x10000, 64, 64, 0, 0)
    rho = L.floats([1] * 5)
    lr = L.floats([1] * 6)
    assert lib.dg_adam_admm_step(C.byref(x), C.byref(x), C.byref(x), C.byref(x), None, None, rho, lr,
                                 0.9, 0.999, 1e-15, 1, 0x50002, None) == L.DG_ERR_INVALID


def test_xstep_part_rejects_bad_arguments_before_launch(lib):
    """dg_xstep_part validates its part, grid bound and z store on the host."""
    from paper_2405_13943_b300 import dogs as D
    arr, plan = D.plan_views([S.cube_camera(32, 32)], [0, 64], 16, 16)
    x = L.DgGaussians(0x10000, 64, 64, 0, 0)
    z = L.DgGaussians(0x20000, 32, 64, 0, 0)
    z1 = L.DgGaussians(0x20000, 32, 64, 1, 0)          # another SH degree
    rho, lr = L.floats([1] * 5), L.floats([1] * 6)
    rect, cams, drec, shared, gid = 0x30000, 0x40000, 0x50000, 0x60000, 0x70000

    def call(part, ctas, zz=None, g=None, sh=shared, d=drec):
        return lib.dg_xstep_part(part, ctas, rect, cams, C.byref(plan), d, C.byref(x), C.byref(x), C.byref(x),
                                 None, sh, rho, lr, 0.9, 0.999, 1e-15, 1, None,
                                 None if zz is None else C.byref(zz), g, None)
    for part, ctas in ((-1, 0), (3, 0), (1, -1)):
        assert call(part, ctas) == L.DG_ERR_INVALID
    assert call(2, 0, d=None) == L.DG_ERR_INVALID             # part 2 needs the record gradients
    assert call(0, 0, z, None) == L.DG_ERR_INVALID            # a z store needs the global ids
    assert call(0, 0, z, gid, sh=None) == L.DG_ERR_INVALID    # ... and the shared flags
    assert call(0, 0, z1, gid) == L.DG_ERR_INVALID            # ... and the same SH degree
    assert call(0, 0, z, gid + 2) == L.DG_ERR_INVALID         # misaligned ids


def test_xstep_stream_rejects_bad_arguments_before_launch(lib):
    """dg_xstep_stream makes dg_xstep_part's checks and checks its grid bound
    and workspace on the host; the workspace is two counters and one list
    entry per group of 128 copies."""
    from paper_2405_13943_b300 import dogs as D
    arr, plan = D.plan_views([S.cube_camera(32, 32)], [0, 300], 16, 16)
    x = L.DgGaussians(0x10000, 300, 300, 0, 0)
    z = L.DgGaussians(0x20000, 32, 64, 0, 0)
    rho, lr = L.floats([1] * 5), L.floats([1] * 6)
    rect, cams, shared, gid, ws = 0x30000, 0x40000, 0x60000, 0x70000, 0x80000
    need = lib.dg_xstep_stream_workspace_size(C.byref(x))
    assert need == 16 + 4 * 3
    assert lib.dg_xstep_stream_workspace_size(C.byref(L.DgGaussians(0x10000, 300, 298, 0, 0))) == 0   # ld < n

    def call(ctas=0, zz=None, g=None, w=ws, nb=need, sh=shared):
        return lib.dg_xstep_stream(ctas, rect, cams, C.byref(plan), C.byref(x), C.byref(x), C.byref(x), None, sh,
                                   rho, lr, 0.9, 0.999, 1e-15, 1, None, None if zz is None else C.byref(zz), g,
                                   w, nb, None)
    assert call(ctas=-1) == L.DG_ERR_INVALID
    assert call(ctas=65536) == L.DG_ERR_INVALID
    assert call(zz=z) == L.DG_ERR_INVALID                    # a z store needs the global ids
    assert call(zz=z, g=gid, sh=None) == L.DG_ERR_INVALID    # ... and the shared flags
    assert call(w=None) == L.DG_ERR_INVALID
    assert call(w=ws + 8) == L.DG_ERR_INVALID                # misaligned workspace
    assert call(nb=need - 1) == L.DG_ERR_WORKSPACE


def test_xstep_listed_rejects_bad_arguments_before_launch(lib):
    """dg_xstep_groups checks the plan, pointers and workspace; dg_xstep_listed
    makes dg_xstep_part's checks, takes parts 1 and 2 only and checks its grid
    bound and workspace, all on the host."""
    from paper_2405_13943_b300 import dogs as D
    arr, plan = D.plan_views([S.cube_camera(32, 32)], [0, 300], 16, 16)
    x = L.DgGaussians(0x10000, 300, 300, 0, 0)
    rho, lr = L.floats([1] * 5), L.floats([1] * 6)
    rect, cams, drec, shared, ws = 0x30000, 0x40000, 0x50000, 0x60000, 0x80000
    need = lib.dg_xstep_stream_workspace_size(C.byref(x))

    def groups(r=rect, w=ws, nb=need, xx=x):
        return lib.dg_xstep_groups(r, cams, C.byref(plan), C.byref(xx), w, nb, None)
    assert groups(r=None) == L.DG_ERR_INVALID
    assert groups(r=rect + 4) == L.DG_ERR_INVALID               # misaligned rectangles
    assert groups(w=None) == L.DG_ERR_INVALID
    assert groups(w=ws + 8) == L.DG_ERR_INVALID
    assert groups(nb=need - 1) == L.DG_ERR_WORKSPACE
    assert groups(xx=L.DgGaussians(0x10000, 200, 200, 0, 0)) == L.DG_ERR_INVALID   # the plan spans 300 copies

    def listed(part=2, ctas=0, d=drec, w=ws, nb=need):
        return lib.dg_xstep_listed(part, ctas, rect, cams, C.byref(plan), d, C.byref(x), C.byref(x), C.byref(x),
                                   None, shared, rho, lr, 0.9, 0.999, 1e-15, 1, None, None, None, w, nb, None)
    for part in (0, 3, -1):
        assert listed(part=part) == L.DG_ERR_INVALID
    assert listed(ctas=-1) == L.DG_ERR_INVALID
    assert listed(ctas=65536) == L.DG_ERR_INVALID
    assert listed(d=None) == L.DG_ERR_INVALID                   # part 2 reads the records' gradients
    assert listed(d=drec + 8) == L.DG_ERR_INVALID
    assert listed(w=ws + 4) == L.DG_ERR_INVALID
    assert listed(nb=need - 4) == L.DG_ERR_WORKSPACE
    assert listed(part=1, nb=need - 4) == L.DG_ERR_WORKSPACE


def test_xstep_calls_on_no_copies_return_ok_without_the_device(lib):
    """With no copies, the x-step entry points check their arguments and
    return DG_OK without any device call (this runs without a GPU)."""
    from paper_2405_13943_b300 import dogs as D
    arr, plan = D.plan_views([S.cube_camera(32, 32)], [0, 0], 16, 16)
    x = L.DgGaussians(0x10000, 0, 0, 0, 0)
    rho, lr = L.floats([1] * 5), L.floats([1] * 6)
    cams, nb = 0x40000, lib.dg_xstep_stream_workspace_size(C.byref(x))
    assert nb == 16
    assert lib.dg_xstep_groups(None, cams, C.byref(plan), C.byref(x), None, nb, None) == L.DG_OK
    for part in (1, 2):
        assert lib.dg_xstep_listed(part, 0, None, cams, C.byref(plan), None, C.byref(x), C.byref(x), C.byref(x),
                                   None, None, rho, lr, 0.9, 0.999, 1e-15, 1, None, None, None, None, nb,
                                   None) == L.DG_OK
        assert lib.dg_xstep_part(part, 0, None, cams, C.byref(plan), None, C.byref(x), C.byref(x), C.byref(x),
                                 None, None, rho, lr, 0.9, 0.999, 1e-15, 1, None, None, None, None) == L.DG_OK
    assert lib.dg_xstep_stream(0, None, cams, C.byref(plan), C.byref(x), C.byref(x), C.byref(x), None, None,
                               rho, lr, 0.9, 0.999, 1e-15, 1, None, None, None, None, nb, None) == L.DG_OK


def test_render_slot_workspace_bounds_every_admissible_batch(lib):
    """The render server sizes a slot's workspace once, on the host, for any
    batch of at most max_batch views and max_batch_pixels pixels: random mixes
    of the served resolutions never need more (host-only queries, no GPU)."""
    from paper_2405_13943_b300 import dogs as D
    from paper_2405_13943_b300 import serve

    class Z:
        n = 6_000_000
    res = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]
    server = serve.RenderServer(Z(), max_batch=8, resolutions=res, inst_per_pixel=2.5)
    bound = server._slot_ws_bytes()
    rng = np.random.default_rng(0)
    for _ in range(200):
        k = int(rng.integers(1, 9))
        pick = [res[i] for i in rng.integers(0, 4, k)]
        cams, npix = [], 0
        for w, h in pick:
            if cams and npix + w * h > server.max_batch_pixels:
                break
            cams.append(S.Camera(w, h, float(w), float(w), w / 2, h / 2, np.eye(3, dtype=np.float32),
                                 np.zeros(3, np.float32), np.zeros(3, np.float32)))
            npix += w * h
        _, plan = D.render_plan(cams, Z.n)
        need = lib.dg_render_workspace_size(C.byref(plan), server._capacity_for(npix))
        assert 0 < need <= bound


def test_slot_backward_rejects_bad_arguments_before_launch(lib):
    from paper_2405_13943_b300 import dogs as D
    arr, plan = D.plan_views([S.cube_camera(32, 32)], [0, 64], 16, 16)
    need = lib.dg_rasterize_bwd_slots_workspace_size(C.byref(plan))
    assert need >= 64 * 8
    bg = L.floats([0, 0, 0])
    launches = lib.dg_launch_count()

    def call(rec=0x10000, rect=0x20000, part=0x90000, cap=100, ws=0xA0000, wsb=need, slots=0xB0000):
        return lib.dg_rasterize_bwd_slots(rec, rect, 0x30000, 0x40000, 0x50000, C.byref(plan), bg, 0x60000,
                                          0x70000, 0x80000, part, cap, ws, wsb, slots, 0xC0000, 0xD0000, None)
    assert call(rec=0x10008) == L.DG_ERR_INVALID          # records are read as float4
    assert call(rect=0x20004) == L.DG_ERR_INVALID         # rectangles as uint2
    assert call(cap=-1) == L.DG_ERR_INVALID
    assert call(part=None) == L.DG_ERR_INVALID
    assert call(slots=0xB0004) == L.DG_ERR_INVALID        # the slot total is 64-bit
    assert call(wsb=need - 8) == L.DG_ERR_WORKSPACE
    assert lib.dg_launch_count() == launches


def test_bin_sort_workspace_sizes(lib):
    """The binning workspace: the full size holds 4 bytes a record more than
    the minimum (the visible-record list), and a workspace below the minimum
    is refused on the host before any launch."""
    from paper_2405_13943_b300 import dogs as D
    cams = [S.cube_camera(64, 48), S.cube_camera(40, 40)]
    cams[1].block = 1
    arr, plan = D.plan_views(cams, [0, 1000, 1600], 16, 16)
    cap = 5000
    full = lib.dg_bin_sort_workspace_size(C.byref(plan), cap)
    small = lib.dg_bin_sort_workspace_min_size(C.byref(plan), cap)
    assert full >= small + 4 * plan.n_rec and full - small <= 4 * plan.n_rec + 255
    assert small > 8 * cap
    call = lambda ws, nb: lib.dg_bin_sort(0x10000, 0x20000, 0x30000, C.byref(plan), cap, None, 0x40000, 0x50000,
                                          0x60000, ws, nb, 0x70000, None)
    assert call(0x100000, small - 1) == L.DG_ERR_WORKSPACE
    assert call(0x100008, full) == L.DG_ERR_INVALID           # the workspace must be 256-byte aligned
    assert call(None, full) == L.DG_ERR_INVALID
