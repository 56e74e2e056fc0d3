"""ctypes binding of libdogs (include/dogs.h): argument marshalling only.

Every function here takes torch tensors (device memory from PyTorch) and
plain Python values, turns them into the C ABI's pointers and structs, calls
the library on the current torch stream, and raises DogsError on a non-zero
status.  No arithmetic of the method happens here.  If libdogs.so is
missing, importing the binding fails: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdogs.so")

DG_OK, DG_ERR_INVALID, DG_ERR_WORKSPACE, DG_ERR_CAPACITY, DG_ERR_CUDA = 0, -1, -2, -3, -4
DG_ERR_TOO_LARGE = -6
DG_ERR_HOST_MEMORY = -7
DG_NOALLOC_MAX_TILES, DG_NOALLOC_MAX_INSTANCES = 262144, 4194304
DG_STATUS_CAPACITY = 1
DG_DENSIFY_KEEP, DG_DENSIFY_PRUNE, DG_DENSIFY_CLONE, DG_DENSIFY_SPLIT = 0, 1, 2, 3
DG_MAX_BLOCKS = 64
DG_MAX_VIEWS = 4096

_ERR = {DG_ERR_INVALID: "invalid argument", DG_ERR_WORKSPACE: "workspace too small",
        DG_ERR_CAPACITY: "capacity", DG_ERR_CUDA: "CUDA launch failed",
        DG_ERR_TOO_LARGE: "beyond the fixed limits of the allocation-free entry point",
        DG_ERR_HOST_MEMORY: "host memory could not be allocated"}


class DogsError(RuntimeError):
    pass


class DgGaussians(C.Structure):
    _fields_ = [("data", C.c_void_p), ("n", C.c_int64), ("ld", C.c_int64),
                ("sh_degree", C.c_int32), ("reserved", C.c_int32)]


class DgCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32),
                ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("R", C.c_float * 9), ("t", C.c_float * 3), ("campos", C.c_float * 3),
                ("near_z", C.c_float), ("block", C.c_int32),
                ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("tile_off", C.c_int32),
                ("reserved", C.c_int32), ("rec_off", C.c_int64), ("pix_off", C.c_int64),
                ("gauss_begin", C.c_int64), ("gauss_end", C.c_int64)]


class DgPlan(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("n_blocks", C.c_int32),
                ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("n_rec", C.c_int64), ("n_tiles", C.c_int64), ("n_pixels", C.c_int64),
                ("blk_off", C.c_int64 * (DG_MAX_BLOCKS + 1)),
                ("blk_view_off", C.c_int32 * (DG_MAX_BLOCKS + 1)),
                ("max_width", C.c_int32), ("max_height", C.c_int32),
                ("raster_warps", C.c_int32), ("raster_stage", C.c_int32),
                ("raster_warps_bwd", C.c_int32), ("raster_stage_bwd", C.c_int32)]


_vp = C.c_void_p
_SIGS = {
    "dg_version": (C.c_char_p, []),
    "dg_launch_count": (C.c_uint64, []),
    "dg_histogram_i32": (C.c_int, [_vp, C.c_int64, C.c_int32, C.c_int, _vp, _vp]),
    "dg_densify_layout_workspace_size": (C.c_size_t, [C.c_int64, C.c_int64]),
    "dg_densify_layout": (C.c_int, [_vp, _vp, C.c_int64, _vp, _vp, _vp, C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp,
                                    C.c_size_t, _vp]),
    "dg_rasterize_bwd_slots_workspace_size": (C.c_size_t, [C.POINTER(DgPlan)]),
    "dg_rasterize_bwd_slots": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(DgPlan), C.POINTER(C.c_float), _vp, _vp,
                                         _vp, _vp, C.c_int64, _vp, C.c_size_t, _vp, _vp, _vp, _vp]),
    "dg_admm_adapt": (C.c_int, [_vp, _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, C.c_int, _vp]),
    "dg_admm_rescale": (C.c_int, [C.POINTER(DgGaussians), C.POINTER(DgGaussians), C.POINTER(DgGaussians), _vp, _vp,
                                  _vp, _vp]),
    "dg_probe_fma": (C.c_int64, [C.c_int, C.c_int, _vp, _vp]),
    "dg_gaussian_floats": (C.c_int64, [C.c_int64, C.c_int]),
    "dg_plan_views": (C.c_int, [C.POINTER(DgCamera), C.c_int, C.POINTER(C.c_int64), C.c_int, C.c_int, C.c_int,
                                C.POINTER(DgPlan)]),
    "dg_project": (C.c_int, [C.POINTER(DgGaussians), _vp, C.POINTER(DgPlan), _vp, _vp, _vp]),
    "dg_bin_sort_workspace_size": (C.c_size_t, [C.POINTER(DgPlan), C.c_int64]),
    "dg_bin_sort_workspace_min_size": (C.c_size_t, [C.POINTER(DgPlan), C.c_int64]),
    "dg_bin_sort": (C.c_int, [_vp, _vp, _vp, C.POINTER(DgPlan), C.c_int64, _vp, _vp, _vp, _vp, _vp, C.c_size_t,
                              _vp, _vp]),
    "dg_bin_sort_noalloc": (C.c_int, [_vp, _vp, _vp, C.POINTER(DgPlan), C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dg_rasterize_fwd": (C.c_int, [_vp, _vp, _vp, _vp, C.POINTER(DgPlan), C.POINTER(C.c_float), _vp, _vp, _vp, _vp]),
    "dg_loss_l1": (C.c_int, [_vp, _vp, _vp, C.POINTER(DgPlan), C.c_float, _vp, _vp, _vp]),
    "dg_loss_workspace_size": (C.c_size_t, [C.POINTER(DgPlan)]),
    "dg_loss_dssim": (C.c_int, [_vp, _vp, _vp, C.POINTER(DgPlan), C.c_float, C.c_float, _vp, _vp, _vp, C.c_size_t,
                                _vp]),
    "dg_rasterize_bwd": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(DgPlan), C.POINTER(C.c_float), _vp, _vp, _vp,
                                   C.POINTER(DgGaussians), _vp, C.POINTER(DgGaussians), _vp]),
    "dg_adam_admm_step": (C.c_int, [C.POINTER(DgGaussians), C.POINTER(DgGaussians), C.POINTER(DgGaussians),
                                    C.POINTER(DgGaussians), C.POINTER(DgGaussians), _vp, C.POINTER(C.c_float),
                                    C.POINTER(C.c_float), C.c_float, C.c_float, C.c_float, C.c_int, _vp, _vp]),
    "dg_admm_consensus": (C.c_int, [C.POINTER(DgGaussians), C.POINTER(DgGaussians), C.POINTER(DgGaussians),
                                    C.POINTER(DgGaussians), _vp, _vp, C.POINTER(C.c_float), C.c_float, _vp, _vp]),
    "dg_admm_anchor": (C.c_int, [C.POINTER(DgGaussians), C.POINTER(DgGaussians), _vp, _vp, C.POINTER(DgGaussians),
                                 _vp]),
    "dg_admm_scale_duals": (C.c_int, [C.POINTER(DgGaussians), _vp, C.POINTER(C.c_float), _vp]),
    "dg_rasterize_count": (C.c_int, [_vp, _vp, _vp, _vp, C.POINTER(DgPlan), C.POINTER(C.c_float), _vp, _vp, _vp,
                                     _vp, _vp]),
    "dg_rasterize_bwd_records": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(DgPlan), C.POINTER(C.c_float), _vp, _vp,
                                            _vp, _vp, _vp]),
    "dg_xstep_from_records": (C.c_int, [_vp, _vp, C.POINTER(DgPlan), _vp, C.POINTER(DgGaussians),
                                         C.POINTER(DgGaussians), C.POINTER(DgGaussians), C.POINTER(DgGaussians), _vp,
                                         C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.c_float, C.c_float,
                                         C.c_int, _vp, _vp]),
    "dg_xstep_part": (C.c_int, [C.c_int, C.c_int, _vp, _vp, C.POINTER(DgPlan), _vp, C.POINTER(DgGaussians),
                                 C.POINTER(DgGaussians), C.POINTER(DgGaussians), C.POINTER(DgGaussians), _vp,
                                 C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.c_float, C.c_float,
                                 C.c_int, _vp, C.POINTER(DgGaussians), _vp, _vp]),
    "dg_xstep_stream_workspace_size": (C.c_size_t, [C.POINTER(DgGaussians)]),
    "dg_xstep_stream": (C.c_int, [C.c_int, _vp, _vp, C.POINTER(DgPlan), C.POINTER(DgGaussians),
                                   C.POINTER(DgGaussians), C.POINTER(DgGaussians), C.POINTER(DgGaussians), _vp,
                                   C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.c_float, C.c_float,
                                   C.c_int, _vp, C.POINTER(DgGaussians), _vp, _vp, C.c_size_t, _vp]),
    "dg_xstep_groups": (C.c_int, [_vp, _vp, C.POINTER(DgPlan), C.POINTER(DgGaussians), _vp, C.c_size_t, _vp]),
    "dg_xstep_listed": (C.c_int, [C.c_int, C.c_int, _vp, _vp, C.POINTER(DgPlan), _vp, C.POINTER(DgGaussians),
                                   C.POINTER(DgGaussians), C.POINTER(DgGaussians), C.POINTER(DgGaussians), _vp,
                                   C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float, C.c_float, C.c_float,
                                   C.c_int, _vp, C.POINTER(DgGaussians), _vp, _vp, C.c_size_t, _vp]),
    "dg_step_advance": (C.c_int, [_vp, _vp]),
    "dg_densify_stats": (C.c_int, [_vp, _vp, C.POINTER(DgPlan), _vp, _vp, _vp]),
    "dg_densify_workspace_size": (C.c_size_t, [C.c_int64]),
    "dg_densify_decide": (C.c_int, [C.POINTER(DgGaussians), _vp, _vp, _vp, C.c_float, C.c_float, C.c_float,
                                    C.c_float, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "dg_densify_emit": (C.c_int, [C.POINTER(DgGaussians), _vp, _vp, _vp, C.POINTER(DgGaussians), _vp, _vp, _vp]),
    "dg_gather_rows": (C.c_int, [C.POINTER(DgGaussians), _vp, C.POINTER(DgGaussians), _vp]),
    "dg_layout_copies": (C.c_int64, [_vp, C.c_int64]),
    "dg_image_u8_to_f32": (C.c_int, [_vp, _vp, C.c_int64, _vp]),
    "dg_image_f32_to_u8": (C.c_int, [_vp, _vp, C.c_int64, _vp]),
    "dg_reset_opacity": (C.c_int, [C.POINTER(DgGaussians), C.c_float, C.POINTER(DgGaussians),
                                   C.POINTER(DgGaussians), _vp]),
    "dg_layout": (C.c_int, [_vp, _vp, C.c_int64, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "dg_layout_membership": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int, _vp, C.c_int64, _vp]),
    "dg_layout_carry": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int64, _vp]),
    "dg_scene_split": (C.c_int, [_vp, C.c_int64, C.c_int, _vp, _vp]),
    "dg_scene_assign": (C.c_int, [_vp, C.c_int64, _vp, C.c_int, C.c_double, _vp, C.c_int, _vp]),
    "dg_render_plan": (C.c_int, [C.POINTER(DgCamera), C.c_int, C.c_int64, C.c_int, C.c_int, C.POINTER(DgPlan)]),
    "dg_render_workspace_size": (C.c_size_t, [C.POINTER(DgPlan), C.c_int64]),
    "dg_render": (C.c_int, [C.POINTER(DgGaussians), _vp, C.POINTER(DgPlan), C.POINTER(C.c_float), C.c_int64, _vp,
                            _vp, C.c_size_t, _vp, _vp, _vp]),
}

_lib = None


def lib():
    """Load libdogs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise DogsError(f"libdogs.so not built ({LIB_PATH}); run paper_2405_13943_b300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def check(rc: int, what: str) -> None:
    if rc != DG_OK:
        raise DogsError(f"{what}: {_ERR.get(rc, rc)}")


def ptr(t) -> Optional[int]:
    """Device (or host) address of a tensor, None for None."""
    if t is None:
        return None
    return t.data_ptr()


def stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def rho_arg(rho):
    """rho[5] for an ABI call: a float array in host memory, or the address
    of a float32 device tensor (read by the kernels when they run)."""
    if hasattr(rho, "data_ptr"):
        import torch
        if rho.dtype != torch.float32 or rho.numel() != 5 or not rho.is_cuda:
            raise ValueError("a device rho is a CUDA float32 tensor of 5 elements")
        return C.cast(C.c_void_p(rho.data_ptr()), C.POINTER(C.c_float))
    return floats(rho)


def floats(vals) -> C.Array:
    a = (C.c_float * len(vals))()
    for i, v in enumerate(vals):
        a[i] = float(v)
    return a
