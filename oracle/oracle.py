"""Python face of the FP64 oracle (TEST INFRASTRUCTURE ONLY).

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this module.  It loads `liboracle.so` (plain C, FP64,
built from `dogs_oracle.c` by `build()` below) and composes its per-view
functions into multi-view renders, the analytic backward, the x-step (Adam on
the loss plus the ADMM penalty, Eq. 8a / 12a) and the consensus step (Eq. 8b-c,
12b-c), in the order the paper states them.  D-SSIM (the lambda term of Eq. 3)
is written here in numpy, from its definition.

Parity status: pinned by tests/test_oracle_*.py (closed forms, brute force,
central finite differences, hand-worked ADMM examples, textbook ADMM
convergence on quadratics; densification by hand-worked decisions and the
split children's distribution against scipy's rotation).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import List, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dogs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-fopenmp", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class OcCam(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("R", C.c_double * 9), ("t", C.c_double * 3), ("campos", C.c_double * 3),
                ("near_z", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp, ip, fp, u32p, u64p, u8p, i64p = (C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                              C.POINTER(C.c_float), C.POINTER(C.c_uint32),
                                              C.POINTER(C.c_uint64), C.POINTER(C.c_uint8),
                                              C.POINTER(C.c_int64))
        _lib.oc_sh_basis.restype = C.c_double
        _lib.oc_sh_basis.argtypes = [C.c_int, C.c_int, dp, dp]
        _lib.oc_project.restype = C.c_int
        _lib.oc_project.argtypes = [C.c_int, C.c_int, dp, C.POINTER(OcCam), C.c_int, C.c_int,
                                    dp, ip, fp, dp]
        _lib.oc_bin_sort.restype = C.c_int64
        _lib.oc_bin_sort.argtypes = [C.c_int64, ip, ip, fp, ip, ip, ip, C.c_int64, C.c_int64,
                                     u64p, u32p, u32p, dp, C.c_int, C.c_int, C.c_int]
        _lib.oc_rasterize_fwd.restype = None
        _lib.oc_rasterize_fwd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, u32p, u32p,
                                          dp, dp, dp, dp, u32p, dp, dp]
        _lib.oc_box_qmin.restype = C.c_double
        _lib.oc_box_qmin.argtypes = [C.c_double] * 7
        _lib.oc_rasterize_counts.restype = None
        _lib.oc_rasterize_counts.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, u32p, u32p,
                                             dp, u32p, u32p]
        _lib.oc_rasterize_bwd.restype = None
        _lib.oc_rasterize_bwd.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, u32p, u32p,
                                          dp, dp, dp, dp]
        _lib.oc_project_bwd.restype = None
        _lib.oc_project_bwd.argtypes = [C.c_int, C.c_int, dp, C.POINTER(OcCam), C.c_int, C.c_int,
                                        dp, dp]
        _lib.oc_adam_admm_step.restype = None
        _lib.oc_adam_admm_step.argtypes = [C.c_int64, C.c_int, dp, dp, dp, dp, dp, dp, ip, u8p, dp, dp,
                                           C.c_double, C.c_double, C.c_double, C.c_int]
        _lib.oc_set_threads.restype = None
        _lib.oc_set_threads.argtypes = [C.c_int]
        _lib.oc_get_threads.restype = C.c_int
        _lib.oc_have_openmp.restype = C.c_int
        _lib.oc_consensus.restype = None
        _lib.oc_consensus.argtypes = [C.c_int64, C.c_int, i64p, ip, dp, dp, dp, C.c_double, dp, dp]
    return _lib


def set_threads(n: int) -> int:
    """Host threads of the per-Gaussian and per-pixel loops (1 by default,
    which keeps every result bit-for-bit reproducible).  Returns the count in
    effect: 1 when the library was built without OpenMP."""
    lib().oc_set_threads(int(n) if lib().oc_have_openmp() else 1)
    return int(lib().oc_get_threads())


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


REC_N = 16
(REC_MX, REC_MY, REC_A, REC_B, REC_C, REC_OP, REC_R, REC_G, REC_BL, REC_DEPTH,
 REC_RAWR, REC_RAWG, REC_RAWB, REC_RADIUS, REC_TILES, REC_VIS) = range(16)


# --------------------------------------------------------------------------
# layout conversion (oracle's own layout: P = 11 + 3K doubles per Gaussian)
# --------------------------------------------------------------------------
def n_params(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


def params_from(g) -> np.ndarray:
    n = g.n
    K = g.sh.shape[1]
    P = 11 + 3 * K
    x = np.empty((n, P), np.float64)
    x[:, 0:3] = g.means
    x[:, 3:7] = g.quats
    x[:, 7:10] = g.log_scales
    x[:, 10:10 + 3 * K] = g.sh.reshape(n, 3 * K)
    x[:, 10 + 3 * K] = g.opacity_logits
    return x


def split_params(x: np.ndarray, sh_degree: int) -> dict:
    """Return parameter groups (the paper's p, q, s, f, o) as views."""
    K = (sh_degree + 1) ** 2
    return {"mean": x[:, 0:3], "quat": x[:, 3:7], "scale": x[:, 7:10],
            "sh": x[:, 10:10 + 3 * K].reshape(-1, K, 3), "opacity": x[:, 10 + 3 * K]}


def cam_struct(c) -> OcCam:
    s = OcCam()
    s.width, s.height = int(c.width), int(c.height)
    s.fx, s.fy, s.cx, s.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
    for i in range(9):
        s.R[i] = float(np.asarray(c.R, np.float32).reshape(9)[i])
    for i in range(3):
        s.t[i] = float(np.asarray(c.t, np.float32)[i])
        s.campos[i] = float(np.asarray(c.campos, np.float32)[i])
    s.near_z = float(np.float32(c.near))
    return s


def sh_basis(l: int, m: int, d) -> tuple:
    d = np.ascontiguousarray(d, np.float64)
    g = np.zeros(3, np.float64)
    v = lib().oc_sh_basis(l, m, _p(d, C.c_double), _p(g, C.c_double))
    return v, g


# --------------------------------------------------------------------------
# per-view pieces
# --------------------------------------------------------------------------
def project(x: np.ndarray, sh_degree: int, cam, tile_w: int, tile_h: int) -> dict:
    x = np.ascontiguousarray(x, np.float64)
    n = x.shape[0]
    rec = np.zeros((n, REC_N), np.float64)
    rect = np.zeros((n, 4), np.int32)
    dk = np.zeros(n, np.float32)
    mg = np.zeros(n, np.float64)
    cs = cam_struct(cam)
    lib().oc_project(n, sh_degree, _p(x, C.c_double), C.byref(cs), tile_w, tile_h,
                     _p(rec, C.c_double), _p(rect, C.c_int32), _p(dk, C.c_float), _p(mg, C.c_double))
    return {"rec": rec, "rect": rect, "depth_key": dk, "margin": mg,
            "visible": rec[:, REC_VIS].astype(np.int32),
            "tiles": rec[:, REC_TILES].astype(np.int64)}


def tiles_of(cam, tile_w: int, tile_h: int) -> tuple:
    return (cam.width + tile_w - 1) // tile_w, (cam.height + tile_h - 1) // tile_h


class ViewPlan:
    """Numbering of records, tiles and pixels over a batch of views.

    View v renders the Gaussians [rows[v][0], rows[v][1]) of the parameter
    array; its records are numbered from rec_off[v] (record = rec_off[v] +
    local index) and its tiles from tile_off[v]."""

    def __init__(self, cams: Sequence, rows: Sequence[tuple], tile_w: int, tile_h: int):
        self.cams, self.rows, self.tw, self.th = list(cams), list(rows), tile_w, tile_h
        self.rec_off, self.tile_off, self.tiles_x = [], [], []
        r = t = 0
        for c, (b, e) in zip(self.cams, self.rows):
            tx, ty = tiles_of(c, tile_w, tile_h)
            self.rec_off.append(r)
            self.tile_off.append(t)
            self.tiles_x.append(tx)
            r += e - b
            t += tx * ty
        self.n_rec, self.n_tiles = r, t


def project_views(x: np.ndarray, sh_degree: int, plan: ViewPlan) -> dict:
    recs, rects, dks, mgs, views = [], [], [], [], []
    for v, (c, (b, e)) in enumerate(zip(plan.cams, plan.rows)):
        p = project(x[b:e], sh_degree, c, plan.tw, plan.th)
        recs.append(p["rec"]); rects.append(p["rect"]); dks.append(p["depth_key"])
        mgs.append(p["margin"]); views.append(np.full(e - b, v, np.int32))
    cat = lambda a, dt, sh: np.concatenate(a) if a else np.zeros(sh, dt)
    return {"rec": cat(recs, np.float64, (0, REC_N)), "rect": cat(rects, np.int32, (0, 4)),
            "depth_key": cat(dks, np.float32, (0,)), "margin": cat(mgs, np.float64, (0,)),
            "view": cat(views, np.int32, (0,))}


def bin_sort(proj: dict, plan: ViewPlan, cull: bool = True) -> dict:
    """Instances of the records' tile rectangles, sorted by (tile, depth,
    record); with cull, tiles no pixel centre of which can reach alpha >=
    1/255 are left out (the images do not depend on it)."""
    n = proj["rec"].shape[0]
    rec = np.ascontiguousarray(proj["rec"], np.float64) if n else np.zeros((1, REC_N))
    vis = np.ascontiguousarray(proj["rec"][:, REC_VIS].astype(np.int32))
    view = np.ascontiguousarray(proj["view"], np.int32)
    rect = np.ascontiguousarray(proj["rect"], np.int32)
    dk = np.ascontiguousarray(proj["depth_key"], np.float32)
    toff = np.asarray(plan.tile_off, np.int32)
    tx = np.asarray(plan.tiles_x, np.int32)
    ranges = np.zeros((plan.n_tiles, 2), np.uint32)
    empty64 = np.zeros(1, np.uint64)
    empty32 = np.zeros(1, np.uint32)
    M = lib().oc_bin_sort(n, _p(view, C.c_int32), _p(rect, C.c_int32), _p(dk, C.c_float),
                          _p(vis, C.c_int32), _p(toff, C.c_int32), _p(tx, C.c_int32),
                          plan.n_tiles, 0, _p(empty64, C.c_uint64), _p(empty32, C.c_uint32),
                          _p(ranges, C.c_uint32), _p(rec, C.c_double), plan.tw, plan.th, int(cull))
    keys = np.zeros(max(M, 1), np.uint64)
    vals = np.zeros(max(M, 1), np.uint32)
    lib().oc_bin_sort(n, _p(view, C.c_int32), _p(rect, C.c_int32), _p(dk, C.c_float),
                      _p(vis, C.c_int32), _p(toff, C.c_int32), _p(tx, C.c_int32),
                      plan.n_tiles, M, _p(keys, C.c_uint64), _p(vals, C.c_uint32),
                      _p(ranges, C.c_uint32), _p(rec, C.c_double), plan.tw, plan.th, int(cull))
    return {"keys": keys[:M], "vals": vals[:M], "ranges": ranges, "M": int(M)}


def rasterize_fwd(proj: dict, bins: dict, plan: ViewPlan, bg=(0.0, 0.0, 0.0)) -> List[dict]:
    out = []
    rec = np.ascontiguousarray(proj["rec"])
    bgv = np.asarray(bg, np.float64)
    vals = np.ascontiguousarray(bins["vals"]) if bins["M"] else np.zeros(1, np.uint32)
    for v, c in enumerate(plan.cams):
        W, H = c.width, c.height
        img = np.zeros((3, H, W)); Tf = np.zeros((H, W)); last = np.zeros((H, W), np.uint32)
        mg = np.zeros((H, W))
        mg2 = np.zeros((H, W))
        lib().oc_rasterize_fwd(W, H, plan.tw, plan.th, plan.tile_off[v], _p(vals, C.c_uint32),
                               _p(bins["ranges"], C.c_uint32), _p(rec, C.c_double),
                               _p(bgv, C.c_double), _p(img, C.c_double), _p(Tf, C.c_double),
                               _p(last, C.c_uint32), _p(mg, C.c_double), _p(mg2, C.c_double))
        # margin: value decisions (1/255 skip, T stop); margin_grad: the 0.99 clamp
        out.append({"image": img, "T_final": Tf, "last": last, "margin": mg, "margin_grad": mg2})
    return out


def rasterize_counts(proj: dict, bins: dict, plan: ViewPlan) -> List[dict]:
    """Per view and pixel: list positions examined by the compositing (up to
    the stop) and Eq. 2 terms composited."""
    out = []
    rec = np.ascontiguousarray(proj["rec"])
    vals = np.ascontiguousarray(bins["vals"]) if bins["M"] else np.zeros(1, np.uint32)
    for v, c in enumerate(plan.cams):
        W, H = c.width, c.height
        seen = np.zeros((H, W), np.uint32); used = np.zeros((H, W), np.uint32)
        lib().oc_rasterize_counts(W, H, plan.tw, plan.th, plan.tile_off[v], _p(vals, C.c_uint32),
                                  _p(bins["ranges"], C.c_uint32), _p(rec, C.c_double),
                                  _p(seen, C.c_uint32), _p(used, C.c_uint32))
        out.append({"seen": seen, "used": used})
    return out


def rasterize_bwd(proj: dict, bins: dict, plan: ViewPlan, dL_dimages: Sequence[np.ndarray],
                  bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    rec = np.ascontiguousarray(proj["rec"])
    drec = np.zeros((rec.shape[0], 9))
    bgv = np.asarray(bg, np.float64)
    vals = np.ascontiguousarray(bins["vals"]) if bins["M"] else np.zeros(1, np.uint32)
    for v, c in enumerate(plan.cams):
        g = np.ascontiguousarray(dL_dimages[v], np.float64)
        lib().oc_rasterize_bwd(c.width, c.height, plan.tw, plan.th, plan.tile_off[v],
                               _p(vals, C.c_uint32), _p(bins["ranges"], C.c_uint32),
                               _p(rec, C.c_double), _p(bgv, C.c_double), _p(g, C.c_double),
                               _p(drec, C.c_double))
    return drec


def project_bwd(x: np.ndarray, sh_degree: int, plan: ViewPlan, drec: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    dx = np.zeros_like(x)
    for v, (c, (b, e)) in enumerate(zip(plan.cams, plan.rows)):
        cs = cam_struct(c)
        r0 = plan.rec_off[v]
        dr = np.ascontiguousarray(drec[r0:r0 + (e - b)])
        part = np.zeros((e - b, x.shape[1]))
        lib().oc_project_bwd(e - b, sh_degree, _p(np.ascontiguousarray(x[b:e]), C.c_double),
                             C.byref(cs), plan.tw, plan.th, _p(dr, C.c_double), _p(part, C.c_double))
        dx[b:e] += part
    return dx


# --------------------------------------------------------------------------
# whole passes
# --------------------------------------------------------------------------
def box_qmin(a, b, c, X0, X1, Y0, Y1) -> float:
    """Minimum of a x^2 + 2 b x y + c y^2 over [X0, X1] x [Y0, Y1]."""
    return lib().oc_box_qmin(a, b, c, X0, X1, Y0, Y1)


def cull_tau(o: float) -> float:
    """Widened bound on q(d) for alpha >= 1/255 (see bin_sort)."""
    return 2.0 * np.log(255.0 * o) * (1.0 + 1.0 / 1024.0) + 1.0 / 64.0


def render(x: np.ndarray, sh_degree: int, plan: ViewPlan, bg=(0.0, 0.0, 0.0), cull: bool = True) -> dict:
    proj = project_views(x, sh_degree, plan)
    bins = bin_sort(proj, plan, cull)
    views = rasterize_fwd(proj, bins, plan, bg)
    return {"proj": proj, "bins": bins, "views": views}


def backward(x: np.ndarray, sh_degree: int, plan: ViewPlan, fwd: dict,
             dL_dimages: Sequence[np.ndarray], bg=(0.0, 0.0, 0.0)) -> dict:
    drec = rasterize_bwd(fwd["proj"], fwd["bins"], plan, dL_dimages, bg)
    return {"drec": drec, "dparams": project_bwd(x, sh_degree, plan, drec)}


# --------------------------------------------------------------------------
# losses (Eq. 3): L1 and D-SSIM, means over all channels and pixels
# --------------------------------------------------------------------------
def l1(img: np.ndarray, tgt: np.ndarray) -> tuple:
    d = np.asarray(img, np.float64) - np.asarray(tgt, np.float64)
    return float(np.abs(d).mean()), np.sign(d) / d.size


def gaussian_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    ax = np.arange(size) - (size - 1) / 2.0
    w = np.exp(-(ax ** 2) / (2.0 * sigma ** 2))
    return w / w.sum()


def _filt(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """'same'-size 2D correlation of each channel with the separable window
    w x w, zero padding (scipy's routine as the library primitive)."""
    from scipy.ndimage import correlate1d
    a = correlate1d(a, w, axis=-1, mode="constant", cval=0.0)
    return correlate1d(a, w, axis=-2, mode="constant", cval=0.0)


def ssim(img: np.ndarray, tgt: np.ndarray, C1: float = 0.01 ** 2, C2: float = 0.03 ** 2) -> tuple:
    """Mean SSIM (Wang et al. 2004) with an 11x11 Gaussian window, sigma 1.5,
    and its gradient w.r.t. img.  S = (2 m1 m2 + C1)(2 s12 + C2) /
    ((m1^2 + m2^2 + C1)(s1 + s2 + C2)), moments taken with the window."""
    x = np.asarray(img, np.float64)
    y = np.asarray(tgt, np.float64)
    w = gaussian_window()
    m1, m2 = _filt(x, w), _filt(y, w)
    e11, e22, e12 = _filt(x * x, w), _filt(y * y, w), _filt(x * y, w)
    s1, s2, s12 = e11 - m1 * m1, e22 - m2 * m2, e12 - m1 * m2
    A1, A2 = 2 * m1 * m2 + C1, 2 * s12 + C2
    B1, B2 = m1 * m1 + m2 * m2 + C1, s1 + s2 + C2
    S = (A1 * A2) / (B1 * B2)
    N = S.size
    # partials of S w.r.t. m1, e11, e12 (m2, e22 do not depend on x)
    dS_dA1 = A2 / (B1 * B2)
    dS_dA2 = A1 / (B1 * B2)
    dS_dB1 = -S / B1
    dS_dB2 = -S / B2
    dS_dm1 = dS_dA1 * 2 * m2 + dS_dA2 * 2 * (-m2) + dS_dB1 * 2 * m1 + dS_dB2 * (-2 * m1)
    dS_de11 = dS_dB2
    dS_de12 = dS_dA2 * 2
    # adjoint of the (symmetric-window) correlation is the same correlation
    g = _filt(dS_dm1 / N, w) + 2 * x * _filt(dS_de11 / N, w) + y * _filt(dS_de12 / N, w)
    return float(S.mean()), g


def dssim_loss(img: np.ndarray, tgt: np.ndarray, lam: float = 0.2) -> tuple:
    """(1 - lam) L1 + lam (1 - SSIM): Eq. 3 with lambda = 0.2."""
    a, ga = l1(img, tgt)
    s, gs = ssim(img, tgt)
    return (1 - lam) * a + lam * (1 - s), (1 - lam) * ga - lam * gs


# --------------------------------------------------------------------------
# ADMM (Eq. 8a-c, 12a-c; Sec. 3.3)
# --------------------------------------------------------------------------
def adam_admm_step(x, grad, m, v, z, u, copy_gid, shared, rho, lr, sh_degree,
                   b1=0.9, b2=0.999, eps=1e-15, step=1) -> None:
    """In place on x, m, v (all n_copies x P, float64, C-contiguous)."""
    for a in (x, grad, m, v, z, u):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gid = np.ascontiguousarray(copy_gid, np.int32)
    sh = np.ascontiguousarray(shared, np.uint8)
    rho = np.ascontiguousarray(rho, np.float64)
    lr = np.ascontiguousarray(lr, np.float64)
    lib().oc_adam_admm_step(x.shape[0], sh_degree, _p(x, C.c_double), _p(grad, C.c_double),
                            _p(m, C.c_double), _p(v, C.c_double), _p(z, C.c_double),
                            _p(u, C.c_double), _p(gid, C.c_int32), _p(sh, C.c_uint8),
                            _p(rho, C.c_double), _p(lr, C.c_double), b1, b2, eps, step)


def consensus(x, u, z, g_off, g_copies, sh_degree, alpha=1.0, rho=(1, 1, 1, 1, 1)) -> np.ndarray:
    """In place on u and z; returns the 10 residual sums (Eq. 9)."""
    for a in (x, u, z):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    go = np.ascontiguousarray(g_off, np.int64)
    gc = np.ascontiguousarray(g_copies, np.int32)
    res = np.zeros(10)
    rr = np.ascontiguousarray(rho, np.float64)
    lib().oc_consensus(z.shape[0], sh_degree, _p(go, C.c_int64), _p(gc, C.c_int32),
                       _p(x, C.c_double), _p(u, C.c_double), _p(z, C.c_double), float(alpha),
                       _p(rr, C.c_double), _p(res, C.c_double))
    return res


# --------------------------------------------------------------------------
# adaptive penalty (Sec. 3.3, Eq. 10) and the rescale of the scaled duals
# --------------------------------------------------------------------------
def adaptive_rho(rho, residuals, t, mu=10.0, tau_inc=2.0, tau_dec=2.0, freeze_after=2000):
    """Eq. 10 per property group: rho * tau_inc if ||r|| > mu ||s||,
    rho / tau_dec if ||s|| > mu ||r||, rho otherwise; no change from
    iteration `freeze_after` on.  residuals = (||r_g||^2 for g in p,q,s,f,o)
    followed by (||s_g||^2 ...)."""
    out = []
    for g in range(5):
        r = float(np.sqrt(residuals[g]))
        s = float(np.sqrt(residuals[5 + g]))
        if t >= freeze_after:
            out.append(float(rho[g]))
        elif r > mu * s:
            out.append(float(rho[g]) * tau_inc)
        elif s > mu * r:
            out.append(float(rho[g]) / tau_dec)
        else:
            out.append(float(rho[g]))
    return out


def scale_duals(u, shared, factor, sh_degree):
    """u <- u * factor[group] on shared copies (u = y / rho keeps y fixed
    when rho changes)."""
    K = (sh_degree + 1) ** 2
    groups = [0] * 3 + [1] * 4 + [2] * 3 + [3] * (3 * K) + [4]
    f = np.array([factor[g] for g in groups])
    u[np.asarray(shared, bool)] *= f


# --------------------------------------------------------------------------
# recursive bipartite scene splitting (Sec. 3.2 "Scene Splitting", Alg. 1)
# and the overlap by a box scale factor s (Sec. 3.2)
# --------------------------------------------------------------------------
def _aabb(xy, idx):
    """Tight ground box (xmin, xmax, ymin, ymax) of the points idx; an empty
    set gives (+inf, -inf, +inf, -inf)."""
    if len(idx) == 0:
        return (np.inf, -np.inf, np.inf, -np.inf)
    p = xy[idx]
    return (p[:, 0].min(), p[:, 0].max(), p[:, 1].min(), p[:, 1].max())


def scene_split(xy, K):
    """Alg. 1 on ground positions xy (n, 2) float64.  Reading: every cell
    carries a budget of leaves (K at the root); a cell with budget k >= 2 is
    cut on the longer side of its tight box (ties: x), the lower child
    getting the first floor(n_c floor(k/2) / k) points in (coordinate, index)
    order and budget floor(k/2); budget-1 cells are popped and pushed back
    unchanged.  Returns (cell (n,) int32, boxes (K, 4))."""
    xy = np.asarray(xy, np.float64)
    n = xy.shape[0]
    # line 1-2: one cell with a tight box over all points
    C = [(np.arange(n), K)]
    # line 3-13: split every current cell until there are K of them
    while len(C) < K:
        C_cur = list(C)
        while len(C_cur) > 0:
            cell = C_cur.pop(0)                 # pop a cell of this level
            C.pop(_index_of(C, cell))           # and remove it from the cells
            idx, k = cell
            if k < 2:
                C.append(cell)
                continue
            box = _aabb(xy, idx)
            axis = 0 if (len(idx) == 0 or box[1] - box[0] >= box[3] - box[2]) else 1
            order = idx[np.lexsort((idx, xy[idx, axis]))]   # group by the cut
            k1 = k // 2
            m = (len(idx) * k1) // k
            C.append((order[:m], k1))
            C.append((order[m:], k - k1))
    # line 14-17: group the points of each cell into its block
    cell_of = np.empty(n, np.int32)
    boxes = np.empty((K, 4))
    for k, (idx, _) in enumerate(C):
        cell_of[idx] = k
        boxes[k] = _aabb(xy, idx)
    return cell_of, boxes


def _index_of(C, cell):
    for i, c in enumerate(C):
        if c is cell:
            return i
    raise ValueError("cell not in the list")


def scene_assign(xy, boxes, s, own=None, nearest=False):
    """Membership (n, K) bool in the boxes expanded about their centres by
    s: centre (lo + hi) / 2, half side s (hi - lo) / 2, closed intervals.
    own adds each point's own cell; nearest gives a point outside every
    expanded box the block of the nearest one (lowest index on ties)."""
    xy = np.asarray(xy, np.float64)
    boxes = np.asarray(boxes, np.float64)
    n, K = xy.shape[0], boxes.shape[0]
    member = np.zeros((n, K), bool)
    ex = np.empty((K, 4))
    empty = np.zeros(K, bool)
    for k in range(K):
        b = boxes[k]
        empty[k] = not (b[0] <= b[1] and b[2] <= b[3])
        if empty[k]:
            continue
        for a in range(2):
            lo, hi = b[2 * a], b[2 * a + 1]
            c = 0.5 * (lo + hi)
            h = 0.5 * s * (hi - lo)
            ex[k, 2 * a], ex[k, 2 * a + 1] = c - h, c + h
    for k in range(K):
        if empty[k]:
            continue
        member[:, k] = ((xy[:, 0] >= ex[k, 0]) & (xy[:, 0] <= ex[k, 1]) &
                        (xy[:, 1] >= ex[k, 2]) & (xy[:, 1] <= ex[k, 3]))
    if own is not None:
        member[np.arange(n), np.asarray(own)] = True
    if nearest:
        for i in np.nonzero(~member.any(1))[0]:
            best, bd = -1, 0.0
            for k in range(K):
                if empty[k]:
                    continue
                x, y = xy[i]
                dx = ex[k, 0] - x if x < ex[k, 0] else (x - ex[k, 1] if x > ex[k, 1] else 0.0)
                dy = ex[k, 2] - y if y < ex[k, 2] else (y - ex[k, 3] if y > ex[k, 3] else 0.0)
                d = dx * dx + dy * dy
                if best < 0 or d < bd:
                    best, bd = k, d
            if best >= 0:
                member[i, best] = True
    return member


# ---------------------------------------------------------------------------
# Densification under consensus (Sec. 4, Implementation Details: densified
# at the intervals of 3DGS; Sec. 5: small Gaussians pruned).  The paper
# follows the 3DGS adaptive density control; its rules are restated here:
#   statistic  per Gaussian, over the iterations since the last densification,
#              the mean over its visible records of the norm of the screen
#              gradient of its projected mean in normalised device units
#              (pixels scaled by W/2 and H/2);
#   prune      opacity sigmoid(o) < min_opacity (the Gaussian and anything
#              it would spawn are dropped);
#   clone      mean statistic >= grad_threshold and largest scale
#              <= percent_dense * extent: the Gaussian and an exact copy;
#   split      mean statistic >= grad_threshold and largest scale larger:
#              two children replace it, each with mean mu + R(q) (S xi)
#              (xi ~ N(0, I), drawn by the caller), scales S / 1.6, the
#              other parameters copied.
# Under consensus the decision is taken on the global model z right after
# a consensus, from the statistics of all copies of each Gaussian summed,
# so every block holding a Gaussian gets the same children; the children
# inherit the parent's sharing set.  Every quantity is formed in FP64 from
# its definition: the mean statistic sum / count, sigmoid(o) and the largest
# scale exp(s).  Each decision reports its relative margin, the distance of
# the compared quantity from its threshold over the threshold, so a test can
# leave out the Gaussians whose decision another precision could flip.
# ---------------------------------------------------------------------------
DENSIFY_KEEP, DENSIFY_PRUNE, DENSIFY_CLONE, DENSIFY_SPLIT = 0, 1, 2, 3


def quat_rotation(q) -> np.ndarray:
    """Rotation matrix of the unit quaternion q / |q| (w, x, y, z)."""
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify_stats(kept: np.ndarray, dmean2d: np.ndarray, view_wh: np.ndarray, copy_of_record: np.ndarray,
                  n_copies: int):
    """One iteration's contribution to the statistic: for every kept record
    r (copy copy_of_record[r] in a view of size view_wh[r]), the norm of its
    mean gradient in normalised device units.  Returns (sum, count) per copy."""
    s = np.zeros(n_copies, np.float64)
    c = np.zeros(n_copies, np.float64)
    g = np.asarray(dmean2d, np.float64) * (0.5 * np.asarray(view_wh, np.float64))
    nrm = np.sqrt((g * g).sum(1))
    for r in np.nonzero(np.asarray(kept, bool))[0]:
        s[copy_of_record[r]] += nrm[r]
        c[copy_of_record[r]] += 1.0
    return s, c


def densify_decide(z: np.ndarray, sh_degree: int, stat_sum, stat_cnt, g_off, g_copies,
                   grad_threshold=2e-4, percent_dense=0.01, extent=1.0, min_opacity=0.005,
                   return_margin: bool = False):
    """The decision per global Gaussian (DENSIFY_* codes), in FP64: prune when
    sigmoid(o) < min_opacity; otherwise, when its copies were seen at all and
    the mean of their summed statistic (sum / count over every copy) reaches
    grad_threshold, split if its largest scale exp(s) exceeds
    percent_dense * extent and clone if not; keep in every other case.

    With return_margin, also the relative margin of the decision: the least,
    over the comparisons on the path that led to the code, of
    |quantity - threshold| / threshold (the opacity comparison always; the
    gradient comparison unless pruned; the scale comparison when the gradient
    rule holds)."""
    zz = split_params(z, sh_degree)
    n = z.shape[0]
    codes = np.zeros(n, np.int32)
    margin = np.full(n, np.inf)
    big_scale = float(percent_dense) * float(extent)
    for i in range(n):
        cps = g_copies[g_off[i]:g_off[i + 1]]
        ssum = float(np.sum(np.asarray(stat_sum, np.float64)[cps]))
        scnt = float(np.sum(np.asarray(stat_cnt, np.float64)[cps]))
        opacity = 1.0 / (1.0 + np.exp(-float(zz["opacity"][i])))
        m = abs(opacity - min_opacity) / min_opacity
        if opacity < min_opacity:
            codes[i] = DENSIFY_PRUNE
        else:
            grad_ok = False
            if scnt > 0:
                mean = ssum / scnt
                m = min(m, abs(mean - grad_threshold) / grad_threshold)
                grad_ok = mean >= grad_threshold
            if grad_ok:
                largest = float(np.exp(np.max(np.asarray(zz["scale"][i], np.float64))))
                m = min(m, abs(largest - big_scale) / big_scale)
                codes[i] = DENSIFY_SPLIT if largest > big_scale else DENSIFY_CLONE
            else:
                codes[i] = DENSIFY_KEEP
        margin[i] = m
    return (codes, margin) if return_margin else codes


def densify_emit(z: np.ndarray, sh_degree: int, codes: np.ndarray, normals: np.ndarray):
    """The densified global set in order (each Gaussian's outputs in place:
    keep -> itself, clone -> itself and its copy, split -> its two children,
    prune -> nothing).  normals: (n, 2, 3) standard normals, row i used if i
    splits.  Returns (z_new, src, original) with src the parent of every new
    Gaussian and original true where it is the parent itself (kept, or the
    first of a clone pair), whose optimiser state and duals carry over."""
    zz = split_params(z, sh_degree)
    out, src, orig = [], [], []
    ln16 = np.log(1.6)
    for i in range(z.shape[0]):
        c = codes[i]
        if c == DENSIFY_PRUNE:
            continue
        if c in (DENSIFY_KEEP, DENSIFY_CLONE):
            out.append(z[i].copy()); src.append(i); orig.append(True)
            if c == DENSIFY_CLONE:
                out.append(z[i].copy()); src.append(i); orig.append(False)
            continue
        R = quat_rotation(zz["quat"][i])
        S = np.exp(zz["scale"][i])
        for h in range(2):
            child = z[i].copy()
            child[0:3] = zz["mean"][i] + R @ (S * normals[i, h])
            child[7:10] = zz["scale"][i] - ln16
            out.append(child); src.append(i); orig.append(False)
    P = z.shape[1]
    z_new = np.array(out, np.float64).reshape(-1, P)
    return z_new, np.array(src, np.int64), np.array(orig, bool)


def reset_opacity(x: np.ndarray, sh_degree: int, cap: float = 0.01) -> np.ndarray:
    """The opacity reset of the 3DGS density control the densification
    follows: every opacity above `cap` is brought down to it (on the logit:
    min(o, logit(cap))).  Returns a new parameter array."""
    y = x.copy()
    o = split_params(y, sh_degree)["opacity"]
    o[:] = np.minimum(o, np.log(cap / (1.0 - cap)))
    return y
