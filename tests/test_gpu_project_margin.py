"""The projection's culling decision at its thresholds.

The kernel decides most culled copies with a float pre-test and leaves the
rest to the exact test (camera depth summed in double, then the lateral
frustum test on it).  The pre-test must never cull a copy the exact test
keeps, nor keep one it would cull in a way that changes the output.  These
copies sit within a few rounding errors of the near plane and of the
lateral frustum edges, in world coordinates of magnitude 1e3 (so the float
depth errs by ~1e-4), and are large enough that every copy passing the
exact test has a non-empty tile rectangle.  The expected decision is the
exact test evaluated on the CPU with correctly rounded float operations
(fma and division emulated exactly), so culled <=> empty rectangle, bit
for bit.  On the CPU, the pre-test itself, evaluated operation for operation
in float32, is checked against the same exact test on the same copies."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from paper_2405_13943_b300 import synth as S

F32 = np.float32


def rn32(q: Fraction) -> F32:
    """q rounded to the nearest float32, ties to even (normal and subnormal
    range; no overflow handling: the test's values are far from it)."""
    if q == 0:
        return F32(0.0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    e = max(e, -126)
    quantum = Fraction(2) ** (e - 23)
    n = a / quantum
    fl = n.numerator // n.denominator
    rem = n - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return F32(sign * float(fl * quantum))


def fma32(a, b, c) -> F32:
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def test_rn32_and_fma32_round_correctly():
    rng = np.random.default_rng(3)
    for x in rng.standard_normal(2000) * 10.0 ** rng.integers(-40, 30, 2000):
        assert rn32(Fraction(float(x))) == F32(x)        # one rounding from double: numpy's is correct
    assert rn32(Fraction(1) + Fraction(1, 2 ** 24)) == F32(1.0)                        # tie to even, down
    assert rn32(Fraction(1) + Fraction(3, 2 ** 24)) == F32(1.0) + F32(2.0 ** -22)       # tie to even, up
    assert rn32(Fraction(1, 2 ** 149)) == F32(2.0 ** -149)
    # an fma whose single rounding differs from rounding the product first
    a = F32(1.0) + F32(2.0 ** -12)
    assert fma32(a, a, F32(-1.0)) == F32(2.0 ** -11 + 2.0 ** -24)
    assert F32(a * a) - F32(1.0) != fma32(a, a, F32(-1.0))


def exact_culled(cam: S.Camera, mu: np.ndarray) -> np.ndarray:
    """The projection's exact culling test: depth = ((R6 x + R7 y) + R8 z) + t2
    in double (exact products), culled if depth <= near; else tz = float(depth),
    tx, ty by the float fma chains, culled if |tx / tz| or |ty / tz| exceeds
    0.65 W / fx or 0.65 H / fy."""
    R = cam.R.astype(F32)
    t = cam.t.astype(F32)
    limx = F32(F32(0.65) * F32(cam.width)) / F32(cam.fx)
    limy = F32(F32(0.65) * F32(cam.height)) / F32(cam.fy)
    near = np.float64(F32(cam.near))
    out = np.empty(len(mu), bool)
    for i, (x, y, z) in enumerate(mu.astype(F32)):
        d = np.float64(R[2, 0]) * np.float64(x)
        d = d + np.float64(R[2, 1]) * np.float64(y)
        d = d + np.float64(R[2, 2]) * np.float64(z)
        d = d + np.float64(t[2])
        if not d > near:
            out[i] = True
            continue
        tz = F32(d)
        tx = fma32(R[0, 0], x, fma32(R[0, 1], y, fma32(R[0, 2], z, t[0])))
        ty = fma32(R[1, 0], x, fma32(R[1, 1], y, fma32(R[1, 2], z, t[1])))
        out[i] = bool(abs(tx / tz) > limx or abs(ty / tz) > limy)
    return out


def boundary_scene(cam: S.Camera, seed: int, n: int = 4000):
    """Copies near the near plane and the four lateral edges, given in camera
    coordinates and mapped to float32 world coordinates (whose rounding
    scatters them across the thresholds)."""
    rng = np.random.default_rng(seed)
    limx = 0.65 * cam.width / cam.fx
    limy = 0.65 * cam.height / cam.fy
    pc = []
    # offsets from a threshold: half within +- 8e-4 (the float depth errs by
    # up to ~5e-4 here), half within +- 0.01 (beyond the pre-test's margin)
    def off():
        return rng.uniform(-1, 1, n) * np.where(rng.random(n) < 0.5, 8e-4, 1e-2)
    # near plane: on axis
    tz = cam.near + off()
    pc.append(np.stack([rng.uniform(-0.05, 0.05, n) * tz, rng.uniform(-0.05, 0.05, n) * tz, tz], 1))
    # lateral edges at depths 1..40
    for axis, lim in ((0, limx), (1, limy)):
        tz = rng.uniform(1.0, 40.0, n)
        side = rng.choice([-1.0, 1.0], n)
        p = np.zeros((n, 3))
        p[:, 2] = tz
        p[:, axis] = side * lim * tz + off()
        p[:, 1 - axis] = rng.uniform(-0.1, 0.1, n) * tz
        pc.append(p)
    pc = np.concatenate(pc)
    R = cam.R.astype(np.float64)
    world = (R.T @ (pc - cam.t.astype(np.float64)).T).T.astype(F32)
    m = len(world)
    # isotropic, a quarter of the depth: screen radius 3 fx s / tz >= 0.75 W
    log_s = np.log(np.maximum(pc[:, 2], cam.near) / 4.0).astype(F32)
    quats = np.tile(np.array([1.0, 0.0, 0.0, 0.0], F32), (m, 1))
    g = S.Gaussians(world, quats, np.repeat(log_s[:, None], 3, 1), np.full(m, 2.0, F32),
                    np.full((m, 1, 3), 0.5, F32))
    return g


def pretest_culled(cam: S.Camera, mu: np.ndarray, margin: float = 2.0 ** -20,
                   widen: float = 1.0 + 2.0 ** -18) -> np.ndarray:
    """The projection's float pre-test, operation for operation in float32
    (fma rounded once): S = |R6 x| + |R7 y| + |R8 z| + |t2|, m = margin S,
    tzf the fma chain; culled if tzf + m < near, or, when tzf - m > max(near, 0),
    if |tx| or |ty| exceeds lim (tzf + m) widen."""
    R = cam.R.astype(F32)
    t = cam.t.astype(F32)
    limx = F32(F32(0.65) * F32(cam.width)) / F32(cam.fx)
    limy = F32(F32(0.65) * F32(cam.height)) / F32(cam.fy)
    near = F32(cam.near)
    out = np.zeros(len(mu), bool)
    for i, (x, y, z) in enumerate(mu.astype(F32)):
        Sm = ((abs(R[2, 0] * x) + abs(R[2, 1] * y)) + abs(R[2, 2] * z)) + abs(t[2])
        if not Sm >= F32(2.0 ** -100):
            continue
        m = Sm * F32(margin)
        tzf = fma32(R[2, 0], x, fma32(R[2, 1], y, fma32(R[2, 2], z, t[2])))
        if tzf + m < near:
            out[i] = True
            continue
        if not tzf - m > max(near, F32(0.0)):
            continue
        tx = fma32(R[0, 0], x, fma32(R[0, 1], y, fma32(R[0, 2], z, t[0])))
        ty = fma32(R[1, 0], x, fma32(R[1, 1], y, fma32(R[1, 2], z, t[1])))
        zb = (tzf + m) * F32(widen)
        out[i] = bool(abs(tx) > limx * zb or abs(ty) > limy * zb)
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_pretest_culls_only_where_the_exact_test_culls(seed):
    """The margin argument of the pre-test, on the CPU: on copies at the
    thresholds it never culls a copy the exact test keeps, and it still
    decides most copies beyond its margin.  With no margin and no widening
    it does cull kept copies on the same data, so the data reaches the
    cases the margin is there for."""
    cam = rotated_far_camera()
    g = boundary_scene(cam, seed)
    exact = exact_culled(cam, g.means)
    pre = pretest_culled(cam, g.means)
    assert not np.any(pre & ~exact), np.flatnonzero(pre & ~exact)[:10]
    assert pre.sum() > 0.3 * exact.sum()
    bare = pretest_culled(cam, g.means, margin=0.0, widen=1.0)
    assert np.any(bare & ~exact)


def rotated_far_camera():
    from scipy.spatial.transform import Rotation
    R = Rotation.from_rotvec([0.7, -0.4, 0.25]).as_matrix().astype(np.float32)
    campos = np.array([1000.5, -2000.25, 500.125], np.float32)
    t = (-(R.astype(np.float64) @ campos.astype(np.float64))).astype(np.float32)
    return S.Camera(64, 48, 64.0, 64.0, 32.0, 24.0, R, t, campos, 0.2)


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [0, 1])
def test_projection_culling_at_its_thresholds(seed):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from paper_2405_13943_b300 import dogs as D
    cam = rotated_far_camera()
    g = boundary_scene(cam, seed)
    expect = exact_culled(cam, g.means)
    xb = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch([cam], [0, g.n], 16, 16)
    D.dg_project(xb, vb)
    torch.cuda.synchronize()
    r = vb.rect.cpu().numpy()[:2 * g.n].reshape(-1, 2).astype(np.uint32)
    x0, y0, x1, y1 = r[:, 0] & 0xFFFF, r[:, 0] >> 16, r[:, 1] & 0xFFFF, r[:, 1] >> 16
    empty = ~((x1 > x0) & (y1 > y0))
    n = g.n // 3
    for fam, name in enumerate(("near", "x edge", "y edge")):
        sl = slice(fam * n, (fam + 1) * n)
        assert 0.2 * n < expect[sl].sum() < 0.8 * n, name        # both sides well populated
        bad = np.flatnonzero(empty[sl] != expect[sl])
        assert bad.size == 0, (name, bad[:10])


# ---- the depth in float arithmetic with an FP64 fallback --------------------
def add32(a, b) -> F32:
    return rn32(Fraction(float(a)) + Fraction(float(b)))


def sub32(a, b) -> F32:
    return rn32(Fraction(float(a)) - Fraction(float(b)))


def mul32(a, b) -> F32:
    return rn32(Fraction(float(a)) * Fraction(float(b)))


def two_sum32(a, b):
    s = add32(a, b)
    bb = sub32(s, a)
    return s, add32(sub32(a, sub32(s, bb)), sub32(b, bb))


def depth_double(R6, R7, R8, t2, near, x, y, z):
    """The FP64 depth as the kernel sums it: (front, float depth)."""
    d = np.float64(R6) * np.float64(x)
    d = d + np.float64(R7) * np.float64(y)
    d = d + np.float64(R8) * np.float64(z)
    d = d + np.float64(t2)
    return bool(d > np.float64(near)), F32(d)


def depth_fast32(R6, R7, R8, t2, near, x, y, z):
    """The kernel's float path, operation for operation with each operation
    rounded once: (front, float depth) where it decides, None where the FP64
    sum must."""
    h6, h7, h8 = mul32(R6, x), mul32(R7, y), mul32(R8, z)
    l6, l7, l8 = fma32(R6, x, -h6), fma32(R7, y, -h7), fma32(R8, z, -h8)
    s, e1 = two_sum32(h6, h7)
    s, e2 = two_sum32(s, h8)
    s, e3 = two_sum32(s, t2)
    lo = add32(add32(add32(l6, l7), add32(l8, e1)), add32(e2, e3))
    S_ = add32(add32(abs(h6), abs(h7)), add32(abs(h8), abs(t2)))
    if not (F32(2.0 ** -80) <= S_ <= F32(2.0 ** 100)):
        return None
    M = mul32(S_, F32(2.0 ** -40))
    dn = sub32(s, near)
    gap = add32(dn, lo)
    Mn = fma32(abs(dn), F32(2.0 ** -22), M)
    if gap < -Mn:
        return False, None
    if not gap > Mn:
        return None
    f = add32(s, lo)
    if not f >= F32(2.0 ** -100):
        return None
    r = add32(sub32(s, f), lo)
    below = sub32(f, np.nextafter(f, F32(0.0)))
    if abs(r) < sub32(mul32(F32(0.5), below), mul32(M, F32(1.0625))):
        return True, f
    return None


def depth_cases(seed, n=1500):
    """Camera rows and means whose FP64 depth lies within 2^-12 of a float
    ulp of a float rounding boundary or within 1e-6 of the near plane (kept
    from many random draws), plus exact ties: R8 = 1 with z + t2 a float
    midpoint."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        m = 200000
        R = rng.standard_normal((m, 3))
        R /= np.linalg.norm(R, axis=1, keepdims=True)
        R = R.astype(F32)
        mu = (rng.uniform(-1500, 1500, (m, 3))).astype(F32)
        t2 = rng.uniform(-2000, 2000, m).astype(F32)
        d = ((R[:, 0].astype(np.float64) * mu[:, 0] + R[:, 1].astype(np.float64) * mu[:, 1])
             + R[:, 2].astype(np.float64) * mu[:, 2]) + t2.astype(np.float64)
        f = d.astype(F32).astype(np.float64)
        ulp = np.abs(np.spacing(d.astype(F32))).astype(np.float64)
        frac = np.abs(np.abs(d - f) / ulp - 0.5)           # 0 at a rounding boundary
        near = np.where(rng.random(m) < 0.5, 0.2, np.abs(d) * (1 + rng.uniform(-1e-6, 1e-6, m))).astype(F32)
        pick = np.flatnonzero((frac < 2.0 ** -12) | (np.abs(d - near) < 1e-6 * np.abs(d)))
        for i in pick[: n - len(out)]:
            out.append((R[i, 0], R[i, 1], R[i, 2], t2[i], near[i], mu[i, 0], mu[i, 1], mu[i, 2]))
    one, zero = F32(1.0), F32(0.0)
    for z, t in ((F32(1.0), F32(2.0 ** -24)), (F32(3.0), F32(2.0 ** -23)), (F32(100.0), F32(2.0 ** -18)),
                 (F32(1.0), F32(3 * 2.0 ** -24))):
        out.append((zero, zero, one, t, F32(0.2), F32(5.0), F32(-7.0), z))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_float_depth_decides_only_where_it_equals_the_fp64_sum(seed):
    """The float path's margin argument, on the CPU: wherever it decides, its
    near-plane decision and float depth equal those of the FP64 sum, on
    depths at float rounding boundaries (exact ties included) and at the
    near plane; it decides most of them and leaves the ties to FP64."""
    decided = fell = 0
    for c in depth_cases(seed):
        want = depth_double(*c)
        got = depth_fast32(*c)
        if got is None:
            fell += 1
            continue
        decided += 1
        assert got[0] == want[0], c
        if want[0]:
            assert got[1].view(np.uint32) == want[1].view(np.uint32), c
    assert decided > 0.5 * (decided + fell) and fell >= 4


@pytest.mark.gpu
def test_projected_depth_bits_at_rounding_ties():
    """On the GPU: copies whose FP64 depth is an exact float midpoint (ties
    to even) or a hair beside one, seen by an axis-aligned camera: the
    record's depth and the keys' depth bits equal the FP64 sum's rounding."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_13943_b300 import build as B
    B.build()
    from paper_2405_13943_b300 import dogs as D
    R = np.eye(3, dtype=F32)
    cam = S.Camera(64, 48, 64.0, 64.0, 32.0, 24.0, R, np.array([0.0, 0.0, 2.0 ** -24], F32),
                   np.array([0.0, 0.0, -(2.0 ** -24)], F32), 0.2)
    zs = []
    for base in (1.0, 3.0, 10.0, 100.0, 1000.0):
        f = F32(base)
        for k in range(-3, 4):
            zs.append(np.nextafter(f, F32(np.inf)) if k > 0 else f)
            f = np.nextafter(f, F32(np.inf))
    zs = np.array(zs, F32)
    n = len(zs)
    means = np.stack([np.zeros(n, F32), np.zeros(n, F32), zs], 1)
    g = S.Gaussians(means, np.tile(np.array([1.0, 0, 0, 0], F32), (n, 1)), np.full((n, 3), -3.0, F32),
                    np.full(n, 2.0, F32), np.full((n, 1, 3), 0.5, F32))
    xb = D.GaussianBuffer.from_synth(g)
    vb = D.ViewBatch([cam], [0, n], 16, 16)
    D.dg_project(xb, vb)
    torch.cuda.synchronize()
    rec = vb.rec.cpu().numpy()[:12 * n].reshape(n, 12)
    for i in range(n):
        front, tz = depth_double(F32(0), F32(0), F32(1), cam.t[2], F32(cam.near), F32(0), F32(0), zs[i])
        assert front
        assert rec[i, 9].astype(F32).view(np.uint32) == tz.view(np.uint32), (i, zs[i], rec[i, 9], tz)
