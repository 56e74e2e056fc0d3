// K1 project_fwd and K8 project_bwd.
//
// Projection of 3D Gaussians (Sec. 3.1: Eq. 1, Sigma = R S S^T R^T) to 2D
// conics with the EWA local-affine approximation J W Sigma W^T J^T + 0.3 I,
// real SH colour of degree <= 3, sigmoid opacity; and its analytic adjoint.
//
// Forward: a CTA takes a run of consecutive local copies, culls them with a
// float pre-test on their means, and projects the rest densely (k_project).
// A copy is loaded once (coalesced float4 SoA for mean/opacity, rotation,
// scale; planar SH) and projected into every view of its block, so the
// parameters are read once per step however many views a block has.
// HBM- and latency-bound.  The adjoint takes one thread per copy.
#include "common.cuh"

namespace dg {

// Real SH basis with the Condon-Shortley phase, k = l*l + l + m, written as
// polynomials in the unit direction (x, y, z).  Coefficients are the closed
// forms 1/2 sqrt(1/pi), sqrt(3/(4pi)), 1/2 sqrt(15/pi), 1/4 sqrt(5/pi),
// 1/4 sqrt(15/pi), 1/4 sqrt(35/(2pi)), 1/2 sqrt(105/pi), 1/4 sqrt(21/(2pi)),
// 1/4 sqrt(7/pi), 1/4 sqrt(105/pi).
#define SH_C0 0.28209479177387814f
#define SH_C1 0.48860251190291992f
#define SH_C2A 1.0925484305920792f
#define SH_C2B 0.31539156525252005f
#define SH_C2C 0.54627421529603959f
#define SH_C3A 0.59004358992664352f
#define SH_C3B 2.8906114426405538f
#define SH_C3C 0.45704579946446572f
#define SH_C3D 0.37317633259011540f
#define SH_C3E 1.4453057213202769f

template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y)
{
    Y[0] = SH_C0;
    if (DEG >= 1) {
        Y[1] = -SH_C1 * y;
        Y[2] = SH_C1 * z;
        Y[3] = -SH_C1 * x;
    }
    if (DEG >= 2) {
        Y[4] = SH_C2A * x * y;
        Y[5] = -SH_C2A * y * z;
        Y[6] = SH_C2B * (3.f * z * z - 1.f);
        Y[7] = -SH_C2A * x * z;
        Y[8] = SH_C2C * (x * x - y * y);
    }
    if (DEG >= 3) {
        Y[9] = -SH_C3A * y * (3.f * x * x - y * y);
        Y[10] = SH_C3B * x * y * z;
        Y[11] = -SH_C3C * y * (5.f * z * z - 1.f);
        Y[12] = SH_C3D * z * (5.f * z * z - 3.f);
        Y[13] = -SH_C3C * x * (5.f * z * z - 1.f);
        Y[14] = SH_C3E * z * (x * x - y * y);
        Y[15] = -SH_C3A * x * (x * x - 3.f * y * y);
    }
}

// sum_k w_k grad Y_k of the polynomials above
template <int DEG>
__device__ __forceinline__ float3 sh_grad_dot(float x, float y, float z, const float* w)
{
    float gx = 0.f, gy = 0.f, gz = 0.f;
    if (DEG >= 1) {
        gy -= SH_C1 * w[1];
        gz += SH_C1 * w[2];
        gx -= SH_C1 * w[3];
    }
    if (DEG >= 2) {
        gx += SH_C2A * y * w[4];            gy += SH_C2A * x * w[4];
        gy -= SH_C2A * z * w[5];            gz -= SH_C2A * y * w[5];
        gz += 6.f * SH_C2B * z * w[6];
        gx -= SH_C2A * z * w[7];            gz -= SH_C2A * x * w[7];
        gx += 2.f * SH_C2C * x * w[8];      gy -= 2.f * SH_C2C * y * w[8];
    }
    if (DEG >= 3) {
        gx -= 6.f * SH_C3A * x * y * w[9];  gy -= SH_C3A * (3.f * x * x - 3.f * y * y) * w[9];
        gx += SH_C3B * y * z * w[10];       gy += SH_C3B * x * z * w[10];   gz += SH_C3B * x * y * w[10];
        gy -= SH_C3C * (5.f * z * z - 1.f) * w[11];                          gz -= 10.f * SH_C3C * y * z * w[11];
        gz += SH_C3D * (15.f * z * z - 3.f) * w[12];
        gx -= SH_C3C * (5.f * z * z - 1.f) * w[13];                          gz -= 10.f * SH_C3C * x * z * w[13];
        gx += 2.f * SH_C3E * x * z * w[14]; gy -= 2.f * SH_C3E * y * z * w[14]; gz += SH_C3E * (x * x - y * y) * w[14];
        gx -= SH_C3A * (3.f * x * x - 3.f * y * y) * w[15];                  gy += 6.f * SH_C3A * x * y * w[15];
    }
    return make_float3(gx, gy, gz);
}

struct CamL {
    float R[9], t[3], cp[3];
    float fx, fy, cx, cy, nearz;
    int W, H, TX, TY;
    int64_t rec_off, gb;
};

__device__ __forceinline__ void load_cam(const dg_camera* cams, int v, CamL& c)
{
    const dg_camera* p = cams + v;
#pragma unroll
    for (int i = 0; i < 9; i++) c.R[i] = __ldg(&p->R[i]);
#pragma unroll
    for (int i = 0; i < 3; i++) { c.t[i] = __ldg(&p->t[i]); c.cp[i] = __ldg(&p->campos[i]); }
    c.fx = __ldg(&p->fx); c.fy = __ldg(&p->fy); c.cx = __ldg(&p->cx); c.cy = __ldg(&p->cy);
    c.nearz = __ldg(&p->near_z);
    c.W = __ldg(&p->width); c.H = __ldg(&p->height);
    c.TX = __ldg(&p->tiles_x); c.TY = __ldg(&p->tiles_y);
    c.rec_off = __ldg(&p->rec_off); c.gb = __ldg(&p->gauss_begin);
}

// camera-frame depth, summed in double in a fixed order: the products of two
// floats are exact in double, so the result rounds identically everywhere
__device__ __forceinline__ double cam_depth(const CamL& c, float3 mu)
{
    double s = __dmul_rn((double)c.R[6], (double)mu.x);
    s = __dadd_rn(s, __dmul_rn((double)c.R[7], (double)mu.y));
    s = __dadd_rn(s, __dmul_rn((double)c.R[8], (double)mu.z));
    return __dadd_rn(s, (double)c.t[2]);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The decisions cam_depth feeds -- depth > near, and the depth's float
// rounding tz -- taken in float arithmetic, FP64 only where that cannot
// decide.  Each product splits exactly into hi + lo (the error of a float
// product is itself a float, given by an FMA); the his are summed by TwoSum
// with their errors, so s + lo lies within 2^-43 S of the exact sum, and
// cam_depth's double within 3 2^-53 S of it (S = |R6 x| + |R7 y| + |R8 z| +
// |t2|).  With the margin M = 2^-40 S:
//   (s - near) + lo > M      =>  depth > near      (s - near is exact when
//   (s - near) + lo < -M     =>  depth <= near      s is within 2x of near;
//                                                    farther, 2^-22 |s - near|
//                                                    covers its rounding);
//   |(s - f) + lo| < ulp/2 - M, f = rn(s + lo), ulp the spacing below f
//                            =>  rn(depth) = f     (no float rounding
//                                                    boundary within M).
// Otherwise (near a threshold or a boundary, S outside [2^-80, 2^100], NaN)
// the FP64 sum decides.  Returns depth > near; tz is set when it is true.
__device__ __forceinline__ bool cam_depth_front(const CamL& c, float3 mu, float& tz)
{
    const float h6 = __fmul_rn(c.R[6], mu.x), h7 = __fmul_rn(c.R[7], mu.y), h8 = __fmul_rn(c.R[8], mu.z);
    const float l6 = __fmaf_rn(c.R[6], mu.x, -h6), l7 = __fmaf_rn(c.R[7], mu.y, -h7);
    const float l8 = __fmaf_rn(c.R[8], mu.z, -h8);
    float s, e1, e2, e3;
    two_sum(h6, h7, s, e1);
    two_sum(s, h8, s, e2);
    two_sum(s, c.t[2], s, e3);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(l6, l7), __fadd_rn(l8, e1)), __fadd_rn(e2, e3));
    const float S = __fadd_rn(__fadd_rn(fabsf(h6), fabsf(h7)), __fadd_rn(fabsf(h8), fabsf(c.t[2])));
    if (S >= 0x1p-80f && S <= 0x1p100f) {
        const float M = __fmul_rn(S, 0x1p-40f);
        const float dn = __fsub_rn(s, c.nearz);
        const float gap = __fadd_rn(dn, lo);
        const float Mn = __fmaf_rn(fabsf(dn), 0x1p-22f, M);
        if (gap < -Mn) return false;
        if (gap > Mn) {
            const float f = __fadd_rn(s, lo);
            if (f >= 0x1p-100f) {
                const float r = __fadd_rn(__fsub_rn(s, f), lo);
                const float below = __fsub_rn(f, __int_as_float(__float_as_int(f) - 1));
                if (fabsf(r) < __fsub_rn(__fmul_rn(0.5f, below), __fmul_rn(M, 1.0625f))) {
                    tz = f;
                    return true;
                }
            }
        }
    }
    const double d = cam_depth(c, mu);
    tz = (float)d;
    return d > (double)c.nearz;
}

// Screen-space geometry of one Gaussian in one view.
struct Geom {
    float tx, ty, tz, xn, yn;
    float Rq[9];          // rotation from the normalised quaternion
    float qn[4], qinv;    // normalised quaternion (w,x,y,z), 1/|q|
    float s[3];           // scales
    float Sig[6];         // Sigma: 00 01 02 11 12 22
    float T0[3], T1[3];   // rows of J W
    float A, B, C, det;   // Sigma' = [[A, B], [B, C]]
    float a, b, c;        // conic
    float mx, my;
};

// The lateral frustum test of geom() on the mean alone (the same expressions,
// so the same decisions), taken before the rest of a copy's parameters load.
__device__ __forceinline__ bool in_frustum(const CamL& cam, float tz, float3 mu)
{
    const float tx = fmaf(cam.R[0], mu.x, fmaf(cam.R[1], mu.y, fmaf(cam.R[2], mu.z, cam.t[0])));
    const float ty = fmaf(cam.R[3], mu.x, fmaf(cam.R[4], mu.y, fmaf(cam.R[5], mu.z, cam.t[1])));
    const float xn = tx / tz, yn = ty / tz;
    const float limx = 0.65f * (float)cam.W / cam.fx, limy = 0.65f * (float)cam.H / cam.fy;
    return !(fabsf(xn) > limx || fabsf(yn) > limy);
}

// A float pre-test that is true only where the test above (with the double
// depth) culls as well, so that most culled copies skip the FP64 arithmetic,
// which is slow on this part.  The float depth tzf (three rounded FMAs) and
// the double sum tzd both lie within 3u S (u = 2^-24 for tzf, 2^-53 for tzd)
// of the exact depth, S = |R6 x| + |R7 y| + |R8 z| + |t2|; so
// |tzf - tzd| < 4u S.  With the margin m = 16u S (each comparison's own
// rounding adds at most u S):
//   tzf + m < near          =>  tzd < near, culled by the near test;
//   tzf - m > max(near, 0)  =>  tzd > near and tzd > 0, and the depth the
//     lateral test divides by, tz = rn(tzd) <= (tzf + m) (1 + u); then
//     |tx| > lim (tzf + m) (1 + 2^-18), rounded three times, still gives
//     |tx| / tz > lim (1 + 58u), whose rounding is above lim, so the lateral
//     test culls.  tx, ty are the same expressions as in in_frustum.
// S >= 2^-100 keeps every rounding error relative (a subnormal partial sum
// errs by 2^-150 at most, far below u S); smaller S, NaN or infinite inputs
// fail a comparison here and take the exact path.
__device__ __forceinline__ bool surely_culled(const CamL& cam, float3 mu)
{
    const float S = fabsf(cam.R[6] * mu.x) + fabsf(cam.R[7] * mu.y) + fabsf(cam.R[8] * mu.z) + fabsf(cam.t[2]);
    if (!(S >= 0x1p-100f)) return false;
    const float m = S * 0x1p-20f;
    const float tzf = fmaf(cam.R[6], mu.x, fmaf(cam.R[7], mu.y, fmaf(cam.R[8], mu.z, cam.t[2])));
    if (tzf + m < cam.nearz) return true;
    if (!(tzf - m > fmaxf(cam.nearz, 0.f))) return false;
    const float tx = fmaf(cam.R[0], mu.x, fmaf(cam.R[1], mu.y, fmaf(cam.R[2], mu.z, cam.t[0])));
    const float ty = fmaf(cam.R[3], mu.x, fmaf(cam.R[4], mu.y, fmaf(cam.R[5], mu.z, cam.t[1])));
    const float limx = 0.65f * (float)cam.W / cam.fx, limy = 0.65f * (float)cam.H / cam.fy;
    const float zb = (tzf + m) * (1.f + 0x1p-18f);
    return fabsf(tx) > limx * zb || fabsf(ty) > limy * zb;
}

// Computes every field; returns false if the Gaussian is culled in this
// view.  The caller has already checked camera z > near_z (exact, in double),
// so no division below is by a non-positive depth.  Fills rect if non-null.
__device__ __forceinline__ bool geom(const CamL& cam, float tz, float3 mu, float4 q, float4 sc, int tw,
                                     int th, Geom& g, uint2* rect_out)
{
    g.tz = tz;
    g.tx = fmaf(cam.R[0], mu.x, fmaf(cam.R[1], mu.y, fmaf(cam.R[2], mu.z, cam.t[0])));
    g.ty = fmaf(cam.R[3], mu.x, fmaf(cam.R[4], mu.y, fmaf(cam.R[5], mu.z, cam.t[1])));
    g.xn = g.tx / g.tz;
    g.yn = g.ty / g.tz;
    float limx = 0.65f * (float)cam.W / cam.fx, limy = 0.65f * (float)cam.H / cam.fy;
    bool vis = !(fabsf(g.xn) > limx || fabsf(g.yn) > limy);
    // rotation from the normalised quaternion (w, x, y, z) = (q.x, q.y, q.z, q.w)
    float qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
    g.qinv = rsqrtf(qq);
    float w = q.x * g.qinv, x = q.y * g.qinv, y = q.z * g.qinv, z = q.w * g.qinv;
    g.qn[0] = w; g.qn[1] = x; g.qn[2] = y; g.qn[3] = z;
    g.Rq[0] = 1.f - 2.f * (y * y + z * z); g.Rq[1] = 2.f * (x * y - w * z); g.Rq[2] = 2.f * (x * z + w * y);
    g.Rq[3] = 2.f * (x * y + w * z); g.Rq[4] = 1.f - 2.f * (x * x + z * z); g.Rq[5] = 2.f * (y * z - w * x);
    g.Rq[6] = 2.f * (x * z - w * y); g.Rq[7] = 2.f * (y * z + w * x); g.Rq[8] = 1.f - 2.f * (x * x + y * y);
    g.s[0] = __expf(sc.x); g.s[1] = __expf(sc.y); g.s[2] = __expf(sc.z);
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M[3 * i + j] = g.Rq[3 * i + j] * g.s[j];
    g.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    g.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    g.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    g.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    g.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    g.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    float fz = cam.fx / g.tz, gz = cam.fy / g.tz;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        g.T0[j] = fz * (cam.R[j] - g.xn * cam.R[6 + j]);
        g.T1[j] = gz * (cam.R[3 + j] - g.yn * cam.R[6 + j]);
    }
    float U0[3], U1[3];
    U0[0] = g.Sig[0] * g.T0[0] + g.Sig[1] * g.T0[1] + g.Sig[2] * g.T0[2];
    U0[1] = g.Sig[1] * g.T0[0] + g.Sig[3] * g.T0[1] + g.Sig[4] * g.T0[2];
    U0[2] = g.Sig[2] * g.T0[0] + g.Sig[4] * g.T0[1] + g.Sig[5] * g.T0[2];
    U1[0] = g.Sig[0] * g.T1[0] + g.Sig[1] * g.T1[1] + g.Sig[2] * g.T1[2];
    U1[1] = g.Sig[1] * g.T1[0] + g.Sig[3] * g.T1[1] + g.Sig[4] * g.T1[2];
    U1[2] = g.Sig[2] * g.T1[0] + g.Sig[4] * g.T1[1] + g.Sig[5] * g.T1[2];
    g.A = g.T0[0] * U0[0] + g.T0[1] * U0[1] + g.T0[2] * U0[2] + 0.3f;
    g.B = g.T0[0] * U1[0] + g.T0[1] * U1[1] + g.T0[2] * U1[2];
    g.C = g.T1[0] * U1[0] + g.T1[1] * U1[1] + g.T1[2] * U1[2] + 0.3f;
    g.det = g.A * g.C - g.B * g.B;
    vis = vis && (g.det > 0.f);
    float id = 1.f / g.det;
    g.a = g.C * id; g.b = -g.B * id; g.c = g.A * id;
    g.mx = cam.fx * g.xn + cam.cx;
    g.my = cam.fy * g.yn + cam.cy;
    if (!vis) return false;
    float mid = 0.5f * (g.A + g.C);
    float lmax = mid + sqrtf(fmaxf(mid * mid - g.det, 0.f));
    float r = ceilf(3.f * sqrtf(lmax));
    int x0 = (int)floorf((g.mx - r) / (float)tw), x1 = (int)floorf((g.mx + r) / (float)tw) + 1;
    int y0 = (int)floorf((g.my - r) / (float)th), y1 = (int)floorf((g.my + r) / (float)th) + 1;
    x0 = min(max(x0, 0), cam.TX); x1 = min(max(x1, 0), cam.TX);
    y0 = min(max(y0, 0), cam.TY); y1 = min(max(y1, 0), cam.TY);
    if (x1 <= x0 || y1 <= y0) return false;
    if (rect_out) *rect_out = make_uint2((uint32_t)x0 | ((uint32_t)y0 << 16), (uint32_t)x1 | ((uint32_t)y1 << 16));
    return true;
}

// Projects copy c (mean and opacity logit mo) into every view of its block:
// a record and a tile rectangle per view (an empty rectangle where it is
// culled).  Called for the copies the float pre-test could not cull, which
// are nearly all kept, so the rotation and scales load up front, in flight
// during the exact depth test.
template <int DEG>
__device__ __forceinline__ void project_copy(const GView& x, const dg_camera* __restrict__ cams, const dg_plan& plan,
                                             int64_t c, float4 mo, float4* __restrict__ rec, uint2* __restrict__ rect)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    int k = find_block(plan, c);
    int v0 = plan.blk_view_off[k], v1 = plan.blk_view_off[k + 1];
    const float3 mu = make_float3(mo.x, mo.y, mo.z);
    const float4 q = x.quat[c], sc = x.scale[c];
    const float opac = 1.f / (1.f + __expf(-mo.w));
    const float* __restrict__ shp = x.sh + c;
    for (int v = v0; v < v1; v++) {
        CamL cam;
        load_cam(cams, v, cam);
        int64_t r = cam.rec_off + (c - cam.gb);
        if (surely_culled(cam, mu)) { rect[r] = make_uint2(0, 0); continue; }
        float tz;
        if (!cam_depth_front(cam, mu, tz) || !in_frustum(cam, tz, mu)) { rect[r] = make_uint2(0, 0); continue; }
        Geom g;
        uint2 rr;
        if (!geom(cam, tz, mu, q, sc, plan.tile_w, plan.tile_h, g, &rr)) { rect[r] = make_uint2(0, 0); continue; }
        float dx = mu.x - cam.cp[0], dy = mu.y - cam.cp[1], dz = mu.z - cam.cp[2];
        float il = rsqrtf(dx * dx + dy * dy + dz * dz);
        float Y[NK];
        sh_eval<DEG>(dx * il, dy * il, dz * il, Y);
        // colour: SH coefficients streamed from their planes (coalesced across the warp)
        float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int kk = 0; kk < NK; kk++)
#pragma unroll
            for (int ch = 0; ch < 3; ch++) col[ch] = fmaf(__ldg(shp + (int64_t)(3 * kk + ch) * x.ld), Y[kk], col[ch]);
        rec[3 * r + 0] = make_float4(g.mx, g.my, g.a, g.b);
        rec[3 * r + 1] = make_float4(g.c, opac, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f));
        rec[3 * r + 2] = make_float4(fmaxf(col[2], 0.f), g.tz, 0.f, 0.f);
        rect[r] = rr;
    }
}

constexpr int kProjThreads = 256;
constexpr int kProjCtasPerSm = 4;     // the register budget of __launch_bounds__ below

// One CTA per kProjThreads * PER consecutive copies, in two passes.
// Culling pass: each thread loads the means of its PER copies at once
// (more loads in flight than one copy per thread) and runs the float
// pre-test in every view of the copy's block; a copy culled in all of them
// gets its empty rectangles here.  The others are listed in shared memory
// in ascending copy order (warp ballots, then one warp's scan of the
// per-warp counts) with their means, and the CTA projects the list densely
// with project_copy, whose exact test decides them.
template <int DEG, int PER>
__global__ void __launch_bounds__(kProjThreads, kProjCtasPerSm) k_project(GView x, const dg_camera* __restrict__ cams,
                                                                          dg_plan plan, float4* __restrict__ rec,
                                                                          uint2* __restrict__ rect)
{
    constexpr int NW = kProjThreads / 32;
    constexpr int kProjPer = PER;
    static_assert(PER >= 1 && PER * NW <= 32, "one warp scans the per-warp counts");
    __shared__ float4 s_mo[kProjThreads * kProjPer];
    __shared__ int s_list[kProjThreads * kProjPer];
    __shared__ int s_off[NW * kProjPer + 1];
    const int64_t n = plan.blk_off[plan.n_blocks];
    const int64_t base = (int64_t)blockIdx.x * (kProjThreads * kProjPer);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float4 mo[kProjPer];
#pragma unroll
    for (int j = 0; j < kProjPer; j++) {
        const int64_t c = base + threadIdx.x + kProjThreads * j;
        mo[j] = c < n ? x.mo[c] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    unsigned bal[kProjPer];
#pragma unroll
    for (int j = 0; j < kProjPer; j++) {
        const int64_t c = base + threadIdx.x + kProjThreads * j;
        bool need = false;
        if (c < n) {
            const int k = find_block(plan, c);
            const int v0 = plan.blk_view_off[k], v1 = plan.blk_view_off[k + 1];
            const float3 mu = make_float3(mo[j].x, mo[j].y, mo[j].z);
            for (int v = v0; v < v1 && !need; v++) {
                CamL cam;
                load_cam(cams, v, cam);
                need = !surely_culled(cam, mu);
            }
            if (!need)
                for (int v = v0; v < v1; v++)
                    rect[__ldg(&cams[v].rec_off) + (c - __ldg(&cams[v].gauss_begin))] = make_uint2(0, 0);
        }
        bal[j] = __ballot_sync(0xffffffffu, need);
        if (lane == 0) s_off[j * NW + warp] = __popc(bal[j]);
    }
    __syncthreads();
    if (warp == 0) {   // exclusive scan of the counts in (pass, warp) order: the list ascends in c
        const int v = lane < NW * kProjPer ? s_off[lane] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane < NW * kProjPer) s_off[lane] = incl - v;
        if (lane == 31) s_off[NW * kProjPer] = incl;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kProjPer; j++)
        if ((bal[j] >> lane) & 1u) {
            const int at = s_off[j * NW + warp] + __popc(bal[j] & ((1u << lane) - 1u));
            s_list[at] = threadIdx.x + kProjThreads * j;
            s_mo[at] = mo[j];
        }
    __syncthreads();
    const int cnt = s_off[NW * kProjPer];
    for (int i = threadIdx.x; i < cnt; i += kProjThreads)
        project_copy<DEG>(x, cams, plan, base + s_list[i], s_mo[i], rec, rect);
}

// ---------------------------------------------------------------------------
// K8: adjoint of the projection, accumulated over the views of the block.
// ---------------------------------------------------------------------------
// Adjoint of one record (copy c seen by one view), in two parts.
// colour_adjoint: from the record's colour gradient (d1.z, d1.w, d2.x) and
// opacity gradient (d1.y), adds dL/d(opacity logit) to go and the view
// direction's share of dL/d(mean) to gmu, and returns the colour gradient gc
// (zero on clamped channels) and the SH basis Y of the view direction, so
// that dL/d f_{k,ch} = gc[ch] Y[k].  f: the copy's SH coefficients (3 NK,
// coefficient-major).
template <int DEG>
__device__ __forceinline__ void colour_adjoint(const CamL& cam, float3 mu, float opac, const float* f, float4 d1,
                                               float4 d2, float* gmu, float& go, float* gc, float* Y)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    // opacity logit
    go += d1.y * opac * (1.f - opac);
    // colour -> SH coefficients and the view direction
    float vx = mu.x - cam.cp[0], vy = mu.y - cam.cp[1], vz = mu.z - cam.cp[2];
    float il = rsqrtf(vx * vx + vy * vy + vz * vz);
    float ux = vx * il, uy = vy * il, uz = vz * il;
    sh_eval<DEG>(ux, uy, uz, Y);
    gc[0] = d1.z; gc[1] = d1.w; gc[2] = d2.x;
#pragma unroll
    for (int ch = 0; ch < 3; ch++) {
        float s = 0.5f;
#pragma unroll
        for (int kk = 0; kk < NK; kk++) s = fmaf(f[3 * kk + ch], Y[kk], s);
        if (!(s > 0.f)) gc[ch] = 0.f;            // clamped channel
    }
    if (DEG > 0) {
        float wk[NK];
#pragma unroll
        for (int kk = 0; kk < NK; kk++) wk[kk] = gc[0] * f[3 * kk] + gc[1] * f[3 * kk + 1] + gc[2] * f[3 * kk + 2];
        float3 gd = sh_grad_dot<DEG>(ux, uy, uz, wk);
        float dd = gd.x * ux + gd.y * uy + gd.z * uz;
        gmu[0] += (gd.x - ux * dd) * il;
        gmu[1] += (gd.y - uy * dd) * il;
        gmu[2] += (gd.z - uz * dd) * il;
    }
}

// geometry_adjoint: from the record's mean2d and conic gradients (d0), adds
// dL/d(mean, rotation, log-scale) of the EWA projection to gmu, gq, gs.
template <int DEG>
__device__ __forceinline__ void geometry_adjoint(const CamL& cam, float3 mu, float4 q, float4 sc, float4 d0,
                                                 float4 d1, int tile_w, int tile_h, float* gmu, float* gq,
                                                 float* gs)
{
    Geom g;
    float tz;
    cam_depth_front(cam, mu, tz);          // a kept record: in front, tz its float depth
    geom(cam, tz, mu, q, sc, tile_w, tile_h, g, nullptr);  // forward's rect decides
    // conic (a, b, c) -> Sigma' entries (A, B, C)
    float da = d0.z, db = d0.w, dc = d1.x;
    float id2 = 1.f / (g.det * g.det);
    float gA = (-g.C * g.C * da + g.B * g.C * db - g.B * g.B * dc) * id2;
    float gB = (2.f * g.B * g.C * da - (g.A * g.C + g.B * g.B) * db + 2.f * g.A * g.B * dc) * id2;
    float gC = (-g.B * g.B * da + g.A * g.B * db - g.A * g.A * dc) * id2;
    // Sigma' = T Sigma T^T: dSigma = T^T G T, dT = 2 G T Sigma, G = [[gA, gB/2], [gB/2, gC]]
    float U0[3], U1[3];
    U0[0] = g.Sig[0] * g.T0[0] + g.Sig[1] * g.T0[1] + g.Sig[2] * g.T0[2];
    U0[1] = g.Sig[1] * g.T0[0] + g.Sig[3] * g.T0[1] + g.Sig[4] * g.T0[2];
    U0[2] = g.Sig[2] * g.T0[0] + g.Sig[4] * g.T0[1] + g.Sig[5] * g.T0[2];
    U1[0] = g.Sig[0] * g.T1[0] + g.Sig[1] * g.T1[1] + g.Sig[2] * g.T1[2];
    U1[1] = g.Sig[1] * g.T1[0] + g.Sig[3] * g.T1[1] + g.Sig[4] * g.T1[2];
    U1[2] = g.Sig[2] * g.T1[0] + g.Sig[4] * g.T1[1] + g.Sig[5] * g.T1[2];
    float dT0[3], dT1[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        dT0[j] = 2.f * gA * U0[j] + gB * U1[j];
        dT1[j] = gB * U0[j] + 2.f * gC * U1[j];
    }
    float hB = 0.5f * gB;
    float dS[6];   // dL/dSigma as a symmetric matrix: 00 01 02 11 12 22
    dS[0] = gA * g.T0[0] * g.T0[0] + 2.f * hB * g.T0[0] * g.T1[0] + gC * g.T1[0] * g.T1[0];
    dS[1] = gA * g.T0[0] * g.T0[1] + hB * (g.T0[0] * g.T1[1] + g.T1[0] * g.T0[1]) + gC * g.T1[0] * g.T1[1];
    dS[2] = gA * g.T0[0] * g.T0[2] + hB * (g.T0[0] * g.T1[2] + g.T1[0] * g.T0[2]) + gC * g.T1[0] * g.T1[2];
    dS[3] = gA * g.T0[1] * g.T0[1] + 2.f * hB * g.T0[1] * g.T1[1] + gC * g.T1[1] * g.T1[1];
    dS[4] = gA * g.T0[1] * g.T0[2] + hB * (g.T0[1] * g.T1[2] + g.T1[1] * g.T0[2]) + gC * g.T1[1] * g.T1[2];
    dS[5] = gA * g.T0[2] * g.T0[2] + 2.f * hB * g.T0[2] * g.T1[2] + gC * g.T1[2] * g.T1[2];
    // rows of T depend on t through fx/tz and x/z; the mean through the pinhole
    const float* W = cam.R;
    float iz = 1.f / g.tz, iz2 = iz * iz, iz3 = iz2 * iz;
    float dT0W0 = dT0[0] * W[0] + dT0[1] * W[1] + dT0[2] * W[2];
    float dT0W2 = dT0[0] * W[6] + dT0[1] * W[7] + dT0[2] * W[8];
    float dT1W1 = dT1[0] * W[3] + dT1[1] * W[4] + dT1[2] * W[5];
    float dT1W2 = dT1[0] * W[6] + dT1[1] * W[7] + dT1[2] * W[8];
    float dtx = -cam.fx * iz2 * dT0W2 + d0.x * cam.fx * iz;
    float dty = -cam.fy * iz2 * dT1W2 + d0.y * cam.fy * iz;
    float dtz = -cam.fx * iz2 * dT0W0 + 2.f * cam.fx * g.tx * iz3 * dT0W2
              - cam.fy * iz2 * dT1W1 + 2.f * cam.fy * g.ty * iz3 * dT1W2
              - d0.x * cam.fx * g.tx * iz2 - d0.y * cam.fy * g.ty * iz2;
    gmu[0] += W[0] * dtx + W[3] * dty + W[6] * dtz;
    gmu[1] += W[1] * dtx + W[4] * dty + W[7] * dtz;
    gmu[2] += W[2] * dtx + W[5] * dty + W[8] * dtz;
    // Sigma = M M^T, M = R diag(s): dM = 2 dSigma M
    float Sf[9] = {dS[0], dS[1], dS[2], dS[1], dS[3], dS[4], dS[2], dS[4], dS[5]};
    float M[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) M[3 * i + j] = g.Rq[3 * i + j] * g.s[j];
    float dR[9];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float ds = 0.f;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            float dM = 2.f * (Sf[3 * i + 0] * M[0 + j] + Sf[3 * i + 1] * M[3 + j] + Sf[3 * i + 2] * M[6 + j]);
            ds += dM * g.Rq[3 * i + j];
            dR[3 * i + j] = dM * g.s[j];
        }
        gs[j] += ds * g.s[j];
    }
    // rotation partials w.r.t. the normalised quaternion, then the normalisation
    float qw = g.qn[0], qx = g.qn[1], qy = g.qn[2], qz = g.qn[3];
    float dqw = 2.f * (qz * (dR[3] - dR[1]) + qy * (dR[2] - dR[6]) + qx * (dR[7] - dR[5]));
    float dqx = 2.f * (qy * (dR[1] + dR[3]) + qz * (dR[2] + dR[6]) + qw * (dR[7] - dR[5])) - 4.f * qx * (dR[4] + dR[8]);
    float dqy = 2.f * (qx * (dR[1] + dR[3]) + qz * (dR[5] + dR[7]) + qw * (dR[2] - dR[6])) - 4.f * qy * (dR[0] + dR[8]);
    float dqz = 2.f * (qx * (dR[2] + dR[6]) + qy * (dR[5] + dR[7]) + qw * (dR[3] - dR[1])) - 4.f * qz * (dR[0] + dR[4]);
    float qd = dqw * qw + dqx * qx + dqy * qy + dqz * qz;
    gq[0] += (dqw - qw * qd) * g.qinv;
    gq[1] += (dqx - qx * qd) * g.qinv;
    gq[2] += (dqy - qy * qd) * g.qinv;
    gq[3] += (dqz - qz * qd) * g.qinv;
}

template <int DEG>
__global__ void __launch_bounds__(128, 4) k_project_bwd(GView x, const dg_camera* __restrict__ cams, dg_plan plan,
                                                        const uint2* __restrict__ rect,
                                                        const float4* __restrict__ drec, GView gr)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= plan.blk_off[plan.n_blocks]) return;
    int k = find_block(plan, c);
    int v0 = plan.blk_view_off[k], v1 = plan.blk_view_off[k + 1];
    float gmu[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, gs[3] = {0, 0, 0}, go = 0.f;
    const float4 mo = x.mo[c];
    const float3 mu = make_float3(mo.x, mo.y, mo.z);
    bool loaded = false, sh_written = false;
    float4 q = make_float4(0, 0, 0, 0), sc = make_float4(0, 0, 0, 0);
    float opac = 0.f;
    const float* __restrict__ shp = x.sh + c;
    float* __restrict__ gsh = gr.sh + c;
    for (int v = v0; v < v1; v++) {
        CamL cam;
        load_cam(cams, v, cam);
        int64_t r = cam.rec_off + (c - cam.gb);
        uint2 rr = rect[r];
        if ((rr.x & 0xFFFFu) == (rr.y & 0xFFFFu)) continue;     // culled in the forward
        if (!loaded) {
            q = x.quat[c];
            sc = x.scale[c];
            opac = 1.f / (1.f + __expf(-mo.w));
            loaded = true;
        }
        const float4 d0 = drec[3 * r + 0], d1 = drec[3 * r + 1], d2 = drec[3 * r + 2];
        {
            float f[3 * NK], gc[3], Y[NK];
#pragma unroll
            for (int j = 0; j < 3 * NK; j++) f[j] = __ldg(shp + (int64_t)j * x.ld);
            colour_adjoint<DEG>(cam, mu, opac, f, d1, d2, gmu, go, gc, Y);
#pragma unroll
            for (int kk = 0; kk < NK; kk++)
#pragma unroll
                for (int ch = 0; ch < 3; ch++) {
                    const int64_t o = (int64_t)(3 * kk + ch) * gr.ld;
                    const float val = gc[ch] * Y[kk];
                    gsh[o] = sh_written ? gsh[o] + val : val;
                }
            sh_written = true;
        }
        geometry_adjoint<DEG>(cam, mu, q, sc, d0, d1, plan.tile_w, plan.tile_h, gmu, gq, gs);
    }
    gr.mo[c] = make_float4(gmu[0], gmu[1], gmu[2], go);
    gr.quat[c] = make_float4(gq[0], gq[1], gq[2], gq[3]);
    gr.scale[c] = make_float4(gs[0], gs[1], gs[2], 0.f);
    if (!sh_written) {
#pragma unroll
        for (int j = 0; j < 3 * NK; j++) gsh[(int64_t)j * gr.ld] = 0.f;
    }
}

// ---- K8 + K9 fused: the projection adjoint feeding the x-step ------------------------
// For batches where every block has at most one view, each copy has at most
// one record, so its gradient is complete once that record's adjoint is
// done: the x-step (Adam + penalty, Eq. 8a / 12a) follows in the same CTA and
// the gradient never goes to memory.  A thread differentiates its copy, steps
// the copy's float4 fields, and leaves the colour gradient gc and SH basis Y
// in shared memory (dL/d f_{k,ch} = gc[ch] Y[k]); the CTA then steps its
// copies' SH planes with float4 accesses, four consecutive copies per thread
// (the same arithmetic as the separate kernels).
//
// The step can be taken in two parts, by CTA of kXsThreads consecutive
// copies: a CTA none of whose copies has a kept record has a zero rendering
// gradient, so its step depends only on x, m, v and the anchors and can run
// as soon as the projection has written the rectangles (k_xstep_idle or
// k_xstep_stream, alongside the compositing kernels); the CTAs with a kept
// record run after the compositing adjoint (k_xstep with PART = 2, or 3 over
// the list k_idle_groups made of them).  All take the step by the same device
// functions, so the result is the same as the one-part step.
constexpr int kXsThreads = 128;

// the record of copy c in its block's view, or -1 if the forward kept none
__device__ __forceinline__ int64_t copy_record(int64_t c, int64_t n, const dg_plan& plan,
                                               const dg_camera* __restrict__ cams, const uint2* __restrict__ rect,
                                               CamL& cam)
{
    if (c >= n || c >= plan.blk_off[plan.n_blocks]) return -1;
    const int k = find_block(plan, c);
    const int v0 = plan.blk_view_off[k];
    if (v0 >= plan.blk_view_off[k + 1]) return -1;
    load_cam(cams, v0, cam);
    const int64_t rr = cam.rec_off + (c - cam.gb);
    const uint2 t = rect[rr];
    return (t.x & 0xFFFFu) != (t.y & 0xFFFFu) ? rr : -1;
}

// Adam + penalty on copy c's float4 fields (mean, opacity logit), rotation,
// (log-scale, padding) with gradients gmu, go, gq, gs
// ZOut: where an unshared copy's stepped value also goes (the consensus's
// z = x for a global held by one block, taken here): z at the copy's global id
struct ZOut {
    GView z;
    const int32_t* gid;   // NULL: no store
};

__device__ __forceinline__ void step_fields(GView& x, GView& m, GView& v, const GView& an, int64_t c, bool s,
                                            const float4& mo, const float4& q, const float4& sc, const float* gmu,
                                            float go, const float* gq, const float* gs, const AdamArgs& a,
                                            float ic1, float ic2, const ZOut& zo)
{
    const int64_t zg = (zo.gid != nullptr && !s) ? (int64_t)zo.gid[c] : -1;
    {
        float xs[4] = {mo.x, mo.y, mo.z, mo.w}, gg[4] = {gmu[0], gmu[1], gmu[2], go};
        const float4 mm = m.mo[c], vv = v.mo[c];
        float ms[4] = {mm.x, mm.y, mm.z, mm.w}, vs[4] = {vv.x, vv.y, vv.z, vv.w};
        const float4 aa = s ? an.mo[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float as[4] = {aa.x, aa.y, aa.z, aa.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float rho = rho_of(a, i < 3 ? 0 : 4), lr = i < 3 ? a.lr[0] : a.lr[5];
            if (s) gg[i] = penalty_add(gg[i], rho, xs[i], as[i]);
            adam_scalar(xs[i], gg[i], ms[i], vs[i], lr, a.b1, a.b2, a.eps, ic1, ic2);
        }
        x.mo[c] = make_float4(xs[0], xs[1], xs[2], xs[3]);
        m.mo[c] = make_float4(ms[0], ms[1], ms[2], ms[3]);
        v.mo[c] = make_float4(vs[0], vs[1], vs[2], vs[3]);
        if (zg >= 0) zo.z.mo[zg] = make_float4(xs[0], xs[1], xs[2], xs[3]);
    }
    {
        const float4 mm = m.quat[c], vv = v.quat[c];
        float xs[4] = {q.x, q.y, q.z, q.w}, ms[4] = {mm.x, mm.y, mm.z, mm.w}, vs[4] = {vv.x, vv.y, vv.z, vv.w};
        const float4 aa = s ? an.quat[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float as[4] = {aa.x, aa.y, aa.z, aa.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            float g = gq[i];
            if (s) g = penalty_add(g, rho_of(a, 1), xs[i], as[i]);
            adam_scalar(xs[i], g, ms[i], vs[i], a.lr[1], a.b1, a.b2, a.eps, ic1, ic2);
        }
        x.quat[c] = make_float4(xs[0], xs[1], xs[2], xs[3]);
        m.quat[c] = make_float4(ms[0], ms[1], ms[2], ms[3]);
        v.quat[c] = make_float4(vs[0], vs[1], vs[2], vs[3]);
        if (zg >= 0) zo.z.quat[zg] = make_float4(xs[0], xs[1], xs[2], xs[3]);
    }
    {
        const float4 mm = m.scale[c], vv = v.scale[c];
        float xs[4] = {sc.x, sc.y, sc.z, sc.w}, ms[4] = {mm.x, mm.y, mm.z, mm.w}, vs[4] = {vv.x, vv.y, vv.z, vv.w};
        const float4 aa = s ? an.scale[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float as[4] = {aa.x, aa.y, aa.z, aa.w};
#pragma unroll
        for (int i = 0; i < 3; i++) {   // lane 3 is padding
            float g = gs[i];
            if (s) g = penalty_add(g, rho_of(a, 2), xs[i], as[i]);
            adam_scalar(xs[i], g, ms[i], vs[i], a.lr[2], a.b1, a.b2, a.eps, ic1, ic2);
        }
        x.scale[c] = make_float4(xs[0], xs[1], xs[2], xs[3]);
        m.scale[c] = make_float4(ms[0], ms[1], ms[2], ms[3]);
        v.scale[c] = make_float4(vs[0], vs[1], vs[2], vs[3]);
        if (zg >= 0) zo.z.scale[zg] = make_float4(xs[0], xs[1], xs[2], xs[3]);
    }
}

// The SH planes of the CTA's copies c0 .. c0 + kXsThreads - 1: thread = (plane
// group tid / 32, quad tid % 32 of four copies), PB planes per batch and
// thread with all loads of a batch issued before its stores.  The gradient of
// plane j (channel j % 3, coefficient j / 3) at copy i of the quad is
// gc[ch][i] Y[k][i] from shared memory, or 0 without a rendering gradient
// (ZERO).
template <int NK, int PB, bool ZERO>
__device__ __forceinline__ void step_planes(GView& x, GView& m, GView& v, const GView& an,
                                            const uint8_t* __restrict__ shared, int64_t c0, const float* s_gc,
                                            const float* s_Y, const AdamArgs& a, float ic1, float ic2,
                                            const ZOut& zo)
{
    const int tid = threadIdx.x;
    const int quad = tid & 31;
    const int64_t cq = c0 + 4 * quad;
    if (cq >= x.ld) return;                       // the quad lies beyond the planes' stride
    bool act[4], sh[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        act[i] = cq + i < x.n;
        sh[i] = act[i] && shared != nullptr && shared[cq + i] != 0;
    }
    const bool any_sh = sh[0] || sh[1] || sh[2] || sh[3];
    int64_t zg[4];                                // global ids of the quad's unshared copies (-1: none)
#pragma unroll
    for (int i = 0; i < 4; i++) zg[i] = (zo.gid != nullptr && act[i] && !sh[i]) ? (int64_t)zo.gid[cq + i] : -1;
    constexpr int G = kXsThreads / 32;          // plane groups (4)
    for (int j0 = tid >> 5; j0 < 3 * NK; j0 += G * PB) {
        float4 xv[PB], mv[PB], vv[PB], av[PB];
#pragma unroll
        for (int b = 0; b < PB; b++) {
            const int j = j0 + b * G;
            if (j >= 3 * NK) break;
            const int64_t u = ((int64_t)j * x.ld + cq) >> 2;
            xv[b] = reinterpret_cast<const float4*>(x.sh)[u];
            mv[b] = reinterpret_cast<const float4*>(m.sh)[u];
            vv[b] = reinterpret_cast<const float4*>(v.sh)[u];
            av[b] = any_sh ? reinterpret_cast<const float4*>(an.sh)[u] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int b = 0; b < PB; b++) {
            const int j = j0 + b * G;
            if (j >= 3 * NK) break;
            const float lr = j < 3 ? a.lr[3] : a.lr[4];
            float gq4[4] = {0.f, 0.f, 0.f, 0.f};
            if (!ZERO) {
                // the quad's four colour gradients and basis values, one 16-byte load each
                const float4 gc4 = *reinterpret_cast<const float4*>(&s_gc[(j % 3) * kXsThreads + 4 * quad]);
                const float4 y4 = *reinterpret_cast<const float4*>(&s_Y[(j / 3) * kXsThreads + 4 * quad]);
                gq4[0] = gc4.x * y4.x; gq4[1] = gc4.y * y4.y; gq4[2] = gc4.z * y4.z; gq4[3] = gc4.w * y4.w;
            }
            float xs[4] = {xv[b].x, xv[b].y, xv[b].z, xv[b].w}, ms[4] = {mv[b].x, mv[b].y, mv[b].z, mv[b].w};
            float vs[4] = {vv[b].x, vv[b].y, vv[b].z, vv[b].w};
            const float as[4] = {av[b].x, av[b].y, av[b].z, av[b].w};
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if (!act[i]) continue;
                float g = gq4[i];
                if (sh[i]) g = penalty_add(g, rho_of(a, 3), xs[i], as[i]);
                adam_scalar(xs[i], g, ms[i], vs[i], lr, a.b1, a.b2, a.eps, ic1, ic2);
            }
            const int64_t u = ((int64_t)j * x.ld + cq) >> 2;
            reinterpret_cast<float4*>(x.sh)[u] = make_float4(xs[0], xs[1], xs[2], xs[3]);
            reinterpret_cast<float4*>(m.sh)[u] = make_float4(ms[0], ms[1], ms[2], ms[3]);
            reinterpret_cast<float4*>(v.sh)[u] = make_float4(vs[0], vs[1], vs[2], vs[3]);
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (zg[i] >= 0) zo.z.sh[(int64_t)j * zo.z.ld + zg[i]] = xs[i];
        }
    }
}

// The fused adjoint + step of the group of kXsThreads copies from c0.  CHECK:
// first find out whether a copy of the group has a kept record and leave the
// group (uniformly) if none has: k_xstep_idle or k_xstep_stream steps it.
template <int DEG, bool CHECK>
__device__ __forceinline__ void xstep_group(int64_t c0, GView& x, GView& m, GView& v, const GView& an,
                                            const uint8_t* __restrict__ shared,
                                            const dg_camera* __restrict__ cams, const dg_plan& plan,
                                            const uint2* __restrict__ rect, const float4* __restrict__ drec,
                                            const AdamArgs& a, float ic1, float ic2, const ZOut& zo,
                                            float* s_gc, float* s_Y)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    const int tid = threadIdx.x;
    const int64_t c = c0 + tid;
    CamL cam;
    const int64_t r = copy_record(c, x.n, plan, cams, rect, cam);
    if (CHECK && !__syncthreads_or(r >= 0)) return;    // uniform
    float gc[3] = {0.f, 0.f, 0.f}, Y[NK];
#pragma unroll
    for (int kk = 0; kk < NK; kk++) Y[kk] = 0.f;
    if (c < x.n) {
        const bool s = shared != nullptr && shared[c] != 0;
        const float4 mo = x.mo[c];
        const float3 mu = make_float3(mo.x, mo.y, mo.z);
        float gmu[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, gs[3] = {0, 0, 0}, go = 0.f;
        const float4 q = x.quat[c], sc = x.scale[c];
        if (r >= 0) {
            {
                float f[3 * NK];
#pragma unroll
                for (int j = 0; j < 3 * NK; j++) f[j] = x.sh[(int64_t)j * x.ld + c];
                colour_adjoint<DEG>(cam, mu, 1.f / (1.f + __expf(-mo.w)), f, drec[3 * r + 1], drec[3 * r + 2], gmu,
                                    go, gc, Y);
            }
            geometry_adjoint<DEG>(cam, mu, q, sc, drec[3 * r + 0], drec[3 * r + 1], plan.tile_w, plan.tile_h, gmu,
                                  gq, gs);
        }
        step_fields(x, m, v, an, c, s, mo, q, sc, gmu, go, gq, gs, a, ic1, ic2, zo);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ch++) s_gc[ch * kXsThreads + tid] = gc[ch];
#pragma unroll
    for (int kk = 0; kk < NK; kk++) s_Y[kk * kXsThreads + tid] = Y[kk];
    __syncthreads();
    step_planes<NK, 6, false>(x, m, v, an, shared, c0, s_gc, s_Y, a, ic1, ic2, zo);
}

// PART 0: every CTA; PART 2: only the CTAs with at least one kept record;
// PART 3: CTA b steps the group alist[-b] of those k_idle_groups listed as
// holding a kept record (the list grows down from alist[0]), and the CTAs
// past the list's length actr[0] leave at once: they all come after the
// stepping CTAs, instead of each taking its slot among them to find out.
template <int DEG, int PART>
__global__ void __launch_bounds__(kXsThreads, 4) k_xstep(GView x, GView m, GView v, GView an,
                                                        const uint8_t* __restrict__ shared,
                                                        const dg_camera* __restrict__ cams, dg_plan plan,
                                                        const uint2* __restrict__ rect,
                                                        const float4* __restrict__ drec, AdamArgs a,
                                                        const int32_t* __restrict__ dev_step, ZOut zo,
                                                        const int32_t* __restrict__ alist,
                                                        const uint32_t* __restrict__ actr)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    __shared__ __align__(16) float s_gc[3 * kXsThreads];
    __shared__ __align__(16) float s_Y[NK * kXsThreads];
    int64_t grp = blockIdx.x;
    if (PART == 3) {
        if (blockIdx.x >= *actr) return;               // uniform
        grp = alist[-(int64_t)blockIdx.x];
        if (grp < 0 || grp * kXsThreads >= x.n) return;   // a list not made for these copies
    }
    float ic1, ic2;
    bias_corr(a, dev_step, ic1, ic2);
    xstep_group<DEG, PART == 2>(grp * kXsThreads, x, m, v, an, shared, cams, plan, rect, drec, a, ic1, ic2, zo,
                                s_gc, s_Y);
}

// the groups of k_xstep<PART 2>'s complement: no copy with a kept record, so
// a zero rendering gradient (the penalty alone on shared copies).  A
// grid-stride loop over the groups of kXsThreads copies, so that a small
// grid (a CTA or two per SM) can run alongside the compositing kernels
// without taking their registers.
template <int DEG>
__global__ void __launch_bounds__(kXsThreads, 6) k_xstep_idle(GView x, GView m, GView v, GView an,
                                                             const uint8_t* __restrict__ shared,
                                                             const dg_camera* __restrict__ cams, dg_plan plan,
                                                             const uint2* __restrict__ rect, AdamArgs a,
                                                             const int32_t* __restrict__ dev_step, ZOut zo)
{
    constexpr int NK = (DEG + 1) * (DEG + 1);
    const int tid = threadIdx.x;
    float ic1, ic2;
    bias_corr(a, dev_step, ic1, ic2);
    const int64_t n_groups = (x.n + kXsThreads - 1) / kXsThreads;
    for (int64_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
        const int64_t c0 = grp * kXsThreads, c = c0 + tid;
        bool kept = false;                          // the test of copy_record, without the camera
        if (c < x.n && c < plan.blk_off[plan.n_blocks]) {
            const int k = find_block(plan, c);
            const int v0 = plan.blk_view_off[k];
            if (v0 < plan.blk_view_off[k + 1]) {
                const uint2 t = rect[__ldg(&cams[v0].rec_off) + (c - __ldg(&cams[v0].gauss_begin))];
                kept = (t.x & 0xFFFFu) != (t.y & 0xFFFFu);
            }
        }
        if (__syncthreads_or(kept)) continue;       // uniform: the group is stepped by k_xstep<PART 2>
        if (c < x.n) {
            const bool s = shared != nullptr && shared[c] != 0;
            const float zero[4] = {0.f, 0.f, 0.f, 0.f};
            step_fields(x, m, v, an, c, s, x.mo[c], x.quat[c], x.scale[c], zero, 0.f, zero, zero, a, ic1, ic2,
                        zo);
        }
        step_planes<NK, 2, true>(x, m, v, an, shared, c0, nullptr, nullptr, a, ic1, ic2, zo);
    }
}

// ---- part 1 streamed through shared memory -------------------------------------------
// The groups without a kept record are listed first (k_idle_groups), then
// stepped by a few persistent CTAs (one per SM by default) that take groups
// in a fixed order.  A group's x, m, v and anchors pass through a ring of
// shared memory by cp.async in segments of 2 KB per array -- the three
// float4 field rows of its 128 copies, then its SH planes four at a time --
// two segments to a pipeline unit.  A thread copies and later steps the same
// 16-byte chunk of every segment, so the ring needs no barrier, and
// kStStages - 1 units (32 KB a CTA) stay in flight while one is stepped:
// enough for HBM speed from one CTA per SM, in registers and shared memory
// that the compositing adjoint leaves free, so this part runs beside it.
// Each element's arithmetic is k_xstep_idle's, so the result is the same bit
// for bit.
constexpr int kStThreads = 128;
#ifndef DG_XSTEP_STAGES
#define DG_XSTEP_STAGES 3   // ring slots of one unit (16 KB each)
#endif
constexpr int kStStages = DG_XSTEP_STAGES;
static_assert(kStStages >= 2, "the ring needs a unit in flight beside the one stepped");

// one warp per group of kXsThreads copies: appends the group to list if none
// of its copies has a kept record, ctr[0] counting them, and else to the
// list's other end (list[n_groups - 1], list[n_groups - 2], ...), ctr[1]
// counting those; each group is listed once, so the two never meet (the
// order within each is unspecified)
__global__ void __launch_bounds__(256) k_idle_groups(int64_t n, int64_t n_groups, const dg_camera* __restrict__ cams,
                                                     dg_plan plan, const uint2* __restrict__ rect,
                                                     int32_t* __restrict__ list, uint32_t* __restrict__ ctr)
{
    const int64_t grp = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (grp * kXsThreads >= n) return;          // uniform over the warp
    bool kept = false;
#pragma unroll
    for (int i = 0; i < kXsThreads / 32; i++) {
        const int64_t c = grp * kXsThreads + lane + 32 * i;
        if (c < n && c < plan.blk_off[plan.n_blocks]) {
            const int k = find_block(plan, c);
            const int v0 = plan.blk_view_off[k];
            if (v0 < plan.blk_view_off[k + 1]) {
                const uint2 t = rect[__ldg(&cams[v0].rec_off) + (c - __ldg(&cams[v0].gauss_begin))];
                kept = kept || (t.x & 0xFFFFu) != (t.y & 0xFFFFu);
            }
        }
    }
    const bool any = __any_sync(0xffffffffu, kept);
    if (lane == 0) {
        if (any) list[n_groups - 1 - (int64_t)atomicAdd(ctr + 1, 1u)] = (int32_t)grp;
        else list[atomicAdd(ctr, 1u)] = (int32_t)grp;
    }
}

// what a thread needs of its group: the copy c0 + tid of the field rows and
// the quad c0 + 4 (tid % 32) .. + 3 of the SH planes.  Loaded raw a group
// ahead (StRaw: the loads only, so that nothing waits on them), decoded
// where first used (StMeta).
struct StRaw {
    int64_t c0;       // first copy of the group; -1: none (past the end of the list)
    uint32_t fs, qs;  // shared flag of the copy; of the quad's copies, a byte each
    int32_t fg;       // global id of the copy
    int32_t qg[4];    // of the quad's copies
};

struct StMeta {
    int64_t c0;       // as in StRaw
    int64_t fo;       // float4 index of the copy in a field row: c0 + tid
    int64_t po;       // float4 index of the quad in plane tid / 32 (segment 3; + ld per later segment)
    uint32_t bits;    // 1: copy active (c < n), 2: copy shared; 1 << (4 + i): quad copy i active,
                      // 1 << (8 + i): shared; 1 << 12: quad inside the planes (cq < ld); 1 << 13: every copy
                      // of the group active (then the rest of the bits hold for the copy and the quad alike)
    int32_t zf;       // global id of an unshared copy for the z store, else -1
    int32_t zq[4];    // the same for the quad's copies
};
constexpr uint32_t kStQuadIn = 1u << 12, kStFull = 1u << 13;

__device__ __forceinline__ void st_load(StRaw& R, int64_t c0, const GView& x, const uint8_t* __restrict__ shared,
                                        const ZOut& zo)
{
    const int tid = threadIdx.x;
    R.c0 = c0;
    R.fs = R.qs = 0;
    R.fg = -1;
#pragma unroll
    for (int i = 0; i < 4; i++) R.qg[i] = -1;
    if (c0 < 0) return;
    const int64_t c = c0 + tid, cq = c0 + 4 * (tid & 31);
    if (c < x.n) {
        if (shared != nullptr) R.fs = shared[c];
        if (zo.gid != nullptr) R.fg = zo.gid[c];
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (cq + i >= x.n) continue;
        if (shared != nullptr) R.qs |= (uint32_t)shared[cq + i] << (8 * i);
        if (zo.gid != nullptr) R.qg[i] = zo.gid[cq + i];
    }
}

__device__ __forceinline__ void st_decode(StMeta& M, const StRaw& R, const GView& x, const ZOut& zo)
{
    const int tid = threadIdx.x;
    M.c0 = R.c0;
    M.bits = 0;
    M.zf = -1;
#pragma unroll
    for (int i = 0; i < 4; i++) M.zq[i] = -1;
    M.fo = M.po = 0;
    if (R.c0 < 0) return;
    const int64_t c = R.c0 + tid, cq = R.c0 + 4 * (tid & 31);
    M.fo = c;
    M.po = ((int64_t)(tid >> 5) * x.ld + cq) >> 2;
    if (cq < x.ld) M.bits |= kStQuadIn;
    if (R.c0 + kXsThreads <= x.n) M.bits |= kStFull;
    if (c < x.n) {
        const bool s = R.fs != 0;
        M.bits |= 1u | (s ? 2u : 0u);
        if (zo.gid != nullptr && !s) M.zf = R.fg;
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (cq + i >= x.n) continue;
        const bool s = ((R.qs >> (8 * i)) & 0xFFu) != 0;
        M.bits |= (1u << (4 + i)) | (s ? 1u << (8 + i) : 0u);
        if (zo.gid != nullptr && !s) M.zq[i] = R.qg[i];
    }
}

__device__ __forceinline__ void st_copy16(float4* dst, const float4* src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// The float4 index (within the row or planes st_row returns) of the chunk
// of segment SEG that this thread copies and steps, or -1 for none.
// Segments 0..2: the field rows (mean and opacity, rotation, scale), one
// copy per thread; from 3 on: SH planes 4 (SEG - 3) .. + 3, a plane per warp
// and a quad of copies per lane.
template <int SEG, int NP>
__device__ __forceinline__ int64_t st_chunk(const StMeta& M, const GView& x)
{
    if (M.c0 < 0) return -1;
    if (SEG < 3) return (M.bits & 1u) ? M.fo : -1;
    if (4 * (SEG - 3) + 3 >= NP && 4 * (SEG - 3) + (int)(threadIdx.x >> 5) >= NP)
        return -1;                                       // the last segment may hold fewer planes
    return (M.bits & kStQuadIn) ? M.po + (int64_t)(SEG - 3) * x.ld : -1;
}

template <int SEG>
__device__ __forceinline__ float4* st_row(const GView& g)
{
    return SEG == 0 ? g.mo : SEG == 1 ? g.quat : SEG == 2 ? g.scale : reinterpret_cast<float4*>(g.sh);
}

// producer: this thread's chunk of x, m, v (and the anchors where its copies
// are shared) of segment SEG into the ring slot s (segments past the
// group's last have none)
template <int SEG, int NSEG, int NP>
__device__ __forceinline__ void st_issue(float4* s, const StMeta& M, const GView& x, const GView& m,
                                         const GView& v, const GView& an)
{
    if constexpr (SEG < NSEG) {
        const int64_t u = st_chunk<SEG, NP>(M, x);
        if (u < 0) return;
        const int tid = threadIdx.x;
        st_copy16(s + tid, st_row<SEG>(x) + u);
        st_copy16(s + kStThreads + tid, st_row<SEG>(m) + u);
        st_copy16(s + 2 * kStThreads + tid, st_row<SEG>(v) + u);
        const bool need_a = SEG < 3 ? (M.bits & 2u) != 0 : ((M.bits >> 8) & 15u) != 0;
        if (need_a) st_copy16(s + 3 * kStThreads + tid, st_row<SEG>(an) + u);
    }
}

struct Rho5 {
    float r[5];   // the penalties of the five groups, read once per CTA
};

// the per-CTA constants of the paired step: Adam's, and (-lr, -lr) and
// (rho, rho) of each parameter class of a segment's float4
struct StPair {
    AdamPair P;
    f32x2 nlr_p, nlr_po, nlr_q, nlr_s, nlr_dc, nlr_rest;   // p, (p, o), q, s, SH DC, SH rest
    f32x2 rho_p, rho_po, rho_q, rho_s, rho_f;
};

__device__ __forceinline__ StPair st_pair_args(const AdamArgs& a, const Rho5& rh, float ic1, float ic2)
{
    StPair S;
    S.P = adam_pair_args(a.b1, a.b2, a.eps, ic1, ic2);
    S.nlr_p = f2_pack(-a.lr[0], -a.lr[0]);
    S.nlr_po = f2_pack(-a.lr[0], -a.lr[5]);
    S.nlr_q = f2_pack(-a.lr[1], -a.lr[1]);
    S.nlr_s = f2_pack(-a.lr[2], -a.lr[2]);
    S.nlr_dc = f2_pack(-a.lr[3], -a.lr[3]);
    S.nlr_rest = f2_pack(-a.lr[4], -a.lr[4]);
    S.rho_p = f2_pack(rh.r[0], rh.r[0]);
    S.rho_po = f2_pack(rh.r[0], rh.r[4]);
    S.rho_q = f2_pack(rh.r[1], rh.r[1]);
    S.rho_s = f2_pack(rh.r[2], rh.r[2]);
    S.rho_f = f2_pack(rh.r[3], rh.r[3]);
    return S;
}

// two parameters (lanes of x2) of a chunk by the paired step: the penalty
// rho (x - a) + 0 where the copy is shared (s0, s1), else a zero gradient
__device__ __forceinline__ void st_pair_step(f32x2& x2, f32x2& m2, f32x2& v2, f32x2 a2, bool s0, bool s1,
                                             f32x2 rho2, f32x2 nlr2, const AdamPair& P)
{
    float p0, p1;
    f2_unpack(f2_fma(rho2, f2_sub(x2, a2), f2_pack(0.f, 0.f)), p0, p1);
    adam_pair(x2, f2_pack(s0 ? p0 : 0.f, s1 ? p1 : 0.f), m2, v2, nlr2, P);
}

// consumer: the Adam + penalty step of this thread's chunk of segment SEG
// from ring slot s, written back to x, m, v (and z for unshared copies).
// A group whose copies are all active takes the paired step with no
// per-element select; the group holding the last copies steps each
// element as k_xstep_idle does and keeps or discards it by a select (a copy
// past n keeps its value).  The scale's padding lane is never stepped.
template <int SEG, int NSEG, int NP>
__device__ __forceinline__ void st_step(const float4* s, const StMeta& M, GView& x, GView& m, GView& v,
                                        const AdamArgs& a, const Rho5& rh, const StPair& SP, float ic1,
                                        float ic2, const ZOut& zo)
{
    if constexpr (SEG < NSEG) {
        const int64_t u = st_chunk<SEG, NP>(M, x);
        if (u < 0) return;
        const int tid = threadIdx.x;
        const float4 X = s[tid], Mo = s[kStThreads + tid], V = s[2 * kStThreads + tid];
        const float4 A = s[3 * kStThreads + tid];   // read only for shared copies (loaded then)
        float xs[4], ms[4], vs[4];
        // plane of this thread's chunk, and whether it is an SH DC plane
        const int j = 4 * (SEG - 3) + (tid >> 5);
        const bool dc = SEG == 3 && j < 3;
        if (M.bits & kStFull) {
            bool sh[4];
#pragma unroll
            for (int i = 0; i < 4; i++) sh[i] = SEG < 3 ? (M.bits & 2u) != 0 : ((M.bits >> (8 + i)) & 1u) != 0;
            f32x2 x01 = f2_pack(X.x, X.y), m01 = f2_pack(Mo.x, Mo.y), v01 = f2_pack(V.x, V.y);
            f32x2 x23 = f2_pack(X.z, X.w), m23 = f2_pack(Mo.z, Mo.w), v23 = f2_pack(V.z, V.w);
            const f32x2 a01 = f2_pack(A.x, A.y), a23 = f2_pack(A.z, A.w);
            f32x2 rho01, rho23, nlr01, nlr23;
            if (SEG == 0) {
                rho01 = SP.rho_p; rho23 = SP.rho_po; nlr01 = SP.nlr_p; nlr23 = SP.nlr_po;
            } else if (SEG == 1) {
                rho01 = rho23 = SP.rho_q; nlr01 = nlr23 = SP.nlr_q;
            } else if (SEG == 2) {
                rho01 = rho23 = SP.rho_s; nlr01 = nlr23 = SP.nlr_s;
            } else {
                rho01 = rho23 = SP.rho_f;
                nlr01 = nlr23 = dc ? SP.nlr_dc : SP.nlr_rest;
            }
            st_pair_step(x01, m01, v01, a01, sh[0], sh[1], rho01, nlr01, SP.P);
            f2_unpack(x01, xs[0], xs[1]); f2_unpack(m01, ms[0], ms[1]); f2_unpack(v01, vs[0], vs[1]);
            if (SEG == 2) {                              // the scale: z stepped alone, w (padding) kept
                xs[2] = X.z; ms[2] = Mo.z; vs[2] = V.z;
                const float g = sh[2] ? penalty_add(0.f, rh.r[2], X.z, A.z) : 0.f;
                adam_scalar(xs[2], g, ms[2], vs[2], a.lr[2], a.b1, a.b2, a.eps, ic1, ic2);
                xs[3] = X.w; ms[3] = Mo.w; vs[3] = V.w;
            } else {
                st_pair_step(x23, m23, v23, a23, sh[2], sh[3], rho23, nlr23, SP.P);
                f2_unpack(x23, xs[2], xs[3]); f2_unpack(m23, ms[2], ms[3]); f2_unpack(v23, vs[2], vs[3]);
            }
        } else {
            const float x0[4] = {X.x, X.y, X.z, X.w}, m0[4] = {Mo.x, Mo.y, Mo.z, Mo.w};
            const float v0[4] = {V.x, V.y, V.z, V.w}, as[4] = {A.x, A.y, A.z, A.w};
#pragma unroll
            for (int i = 0; i < 4; i++) {
                // step, penalty and learning rate of element i (constants of SEG and i)
                bool step;
                float rho, lr;
                if (SEG == 0) {
                    step = (M.bits & 1u) != 0;
                    rho = rh.r[i < 3 ? 0 : 4];
                    lr = i < 3 ? a.lr[0] : a.lr[5];
                } else if (SEG == 1) {
                    step = (M.bits & 1u) != 0;
                    rho = rh.r[1];
                    lr = a.lr[1];
                } else if (SEG == 2) {
                    step = i < 3 && (M.bits & 1u) != 0;
                    rho = rh.r[2];
                    lr = a.lr[2];
                } else {
                    step = ((M.bits >> (4 + i)) & 1u) != 0;
                    rho = rh.r[3];
                    lr = dc ? a.lr[3] : a.lr[4];
                }
                const bool sh = SEG < 3 ? (M.bits & 2u) != 0 : ((M.bits >> (8 + i)) & 1u) != 0;
                const float g = sh ? penalty_add(0.f, rho, x0[i], as[i]) : 0.f;
                float xi = x0[i], mi = m0[i], vi = v0[i];
                adam_scalar(xi, g, mi, vi, lr, a.b1, a.b2, a.eps, ic1, ic2);
                xs[i] = step ? xi : x0[i];
                ms[i] = step ? mi : m0[i];
                vs[i] = step ? vi : v0[i];
            }
        }
        st_row<SEG>(x)[u] = make_float4(xs[0], xs[1], xs[2], xs[3]);
        st_row<SEG>(m)[u] = make_float4(ms[0], ms[1], ms[2], ms[3]);
        st_row<SEG>(v)[u] = make_float4(vs[0], vs[1], vs[2], vs[3]);
        if (SEG < 3) {
            if (M.zf >= 0) st_row<SEG>(zo.z)[M.zf] = make_float4(xs[0], xs[1], xs[2], xs[3]);
        } else {
            float* zj = zo.z.sh + (int64_t)j * zo.z.ld;
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (M.zq[i] >= 0) zj[M.zq[i]] = xs[i];
        }
    }
}

template <int N>
__device__ __forceinline__ void st_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ void st_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// The pipeline's unit is two segments (one commit group, a ring slot of
// 2 x 4 x kStThreads float4): unit k of a CTA's sequence lives in slot
// k mod NS, and a group's first unit in slot `base`.
template <int NS>
__device__ __forceinline__ float4* st_slot(float4* ring, int base, int k)
{
    return ring + ((base + k) % NS) * 8 * kStThreads;
}

template <int U, int NSEG, int NP>
__device__ __forceinline__ void st_issue_unit(float4* s, const StMeta& M, const GView& x, const GView& m,
                                              const GView& v, const GView& an)
{
    st_issue<2 * U, NSEG, NP>(s, M, x, m, v, an);
    st_issue<2 * U + 1, NSEG, NP>(s + 4 * kStThreads, M, x, m, v, an);
    st_commit();
}

// unit U of a group: the producer's unit U + NS - 1 (of this group, or past
// its last unit the next group's, with nm -- decoded from its raw loads
// just before its first use), then the consumer's unit U
template <int U, int NU, int NSEG, int NS, int NP>
__device__ __forceinline__ void st_unit(float4* ring, int base, const StMeta& cm, StMeta& nm, const StRaw& nr,
                                        GView& x, GView& m, GView& v, const GView& an, const AdamArgs& a,
                                        const Rho5& rh, const StPair& sp, float ic1, float ic2, const ZOut& zo)
{
    constexpr int P = U + NS - 1;
    if constexpr (P < NU) {
        st_issue_unit<P, NSEG, NP>(st_slot<NS>(ring, base, P), cm, x, m, v, an);
    } else {
        if constexpr (P == NU) st_decode(nm, nr, x, zo);
        st_issue_unit<P - NU, NSEG, NP>(st_slot<NS>(ring, base, P), nm, x, m, v, an);
    }
    st_wait<NS - 1>();
    float4* s = st_slot<NS>(ring, base, U);
    st_step<2 * U, NSEG, NP>(s, cm, x, m, v, a, rh, sp, ic1, ic2, zo);
    st_step<2 * U + 1, NSEG, NP>(s + 4 * kStThreads, cm, x, m, v, a, rh, sp, ic1, ic2, zo);
    if constexpr (U + 1 < NU)
        st_unit<U + 1, NU, NSEG, NS, NP>(ring, base, cm, nm, nr, x, m, v, an, a, rh, sp, ic1, ic2, zo);
}

template <int U, int NS, int NSEG, int NP>
__device__ __forceinline__ void st_prologue(float4* ring, const StMeta& cm, const GView& x, const GView& m,
                                            const GView& v, const GView& an)
{
    if constexpr (U < NS - 1) {
        st_issue_unit<U, NSEG, NP>(ring + U * 8 * kStThreads, cm, x, m, v, an);
        st_prologue<U + 1, NS, NSEG, NP>(ring, cm, x, m, v, an);
    }
}

// the persistent streamed part 1 over list[0 .. ctr[0]) (ctr[0] written by
// k_idle_groups): CTA b takes the entries b, b + G, b + 2 G, ... (G CTAs),
// one group per iteration with its NU units unrolled.  Producer and consumer
// are the same threads, the producer NS - 1 units ahead (NS <= NU), so its
// last NS - 1 units of an iteration are the next group's first.  The next
// group's metadata is loaded raw a group ahead and the list entry after it
// two, so no load is waited for.
template <int DEG>
__global__ void __launch_bounds__(kStThreads) k_xstep_stream(GView x, GView m, GView v, GView an,
                                                            const uint8_t* __restrict__ shared,
                                                            const int32_t* __restrict__ list,
                                                            const uint32_t* __restrict__ ctr, AdamArgs a,
                                                            const int32_t* __restrict__ dev_step, ZOut zo)
{
    constexpr int NK = (DEG + 1) * (DEG + 1), NP = 3 * NK, NSEG = 3 + (NP + 3) / 4, NU = (NSEG + 1) / 2;
    constexpr int NS = kStStages < NU ? kStStages : NU;
    extern __shared__ __align__(16) float4 s_ring[];   // [NS][2 segments][x, m, v, anchor][kStThreads]
    float ic1, ic2;
    bias_corr(a, dev_step, ic1, ic2);
    Rho5 rh;
#pragma unroll
    for (int k = 0; k < 5; k++) rh.r[k] = rho_of(a, k);
    const StPair sp = st_pair_args(a, rh, ic1, ic2);
    const int64_t n_groups = (x.n + kXsThreads - 1) / kXsThreads;
    const uint32_t n_list = (uint32_t)min((int64_t)ctr[0], n_groups), G = gridDim.x;
    uint32_t li = blockIdx.x;
    // an entry outside the copies (a list not made for them) ends the CTA's walk
    auto entry = [&](uint32_t i) {
        const int64_t g = i < n_list ? (int64_t)list[i] : (int64_t)-1;
        return g >= 0 && g < n_groups ? g * kXsThreads : (int64_t)-1;
    };
    StRaw nr;
    StMeta cm, nm;
    st_load(nr, entry(li), x, shared, zo);
    st_decode(cm, nr, x, zo);
    st_load(nr, entry(li + G), x, shared, zo);
    int64_t c0_ahead = entry(li + 2 * G);
    li += 3 * G;
    st_prologue<0, NS, NSEG, NP>(s_ring, cm, x, m, v, an);
    int base = 0;
#pragma unroll 1
    while (cm.c0 >= 0) {
        st_unit<0, NU, NSEG, NS, NP>(s_ring, base, cm, nm, nr, x, m, v, an, a, rh, sp, ic1, ic2, zo);
        base = (base + NU) % NS;
        cm = nm;
        st_load(nr, c0_ahead, x, shared, zo);
        c0_ahead = entry(li);
        li += G;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int DEG>
constexpr size_t st_smem_bytes()
{
    constexpr int NK = (DEG + 1) * (DEG + 1), NSEG = 3 + (3 * NK + 3) / 4, NU = (NSEG + 1) / 2;
    return (size_t)(kStStages < NU ? kStStages : NU) * 8 * kStThreads * sizeof(float4);
}

// once per device (ensure_init): the ring's dynamic shared memory, and the
// shared-memory carveout at its maximum so that a CTA fits beside the
// compositing adjoint's
int xstep_stream_init()
{
#define DG_ST_INIT(D)                                                                                   \
    if (cudaFuncSetAttribute(k_xstep_stream<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                             (int)st_smem_bytes<D>()) != cudaSuccess ||                                 \
        cudaFuncSetAttribute(k_xstep_stream<D>, cudaFuncAttributePreferredSharedMemoryCarveout,       \
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)                       \
        return DG_ERR_CUDA;
    DG_ST_INIT(0) DG_ST_INIT(1) DG_ST_INIT(2) DG_ST_INIT(3)
#undef DG_ST_INIT
    return DG_OK;
}

// workspace of the listed steps: two counters (16 bytes), then the list of
// one entry per group (the groups without a kept record from the front, the
// others from the back)
size_t xstep_stream_ws_bytes(int64_t n)
{
    return 16 + 4 * (size_t)((n + kXsThreads - 1) / kXsThreads);
}

// both lists of k_idle_groups into ws
int launch_xstep_groups(const dg_gaussians* x, const dg_camera* cams, const dg_plan& plan, const uint2* rect,
                        void* ws, cudaStream_t st)
{
    if (x->n == 0) return DG_OK;
    uint32_t* ctr = static_cast<uint32_t*>(ws);
    int32_t* list = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + 16);
    const int64_t n_groups = (x->n + kXsThreads - 1) / kXsThreads;
    if (cudaMemsetAsync(ctr, 0, 8, st) != cudaSuccess) return DG_ERR_CUDA;
    k_idle_groups<<<(unsigned)((n_groups + 7) / 8), 256, 0, st>>>(x->n, n_groups, cams, plan, rect, list, ctr);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// build_lists: list the groups first (launch_xstep_groups); else step the
// list an earlier launch_xstep_groups left in ws
int launch_xstep_stream(int ctas, dg_gaussians* x, dg_gaussians* m, dg_gaussians* v, const dg_gaussians* anchor,
                        const uint8_t* shared, const dg_camera* cams, const dg_plan& plan, const uint2* rect,
                        const AdamArgs& a, const int32_t* dev_step, dg_gaussians* z, const int32_t* gid, void* ws,
                        bool build_lists, cudaStream_t st)
{
    if (x->n == 0) return DG_OK;
    GView xv = gview(x), mv = gview(m), vv = gview(v);
    GView av = anchor ? gview(anchor) : xv;
    ZOut zo;
    zo.z = z ? gview(z) : xv;
    zo.gid = z ? gid : nullptr;
    uint32_t* ctr = static_cast<uint32_t*>(ws);
    int32_t* list = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + 16);
    if (build_lists) {
        const int rc = launch_xstep_groups(x, cams, plan, rect, ws, st);
        if (rc != DG_OK) return rc;
    }
    int dev = 0, sms = 0, least = 0, greatest = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess)
        return DG_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ctas > 0 ? ctas : sms));
    cfg.blockDim = dim3(kStThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;       // ahead of the compositing's CTAs for the free slots
    attr[0].val.priority = greatest;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    const int32_t* cl = list;
#define DG_ST_CASE(D)                                                                                        \
    case D:                                                                                                  \
        cfg.dynamicSmemBytes = st_smem_bytes<D>();                                                           \
        e = cudaLaunchKernelEx(&cfg, k_xstep_stream<D>, xv, mv, vv, av, shared, cl, ctr, a, dev_step, zo);   \
        break;
    switch (x->sh_degree) {
    DG_ST_CASE(0)
    DG_ST_CASE(1)
    DG_ST_CASE(2)
    default:
    DG_ST_CASE(3)
    }
#undef DG_ST_CASE
    note_launch();
    if (e != cudaSuccess) return DG_ERR_CUDA;
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// part 0: the whole step; 1: the groups without a kept record (drec unused;
// `ctas` CTAs, 0 = one per group); 2: the groups with one; 3: the groups
// with one as listed in ws by launch_xstep_groups.  z / gid not NULL:
// unshared copies also stored to z at their global ids.
int launch_xstep(int part, int ctas, dg_gaussians* x, dg_gaussians* m, dg_gaussians* v, const dg_gaussians* anchor,
                 const uint8_t* shared, const dg_camera* cams, const dg_plan& plan, const uint2* rect,
                 const float4* drec, const AdamArgs& a, const int32_t* dev_step, dg_gaussians* z,
                 const int32_t* gid, const void* ws, cudaStream_t st)
{
    if (x->n == 0) return DG_OK;
    GView xv = gview(x), mv = gview(m), vv = gview(v);
    GView av = anchor ? gview(anchor) : xv;
    ZOut zo;
    zo.z = z ? gview(z) : xv;
    zo.gid = z ? gid : nullptr;
    const int64_t n_groups = (x->n + kXsThreads - 1) / kXsThreads;
    dim3 grid((unsigned)n_groups);
    dim3 grid_idle((unsigned)(ctas > 0 && ctas < n_groups ? ctas : n_groups));
    const uint32_t* actr = part == 3 ? static_cast<const uint32_t*>(ws) + 1 : nullptr;
    const int32_t* alist = part == 3 ? reinterpret_cast<const int32_t*>(static_cast<const char*>(ws) + 16) +
                                           (n_groups - 1)
                                     : nullptr;
#define DG_XSTEP_CASE(DEG)                                                                                      \
    case DEG:                                                                                                   \
        if (part == 0)                                                                                          \
            k_xstep<DEG, 0><<<grid, kXsThreads, 0, st>>>(xv, mv, vv, av, shared, cams, plan, rect, drec, a,     \
                                                         dev_step, zo, nullptr, nullptr);                       \
        else if (part == 2)                                                                                     \
            k_xstep<DEG, 2><<<grid, kXsThreads, 0, st>>>(xv, mv, vv, av, shared, cams, plan, rect, drec, a,     \
                                                         dev_step, zo, nullptr, nullptr);                       \
        else if (part == 3)                                                                                     \
            k_xstep<DEG, 3><<<grid, kXsThreads, 0, st>>>(xv, mv, vv, av, shared, cams, plan, rect, drec, a,     \
                                                         dev_step, zo, alist, actr);                            \
        else                                                                                                    \
            k_xstep_idle<DEG><<<grid_idle, kXsThreads, 0, st>>>(xv, mv, vv, av, shared, cams, plan, rect, a,      \
                                                                dev_step, zo);                                  \
        break;
    switch (x->sh_degree) {
    DG_XSTEP_CASE(0)
    DG_XSTEP_CASE(1)
    DG_XSTEP_CASE(2)
    default:
    DG_XSTEP_CASE(3)
    }
#undef DG_XSTEP_CASE
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_project(const dg_gaussians* x, const dg_camera* cams, const dg_plan& plan, float4* rec, uint2* rect,
                   cudaStream_t st)
{
    int64_t n = plan.blk_off[plan.n_blocks];
    if (n == 0) return DG_OK;
    GView xv = gview(x);
    // Four copies per thread while the grid still spans 8 waves of resident
    // CTAs; below that the CTAs whose copies are mostly kept, which project
    // four copies per thread one after another, would form the tail, so one.
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DG_ERR_CUDA;
    const int64_t slots = (int64_t)sms * kProjCtasPerSm;
    const bool four = (n + 4 * kProjThreads - 1) / (4 * kProjThreads) >= 8 * slots;
    const int64_t per_cta = (int64_t)kProjThreads * (four ? 4 : 1);
    dim3 grid((unsigned)((n + per_cta - 1) / per_cta));
#define DG_PROJECT_CASE(D)                                                                    \
    case D:                                                                                   \
        if (four) k_project<D, 4><<<grid, kProjThreads, 0, st>>>(xv, cams, plan, rec, rect);  \
        else k_project<D, 1><<<grid, kProjThreads, 0, st>>>(xv, cams, plan, rec, rect);       \
        break;
    switch (x->sh_degree) {
    DG_PROJECT_CASE(0)
    DG_PROJECT_CASE(1)
    DG_PROJECT_CASE(2)
    default:
    DG_PROJECT_CASE(3)
    }
#undef DG_PROJECT_CASE
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_project_bwd(const dg_gaussians* x, const dg_camera* cams, const dg_plan& plan, const uint2* rect,
                       const float4* drec, dg_gaussians* grads, cudaStream_t st)
{
    int64_t n = plan.blk_off[plan.n_blocks];
    if (n == 0) return DG_OK;
    GView xv = gview(x), gv = gview(grads);
    dim3 grid((unsigned)((n + 127) / 128));
    switch (x->sh_degree) {
    case 0: k_project_bwd<0><<<grid, 128, 0, st>>>(xv, cams, plan, rect, drec, gv); break;
    case 1: k_project_bwd<1><<<grid, 128, 0, st>>>(xv, cams, plan, rect, drec, gv); break;
    case 2: k_project_bwd<2><<<grid, 128, 0, st>>>(xv, cams, plan, rect, drec, gv); break;
    default: k_project_bwd<3><<<grid, 128, 0, st>>>(xv, cams, plan, rect, drec, gv); break;
    }
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg
