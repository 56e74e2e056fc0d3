// Internal helpers shared by the libdogs kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dogs.h"

namespace dg {

// launch accounting (dg_launch_count)
void note_launch(int n = 1);

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
// log2(1/255) rounded to float: a pair is composited when its alpha exponent
// e = log2(o G) is at least this (alpha >= 1/255 in the log domain, decided
// before 2^e is formed)
constexpr float kQMin = -7.99435329f;
// log2(0.99) rounded to float: alpha = min(o G, 0.99) is formed as
// 2^min(e, kLogAlphaMax), the clamp taken in the exponent
constexpr float kLogAlphaMax = -0.0144995693f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;

// ---- parameter-set views ----------------------------------------------------
struct GView {
    float4* mo;     // (p.xyz, opacity logit)
    float4* quat;   // (w, x, y, z)
    float4* scale;  // (log s.xyz, 0)
    float* sh;      // planes, plane j at sh + j * ld
    int64_t n, ld;
    int deg;
};

inline GView gview(const dg_gaussians* g)
{
    GView v;
    v.mo = reinterpret_cast<float4*>(g->data);
    v.quat = reinterpret_cast<float4*>(g->data + 4 * g->ld);
    v.scale = reinterpret_cast<float4*>(g->data + 8 * g->ld);
    v.sh = g->data + 12 * g->ld;
    v.n = g->n;
    v.ld = g->ld;
    v.deg = g->sh_degree;
    return v;
}

__host__ __device__ inline int sh_coefs(int deg) { return (deg + 1) * (deg + 1); }

// block of a copy index (blk_off has n_blocks + 1 ascending entries)
__device__ __forceinline__ int find_block(const dg_plan& p, int64_t c)
{
    int lo = 0, hi = p.n_blocks - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (p.blk_off[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// view owning global tile index t (cams sorted by tile_off)
__device__ __forceinline__ int find_view_of_tile(const dg_camera* cams, int n_views, int64_t t)
{
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&cams[mid].tile_off) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_view_of_rec(const dg_camera* cams, int n_views, int64_t r)
{
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&cams[mid].rec_off) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- compositing decision shared by the forward and the backward -------------
// A staged instance: exponent coefficients in log2 units and log2(opacity):
// power2 = A dx^2 + B dx dy + C dy^2, alpha = 2^(power2 + lo).  An instance
// whose opacity alone is below 1/255 (lo < kQMin; binning keeps a few, its
// cull being widened) can reach no pixel: its lo is staged as -1e30, so that
// every exponent of it fails the first test.
struct Staged {
    float mx, my, A, B, C, lo;
};

__device__ __forceinline__ Staged stage_geometry(float4 r0, float4 r1)
{
    Staged s;
    s.mx = r0.x;
    s.my = r0.y;
    s.A = __fmul_rn(-0.5f * kLog2e, r0.z);
    s.B = __fmul_rn(-kLog2e, r0.w);
    s.C = __fmul_rn(-0.5f * kLog2e, r1.x);
    s.lo = __log2f(r1.y);
    if (!(s.lo >= kQMin)) s.lo = -1e30f;
    return s;
}

// ---- paired FP32 arithmetic (two lanes per instruction, each rounded as the
// scalar operation rounds) ------------------------------------------------------
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f32x2 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- Adam with the ADMM penalty (Eq. 8a / 12a), shared by the x-step kernels ----
struct AdamArgs {
    float rho[5];   // groups p, q, s, f, o
    float lr[6];    // p, q, s, f_dc, f_rest, o
    float b1, b2, eps;
    int step;
    const float* dev_rho;   // non-null: rho read from this device array when the kernel runs
};

// the penalty of group g (rho from the launch, or from device memory)
template <class Args>
__device__ __forceinline__ float rho_of(const Args& a, int g)
{
    return a.dev_rho ? __ldg(a.dev_rho + g) : a.rho[g];
}

// rho[5] of an ABI call points to host memory (read now into dst) or to
// device memory (left to the kernels: *dev = rho), told apart by the driver
inline void take_rho(const float* rho, float* dst, const float** dev)
{
    cudaPointerAttributes at;
    bool on_dev = false;
    if (cudaPointerGetAttributes(&at, rho) == cudaSuccess)
        on_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    else
        cudaGetLastError();
    *dev = on_dev ? rho : nullptr;
    for (int i = 0; i < 5; i++) dst[i] = on_dev ? 0.f : rho[i];
}

__device__ __forceinline__ void bias_corr(const AdamArgs& a, const int32_t* dev_step, float& ic1, float& ic2)
{
    float t = (float)(dev_step ? *dev_step : a.step);
    ic1 = 1.f / (1.f - powf(a.b1, t));
    ic2 = 1.f / (1.f - powf(a.b2, t));
}

// The rounding of every operation below is pinned (explicit fused or
// unfused intrinsics, no contraction left to the compiler), so that each
// x-step kernel -- whatever code surrounds the inlined step -- gives a
// parameter the same bits.

// g + rho (x - a): the gradient of the ADMM penalty rho/2 |x - a|^2 added to g
__device__ __forceinline__ float penalty_add(float g, float rho, float x, float a)
{
    return __fmaf_rn(rho, __fsub_rn(x, a), g);
}

// square root and reciprocal by the SFU (PTX sqrt.approx.ftz and
// rcp.approx.ftz: about 1 ulp each, one instruction and no branch, so that
// the updates of several parameters interleave)
__device__ __forceinline__ float sqrt_sfu(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_sfu(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// one Adam step of one parameter; g already holds the penalty term:
// m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
// x <- x - lr (m ic1) / (sqrt(v ic2) + eps) with ic1, ic2 the bias corrections
__device__ __forceinline__ void adam_scalar(float& x, float g, float& m, float& v, float lr, float b1, float b2,
                                            float eps, float ic1, float ic2)
{
    m = __fmaf_rn(b1, m, __fmul_rn(1.f - b1, g));
    v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(1.f - b2, g), g));
    const float d = __fadd_rn(sqrt_sfu(__fmul_rn(v, ic2)), eps);
    x = __fmaf_rn(-lr, __fmul_rn(__fmul_rn(m, ic1), rcp_sfu(d)), x);
}

// the same step of two parameters at once, by paired FP32 instructions
// where the operation pairs (each lane rounded exactly as adam_scalar rounds
// it, so the two give the same bits)
struct AdamPair {
    f32x2 b1, c1, b2, c2, ic1, ic2, eps;   // c1 = 1 - b1, c2 = 1 - b2, as adam_scalar forms them
};

__device__ __forceinline__ AdamPair adam_pair_args(float b1, float b2, float eps, float ic1, float ic2)
{
    AdamPair P;
    P.b1 = f2_pack(b1, b1);
    P.c1 = f2_pack(1.f - b1, 1.f - b1);
    P.b2 = f2_pack(b2, b2);
    P.c2 = f2_pack(1.f - b2, 1.f - b2);
    P.ic1 = f2_pack(ic1, ic1);
    P.ic2 = f2_pack(ic2, ic2);
    P.eps = f2_pack(eps, eps);
    return P;
}

// nlr = (-lr, -lr) of the two parameters
__device__ __forceinline__ void adam_pair(f32x2& x, f32x2 g, f32x2& m, f32x2& v, f32x2 nlr, const AdamPair& P)
{
    m = f2_fma(P.b1, m, f2_mul(P.c1, g));
    v = f2_fma(P.b2, v, f2_mul(f2_mul(P.c2, g), g));
    float s0, s1;
    f2_unpack(f2_mul(v, P.ic2), s0, s1);
    float d0, d1;
    f2_unpack(f2_add(f2_pack(sqrt_sfu(s0), sqrt_sfu(s1)), P.eps), d0, d1);
    x = f2_fma(nlr, f2_mul(f2_mul(m, P.ic1), f2_pack(rcp_sfu(d0), rcp_sfu(d1))), x);
}

}  // namespace dg

#define DG_CHECK_LAUNCH()                                      \
    do {                                                       \
        cudaError_t _e = cudaGetLastError();                   \
        if (_e != cudaSuccess) return DG_ERR_CUDA;             \
    } while (0)
