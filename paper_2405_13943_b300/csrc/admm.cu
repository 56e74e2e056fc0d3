// K9 and K10: the block ADMM of Sec. 3.2 over the batched block-local copies.
//
// K9 (x-step, Eq. 8a / 12a): one Adam step on every copy with the gradient
// of f_k plus rho_grp (x - z + u) on shared copies; z - u is kept per shared
// copy as the "anchor" so the step reads one extra float per shared float.
// Elementwise over the whole parameter buffer in float4 units; HBM-bound.
//
// K10 (consensus, Eq. 8b-c / 12b-c, over-relaxation of Sec. 3.3, residuals of
// Eq. 9): one thread per global Gaussian gathers its n_i copies through the
// CSR sharing map.  HBM-bound.
#include "common.cuh"

namespace dg {

// The x-step runs as two launches with contiguous warp accesses and no
// per-element index division: the float4 fields (four copies per thread,
// copies strided by the CTA width) and the SH planes (a 2D grid of quads of
// copies x planes, four quads per thread).
__device__ __forceinline__ void adam_unit(float4* __restrict__ x, const float4* __restrict__ g,
                                          float4* __restrict__ m, float4* __restrict__ v,
                                          const float4* __restrict__ anchor, int64_t u, const float* rho,
                                          const float* lr, const bool* act, const bool* sh, float b1, float b2,
                                          float eps, float ic1, float ic2)
{
    float4 xv = x[u], gv = g[u], mv = m[u], vv = v[u];
    float xs[4] = {xv.x, xv.y, xv.z, xv.w}, gs[4] = {gv.x, gv.y, gv.z, gv.w};
    float ms[4] = {mv.x, mv.y, mv.z, mv.w}, vs[4] = {vv.x, vv.y, vv.z, vv.w};
    if (sh[0] || sh[1] || sh[2] || sh[3]) {
        float4 av = anchor[u];
        float as[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (sh[i]) gs[i] = penalty_add(gs[i], rho[i], xs[i], as[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
        if (act[i]) adam_scalar(xs[i], gs[i], ms[i], vs[i], lr[i], b1, b2, eps, ic1, ic2);
    x[u] = make_float4(xs[0], xs[1], xs[2], xs[3]);
    m[u] = make_float4(ms[0], ms[1], ms[2], ms[3]);
    v[u] = make_float4(vs[0], vs[1], vs[2], vs[3]);
}

constexpr int kAdamThreads = 256, kAdamPer = 4;

__global__ void __launch_bounds__(kAdamThreads) k_adam_fields(float4* __restrict__ x, const float4* __restrict__ g,
                                                              float4* __restrict__ m, float4* __restrict__ v,
                                                              const float4* __restrict__ anchor,
                                                              const uint8_t* __restrict__ shared, int64_t n,
                                                              int64_t ld, AdamArgs a, const int32_t* __restrict__ dev_step)
{
    float ic1, ic2;
    bias_corr(a, dev_step, ic1, ic2);
    const float p0 = rho_of(a, 0), p1 = rho_of(a, 1), p2 = rho_of(a, 2), p4 = rho_of(a, 4);
    const float rho0[4] = {p0, p0, p0, p4}, lr0[4] = {a.lr[0], a.lr[0], a.lr[0], a.lr[5]};
    const float rho1[4] = {p1, p1, p1, p1}, lr1[4] = {a.lr[1], a.lr[1], a.lr[1], a.lr[1]};
    const float rho2[4] = {p2, p2, p2, p2}, lr2[4] = {a.lr[2], a.lr[2], a.lr[2], a.lr[2]};
    const bool all4[4] = {true, true, true, true}, three[4] = {true, true, true, false};
    int64_t base = (int64_t)blockIdx.x * (kAdamThreads * kAdamPer) + threadIdx.x;
#pragma unroll
    for (int i = 0; i < kAdamPer; i++) {
        int64_t c = base + i * kAdamThreads;
        if (c >= n) break;
        bool s = shared && shared[c];
        bool s4[4] = {s, s, s, s};
        adam_unit(x, g, m, v, anchor, c, rho0, lr0, all4, s4, a.b1, a.b2, a.eps, ic1, ic2);          // p, o
        adam_unit(x, g, m, v, anchor, ld + c, rho1, lr1, all4, s4, a.b1, a.b2, a.eps, ic1, ic2);     // q
        adam_unit(x, g, m, v, anchor, 2 * ld + c, rho2, lr2, three, s4, a.b1, a.b2, a.eps, ic1, ic2); // s (+pad)
    }
}

__global__ void __launch_bounds__(kAdamThreads) k_adam_planes(float4* __restrict__ x, const float4* __restrict__ g,
                                                              float4* __restrict__ m, float4* __restrict__ v,
                                                              const float4* __restrict__ anchor,
                                                              const uint8_t* __restrict__ shared, int64_t n,
                                                              int64_t ld, AdamArgs a, const int32_t* __restrict__ dev_step)
{
    float ic1, ic2;
    bias_corr(a, dev_step, ic1, ic2);
    const int p = blockIdx.y;
    const float l = p < 3 ? a.lr[3] : a.lr[4];
    const float p3 = rho_of(a, 3);
    const float rho[4] = {p3, p3, p3, p3}, lr[4] = {l, l, l, l};
    const int64_t q4 = ld >> 2;
    const int64_t row = 3 * ld + (int64_t)p * q4;
    int64_t base = (int64_t)blockIdx.x * (kAdamThreads * kAdamPer) + threadIdx.x;
#pragma unroll
    for (int i = 0; i < kAdamPer; i++) {
        int64_t q = base + i * kAdamThreads;
        int64_t c0 = 4 * q;
        if (c0 >= n) break;
        bool act[4], sh[4];
        // byte loads: copy_shared carries no alignment guarantee
#pragma unroll
        for (int k = 0; k < 4; k++) {
            act[k] = c0 + k < n;
            sh[k] = act[k] && shared && shared[c0 + k];
        }
        adam_unit(x, g, m, v, anchor, row + q, rho, lr, act, sh, a.b1, a.b2, a.eps, ic1, ic2);
    }
}

// ---- the x-step's step counter ----------------------------------------------------------
__global__ void k_step_advance(int32_t* __restrict__ dev_step) { *dev_step += 1; }

int launch_step_advance(int32_t* dev_step, cudaStream_t st)
{
    k_step_advance<<<1, 1, 0, st>>>(dev_step);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// ---- consensus ---------------------------------------------------------------------
struct ConsArgs {
    float rho[5];
    float alpha;
    int n_planes;
    const float* dev_rho;   // non-null: rho read from this device array when the kernel runs
};

// Up to kFast copies per global are handled with all their loads issued
// together; globals held by more blocks take the loop below.
constexpr int kFast = 4;

struct ResAcc {
    float rp[5], rd[5];
};

// One float4 field (lanes l: group grp[l]; lane 3 of the scale field is padding).
__device__ __forceinline__ void cons_field4(const float4* __restrict__ X, float4* __restrict__ U,
                                            float4* __restrict__ A, float4* __restrict__ Z, int64_t i,
                                            const int32_t* cp, int n, const int* grp, float alpha, const float* rho,
                                            ResAcc& r)
{
    float4 xs[kFast], us[kFast];
#pragma unroll
    for (int k = 0; k < kFast; k++)
        if (k < n) { xs[k] = X[cp[k]]; us[k] = U[cp[k]]; }
    const float4 zo = Z[i];
    const float zp[4] = {zo.x, zo.y, zo.z, zo.w};
    float zn[4];
    const float inv = 1.f / (float)n;
#pragma unroll
    for (int l = 0; l < 4; l++) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kFast; k++)
            if (k < n) {
                const float xv = (&xs[k].x)[l];
                acc += alpha * xv + (1.f - alpha) * zp[l] + (&us[k].x)[l];
            }
        zn[l] = acc * inv;
    }
#pragma unroll
    for (int k = 0; k < kFast; k++) {
        if (k >= n) continue;
        float un[4], an[4];
#pragma unroll
        for (int l = 0; l < 4; l++) {
            const float xv = (&xs[k].x)[l];
            const float xh = alpha * xv + (1.f - alpha) * zp[l];
            un[l] = (&us[k].x)[l] + xh - zn[l];
            an[l] = zn[l] - un[l];
            if (grp[l] >= 0) r.rp[grp[l]] += (xv - zn[l]) * (xv - zn[l]);
        }
        U[cp[k]] = make_float4(un[0], un[1], un[2], un[3]);
        A[cp[k]] = make_float4(an[0], an[1], an[2], an[3]);
    }
#pragma unroll
    for (int l = 0; l < 4; l++)
        if (grp[l] >= 0) {
            const float dz = zn[l] - zp[l];
            r.rd[grp[l]] += rho[grp[l]] * rho[grp[l]] * (float)n * dz * dz;
        }
    Z[i] = make_float4(zn[0], zn[1], zn[2], zn[3]);
}

// generic path: one scalar element, any number of copies
__device__ __forceinline__ float cons_elem(const float* xp, float* up, float* ap, const int32_t* cp, int n,
                                           int64_t stride, float zprev, float alpha, float& r_primal)
{
    float acc = 0.f;
    for (int k = 0; k < n; k++) {
        int64_t c = (int64_t)cp[k] * stride;
        acc += alpha * xp[c] + (1.f - alpha) * zprev + up[c];
    }
    float z = acc / (float)n;
    for (int k = 0; k < n; k++) {
        int64_t c = (int64_t)cp[k] * stride;
        float xv = xp[c];
        float un = up[c] + alpha * xv + (1.f - alpha) * zprev - z;
        up[c] = un;
        ap[c] = z - un;
        r_primal += (xv - z) * (xv - z);
    }
    return z;
}

// globals held by more than kFast blocks (rare): element by element
__device__ __noinline__ void cons_generic(GView x, GView u, GView z, GView an, int64_t i, const int32_t* cpg, int n,
                                          const ConsArgs& a, ResAcc& r)
{
    float4* xf[3] = {x.mo, x.quat, x.scale};
    float4* uf[3] = {u.mo, u.quat, u.scale};
    float4* zf[3] = {z.mo, z.quat, z.scale};
    float4* af[3] = {an.mo, an.quat, an.scale};
    for (int f = 0; f < 3; f++) {
        float4 zo = zf[f][i];
        float zp[4] = {zo.x, zo.y, zo.z, zo.w}, zn[4];
        for (int l = 0; l < 4; l++) {
            int grp = f == 0 ? (l < 3 ? 0 : 4) : (f == 1 ? 1 : 2);
            float rr = 0.f;
            zn[l] = cons_elem((const float*)xf[f] + l, (float*)uf[f] + l, (float*)af[f] + l, cpg, n, 4, zp[l],
                              a.alpha, rr);
            if (!(f == 2 && l == 3)) {
                r.rp[grp] += rr;
                float dz = zn[l] - zp[l];
                const float rg = rho_of(a, grp);
                r.rd[grp] += rg * rg * (float)n * dz * dz;
            }
        }
        zf[f][i] = make_float4(zn[0], zn[1], zn[2], zn[3]);
    }
    for (int j = 0; j < a.n_planes; j++) {
        float zo = z.sh[(int64_t)j * z.ld + i];
        float rr = 0.f;
        float zn = cons_elem(x.sh + (int64_t)j * x.ld, u.sh + (int64_t)j * u.ld, an.sh + (int64_t)j * an.ld, cpg, n,
                             1, zo, a.alpha, rr);
        z.sh[(int64_t)j * z.ld + i] = zn;
        r.rp[3] += rr;
        const float r3 = rho_of(a, 3);
        r.rd[3] += r3 * r3 * (float)n * (zn - zo) * (zn - zo);
    }
}

#ifndef DG_CONS_CTAS
#define DG_CONS_CTAS 8   // 64 registers: 32 warps per SM (with CH = 2 below; measured best, see CH)
#endif
template <int NP>
__global__ void __launch_bounds__(128, DG_CONS_CTAS) k_consensus(GView x, GView u, GView z, GView an,
                                                   const int64_t* __restrict__ g_off,
                                                   const int32_t* __restrict__ g_copies, int64_t n_glob,
                                                   ConsArgs a, double* __restrict__ res)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    ResAcc r;
#pragma unroll
    for (int k = 0; k < 5; k++) { r.rp[k] = 0.f; r.rd[k] = 0.f; }
    if (i < n_glob) {
        const int64_t b = g_off[i];
        const int n = (int)(g_off[i + 1] - b);
        const int32_t* cpg = g_copies + b;
        if (n == 1) {
            // unshared: z = x; every load is issued before the first store
            const int64_t c = cpg[0];
            const float4 m0 = x.mo[c], q0 = x.quat[c], s0 = x.scale[c];
            float f[NP];
#pragma unroll
            for (int j = 0; j < NP; j++) f[j] = x.sh[(int64_t)j * x.ld + c];
            z.mo[i] = m0;
            z.quat[i] = q0;
            z.scale[i] = s0;
#pragma unroll
            for (int j = 0; j < NP; j++) z.sh[(int64_t)j * z.ld + i] = f[j];
        } else if (n > 1 && n <= kFast) {
            int32_t cp[kFast];
#pragma unroll
            for (int k = 0; k < kFast; k++) cp[k] = k < n ? cpg[k] : 0;
            const int g_mo[4] = {0, 0, 0, 4}, g_q[4] = {1, 1, 1, 1}, g_s[4] = {2, 2, 2, -1};
            float rh[5];
#pragma unroll
            for (int k = 0; k < 5; k++) rh[k] = rho_of(a, k);
            cons_field4(x.mo, u.mo, an.mo, z.mo, i, cp, n, g_mo, a.alpha, rh, r);
            cons_field4(x.quat, u.quat, an.quat, z.quat, i, cp, n, g_q, a.alpha, rh, r);
            cons_field4(x.scale, u.scale, an.scale, z.scale, i, cp, n, g_s, a.alpha, rh, r);
            const float rho3 = rh[3];
            const float inv = 1.f / (float)n;
            // planes per batch of loads; same-box A/B on the 6M step (CTAs per SM, CH):
            // (6, 4) 0.359 ms, (6, 2) 0.351, (7, 3) 0.336, (8, 2) 0.329.  Larger batches
            // at a given register budget spill more than their extra loads in flight gain.
            constexpr int CH = 2;
#pragma unroll
            for (int j0 = 0; j0 < NP; j0 += CH) {
                float xs[CH][kFast], us[CH][kFast], zo[CH];
#pragma unroll
                for (int jj = 0; jj < CH; jj++) {
                    const int j = j0 + jj;
                    if (j >= NP) continue;
                    zo[jj] = z.sh[(int64_t)j * z.ld + i];
#pragma unroll
                    for (int k = 0; k < kFast; k++)
                        if (k < n) {
                            xs[jj][k] = x.sh[(int64_t)j * x.ld + cp[k]];
                            us[jj][k] = u.sh[(int64_t)j * u.ld + cp[k]];
                        }
                }
#pragma unroll
                for (int jj = 0; jj < CH; jj++) {
                    const int j = j0 + jj;
                    if (j >= NP) continue;
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < kFast; k++)
                        if (k < n) acc += a.alpha * xs[jj][k] + (1.f - a.alpha) * zo[jj] + us[jj][k];
                    const float zn = acc * inv;
#pragma unroll
                    for (int k = 0; k < kFast; k++)
                        if (k < n) {
                            const float un = us[jj][k] + a.alpha * xs[jj][k] + (1.f - a.alpha) * zo[jj] - zn;
                            u.sh[(int64_t)j * u.ld + cp[k]] = un;
                            an.sh[(int64_t)j * an.ld + cp[k]] = zn - un;
                            r.rp[3] += (xs[jj][k] - zn) * (xs[jj][k] - zn);
                        }
                    z.sh[(int64_t)j * z.ld + i] = zn;
                    r.rd[3] += rho3 * rho3 * (float)n * (zn - zo[jj]) * (zn - zo[jj]);
                }
            }
        } else if (n > kFast) {
            cons_generic(x, u, z, an, i, cpg, n, a, r);
        }
    }
    if (res) {
        __shared__ float s_r[4][10];
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 5; k++) {
            float a0 = r.rp[k], a1 = r.rd[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            }
            if (lane == 0) { s_r[w][k] = a0; s_r[w][5 + k] = a1; }
        }
        __syncthreads();
        if (threadIdx.x < 10) {
            double t = 0.0;
            for (int ww = 0; ww < 4; ww++) t += s_r[ww][threadIdx.x];
            if (t != 0.0) atomicAdd(&res[threadIdx.x], t);
        }
    }
}

// anchor = z[gid] - u for shared copies
__global__ void __launch_bounds__(256) k_anchor(GView z, GView u, GView an, const int32_t* __restrict__ gid,
                                                const uint8_t* __restrict__ shared, int64_t n, int n_planes)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || !shared[c]) return;
    int64_t gI = gid[c];
    float4 a, b;
    a = z.mo[gI]; b = u.mo[c]; an.mo[c] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    a = z.quat[gI]; b = u.quat[c]; an.quat[c] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    a = z.scale[gI]; b = u.scale[c]; an.scale[c] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    for (int j = 0; j < n_planes; j++)
        an.sh[(int64_t)j * an.ld + c] = z.sh[(int64_t)j * z.ld + gI] - u.sh[(int64_t)j * u.ld + c];
}

// u_grp *= factor[grp] on shared copies (the scaled duals follow a change of
// rho: u = y / rho, so rho -> rho' rescales u by rho / rho')
__global__ void __launch_bounds__(256) k_scale_duals(GView u, const uint8_t* __restrict__ shared, int64_t n,
                                                     int n_planes, float f0, float f1, float f2, float f3, float f4)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || !shared[c]) return;
    float4 m = u.mo[c];
    u.mo[c] = make_float4(m.x * f0, m.y * f0, m.z * f0, m.w * f4);
    float4 q = u.quat[c];
    u.quat[c] = make_float4(q.x * f1, q.y * f1, q.z * f1, q.w * f1);
    float4 s = u.scale[c];
    u.scale[c] = make_float4(s.x * f2, s.y * f2, s.z * f2, s.w * f2);
    for (int j = 0; j < n_planes; j++) u.sh[(int64_t)j * u.ld + c] *= f3;
}

int launch_scale_duals(dg_gaussians* u, const uint8_t* shared, const float* f, cudaStream_t st)
{
    if (u->n == 0) return DG_OK;
    k_scale_duals<<<(unsigned)((u->n + 255) / 256), 256, 0, st>>>(gview(u), shared, u->n, 3 * sh_coefs(u->sh_degree),
                                                                  f[0], f[1], f[2], f[3], f[4]);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// ---- Eq. 10 on the device ------------------------------------------------------------
// One thread per group g: with r = sqrt(primal_g), s = sqrt(dual_g) from
// the consensus just run, rho_g *= tau_inc when r > mu s, rho_g /= tau_dec
// when s > mu r, unchanged otherwise, and only while the iteration
// t = *dev_step - 1 is below freeze_after; factor_g = old rho_g / new rho_g,
// the rescale of the scaled duals (u = y / rho).  Compared in FP64 as the
// host rule does.
__global__ void k_admm_adapt(const double* __restrict__ res, float* __restrict__ rho, float* __restrict__ factor,
                             const int32_t* __restrict__ dev_step, float mu, float tau_inc, float tau_dec,
                             int freeze_after)
{
    const int g = threadIdx.x;
    if (g >= 5) return;
    const int t = *dev_step - 1;
    const float old = rho[g];
    float nw = old;
    if (t < freeze_after) {
        const double r = sqrt(fmax(res[g], 0.0)), s = sqrt(fmax(res[5 + g], 0.0));
        if (r > (double)mu * s)
            nw = (float)((double)old * (double)tau_inc);
        else if (s > (double)mu * r)
            nw = (float)((double)old / (double)tau_dec);
    }
    rho[g] = nw;
    factor[g] = old / nw;
}

// After a change of rho: u_grp *= factor[grp] on the shared copies and their
// anchors z - u rebuilt, in one pass; returns at once when every factor is 1.
__global__ void __launch_bounds__(256) k_admm_rescale(GView u, GView z, GView an, const int32_t* __restrict__ gid,
                                                      const uint8_t* __restrict__ shared, int64_t n, int n_planes,
                                                      const float* __restrict__ factor)
{
    const float f0 = __ldg(factor), f1 = __ldg(factor + 1), f2 = __ldg(factor + 2), f3 = __ldg(factor + 3),
                f4 = __ldg(factor + 4);
    if (f0 == 1.f && f1 == 1.f && f2 == 1.f && f3 == 1.f && f4 == 1.f) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || !shared[c]) return;
    const int64_t gI = gid[c];
    float4 m = u.mo[c], a = z.mo[gI];
    m = make_float4(m.x * f0, m.y * f0, m.z * f0, m.w * f4);
    u.mo[c] = m;
    an.mo[c] = make_float4(a.x - m.x, a.y - m.y, a.z - m.z, a.w - m.w);
    float4 q = u.quat[c];
    a = z.quat[gI];
    q = make_float4(q.x * f1, q.y * f1, q.z * f1, q.w * f1);
    u.quat[c] = q;
    an.quat[c] = make_float4(a.x - q.x, a.y - q.y, a.z - q.z, a.w - q.w);
    float4 sc = u.scale[c];
    a = z.scale[gI];
    sc = make_float4(sc.x * f2, sc.y * f2, sc.z * f2, sc.w * f2);
    u.scale[c] = sc;
    an.scale[c] = make_float4(a.x - sc.x, a.y - sc.y, a.z - sc.z, a.w - sc.w);
    for (int j = 0; j < n_planes; j++) {
        const float un = u.sh[(int64_t)j * u.ld + c] * f3;
        u.sh[(int64_t)j * u.ld + c] = un;
        an.sh[(int64_t)j * an.ld + c] = z.sh[(int64_t)j * z.ld + gI] - un;
    }
}

int launch_admm_adapt(const double* res, float* rho, float* factor, const int32_t* dev_step, float mu,
                      float tau_inc, float tau_dec, int freeze_after, cudaStream_t st)
{
    k_admm_adapt<<<1, 32, 0, st>>>(res, rho, factor, dev_step, mu, tau_inc, tau_dec, freeze_after);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_admm_rescale(dg_gaussians* u, const dg_gaussians* z, dg_gaussians* an, const int32_t* gid,
                        const uint8_t* shared, const float* factor, cudaStream_t st)
{
    if (u->n == 0) return DG_OK;
    k_admm_rescale<<<(unsigned)((u->n + 255) / 256), 256, 0, st>>>(gview(u), gview(z), gview(an), gid, shared, u->n,
                                                                   3 * sh_coefs(u->sh_degree), factor);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_adam_admm(dg_gaussians* x, const dg_gaussians* g, dg_gaussians* m, dg_gaussians* v,
                     const dg_gaussians* anchor, const uint8_t* shared, const float* rho, const float* lr,
                     float b1, float b2, float eps, int step, const int32_t* dev_step, cudaStream_t st)
{
    if (x->n == 0) return DG_OK;
    AdamArgs a;
    take_rho(rho, a.rho, &a.dev_rho);
    for (int i = 0; i < 6; i++) a.lr[i] = lr[i];
    a.b1 = b1; a.b2 = b2; a.eps = eps; a.step = step;
    const float4* an = anchor ? reinterpret_cast<const float4*>(anchor->data) : nullptr;
    float4* X = reinterpret_cast<float4*>(x->data);
    const float4* G = reinterpret_cast<const float4*>(g->data);
    float4* M = reinterpret_cast<float4*>(m->data);
    float4* V = reinterpret_cast<float4*>(v->data);
    const int64_t per = kAdamThreads * kAdamPer;
    k_adam_fields<<<(unsigned)((x->n + per - 1) / per), kAdamThreads, 0, st>>>(X, G, M, V, an, shared, x->n, x->ld,
                                                                               a, dev_step);
    dim3 grid((unsigned)(((x->n + 3) / 4 + per - 1) / per), (unsigned)(3 * sh_coefs(x->sh_degree)));
    k_adam_planes<<<grid, kAdamThreads, 0, st>>>(X, G, M, V, an, shared, x->n, x->ld, a, dev_step);
    note_launch(2);
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_consensus(const dg_gaussians* x, dg_gaussians* u, dg_gaussians* z, dg_gaussians* an,
                     const int64_t* g_off, const int32_t* g_copies, const float* rho, float alpha, double* res,
                     cudaStream_t st)
{
    if (res && cudaMemsetAsync(res, 0, 10 * sizeof(double), st) != cudaSuccess) return DG_ERR_CUDA;
    if (z->n == 0) return DG_OK;
    ConsArgs a;
    take_rho(rho, a.rho, &a.dev_rho);
    a.alpha = alpha;
    a.n_planes = 3 * sh_coefs(x->sh_degree);
    const unsigned grid = (unsigned)((z->n + 127) / 128);
    switch (x->sh_degree) {
    case 0: k_consensus<3><<<grid, 128, 0, st>>>(gview(x), gview(u), gview(z), gview(an), g_off, g_copies, z->n, a, res); break;
    case 1: k_consensus<12><<<grid, 128, 0, st>>>(gview(x), gview(u), gview(z), gview(an), g_off, g_copies, z->n, a, res); break;
    case 2: k_consensus<27><<<grid, 128, 0, st>>>(gview(x), gview(u), gview(z), gview(an), g_off, g_copies, z->n, a, res); break;
    default: k_consensus<48><<<grid, 128, 0, st>>>(gview(x), gview(u), gview(z), gview(an), g_off, g_copies, z->n, a, res); break;
    }
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_anchor(const dg_gaussians* z, const dg_gaussians* u, const int32_t* gid, const uint8_t* shared,
                  dg_gaussians* an, cudaStream_t st)
{
    if (u->n == 0) return DG_OK;
    k_anchor<<<(unsigned)((u->n + 255) / 256), 256, 0, st>>>(gview(z), gview(u), gview(an), gid, shared, u->n,
                                                             3 * sh_coefs(z->sh_degree));
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg
