// K6 / K11: the training loss of Eq. 3, L = w_l1 * L1 + w_ssim * (1 - SSIM),
// per view, with dL/d(image).
//
// SSIM: 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, zero
// padding, "same" size.  The forward computes the local moments with a
// separable filter in shared memory (output tile 32x54 plus a 5-pixel halo):
// the means of x and y, of xy, and of x^2 + y^2 -- the two variances enter
// SSIM only as their sum s1 + s2 = E[x^2 + y^2] - mx^2 - my^2, so four
// filtered maps where the five moments would take five -- then the SSIM
// map and the three per-pixel partials dS/d(mean_x), dS/d(E[x^2]),
// dS/d(E[xy]); the backward applies the same (symmetric) filter to those
// partials: dL/dx = F(a) + 2 x F(b) + y F(c).
#include <algorithm>

#include "common.cuh"

namespace dg {

constexpr int kR = 5, kWin = 11;

struct Win { float w[kWin]; };

static Win gaussian_window()
{
    Win g;
    double s = 0.0, v[kWin];
    for (int i = 0; i < kWin; i++) { double d = i - kR; v[i] = exp(-d * d / (2.0 * 1.5 * 1.5)); s += v[i]; }
    for (int i = 0; i < kWin; i++) g.w[i] = (float)(v[i] / s);
    return g;
}

// ---- L1 --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_l1(const float* __restrict__ img, const float* __restrict__ tgt,
                                            const dg_camera* __restrict__ cams, float w_l1,
                                            double* __restrict__ sums, float* __restrict__ grad)
{
    int v = blockIdx.y;
    int64_t HW = (int64_t)__ldg(&cams[v].width) * __ldg(&cams[v].height);
    int64_t off = 3 * __ldg(&cams[v].pix_off);
    float inv = w_l1 / (float)(3 * HW);
    float acc = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * HW; i += (int64_t)gridDim.x * blockDim.x) {
        float d = img[off + i] - tgt[off + i];
        acc += fabsf(d);
        grad[off + i] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s_w[8];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; i++) t += s_w[i];
        atomicAdd(&sums[v], t);
    }
}

// loss[v] holds sum |I - I*| on entry; ssim_sum (may be NULL) sum of the SSIM map
__global__ void k_loss_final(const dg_camera* __restrict__ cams, int n_views, float w_l1, float w_ssim,
                             const double* __restrict__ ssim_sum, double* __restrict__ loss)
{
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    double N = 3.0 * (double)__ldg(&cams[v].width) * (double)__ldg(&cams[v].height);
    loss[v] = (double)w_l1 * loss[v] / N + (ssim_sum ? (double)w_ssim * (1.0 - ssim_sum[v] / N) : 0.0);
}

// ---- SSIM ------------------------------------------------------------------------
// Output tile 32 x 54 per CTA (256 threads) with a 5-pixel halo, so the input
// tile is 42 x 64: the horizontal pass is exactly one task per thread (64
// input rows x 4 blocks of 8 columns) and the vertical pass 224 tasks (32
// columns x 7 blocks of 8 rows).  Both passes are register-blocked: a thread
// produces 8 consecutive outputs from a window of 18 inputs held in
// registers, so each input is read from shared memory once per pass.
constexpr int kTW = 32;                 // output tile width
constexpr int kTH = 54;                 // output tile height
constexpr int kIH = kTH + 2 * kR;       // input tile height (64)
constexpr int kBlk = 8;                 // outputs per thread per pass
constexpr int kWin8 = kBlk + 2 * kR;    // 18 inputs per 8 outputs
constexpr int kSsimThreads = 256;
// The input rows are staged from global column x0 - 8 (16-byte aligned when
// the image width is a multiple of 4) over 48 columns, 12 chunks of four;
// tile column c (global x0 - 5 + c) sits at staged column c + 3.  Row stride
// 52 floats: a multiple of four for the 16-byte copies, and with it the
// horizontal pass's 16-byte reads (two rows x four column blocks per
// quarter-warp) fall in distinct banks.
constexpr int kIWv = 48;                // staged columns
constexpr int kIWP = 52;                // staged row stride
constexpr int kTWP = kTW + 1;           // 33: horizontal-pass output stride (odd: conflict-free columns)
constexpr int kVBlocks = (kTH + kBlk - 1) / kBlk;   // 7 row blocks in the vertical pass
constexpr int kTHP = kVBlocks * kBlk + 2 * kR;      // 66 rows of horizontal output read by the vertical pass

// horizontal pass over NM maps, one task per thread: input row r = tid / 4,
// output columns c0 .. c0 + 7 with c0 = 8 (tid % 4): tmp[m][r][c] = sum_k w_k in_m[r][c + k].
// The 18 inputs of the task are staged columns c0 + 3 .. c0 + 20, read as six
// 16-byte chunks (staged columns c0 .. c0 + 23).
template <int NM, int NIN, typename Make>
__device__ __forceinline__ void hpass(const Win& g, const float* const* in_maps, float (*tmp)[kTHP][kTWP], Make make)
{
    const int r = threadIdx.x >> 2, c0 = (threadIdx.x & 3) * kBlk;
    float raw[NIN][24];
#pragma unroll
    for (int n = 0; n < NIN; n++)
#pragma unroll
        for (int q = 0; q < 6; q++) {
            const float4 v = *reinterpret_cast<const float4*>(in_maps[n] + r * kIWP + c0 + 4 * q);
            raw[n][4 * q] = v.x; raw[n][4 * q + 1] = v.y; raw[n][4 * q + 2] = v.z; raw[n][4 * q + 3] = v.w;
        }
    float in[NM][kWin8];
#pragma unroll
    for (int i = 0; i < kWin8; i++) make(raw, 3 + i, in, i);
#pragma unroll
    for (int m = 0; m < NM; m++)
#pragma unroll
        for (int j = 0; j < kBlk; j++) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; k++) s = fmaf(g.w[k], in[m][j + k], s);
            tmp[m][r][c0 + j] = s;
        }
}

// vertical pass: out[m][j] = sum_k w_k tmp[m][r0 + j + k][c] for column c and
// rows r0 .. r0 + 7 (rows past the tile's input are read from the padding
// rows and never stored)
template <int NM>
__device__ __forceinline__ void vpass(const Win& g, float (*tmp)[kTHP][kTWP], int c, int r0, float out[][kBlk])
{
#pragma unroll
    for (int m = 0; m < NM; m++) {
        float col[kWin8];
#pragma unroll
        for (int i = 0; i < kWin8; i++) col[i] = tmp[m][r0 + i][c];
#pragma unroll
        for (int j = 0; j < kBlk; j++) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; k++) s = fmaf(g.w[k], col[j + k], s);
            out[m][j] = s;
        }
    }
}

// ---- persistent, double-buffered SSIM passes ---------------------------------------
// Each CTA walks work items (view, channel, tile) with a stride of the grid;
// the input halo of the next item is copied into the other shared-memory
// buffer by cp.async (zero-filled outside the image) while the current item
// is filtered, so the loads' latency hides behind the arithmetic.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool ok)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

struct SsimItem {
    int v, ch, x0, y0, W, H;
    int64_t HW, pix;
    bool ok;
};

__device__ __forceinline__ SsimItem ssim_item(const dg_camera* __restrict__ cams, int w, int TX, int TY)
{
    SsimItem it;
    const int per = TX * TY, z = w / per, rem = w - z * per;
    it.v = z / 3;
    it.ch = z - 3 * it.v;
    it.x0 = (rem % TX) * kTW;
    it.y0 = (rem / TX) * kTH;
    it.W = __ldg(&cams[it.v].width);
    it.H = __ldg(&cams[it.v].height);
    it.HW = (int64_t)it.W * it.H;
    it.pix = __ldg(&cams[it.v].pix_off);
    it.ok = it.x0 < it.W && it.y0 < it.H;
    return it;
}

// the view of work item w (the items of a view are consecutive)
__device__ __forceinline__ int ssim_view(int w, int TX, int TY) { return w / (3 * TX * TY); }

// A thread's share of a per-view sum (the SSIM map, the L1 term) over the
// CTA's consecutive items of one view, added to sum[v] when the next item is
// of another view or there is none: one atomic per warp and view run, and no
// barrier or double arithmetic per item.
__device__ __forceinline__ void ssim_flush(float& part, int w, int n_work, int v, int TX, int TY,
                                           double* __restrict__ sum)
{
    const int wn = w + (int)gridDim.x;
    if (wn < n_work && ssim_view(wn, TX, TY) == v) return;     // uniform over the CTA
    float s = part;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s != 0.f) atomicAdd(&sum[v], (double)s);
    part = 0.f;
}

// copy NP planes (plane m at pl[m], an item's channel plane) of item `it`'s
// input rows, global columns x0 - 8 .. x0 + 39, into dst[m][kIH][kIWP]: by
// 16-byte chunks when the width and the planes allow it (a chunk is then
// wholly inside or wholly outside the image), else element by element.  The
// planes are taken one after another with a constant index, so their
// pointers stay in registers.
struct Planes {
    const float* p[3];
};

template <int NP>
__device__ __forceinline__ void ssim_issue(const SsimItem& it, const Planes& pl, float* dst)
{
    if (!it.ok) return;
    const int gx0 = it.x0 - 8, gy0 = it.y0 - kR;
    bool vec = (it.W & 3) == 0;
#pragma unroll
    for (int m = 0; m < NP; m++) vec = vec && (((uintptr_t)pl.p[m] & 15u) == 0);
    if (vec) {
        constexpr int CH = kIWv / 4;                  // 16-byte chunks per row
        static_assert((kIH * CH) % kSsimThreads == 0, "whole chunks per thread");
#pragma unroll
        for (int m = 0; m < NP; m++)
#pragma unroll
            for (int k = 0; k < kIH * CH / kSsimThreads; k++) {
                const int i = (int)threadIdx.x + k * kSsimThreads;
                const int r = i / CH, q = i - r * CH;
                const int gx = gx0 + 4 * q, gy = gy0 + r;
                const bool ok = gx >= 0 && gx < it.W && gy >= 0 && gy < it.H;
                const float* src = pl.p[m] + (ok ? (int64_t)gy * it.W + gx : 0);
                cp_async16(dst + (m * kIH + r) * kIWP + 4 * q, src, ok);
            }
    } else {
        for (int i = threadIdx.x; i < kIH * kIWv; i += kSsimThreads) {
            const int r = i / kIWv, c = i - r * kIWv;
            const int gx = gx0 + c, gy = gy0 + r;
            const bool ok = gx >= 0 && gx < it.W && gy >= 0 && gy < it.H;
            const int64_t p = ok ? (int64_t)gy * it.W + gx : 0;
#pragma unroll
            for (int m = 0; m < NP; m++)
                cp_async4(dst + (m * kIH + r) * kIWP + c, pl.p[m] + p, ok);
        }
    }
}

__global__ void __launch_bounds__(kSsimThreads) k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                          const dg_camera* __restrict__ cams, Win g, float w_ssim,
                                                          double* __restrict__ sums, float* __restrict__ partial,
                                                          int TX, int TY, int n_work)
{
    extern __shared__ float s_dyn[];
    float* s_in = s_dyn;                                   // [2 buffers][x, y][kIH][kIWP]
    float (*s_tmp)[kTHP][kTWP] = reinterpret_cast<float (*)[kTHP][kTWP]>(s_dyn + 4 * kIH * kIWP);   // 4 maps
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float part = 0.f;   // this thread's SSIM sum over the current view's items
    int buf = 0;
    {
        const int w = blockIdx.x;
        if (w < n_work) {
            const SsimItem it = ssim_item(cams, w, TX, TY);
            const Planes bp = {{img + 3 * it.pix + it.ch * it.HW, tgt + 3 * it.pix + it.ch * it.HW, nullptr}};
            ssim_issue<2>(it, bp, s_in);
        }
        cp_async_commit();
    }
    for (int w = blockIdx.x; w < n_work; w += gridDim.x, buf ^= 1) {
        const int wn = w + gridDim.x;
        if (wn < n_work) {
            const SsimItem nt = ssim_item(cams, wn, TX, TY);
            const Planes bp = {{img + 3 * nt.pix + nt.ch * nt.HW, tgt + 3 * nt.pix + nt.ch * nt.HW, nullptr}};
            ssim_issue<2>(nt, bp, s_in + (buf ^ 1) * 2 * kIH * kIWP);
        }
        cp_async_commit();
        cp_async_wait_prev();
        __syncthreads();
        const SsimItem it = ssim_item(cams, w, TX, TY);
        if (!it.ok) {                                 // uniform over the CTA
            ssim_flush(part, w, n_work, it.v, TX, TY, sums);
            continue;
        }
        const float* maps[2] = {s_in + buf * 2 * kIH * kIWP, s_in + (buf * 2 + 1) * kIH * kIWP};
        hpass<4, 2>(g, maps, s_tmp, [&](float (*raw)[24], int c, float (*in)[kWin8], int i) {
            const float a = raw[0][c], b = raw[1][c];
            in[0][i] = a; in[1][i] = b; in[2][i] = fmaf(a, a, b * b); in[3][i] = a * b;
        });
        __syncthreads();
        const float sc = -w_ssim / (float)(3 * it.HW);
        float* P = partial + 9 * it.pix + 3 * it.ch * it.HW;
        if (threadIdx.x < kTW * kVBlocks) {
            const int c = threadIdx.x % kTW, r0 = (threadIdx.x / kTW) * kBlk;
            float mo[4][kBlk];
            vpass<4>(g, s_tmp, c, r0, mo);
            const int gx = it.x0 + c;
#pragma unroll
            for (int j = 0; j < kBlk; j++) {
                const int gy = it.y0 + r0 + j;
                if (r0 + j >= kTH || gx >= it.W || gy >= it.H) continue;
                const float m1 = mo[0][j], m2 = mo[1][j];
                const float mm = m1 * m1 + m2 * m2;
                const float s12 = mo[3][j] - m1 * m2;      // s1 + s2 = mo[2] - mm
                const float A1 = 2.f * m1 * m2 + C1, A2 = 2.f * s12 + C2;
                const float B1 = mm + C1, B2 = (mo[2][j] - mm) + C2;
                const float iB = __fdividef(1.f, B1 * B2);
                const float S = A1 * A2 * iB;
                part += S;
                // dS/dA1, dS/dA2, dS/dB1 = -S / B1 = -S B2 iB, dS/dB2 = -S B1 iB
                const float dA1 = A2 * iB, dA2 = A1 * iB, dB1 = -S * B2 * iB, dB2 = -S * B1 * iB;
                const float dm1 = 2.f * m2 * dA1 - 2.f * m2 * dA2 + 2.f * m1 * dB1 - 2.f * m1 * dB2;
                const int64_t p = (int64_t)gy * it.W + gx;
                P[p] = sc * dm1;
                P[it.HW + p] = sc * dB2;
                P[2 * it.HW + p] = sc * 2.f * dA2;
            }
        }
        ssim_flush(part, w, n_work, it.v, TX, TY, sums);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

constexpr size_t kSsimFwdSmem = sizeof(float) * (4 * kIH * kIWP + 4 * kTHP * kTWP);
constexpr size_t kSsimBwdSmem = sizeof(float) * (6 * kIH * kIWP + 3 * kTHP * kTWP);

// dL/dx = w_l1 sign(x - y) / N + F(a) + 2 x F(b) + y F(c); the L1 sum of the
// tile is added to l1_sum[v].  The output pixels' x and y are loaded before the
// filter passes so that their latency overlaps the shared-memory work.
__global__ void __launch_bounds__(kSsimThreads) k_ssim_bwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                          const dg_camera* __restrict__ cams, Win g, float w_l1,
                                                          const float* __restrict__ partial, float* __restrict__ grad,
                                                          double* __restrict__ l1_sum, int TX, int TY, int n_work)
{
    extern __shared__ float s_dyn[];
    float* s_in = s_dyn;                                   // [2 buffers][3 maps][kIH][kIWP]
    float (*s_tmp)[kTHP][kTWP] = reinterpret_cast<float (*)[kTHP][kTWP]>(s_dyn + 6 * kIH * kIWP);
    const bool has_out = threadIdx.x < kTW * kVBlocks;
    float part = 0.f;   // this thread's L1 sum over the current view's items
    const int c = threadIdx.x % kTW, r0 = (threadIdx.x / kTW) * kBlk;
    int buf = 0;
    {
        const int w = blockIdx.x;
        if (w < n_work) {
            const SsimItem it = ssim_item(cams, w, TX, TY);
            const float* P = partial + 9 * it.pix + 3 * it.ch * it.HW;
            const Planes bp = {{P, P + it.HW, P + 2 * it.HW}};
            ssim_issue<3>(it, bp, s_in);
        }
        cp_async_commit();
    }
    for (int w = blockIdx.x; w < n_work; w += gridDim.x, buf ^= 1) {
        const int wn = w + gridDim.x;
        if (wn < n_work) {
            const SsimItem nt = ssim_item(cams, wn, TX, TY);
            const float* P = partial + 9 * nt.pix + 3 * nt.ch * nt.HW;
            const Planes bp = {{P, P + nt.HW, P + 2 * nt.HW}};
            ssim_issue<3>(nt, bp, s_in + (buf ^ 1) * 3 * kIH * kIWP);
        }
        cp_async_commit();
        const SsimItem it = ssim_item(cams, w, TX, TY);
        // this thread's outputs: column c, rows r0 .. r0 + 7
        const float* X = img + 3 * it.pix + it.ch * it.HW;
        const float* Y = tgt + 3 * it.pix + it.ch * it.HW;
        const int gx = it.x0 + c;
        float xv[kBlk], yv[kBlk];
#pragma unroll
        for (int j = 0; j < kBlk; j++) {
            const int gy = it.y0 + r0 + j;
            const bool ok = it.ok && has_out && r0 + j < kTH && gx < it.W && gy < it.H;
            const int64_t p = (int64_t)gy * it.W + gx;
            xv[j] = ok ? X[p] : 0.f;
            yv[j] = ok ? Y[p] : 0.f;
        }
        cp_async_wait_prev();
        __syncthreads();
        if (!it.ok) {                                 // uniform over the CTA
            ssim_flush(part, w, n_work, it.v, TX, TY, l1_sum);
            continue;
        }
        const float* sp0 = s_in + buf * 3 * kIH * kIWP;
        const float* maps[3] = {sp0, sp0 + kIH * kIWP, sp0 + 2 * kIH * kIWP};
        hpass<3, 3>(g, maps, s_tmp, [&](float (*raw)[24], int c, float (*in)[kWin8], int i) {
            in[0][i] = raw[0][c]; in[1][i] = raw[1][c]; in[2][i] = raw[2][c];
        });
        __syncthreads();
        if (has_out) {
            float fo[3][kBlk];
            vpass<3>(g, s_tmp, c, r0, fo);
            const float wl = w_l1 / (float)(3 * it.HW);
            float* G = grad + 3 * it.pix + it.ch * it.HW;
#pragma unroll
            for (int j = 0; j < kBlk; j++) {
                const int gy = it.y0 + r0 + j;
                if (r0 + j >= kTH || gx >= it.W || gy >= it.H) continue;
                const int64_t p = (int64_t)gy * it.W + gx;
                const float d = xv[j] - yv[j];
                part += fabsf(d);
                const float l1g = d > 0.f ? wl : (d < 0.f ? -wl : 0.f);
                G[p] = l1g + fo[0][j] + 2.f * xv[j] * fo[1][j] + yv[j] * fo[2][j];
            }
        }
        ssim_flush(part, w, n_work, it.v, TX, TY, l1_sum);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---- 8-bit images ---------------------------------------------------------------
// Training images are 8-bit; they cross the host link as bytes and widen on
// the device (v / 255, correctly rounded), four per thread.
__global__ void __launch_bounds__(256) k_u8_to_f32(const uint8_t* __restrict__ src, float* __restrict__ dst,
                                                   int64_t n)
{
    const int64_t n4 = n / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const uchar4 b = reinterpret_cast<const uchar4*>(src)[i];
        reinterpret_cast<float4*>(dst)[i] = make_float4(__fdiv_rn((float)b.x, 255.f), __fdiv_rn((float)b.y, 255.f),
                                                        __fdiv_rn((float)b.z, 255.f), __fdiv_rn((float)b.w, 255.f));
    }
    if (blockIdx.x == 0 && threadIdx.x < (unsigned)(n - 4 * n4))   // the last n mod 4 bytes
        dst[4 * n4 + threadIdx.x] = __fdiv_rn((float)src[4 * n4 + threadIdx.x], 255.f);
}

// round(clamp(v, 0, 1) * 255)
__global__ void __launch_bounds__(256) k_f32_to_u8(const float* __restrict__ src, uint8_t* __restrict__ dst,
                                                   int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (uint8_t)__float2int_rn(fminf(fmaxf(src[i], 0.f), 1.f) * 255.f);
}

int launch_u8_to_f32(const uint8_t* src, float* dst, int64_t n, cudaStream_t st)
{
    if (n == 0) return DG_OK;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n / 4 + 255) / 256, 148 * 16));
    k_u8_to_f32<<<g, 256, 0, st>>>(src, dst, n);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_f32_to_u8(const float* src, uint8_t* dst, int64_t n, cudaStream_t st)
{
    if (n == 0) return DG_OK;
    const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 148 * 16);
    k_f32_to_u8<<<g, 256, 0, st>>>(src, dst, n);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

static int g_ssim_ctas[2] = {0, 0};   // resident CTAs per SM x SMs, for the forward and the backward

int loss_init()
{
    if (cudaFuncSetAttribute(k_ssim_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsimFwdSmem) != cudaSuccess)
        return DG_ERR_CUDA;
    if (cudaFuncSetAttribute(k_ssim_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsimBwdSmem) != cudaSuccess)
        return DG_ERR_CUDA;
    int dev = 0, sms = 0, bf = 0, bb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bf, k_ssim_fwd, kSsimThreads, kSsimFwdSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bb, k_ssim_bwd, kSsimThreads, kSsimBwdSmem) != cudaSuccess)
        return DG_ERR_CUDA;
    g_ssim_ctas[0] = sms * (bf > 0 ? bf : 1);
    g_ssim_ctas[1] = sms * (bb > 0 ? bb : 1);
    return DG_OK;
}

static size_t sums_bytes(const dg_plan& plan) { return ((size_t)plan.n_views * sizeof(double) + 255) / 256 * 256; }

size_t loss_ws_bytes(const dg_plan& plan) { return sums_bytes(plan) + (size_t)9 * plan.n_pixels * sizeof(float); }

// ws may be NULL when w_ssim == 0
int launch_loss(const float* img, const float* tgt, const dg_camera* cams, const dg_plan& plan, float w_l1,
                float w_ssim, double* loss, float* grad, void* ws, cudaStream_t st)
{
    if (cudaMemsetAsync(loss, 0, (size_t)plan.n_views * sizeof(double), st) != cudaSuccess) return DG_ERR_CUDA;
    double* ssum = nullptr;
    if (w_ssim == 0.f) {
        int64_t nblk = (3 * (int64_t)plan.max_width * plan.max_height + 255) / 256;
        unsigned gx = (unsigned)(nblk < 2048 ? nblk : 2048);
        k_l1<<<dim3(gx, plan.n_views), 256, 0, st>>>(img, tgt, cams, w_l1, loss, grad);
        note_launch();
    } else {
        // SSIM forward (moments, map, partials), then one backward pass that
        // writes the whole gradient (L1 + SSIM terms) and the L1 sums
        ssum = (double*)ws;
        float* partial = (float*)((char*)ws + sums_bytes(plan));
        if (cudaMemsetAsync(ssum, 0, (size_t)plan.n_views * sizeof(double), st) != cudaSuccess) return DG_ERR_CUDA;
        Win g = gaussian_window();
        const int TX = (plan.max_width + kTW - 1) / kTW, TY = (plan.max_height + kTH - 1) / kTH;
        const int64_t n_work = 3 * (int64_t)plan.n_views * TX * TY;
        if (n_work >= (int64_t)1 << 31) return DG_ERR_INVALID;
        const int gf = (int)(n_work < g_ssim_ctas[0] ? n_work : g_ssim_ctas[0]);
        const int gb = (int)(n_work < g_ssim_ctas[1] ? n_work : g_ssim_ctas[1]);
        k_ssim_fwd<<<gf, kSsimThreads, kSsimFwdSmem, st>>>(img, tgt, cams, g, w_ssim, ssum, partial, TX, TY,
                                                            (int)n_work);
        k_ssim_bwd<<<gb, kSsimThreads, kSsimBwdSmem, st>>>(img, tgt, cams, g, w_l1, partial, grad, loss, TX, TY,
                                                            (int)n_work);
        note_launch(2);
    }
    k_loss_final<<<(plan.n_views + 127) / 128, 128, 0, st>>>(cams, plan.n_views, w_l1, w_ssim, ssum, loss);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg
