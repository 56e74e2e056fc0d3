// K6 / K11: the training loss of Eq. 3, L = w_l1 * L1 + w_ssim * (1 - SSIM),
// per view, with dL/d(image).
//
// SSIM: 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, zero
// padding, "same" size.  The forward computes the five local moments with a
// separable filter in shared memory (tile 32x16 plus a 5-pixel halo), the SSIM
// map, and the three per-pixel partials dS/d(mean_x), dS/d(E[x^2]),
// dS/d(E[xy]); the backward applies the same (symmetric) filter to those
// partials: dL/dx = F(a) + 2 x F(b) + y F(c).
#include "common.cuh"

namespace dg {

constexpr int kSW = 32, kSH = 16, kR = 5, kWin = 11;
constexpr int kInW = kSW + 2 * kR, kInH = kSH + 2 * kR;

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
// Separable filtering of NM maps held in shared memory (kInH x kInW) into
// kSH x kSW outputs; tmp is kInH x kSW per map.
template <int NM>
__device__ __forceinline__ void filter_tile(float (*in)[kInH][kInW], float (*tmp)[kInH][kSW], const Win& g,
                                            float out[][2])
{
    for (int i = threadIdx.x; i < kInH * kSW; i += blockDim.x) {
        int r = i / kSW, c = i % kSW;
#pragma unroll
        for (int m = 0; m < NM; m++) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; k++) s = fmaf(g.w[k], in[m][r][c + k], s);
            tmp[m][r][c] = s;
        }
    }
    __syncthreads();
    // each thread: column threadIdx.x % 32, rows (threadIdx.x / 32) + 8 * e
#pragma unroll
    for (int e = 0; e < 2; e++) {
        int c = threadIdx.x % kSW, r = threadIdx.x / kSW + 8 * e;
#pragma unroll
        for (int m = 0; m < NM; m++) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; k++) s = fmaf(g.w[k], tmp[m][r + k][c], s);
            out[m][e] = s;
        }
    }
}

__global__ void __launch_bounds__(256) k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  const dg_camera* __restrict__ cams, Win g, float w_ssim,
                                                  double* __restrict__ sums, float* __restrict__ partial)
{
    __shared__ float s_in[5][kInH][kInW];
    __shared__ float s_tmp[5][kInH][kSW];
    int v = blockIdx.z / 3, ch = blockIdx.z % 3;
    int W = __ldg(&cams[v].width), H = __ldg(&cams[v].height);
    int x0 = blockIdx.x * kSW, y0 = blockIdx.y * kSH;
    if (x0 >= W || y0 >= H) return;
    int64_t HW = (int64_t)W * H;
    int64_t pix = __ldg(&cams[v].pix_off);
    const float* X = img + 3 * pix + ch * HW;
    const float* Y = tgt + 3 * pix + ch * HW;
    for (int i = threadIdx.x; i < kInH * kInW; i += blockDim.x) {
        int r = i / kInW, c = i % kInW;
        int gx = x0 + c - kR, gy = y0 + r - kR;
        float a = 0.f, b = 0.f;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) { a = X[(int64_t)gy * W + gx]; b = Y[(int64_t)gy * W + gx]; }
        s_in[0][r][c] = a; s_in[1][r][c] = b;
        s_in[2][r][c] = a * a; s_in[3][r][c] = b * b; s_in[4][r][c] = a * b;
    }
    __syncthreads();
    float mo[5][2];
    filter_tile<5>(s_in, s_tmp, g, mo);
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float invN = 1.f / (float)(3 * HW);
    float acc = 0.f;
#pragma unroll
    for (int e = 0; e < 2; e++) {
        int c = threadIdx.x % kSW, r = threadIdx.x / kSW + 8 * e;
        int gx = x0 + c, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        float m1 = mo[0][e], m2 = mo[1][e];
        float s1 = mo[2][e] - m1 * m1, s2 = mo[3][e] - m2 * m2, s12 = mo[4][e] - m1 * m2;
        float A1 = 2.f * m1 * m2 + C1, A2 = 2.f * s12 + C2;
        float B1 = m1 * m1 + m2 * m2 + C1, B2 = s1 + s2 + C2;
        float iB = 1.f / (B1 * B2);
        float S = A1 * A2 * iB;
        acc += S;
        float dA1 = A2 * iB, dA2 = A1 * iB, dB1 = -S / B1, dB2 = -S / B2;
        float dm1 = 2.f * m2 * dA1 - 2.f * m2 * dA2 + 2.f * m1 * dB1 - 2.f * m1 * dB2;
        // loss term w_ssim * (1 - mean S): scale partials by -w_ssim / N
        float sc = -w_ssim * invN;
        int64_t p = (int64_t)gy * W + gx;
        float* P = partial + 9 * pix + 3 * ch * HW;
        P[p] = sc * dm1;
        P[HW + p] = sc * dB2;
        P[2 * HW + p] = sc * 2.f * dA2;
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

// dL/dx += F(a) + 2 x F(b) + y F(c), added onto the L1 gradient already in grad
__global__ void __launch_bounds__(256) k_ssim_bwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                  const dg_camera* __restrict__ cams, Win g,
                                                  const float* __restrict__ partial, float* __restrict__ grad)
{
    __shared__ float s_in[3][kInH][kInW];
    __shared__ float s_tmp[3][kInH][kSW];
    int v = blockIdx.z / 3, ch = blockIdx.z % 3;
    int W = __ldg(&cams[v].width), H = __ldg(&cams[v].height);
    int x0 = blockIdx.x * kSW, y0 = blockIdx.y * kSH;
    if (x0 >= W || y0 >= H) return;
    int64_t HW = (int64_t)W * H;
    int64_t pix = __ldg(&cams[v].pix_off);
    const float* P = partial + 9 * pix + 3 * ch * HW;
    for (int i = threadIdx.x; i < kInH * kInW; i += blockDim.x) {
        int r = i / kInW, c = i % kInW;
        int gx = x0 + c - kR, gy = y0 + r - kR;
        bool ok = gx >= 0 && gx < W && gy >= 0 && gy < H;
        int64_t p = (int64_t)gy * W + gx;
#pragma unroll
        for (int m = 0; m < 3; m++) s_in[m][r][c] = ok ? P[m * HW + p] : 0.f;
    }
    __syncthreads();
    float fo[3][2];
    filter_tile<3>(s_in, s_tmp, g, fo);
    const float* X = img + 3 * pix + ch * HW;
    const float* Y = tgt + 3 * pix + ch * HW;
    float* G = grad + 3 * pix + ch * HW;
#pragma unroll
    for (int e = 0; e < 2; e++) {
        int c = threadIdx.x % kSW, r = threadIdx.x / kSW + 8 * e;
        int gx = x0 + c, gy = y0 + r;
        if (gx >= W || gy >= H) continue;
        int64_t p = (int64_t)gy * W + gx;
        G[p] += fo[0][e] + 2.f * X[p] * fo[1][e] + Y[p] * fo[2][e];
    }
}

static size_t sums_bytes(const dg_plan& plan) { return ((size_t)plan.n_views * sizeof(double) + 255) / 256 * 256; }

size_t loss_ws_bytes(const dg_plan& plan) { return sums_bytes(plan) + (size_t)9 * plan.n_pixels * sizeof(float); }

// ws may be NULL when w_ssim == 0
int launch_loss(const float* img, const float* tgt, const dg_camera* cams, const dg_plan& plan, float w_l1,
                float w_ssim, double* loss, float* grad, void* ws, cudaStream_t st)
{
    if (cudaMemsetAsync(loss, 0, (size_t)plan.n_views * sizeof(double), st) != cudaSuccess) return DG_ERR_CUDA;
    int64_t nblk = (3 * (int64_t)plan.max_width * plan.max_height + 255) / 256;
    unsigned gx = (unsigned)(nblk < 2048 ? nblk : 2048);
    k_l1<<<dim3(gx, plan.n_views), 256, 0, st>>>(img, tgt, cams, w_l1, loss, grad);
    note_launch();
    double* ssum = nullptr;
    if (w_ssim != 0.f) {
        ssum = (double*)ws;
        float* partial = (float*)((char*)ws + sums_bytes(plan));
        if (cudaMemsetAsync(ssum, 0, (size_t)plan.n_views * sizeof(double), st) != cudaSuccess) return DG_ERR_CUDA;
        Win g = gaussian_window();
        dim3 grid((unsigned)((plan.max_width + kSW - 1) / kSW), (unsigned)((plan.max_height + kSH - 1) / kSH),
                  (unsigned)(3 * plan.n_views));
        k_ssim_fwd<<<grid, 256, 0, st>>>(img, tgt, cams, g, w_ssim, ssum, partial);
        k_ssim_bwd<<<grid, 256, 0, st>>>(img, tgt, cams, g, partial, grad);
        note_launch(2);
    }
    k_loss_final<<<(plan.n_views + 127) / 128, 128, 0, st>>>(cams, plan.n_views, w_l1, w_ssim, ssum, loss);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg
