// dg_probe_fma: the FP32 roofline denominator of the compositing kernels,
// measured on the device that runs them.  Every thread runs 8 independent
// chains of fused multiply-adds (a <- a * b + c, b just below 1 so the
// values stay finite); the caller times the launch and divides
// 2 x 8 x 16 x iters x threads FLOPs by its duration.  Nothing of the method
// runs here.
#include "common.cuh"

namespace dg {

constexpr int kProbeChains = 8, kProbeUnroll = 16;

__global__ void __launch_bounds__(256) k_probe_fma(int iters, float b, float c, float* __restrict__ out)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    float a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; k++) a[k] = 1.0f + 1e-3f * (float)k + 1e-9f * (float)gid;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; u++) {
#pragma unroll
            for (int k = 0; k < kProbeChains; k++) a[k] = __fmaf_rn(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kProbeChains; k++) s += a[k];
    out[gid] = s;
}

}  // namespace dg

extern "C" int64_t dg_probe_fma(int iters, int blocks, float* out, void* stream)
{
    using namespace dg;
    if (iters < 1 || blocks < 1 || !out || ((uintptr_t)out & 3u)) return -1;
    k_probe_fma<<<blocks, 256, 0, (cudaStream_t)stream>>>(iters, 0.99999994f, 1e-7f, out);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) return -1;
    return 2LL * kProbeChains * kProbeUnroll * (int64_t)iters * 256 * blocks;
}
