// K5 blend_fwd and K7 blend_bwd: per-tile front-to-back alpha compositing
// (Sec. 3.1, Eq. 2) and its adjoint.
//
// One CTA per (view, tile).  Batches of the tile's instances are staged in
// shared memory (one record per thread per batch); each thread then walks
// the batch for its pixel(s).  The forward stops a tile as soon as every
// pixel's transmittance has hit the cut.  The backward walks each tile back
// to front starting from the stored T_final and last index, recovering
// T_i = T_{i+1} / (1 - alpha_i) and the colour behind each instance by the
// recurrence B_{i-1} = c_i alpha_i + (1 - alpha_i) B_i (B = background behind
// the last composited instance), and reduces the nine per-record gradients
// across the warp (reduce-scatter by shuffles) before the global atomics.
#include "common.cuh"

namespace dg {

constexpr int kRasterThreads = 256;   // one pixel per thread, tile_w * tile_h == 256

struct TileInfo {
    int v, W, H, px0, py0;
    int64_t pix_off;
    uint32_t start, end;
};

__device__ __forceinline__ void tile_info(const dg_camera* cams, int n_views, int tw, int th,
                                          const uint32_t* ranges, TileInfo& ti)
{
    int64_t t = blockIdx.x;
    int v = find_view_of_tile(cams, n_views, t);
    int64_t local = t - __ldg(&cams[v].tile_off);
    int TX = __ldg(&cams[v].tiles_x);
    ti.v = v;
    ti.W = __ldg(&cams[v].width);
    ti.H = __ldg(&cams[v].height);
    ti.px0 = (int)(local % TX) * tw;
    ti.py0 = (int)(local / TX) * th;
    ti.pix_off = __ldg(&cams[v].pix_off);
    ti.start = ranges[2 * t];
    ti.end = ranges[2 * t + 1];
}

__global__ void __launch_bounds__(kRasterThreads) k_raster_fwd(const float4* __restrict__ rec,
                                                               const uint32_t* __restrict__ vals,
                                                               const uint32_t* __restrict__ ranges,
                                                               const dg_camera* __restrict__ cams, int n_views,
                                                               int tw, int th, float bg0, float bg1, float bg2,
                                                               float* __restrict__ image, float* __restrict__ T_final,
                                                               uint32_t* __restrict__ last_out)
{
    __shared__ float4 s_g[kRasterThreads];   // mx, my, A, B
    __shared__ float2 s_h[kRasterThreads];   // C, log2 opacity
    __shared__ float4 s_c[kRasterThreads];   // colour
    TileInfo ti;
    tile_info(cams, n_views, tw, th, ranges, ti);
    int lx = threadIdx.x % tw, ly = threadIdx.x / tw;
    int px = ti.px0 + lx, py = ti.py0 + ly;
    bool inside = px < ti.W && py < ti.H;
    float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    uint32_t n = ti.end - ti.start;
    for (uint32_t base = 0; base < n; base += kRasterThreads) {
        if (__syncthreads_count(done) == kRasterThreads) break;
        uint32_t idx = base + threadIdx.x;
        if (idx < n) {
            uint32_t r = vals[ti.start + idx];
            float4 r0 = rec[3 * (int64_t)r], r1 = rec[3 * (int64_t)r + 1], r2 = rec[3 * (int64_t)r + 2];
            Staged s = stage_geometry(r0, r1);
            s_g[threadIdx.x] = make_float4(s.mx, s.my, s.A, s.B);
            s_h[threadIdx.x] = make_float2(s.C, s.lo);
            s_c[threadIdx.x] = make_float4(r1.z, r1.w, r2.x, 0.f);
        }
        __syncthreads();
        if (!done) {
            uint32_t cnt = min((uint32_t)kRasterThreads, n - base);
            for (uint32_t j = 0; j < cnt; j++) {
                float4 g = s_g[j];
                float2 h = s_h[j];
                float dx, dy, raw;
                float a = pair_alpha(g.x, g.y, g.z, g.w, h.x, h.y, fpx, fpy, dx, dy, raw);
                if (a == 0.f) continue;
                float Tn = T * (1.f - a);
                if (Tn < kTMin) { done = true; break; }
                float4 c = s_c[j];
                float w = a * T;
                C0 = fmaf(c.x, w, C0);
                C1 = fmaf(c.y, w, C1);
                C2 = fmaf(c.z, w, C2);
                T = Tn;
                last = base + j + 1;
            }
        }
    }
    if (inside) {
        int64_t HW = (int64_t)ti.W * ti.H;
        int64_t p = (int64_t)py * ti.W + px;
        float* im = image + 3 * ti.pix_off;
        im[p] = fmaf(T, bg0, C0);
        im[HW + p] = fmaf(T, bg1, C1);
        im[2 * HW + p] = fmaf(T, bg2, C2);
        T_final[ti.pix_off + p] = T;
        last_out[ti.pix_off + p] = last;
    }
}

// Sum v[0..7] and v8 over the warp; lane L with (L & 3) == 0 ends up holding
// the total of value index ((L >> 4) & 1) * 4 + ((L >> 3) & 1) * 2 + ((L >> 2) & 1),
// lane 0 also holds the total of v8.
__device__ __forceinline__ float warp_reduce_scatter8(const float* v, float& v8, int lane)
{
    float w[4], u[2];
    bool hi = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float send = hi ? v[i] : v[4 + i];
        float keep = hi ? v[4 + i] : v[i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    hi = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        float send = hi ? w[i] : w[2 + i];
        float keep = hi ? w[2 + i] : w[i];
        u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    hi = lane & 4;
    float s = (hi ? u[1] : u[0]) + __shfl_xor_sync(0xffffffffu, hi ? u[0] : u[1], 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v8 += __shfl_xor_sync(0xffffffffu, v8, o);
    return s;
}

__global__ void __launch_bounds__(kRasterThreads) k_raster_bwd(const float4* __restrict__ rec,
                                                               const uint32_t* __restrict__ vals,
                                                               const uint32_t* __restrict__ ranges,
                                                               const dg_camera* __restrict__ cams, int n_views,
                                                               int tw, int th, float bg0, float bg1, float bg2,
                                                               const float* __restrict__ T_final,
                                                               const uint32_t* __restrict__ last_in,
                                                               const float* __restrict__ dL_dimage,
                                                               float* __restrict__ drec)
{
    __shared__ float4 s_g[kRasterThreads];   // mx, my, A, B   (log2-scaled exponent)
    __shared__ float4 s_h[kRasterThreads];   // C, log2 o, o, -
    __shared__ float4 s_k[kRasterThreads];   // conic a, b, c, -
    __shared__ float4 s_c[kRasterThreads];   // colour
    __shared__ uint32_t s_rid[kRasterThreads];
    __shared__ uint32_t s_maxlast;
    TileInfo ti;
    tile_info(cams, n_views, tw, th, ranges, ti);
    int lane = threadIdx.x & 31;
    int lx = threadIdx.x % tw, ly = threadIdx.x / tw;
    int px = ti.px0 + lx, py = ti.py0 + ly;
    bool inside = px < ti.W && py < ti.H;
    float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t last = 0;
    if (threadIdx.x == 0) s_maxlast = 0;
    if (inside) {
        int64_t HW = (int64_t)ti.W * ti.H;
        int64_t p = (int64_t)py * ti.W + px;
        const float* gi = dL_dimage + 3 * ti.pix_off;
        g0 = gi[p]; g1 = gi[HW + p]; g2 = gi[2 * HW + p];
        T = T_final[ti.pix_off + p];
        last = last_in[ti.pix_off + p];
    }
    __syncthreads();
    if (last) atomicMax(&s_maxlast, last);
    __syncthreads();
    uint32_t maxlast = s_maxlast;
    float B0 = bg0, B1 = bg1, B2 = bg2;   // colour behind, normalised by the transmittance in front of it
    if (maxlast == 0) return;
    int rounds = (int)((maxlast + kRasterThreads - 1) / kRasterThreads);
    for (int rd = rounds - 1; rd >= 0; rd--) {
        uint32_t base = (uint32_t)rd * kRasterThreads;
        uint32_t idx = base + threadIdx.x;
        __syncthreads();
        if (idx < maxlast) {
            uint32_t r = vals[ti.start + idx];
            float4 r0 = rec[3 * (int64_t)r], r1 = rec[3 * (int64_t)r + 1], r2 = rec[3 * (int64_t)r + 2];
            Staged s = stage_geometry(r0, r1);
            s_g[threadIdx.x] = make_float4(s.mx, s.my, s.A, s.B);
            s_h[threadIdx.x] = make_float4(s.C, s.lo, r1.y, 0.f);
            s_k[threadIdx.x] = make_float4(r0.z, r0.w, r1.x, 0.f);
            s_c[threadIdx.x] = make_float4(r1.z, r1.w, r2.x, 0.f);
            s_rid[threadIdx.x] = r;
        }
        __syncthreads();
        int cnt = (int)min((uint32_t)kRasterThreads, maxlast - base);
        for (int j = cnt - 1; j >= 0; j--) {
            uint32_t pos = base + (uint32_t)j;
            float gr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            float g8 = 0.f;
            bool contrib = false;
            if (pos < last) {
                float4 g = s_g[j];
                float4 h = s_h[j];
                float dx, dy, raw = 0.f;
                float a = pair_alpha(g.x, g.y, g.z, g.w, h.x, h.y, fpx, fpy, dx, dy, raw);
                if (a > 0.f) {
                    contrib = true;
                    float4 c = s_c[j];
                    float Tj = T / (1.f - a);
                    float wT = a * Tj;
                    gr[6] = g0 * wT;
                    gr[7] = g1 * wT;
                    g8 = g2 * wT;
                    float dLda = Tj * (g0 * (c.x - B0) + g1 * (c.y - B1) + g2 * (c.z - B2));
                    B0 = fmaf(c.x, a, (1.f - a) * B0);
                    B1 = fmaf(c.y, a, (1.f - a) * B1);
                    B2 = fmaf(c.z, a, (1.f - a) * B2);
                    T = Tj;
                    if (raw < kAlphaMax) {
                        float4 k = s_k[j];
                        float dLdp = dLda * a;             // d alpha / d power = alpha
                        gr[5] = dLda * a / h.z;            // d alpha / d opacity = G
                        gr[0] = -dLdp * (k.x * dx + k.y * dy);
                        gr[1] = -dLdp * (k.y * dx + k.z * dy);
                        gr[2] = -0.5f * dLdp * dx * dx;
                        gr[3] = -dLdp * dx * dy;
                        gr[4] = -0.5f * dLdp * dy * dy;
                    }
                }
            }
            if (!__any_sync(0xffffffffu, contrib)) continue;
            float s = warp_reduce_scatter8(gr, g8, lane);
            float* d = drec + 12 * (int64_t)s_rid[j];
            if ((lane & 3) == 0) {
                int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                atomicAdd(d + vi, s);
            }
            if (lane == 0) atomicAdd(d + 8, g8);
        }
    }
}

int launch_raster_fwd(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                      const dg_plan& plan, const float* bg, float* image, float* T_final, uint32_t* last,
                      cudaStream_t st)
{
    if (plan.n_tiles == 0) return DG_OK;
    k_raster_fwd<<<(unsigned)plan.n_tiles, kRasterThreads, 0, st>>>(rec, vals, ranges, cams, plan.n_views,
                                                                      plan.tile_w, plan.tile_h, bg[0], bg[1], bg[2],
                                                                      image, T_final, last);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_raster_bwd(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                      const dg_plan& plan, const float* bg, const float* T_final, const uint32_t* last,
                      const float* dL_dimage, float* drec, cudaStream_t st)
{
    if (plan.n_tiles == 0) return DG_OK;
    k_raster_bwd<<<(unsigned)plan.n_tiles, kRasterThreads, 0, st>>>(rec, vals, ranges, cams, plan.n_views,
                                                                      plan.tile_w, plan.tile_h, bg[0], bg[1], bg[2],
                                                                      T_final, last, dL_dimage, drec);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg
