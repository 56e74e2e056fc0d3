// K5 blend_fwd and K7 blend_bwd: per-tile front-to-back alpha compositing
// (Sec. 3.1, Eq. 2) and its adjoint.
//
// One CTA of 128 threads per (view, tile) of 256 pixels; each thread owns two
// pixels of the tile (rows r and r + tile_h / 2).  Batches of 256 of the
// tile's instances are staged in shared memory (two per thread per batch);
// each thread then walks the batch for both of its pixels, so one set of
// shared-memory loads serves two pixels.  The forward stops a tile as soon as
// every pixel's transmittance has hit the cut.  The backward walks each tile
// back to front from the stored T_final and last index, recovering
// T_i = T_{i+1} / (1 - alpha_i) and the colour behind each instance by the
// recurrence B_{i-1} = c_i alpha_i + (1 - alpha_i) B_i (B = background behind
// the last composited instance); each lane sums its two pixels' gradients,
// and the nine per-instance gradients are reduced across the warp by a
// shuffle reduce-scatter before one set of global atomics per warp.
#include "common.cuh"

namespace dg {

constexpr int kRasterThreads = 128;   // two pixels per thread, tile_w * tile_h == 256
constexpr int kBatch = 256;           // instances staged per round

struct TileInfo {
    int v, W, H, px0, py0;
    int64_t pix_off;
    uint32_t start, end;
};

__device__ __forceinline__ void tile_info(const dg_camera* cams, int n_views, int tw, const uint32_t* ranges,
                                          int th, TileInfo& ti)
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

struct Pix {
    int px, py;
    float fx, fy;
    bool inside;
};

__device__ __forceinline__ Pix pixel_of(const TileInfo& ti, int tw, int q)
{
    Pix p;
    p.px = ti.px0 + q % tw;
    p.py = ti.py0 + q / tw;
    p.inside = p.px < ti.W && p.py < ti.H;
    p.fx = (float)p.px + 0.5f;
    p.fy = (float)p.py + 0.5f;
    return p;
}

__global__ void __launch_bounds__(kRasterThreads) k_raster_fwd(const float4* __restrict__ rec,
                                                               const uint32_t* __restrict__ vals,
                                                               const uint32_t* __restrict__ ranges,
                                                               const dg_camera* __restrict__ cams, int n_views,
                                                               int tw, int th, float bg0, float bg1, float bg2,
                                                               float* __restrict__ image, float* __restrict__ T_final,
                                                               uint32_t* __restrict__ last_out)
{
    __shared__ float4 s_g[kBatch];   // mx, my, A, B
    __shared__ float2 s_h[kBatch];   // C, log2 opacity
    __shared__ float4 s_c[kBatch];   // colour
    TileInfo ti;
    tile_info(cams, n_views, tw, ranges, th, ti);
    Pix P[2] = {pixel_of(ti, tw, threadIdx.x), pixel_of(ti, tw, threadIdx.x + kRasterThreads)};
    float T[2] = {1.f, 1.f}, C[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    uint32_t last[2] = {0, 0};
    bool done[2] = {!P[0].inside, !P[1].inside};
    uint32_t n = ti.end - ti.start;
    for (uint32_t base = 0; base < n; base += kBatch) {
        if (__syncthreads_count(done[0] && done[1]) == kRasterThreads) break;
#pragma unroll
        for (int k = 0; k < kBatch / kRasterThreads; k++) {
            uint32_t idx = base + threadIdx.x + k * kRasterThreads;
            if (idx < n) {
                uint32_t r = vals[ti.start + idx];
                float4 r0 = rec[3 * (int64_t)r], r1 = rec[3 * (int64_t)r + 1], r2 = rec[3 * (int64_t)r + 2];
                Staged s = stage_geometry(r0, r1);
                int j = threadIdx.x + k * kRasterThreads;
                s_g[j] = make_float4(s.mx, s.my, s.A, s.B);
                s_h[j] = make_float2(s.C, s.lo);
                s_c[j] = make_float4(r1.z, r1.w, r2.x, 0.f);
            }
        }
        __syncthreads();
        if (!(done[0] && done[1])) {
            uint32_t cnt = min((uint32_t)kBatch, n - base);
            for (uint32_t j = 0; j < cnt; j++) {
                float4 g = s_g[j];
                float2 h = s_h[j];
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    if (done[k]) continue;
                    float dx, dy, raw;
                    float a = pair_alpha(g.x, g.y, g.z, g.w, h.x, h.y, P[k].fx, P[k].fy, dx, dy, raw);
                    if (a == 0.f) continue;
                    float Tn = T[k] * (1.f - a);
                    if (Tn < kTMin) { done[k] = true; continue; }
                    float4 c = s_c[j];
                    float w = a * T[k];
                    C[k][0] = fmaf(c.x, w, C[k][0]);
                    C[k][1] = fmaf(c.y, w, C[k][1]);
                    C[k][2] = fmaf(c.z, w, C[k][2]);
                    T[k] = Tn;
                    last[k] = base + j + 1;
                }
                if (done[0] && done[1]) break;
            }
        }
    }
    int64_t HW = (int64_t)ti.W * ti.H;
    float* im = image + 3 * ti.pix_off;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        if (!P[k].inside) continue;
        int64_t p = (int64_t)P[k].py * ti.W + P[k].px;
        im[p] = fmaf(T[k], bg0, C[k][0]);
        im[HW + p] = fmaf(T[k], bg1, C[k][1]);
        im[2 * HW + p] = fmaf(T[k], bg2, C[k][2]);
        T_final[ti.pix_off + p] = T[k];
        last_out[ti.pix_off + p] = last[k];
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

struct BwdPix {
    float T, B0, B1, B2, g0, g1, g2;
    uint32_t last;
};

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
    __shared__ float4 s_g[kBatch];   // mx, my, A, B   (log2-scaled exponent)
    __shared__ float4 s_h[kBatch];   // C, log2 o, 1 / o, -
    __shared__ float4 s_k[kBatch];   // conic a, b, c, -
    __shared__ float4 s_c[kBatch];   // colour
    __shared__ uint32_t s_rid[kBatch];
    __shared__ uint32_t s_maxlast;
    TileInfo ti;
    tile_info(cams, n_views, tw, ranges, th, ti);
    int lane = threadIdx.x & 31;
    Pix P[2] = {pixel_of(ti, tw, threadIdx.x), pixel_of(ti, tw, threadIdx.x + kRasterThreads)};
    BwdPix S[2];
    int64_t HW = (int64_t)ti.W * ti.H;
    const float* gi = dL_dimage + 3 * ti.pix_off;
    if (threadIdx.x == 0) s_maxlast = 0;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        S[k].T = 1.f; S[k].g0 = S[k].g1 = S[k].g2 = 0.f; S[k].last = 0;
        S[k].B0 = bg0; S[k].B1 = bg1; S[k].B2 = bg2;
        if (P[k].inside) {
            int64_t p = (int64_t)P[k].py * ti.W + P[k].px;
            S[k].g0 = gi[p]; S[k].g1 = gi[HW + p]; S[k].g2 = gi[2 * HW + p];
            S[k].T = T_final[ti.pix_off + p];
            S[k].last = last_in[ti.pix_off + p];
        }
    }
    __syncthreads();
    uint32_t ml = max(S[0].last, S[1].last);
    if (ml) atomicMax(&s_maxlast, ml);
    __syncthreads();
    uint32_t maxlast = s_maxlast;
    if (maxlast == 0) return;
    int rounds = (int)((maxlast + kBatch - 1) / kBatch);
    for (int rd = rounds - 1; rd >= 0; rd--) {
        uint32_t base = (uint32_t)rd * kBatch;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kBatch / kRasterThreads; k++) {
            uint32_t idx = base + threadIdx.x + k * kRasterThreads;
            if (idx < maxlast) {
                uint32_t r = vals[ti.start + idx];
                float4 r0 = rec[3 * (int64_t)r], r1 = rec[3 * (int64_t)r + 1], r2 = rec[3 * (int64_t)r + 2];
                Staged s = stage_geometry(r0, r1);
                int j = threadIdx.x + k * kRasterThreads;
                s_g[j] = make_float4(s.mx, s.my, s.A, s.B);
                s_h[j] = make_float4(s.C, s.lo, __frcp_rn(r1.y), 0.f);
                s_k[j] = make_float4(r0.z, r0.w, r1.x, 0.f);
                s_c[j] = make_float4(r1.z, r1.w, r2.x, 0.f);
                s_rid[j] = r;
            }
        }
        __syncthreads();
        int cnt = (int)min((uint32_t)kBatch, maxlast - base);
        for (int j = cnt - 1; j >= 0; j--) {
            uint32_t pos = base + (uint32_t)j;
            float4 g = s_g[j];
            float4 h = s_h[j];
            float a[2] = {0.f, 0.f}, raw[2] = {0.f, 0.f}, dx[2] = {0.f, 0.f}, dy[2] = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 2; k++)
                if (pos < S[k].last) a[k] = pair_alpha(g.x, g.y, g.z, g.w, h.x, h.y, P[k].fx, P[k].fy, dx[k], dy[k], raw[k]);
            bool any = a[0] > 0.f || a[1] > 0.f;
            if (!__any_sync(0xffffffffu, any)) continue;
            float gr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            float g8 = 0.f;
            if (any) {
                float4 c = s_c[j];
                float4 kc = s_k[j];
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    if (!(a[k] > 0.f)) continue;
                    float ak = a[k];
                    float Tj = S[k].T * __fdividef(1.f, 1.f - ak);
                    float wT = ak * Tj;
                    gr[6] = fmaf(S[k].g0, wT, gr[6]);
                    gr[7] = fmaf(S[k].g1, wT, gr[7]);
                    g8 = fmaf(S[k].g2, wT, g8);
                    float dLda = Tj * (S[k].g0 * (c.x - S[k].B0) + S[k].g1 * (c.y - S[k].B1) + S[k].g2 * (c.z - S[k].B2));
                    float om = 1.f - ak;
                    S[k].B0 = fmaf(c.x, ak, om * S[k].B0);
                    S[k].B1 = fmaf(c.y, ak, om * S[k].B1);
                    S[k].B2 = fmaf(c.z, ak, om * S[k].B2);
                    S[k].T = Tj;
                    if (raw[k] < kAlphaMax) {
                        float dLdp = dLda * ak;              // d alpha / d power = alpha
                        float ddx = dx[k], ddy = dy[k];
                        gr[5] = fmaf(dLdp, h.z, gr[5]);      // d alpha / d opacity = alpha / opacity
                        gr[0] = fmaf(-dLdp, kc.x * ddx + kc.y * ddy, gr[0]);
                        gr[1] = fmaf(-dLdp, kc.y * ddx + kc.z * ddy, gr[1]);
                        gr[2] = fmaf(-0.5f * dLdp, ddx * ddx, gr[2]);
                        gr[3] = fmaf(-dLdp, ddx * ddy, gr[3]);
                        gr[4] = fmaf(-0.5f * dLdp, ddy * ddy, gr[4]);
                    }
                }
            }
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
