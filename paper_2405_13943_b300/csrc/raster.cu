// K5 blend_fwd and K7 blend_bwd: per-tile front-to-back alpha compositing
// (Sec. 3.1, Eq. 2) and its adjoint.
//
// One warp per (view, tile) of 256 pixels, eight pixels per lane (pixel
// q = lane + 32 k of the tile, k = 0..7); four independent warps per CTA.
// Each warp stages 32 of its tile's instances at a time in its own slice of
// shared memory (one per lane, warp-synchronous: no CTA barrier) and walks
// them for all eight of its pixels, so one set of shared-memory loads and
// one per-instance decision serve 256 pixels.  The forward stops a warp as
// soon as all of its pixels have hit the transmittance cut.  The backward
// walks the tile back to front from the stored T_final and last index,
// recovering T_i = T_{i+1} / (1 - alpha_i) and the colour behind each
// instance by the recurrence B_{i-1} = c_i alpha_i + (1 - alpha_i) B_i
// (B = background behind the last composited instance); each lane sums its
// eight pixels' gradients, and the nine per-instance gradients are reduced
// across the warp by a shuffle reduce-scatter, then added to global memory
// by nine lanes -- one set of atomics per (instance, tile).
#include "common.cuh"

namespace dg {

constexpr int kWarps = 4;          // tiles per CTA
constexpr int kPPL = 8;            // pixels per lane
constexpr int kStage = 32;         // instances staged per warp per round

struct TileInfo {
    int v, W, H, px0, py0;
    int64_t pix_off;
    uint32_t start, end;
};

__device__ __forceinline__ void tile_info(const dg_camera* cams, int n_views, int64_t t, int tw, int th,
                                          const uint32_t* ranges, TileInfo& ti)
{
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

__global__ void __launch_bounds__(32 * kWarps) k_raster_fwd(const float4* __restrict__ rec,
                                                            const uint32_t* __restrict__ vals,
                                                            const uint32_t* __restrict__ ranges,
                                                            const dg_camera* __restrict__ cams, int n_views,
                                                            int64_t n_tiles, int tw, int th, float bg0, float bg1,
                                                            float bg2, float* __restrict__ image,
                                                            float* __restrict__ T_final,
                                                            uint32_t* __restrict__ last_out)
{
    __shared__ float4 s_g[kWarps][kStage];   // mx, my, A, B
    __shared__ float2 s_h[kWarps][kStage];   // C, log2 opacity
    __shared__ float4 s_c[kWarps][kStage];   // colour
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * kWarps + w;
    if (t >= n_tiles) return;
    TileInfo ti;
    tile_info(cams, n_views, t, tw, th, ranges, ti);
    float fx[kPPL], fy[kPPL], T[kPPL], C0[kPPL], C1[kPPL], C2[kPPL];
    uint32_t last[kPPL];
    uint32_t live = 0;   // bit k: pixel k inside the image and not yet stopped
#pragma unroll
    for (int k = 0; k < kPPL; k++) {
        int q = lane + 32 * k;
        int px = ti.px0 + q % tw, py = ti.py0 + q / tw;
        fx[k] = (float)px + 0.5f;
        fy[k] = (float)py + 0.5f;
        T[k] = 1.f; C0[k] = C1[k] = C2[k] = 0.f; last[k] = 0;
        if (px < ti.W && py < ti.H) live |= 1u << k;
    }
    const uint32_t n = ti.end - ti.start;
    for (uint32_t base = 0; base < n; base += kStage) {
        if (!__any_sync(0xffffffffu, live != 0)) break;
        uint32_t idx = base + lane;
        if (idx < n) {
            uint32_t r = vals[ti.start + idx];
            float4 r0 = rec[3 * (int64_t)r], r1 = rec[3 * (int64_t)r + 1], r2 = rec[3 * (int64_t)r + 2];
            Staged s = stage_geometry(r0, r1);
            s_g[w][lane] = make_float4(s.mx, s.my, s.A, s.B);
            s_h[w][lane] = make_float2(s.C, s.lo);
            s_c[w][lane] = make_float4(r1.z, r1.w, r2.x, 0.f);
        }
        __syncwarp();
        const uint32_t cnt = min((uint32_t)kStage, n - base);
        for (uint32_t j = 0; j < cnt && live; j++) {
            const float4 g = s_g[w][j];
            const float2 h = s_h[w][j];
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
            bool have_c = false;
#pragma unroll
            for (int k = 0; k < kPPL; k++) {
                if (!(live >> k & 1u)) continue;
                float dx, dy, raw;
                const float a = pair_alpha(g.x, g.y, g.z, g.w, h.x, h.y, fx[k], fy[k], dx, dy, raw);
                if (a == 0.f) continue;
                const float Tn = T[k] * (1.f - a);
                if (Tn < kTMin) { live &= ~(1u << k); continue; }
                if (!have_c) { c = s_c[w][j]; have_c = true; }
                const float wt = a * T[k];
                C0[k] = fmaf(c.x, wt, C0[k]);
                C1[k] = fmaf(c.y, wt, C1[k]);
                C2[k] = fmaf(c.z, wt, C2[k]);
                T[k] = Tn;
                last[k] = base + j + 1;
            }
        }
        __syncwarp();
    }
    const int64_t HW = (int64_t)ti.W * ti.H;
    float* im = image + 3 * ti.pix_off;
#pragma unroll
    for (int k = 0; k < kPPL; k++) {
        int q = lane + 32 * k;
        int px = ti.px0 + q % tw, py = ti.py0 + q / tw;
        if (px >= ti.W || py >= ti.H) continue;
        int64_t p = (int64_t)py * ti.W + px;
        im[p] = fmaf(T[k], bg0, C0[k]);
        im[HW + p] = fmaf(T[k], bg1, C1[k]);
        im[2 * HW + p] = fmaf(T[k], bg2, C2[k]);
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

__global__ void __launch_bounds__(32 * kWarps) k_raster_bwd(const float4* __restrict__ rec,
                                                            const uint32_t* __restrict__ vals,
                                                            const uint32_t* __restrict__ ranges,
                                                            const dg_camera* __restrict__ cams, int n_views,
                                                            int64_t n_tiles, int tw, int th, float bg0, float bg1,
                                                            float bg2, const float* __restrict__ T_final,
                                                            const uint32_t* __restrict__ last_in,
                                                            const float* __restrict__ dL_dimage,
                                                            float* __restrict__ drec)
{
    __shared__ float4 s_g[kWarps][kStage];   // mx, my, A, B   (log2-scaled exponent)
    __shared__ float4 s_h[kWarps][kStage];   // C, log2 o, 1 / o, record index (bits)
    __shared__ float4 s_k[kWarps][kStage];   // conic a, b, c, -
    __shared__ float4 s_c[kWarps][kStage];   // colour
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * kWarps + w;
    if (t >= n_tiles) return;
    TileInfo ti;
    tile_info(cams, n_views, t, tw, th, ranges, ti);
    const int64_t HW = (int64_t)ti.W * ti.H;
    const float* gi = dL_dimage + 3 * ti.pix_off;
    float fx[kPPL], fy[kPPL], T[kPPL], B0[kPPL], B1[kPPL], B2[kPPL], G0[kPPL], G1[kPPL], G2[kPPL];
    uint32_t last[kPPL];
    uint32_t ml = 0;
#pragma unroll
    for (int k = 0; k < kPPL; k++) {
        int q = lane + 32 * k;
        int px = ti.px0 + q % tw, py = ti.py0 + q / tw;
        fx[k] = (float)px + 0.5f;
        fy[k] = (float)py + 0.5f;
        T[k] = 1.f; G0[k] = G1[k] = G2[k] = 0.f; last[k] = 0;
        B0[k] = bg0; B1[k] = bg1; B2[k] = bg2;
        if (px < ti.W && py < ti.H) {
            int64_t p = (int64_t)py * ti.W + px;
            G0[k] = gi[p]; G1[k] = gi[HW + p]; G2[k] = gi[2 * HW + p];
            T[k] = T_final[ti.pix_off + p];
            last[k] = last_in[ti.pix_off + p];
            ml = max(ml, last[k]);
        }
    }
    const uint32_t maxlast = __reduce_max_sync(0xffffffffu, ml);
    if (maxlast == 0) return;
    const int rounds = (int)((maxlast + kStage - 1) / kStage);
    for (int rd = rounds - 1; rd >= 0; rd--) {
        const uint32_t base = (uint32_t)rd * kStage;
        const uint32_t idx = base + lane;
        __syncwarp();
        if (idx < maxlast) {
            uint32_t r = vals[ti.start + idx];
            float4 r0 = rec[3 * (int64_t)r], r1 = rec[3 * (int64_t)r + 1], r2 = rec[3 * (int64_t)r + 2];
            Staged s = stage_geometry(r0, r1);
            s_g[w][lane] = make_float4(s.mx, s.my, s.A, s.B);
            s_h[w][lane] = make_float4(s.C, s.lo, __frcp_rn(r1.y), __uint_as_float(r));
            s_k[w][lane] = make_float4(r0.z, r0.w, r1.x, 0.f);
            s_c[w][lane] = make_float4(r1.z, r1.w, r2.x, 0.f);
        }
        __syncwarp();
        const int cnt = (int)min((uint32_t)kStage, maxlast - base);
        for (int j = cnt - 1; j >= 0; j--) {
            const uint32_t pos = base + (uint32_t)j;
            const float4 g = s_g[w][j];
            const float4 h = s_h[w][j];
            float gr[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            float g8 = 0.f;
            bool any = false;
            float4 c = make_float4(0.f, 0.f, 0.f, 0.f), kc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < kPPL; k++) {
                if (pos >= last[k]) continue;
                float dx, dy, raw = 0.f;
                const float a = pair_alpha(g.x, g.y, g.z, g.w, h.x, h.y, fx[k], fy[k], dx, dy, raw);
                if (!(a > 0.f)) continue;
                if (!any) { c = s_c[w][j]; kc = s_k[w][j]; any = true; }
                const float Tj = T[k] * __fdividef(1.f, 1.f - a);
                const float wT = a * Tj;
                gr[6] = fmaf(G0[k], wT, gr[6]);
                gr[7] = fmaf(G1[k], wT, gr[7]);
                g8 = fmaf(G2[k], wT, g8);
                const float dLda = Tj * (G0[k] * (c.x - B0[k]) + G1[k] * (c.y - B1[k]) + G2[k] * (c.z - B2[k]));
                const float om = 1.f - a;
                B0[k] = fmaf(c.x, a, om * B0[k]);
                B1[k] = fmaf(c.y, a, om * B1[k]);
                B2[k] = fmaf(c.z, a, om * B2[k]);
                T[k] = Tj;
                if (raw < kAlphaMax) {
                    const float dLdp = dLda * a;             // d alpha / d power = alpha
                    gr[5] = fmaf(dLdp, h.z, gr[5]);         // d alpha / d opacity = alpha / opacity
                    gr[0] = fmaf(-dLdp, kc.x * dx + kc.y * dy, gr[0]);
                    gr[1] = fmaf(-dLdp, kc.y * dx + kc.z * dy, gr[1]);
                    gr[2] = fmaf(-0.5f * dLdp, dx * dx, gr[2]);
                    gr[3] = fmaf(-dLdp, dx * dy, gr[3]);
                    gr[4] = fmaf(-0.5f * dLdp, dy * dy, gr[4]);
                }
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const float s = warp_reduce_scatter8(gr, g8, lane);
            float* d = drec + 12 * (int64_t)__float_as_uint(h.w);
            if ((lane & 3) == 0) {
                const int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                if (s != 0.f) atomicAdd(d + vi, s);
            }
            if (lane == 0 && g8 != 0.f) atomicAdd(d + 8, g8);
        }
    }
}

int launch_raster_fwd(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                      const dg_plan& plan, const float* bg, float* image, float* T_final, uint32_t* last,
                      cudaStream_t st)
{
    if (plan.n_tiles == 0) return DG_OK;
    unsigned grid = (unsigned)((plan.n_tiles + kWarps - 1) / kWarps);
    k_raster_fwd<<<grid, 32 * kWarps, 0, st>>>(rec, vals, ranges, cams, plan.n_views, plan.n_tiles, plan.tile_w,
                                                plan.tile_h, bg[0], bg[1], bg[2], image, T_final, last);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_raster_bwd(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                      const dg_plan& plan, const float* bg, const float* T_final, const uint32_t* last,
                      const float* dL_dimage, float* drec, cudaStream_t st)
{
    if (plan.n_tiles == 0) return DG_OK;
    unsigned grid = (unsigned)((plan.n_tiles + kWarps - 1) / kWarps);
    k_raster_bwd<<<grid, 32 * kWarps, 0, st>>>(rec, vals, ranges, cams, plan.n_views, plan.n_tiles, plan.tile_w,
                                                plan.tile_h, bg[0], bg[1], bg[2], T_final, last, dL_dimage, drec);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg
