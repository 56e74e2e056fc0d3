// K5 blend_fwd and K7 blend_bwd: per-tile front-to-back alpha compositing
// (Sec. 3.1, Eq. 2) and its adjoint.
//
// One CTA per (view, tile) of 256 pixels with NW warps, the tiles taken in
// the work order dg_bin_sort leaves after the ranges (descending instance
// count, so the heavy tiles start first); each thread owns
// PPL = 8 / NW pixels of the tile (pixel q = tid + 32 NW k), so a thread's
// pixels share a column and need no coordinate registers.  Rounds of
// 32 NW S instances (S per thread) are staged in shared memory -- fetched
// into registers one round ahead so the gather overlaps compositing -- and
// every thread walks the round for all of its pixels: one set of
// shared-memory loads and one decision path serve PPL pixels.  The forward
// stops a tile as soon as every pixel has hit the transmittance cut.  The
// backward walks the tile back to front from the stored T_final and last
// index, recovering T_i = T_{i+1} / (1 - alpha_i) and the colour behind each
// instance by the recurrence B_{i-1} = c_i alpha_i + (1 - alpha_i) B_i (B =
// background behind the last composited instance), kept as its projection
// G . B on the pixel's dL/dpixel G, the only form the adjoint needs; each lane sums its
// pixels' gradients, the nine per-instance gradients are reduced across the
// warp by a shuffle reduce-scatter, and nine lanes add them to global
// memory (NW sets of atomics per instance and tile).
//
// The variant (NW in {1, 2, 4, 8}, S in {1, 2}) and the tile shape are
// chosen per workload by the autotuner (plan.raster_warps / raster_stage,
// and raster_warps_bwd / raster_stage_bwd for the backward).
#include "common.cuh"

namespace dg {

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

// Thread pixels: column tid % tw, rows tid / tw + k * (32 NW / tw).
struct LaneGeom {
    float fx, fy0, dy;
    int px, py0, dpy;
};

__device__ __forceinline__ LaneGeom lane_geom(const TileInfo& ti, int tw, int tid, int nthreads)
{
    LaneGeom L;
    L.px = ti.px0 + tid % tw;
    L.py0 = ti.py0 + tid / tw;
    L.dpy = nthreads / tw;
    L.fx = (float)L.px + 0.5f;
    L.fy0 = (float)L.py0 + 0.5f;
    L.dy = (float)L.dpy;
    return L;
}

// The exponent of alpha (log2 units) of one instance at pixel k of a
// thread's strip (fixed column fx, rows fy0 + k dy): e = p + log2 o with
// p = A dx^2 + B dx dy_k + C dy_k^2, dx = mx - fx and dy_k = (my - fy0) - k dy.
// It is evaluated for every pixel from its own dy_k by Horner's rule in
// dy_k, q = (C dy_k + B dx) dy_k + (A dx^2 + log2 o), the column terms formed
// once per instance (no expansion from the strip's first pixel, whose large
// terms would cancel near the Gaussian's centre).  The conic is positive
// definite, so p is never positive in exact arithmetic; a positive value is
// rounding and is taken as 0, i.e. e = min(q, log2 o).  A pair is
// composited when e >= kQMin = log2(1/255), the skip rule of Eq. 2 in the
// log domain; since every staged instance has log2 o >= kQMin, that is
// q >= kQMin, one test taken before 2^e is formed.  The forward and the
// backward evaluate q, e and alpha by the same instructions, so both take
// the same decisions.
struct Strip {
    float E0, Bdx, C, dy0, ddy;
};

__device__ __forceinline__ float strip_q(const Strip& s, int k)
{
    const float dy = __fmaf_rn(-(float)k, s.ddy, s.dy0);
    return __fmaf_rn(__fmaf_rn(s.C, dy, s.Bdx), dy, s.E0);
}

// the same with the row offset k dy given (k dy is exact, so dy0 - off rounds
// exactly as the fused multiply-add above); an offset of -kDeadRow moves a
// pixel so far from every instance that it fails q >= kQMin
constexpr float kDeadRow = 1e15f;
__device__ __forceinline__ float strip_q_off(const Strip& s, float off)
{
    const float dy = __fsub_rn(s.dy0, off);
    return __fmaf_rn(__fmaf_rn(s.C, dy, s.Bdx), dy, s.E0);
}

// q of every pixel of the strip, two pixels per paired instruction where PPL
// is even (each lane rounded exactly as strip_q / strip_q_off round).
// off == nullptr: row offsets k dy (strip_q); else off[k] (strip_q_off).
template <int PPL>
__device__ __forceinline__ void strip_q_all(const Strip& s, const float* off, float* q)
{
    if constexpr (PPL % 2 == 0) {
        const f32x2 C2 = f2_pack(s.C, s.C), B2 = f2_pack(s.Bdx, s.Bdx), E2 = f2_pack(s.E0, s.E0);
        const f32x2 D2 = f2_pack(s.dy0, s.dy0);
#pragma unroll
        for (int j = 0; j < PPL / 2; j++) {
            f32x2 dy;
            if (off)
                dy = f2_sub(D2, f2_pack(off[2 * j], off[2 * j + 1]));
            else
                dy = f2_fma(f2_pack(-(float)(2 * j), -(float)(2 * j + 1)), f2_pack(s.ddy, s.ddy), D2);
            const f32x2 qq = f2_fma(f2_fma(C2, dy, B2), dy, E2);
            f2_unpack(qq, q[2 * j], q[2 * j + 1]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < PPL; k++) q[k] = off ? strip_q_off(s, off[k]) : strip_q(s, k);
    }
}

template <int PPL>
__device__ __forceinline__ Strip strip_setup(float mx, float my, float A, float B, float C, float lo, float fx,
                                             float fy0, float ddy)
{
    Strip st;
    const float dx = __fsub_rn(mx, fx);
    st.E0 = __fmaf_rn(__fmul_rn(A, dx), dx, lo);
    st.Bdx = __fmul_rn(B, dx);
    st.C = C;
    st.dy0 = __fsub_rn(my, fy0);
    st.ddy = ddy;
    return st;
}

// 2^x by the SFU (PTX ex2.approx.ftz; x >= kQMin > -8 here, so no denormal result)
__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// alpha of a composited pair (q >= kQMin): 2^min(q, loc) with loc =
// min(log2 o, log2 0.99) staged per instance, i.e. min(o G, 0.99) with the
// clamp taken in the exponent (and a positive rounding of p taken as 0)
__device__ __forceinline__ float strip_alpha(float q, float loc) { return ex2(fminf(q, loc)); }

struct Fetch {
    float4 r0, r1, r2;
    uint32_t r;
};

__device__ __forceinline__ void fetch(const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
                                      uint32_t start, uint32_t idx, uint32_t lim, Fetch& f)
{
    if (idx < lim) {
        f.r = vals[start + idx];
        f.r0 = rec[3 * (int64_t)f.r];
        f.r1 = rec[3 * (int64_t)f.r + 1];
        f.r2 = rec[3 * (int64_t)f.r + 2];
    }
}

template <int NW>
__device__ __forceinline__ void cta_sync()
{
    if (NW == 1) __syncwarp(); else __syncthreads();
}

// CNT = true is the counting instantiation behind dg_rasterize_count: the same
// compositing, plus the number of (pixel, instance) pairs examined while the
// pixel was live and the number that contributed, added into counts[0..1].
template <int NW, int S, bool CNT = false>
__global__ void __launch_bounds__(32 * NW) k_raster_fwd(const float4* __restrict__ rec,
                                                        const uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ ranges,
                                                        const uint32_t* __restrict__ order,
                                                        const dg_camera* __restrict__ cams, int n_views, int tw,
                                                        int th, float bg0, float bg1, float bg2,
                                                        float* __restrict__ image, float* __restrict__ T_final,
                                                        uint32_t* __restrict__ last_out,
                                                        unsigned long long* __restrict__ counts)
{
    uint32_t n_seen = 0, n_used = 0;
    constexpr int NT = 32 * NW, PPL = 8 / NW, R = NT * S;
    __shared__ float4 s_g[R];   // mx, my, A, B
    __shared__ float2 s_h[R];   // C, log2 opacity
    __shared__ float4 s_c[R];   // colour
    const int tid = threadIdx.x;
    TileInfo ti;
    tile_info(cams, n_views, order[blockIdx.x], tw, th, ranges, ti);
    const LaneGeom G = lane_geom(ti, tw, tid, NT);
    float T[PPL], C0[PPL], C1[PPL], C2[PPL], off[PPL];
    uint32_t last[PPL];
    uint32_t live = 0;   // bit k: pixel k inside the image and not yet stopped
    // row offset of pixel k, or -kDeadRow once it is outside the image or
    // stopped: a dead pixel then fails the first test like a distant one,
    // with no per-pixel live test in the loop
#pragma unroll
    for (int k = 0; k < PPL; k++) {
        T[k] = 1.f; C0[k] = C1[k] = C2[k] = 0.f; last[k] = 0;
        off[k] = -kDeadRow;
        if (G.px < ti.W && G.py0 + k * G.dpy < ti.H) {
            live |= 1u << k;
            off[k] = (float)k * G.dy;
        }
    }
    const uint32_t n = ti.end - ti.start;
    Fetch nx[S];
#pragma unroll
    for (int s = 0; s < S; s++) fetch(rec, vals, ti.start, tid + s * NT, n, nx[s]);
    for (uint32_t base = 0; base < n; base += R) {
        bool all_done = NW == 1 ? !__any_sync(0xffffffffu, live != 0) : __syncthreads_count(live != 0) == 0;
        if (all_done) break;
#pragma unroll
        for (int s = 0; s < S; s++) {
            const int j = tid + s * NT;
            if (base + j < n) {
                Staged st = stage_geometry(nx[s].r0, nx[s].r1);
                s_g[j] = make_float4(st.mx, st.my, st.A, st.B);
                s_h[j] = make_float2(st.C, st.lo);
                s_c[j] = make_float4(nx[s].r1.z, nx[s].r1.w, nx[s].r2.x, fminf(st.lo, kLogAlphaMax));
            }
        }
        cta_sync<NW>();
#pragma unroll
        for (int s = 0; s < S; s++) fetch(rec, vals, ti.start, base + R + tid + s * NT, n, nx[s]);
        const uint32_t cnt = min((uint32_t)R, n - base);
        // stopped pixels fail the first test by their dead-row offset, so the
        // walk needs no per-instance live test (the round's vote ends the tile)
        for (uint32_t j = 0; j < cnt; j++) {
            const float4 g = s_g[j];
            const float2 h = s_h[j];
            if (CNT) n_seen += __popc(live);
            const Strip sp = strip_setup<PPL>(g.x, g.y, g.z, g.w, h.x, h.y, G.fx, G.fy0, G.dy);
            const float4 c = s_c[j];
            float qs[PPL];
            strip_q_all<PPL>(sp, off, qs);
#pragma unroll
            for (int k = 0; k < PPL; k++) {
                const float q = qs[k];
                if (!(q >= kQMin)) continue;
                const float a = strip_alpha(q, c.w);
                const float wt = a * T[k];
                const float Tn = T[k] - wt;                // T (1 - alpha), by the weight already formed
                if (Tn < kTMin) { live &= ~(1u << k); off[k] = -kDeadRow; continue; }
                C0[k] = fmaf(c.x, wt, C0[k]);
                C1[k] = fmaf(c.y, wt, C1[k]);
                C2[k] = fmaf(c.z, wt, C2[k]);
                T[k] = Tn;
                last[k] = base + j + 1;
                if (CNT) n_used++;
            }
        }
        cta_sync<NW>();
    }
    if (CNT) {
        n_seen = __reduce_add_sync(0xffffffffu, n_seen);
        n_used = __reduce_add_sync(0xffffffffu, n_used);
        if ((tid & 31) == 0) {
            atomicAdd(counts, (unsigned long long)n_seen);
            atomicAdd(counts + 1, (unsigned long long)n_used);
        }
    }
    const int64_t HW = (int64_t)ti.W * ti.H;
    float* im = image + 3 * ti.pix_off;
#pragma unroll
    for (int k = 0; k < PPL; k++) {
        int py = G.py0 + k * G.dpy;
        if (G.px >= ti.W || py >= ti.H) continue;
        int64_t p = (int64_t)py * ti.W + G.px;
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

// Per-pixel inputs of the backward that are read only when a pair
// contributes (dL/dpixel) or when a pixel joins the walk (last) live in
// shared memory, indexed by the pixel's slot q = tid + 32 NW k (conflict
// free: slot q is in bank tid % 32); T and the colour behind B, updated at
// every composited pair, stay in registers.  A pixel joins the back-to-front
// walk at position last - 1; each thread keeps a mask of its joined pixels
// and the next position at which another one joins, so the per-pair test is
// one bit.
// register budget: 24 resident single-warp CTAs per SM for NW = 1; for the
// wider variants 32 warps per SM with one staged instance per thread and 24
// with two (the budgets that compile without spilling)
#ifndef DG_BWD_CTAS_1W
#define DG_BWD_CTAS_1W 24   // measured best of 20, 24, 28
#endif
template <int NW, int S>
constexpr int bwd_min_blocks() { return NW == 1 ? DG_BWD_CTAS_1W : (S == 1 ? 32 : 24) / NW; }

// Where the backward's per-(instance, tile) gradient goes.  Accumulated:
// atomics into the record's 12 floats of drec.  Slots (deterministic mode,
// one warp per tile): a plain store into the (record, tile) slot
// slot_off[r] + (ty - y0) w + (tx - x0) of part (9 floats per slot), summed
// per record in a fixed order by k_slot_reduce afterwards.
struct SlotOut {
    const uint2* rect;
    const uint64_t* slot_off;
    float* part;
    uint64_t cap;
};

// The adjoint of one instance at the pixels of a thread's strip that
// composited it (bits of todo), back to front: T and G . B of each pixel
// stepped over the instance, the colour sums and the moments S0, S1, S2 of
// dL/dpower along the strip (dy_k = dy0 - k dy).  CLAMP: the instance may
// reach the 0.99 alpha clamp (exponent q at or above qc), where d alpha /
// d power is zero.
template <int PPL, int NT, bool CLAMP>
__device__ __forceinline__ void bwd_rows(uint32_t todo, const float* qk, const float4& c, float qc,
                                         const float4* s_Gl, int tid, float* T, float* Bg, float& c0, float& c1,
                                         float& c2, float& S0, float& S1, float& S2)
{
#pragma unroll
    for (int k = 0; k < PPL; k++) {
        if (!(todo >> k & 1u)) continue;
        const float a = strip_alpha(qk[k], c.w);
        const float4 Gk = s_Gl[tid + NT * k];
        const float Tj = T[k] * __fdividef(1.f, 1.f - a);
        const float wT = a * Tj;
        c0 = fmaf(Gk.x, wT, c0);
        c1 = fmaf(Gk.y, wT, c1);
        c2 = fmaf(Gk.z, wT, c2);
        // dL/dalpha = T_j (G . c - G . B); d alpha / d power = alpha below the clamp
        const float gd = fmaf(Gk.x, c.x, fmaf(Gk.y, c.y, fmaf(Gk.z, c.z, -Bg[k])));
        Bg[k] = fmaf(a, gd, Bg[k]);      // G . B <- a G . c + (1 - a) G . B
        T[k] = Tj;
        const float dLdp = (!CLAMP || qk[k] < qc) ? wT * gd : 0.f;
        S0 += dLdp;
        S1 = fmaf(dLdp, (float)k, S1);
        S2 = fmaf(dLdp, (float)(k * k), S2);
    }
}

template <int NW, int S, bool SLOT = false>
__global__ void __launch_bounds__(32 * NW, bwd_min_blocks<NW, S>()) k_raster_bwd(const float4* __restrict__ rec,
                                                        const uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ ranges,
                                                        const uint32_t* __restrict__ order,
                                                        const dg_camera* __restrict__ cams, int n_views, int tw,
                                                        int th, float bg0, float bg1, float bg2,
                                                        const float* __restrict__ T_final,
                                                        const uint32_t* __restrict__ last_in,
                                                        const float* __restrict__ dL_dimage,
                                                        float* __restrict__ drec, SlotOut so)
{
    static_assert(!SLOT || NW == 1, "slots take one warp per tile");
    constexpr int NT = 32 * NW, PPL = 8 / NW, R = NT * S;
    __shared__ float4 s_g[R];   // mx, my, A, B   (log2-scaled exponent)
    __shared__ float4 s_h[R];   // C, log2 o, 1 / o, record index (bits)
    __shared__ float4 s_k[R];   // conic a, b, c, -
    __shared__ float4 s_c[R];   // colour
    __shared__ float4 s_Gl[256];        // dL/dpixel (3) and last (bits) per slot
    __shared__ uint32_t s_max;
    const int tid = threadIdx.x, lane = tid & 31;
    TileInfo ti;
    tile_info(cams, n_views, order[blockIdx.x], tw, th, ranges, ti);
    const LaneGeom Lg = lane_geom(ti, tw, tid, NT);
    const int64_t HW = (int64_t)ti.W * ti.H;
    const float* gi = dL_dimage + 3 * ti.pix_off;
    // per pixel: T and, in place of the colour B behind the walk, its
    // projection Bg = G . B on the pixel's dL/dpixel G, the only form of B
    // the adjoint uses (dL/dalpha = T_j G . (c - B)); its recurrence
    // Bg <- alpha (G . c) + (1 - alpha) Bg follows from B's
    float T[PPL], Bg[PPL];
    uint32_t ml = 0;
#pragma unroll
    for (int k = 0; k < PPL; k++) {
        const int q = tid + NT * k;
        int py = Lg.py0 + k * Lg.dpy;
        T[k] = 1.f;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        uint32_t lk = 0;
        if (Lg.px < ti.W && py < ti.H) {
            int64_t p = (int64_t)py * ti.W + Lg.px;
            g0 = gi[p]; g1 = gi[HW + p]; g2 = gi[2 * HW + p];
            T[k] = T_final[ti.pix_off + p];
            lk = last_in[ti.pix_off + p];
        }
        Bg[k] = fmaf(g0, bg0, fmaf(g1, bg1, g2 * bg2));
        s_Gl[q] = make_float4(g0, g1, g2, __uint_as_float(lk));
        ml = max(ml, lk);
    }
    uint32_t maxlast = __reduce_max_sync(0xffffffffu, ml);
    if (NW > 1) {
        if (tid == 0) s_max = 0;
        __syncthreads();
        if (lane == 0 && maxlast) atomicMax(&s_max, maxlast);
        __syncthreads();
        maxlast = s_max;
    }
    if (maxlast == 0) return;
    // joined pixels: bit k set once the walk is below last[k]
    uint32_t joined = 0, next_join = ml;
    const int rounds = (int)((maxlast + R - 1) / R);
    Fetch nx[S];
#pragma unroll
    for (int s = 0; s < S; s++) fetch(rec, vals, ti.start, (uint32_t)(rounds - 1) * R + tid + s * NT, maxlast, nx[s]);
    for (int rd = rounds - 1; rd >= 0; rd--) {
        const uint32_t base = (uint32_t)rd * R;
        cta_sync<NW>();
#pragma unroll
        for (int s = 0; s < S; s++) {
            const int j = tid + s * NT;
            if (base + j < maxlast) {
                Staged st = stage_geometry(nx[s].r0, nx[s].r1);
                s_g[j] = make_float4(st.mx, st.my, st.A, st.B);
                s_h[j] = make_float4(st.C, st.lo, __frcp_rn(nx[s].r1.y), __uint_as_float(nx[s].r));
                // s_k.w: the exponent at and above which alpha is clamped
                // (kLogAlphaMax, or +inf for an instance whose opacity is below
                // 0.99: min(q, log2 o) >= kLogAlphaMax exactly when q >= it)
                s_k[j] = make_float4(nx[s].r0.z, nx[s].r0.w, nx[s].r1.x,
                                     st.lo >= kLogAlphaMax ? kLogAlphaMax : __int_as_float(0x7f800000));
                s_c[j] = make_float4(nx[s].r1.z, nx[s].r1.w, nx[s].r2.x, fminf(st.lo, kLogAlphaMax));
            }
        }
        cta_sync<NW>();
        if (rd > 0) {
#pragma unroll
            for (int s = 0; s < S; s++) fetch(rec, vals, ti.start, base - R + tid + s * NT, maxlast, nx[s]);
        }
        const int cnt = (int)min((uint32_t)R, maxlast - base);
        for (int j = cnt - 1; j >= 0; j--) {
            const uint32_t pos = base + (uint32_t)j;
            if (pos < next_join) {              // pixels whose last composited pair is at or after pos
                next_join = 0;
#pragma unroll
                for (int k = 0; k < PPL; k++) {
                    const uint32_t lk = __float_as_uint(s_Gl[tid + NT * k].w);
                    if (pos < lk) joined |= 1u << k;
                    else next_join = max(next_join, lk);
                }
            }
            const float4 g = s_g[j];
            const float4 h = s_h[j];
            const Strip sp = strip_setup<PPL>(g.x, g.y, g.z, g.w, h.x, h.y, Lg.fx, Lg.fy0, Lg.dy);
            // the first test for the whole strip, without branches
            float qk[PPL];
            strip_q_all<PPL>(sp, nullptr, qk);
            uint32_t reach = 0;
#pragma unroll
            for (int k = 0; k < PPL; k++) reach |= (uint32_t)(qk[k] >= kQMin) << k;
            const uint32_t todo = joined & reach;
            if (!__any_sync(0xffffffffu, todo != 0u)) continue;
            const float4 c = s_c[j];
            const float4 kc = s_k[j];
            // colour sums and the moments of dL/dpower along the strip:
            // S0 = sum dLdp, S1 = sum k dLdp, S2 = sum k^2 dLdp (dy_k = dy0 - k dy)
            float c0 = 0.f, c1 = 0.f, c2 = 0.f, S0 = 0.f, S1 = 0.f, S2 = 0.f;
            // an instance below 0.99 opacity (kc.w = +inf, nearly all) is never
            // clamped: its pixels take the adjoint without the clamp test
            if (kc.w == __int_as_float(0x7f800000))     // uniform over the warp
                bwd_rows<PPL, NT, false>(todo, qk, c, kc.w, s_Gl, tid, T, Bg, c0, c1, c2, S0, S1, S2);
            else
                bwd_rows<PPL, NT, true>(todo, qk, c, kc.w, s_Gl, tid, T, Bg, c0, c1, c2, S0, S1, S2);
            // power = -(a dx^2 + 2 b dx dy + c dy^2) / 2 with dx = mx - px,
            // dy = my - py; its gradients summed over the strip's pixels.  Every
            // lane forms them (the warp runs this for any lane with work); a lane
            // with no composited pixel has zero sums and gives (signed) zeros.
            float gr[8];
            {
                const float dx = g.x - Lg.fx, dy0 = g.y - Lg.fy0;
                const float Sy = fmaf(-Lg.dy, S1, dy0 * S0);                                  // sum dLdp dy
                const float Syy = fmaf(Lg.dy * Lg.dy, S2, fmaf(-2.f * dy0 * Lg.dy, S1, dy0 * dy0 * S0));  // sum dLdp dy^2
                gr[0] = -fmaf(kc.x * dx, S0, kc.y * Sy);
                gr[1] = -fmaf(kc.y * dx, S0, kc.z * Sy);
                gr[2] = -0.5f * dx * dx * S0;
                gr[3] = -dx * Sy;
                gr[4] = -0.5f * Syy;
                gr[5] = S0 * h.z;                       // d alpha / d opacity = alpha / opacity
                gr[6] = c0;
                gr[7] = c1;
            }
            float g8 = c2;
            const float sred = warp_reduce_scatter8(gr, g8, lane);
            const uint32_t rid = __float_as_uint(h.w);
            if (SLOT) {
                if ((lane & 3) == 0) {
                    const uint2 rr = so.rect[rid];
                    const uint32_t x0 = rr.x & 0xFFFFu, y0 = rr.x >> 16, w = (rr.y & 0xFFFFu) - x0;
                    const uint32_t tx = (uint32_t)(ti.px0 / tw), ty = (uint32_t)(ti.py0 / th);
                    const uint64_t slot = so.slot_off[rid] + (uint64_t)((ty - y0) * w + (tx - x0));
                    if (slot < so.cap) {
                        const int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                        so.part[9 * slot + vi] = sred;
                        if (lane == 0) so.part[9 * slot + 8] = g8;
                    }
                }
            } else {
                float* d = drec + 12 * (int64_t)rid;
                if ((lane & 3) == 0) {
                    const int vi = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
                    if (sred != 0.f) atomicAdd(d + vi, sred);
                }
                if (lane == 0 && g8 != 0.f) atomicAdd(d + 8, g8);
            }
        }
    }
}

template <int NW, int S>
static void fwd_launch(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                       const dg_plan& p, const float* bg, float* image, float* T_final, uint32_t* last,
                       cudaStream_t st)
{
    k_raster_fwd<NW, S><<<(unsigned)p.n_tiles, 32 * NW, 0, st>>>(rec, vals, ranges, ranges + 2 * p.n_tiles, cams,
                                                                 p.n_views, p.tile_w,
                                                                 p.tile_h, bg[0], bg[1], bg[2], image, T_final, last,
                                                                 nullptr);
}

template <int NW, int S>
static void count_launch(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                         const dg_plan& p, const float* bg, float* image, float* T_final, uint32_t* last,
                         unsigned long long* counts, cudaStream_t st)
{
    k_raster_fwd<NW, S, true><<<(unsigned)p.n_tiles, 32 * NW, 0, st>>>(rec, vals, ranges, ranges + 2 * p.n_tiles,
                                                                       cams, p.n_views,
                                                                       p.tile_w, p.tile_h, bg[0], bg[1], bg[2],
                                                                       image, T_final, last, counts);
}

template <int NW, int S>
static void bwd_launch(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                       const dg_plan& p, const float* bg, const float* T_final, const uint32_t* last,
                       const float* dL_dimage, float* drec, cudaStream_t st)
{
    k_raster_bwd<NW, S><<<(unsigned)p.n_tiles, 32 * NW, 0, st>>>(rec, vals, ranges, ranges + 2 * p.n_tiles, cams,
                                                                 p.n_views, p.tile_w,
                                                                 p.tile_h, bg[0], bg[1], bg[2], T_final, last,
                                                                 dL_dimage, drec, SlotOut{});
}

// once per device: the backward's shared-memory carveout at its maximum,
// so that every SM keeps room beside its CTAs for the persistent x-step
// that runs with it (dg_xstep_stream)
int raster_bwd_init()
{
    const int c = (int)cudaSharedmemCarveoutMaxShared;
    const cudaFuncAttribute at = cudaFuncAttributePreferredSharedMemoryCarveout;
    if (cudaFuncSetAttribute(k_raster_bwd<1, 1>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<1, 2>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<2, 1>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<2, 2>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<4, 1>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<4, 2>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<8, 1>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<8, 2>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<1, 1, true>, at, c) != cudaSuccess ||
        cudaFuncSetAttribute(k_raster_bwd<1, 2, true>, at, c) != cudaSuccess)
        return DG_ERR_CUDA;
    return DG_OK;
}

#define DG_RASTER_DISPATCH(P, FN, ...)                                       \
    switch (P.raster_warps * 10 + P.raster_stage) {                          \
    case 11: FN<1, 1>(__VA_ARGS__); break;                                   \
    case 12: FN<1, 2>(__VA_ARGS__); break;                                   \
    case 21: FN<2, 1>(__VA_ARGS__); break;                                   \
    case 22: FN<2, 2>(__VA_ARGS__); break;                                   \
    case 41: FN<4, 1>(__VA_ARGS__); break;                                   \
    case 42: FN<4, 2>(__VA_ARGS__); break;                                   \
    case 81: FN<8, 1>(__VA_ARGS__); break;                                   \
    case 82: FN<8, 2>(__VA_ARGS__); break;                                   \
    default: return DG_ERR_INVALID;                                          \
    }

int launch_raster_fwd(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                      const dg_plan& plan, const float* bg, float* image, float* T_final, uint32_t* last,
                      cudaStream_t st)
{
    if (plan.n_tiles == 0) return DG_OK;
    DG_RASTER_DISPATCH(plan, fwd_launch, rec, vals, ranges, cams, plan, bg, image, T_final, last, st)
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_raster_count(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                        const dg_plan& plan, const float* bg, float* image, float* T_final, uint32_t* last,
                        unsigned long long* counts, cudaStream_t st)
{
    if (cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), st) != cudaSuccess) return DG_ERR_CUDA;
    if (plan.n_tiles == 0) return DG_OK;
    DG_RASTER_DISPATCH(plan, count_launch, rec, vals, ranges, cams, plan, bg, image, T_final, last, counts, st)
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_raster_bwd(const float4* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* cams,
                      const dg_plan& plan, const float* bg, const float* T_final, const uint32_t* last,
                      const float* dL_dimage, float* drec, cudaStream_t st)
{
    if (plan.n_tiles == 0) return DG_OK;
    dg_plan pb = plan;   // the backward's own variant, if set
    if (plan.raster_warps_bwd != 0) {
        pb.raster_warps = plan.raster_warps_bwd;
        pb.raster_stage = plan.raster_stage_bwd;
    }
    DG_RASTER_DISPATCH(pb, bwd_launch, rec, vals, ranges, cams, pb, bg, T_final, last, dL_dimage, drec, st)
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// drec's 12 floats zeroed for the records with a non-empty rectangle (the
// only ones the compositing adjoint adds to and the projection adjoint
// reads); four records per thread, so four rectangle loads are in flight
constexpr int kZeroPer = 4;

__global__ void __launch_bounds__(256) k_zero_kept(const uint2* __restrict__ rect, int64_t n_rec,
                                                   float4* __restrict__ drec)
{
    const int64_t base = (int64_t)blockIdx.x * (256 * kZeroPer) + threadIdx.x;
    uint2 rr[kZeroPer];
#pragma unroll
    for (int j = 0; j < kZeroPer; j++) {
        const int64_t r = base + 256 * j;
        rr[j] = r < n_rec ? rect[r] : make_uint2(0, 0);
    }
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < kZeroPer; j++) {
        if ((rr[j].x & 0xFFFFu) == (rr[j].y & 0xFFFFu)) continue;
        const int64_t r = base + 256 * j;
        drec[3 * r] = z;
        drec[3 * r + 1] = z;
        drec[3 * r + 2] = z;
    }
}

int launch_zero_kept(const uint2* rect, int64_t n_rec, float* drec, cudaStream_t st)
{
    if (n_rec == 0) return DG_OK;
    const int64_t per = 256 * kZeroPer;
    k_zero_kept<<<(unsigned)((n_rec + per - 1) / per), 256, 0, st>>>(rect, n_rec, (float4*)drec);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// ---- deterministic mode: (record, tile) slots ---------------------------------------
// slot_off[r] = the sum of the rectangle areas (in tiles) of the records
// before r, by a three-pass scan (chunks of kSlotChunk records per CTA).
constexpr int kSlotT = 512, kSlotPer = 8, kSlotChunk = kSlotT * kSlotPer;

__device__ __forceinline__ uint32_t rect_area(uint2 rr)
{
    const uint32_t x0 = rr.x & 0xFFFFu, y0 = rr.x >> 16, x1 = rr.y & 0xFFFFu, y1 = rr.y >> 16;
    return (x1 > x0 && y1 > y0) ? (x1 - x0) * (y1 - y0) : 0u;
}

__device__ __forceinline__ uint64_t slot_block_scan(uint64_t v, uint64_t* s_warp, uint64_t& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = lane < nw ? s_warp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[nw - 1];
    const uint64_t before = wid > 0 ? s_warp[wid - 1] : 0ull;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kSlotT) k_slot_reduce_chunks(const uint2* __restrict__ rect, int64_t n,
                                                                uint64_t* __restrict__ partials)
{
    __shared__ uint64_t s_warp[32];
    const int64_t b = (int64_t)blockIdx.x * kSlotChunk + (int64_t)threadIdx.x * kSlotPer;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kSlotPer; i++)
        if (b + i < n) s += rect_area(rect[b + i]);
    uint64_t tot;
    slot_block_scan(s, s_warp, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kSlotT) k_slot_scan_top(uint64_t* __restrict__ partials, int64_t n_chunks,
                                                          int64_t cap, uint64_t* __restrict__ dev_slots,
                                                          uint32_t* __restrict__ dev_status)
{
    __shared__ uint64_t s_warp[32];
    uint64_t carry = 0;
    for (int64_t base = 0; base < n_chunks; base += kSlotT) {
        const int64_t i = base + threadIdx.x;
        const uint64_t v = i < n_chunks ? partials[i] : 0ull;
        uint64_t tot;
        const uint64_t ex = slot_block_scan(v, s_warp, tot);
        if (i < n_chunks) partials[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        *dev_slots = carry;
        if ((int64_t)carry > cap) atomicOr(dev_status, DG_STATUS_CAPACITY);
    }
}

__global__ void __launch_bounds__(kSlotT) k_slot_scan_down(const uint2* __restrict__ rect, int64_t n,
                                                           const uint64_t* __restrict__ partials,
                                                           uint64_t* __restrict__ slot_off)
{
    __shared__ uint64_t s_warp[32];
    const int64_t b = (int64_t)blockIdx.x * kSlotChunk + (int64_t)threadIdx.x * kSlotPer;
    uint32_t a[kSlotPer];
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kSlotPer; i++) {
        a[i] = b + i < n ? rect_area(rect[b + i]) : 0u;
        s += a[i];
    }
    uint64_t tot;
    uint64_t run = partials[blockIdx.x] + slot_block_scan(s, s_warp, tot);
#pragma unroll
    for (int i = 0; i < kSlotPer; i++)
        if (b + i < n) {
            slot_off[b + i] = run;
            run += a[i];
        }
}

// drec[r] = the sum of record r's slots in tile order (fixed, so the result
// does not depend on which tile's warp finished first); the three unused
// floats of each record are zeroed.
__global__ void __launch_bounds__(256) k_slot_reduce(const uint2* __restrict__ rect,
                                                     const uint64_t* __restrict__ slot_off,
                                                     const float* __restrict__ part, uint64_t cap, int64_t n,
                                                     float* __restrict__ drec)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t area = rect_area(rect[r]);
    const uint64_t so = slot_off[r];
    float acc[9];
#pragma unroll
    for (int v = 0; v < 9; v++) acc[v] = 0.f;
    if (so + area <= cap)
        for (uint32_t i = 0; i < area; i++) {
            const float* p = part + 9 * (so + i);
#pragma unroll
            for (int v = 0; v < 9; v++) acc[v] += p[v];
        }
    float4* d = reinterpret_cast<float4*>(drec + 12 * r);
    d[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
    d[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
    d[2] = make_float4(acc[8], 0.f, 0.f, 0.f);
}

size_t raster_slots_ws_bytes(int64_t n_rec)
{
    const int64_t n_chunks = (n_rec + kSlotChunk - 1) / kSlotChunk;
    return (size_t)(n_rec + n_chunks + 1) * sizeof(uint64_t) + 256;
}

int launch_raster_bwd_slots(const float4* rec, const uint2* rect, const uint32_t* vals, const uint32_t* ranges,
                            const dg_camera* cams, const dg_plan& plan, const float* bg, const float* T_final,
                            const uint32_t* last, const float* dL_dimage, float* part, int64_t cap, void* ws,
                            uint64_t* dev_slots, uint32_t* dev_status, float* drec, cudaStream_t st)
{
    const int64_t n = plan.n_rec;
    if (n == 0) return cudaMemsetAsync(dev_slots, 0, sizeof(uint64_t), st) == cudaSuccess ? DG_OK : DG_ERR_CUDA;
    uint64_t* slot_off = reinterpret_cast<uint64_t*>(ws);
    uint64_t* partials = slot_off + n;
    const int64_t n_chunks = (n + kSlotChunk - 1) / kSlotChunk;
    k_slot_reduce_chunks<<<(unsigned)n_chunks, kSlotT, 0, st>>>(rect, n, partials);
    k_slot_scan_top<<<1, kSlotT, 0, st>>>(partials, n_chunks, cap, dev_slots, dev_status);
    k_slot_scan_down<<<(unsigned)n_chunks, kSlotT, 0, st>>>(rect, n, partials, slot_off);
    if (cap > 0 && cudaMemsetAsync(part, 0, (size_t)cap * 9 * sizeof(float), st) != cudaSuccess) return DG_ERR_CUDA;
    note_launch(3);
    if (plan.n_tiles > 0) {
        const SlotOut so{rect, slot_off, part, (uint64_t)cap};
        const int S = plan.raster_warps_bwd != 0 ? plan.raster_stage_bwd : plan.raster_stage;
        if (S == 2)
            k_raster_bwd<1, 2, true><<<(unsigned)plan.n_tiles, 32, 0, st>>>(
                rec, vals, ranges, ranges + 2 * plan.n_tiles, cams, plan.n_views, plan.tile_w, plan.tile_h, bg[0], bg[1],
                bg[2], T_final, last,
                dL_dimage, drec, so);
        else
            k_raster_bwd<1, 1, true><<<(unsigned)plan.n_tiles, 32, 0, st>>>(
                rec, vals, ranges, ranges + 2 * plan.n_tiles, cams, plan.n_views, plan.tile_w, plan.tile_h, bg[0], bg[1],
                bg[2], T_final, last,
                dL_dimage, drec, so);
        note_launch();
    }
    k_slot_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rect, slot_off, part, (uint64_t)cap, n, drec);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg
