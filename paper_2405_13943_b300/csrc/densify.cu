// Densification under consensus (Sec. 4: densified at the intervals of 3DGS,
// with its adaptive density control; Sec. 5: small Gaussians pruned).
//
// Four data-parallel passes; the host orchestrates them right after a
// consensus and rebuilds the block layout from their output:
//   k_densify_stats   every iteration: for every kept record, the norm of
//                     its projected mean's gradient in normalised device
//                     units (pixels scaled by W/2, H/2), summed per copy with
//                     a count of the iterations it was seen;
//   k_densify_decide  per global Gaussian, from the statistics of all its
//                     copies (summed in the sharing map's order): prune if
//                     the opacity logit is below logit(min_opacity), else
//                     clone or split if sum >= grad_threshold * count (split
//                     when the largest log-scale is above
//                     log(percent_dense * extent)), else keep; its number of
//                     outputs (0, 1, 2, 2);
//   exclusive scan    of the output counts (three passes, no inter-CTA wait);
//   k_densify_emit    each Gaussian's outputs at its offset: itself, itself
//                     and a copy, or two children mu + R(q) (S xi) with
//                     scales S / 1.6 (xi drawn by the caller), and for every
//                     output its parent and whether it is the parent itself.
// k_gather_rows gathers parameter rows by index, the data movement of the
// rebuild.  All decisions are FP32 comparisons of the raw
// parameters against thresholds formed once on the host.
#include "common.cuh"

namespace dg {

constexpr int kDensifyThreads = 256;

__global__ void __launch_bounds__(kDensifyThreads) k_densify_stats(const uint2* __restrict__ rect,
                                                                   const float* __restrict__ drec,
                                                                   const dg_camera* __restrict__ cams, int n_views,
                                                                   int64_t n_rec, float* __restrict__ stats)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rec) return;
    const uint2 t = rect[r];
    if ((t.x & 0xFFFFu) == (t.y & 0xFFFFu)) return;              // not kept by the forward
    const int v = find_view_of_rec(cams, n_views, r);
    const int64_t c = __ldg(&cams[v].gauss_begin) + (r - __ldg(&cams[v].rec_off));
    const float gx = drec[12 * r] * (0.5f * (float)__ldg(&cams[v].width));
    const float gy = drec[12 * r + 1] * (0.5f * (float)__ldg(&cams[v].height));
    atomicAdd(&stats[2 * c], sqrtf(gx * gx + gy * gy));
    atomicAdd(&stats[2 * c + 1], 1.0f);
}

struct DensifyArgs {
    float grad_threshold, logit_min, log_big;
};

__global__ void __launch_bounds__(kDensifyThreads) k_densify_decide(GView z, const int64_t* __restrict__ g_off,
                                                                    const int32_t* __restrict__ g_copies,
                                                                    const float* __restrict__ stats, DensifyArgs a,
                                                                    int32_t* __restrict__ codes,
                                                                    uint32_t* __restrict__ counts)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.n) return;
    float ssum = 0.f, scnt = 0.f;
    for (int64_t e = g_off[i]; e < g_off[i + 1]; e++) {
        const int64_t c = g_copies[e];
        ssum = __fadd_rn(ssum, stats[2 * c]);
        scnt = __fadd_rn(scnt, stats[2 * c + 1]);
    }
    const float4 mo = z.mo[i], sc = z.scale[i];
    int32_t code;
    if (mo.w < a.logit_min) {
        code = DG_DENSIFY_PRUNE;
    } else if (scnt > 0.f && ssum >= __fmul_rn(a.grad_threshold, scnt)) {
        const float smax = fmaxf(fmaxf(sc.x, sc.y), sc.z);
        code = smax > a.log_big ? DG_DENSIFY_SPLIT : DG_DENSIFY_CLONE;
    } else {
        code = DG_DENSIFY_KEEP;
    }
    codes[i] = code;
    counts[i] = code == DG_DENSIFY_PRUNE ? 0u : (code == DG_DENSIFY_KEEP ? 1u : 2u);
}

// ---- exclusive scan of n uint32 counts (chunks of 4096 per CTA) ------------------
constexpr int kScanT = 1024, kScanPerT = 4, kScanChunkN = kScanT * kScanPerT;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    total = s_warp[31];
    const uint32_t before = wid > 0 ? s_warp[wid - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanT) k_dscan_reduce(const uint32_t* __restrict__ counts, int64_t n,
                                                         uint32_t* __restrict__ partials)
{
    __shared__ uint32_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunkN + (int64_t)threadIdx.x * kScanPerT;
    uint32_t v = 0;
#pragma unroll
    for (int i = 0; i < kScanPerT; i++) v += base + i < n ? counts[base + i] : 0u;
    uint32_t total;
    block_exclusive_scan(v, s_warp, total);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// one CTA: exclusive scan of the chunk totals in place, grand total at partials[n_chunks]
__global__ void __launch_bounds__(kScanT) k_dscan_top(uint32_t* __restrict__ partials, int64_t n_chunks)
{
    __shared__ uint32_t s_warp[32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < n_chunks; b += kScanT) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < n_chunks ? partials[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(v, s_warp, total);
        if (i < n_chunks) partials[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) partials[n_chunks] = carry;
}

__global__ void __launch_bounds__(kScanT) k_dscan_down(const uint32_t* __restrict__ counts, int64_t n,
                                                       const uint32_t* __restrict__ partials,
                                                       uint32_t* __restrict__ offsets)
{
    __shared__ uint32_t s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunkN + (int64_t)threadIdx.x * kScanPerT;
    uint32_t c[kScanPerT], v = 0;
#pragma unroll
    for (int i = 0; i < kScanPerT; i++) {
        c[i] = base + i < n ? counts[base + i] : 0u;
        v += c[i];
    }
    uint32_t total;
    uint32_t run = partials[blockIdx.x] + block_exclusive_scan(v, s_warp, total);
#pragma unroll
    for (int i = 0; i < kScanPerT; i++) {
        if (base + i < n) offsets[base + i] = run;
        run += c[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) offsets[n] = partials[gridDim.x];
}

// ---- emission ------------------------------------------------------------------------
__device__ __forceinline__ void copy_row(const GView& s, int64_t i, GView& d, int64_t o, int np)
{
    d.mo[o] = s.mo[i];
    d.quat[o] = s.quat[i];
    d.scale[o] = s.scale[i];
    for (int j = 0; j < np; j++) d.sh[(int64_t)j * d.ld + o] = s.sh[(int64_t)j * s.ld + i];
}

__global__ void __launch_bounds__(kDensifyThreads) k_densify_emit(GView z, const int32_t* __restrict__ codes,
                                                                  const uint32_t* __restrict__ offsets,
                                                                  const float* __restrict__ normals, GView out,
                                                                  int32_t* __restrict__ src,
                                                                  uint8_t* __restrict__ original, int np)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= z.n) return;
    const int32_t code = codes[i];
    if (code == DG_DENSIFY_PRUNE) return;
    const int64_t o = offsets[i];
    if (code != DG_DENSIFY_SPLIT) {
        copy_row(z, i, out, o, np);
        src[o] = (int32_t)i;
        original[o] = 1;
        if (code == DG_DENSIFY_CLONE) {
            copy_row(z, i, out, o + 1, np);
            src[o + 1] = (int32_t)i;
            original[o + 1] = 0;
        }
        return;
    }
    // split: two children around the parent, rotation of the normalised quaternion (w, x, y, z)
    const float4 mo = z.mo[i], q = z.quat[i], sc = z.scale[i];
    const float qi = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * qi, x = q.y * qi, y = q.z * qi, zq = q.w * qi;
    const float R[9] = {1.f - 2.f * (y * y + zq * zq), 2.f * (x * y - w * zq), 2.f * (x * zq + w * y),
                        2.f * (x * y + w * zq), 1.f - 2.f * (x * x + zq * zq), 2.f * (y * zq - w * x),
                        2.f * (x * zq - w * y), 2.f * (y * zq + w * x), 1.f - 2.f * (x * x + y * y)};
    const float s3[3] = {expf(sc.x), expf(sc.y), expf(sc.z)};
    const float ln16 = 0.47000362924573558f;                    // ln 1.6
    for (int h = 0; h < 2; h++) {
        const int64_t oh = o + h;
        copy_row(z, i, out, oh, np);
        const float* xi = normals + 6 * i + 3 * h;
        const float e0 = s3[0] * xi[0], e1 = s3[1] * xi[1], e2 = s3[2] * xi[2];
        out.mo[oh] = make_float4(mo.x + (R[0] * e0 + R[1] * e1 + R[2] * e2), mo.y + (R[3] * e0 + R[4] * e1 + R[5] * e2),
                                 mo.z + (R[6] * e0 + R[7] * e1 + R[8] * e2), mo.w);
        out.scale[oh] = make_float4(sc.x - ln16, sc.y - ln16, sc.z - ln16, sc.w);
        src[oh] = (int32_t)i;
        original[oh] = 0;
    }
}

// dst row r = src row idx[r] (idx < 0: left as it is), every field and plane
__global__ void __launch_bounds__(kDensifyThreads) k_gather_rows(GView s, const int32_t* __restrict__ idx, GView d,
                                                                 int np)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= d.n) return;
    const int64_t i = idx[r];
    if (i >= 0) copy_row(s, i, d, r, np);
}

// opacity reset: logit = min(logit, cap) on every row; where the moments are
// given, their opacity lanes restart from zero
__global__ void __launch_bounds__(kDensifyThreads) k_reset_opacity(GView g, float cap, float4* __restrict__ m,
                                                                   float4* __restrict__ v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    float4 mo = g.mo[i];
    mo.w = fminf(mo.w, cap);
    g.mo[i] = mo;
    if (m) m[i].w = 0.f;
    if (v) v[i].w = 0.f;
}

static unsigned blocks_of(int64_t n) { return (unsigned)((n + kDensifyThreads - 1) / kDensifyThreads); }

__global__ void k_dl_close(const uint32_t* __restrict__ offsets, int64_t n_g, const uint32_t* __restrict__ copy_off,
                           int64_t n_c, int64_t* __restrict__ new_g_off)
{
    new_g_off[offsets[n_g]] = (int64_t)copy_off[n_c];
}

int launch_densify_stats(const uint2* rect, const float* drec, const dg_camera* cams, const dg_plan& plan,
                         float* stats, cudaStream_t st)
{
    if (plan.n_rec == 0) return DG_OK;
    k_densify_stats<<<blocks_of(plan.n_rec), kDensifyThreads, 0, st>>>(rect, drec, cams, plan.n_views, plan.n_rec,
                                                                       stats);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

size_t densify_scan_ws_bytes(int64_t n) { return sizeof(uint32_t) * (size_t)((n + kScanChunkN - 1) / kScanChunkN + 1); }

int launch_densify_decide(const dg_gaussians* z, const int64_t* g_off, const int32_t* g_copies, const float* stats,
                          float grad_threshold, float logit_min, float log_big, int32_t* codes, uint32_t* counts,
                          uint32_t* offsets, void* ws, cudaStream_t st)
{
    const int64_t n = z->n;
    if (n == 0) return cudaMemsetAsync(offsets, 0, sizeof(uint32_t), st) == cudaSuccess ? DG_OK : DG_ERR_CUDA;
    DensifyArgs a{grad_threshold, logit_min, log_big};
    k_densify_decide<<<blocks_of(n), kDensifyThreads, 0, st>>>(gview(z), g_off, g_copies, stats, a, codes, counts);
    const int64_t n_chunks = (n + kScanChunkN - 1) / kScanChunkN;
    uint32_t* partials = (uint32_t*)ws;
    k_dscan_reduce<<<(unsigned)n_chunks, kScanT, 0, st>>>(counts, n, partials);
    k_dscan_top<<<1, kScanT, 0, st>>>(partials, n_chunks);
    k_dscan_down<<<(unsigned)n_chunks, kScanT, 0, st>>>(counts, n, partials, offsets);
    note_launch(4);
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_densify_emit(const dg_gaussians* z, const int32_t* codes, const uint32_t* offsets, const float* normals,
                        dg_gaussians* out, int32_t* src, uint8_t* original, cudaStream_t st)
{
    if (z->n == 0) return DG_OK;
    const int np = 3 * (z->sh_degree + 1) * (z->sh_degree + 1);
    k_densify_emit<<<blocks_of(z->n), kDensifyThreads, 0, st>>>(gview(z), codes, offsets, normals, gview(out), src,
                                                                original, np);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// ---- the densified copy layout, in place of the old one ------------------------------
// Each Gaussian's outputs take its place: global p's outputs are the new
// globals offsets[p] + h, and each of p's copies c (block k) becomes the new
// copies copy_off[c] + h of block k, copy_off being the exclusive scan over
// the old copies (blocks concatenated) of their Gaussian's output count.
__device__ __forceinline__ uint32_t n_outputs(int32_t code)
{
    return code == DG_DENSIFY_PRUNE ? 0u : (code == DG_DENSIFY_KEEP ? 1u : 2u);
}

__global__ void __launch_bounds__(kDensifyThreads) k_dl_copy_counts(const int32_t* __restrict__ copy_gid, int64_t n_c,
                                                                    const int32_t* __restrict__ codes,
                                                                    uint32_t* __restrict__ cnt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_c) cnt[c] = n_outputs(codes[copy_gid[c]]);
}

__global__ void __launch_bounds__(kDensifyThreads) k_dl_global_counts(const int64_t* __restrict__ g_off, int64_t n_g,
                                                                      const int32_t* __restrict__ codes,
                                                                      uint32_t* __restrict__ cnt)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_g) cnt[p] = n_outputs(codes[p]) * (uint32_t)(g_off[p + 1] - g_off[p]);
}

__global__ void __launch_bounds__(kDensifyThreads) k_dl_emit(const int64_t* __restrict__ g_off,
                                                             const int32_t* __restrict__ g_copies, int64_t n_g,
                                                             const int32_t* __restrict__ codes,
                                                             const uint32_t* __restrict__ offsets,
                                                             const uint32_t* __restrict__ copy_off,
                                                             const uint32_t* __restrict__ gscan,
                                                             int64_t* __restrict__ new_g_off,
                                                             int32_t* __restrict__ new_g_copies,
                                                             int32_t* __restrict__ new_copy_gid,
                                                             int32_t* __restrict__ carry)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_g) return;
    const int32_t code = codes[p];
    const uint32_t nout = n_outputs(code);
    const int64_t b = g_off[p];
    const uint32_t np = (uint32_t)(g_off[p + 1] - b);
    for (uint32_t h = 0; h < nout; h++) {
        const int64_t j = (int64_t)offsets[p] + h;
        const int64_t base = (int64_t)gscan[p] + (int64_t)h * np;
        new_g_off[j] = base;
        for (uint32_t i = 0; i < np; i++) {
            const int32_t c = g_copies[b + i];
            const int64_t nc = (int64_t)copy_off[c] + h;
            new_g_copies[base + i] = (int32_t)nc;
            new_copy_gid[nc] = (int32_t)j;
            carry[nc] = (h == 0 && code != DG_DENSIFY_SPLIT) ? c : -1;
        }
    }
}

// counts[b] += #{i : v[i] == lo + b} for b < nb (values outside [lo, lo + nb) are not
// counted); a shared-memory histogram per CTA, then one atomic per bin and CTA
__global__ void __launch_bounds__(kDensifyThreads) k_histogram(const int32_t* __restrict__ v, int64_t n, int32_t lo,
                                                               int nb, uint32_t* __restrict__ counts)
{
    __shared__ uint32_t s_h[64];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s_h[b] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = v[i] - lo;
        if (b >= 0 && b < nb) atomicAdd(&s_h[b], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (s_h[b]) atomicAdd(&counts[b], s_h[b]);
}

int launch_histogram(const int32_t* v, int64_t n, int32_t lo, int nb, uint32_t* counts, cudaStream_t st)
{
    if (cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)nb, st) != cudaSuccess) return DG_ERR_CUDA;
    if (n == 0) return DG_OK;
    const int64_t want = (n + kDensifyThreads - 1) / kDensifyThreads;
    const unsigned grid = (unsigned)(want < 148 * 8 ? want : 148 * 8);
    k_histogram<<<grid, kDensifyThreads, 0, st>>>(v, n, lo, nb, counts);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

// exclusive scan of n uint32 into out[0..n] (total at out[n]), ws: partials
static void scan_u32(const uint32_t* cnt, int64_t n, uint32_t* out, uint32_t* partials, cudaStream_t st)
{
    const int64_t n_chunks = (n + kScanChunkN - 1) / kScanChunkN;
    k_dscan_reduce<<<(unsigned)n_chunks, kScanT, 0, st>>>(cnt, n, partials);
    k_dscan_top<<<1, kScanT, 0, st>>>(partials, n_chunks);
    k_dscan_down<<<(unsigned)n_chunks, kScanT, 0, st>>>(cnt, n, partials, out);
    note_launch(3);
}

size_t densify_layout_ws_bytes(int64_t n_g, int64_t n_c)
{
    const auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up(sizeof(uint32_t) * (size_t)(n_c > n_g ? n_c : n_g)) + up(sizeof(uint32_t) * (size_t)(n_g + 1)) +
           up(densify_scan_ws_bytes(n_c > n_g ? n_c : n_g));
}

int launch_densify_layout(const int32_t* codes, const uint32_t* offsets, int64_t n_g, const int64_t* g_off,
                          const int32_t* g_copies, const int32_t* copy_gid, int64_t n_c, int64_t* new_g_off,
                          int32_t* new_g_copies, int32_t* new_copy_gid, int32_t* carry, uint32_t* copy_off,
                          void* ws, cudaStream_t st)
{
    const auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    char* w = (char*)ws;
    uint32_t* cnt = (uint32_t*)w;
    uint32_t* gscan = (uint32_t*)(w + up(sizeof(uint32_t) * (size_t)(n_c > n_g ? n_c : n_g)));
    uint32_t* partials = (uint32_t*)((char*)gscan + up(sizeof(uint32_t) * (size_t)(n_g + 1)));
    if (n_c == 0) {
        if (cudaMemsetAsync(copy_off, 0, sizeof(uint32_t), st) != cudaSuccess) return DG_ERR_CUDA;
    } else {
        k_dl_copy_counts<<<blocks_of(n_c), kDensifyThreads, 0, st>>>(copy_gid, n_c, codes, cnt);
        note_launch();
        scan_u32(cnt, n_c, copy_off, partials, st);
    }
    if (n_g > 0) {
        k_dl_global_counts<<<blocks_of(n_g), kDensifyThreads, 0, st>>>(g_off, n_g, codes, cnt);
        note_launch();
        scan_u32(cnt, n_g, gscan, partials, st);
        k_dl_emit<<<blocks_of(n_g), kDensifyThreads, 0, st>>>(g_off, g_copies, n_g, codes, offsets, copy_off, gscan,
                                                              new_g_off, new_g_copies, new_copy_gid, carry);
        note_launch();
    }
    // the closing offset of the new sharing map: the total of the new copies
    k_dl_close<<<1, 1, 0, st>>>(offsets, n_g, copy_off, n_c, new_g_off);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int launch_gather_rows(const dg_gaussians* s, const int32_t* idx, dg_gaussians* d, cudaStream_t st)
{
    if (d->n == 0) return DG_OK;
    const int np = 3 * (s->sh_degree + 1) * (s->sh_degree + 1);
    k_gather_rows<<<blocks_of(d->n), kDensifyThreads, 0, st>>>(gview(s), idx, gview(d), np);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

}  // namespace dg

namespace dg {
int launch_reset_opacity(dg_gaussians* g, float cap, dg_gaussians* m, dg_gaussians* v, cudaStream_t st)
{
    if (g->n == 0) return DG_OK;
    k_reset_opacity<<<blocks_of(g->n), kDensifyThreads, 0, st>>>(gview(g), cap, m ? gview(m).mo : nullptr,
                                                                 v ? gview(v).mo : nullptr);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}
}  // namespace dg
