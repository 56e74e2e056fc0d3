// K2-K4: tile binning and the 64-bit (tile | depth) key sort.
//
// Each projected record covers a rectangle of tiles; every (record, tile)
// pair whose tile the record can reach at alpha >= 1/255 (tile culling,
// below) is an instance with key (tile << 32) | bits(depth) and value =
// record index.  The instances are sorted by (key, value): by tile first, then by
// depth, ties broken by record index (Sec. 3.1, Eq. 2 composites in depth
// order within each tile).
//
// Sort design (a most-significant-digit radix sort): the tile id is one
// wide digit.  Pass 1 histograms instances per tile with atomics; an
// exclusive scan of the histogram gives every tile's range (K4's output
// directly); pass 2 scatters (depth bits, record) pairs into their tile's
// range; then each tile's segment is sorted by (depth bits, record) in shared
// memory with a bitonic network (segments above the shared-memory limit
// fall back to the same network in global memory).  Instance data crosses
// HBM about three times (scatter write, sort read, value write) instead of
// twice per digit of an LSD sort.  No kernel waits on another CTA.
#include <algorithm>

#include "common.cuh"

namespace dg {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanChunk = kScanThreads * kScanPer;   // tiles per scan CTA
constexpr int kSmallCap = 2048;                       // segment sorted by a 256-thread CTA
constexpr int kBigCap = 16384;                        // segment sorted by a 1024-thread CTA in smem

// The compositing's work order: tiles by descending instance count, in
// buckets a quarter octave wide (clz(count) and the two bits after the
// leading one; empty tiles last), written after the ranges as
// ranges[2 n_tiles + i].  Heavy tiles
// then start first instead of in image order, so no long tile is left to run
// alone at the end of a compositing launch.
constexpr int kOrderBuckets = 129;
// counters after the per-tile counts: [0] big, [1] huge, [2] mid tile lists, [3] visible records
constexpr int kCtrs = 4;

// bucket 4 clz(n) + (3 - the two bits after n's leading one): a quarter
// octave wide, ascending as n descends; 128 for an empty tile
__device__ __forceinline__ int order_bucket(uint32_t n)
{
    if (n == 0) return 128;
    const int z = __clz(n);
    return 4 * z + 3 - (int)(((n << z) >> 29) & 3u);
}

struct BinWs {
    uint32_t* counts;     // n_tiles + 4 (four counters at the end: three tile lists, the visible records) + order_ctr, zeroed together
    uint32_t* cursor;     // n_tiles
    uint32_t* partials;   // n_chunks + 1
    uint32_t* big_list;   // n_tiles
    uint32_t* huge_list;  // n_tiles
    uint32_t* mid_list;   // n_tiles
    uint64_t* pairs;      // capacity
    uint32_t* order_ctr;  // counts + n_tiles + 4: 2 kOrderBuckets -- tiles per bucket, then the buckets' fill cursors
    uint32_t* vis_list;   // list_records (0: no list; the expansion then scans every record)
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t bin_ws_layout(int64_t n_tiles, int64_t capacity, int64_t list_records, BinWs* w, char* base)
{
    int64_t n_chunks = (n_tiles + kScanChunk - 1) / kScanChunk;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off += align256(bytes); return p; };
    BinWs t;
    t.counts = (uint32_t*)take(4 * (size_t)(n_tiles + kCtrs + 2 * kOrderBuckets));
    t.order_ctr = t.counts ? t.counts + n_tiles + kCtrs : nullptr;
    t.cursor = (uint32_t*)take(4 * (size_t)(n_tiles + 1));
    t.partials = (uint32_t*)take(4 * (size_t)(n_chunks + 1));
    t.big_list = (uint32_t*)take(4 * (size_t)(n_tiles + 1));
    t.huge_list = (uint32_t*)take(4 * (size_t)(n_tiles + 1));
    t.mid_list = (uint32_t*)take(4 * (size_t)(n_tiles + 1));
    t.pairs = (uint64_t*)take(8 * (size_t)(capacity > 0 ? capacity : 1));
    t.vis_list = list_records > 0 ? (uint32_t*)take(4 * (size_t)list_records) : nullptr;
    if (w) *w = t;
    return off;
}

size_t bin_sort_ws_bytes(int64_t n_tiles, int64_t capacity, int64_t list_records)
{
    return bin_ws_layout(n_tiles, capacity, list_records, nullptr, nullptr);
}

// ---- tile culling --------------------------------------------------------------
// A pixel at offset d from the mean is composited only if o exp(-q(d)/2) >=
// 1/255 with q(d) = a dx^2 + 2 b dx dy + c dy^2 (Eq. 2's skip rule).  A tile
// of a record's rectangle is binned only if the minimum of q over the box of
// its pixel centres is at most tau = 2 ln(255 o) (1 + 2^-10) + 2^-6; the
// widening keeps every pair the compositing could take, so culling changes
// no image, transmittance or gradient.  q is convex, so its minimum over the
// box is 0 when the box holds the mean and otherwise lies on an edge, at the
// edge's unconstrained minimiser clamped to the edge.  Rounding is pinned
// (no contraction) so that the count and the scatter decide alike.
struct CullRec {
    float mx, my, a, b, c, tau, b_c, b_a;   // b_c = b / c, b_a = b / a: one division each per record
};

__device__ __forceinline__ CullRec cull_rec(const float4* __restrict__ rec, int64_t r)
{
    const float4 g0 = rec[3 * r], g1 = rec[3 * r + 1];
    CullRec k;
    k.mx = g0.x; k.my = g0.y; k.a = g0.z; k.b = g0.w; k.c = g1.x;
    k.tau = __fmaf_rn(__fmul_rn(2.f, __logf(__fmul_rn(255.f, g1.y))), 1.f + 1.f / 1024.f, 1.f / 64.f);
    k.b_c = __fdiv_rn(k.b, k.c);
    k.b_a = __fdiv_rn(k.b, k.a);
    return k;
}

// minimum over t in [lo, hi] of a X^2 + 2 b X t + c t^2 (b_c = b / c: the
// unconstrained minimiser is -X b / c)
__device__ __forceinline__ float edge_qmin(float a, float b, float c, float b_c, float X, float lo, float hi)
{
    const float t = fminf(fmaxf(-__fmul_rn(X, b_c), lo), hi);
    return __fmaf_rn(__fmul_rn(c, t), t, __fmul_rn(X, __fmaf_rn(__fmul_rn(2.f, b), t, __fmul_rn(a, X))));
}

__device__ __forceinline__ bool tile_reached(const CullRec& k, uint32_t tx, uint32_t ty, int tw, int th)
{
    const float X0 = __fsub_rn(__fadd_rn((float)(tx * tw), 0.5f), k.mx);
    const float X1 = __fsub_rn(__fsub_rn((float)(tx * tw + tw), 0.5f), k.mx);
    const float Y0 = __fsub_rn(__fadd_rn((float)(ty * th), 0.5f), k.my);
    const float Y1 = __fsub_rn(__fsub_rn((float)(ty * th + th), 0.5f), k.my);
    if (X0 <= 0.f && X1 >= 0.f && Y0 <= 0.f && Y1 >= 0.f) return 0.f <= k.tau;
    const float qx = fminf(edge_qmin(k.a, k.b, k.c, k.b_c, X0, Y0, Y1), edge_qmin(k.a, k.b, k.c, k.b_c, X1, Y0, Y1));
    const float qy = fminf(edge_qmin(k.c, k.b, k.a, k.b_a, Y0, X0, X1), edge_qmin(k.c, k.b, k.a, k.b_a, Y1, X0, X1));
    const float m = fminf(qx, qy);
    return m <= k.tau;
}

// ---- passes 1 and 2: expansion of (record, tile) candidates ---------------------
// Each lane owns one record; the candidate pairs of the warp's 32 records
// (every tile of each rectangle) are numbered by a warp scan and dealt out 32
// at a time, so the lanes stay busy however the rectangle sizes vary.  A
// lane finds the owner of its candidate by a five-step search over the scan
// and reads the owner's fields from the warp's slice of shared memory (four
// 16-byte loads, where shuffles took one instruction a field).  Pass 1
// (SCATTER = false) counts the kept pairs per tile; pass 2 writes them into
// the tiles' ranges.  Both take the same decisions: the same inputs go
// through the same instructions.
//
// A candidate's row in its record's rectangle is li / w, formed as
// (li + 1/2) * rn(1/w) truncated: the exact quotient (li + 1/2) / w lies at
// least 1/(2w) from an integer, and the two roundings move it by at most
// 2^-23 (li + 1/2) / w, less than that for li < 2^21 (integer division
// above, never reached by a rectangle of this library's tile counts).
constexpr int kExpandThreads = 256;
struct ExpandSlice { float4 q[4][32]; };   // field group g of lane L's record at q[g][L]

// The expansion of one warp's 32 records (lane: record r when `own`); every
// lane of the warp calls it together.
template <bool SCATTER>
__device__ __forceinline__ void expand_warp(bool own, int64_t r, const uint2* __restrict__ rect,
                                            const float4* __restrict__ rec, const dg_camera* __restrict__ cams,
                                            int n_views, int tw, int th, uint32_t* __restrict__ counts,
                                            const uint32_t* __restrict__ ranges, uint32_t* __restrict__ cursor,
                                            uint64_t* __restrict__ pairs, ExpandSlice& sl)
{
    const int lane = threadIdx.x & 31;
    uint32_t xy0 = 0, w = 0, n = 0, toff = 0, TX = 0, dbits = 0;
    CullRec k = {0.f, 0.f, 0.f, 0.f, 0.f, -1.f, 0.f, 0.f};
    if (own) {
        const uint2 rr = rect[r];
        xy0 = rr.x;
        const uint32_t x0 = rr.x & 0xFFFFu, y0 = rr.x >> 16, x1 = rr.y & 0xFFFFu, y1 = rr.y >> 16;
        if (x1 > x0 && y1 > y0) {
            w = x1 - x0;
            n = w * (y1 - y0);
            const int v = find_view_of_rec(cams, n_views, r);
            toff = (uint32_t)__ldg(&cams[v].tile_off);
            TX = (uint32_t)__ldg(&cams[v].tiles_x);
            k = cull_rec(rec, r);
            if (SCATTER) dbits = __float_as_uint(rec[3 * r + 2].y);
        }
    }
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;                     // uniform over the warp
    const uint32_t excl = incl - n;
    __syncwarp();                               // the previous call's reads of the slice are done
    sl.q[0][lane] = make_float4(k.mx, k.my, k.a, k.b);
    sl.q[1][lane] = make_float4(k.c, k.tau, k.b_c, k.b_a);
    sl.q[2][lane] = make_float4(__uint_as_float(xy0), __uint_as_float(w), __uint_as_float(excl),
                                w ? __frcp_rn((float)w) : 0.f);
    sl.q[3][lane] = make_float4(__uint_as_float(toff), __uint_as_float(TX), __uint_as_float(dbits),
                                __uint_as_float((uint32_t)r));   // low 32 bits suffice: n_rec < 2^32
    __syncwarp();
    for (uint32_t base = 0; base < total; base += 32) {
        const uint32_t item = base + (uint32_t)lane;
        int o = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1)
            if (__shfl_sync(0xffffffffu, incl, o + st - 1) <= item) o += st;
        if (item >= total) continue;
        const int src = o < 31 ? o : 31;
        const float4 g0 = sl.q[0][src], g1 = sl.q[1][src], g2 = sl.q[2][src], g3 = sl.q[3][src];
        CullRec ok;
        ok.mx = g0.x; ok.my = g0.y; ok.a = g0.z; ok.b = g0.w;
        ok.c = g1.x; ok.tau = g1.y; ok.b_c = g1.z; ok.b_a = g1.w;
        const uint32_t oxy = __float_as_uint(g2.x), ow = __float_as_uint(g2.y);
        const uint32_t li = item - __float_as_uint(g2.z);
        const uint32_t dy = li < (1u << 21) ? __float2uint_rz(__fmul_rn(__fadd_rn(__uint2float_rn(li), 0.5f), g2.w))
                                            : li / ow;
        const uint32_t dx = li - dy * ow;
        const uint32_t tx = (oxy & 0xFFFFu) + dx, ty = (oxy >> 16) + dy;
        if (!tile_reached(ok, tx, ty, tw, th)) continue;
        const uint32_t t = __float_as_uint(g3.x) + ty * __float_as_uint(g3.y) + tx;
        if (!SCATTER) {
            atomicAdd(&counts[t], 1u);
        } else {
            const uint32_t pos = atomicAdd(&cursor[t], 1u);
            if (pos < ranges[2 * t + 1])   // never false
                pairs[pos] = ((uint64_t)__float_as_uint(g3.z) << 32) | (uint64_t)__float_as_uint(g3.w);
        }
    }
}

// LIST = false: one thread per record of the batch (most of them empty in a
// large scene).  LIST = true: a persistent grid over the list of records
// with a non-empty rectangle that k_visible built, so every warp holds 32
// records to expand instead of the few a run of 32 consecutive records has,
// and the rectangle -> record load chain before the expansion is paid once
// per 32 visible records.  The list's order is unspecified; the counts do
// not depend on it, nor do the sorted segments (the pairs are sorted by
// their full (depth, record) key).
template <bool SCATTER, bool LIST>
__global__ void __launch_bounds__(kExpandThreads) k_expand(const uint2* __restrict__ rect, const float4* __restrict__ rec,
                                                const dg_camera* __restrict__ cams, int n_views, int64_t n_rec,
                                                int tw, int th, uint32_t* __restrict__ counts,
                                                const uint32_t* __restrict__ dev_count, int64_t capacity,
                                                const uint32_t* __restrict__ ranges, uint32_t* __restrict__ cursor,
                                                uint64_t* __restrict__ pairs, const uint32_t* __restrict__ list,
                                                const uint32_t* __restrict__ n_list)
{
    if (SCATTER && (int64_t)(*dev_count) > capacity) return;   // uniform over the grid
    __shared__ ExpandSlice s_sl[kExpandThreads / 32];
    ExpandSlice& sl = s_sl[threadIdx.x >> 5];
    if (LIST) {
        const uint32_t cnt = *n_list;
        for (uint32_t b = blockIdx.x * blockDim.x; b < cnt; b += gridDim.x * blockDim.x) {
            const uint32_t i = b + threadIdx.x;
            const bool own = i < cnt;
            expand_warp<SCATTER>(own, own ? (int64_t)list[i] : 0, rect, rec, cams, n_views, tw, th, counts, ranges,
                                 cursor, pairs, sl);
        }
    } else {
        const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        expand_warp<SCATTER>(r < n_rec, r, rect, rec, cams, n_views, tw, th, counts, ranges, cursor, pairs, sl);
    }
}

// The records with a non-empty rectangle, appended to list in no particular
// order (one atomic per warp); four records per thread keep four rectangle
// loads in flight.
constexpr int kVisPer = 4;

__global__ void __launch_bounds__(256) k_visible(const uint2* __restrict__ rect, int64_t n_rec,
                                                 uint32_t* __restrict__ list, uint32_t* __restrict__ n_list)
{
    const int64_t base = (int64_t)blockIdx.x * (256 * kVisPer) + threadIdx.x;
    const int lane = threadIdx.x & 31;
    uint2 rr[kVisPer];
#pragma unroll
    for (int j = 0; j < kVisPer; j++) {
        const int64_t r = base + 256 * j;
        rr[j] = r < n_rec ? rect[r] : make_uint2(0, 0);
    }
    unsigned bal[kVisPer];
    uint32_t tot = 0;
#pragma unroll
    for (int j = 0; j < kVisPer; j++) {
        const bool vis = (rr[j].y & 0xFFFFu) > (rr[j].x & 0xFFFFu) && (rr[j].y >> 16) > (rr[j].x >> 16);
        bal[j] = __ballot_sync(0xffffffffu, vis);
        tot += __popc(bal[j]);
    }
    uint32_t at = 0;
    if (lane == 0 && tot) at = atomicAdd(n_list, tot);
    at = __shfl_sync(0xffffffffu, at, 0);
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kVisPer; j++) {
        if ((bal[j] >> lane) & 1u) list[at + __popc(bal[j] & below)] = (uint32_t)(base + 256 * j);
        at += __popc(bal[j]);
    }
}

// ---- CTA-wide exclusive scan of one value per thread (1024 threads) -----------
__device__ __forceinline__ uint32_t cta_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& total)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) s_warp[lane] = w;   // inclusive warp prefix
    }
    __syncthreads();
    total = s_warp[(blockDim.x >> 5) - 1];
    uint32_t before = wid > 0 ? s_warp[wid - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ counts, int64_t n_tiles,
                                                              uint32_t* __restrict__ partials)
{
    __shared__ uint32_t s_warp[32];
    int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; i++)
        if (base + i < n_tiles) s += counts[base + i];
    uint32_t tot;
    cta_exclusive_scan(s, s_warp, tot);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(uint32_t* __restrict__ partials, int64_t n_chunks,
                                                           int64_t capacity, uint32_t* __restrict__ dev_count,
                                                           uint32_t* __restrict__ dev_status)
{
    __shared__ uint32_t s_warp[32];
    // 64-bit running total so an overflow of the 32-bit instance count is seen
    uint64_t carry = 0;
    for (int64_t base = 0; base < n_chunks; base += (int64_t)kScanThreads * kScanPer) {
        int64_t i0 = base + (int64_t)threadIdx.x * kScanPer;
        uint32_t v[kScanPer];
        uint32_t s = 0;
#pragma unroll
        for (int i = 0; i < kScanPer; i++) { v[i] = (i0 + i < n_chunks) ? partials[i0 + i] : 0u; s += v[i]; }
        uint32_t tot;
        uint32_t ex = cta_exclusive_scan(s, s_warp, tot);
        uint64_t run = carry + ex;
#pragma unroll
        for (int i = 0; i < kScanPer; i++) {
            if (i0 + i < n_chunks) partials[i0 + i] = (uint32_t)run;
            run += v[i];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        partials[n_chunks] = (uint32_t)carry;
        *dev_count = carry > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)carry;
        if ((int64_t)carry > capacity) atomicOr(dev_status, DG_STATUS_CAPACITY);
    }
}

// ... and the histogram of the ranges' sizes over the work order's buckets
// (from the values written, so that the order's scatter sees the same)
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ counts, int64_t n_tiles,
                                                            const uint32_t* __restrict__ partials, int64_t n_chunks,
                                                            const uint32_t* __restrict__ dev_count, int64_t capacity,
                                                            uint32_t* __restrict__ ranges, uint32_t* __restrict__ cursor,
                                                            uint32_t* __restrict__ order_hist)
{
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_h[kOrderBuckets];
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_h[b] = 0;
    __syncthreads();
    bool overflow = (int64_t)(*dev_count) > capacity;
    int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanPer;
    uint32_t v[kScanPer], s = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; i++) { v[i] = base + i < n_tiles ? counts[base + i] : 0u; s += v[i]; }
    uint32_t tot;
    uint32_t run = partials[blockIdx.x] + cta_exclusive_scan(s, s_warp, tot);
#pragma unroll
    for (int i = 0; i < kScanPer; i++) {
        int64_t t = base + i;
        if (t < n_tiles) {
            uint32_t b = overflow ? 0u : run, e = overflow ? 0u : run + v[i];
            ranges[2 * t] = b;
            ranges[2 * t + 1] = e;
            cursor[t] = b;
            atomicAdd(&s_h[order_bucket(e - b)], 1u);
        }
        run += v[i];
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x)
        if (s_h[b]) atomicAdd(&order_hist[b], s_h[b]);
}

// ---- pass 2: scatter (depth bits, record) into tile segments ------------------------
// ---- per-segment sort ----------------------------------------------------------------
// Bitonic network in its "all ascending" form: for each merge size k the
// first step compares i with its mirror in the k-block, later steps compare
// i with i + j.  The smaller element always goes to the lower index, so
// positions >= n behave as +infinity and need no storage (virtual padding).
// (k, half and j are powers of two: block and offset by shifts and masks)
template <int NT>
__device__ __forceinline__ void bitonic_sort(uint64_t* s, uint32_t n)
{
    uint32_t N = 1;
    while (N < n) N <<= 1;
    for (uint32_t lk = 1; (1u << lk) <= N; lk++) {
        const uint32_t k = 1u << lk, lh = lk - 1;
        for (uint32_t p = threadIdx.x; p < N / 2; p += NT) {
            const uint32_t blk = p >> lh, off = p & ((1u << lh) - 1u);
            const uint32_t i = (blk << lk) + off, l = (blk << lk) + k - 1 - off;
            if (l < n) {
                uint64_t a = s[i], b = s[l];
                if (a > b) { s[i] = b; s[l] = a; }
            }
        }
        __syncthreads();
        for (int lj = (int)lh - 1; lj >= 0; lj--) {
            const uint32_t j = 1u << lj;
            for (uint32_t p = threadIdx.x; p < N / 2; p += NT) {
                const uint32_t i = ((p >> lj) << (lj + 1)) + (p & (j - 1u)), l = i + j;
                if (l < n) {
                    uint64_t a = s[i], b = s[l];
                    if (a > b) { s[i] = b; s[l] = a; }
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ void write_segment(const uint64_t* s, uint32_t n, uint32_t start, uint64_t tile,
                                              uint32_t* vals, uint64_t* keys, int nt)
{
    for (uint32_t i = threadIdx.x; i < n; i += nt) {
        uint64_t p = s[i];
        vals[start + i] = (uint32_t)p;
        if (keys) keys[start + i] = (tile << 32) | (p >> 32);
    }
}

// Segments of up to 256 instances: one warp per tile, a bitonic network on
// 64-bit (depth bits, record) keys held in registers -- element e = i * 32 +
// lane in register i of the lane -- with lane shuffles for distances below 32
// and register exchanges above.  The network is the "all ascending" form
// (each merge compares an element with its mirror in its k-block first, then
// e with e ^ j for j = k/4 .. 1, the smaller always to the lower position),
// so positions >= n hold +infinity at every stage: a compare-exchange whose
// upper partner is all padding changes nothing, and registers with i * 32 >=
// n are skipped.  A compare-exchange keeps one value by a single 64-bit
// comparison (equal values, only padding, may go either way).  No barriers.
// the half-cleaners of a merge in one warp's registers: e against e ^ j for
// j = JTOP, JTOP / 2, .. 1, the smaller to the lower position (registers
// with i * 32 >= n hold only padding and are skipped)
template <int NR, int JTOP>
__device__ __forceinline__ void warp_cleaners(uint64_t* v, int lane, uint32_t n)
{
#pragma unroll
    for (int j = JTOP; j > 0; j >>= 1) {
        if (j >= 32) {
            const int ri = j >> 5;
#pragma unroll
            for (int i = 0; i < NR; i++) {
                if (i & ri) continue;
                if ((uint32_t)((i | ri) * 32) >= n) continue;
                const uint64_t a = v[i], b = v[i | ri];
                const bool sw = b < a;
                v[i] = sw ? b : a;
                v[i | ri] = sw ? a : b;
            }
        } else {
            const bool lo = (lane & j) == 0;
#pragma unroll
            for (int i = 0; i < NR; i++) {
                if ((uint32_t)(i * 32) >= n) continue;
                const uint64_t w = __shfl_xor_sync(0xffffffffu, v[i], j);
                v[i] = ((w < v[i]) == lo) ? w : v[i];
            }
        }
    }
}

template <int NR, int K>
__device__ __forceinline__ void warp_merge(uint64_t* v, int lane, uint32_t n)
{
    if constexpr (K <= 32) {                // mirror within the lanes of one register
        const bool lo = (lane & (K >> 1)) == 0;
#pragma unroll
        for (int i = 0; i < NR; i++) {
            if ((uint32_t)(i * 32) >= n) continue;
            const uint64_t w = __shfl_xor_sync(0xffffffffu, v[i], K - 1);
            v[i] = ((w < v[i]) == lo) ? w : v[i];
        }
    } else {                                // mirror across registers: lane L of i meets lane 31 - L of ip
        constexpr int KR = K >> 5;
#pragma unroll
        for (int i = 0; i < NR; i++) {
            if ((i % KR) >= KR / 2) continue;
            const int ip = (i / KR) * KR + (KR - 1 - (i % KR));
            if ((uint32_t)(ip * 32) >= n) continue;
            const uint64_t a = v[i], b = v[ip];
            const uint64_t wa = __shfl_xor_sync(0xffffffffu, b, 31);
            const uint64_t wb = __shfl_xor_sync(0xffffffffu, a, 31);
            v[i] = wa < a ? wa : a;
            v[ip] = wb < b ? b : wb;
        }
    }
    warp_cleaners<NR, (K >> 2)>(v, lane, n);
}

template <int NR, int K = 2>
__device__ __forceinline__ void warp_bitonic(uint64_t* v, int lane, uint32_t n)
{
    if constexpr (K <= 32 * NR) {
        warp_merge<NR, K>(v, lane, n);
        warp_bitonic<NR, 2 * K>(v, lane, n);
    }
}

template <int NR>
__device__ __forceinline__ void warp_sort_segment(const uint64_t* __restrict__ pairs, uint32_t start, uint32_t n,
                                                  uint64_t tile, uint32_t* __restrict__ vals,
                                                  uint64_t* __restrict__ keys, int lane)
{
    uint64_t v[NR];
#pragma unroll
    for (int i = 0; i < NR; i++) {
        const uint32_t e = (uint32_t)(i * 32 + lane);
        v[i] = e < n ? pairs[start + e] : ~0ull;
    }
    warp_bitonic<NR>(v, lane, n);
#pragma unroll
    for (int i = 0; i < NR; i++) {
        const uint32_t e = (uint32_t)(i * 32 + lane);
        if (e < n) {
            vals[start + e] = (uint32_t)v[i];
            if (keys) keys[start + e] = (tile << 32) | (v[i] >> 32);
        }
    }
}

constexpr int kWarpSortMax = 256;

__global__ void __launch_bounds__(128) k_sort_warp(const uint32_t* __restrict__ ranges, int64_t n_tiles,
                                                   const uint64_t* __restrict__ pairs, uint32_t* __restrict__ vals,
                                                   uint64_t* __restrict__ keys, uint32_t* __restrict__ counters,
                                                   uint32_t* __restrict__ mid_list, uint32_t* __restrict__ big_list,
                                                   uint32_t* __restrict__ huge_list)
{
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    if (t >= n_tiles) return;
    const uint32_t start = ranges[2 * t], n = ranges[2 * t + 1] - start;
    if (n == 0) return;
    if (n > kWarpSortMax) {
        if (lane == 0) {
            if (n <= kSmallCap) mid_list[atomicAdd(&counters[2], 1u)] = (uint32_t)t;
            else if (n <= kBigCap) big_list[atomicAdd(&counters[0], 1u)] = (uint32_t)t;
            else huge_list[atomicAdd(&counters[1], 1u)] = (uint32_t)t;
        }
        return;
    }
    if (n <= 32) warp_sort_segment<1>(pairs, start, n, (uint64_t)t, vals, keys, lane);
    else if (n <= 64) warp_sort_segment<2>(pairs, start, n, (uint64_t)t, vals, keys, lane);
    else if (n <= 128) warp_sort_segment<4>(pairs, start, n, (uint64_t)t, vals, keys, lane);
    else warp_sort_segment<8>(pairs, start, n, (uint64_t)t, vals, keys, lane);
}

// Segments of 257 .. kSmallCap instances: one 256-thread CTA each, 8 warps
// of E = N / 256 keys a lane (N the network's power-of-two size, 512 ..
// 2048; element e = warp * 32 E + i * 32 + lane in register i).  Each warp
// first sorts its 32 E keys in registers (the warp network above); every
// later merge then takes its mirror step, and its half-cleaners of distance
// 32 E or more, through shared memory (a barrier each), and the rest in the
// warps' registers -- 6 barriered steps at N = 2048 instead of the 66 of a
// network wholly in shared memory.  The form is the all-ascending one
// throughout, so padding (+infinity) stays at the end.
template <int E>
__device__ __forceinline__ void cta_sort_segment(const uint64_t* __restrict__ pairs, uint32_t start, uint32_t n,
                                                 uint64_t tile, uint32_t* __restrict__ vals,
                                                 uint64_t* __restrict__ keys, uint64_t* s)
{
    constexpr int PW = 32 * E, N = 256 * E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t e0 = (uint32_t)(warp * PW + lane);
    uint64_t v[E];
#pragma unroll
    for (int i = 0; i < E; i++) {
        const uint32_t e = e0 + 32 * i;
        v[i] = e < n ? pairs[start + e] : ~0ull;
    }
    const uint32_t nl = n > (uint32_t)(warp * PW) ? min(n - (uint32_t)(warp * PW), (uint32_t)PW) : 0u;
    warp_bitonic<E>(v, lane, nl);
#pragma unroll 1
    for (uint32_t k = 2 * PW; k <= (uint32_t)N; k <<= 1) {
        __syncthreads();                           // the previous step's reads of s are done
#pragma unroll
        for (int i = 0; i < E; i++) s[e0 + 32 * i] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < E; i++) {              // e against its mirror in its k-block
            const uint32_t e = e0 + 32 * i, off = e & (k - 1);
            const uint64_t w = s[(e - off) + (k - 1 - off)];
            v[i] = off < (k >> 1) ? (w < v[i] ? w : v[i]) : (w < v[i] ? v[i] : w);
        }
#pragma unroll 1
        for (uint32_t j = k >> 2; j >= (uint32_t)PW; j >>= 1) {
            __syncthreads();
#pragma unroll
            for (int i = 0; i < E; i++) s[e0 + 32 * i] = v[i];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < E; i++) {          // e against e ^ j, the smaller to the lower position
                const uint32_t e = e0 + 32 * i;
                const uint64_t w = s[e ^ j];
                v[i] = (e & j) == 0 ? (w < v[i] ? w : v[i]) : (w < v[i] ? v[i] : w);
            }
        }
        warp_cleaners<E, PW / 2>(v, lane, nl);
    }
#pragma unroll
    for (int i = 0; i < E; i++) {
        const uint32_t e = e0 + 32 * i;
        if (e < n) {
            vals[start + e] = (uint32_t)v[i];
            if (keys) keys[start + e] = (tile << 32) | (v[i] >> 32);
        }
    }
}

// persistent over the list k_sort_warp fills
__global__ void __launch_bounds__(256) k_sort_small(const uint32_t* __restrict__ ranges,
                                                    const uint64_t* __restrict__ pairs, uint32_t* __restrict__ vals,
                                                    uint64_t* __restrict__ keys, const uint32_t* __restrict__ counters,
                                                    const uint32_t* __restrict__ mid_list)
{
    __shared__ uint64_t s[kSmallCap];
    const uint32_t nm = counters[2];
    for (uint32_t i = blockIdx.x; i < nm; i += gridDim.x) {
        const uint32_t t = mid_list[i];
        const uint32_t start = ranges[2 * (int64_t)t], n = ranges[2 * (int64_t)t + 1] - start;
        __syncthreads();                           // the previous segment's reads of s are done
        if (n <= 512) cta_sort_segment<2>(pairs, start, n, (uint64_t)t, vals, keys, s);
        else if (n <= 1024) cta_sort_segment<4>(pairs, start, n, (uint64_t)t, vals, keys, s);
        else cta_sort_segment<8>(pairs, start, n, (uint64_t)t, vals, keys, s);
    }
}

__global__ void __launch_bounds__(1024) k_sort_big(const uint32_t* __restrict__ ranges,
                                                   const uint64_t* __restrict__ pairs, uint32_t* __restrict__ vals,
                                                   uint64_t* __restrict__ keys, const uint32_t* __restrict__ counters,
                                                   const uint32_t* __restrict__ big_list)
{
    extern __shared__ uint64_t s_big[];
    uint32_t nb = counters[0];
    for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
        uint32_t t = big_list[i];
        uint32_t start = ranges[2 * (int64_t)t], n = ranges[2 * (int64_t)t + 1] - start;
        for (uint32_t j = threadIdx.x; j < n; j += 1024) s_big[j] = pairs[start + j];
        __syncthreads();
        bitonic_sort<1024>(s_big, n);
        write_segment(s_big, n, start, (uint64_t)t, vals, keys, 1024);
        __syncthreads();
    }
}

// Segments larger than shared memory: the same network in place in global
// memory (one CTA per segment; rare for the workloads here).
__global__ void __launch_bounds__(1024) k_sort_huge(const uint32_t* __restrict__ ranges, uint64_t* __restrict__ pairs,
                                                    uint32_t* __restrict__ vals, uint64_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ counters,
                                                    const uint32_t* __restrict__ huge_list)
{
    uint32_t nh = counters[1];
    for (uint32_t i = blockIdx.x; i < nh; i += gridDim.x) {
        uint32_t t = huge_list[i];
        uint32_t start = ranges[2 * (int64_t)t], n = ranges[2 * (int64_t)t + 1] - start;
        bitonic_sort<1024>(pairs + start, n);
        __threadfence_block();
        write_segment(pairs + start, n, start, (uint64_t)t, vals, keys, 1024);
        __syncthreads();
    }
}

// Each CTA takes 256 tiles at a time: their ranks within their buckets from
// shared-memory counters, then one global atomic per bucket the 256 touch
// (the work order's few buckets would otherwise take every tile's atomic on
// a handful of addresses).
__global__ void __launch_bounds__(256) k_order_scatter(uint32_t* __restrict__ ranges, int64_t n_tiles,
                                                       uint32_t* __restrict__ ctr)
{
    // exclusive scan of the bucket counts by warp 0, five buckets a lane
    constexpr int kPer = (kOrderBuckets + 31) / 32;
    __shared__ uint32_t s_off[kOrderBuckets];
    __shared__ uint32_t s_cnt[kOrderBuckets], s_base[kOrderBuckets];
    if (threadIdx.x < 32) {
        uint32_t c[kPer], sum = 0;
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const int b = threadIdx.x * kPer + j;
            c[j] = b < kOrderBuckets ? ctr[b] : 0u;
            sum += c[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
            if ((int)threadIdx.x >= d) incl += v;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            const int b = threadIdx.x * kPer + j;
            if (b < kOrderBuckets) s_off[b] = run;
            run += c[j];
        }
    }
    uint32_t* order = ranges + 2 * n_tiles;
    uint32_t* cursor = ctr + kOrderBuckets;
    for (int64_t c0 = (int64_t)blockIdx.x * 256; c0 < n_tiles; c0 += (int64_t)gridDim.x * 256) {
        for (int b = threadIdx.x; b < kOrderBuckets; b += 256) s_cnt[b] = 0;
        __syncthreads();
        const int64_t t = c0 + threadIdx.x;
        int b = 0;
        uint32_t rank = 0;
        if (t < n_tiles) {
            b = order_bucket(ranges[2 * t + 1] - ranges[2 * t]);
            rank = atomicAdd(&s_cnt[b], 1u);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < kOrderBuckets; q += 256)
            if (s_cnt[q]) s_base[q] = s_off[q] + atomicAdd(&cursor[q], s_cnt[q]);
        __syncthreads();
        if (t < n_tiles) order[s_base[b] + rank] = (uint32_t)t;
    }
}

// with_list: ws was laid out with room for a list of plan.n_rec records
int launch_bin_sort(const float4* rec, const uint2* rect, const dg_camera* cams, const dg_plan& plan,
                    int64_t capacity, uint64_t* keys, uint32_t* vals, uint32_t* ranges, uint32_t* dev_count,
                    void* ws, bool with_list, uint32_t* dev_status, cudaStream_t st)
{
    BinWs w;
    bin_ws_layout(plan.n_tiles, capacity, with_list ? plan.n_rec : 0, &w, (char*)ws);
    int64_t n_chunks = (plan.n_tiles + kScanChunk - 1) / kScanChunk;
    if (cudaMemsetAsync(w.counts, 0, 4 * (size_t)(plan.n_tiles + kCtrs + 2 * kOrderBuckets), st) != cudaSuccess)
        return DG_ERR_CUDA;
    uint32_t* counters = w.counts + plan.n_tiles;
    const bool listed = with_list && plan.n_rec > 0;
    unsigned exp_grid = (unsigned)((plan.n_rec + 255) / 256);
    if (listed) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return DG_ERR_CUDA;
        k_visible<<<(unsigned)((plan.n_rec + 256 * kVisPer - 1) / (256 * kVisPer)), 256, 0, st>>>(
            rect, plan.n_rec, w.vis_list, counters + 3);
        note_launch();
        exp_grid = (unsigned)std::min<int64_t>(exp_grid, (int64_t)sms * 8);   // 8 CTAs of 256 fit an SM
    }
    if (plan.n_rec > 0) {
        if (listed)
            k_expand<false, true><<<exp_grid, 256, 0, st>>>(rect, rec, cams, plan.n_views, plan.n_rec, plan.tile_w,
                                                           plan.tile_h, w.counts, nullptr, 0, nullptr, nullptr,
                                                           nullptr, w.vis_list, counters + 3);
        else
            k_expand<false, false><<<exp_grid, 256, 0, st>>>(rect, rec, cams, plan.n_views, plan.n_rec, plan.tile_w,
                                                            plan.tile_h, w.counts, nullptr, 0, nullptr, nullptr,
                                                            nullptr, nullptr, nullptr);
        note_launch();
    }
    k_scan_reduce<<<(unsigned)n_chunks, kScanThreads, 0, st>>>(w.counts, plan.n_tiles, w.partials);
    k_scan_top<<<1, kScanThreads, 0, st>>>(w.partials, n_chunks, capacity, dev_count, dev_status);
    k_scan_down<<<(unsigned)n_chunks, kScanThreads, 0, st>>>(w.counts, plan.n_tiles, w.partials, n_chunks, dev_count,
                                                             capacity, ranges, w.cursor, w.order_ctr);
    note_launch(3);
    if (plan.n_rec > 0) {
        if (listed)
            k_expand<true, true><<<exp_grid, 256, 0, st>>>(rect, rec, cams, plan.n_views, plan.n_rec, plan.tile_w,
                                                          plan.tile_h, nullptr, dev_count, capacity, ranges,
                                                          w.cursor, w.pairs, w.vis_list, counters + 3);
        else
            k_expand<true, false><<<exp_grid, 256, 0, st>>>(rect, rec, cams, plan.n_views, plan.n_rec, plan.tile_w,
                                                           plan.tile_h, nullptr, dev_count, capacity, ranges,
                                                           w.cursor, w.pairs, nullptr, nullptr);
        note_launch();
    }
    k_sort_warp<<<(unsigned)((plan.n_tiles + 3) / 4), 128, 0, st>>>(ranges, plan.n_tiles, w.pairs, vals, keys,
                                                                    counters, w.mid_list, w.big_list, w.huge_list);
    k_sort_small<<<148 * 4, 256, 0, st>>>(ranges, w.pairs, vals, keys, counters, w.mid_list);
    k_sort_big<<<148, 1024, kBigCap * sizeof(uint64_t), st>>>(ranges, w.pairs, vals, keys, counters, w.big_list);
    k_sort_huge<<<148, 1024, 0, st>>>(ranges, w.pairs, vals, keys, counters, w.huge_list);
    note_launch(4);
    // the compositing's work order, after the ranges (bucket sizes from k_scan_down)
    const unsigned og = (unsigned)std::min<int64_t>((plan.n_tiles + 255) / 256, 148 * 2);
    k_order_scatter<<<og, 256, 0, st>>>(ranges, plan.n_tiles, w.order_ctr);
    note_launch();
    DG_CHECK_LAUNCH();
    return DG_OK;
}

int bin_sort_init()
{
    if (cudaFuncSetAttribute(k_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kBigCap * sizeof(uint64_t))) != cudaSuccess)
        return DG_ERR_CUDA;
    return DG_OK;
}

}  // namespace dg
