// The copy layout of a block membership (host): global numbering, the
// block-local copies and the sharing map, as the batched trainer lays them
// out.  Run when the global set changes (a densification): the same rule as
// the initial layout, in linear passes.
//
// Rule: globals held by two or more blocks are numbered first, then the
// others; within each part by (first holding block, Z-order of the ground
// position), the Z-order being the 16-bit Morton code of (x, y) quantised
// over the points' bounding box (x in the even bits).  Block k's copies are
// its shared globals in ascending id, then its unshared ones; the sharing
// map lists each global's copies in ascending block.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "dogs.h"

namespace {

uint64_t spread16(uint64_t v) {
    v = (v | (v << 8)) & 0x00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0Full;
    v = (v | (v << 2)) & 0x33333333ull;
    return (v | (v << 1)) & 0x55555555ull;
}

// stable LSD radix sort of idx by key (8-bit digits over the key's used bytes)
void radix_sort(std::vector<uint64_t>& key, std::vector<int32_t>& idx, int bytes) {
    const size_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<int32_t> i2(n);
    for (int b = 0; b < bytes; b++) {
        const int sh = 8 * b;
        size_t cnt[257] = {0};
        for (size_t i = 0; i < n; i++) cnt[((key[i] >> sh) & 0xFF) + 1]++;
        for (int d = 0; d < 256; d++) cnt[d + 1] += cnt[d];
        for (size_t i = 0; i < n; i++) {
            const size_t p = cnt[(key[i] >> sh) & 0xFF]++;
            k2[p] = key[i];
            i2[p] = idx[i];
        }
        key.swap(k2);
        idx.swap(i2);
    }
}

}  // namespace

extern "C" int64_t dg_layout_copies(const uint64_t* member, int64_t n) {
    if (n < 0 || (n > 0 && !member)) return -1;
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) c += __builtin_popcountll(member[i]);
    return c;
}

extern "C" int dg_layout(const double* xy, const uint64_t* member, int64_t n, int K, int32_t* order,
                         int32_t* copy_gid, int64_t* blk_off, int64_t* blk_nshared, int64_t* g_off,
                         int32_t* g_copies, int64_t* n_shared) {
    if (n < 0 || K < 1 || K > DG_MAX_BLOCKS || !blk_off || !blk_nshared || !n_shared) return DG_ERR_INVALID;
    if (n >= ((int64_t)1 << 31)) return DG_ERR_INVALID;
    if (n > 0 && (!xy || !member || !order || !copy_gid || !g_off || !g_copies)) return DG_ERR_INVALID;
    const uint64_t valid = K == 64 ? ~0ull : ((1ull << K) - 1);
    for (int64_t i = 0; i < n; i++)
        if (member[i] == 0 || (member[i] & ~valid)) return DG_ERR_INVALID;   // every point in some block
    // Morton codes over the bounding box (the quantisation of the numpy rule:
    // (v - lo) / max(hi - lo, 1e-30) * 65535, clipped to [0, 65535], truncated)
    double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 2; a++) {
            lo[a] = std::min(lo[a], xy[2 * i + a]);
            hi[a] = std::max(hi[a], xy[2 * i + a]);
        }
    std::vector<uint64_t> key((size_t)n);
    std::vector<int32_t> idx((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        uint64_t q[2];
        for (int a = 0; a < 2; a++) {
            double v = (xy[2 * i + a] - lo[a]) / std::max(hi[a] - lo[a], 1e-30) * 65535.0;
            v = std::min(std::max(v, 0.0), 65535.0);
            q[a] = (uint64_t)v;
        }
        const uint64_t first = (uint64_t)__builtin_ctzll(member[i]);
        key[i] = (first << 32) | spread16(q[0]) | (spread16(q[1]) << 1);
        idx[i] = (int32_t)i;
    }
    radix_sort(key, idx, 5);                      // 32 Morton bits + 6 block bits
    // shared first, each part in key order; mg[g]: the membership of global g
    std::vector<uint64_t> ms((size_t)n);
    for (int64_t j = 0; j < n; j++) ms[j] = member[idx[j]];
    std::vector<uint64_t> mg((size_t)n);
    int64_t ns = 0, o = 0;
    for (int64_t j = 0; j < n; j++)
        if (__builtin_popcountll(ms[j]) >= 2) { mg[o] = ms[j]; order[o++] = idx[j]; }
    ns = o;
    for (int64_t j = 0; j < n; j++)
        if (__builtin_popcountll(ms[j]) < 2) { mg[o] = ms[j]; order[o++] = idx[j]; }
    *n_shared = ns;
    // block-local copies: shared globals of the block, then unshared, ascending id
    int64_t c = 0;
    blk_off[0] = 0;
    for (int k = 0; k < K; k++) {
        const uint64_t bit = 1ull << k;
        int64_t nsh = 0;
        for (int64_t g = 0; g < ns; g++)
            if (mg[g] & bit) { copy_gid[c++] = (int32_t)g; nsh++; }
        for (int64_t g = ns; g < n; g++)
            if (mg[g] & bit) copy_gid[c++] = (int32_t)g;
        blk_nshared[k] = nsh;
        blk_off[k + 1] = c;
    }
    // sharing map: each global's copies in ascending block (copies are block-major)
    if (n == 0 && g_off) g_off[0] = 0;
    if (n > 0) {
        std::fill(g_off, g_off + n + 1, 0);
        for (int64_t e = 0; e < c; e++) g_off[copy_gid[e] + 1]++;
        for (int64_t g = 0; g < n; g++) g_off[g + 1] += g_off[g];
        std::vector<int64_t> cur(g_off, g_off + n);
        for (int64_t e = 0; e < c; e++) g_copies[cur[copy_gid[e]]++] = (int32_t)e;
    }
    return DG_OK;
}
