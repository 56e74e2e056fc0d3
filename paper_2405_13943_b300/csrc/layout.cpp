// The copy layout of a block membership (host): global numbering, the
// block-local copies and the sharing map, as the batched trainer lays them
// out.  Run when the global set changes (a densification): the same rule as
// the initial layout, in linear passes spread over host threads.
//
// Rule: globals held by two or more blocks are numbered first, then the
// others; within each part by (first holding block, Z-order of the ground
// position), the Z-order being the 16-bit Morton code of (x, y) quantised
// over the points' bounding box (x in the even bits).  Block k's copies are
// its shared globals in ascending id, then its unshared ones; the sharing
// map lists each global's copies in ascending block.
//
// Passes: the points are bucketed by (shared or not, first block) in a
// stable counting pass over contiguous chunks, one per thread; each bucket is
// sorted by Morton code (stable radix sort), and the buckets in sequence are
// the global numbering.  The copies and the sharing map are then written
// chunk by chunk of globals, the place of each copy known from per-chunk
// counts (no pass over all globals per block).  Every pass is deterministic,
// so the result does not depend on the thread count.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <memory>
#include <new>
#include <thread>
#include <vector>

#include <sched.h>

#include "dogs.h"

namespace {

uint64_t spread16(uint64_t v) {
    v = (v | (v << 8)) & 0x00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0Full;
    v = (v | (v << 2)) & 0x33333333ull;
    return (v | (v << 1)) & 0x55555555ull;
}

// CPUs this process may run on (its affinity mask), else the online count.
unsigned usable_cpus() {
    cpu_set_t set;
    if (sched_getaffinity(0, sizeof(set), &set) == 0) {
        const int c = CPU_COUNT(&set);
        if (c > 0) return (unsigned)c;
    }
    const unsigned h = std::thread::hardware_concurrency();
    return h ? h : 1u;
}

// Threads for a host pass over n items: one per 64K items, at most 16 and at
// most the usable CPUs.
unsigned threads_for(int64_t n) {
    const unsigned h = usable_cpus();
    const int64_t want = n / 65536 + 1;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(std::min<unsigned>(h, 16u), want));
}

// f(t) for t in [0, T): T - 1 threads and the caller.  A task whose thread
// cannot be started runs on the caller.  f must not throw.
template <class F>
void parallel_for(unsigned T, const F& f) {
    std::vector<std::thread> th;
    unsigned started = 1;
    try {
        th.reserve(T);
        for (unsigned t = 1; t < T; t++) {
            th.emplace_back([&f, t] { f(t); });
            started++;
        }
    } catch (...) {
    }
    f(0u);
    for (unsigned t = started; t < T; t++) f(t);
    for (auto& x : th) x.join();
}

// [lo, hi) of chunk t of T over n items
inline int64_t chunk_lo(int64_t n, unsigned T, unsigned t) { return n * (int64_t)t / (int64_t)T; }

// Stable LSD radix sort of (key, idx)[0, n) by the 32-bit key, in digits of
// BITS bits: one read pass counts every digit, then one scatter pass per
// digit through the scratch arrays k2, i2 (n each), skipping a digit that
// all keys share; the result ends in key, idx.
template <int BITS>
void radix32(uint32_t* key, int32_t* idx, uint32_t* k2, int32_t* i2, int64_t n) {
    constexpr int P = (32 + BITS - 1) / BITS, R = 1 << BITS;
    int64_t cnt[P][R + 1];
    for (int p = 0; p < P; p++) std::fill(cnt[p], cnt[p] + R + 1, (int64_t)0);
    for (int64_t i = 0; i < n; i++) {
        const uint32_t k = key[i];
        for (int p = 0; p < P; p++) cnt[p][((k >> (p * BITS)) & (R - 1)) + 1]++;
    }
    uint32_t *ka = key, *kb = k2;
    int32_t *ia = idx, *ib = i2;
    for (int p = 0; p < P; p++) {
        int64_t* c = cnt[p];
        bool shared_digit = false;
        for (int d = 0; d < R && !shared_digit; d++) shared_digit = c[d + 1] == n;
        if (shared_digit) continue;
        for (int d = 0; d < R; d++) c[d + 1] += c[d];
        const int sh = p * BITS;
        for (int64_t i = 0; i < n; i++) {
            const int64_t q = c[(ka[i] >> sh) & (R - 1)]++;
            kb[q] = ka[i];
            ib[q] = ia[i];
        }
        std::swap(ka, kb);
        std::swap(ia, ib);
    }
    if (ka != key) {
        std::copy(ka, ka + n, key);
        std::copy(ia, ia + n, idx);
    }
}

}  // namespace

extern "C" int64_t dg_layout_copies(const uint64_t* member, int64_t n) {
    if (n < 0 || (n > 0 && !member)) return -1;
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) c += __builtin_popcountll(member[i]);
    return c;
}

namespace {

template <class T>
std::unique_ptr<T[]> host_array(int64_t n) {   // uninitialised; every element is written before it is read
    return std::unique_ptr<T[]>(new T[(size_t)std::max<int64_t>(n, 1)]);
}

void layout_impl(const double* xy, const uint64_t* member, int64_t n, int K, int32_t* order, int32_t* copy_gid,
                 int64_t* blk_off, int64_t* blk_nshared, int64_t* g_off, int32_t* g_copies, int64_t* n_shared) {
    const unsigned T = threads_for(n);
    const size_t TK = (size_t)T * (size_t)K;
    // bounding box: per chunk, then combined (min and max do not depend on the split)
    std::vector<double> box((size_t)T * 4);
    parallel_for(T, [&](unsigned t) {
        double l0 = INFINITY, l1 = INFINITY, h0 = -INFINITY, h1 = -INFINITY;
        for (int64_t i = chunk_lo(n, T, t); i < chunk_lo(n, T, t + 1); i++) {
            l0 = std::min(l0, xy[2 * i]);
            h0 = std::max(h0, xy[2 * i]);
            l1 = std::min(l1, xy[2 * i + 1]);
            h1 = std::max(h1, xy[2 * i + 1]);
        }
        box[4 * t] = l0; box[4 * t + 1] = l1; box[4 * t + 2] = h0; box[4 * t + 3] = h1;
    });
    double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
    for (unsigned t = 0; t < T; t++)
        for (int a = 0; a < 2; a++) {
            lo[a] = std::min(lo[a], box[4 * t + a]);
            hi[a] = std::max(hi[a], box[4 * t + 2 + a]);
        }
    // Morton codes (the quantisation (v - lo) / max(hi - lo, 1e-30) * 65535, clipped to
    // [0, 65535], truncated) and buckets: bucket f < K holds the shared points whose
    // first block is f, bucket K + f the unshared ones; per chunk the count of each
    const int NB = 2 * K;
    const size_t TB2 = (size_t)T * (size_t)NB;
    auto mort = host_array<uint32_t>(n);
    auto bucket = host_array<uint8_t>(n);
    std::vector<int64_t> ccount(TB2, 0);
    parallel_for(T, [&](unsigned t) {
        int64_t* cc = &ccount[(size_t)t * NB];
        for (int64_t i = chunk_lo(n, T, t); i < chunk_lo(n, T, t + 1); i++) {
            uint64_t q[2];
            for (int a = 0; a < 2; a++) {
                double v = (xy[2 * i + a] - lo[a]) / std::max(hi[a] - lo[a], 1e-30) * 65535.0;
                v = std::min(std::max(v, 0.0), 65535.0);
                q[a] = (uint64_t)v;
            }
            mort[i] = (uint32_t)(spread16(q[0]) | (spread16(q[1]) << 1));
            const uint64_t m = member[i];
            const int b = __builtin_ctzll(m) + (__builtin_popcountll(m) >= 2 ? 0 : K);
            bucket[i] = (uint8_t)b;
            cc[b]++;
        }
    });
    // stable bucketing: bucket b holds its points in ascending index
    std::vector<int64_t> boff((size_t)NB + 1, 0);
    for (int b = 0; b < NB; b++) {
        int64_t s = 0;
        for (unsigned t = 0; t < T; t++) s += ccount[(size_t)t * NB + b];
        boff[b + 1] = boff[b] + s;
    }
    std::vector<int64_t> cpos(TB2);
    for (int b = 0; b < NB; b++) {
        int64_t p = boff[b];
        for (unsigned t = 0; t < T; t++) {
            cpos[(size_t)t * NB + b] = p;
            p += ccount[(size_t)t * NB + b];
        }
    }
    auto bkey = host_array<uint32_t>(n), k2 = host_array<uint32_t>(n);
    auto k2i = host_array<int32_t>(n);
    parallel_for(T, [&](unsigned t) {
        int64_t pos[2 * DG_MAX_BLOCKS];
        for (int b = 0; b < NB; b++) pos[b] = cpos[(size_t)t * NB + b];
        for (int64_t i = chunk_lo(n, T, t); i < chunk_lo(n, T, t + 1); i++) {
            const int64_t p = pos[bucket[i]]++;
            bkey[p] = mort[i];
            order[p] = (int32_t)i;
        }
    });
    // each bucket by Morton code (stable: ties keep ascending index); buckets go to
    // threads round-robin.  The buckets in sequence are the global numbering: the
    // shared globals (by first block, then Z-order), then the unshared ones.
    const unsigned TS = std::max(1u, std::min<unsigned>(T, (unsigned)NB));
    parallel_for(TS, [&](unsigned t) {
        for (int b = (int)t; b < NB; b += (int)TS)
            radix32<8>(&bkey[boff[b]], &order[boff[b]], &k2[boff[b]], &k2i[boff[b]], boff[b + 1] - boff[b]);
    });
    const int64_t ns = boff[K];
    auto mg = host_array<uint64_t>(n);   // mg[g]: the membership of global g
    parallel_for(T, [&](unsigned t) {
        for (int64_t g = chunk_lo(n, T, t); g < chunk_lo(n, T, t + 1); g++) mg[g] = member[order[g]];
    });
    *n_shared = ns;
    // per chunk of globals and per block: how many shared and unshared copies
    std::vector<int64_t> cs(TK, 0), cu(TK, 0), gc(T, 0);
    parallel_for(T, [&](unsigned t) {
        int64_t* s = &cs[(size_t)t * K];
        int64_t* u = &cu[(size_t)t * K];
        int64_t c = 0;
        for (int64_t g = chunk_lo(n, T, t); g < chunk_lo(n, T, t + 1); g++) {
            uint64_t m = mg[g];
            c += __builtin_popcountll(m);
            int64_t* d = g < ns ? s : u;
            for (; m; m &= m - 1) d[__builtin_ctzll(m)]++;
        }
        gc[t] = c;
    });
    // block offsets; each chunk's first place in each block's shared and unshared parts
    blk_off[0] = 0;
    for (int k = 0; k < K; k++) {
        int64_t a = 0, b = 0;
        for (unsigned t = 0; t < T; t++) {
            a += cs[(size_t)t * K + k];
            b += cu[(size_t)t * K + k];
        }
        blk_nshared[k] = a;
        blk_off[k + 1] = blk_off[k] + a + b;
        int64_t ps = blk_off[k], pu = blk_off[k] + a;
        for (unsigned t = 0; t < T; t++) {
            const int64_t x = cs[(size_t)t * K + k], y = cu[(size_t)t * K + k];
            cs[(size_t)t * K + k] = ps;
            cu[(size_t)t * K + k] = pu;
            ps += x;
            pu += y;
        }
    }
    if (n == 0) {
        if (g_off) g_off[0] = 0;
        return;
    }
    std::vector<int64_t> gstart(T, 0);
    for (unsigned t = 1; t < T; t++) gstart[t] = gstart[t - 1] + gc[t - 1];
    // copies (block-major) and the sharing map: the copy of global g in block k is
    // g_copies[g_off[g] + (the number of g's blocks below k)]
    parallel_for(T, [&](unsigned t) {
        int64_t ps[64], pu[64];
        for (int k = 0; k < K; k++) {
            ps[k] = cs[(size_t)t * K + k];
            pu[k] = cu[(size_t)t * K + k];
        }
        int64_t go = gstart[t];
        for (int64_t g = chunk_lo(n, T, t); g < chunk_lo(n, T, t + 1); g++) {
            g_off[g] = go;
            int64_t* p = g < ns ? ps : pu;
            for (uint64_t m = mg[g]; m; m &= m - 1) {
                const int64_t e = p[__builtin_ctzll(m)]++;
                copy_gid[e] = (int32_t)g;
                g_copies[go++] = (int32_t)e;
            }
        }
    });
    g_off[n] = blk_off[K];
}

}  // namespace

extern "C" int dg_layout(const double* xy, const uint64_t* member, int64_t n, int K, int32_t* order,
                         int32_t* copy_gid, int64_t* blk_off, int64_t* blk_nshared, int64_t* g_off,
                         int32_t* g_copies, int64_t* n_shared) {
    if (n < 0 || K < 1 || K > DG_MAX_BLOCKS || !blk_off || !blk_nshared || !n_shared) return DG_ERR_INVALID;
    if (n >= ((int64_t)1 << 31)) return DG_ERR_INVALID;
    if (n > 0 && (!xy || !member || !order || !copy_gid || !g_off || !g_copies)) return DG_ERR_INVALID;
    const uint64_t valid = K == 64 ? ~0ull : ((1ull << K) - 1);
    for (int64_t i = 0; i < n; i++)
        if (member[i] == 0 || (member[i] & ~valid)) return DG_ERR_INVALID;   // every point in some block
    // copy numbers are int32 throughout the layout
    if (n > 0 && dg_layout_copies(member, n) >= ((int64_t)1 << 31)) return DG_ERR_INVALID;
    // the Z-order key converts the ground position to an integer
    for (int64_t i = 0; i < 2 * n; i++)
        if (!std::isfinite(xy[i])) return DG_ERR_INVALID;
    try {
        layout_impl(xy, member, n, K, order, copy_gid, blk_off, blk_nshared, g_off, g_copies, n_shared);
    } catch (const std::bad_alloc&) {
        return DG_ERR_HOST_MEMORY;
    } catch (...) {
        return DG_ERR_INVALID;
    }
    return DG_OK;
}

extern "C" int dg_layout_carry(const int64_t* old_blk_off, const int64_t* old_g_off, const int32_t* old_g_copies,
                               int64_t n_old, int K, const int64_t* new_blk_off, const int64_t* new_g_off,
                               const int32_t* new_g_copies, const int32_t* parent, const uint8_t* original,
                               int64_t n_new, int32_t* carry) {
    if (K < 1 || K > DG_MAX_BLOCKS || n_old < 0 || n_new < 0 || !old_blk_off || !new_blk_off || !old_g_off ||
        !new_g_off)
        return DG_ERR_INVALID;
    const int64_t nc = new_blk_off[K], oc = old_blk_off[K];
    if (new_blk_off[0] != 0 || old_blk_off[0] != 0 || nc < 0 || oc < 0 || old_g_off[n_old] != oc ||
        new_g_off[0] != 0 || new_g_off[n_new] != nc)
        return DG_ERR_INVALID;
    for (int k = 0; k < K; k++)
        if (new_blk_off[k + 1] < new_blk_off[k] || old_blk_off[k + 1] < old_blk_off[k]) return DG_ERR_INVALID;
    if (nc > 0 && (!new_g_copies || !parent || !original || !carry)) return DG_ERR_INVALID;
    if (oc > 0 && !old_g_copies) return DG_ERR_INVALID;
    auto block_of = [K](const int64_t* off, int64_t c) {
        return (int)(std::upper_bound(off, off + K + 1, c) - off) - 1;
    };
    std::atomic<bool> bad{false};
    // by new global: its copies (new sharing map, ascending block) against its
    // parent's copies (old sharing map, ascending block), merged by block
    const unsigned T = threads_for(nc);
    parallel_for(T, [&](unsigned t) {
        for (int64_t g = chunk_lo(n_new, T, t); g < chunk_lo(n_new, T, t + 1); g++) {
            const int64_t a0 = new_g_off[g], a1 = new_g_off[g + 1];
            if (a0 < 0 || a1 < a0 || a1 > nc) { bad = true; continue; }
            int64_t j = 0, j1 = 0;
            const int32_t p = original[g] ? parent[g] : -1;
            if (original[g]) {
                if (p < 0 || p >= n_old || old_g_off[p] < 0 || old_g_off[p + 1] < old_g_off[p] ||
                    old_g_off[p + 1] > oc) {
                    bad = true;
                    continue;
                }
                j = old_g_off[p];
                j1 = old_g_off[p + 1];
            }
            int ob = -1;                             // block of old copy j
            for (int64_t a = a0; a < a1; a++) {
                const int32_t e = new_g_copies[a];
                if (e < 0 || e >= nc) { bad = true; break; }
                const int b = block_of(new_blk_off, e);
                int32_t hit = -1;
                while (j < j1) {
                    const int32_t c = old_g_copies[j];
                    if (c < 0 || c >= oc) { bad = true; j = j1; break; }
                    if (ob < 0) ob = block_of(old_blk_off, c);
                    if (ob < b) { j++; ob = -1; continue; }
                    if (ob == b) hit = c;
                    break;
                }
                carry[e] = hit;
            }
        }
    });
    return bad ? DG_ERR_INVALID : DG_OK;
}

extern "C" int dg_layout_membership(const int64_t* old_blk_off, const int64_t* old_g_off, const int32_t* old_g_copies,
                                    int64_t n_old, int K, const int32_t* parent, int64_t n_new, uint64_t* member) {
    if (K < 1 || K > DG_MAX_BLOCKS || n_old < 0 || n_new < 0 || !old_blk_off || !old_g_off) return DG_ERR_INVALID;
    const int64_t oc = old_blk_off[K];
    if (old_blk_off[0] != 0 || oc < 0 || old_g_off[n_old] != oc) return DG_ERR_INVALID;
    for (int k = 0; k < K; k++)
        if (old_blk_off[k + 1] < old_blk_off[k]) return DG_ERR_INVALID;
    if (n_new > 0 && (!parent || !member)) return DG_ERR_INVALID;
    if (oc > 0 && !old_g_copies) return DG_ERR_INVALID;
    std::atomic<bool> bad{false};
    const unsigned T = threads_for(n_new);
    parallel_for(T, [&](unsigned t) {
        for (int64_t j = chunk_lo(n_new, T, t); j < chunk_lo(n_new, T, t + 1); j++) {
            uint64_t m = 0;
            const int32_t p = parent[j];
            if (p < 0 || p >= n_old || old_g_off[p] < 0 || old_g_off[p + 1] < old_g_off[p] || old_g_off[p + 1] > oc) {
                bad = true;
                member[j] = 0;
                continue;
            }
            for (int64_t a = old_g_off[p]; a < old_g_off[p + 1]; a++) {
                const int32_t c = old_g_copies[a];
                if (c < 0 || c >= oc) { bad = true; break; }
                m |= 1ull << ((std::upper_bound(old_blk_off, old_blk_off + K + 1, (int64_t)c) - old_blk_off) - 1);
            }
            member[j] = m;
        }
    });
    return bad ? DG_ERR_INVALID : DG_OK;
}
