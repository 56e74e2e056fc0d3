// dg_bin_sort_noalloc: tile binning and key sort with its scratch in a
// library-owned static device array instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they bin:
// for example a plugin inside an application whose allocator owns the whole
// device budget, or a latency-critical loop that must not pay cudaMalloc's
// implicit synchronisation.  They still pass every input and output buffer;
// only the scratch (per-tile counters and cursors, scan partials, big-tile
// lists, the unsorted (depth, record) pairs) comes from the array below.
//
// The array is reserved on every GPU that loads this library, for the life
// of the process, whether or not this entry point is ever called.  All calls
// share it and it keeps the previous call's contents; the binning pass
// clears the counters that must start at zero before using them.  Two calls
// whose work overlaps on the GPU (different streams without ordering, or
// different host threads) race on the array and give wrong results.
#include <mutex>

#include "common.cuh"

namespace dg {

size_t bin_sort_ws_bytes(int64_t n_tiles, int64_t capacity, int64_t list_records);
int launch_bin_sort(const float4*, const uint2*, const dg_camera*, const dg_plan&, int64_t, uint64_t*, uint32_t*,
                    uint32_t*, uint32_t*, void*, bool, uint32_t*, cudaStream_t);
int ensure_init();
int bin_sort_args(const float* rec, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                  int64_t capacity, const uint64_t* keys, const uint32_t* vals, const uint32_t* ranges,
                  const uint32_t* dev_count, const uint32_t* dev_status);

// Sized for DG_NOALLOC_MAX_TILES tiles and DG_NOALLOC_MAX_INSTANCES instances
// (the pairs take 8 bytes each; the per-tile arrays 16 bytes per tile).
constexpr size_t kNoallocScratchBytes = 40u << 20;
static __device__ __align__(256) unsigned char g_binsort_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the static array on the current device, looked up once
// per device.  The array's name in host code is only a host-side stand-in for
// the symbol, so it is never passed to a kernel directly.
static int scratch_address(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DG_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_binsort_scratch) != cudaSuccess || !p) return DG_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DG_OK;
}

}  // namespace dg

extern "C" int dg_bin_sort_noalloc(const float* rec, const uint32_t* rect, const dg_camera* dev_cams,
                                   const dg_plan* plan, int64_t capacity, uint64_t* keys, uint32_t* vals,
                                   uint32_t* ranges, uint32_t* dev_count, uint32_t* dev_status, void* stream)
{
    using namespace dg;
    // the same host-side checks as dg_bin_sort, then the fixed limits
    int rc = bin_sort_args(rec, rect, dev_cams, plan, capacity, keys, vals, ranges, dev_count, dev_status);
    if (rc != DG_OK || plan->n_tiles == 0) return rc;
    if (plan->n_tiles > DG_NOALLOC_MAX_TILES || capacity > DG_NOALLOC_MAX_INSTANCES) return DG_ERR_TOO_LARGE;
    if (bin_sort_ws_bytes(plan->n_tiles, capacity, 0) > kNoallocScratchBytes) return DG_ERR_TOO_LARGE;
    // the list of visible records when the array has room for it (it only
    // speeds the expansion up; the output is the same without it)
    const bool with_list = bin_sort_ws_bytes(plan->n_tiles, capacity, plan->n_rec) <= kNoallocScratchBytes;
    void* ws = nullptr;
    rc = scratch_address(&ws);
    if (rc != DG_OK) return rc;
    rc = ensure_init();
    if (rc != DG_OK) return rc;
    return launch_bin_sort((const float4*)rec, (const uint2*)rect, dev_cams, *plan, capacity, keys, vals, ranges,
                           dev_count, ws, with_list, dev_status, (cudaStream_t)stream);
}
