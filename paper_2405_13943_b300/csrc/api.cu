// C ABI of libdogs: argument checks, batch planning, workspace carving and
// the launch sequences.  No allocation, no synchronisation.
#include <atomic>
#include <cstring>

#include "common.cuh"

namespace dg {

static std::atomic<uint64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int launch_project(const dg_gaussians*, const dg_camera*, const dg_plan&, float4*, uint2*, cudaStream_t);
int launch_project_bwd(const dg_gaussians*, const dg_camera*, const dg_plan&, const uint2*, const float4*,
                       dg_gaussians*, cudaStream_t);
size_t bin_sort_ws_bytes(int64_t n_tiles, int64_t capacity, int64_t list_records);
int launch_bin_sort(const float4*, const uint2*, const dg_camera*, const dg_plan&, int64_t, uint64_t*, uint32_t*,
                    uint32_t*, uint32_t*, void*, bool, uint32_t*, cudaStream_t);
int bin_sort_init();
size_t raster_slots_ws_bytes(int64_t n_rec);
size_t densify_layout_ws_bytes(int64_t n_g, int64_t n_c);
int launch_histogram(const int32_t* v, int64_t n, int32_t lo, int nb, uint32_t* counts, cudaStream_t st);
int launch_densify_layout(const int32_t* codes, const uint32_t* offsets, int64_t n_g, const int64_t* g_off,
                          const int32_t* g_copies, const int32_t* copy_gid, int64_t n_c, int64_t* new_g_off,
                          int32_t* new_g_copies, int32_t* new_copy_gid, int32_t* carry, uint32_t* copy_off,
                          void* ws, cudaStream_t st);
int launch_raster_bwd_slots(const float4* rec, const uint2* rect, const uint32_t* vals, const uint32_t* ranges,
                            const dg_camera* cams, const dg_plan& plan, const float* bg, const float* T_final,
                            const uint32_t* last, const float* dL_dimage, float* part, int64_t cap, void* ws,
                            uint64_t* dev_slots, uint32_t* dev_status, float* drec, cudaStream_t st);
int launch_admm_adapt(const double* res, float* rho, float* factor, const int32_t* dev_step, float mu,
                      float tau_inc, float tau_dec, int freeze_after, cudaStream_t st);
int launch_admm_rescale(dg_gaussians* u, const dg_gaussians* z, dg_gaussians* an, const int32_t* gid,
                        const uint8_t* shared, const float* factor, cudaStream_t st);
int loss_init();
int launch_raster_fwd(const float4*, const uint32_t*, const uint32_t*, const dg_camera*, const dg_plan&,
                      const float*, float*, float*, uint32_t*, cudaStream_t);
int launch_raster_count(const float4*, const uint32_t*, const uint32_t*, const dg_camera*, const dg_plan&,
                        const float*, float*, float*, uint32_t*, unsigned long long*, cudaStream_t);
int launch_raster_bwd(const float4*, const uint32_t*, const uint32_t*, const dg_camera*, const dg_plan&,
                      const float*, const float*, const uint32_t*, const float*, float*, cudaStream_t);
int launch_zero_kept(const uint2* rect, int64_t n_rec, float* drec, cudaStream_t st);
size_t loss_ws_bytes(const dg_plan&);
int launch_loss(const float*, const float*, const dg_camera*, const dg_plan&, float, float, double*, float*, void*,
                cudaStream_t);
int launch_adam_admm(dg_gaussians*, const dg_gaussians*, dg_gaussians*, dg_gaussians*, const dg_gaussians*,
                     const uint8_t*, const float*, const float*, float, float, float, int, const int32_t*,
                     cudaStream_t);
int launch_consensus(const dg_gaussians*, dg_gaussians*, dg_gaussians*, dg_gaussians*, const int64_t*,
                     const int32_t*, const float*, float, double*, cudaStream_t);
int launch_anchor(const dg_gaussians*, const dg_gaussians*, const int32_t*, const uint8_t*, dg_gaussians*,
                  cudaStream_t);
int launch_scale_duals(dg_gaussians*, const uint8_t*, const float*, cudaStream_t);
int launch_step_advance(int32_t*, cudaStream_t);
int launch_densify_stats(const uint2*, const float*, const dg_camera*, const dg_plan&, float*, cudaStream_t);
size_t densify_scan_ws_bytes(int64_t);
int launch_densify_decide(const dg_gaussians*, const int64_t*, const int32_t*, const float*, float, float, float,
                          int32_t*, uint32_t*, uint32_t*, void*, cudaStream_t);
int launch_densify_emit(const dg_gaussians*, const int32_t*, const uint32_t*, const float*, dg_gaussians*, int32_t*,
                        uint8_t*, cudaStream_t);
int launch_gather_rows(const dg_gaussians*, const int32_t*, dg_gaussians*, cudaStream_t);
int launch_reset_opacity(dg_gaussians*, float, dg_gaussians*, dg_gaussians*, cudaStream_t);
int launch_u8_to_f32(const uint8_t*, float*, int64_t, cudaStream_t);
int launch_f32_to_u8(const float*, uint8_t*, int64_t, cudaStream_t);
int launch_xstep(int, int, dg_gaussians*, dg_gaussians*, dg_gaussians*, const dg_gaussians*, const uint8_t*,
                 const dg_camera*, const dg_plan&, const uint2*, const float4*, const AdamArgs&, const int32_t*,
                 dg_gaussians*, const int32_t*, const void*, cudaStream_t);
int xstep_stream_init();
int raster_bwd_init();
size_t xstep_stream_ws_bytes(int64_t n);
int launch_xstep_groups(const dg_gaussians*, const dg_camera*, const dg_plan&, const uint2*, void*, cudaStream_t);
int launch_xstep_stream(int, dg_gaussians*, dg_gaussians*, dg_gaussians*, const dg_gaussians*, const uint8_t*,
                        const dg_camera*, const dg_plan&, const uint2*, const AdamArgs&, const int32_t*,
                        dg_gaussians*, const int32_t*, void*, bool, cudaStream_t);

static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
static bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

static bool valid_gauss(const dg_gaussians* g)
{
    if (!g) return false;
    if (g->n < 0 || g->ld < g->n || (g->ld & 3) || g->sh_degree < 0 || g->sh_degree > 3) return false;
    if (g->n > 0 && (!g->data || !aligned16(g->data))) return false;
    return true;
}

static bool same_layout(const dg_gaussians* a, const dg_gaussians* b)
{
    return a->n == b->n && a->ld == b->ld && a->sh_degree == b->sh_degree;
}

static bool valid_plan(const dg_plan* p)
{
    if (!p || p->n_views < 0 || p->n_views > DG_MAX_VIEWS || p->n_blocks < 1 || p->n_blocks > DG_MAX_BLOCKS) return false;
    if (!((p->tile_w == 16 && p->tile_h == 16) || (p->tile_w == 32 && p->tile_h == 8) || (p->tile_w == 8 && p->tile_h == 32)))
        return false;
    if (p->n_rec < 0 || p->n_rec >= (int64_t)0xFFFFFFFFll || p->n_tiles < 0 || p->n_tiles > (int64_t)1 << 24) return false;
    if (!(p->raster_warps == 1 || p->raster_warps == 2 || p->raster_warps == 4 || p->raster_warps == 8)) return false;
    if (!(p->raster_stage == 1 || p->raster_stage == 2)) return false;
    const int wb = p->raster_warps_bwd, sb = p->raster_stage_bwd;
    if (!((wb == 0 && sb == 0) || ((wb == 1 || wb == 2 || wb == 4 || wb == 8) && (sb == 1 || sb == 2)))) return false;
    return true;
}

// per-device one-time function attributes
int ensure_init()
{
    static std::atomic<uint64_t> done_mask{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
    uint64_t bit = 1ull << (dev & 63);
    if (done_mask.load() & bit) return DG_OK;
    int rc = bin_sort_init();
    if (rc == DG_OK) rc = loss_init();
    if (rc == DG_OK) rc = xstep_stream_init();
    if (rc == DG_OK) rc = raster_bwd_init();
    if (rc == DG_OK) done_mask.fetch_or(bit);
    return rc;
}

// The host-side argument checks of the binning entry points (every one
// before any launch): the plan, the capacity (instance numbers are 32-bit),
// the buffers a non-empty plan needs, and the alignment of every buffer the
// kernels read as vectors.
int bin_sort_args(const float* rec, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                  int64_t capacity, const uint64_t* keys, const uint32_t* vals, const uint32_t* ranges,
                  const uint32_t* dev_count, const uint32_t* dev_status)
{
    if (!valid_plan(plan) || capacity < 0 || capacity >= (int64_t)0xFFFFFFFFll) return DG_ERR_INVALID;
    if (plan->n_tiles == 0) return DG_OK;
    if (!dev_cams || !ranges || !dev_count || !dev_status || !vals) return DG_ERR_INVALID;
    if (plan->n_rec > 0 && (!rec || !rect)) return DG_ERR_INVALID;
    if (!aligned16(rec) || !aligned8(rect) || !aligned8(dev_cams) || !aligned8(keys)) return DG_ERR_INVALID;
    return DG_OK;
}

}  // namespace dg

using namespace dg;

extern "C" {

const char* dg_version(void) { return "libdogs 0.1 sm_103a"; }

uint64_t dg_launch_count(void) { return g_launches.load(); }

int64_t dg_gaussian_floats(int64_t ld, int sh_degree)
{
    if (ld < 0 || sh_degree < 0 || sh_degree > 3) return -1;
    return (12 + 3 * (int64_t)sh_coefs(sh_degree)) * ld;
}

int dg_plan_views(dg_camera* cams, int n_views, const int64_t* blk_off, int n_blocks, int tile_w, int tile_h,
                  dg_plan* plan)
{
    if (!cams || !blk_off || !plan || n_views < 1 || n_views > DG_MAX_VIEWS || n_blocks < 1 || n_blocks > DG_MAX_BLOCKS)
        return DG_ERR_INVALID;
    dg_plan p;
    memset(&p, 0, sizeof p);
    p.n_views = n_views;
    p.n_blocks = n_blocks;
    p.tile_w = tile_w;
    p.tile_h = tile_h;
    p.raster_warps = 4;
    p.raster_stage = 2;
    p.raster_warps_bwd = 0;
    p.raster_stage_bwd = 0;
    if (blk_off[0] != 0) return DG_ERR_INVALID;
    for (int k = 0; k <= n_blocks; k++) {
        if (k > 0 && blk_off[k] < blk_off[k - 1]) return DG_ERR_INVALID;
        p.blk_off[k] = blk_off[k];
    }
    if (blk_off[n_blocks] >= (int64_t)0x7FFFFFFFll) return DG_ERR_INVALID;
    int64_t rec = 0, tiles = 0, pix = 0;
    int prev_block = 0;
    for (int k = 0; k <= n_blocks; k++) p.blk_view_off[k] = 0;
    for (int v = 0; v < n_views; v++) {
        dg_camera& c = cams[v];
        if (c.block < prev_block || c.block >= n_blocks) return DG_ERR_INVALID;
        if (c.width <= 0 || c.height <= 0 || !(c.fx > 0.f) || !(c.fy > 0.f)) return DG_ERR_INVALID;
        prev_block = c.block;
        c.tiles_x = (c.width + tile_w - 1) / tile_w;
        c.tiles_y = (c.height + tile_h - 1) / tile_h;
        if (c.tiles_x > 65535 || c.tiles_y > 65535) return DG_ERR_INVALID;
        c.tile_off = (int32_t)tiles;
        c.reserved = 0;
        c.rec_off = rec;
        c.pix_off = pix;
        c.gauss_begin = blk_off[c.block];
        c.gauss_end = blk_off[c.block + 1];
        rec += c.gauss_end - c.gauss_begin;
        tiles += (int64_t)c.tiles_x * c.tiles_y;
        pix += (int64_t)c.width * c.height;
        if (c.width > p.max_width) p.max_width = c.width;
        if (c.height > p.max_height) p.max_height = c.height;
        if (tiles > ((int64_t)1 << 24) || rec >= (int64_t)0xFFFFFFFFll) return DG_ERR_INVALID;
        p.blk_view_off[c.block + 1] = v + 1;
    }
    // blocks with no views: their view range is empty
    for (int k = 1; k <= n_blocks; k++)
        if (p.blk_view_off[k] < p.blk_view_off[k - 1]) p.blk_view_off[k] = p.blk_view_off[k - 1];
    p.n_rec = rec;
    p.n_tiles = tiles;
    p.n_pixels = pix;
    if (!valid_plan(&p)) return DG_ERR_INVALID;
    *plan = p;
    return DG_OK;
}

int dg_project(const dg_gaussians* x, const dg_camera* dev_cams, const dg_plan* plan, float* rec, uint32_t* rect,
               void* stream)
{
    if (!valid_gauss(x) || !valid_plan(plan)) return DG_ERR_INVALID;
    if (plan->blk_off[plan->n_blocks] > x->n) return DG_ERR_INVALID;
    if (plan->n_rec > 0 && (!dev_cams || !rec || !rect || !aligned16(rec) || !aligned8(rect) || !aligned8(dev_cams)))
        return DG_ERR_INVALID;
    return launch_project(x, dev_cams, *plan, (float4*)rec, (uint2*)rect, (cudaStream_t)stream);
}

size_t dg_bin_sort_workspace_size(const dg_plan* plan, int64_t capacity)
{
    if (!valid_plan(plan) || capacity < 0) return 0;
    return bin_sort_ws_bytes(plan->n_tiles, capacity, plan->n_rec);
}

size_t dg_bin_sort_workspace_min_size(const dg_plan* plan, int64_t capacity)
{
    if (!valid_plan(plan) || capacity < 0) return 0;
    return bin_sort_ws_bytes(plan->n_tiles, capacity, 0);
}

int dg_bin_sort(const float* rec, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                int64_t capacity, uint64_t* keys, uint32_t* vals, uint32_t* ranges, uint32_t* dev_count, void* ws,
                size_t ws_bytes, uint32_t* dev_status, void* stream)
{
    int rc = bin_sort_args(rec, rect, dev_cams, plan, capacity, keys, vals, ranges, dev_count, dev_status);
    if (rc != DG_OK || plan->n_tiles == 0) return rc;
    if (!ws || ((uintptr_t)ws & 255u)) return DG_ERR_INVALID;
    if (ws_bytes < bin_sort_ws_bytes(plan->n_tiles, capacity, 0)) return DG_ERR_WORKSPACE;
    const bool with_list = ws_bytes >= bin_sort_ws_bytes(plan->n_tiles, capacity, plan->n_rec);
    rc = ensure_init();
    if (rc != DG_OK) return rc;
    return launch_bin_sort((const float4*)rec, (const uint2*)rect, dev_cams, *plan, capacity, keys, vals, ranges,
                           dev_count, ws, with_list, dev_status, (cudaStream_t)stream);
}

int dg_rasterize_fwd(const float* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* dev_cams,
                     const dg_plan* plan, const float* bg, float* image, float* T_final, uint32_t* last, void* stream)
{
    if (!valid_plan(plan) || !bg) return DG_ERR_INVALID;
    if (plan->n_tiles == 0) return DG_OK;
    if (!dev_cams || !ranges || !vals || !image || !T_final || !last) return DG_ERR_INVALID;
    if (!aligned16(rec) || !aligned8(dev_cams)) return DG_ERR_INVALID;
    return launch_raster_fwd((const float4*)rec, vals, ranges, dev_cams, *plan, bg, image, T_final, last,
                             (cudaStream_t)stream);
}

int dg_rasterize_count(const float* rec, const uint32_t* vals, const uint32_t* ranges, const dg_camera* dev_cams,
                       const dg_plan* plan, const float* bg, float* image, float* T_final, uint32_t* last,
                       uint64_t* counts, void* stream)
{
    if (!valid_plan(plan) || !bg || !counts || !aligned8(counts)) return DG_ERR_INVALID;
    if (plan->n_tiles > 0 && (!dev_cams || !ranges || !vals || !image || !T_final || !last)) return DG_ERR_INVALID;
    if (!aligned16(rec) || !aligned8(dev_cams)) return DG_ERR_INVALID;
    return launch_raster_count((const float4*)rec, vals, ranges, dev_cams, *plan, bg, image, T_final, last,
                               (unsigned long long*)counts, (cudaStream_t)stream);
}

int dg_loss_l1(const float* image, const float* target, const dg_camera* dev_cams, const dg_plan* plan, float w_l1,
               double* loss, float* dL_dimage, void* stream)
{
    if (!valid_plan(plan) || plan->n_views == 0) return DG_ERR_INVALID;
    if (!image || !target || !dev_cams || !loss || !dL_dimage) return DG_ERR_INVALID;
    if (!aligned8(dev_cams) || !aligned8(loss)) return DG_ERR_INVALID;
    return launch_loss(image, target, dev_cams, *plan, w_l1, 0.f, loss, dL_dimage, nullptr, (cudaStream_t)stream);
}

size_t dg_loss_workspace_size(const dg_plan* plan)
{
    if (!valid_plan(plan)) return 0;
    return loss_ws_bytes(*plan);
}

int dg_loss_dssim(const float* image, const float* target, const dg_camera* dev_cams, const dg_plan* plan,
                  float w_l1, float w_ssim, double* loss, float* dL_dimage, void* ws, size_t ws_bytes, void* stream)
{
    if (!valid_plan(plan) || plan->n_views == 0) return DG_ERR_INVALID;
    if (!image || !target || !dev_cams || !loss || !dL_dimage) return DG_ERR_INVALID;
    if (!aligned8(dev_cams) || !aligned8(loss) || ((uintptr_t)ws & 7u)) return DG_ERR_INVALID;
    if (w_ssim != 0.f && (!ws || ws_bytes < loss_ws_bytes(*plan))) return DG_ERR_WORKSPACE;
    int rc = ensure_init();
    if (rc != DG_OK) return rc;
    return launch_loss(image, target, dev_cams, *plan, w_l1, w_ssim, loss, dL_dimage, ws, (cudaStream_t)stream);
}

int dg_rasterize_bwd(const float* rec, const uint32_t* rect, const uint32_t* vals, const uint32_t* ranges,
                     const dg_camera* dev_cams, const dg_plan* plan, const float* bg, const float* T_final,
                     const uint32_t* last, const float* dL_dimage, const dg_gaussians* x, float* drec,
                     dg_gaussians* grads, void* stream)
{
    if (!valid_plan(plan) || !bg || !valid_gauss(x) || !valid_gauss(grads) || !same_layout(x, grads))
        return DG_ERR_INVALID;
    if (plan->blk_off[plan->n_blocks] > x->n) return DG_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->n_rec > 0) {
        if (!rec || !rect || !vals || !ranges || !dev_cams || !T_final || !last || !dL_dimage || !drec)
            return DG_ERR_INVALID;
        if (!aligned16(rec) || !aligned8(rect) || !aligned8(dev_cams) || !aligned16(drec)) return DG_ERR_INVALID;
        if (cudaMemsetAsync(drec, 0, (size_t)plan->n_rec * 12 * sizeof(float), st) != cudaSuccess) return DG_ERR_CUDA;
        int rc = launch_raster_bwd((const float4*)rec, vals, ranges, dev_cams, *plan, bg, T_final, last, dL_dimage,
                                   drec, st);
        if (rc != DG_OK) return rc;
    }
    // K8 writes every copy in [0, blk_off[K]); zero the rest only when there is a rest
    if (plan->blk_off[plan->n_blocks] < x->n && cudaMemsetAsync(grads->data, 0, (size_t)dg_gaussian_floats(grads->ld, grads->sh_degree) * 4, st)
                        != cudaSuccess)
        return DG_ERR_CUDA;
    return launch_project_bwd(x, dev_cams, *plan, (const uint2*)rect, (const float4*)drec, grads, st);
}

int dg_adam_admm_step(dg_gaussians* x, const dg_gaussians* g, dg_gaussians* m, dg_gaussians* v,
                      const dg_gaussians* anchor, const uint8_t* copy_shared, const float* rho, const float* lr,
                      float beta1, float beta2, float eps, int step, const int32_t* dev_step, void* stream)
{
    if (!valid_gauss(x) || !valid_gauss(g) || !valid_gauss(m) || !valid_gauss(v)) return DG_ERR_INVALID;
    if (!same_layout(x, g) || !same_layout(x, m) || !same_layout(x, v)) return DG_ERR_INVALID;
    if (anchor && (!valid_gauss(anchor) || !same_layout(x, anchor))) return DG_ERR_INVALID;
    if (!rho || !lr || (!dev_step && step < 1)) return DG_ERR_INVALID;
    if ((uintptr_t)dev_step & 3u) return DG_ERR_INVALID;
    if (x->n > 0 && anchor && !copy_shared) return DG_ERR_INVALID;
    return launch_adam_admm(x, g, m, v, anchor, anchor ? copy_shared : nullptr, rho, lr, beta1, beta2, eps, step,
                            dev_step, (cudaStream_t)stream);
}

int dg_rasterize_bwd_records(const float* rec, const uint32_t* rect, const uint32_t* vals, const uint32_t* ranges,
                             const dg_camera* dev_cams, const dg_plan* plan, const float* bg, const float* T_final,
                             const uint32_t* last, const float* dL_dimage, float* drec, void* stream)
{
    if (!valid_plan(plan) || !bg) return DG_ERR_INVALID;
    if (plan->n_rec == 0) return DG_OK;
    if (!rec || !vals || !ranges || !dev_cams || !T_final || !last || !dL_dimage || !drec) return DG_ERR_INVALID;
    if (!aligned16(rec) || !aligned8(dev_cams) || !aligned16(drec) || !aligned8(rect)) return DG_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (rect) {
        int rc = launch_zero_kept((const uint2*)rect, plan->n_rec, drec, st);
        if (rc != DG_OK) return rc;
    } else if (cudaMemsetAsync(drec, 0, (size_t)plan->n_rec * 12 * sizeof(float), st) != cudaSuccess) {
        return DG_ERR_CUDA;
    }
    return launch_raster_bwd((const float4*)rec, vals, ranges, dev_cams, *plan, bg, T_final, last, dL_dimage, drec,
                             st);
}

size_t dg_rasterize_bwd_slots_workspace_size(const dg_plan* plan)
{
    if (!valid_plan(plan)) return 0;
    return raster_slots_ws_bytes(plan->n_rec);
}

int dg_rasterize_bwd_slots(const float* rec, const uint32_t* rect, const uint32_t* vals, const uint32_t* ranges,
                           const dg_camera* dev_cams, const dg_plan* plan, const float* bg, const float* T_final,
                           const uint32_t* last, const float* dL_dimage, float* part, int64_t slot_capacity,
                           void* ws, size_t ws_bytes, uint64_t* dev_slots, uint32_t* dev_status, float* drec,
                           void* stream)
{
    if (!valid_plan(plan) || !bg || slot_capacity < 0) return DG_ERR_INVALID;
    if (!dev_slots || !dev_status || !ws || ((uintptr_t)dev_slots & 7u) || ((uintptr_t)ws & 7u))
        return DG_ERR_INVALID;
    if (plan->n_rec > 0) {
        if (!rec || !rect || !vals || !ranges || !dev_cams || !T_final || !last || !dL_dimage || !drec)
            return DG_ERR_INVALID;
        if (slot_capacity > 0 && (!part || ((uintptr_t)part & 3u))) return DG_ERR_INVALID;
        if (!aligned16(rec) || !aligned8(rect) || !aligned8(dev_cams) || !aligned16(drec)) return DG_ERR_INVALID;
    }
    if (ws_bytes < raster_slots_ws_bytes(plan->n_rec)) return DG_ERR_WORKSPACE;
    return launch_raster_bwd_slots((const float4*)rec, (const uint2*)rect, vals, ranges, dev_cams, *plan, bg, T_final,
                                   last, dL_dimage, part, slot_capacity, ws, dev_slots, dev_status, drec,
                                   (cudaStream_t)stream);
}

static int xstep_args(int part, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                      const float* drec, const dg_gaussians* x, const dg_gaussians* m, const dg_gaussians* v,
                      const dg_gaussians* anchor, const uint8_t* copy_shared, const float* rho, const float* lr,
                      float beta1, float beta2, float eps, int step, const int32_t* dev_step,
                      const dg_gaussians* z_unshared, const int32_t* copy_gid, AdamArgs& a);

int dg_xstep_part(int part, int ctas, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                  const float* drec, dg_gaussians* x, dg_gaussians* m, dg_gaussians* v, const dg_gaussians* anchor,
                  const uint8_t* copy_shared, const float* rho, const float* lr, float beta1, float beta2, float eps,
                  int step, const int32_t* dev_step, dg_gaussians* z_unshared, const int32_t* copy_gid,
                  void* stream)
{
    if (part < 0 || part > 2 || ctas < 0) return DG_ERR_INVALID;
    AdamArgs a;
    const int rc = xstep_args(part, rect, dev_cams, plan, drec, x, m, v, anchor, copy_shared, rho, lr, beta1, beta2,
                              eps, step, dev_step, z_unshared, copy_gid, a);
    if (rc != DG_OK) return rc;
    return launch_xstep(part, ctas, x, m, v, anchor, (anchor || z_unshared) ? copy_shared : nullptr, dev_cams, *plan,
                        (const uint2*)rect, (const float4*)drec, a, dev_step, z_unshared, copy_gid, nullptr,
                        (cudaStream_t)stream);
}

// the host-side checks shared by dg_xstep_part and dg_xstep_stream (part 1:
// drec is not read), and the Adam arguments they launch with
static int xstep_args(int part, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                      const float* drec, const dg_gaussians* x, const dg_gaussians* m, const dg_gaussians* v,
                      const dg_gaussians* anchor, const uint8_t* copy_shared, const float* rho, const float* lr,
                      float beta1, float beta2, float eps, int step, const int32_t* dev_step,
                      const dg_gaussians* z_unshared, const int32_t* copy_gid, AdamArgs& a)
{
    if (!valid_plan(plan) || !valid_gauss(x) || !valid_gauss(m) || !valid_gauss(v)) return DG_ERR_INVALID;
    if (!same_layout(x, m) || !same_layout(x, v)) return DG_ERR_INVALID;
    if (anchor && (!valid_gauss(anchor) || !same_layout(x, anchor))) return DG_ERR_INVALID;
    if (!rho || !lr || (!dev_step && step < 1) || ((uintptr_t)dev_step & 3u)) return DG_ERR_INVALID;
    if (x->n > 0 && anchor && !copy_shared) return DG_ERR_INVALID;
    if (z_unshared && (!valid_gauss(z_unshared) || z_unshared->sh_degree != x->sh_degree ||
                       (x->n > 0 && (!copy_gid || !copy_shared)) || ((uintptr_t)copy_gid & 3u)))
        return DG_ERR_INVALID;
    if (plan->blk_off[plan->n_blocks] > x->n) return DG_ERR_INVALID;
    for (int k = 0; k < plan->n_blocks; k++)
        if (plan->blk_view_off[k + 1] - plan->blk_view_off[k] > 1) return DG_ERR_INVALID;   // one view per block
    if (plan->n_rec > 0 && (!rect || !dev_cams || (part != 1 && !drec))) return DG_ERR_INVALID;
    if (!aligned8(rect) || !aligned8(dev_cams) || !aligned16(drec)) return DG_ERR_INVALID;
    take_rho(rho, a.rho, &a.dev_rho);
    for (int i = 0; i < 6; i++) a.lr[i] = lr[i];
    a.b1 = beta1; a.b2 = beta2; a.eps = eps; a.step = step;
    return DG_OK;
}

size_t dg_xstep_stream_workspace_size(const dg_gaussians* x)
{
    return valid_gauss(x) ? xstep_stream_ws_bytes(x->n) : 0;
}

int dg_xstep_stream(int ctas, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan, dg_gaussians* x,
                    dg_gaussians* m, dg_gaussians* v, const dg_gaussians* anchor, const uint8_t* copy_shared,
                    const float* rho, const float* lr, float beta1, float beta2, float eps, int step,
                    const int32_t* dev_step, dg_gaussians* z_unshared, const int32_t* copy_gid, void* ws,
                    size_t ws_bytes, void* stream)
{
    if (ctas < 0 || ctas > 65535) return DG_ERR_INVALID;
    AdamArgs a;
    int rc = xstep_args(1, rect, dev_cams, plan, nullptr, x, m, v, anchor, copy_shared, rho, lr, beta1, beta2, eps,
                        step, dev_step, z_unshared, copy_gid, a);
    if (rc != DG_OK) return rc;
    if (x->n > 0 && (!ws || !aligned16(ws))) return DG_ERR_INVALID;
    if (ws_bytes < xstep_stream_ws_bytes(x->n)) return DG_ERR_WORKSPACE;
    if (x->n == 0) return DG_OK;                  // nothing to step: no device call
    rc = ensure_init();
    if (rc != DG_OK) return rc;
    return launch_xstep_stream(ctas, x, m, v, anchor, (anchor || z_unshared) ? copy_shared : nullptr, dev_cams,
                               *plan, (const uint2*)rect, a, dev_step, z_unshared, copy_gid, ws, true,
                               (cudaStream_t)stream);
}

int dg_xstep_groups(const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan, const dg_gaussians* x,
                    void* ws, size_t ws_bytes, void* stream)
{
    if (!valid_plan(plan) || !valid_gauss(x) || plan->blk_off[plan->n_blocks] > x->n) return DG_ERR_INVALID;
    for (int k = 0; k < plan->n_blocks; k++)
        if (plan->blk_view_off[k + 1] - plan->blk_view_off[k] > 1) return DG_ERR_INVALID;   // one view per block
    if (plan->n_rec > 0 && (!rect || !dev_cams)) return DG_ERR_INVALID;
    if (!aligned8(rect) || !aligned8(dev_cams)) return DG_ERR_INVALID;
    if (x->n > 0 && (!ws || !aligned16(ws))) return DG_ERR_INVALID;
    if (ws_bytes < xstep_stream_ws_bytes(x->n)) return DG_ERR_WORKSPACE;
    return launch_xstep_groups(x, dev_cams, *plan, (const uint2*)rect, ws, (cudaStream_t)stream);
}

int dg_xstep_listed(int part, int ctas, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                    const float* drec, dg_gaussians* x, dg_gaussians* m, dg_gaussians* v, const dg_gaussians* anchor,
                    const uint8_t* copy_shared, const float* rho, const float* lr, float beta1, float beta2,
                    float eps, int step, const int32_t* dev_step, dg_gaussians* z_unshared,
                    const int32_t* copy_gid, void* ws, size_t ws_bytes, void* stream)
{
    if ((part != 1 && part != 2) || ctas < 0 || ctas > 65535) return DG_ERR_INVALID;
    AdamArgs a;
    int rc = xstep_args(part, rect, dev_cams, plan, drec, x, m, v, anchor, copy_shared, rho, lr, beta1, beta2, eps,
                        step, dev_step, z_unshared, copy_gid, a);
    if (rc != DG_OK) return rc;
    if (x->n > 0 && (!ws || !aligned16(ws))) return DG_ERR_INVALID;
    if (ws_bytes < xstep_stream_ws_bytes(x->n)) return DG_ERR_WORKSPACE;
    const uint8_t* sh = (anchor || z_unshared) ? copy_shared : nullptr;
    if (x->n == 0) return DG_OK;                  // nothing to step: no device call
    if (part == 1) {
        rc = ensure_init();
        if (rc != DG_OK) return rc;
        return launch_xstep_stream(ctas, x, m, v, anchor, sh, dev_cams, *plan, (const uint2*)rect, a, dev_step,
                                   z_unshared, copy_gid, ws, false, (cudaStream_t)stream);
    }
    return launch_xstep(3, ctas, x, m, v, anchor, sh, dev_cams, *plan, (const uint2*)rect, (const float4*)drec, a,
                        dev_step, z_unshared, copy_gid, ws, (cudaStream_t)stream);
}

int dg_xstep_from_records(const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan, const float* drec,
                          dg_gaussians* x, dg_gaussians* m, dg_gaussians* v, const dg_gaussians* anchor,
                          const uint8_t* copy_shared, const float* rho, const float* lr, float beta1, float beta2,
                          float eps, int step, const int32_t* dev_step, void* stream)
{
    return dg_xstep_part(0, 0, rect, dev_cams, plan, drec, x, m, v, anchor, copy_shared, rho, lr, beta1, beta2, eps,
                         step, dev_step, nullptr, nullptr, stream);
}

int dg_admm_consensus(const dg_gaussians* x, dg_gaussians* u, dg_gaussians* z, dg_gaussians* anchor,
                      const int64_t* g_off, const int32_t* g_copies, const float* rho, float alpha,
                      double* residuals, void* stream)
{
    if (!valid_gauss(x) || !valid_gauss(u) || !valid_gauss(z) || !valid_gauss(anchor)) return DG_ERR_INVALID;
    if (!same_layout(x, u) || !same_layout(x, anchor) || z->sh_degree != x->sh_degree) return DG_ERR_INVALID;
    if (!rho || !(alpha > 0.f && alpha < 2.f)) return DG_ERR_INVALID;
    if (z->n > 0 && (!g_off || !g_copies)) return DG_ERR_INVALID;
    if (!aligned8(g_off) || ((uintptr_t)g_copies & 3u) || !aligned8(residuals)) return DG_ERR_INVALID;
    return launch_consensus(x, u, z, anchor, g_off, g_copies, rho, alpha, residuals, (cudaStream_t)stream);
}

int dg_admm_anchor(const dg_gaussians* z, const dg_gaussians* u, const int32_t* copy_gid, const uint8_t* copy_shared,
                   dg_gaussians* anchor, void* stream)
{
    if (!valid_gauss(z) || !valid_gauss(u) || !valid_gauss(anchor) || !same_layout(u, anchor)) return DG_ERR_INVALID;
    if (z->sh_degree != u->sh_degree) return DG_ERR_INVALID;
    if (u->n > 0 && (!copy_gid || !copy_shared)) return DG_ERR_INVALID;
    if ((uintptr_t)copy_gid & 3u) return DG_ERR_INVALID;
    return launch_anchor(z, u, copy_gid, copy_shared, anchor, (cudaStream_t)stream);
}

int dg_step_advance(int32_t* dev_step, void* stream)
{
    if (!dev_step || ((uintptr_t)dev_step & 3u)) return DG_ERR_INVALID;
    return launch_step_advance(dev_step, (cudaStream_t)stream);
}

int dg_densify_stats(const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan, const float* drec,
                     float* stats, void* stream)
{
    if (!valid_plan(plan)) return DG_ERR_INVALID;
    if (plan->n_rec > 0 && (!rect || !dev_cams || !drec || !stats)) return DG_ERR_INVALID;
    if (!aligned8(rect) || !aligned8(dev_cams) || !aligned16(drec) || ((uintptr_t)stats & 3u)) return DG_ERR_INVALID;
    return launch_densify_stats((const uint2*)rect, drec, dev_cams, *plan, stats, (cudaStream_t)stream);
}

size_t dg_densify_workspace_size(int64_t n_global) { return densify_scan_ws_bytes(n_global < 0 ? 0 : n_global); }

int dg_densify_decide(const dg_gaussians* z, const int64_t* g_off, const int32_t* g_copies, const float* stats,
                      float grad_threshold, float percent_dense, float extent, float min_opacity, int32_t* codes,
                      uint32_t* counts, uint32_t* offsets, void* ws, size_t ws_bytes, void* stream)
{
    if (!valid_gauss(z) || !offsets) return DG_ERR_INVALID;
    if (z->n > 0 && (!g_off || !g_copies || !stats || !codes || !counts || !ws)) return DG_ERR_INVALID;
    if (z->n >= ((int64_t)1 << 31) || ws_bytes < densify_scan_ws_bytes(z->n)) return DG_ERR_INVALID;
    if (!(percent_dense > 0.f) || !(extent > 0.f) || !(min_opacity > 0.f && min_opacity < 1.f))
        return DG_ERR_INVALID;
    // thresholds on the raw parameters, formed in double and rounded once
    const double m = (double)min_opacity;
    const float logit_min = (float)log(m / (1.0 - m));
    const float log_big = (float)log((double)percent_dense * (double)extent);
    return launch_densify_decide(z, g_off, g_copies, stats, grad_threshold, logit_min, log_big, codes, counts,
                                 offsets, ws, (cudaStream_t)stream);
}

int dg_densify_emit(const dg_gaussians* z, const int32_t* codes, const uint32_t* offsets, const float* normals,
                    dg_gaussians* out, int32_t* src, uint8_t* original, void* stream)
{
    if (!valid_gauss(z) || !valid_gauss(out) || out->sh_degree != z->sh_degree) return DG_ERR_INVALID;
    if (z->n > 0 && (!codes || !offsets || !normals || !src || !original)) return DG_ERR_INVALID;
    return launch_densify_emit(z, codes, offsets, normals, out, src, original, (cudaStream_t)stream);
}

size_t dg_densify_layout_workspace_size(int64_t n_global, int64_t n_copies)
{
    if (n_global < 0 || n_copies < 0) return 0;
    return densify_layout_ws_bytes(n_global, n_copies);
}

int dg_densify_layout(const int32_t* codes, const uint32_t* offsets, int64_t n_global, const int64_t* g_off,
                      const int32_t* g_copies, const int32_t* copy_gid, int64_t n_copies, int64_t* new_g_off,
                      int32_t* new_g_copies, int32_t* new_copy_gid, int32_t* carry, uint32_t* copy_offsets,
                      void* ws, size_t ws_bytes, void* stream)
{
    if (n_global < 0 || n_copies < 0 || n_global >= ((int64_t)1 << 30) || n_copies >= ((int64_t)1 << 30))
        return DG_ERR_INVALID;
    if (!offsets || !new_g_off || !copy_offsets || !ws) return DG_ERR_INVALID;
    if (n_global > 0 && (!codes || !g_off || !g_copies)) return DG_ERR_INVALID;
    if (n_copies > 0 && (!copy_gid || !new_g_copies || !new_copy_gid || !carry)) return DG_ERR_INVALID;
    if (((uintptr_t)new_g_off & 7u) || ((uintptr_t)g_off & 7u) || ((uintptr_t)ws & 255u)) return DG_ERR_INVALID;
    if (ws_bytes < densify_layout_ws_bytes(n_global, n_copies)) return DG_ERR_WORKSPACE;
    return launch_densify_layout(codes, offsets, n_global, g_off, g_copies, copy_gid, n_copies, new_g_off,
                                 new_g_copies, new_copy_gid, carry, copy_offsets, ws, (cudaStream_t)stream);
}

int dg_histogram_i32(const int32_t* v, int64_t n, int32_t lo, int n_bins, uint32_t* counts, void* stream)
{
    if (n < 0 || n_bins < 1 || n_bins > 64 || !counts || (n > 0 && !v) || ((uintptr_t)v & 3u) ||
        ((uintptr_t)counts & 3u))
        return DG_ERR_INVALID;
    return launch_histogram(v, n, lo, n_bins, counts, (cudaStream_t)stream);
}

int dg_gather_rows(const dg_gaussians* src, const int32_t* idx, dg_gaussians* dst, void* stream)
{
    if (!valid_gauss(src) || !valid_gauss(dst) || src->sh_degree != dst->sh_degree) return DG_ERR_INVALID;
    if (dst->n > 0 && !idx) return DG_ERR_INVALID;
    return launch_gather_rows(src, idx, dst, (cudaStream_t)stream);
}

int dg_image_u8_to_f32(const uint8_t* src, float* dst, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!src || !dst)) || ((uintptr_t)src & 3u) || !aligned16(dst))
        return DG_ERR_INVALID;
    return launch_u8_to_f32(src, dst, n, (cudaStream_t)stream);
}

int dg_image_f32_to_u8(const float* src, uint8_t* dst, int64_t n, void* stream)
{
    if (n < 0 || (n > 0 && (!src || !dst))) return DG_ERR_INVALID;
    return launch_f32_to_u8(src, dst, n, (cudaStream_t)stream);
}

int dg_reset_opacity(dg_gaussians* g, float cap, dg_gaussians* m, dg_gaussians* v, void* stream)
{
    if (!valid_gauss(g) || !(cap > 0.f && cap < 1.f)) return DG_ERR_INVALID;
    if ((m && !same_layout(g, m)) || (v && !same_layout(g, v))) return DG_ERR_INVALID;
    const double c = (double)cap;
    return launch_reset_opacity(g, (float)log(c / (1.0 - c)), m, v, (cudaStream_t)stream);
}

int dg_admm_scale_duals(dg_gaussians* u, const uint8_t* copy_shared, const float* factor, void* stream)
{
    if (!valid_gauss(u) || !factor) return DG_ERR_INVALID;
    if (u->n > 0 && !copy_shared) return DG_ERR_INVALID;
    return launch_scale_duals(u, copy_shared, factor, (cudaStream_t)stream);
}

int dg_admm_adapt(const double* residuals, float* rho, float* factor, const int32_t* dev_step, float mu,
                  float tau_inc, float tau_dec, int freeze_after, void* stream)
{
    if (!residuals || !rho || !factor || !dev_step) return DG_ERR_INVALID;
    if (((uintptr_t)residuals & 7u) || ((uintptr_t)rho & 3u) || ((uintptr_t)factor & 3u) || ((uintptr_t)dev_step & 3u))
        return DG_ERR_INVALID;
    if (!(mu >= 1.f) || !(tau_inc >= 1.f) || !(tau_dec >= 1.f)) return DG_ERR_INVALID;
    return launch_admm_adapt(residuals, rho, factor, dev_step, mu, tau_inc, tau_dec, freeze_after,
                             (cudaStream_t)stream);
}

int dg_admm_rescale(dg_gaussians* u, const dg_gaussians* z, dg_gaussians* anchor, const int32_t* copy_gid,
                    const uint8_t* copy_shared, const float* factor, void* stream)
{
    if (!valid_gauss(u) || !valid_gauss(z) || !valid_gauss(anchor) || !same_layout(u, anchor) || !factor)
        return DG_ERR_INVALID;
    if (z->sh_degree != u->sh_degree || ((uintptr_t)factor & 3u) || ((uintptr_t)copy_gid & 3u)) return DG_ERR_INVALID;
    if (u->n > 0 && (!copy_gid || !copy_shared)) return DG_ERR_INVALID;
    return launch_admm_rescale(u, z, anchor, copy_gid, copy_shared, factor, (cudaStream_t)stream);
}

int dg_render_plan(dg_camera* host_cams, int n_views, int64_t n_gauss, int tile_w, int tile_h, dg_plan* plan)
{
    if (!host_cams || n_gauss < 0) return DG_ERR_INVALID;
    int64_t off[2] = {0, n_gauss};
    for (int v = 0; v < n_views; v++) host_cams[v].block = 0;
    return dg_plan_views(host_cams, n_views, off, 1, tile_w, tile_h, plan);
}

struct RenderWs {
    float4* rec;
    uint2* rect;
    uint32_t* vals;
    uint32_t* ranges;
    float* T_final;
    uint32_t* last;
    void* bin;
    size_t bin_bytes;
};

static size_t render_ws_layout(const dg_plan& p, int64_t capacity, char* base, RenderWs* w)
{
    size_t off = 0;
    auto take = [&](size_t b) { char* q = base ? base + off : nullptr; off += a256(b); return q; };
    RenderWs r;
    r.rec = (float4*)take((size_t)p.n_rec * 48 + 16);
    r.rect = (uint2*)take((size_t)p.n_rec * 8 + 8);
    r.vals = (uint32_t*)take((size_t)(capacity > 0 ? capacity : 1) * 4);
    r.ranges = (uint32_t*)take((size_t)p.n_tiles * 12 + 8);   // ranges, then the work order
    r.T_final = (float*)take((size_t)p.n_pixels * 4 + 4);
    r.last = (uint32_t*)take((size_t)p.n_pixels * 4 + 4);
    r.bin_bytes = bin_sort_ws_bytes(p.n_tiles, capacity, p.n_rec);
    r.bin = take(r.bin_bytes);
    if (w) *w = r;
    return off;
}

size_t dg_render_workspace_size(const dg_plan* plan, int64_t capacity)
{
    if (!valid_plan(plan) || capacity < 0) return 0;
    return render_ws_layout(*plan, capacity, nullptr, nullptr);
}

int dg_render(const dg_gaussians* z, const dg_camera* dev_cams, const dg_plan* plan, const float* bg,
              int64_t capacity, float* image, void* ws, size_t ws_bytes, uint32_t* dev_count, uint32_t* dev_status,
              void* stream)
{
    if (!valid_gauss(z) || !valid_plan(plan) || !bg || plan->n_blocks != 1 || plan->blk_off[1] != z->n)
        return DG_ERR_INVALID;
    if (plan->n_tiles == 0) return DG_OK;
    if (!dev_cams || !image || !ws || !dev_count || !dev_status) return DG_ERR_INVALID;
    if (!aligned8(dev_cams) || ((uintptr_t)ws & 255u)) return DG_ERR_INVALID;
    if (capacity < 0 || capacity >= (int64_t)0xFFFFFFFFll) return DG_ERR_INVALID;
    if (ws_bytes < render_ws_layout(*plan, capacity, nullptr, nullptr)) return DG_ERR_WORKSPACE;
    RenderWs w;
    render_ws_layout(*plan, capacity, (char*)ws, &w);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_project(z, dev_cams, *plan, w.rec, w.rect, st);
    if (rc != DG_OK) return rc;
    rc = ensure_init();
    if (rc != DG_OK) return rc;
    rc = launch_bin_sort(w.rec, w.rect, dev_cams, *plan, capacity, nullptr, w.vals, w.ranges, dev_count, w.bin,
                         true, dev_status, st);
    if (rc != DG_OK) return rc;
    return launch_raster_fwd(w.rec, w.vals, w.ranges, dev_cams, *plan, bg, image, w.T_final, w.last, st);
}

}  // extern "C"
