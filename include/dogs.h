/*
 * dogs.h -- C ABI of libdogs, the B300 (sm_103a) hot path of DOGS
 * (distributed 3D Gaussian Splatting by ADMM Gaussian consensus).
 *
 * The library computes, on one GPU:
 *   - the differentiable tile rasteriser of 3D Gaussian Splatting (Sec. 3.1:
 *     Gaussian primitive, Eq. 1; Sigma = R S S^T R^T; alpha blending, Eq. 2):
 *     dg_project, dg_bin_sort, dg_rasterize_fwd, dg_rasterize_bwd, and the
 *     loss of Eq. 3 (dg_loss_l1, dg_loss_dssim);
 *   - the block ADMM of Sec. 3.2: the x-step (Eq. 8a / 12a) as one Adam step
 *     on the loss plus the penalty rho/2 ||x - z + u||^2 (dg_adam_admm_step),
 *     and the consensus z = mean(x + u), u += x - z (Eq. 8b-c / 12b-c, with
 *     over-relaxation and the residuals of Sec. 3.3) (dg_admm_consensus);
 *   - rendering of the global model for serving (dg_render).
 * The K block-local models are batched instances in one launch per step.
 *
 * Conventions shared by every entry point:
 *   - Every call returns an int status (DG_OK or a DG_ERR_* code below).
 *     Host-side argument errors are detected before anything is launched.
 *   - The caller owns all memory.  No call allocates, frees or synchronises;
 *     device buffers are passed as plain device pointers, host tables as
 *     host pointers, and work is enqueued on the cudaStream_t passed as
 *     `stream` (NULL = legacy default stream).  Calls are re-entrant and can
 *     be captured in a CUDA graph.
 *   - Conditions found on the device (instance capacity exceeded) are OR-ed
 *     into the caller's device word `dev_status` (DG_STATUS_* bits), to be
 *     read after the stream is synchronised.
 *   - n = 0 Gaussians is valid and renders the background.
 *   - Alignment (checked on the host, DG_ERR_INVALID otherwise): parameter
 *     buffers and projected records 16 bytes; tile rectangles, keys, camera
 *     tables, int64 and double arrays 8 bytes; int32 arrays 4 bytes; the
 *     bin-sort and render workspaces 256 bytes.  Byte arrays (copy_shared)
 *     need none.
 */
#ifndef DOGS_H
#define DOGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define DG_OK 0
#define DG_ERR_INVALID (-1)   /* null pointer with work to do, bad size, bad layout */
#define DG_ERR_WORKSPACE (-2) /* workspace smaller than the matching *_workspace_size */
#define DG_ERR_CAPACITY (-3)  /* reserved: host-visible capacity failure */
#define DG_ERR_CUDA (-4)      /* a CUDA launch or memset failed */
#define DG_ERR_TOO_LARGE (-6) /* sizes beyond the fixed limits of dg_bin_sort_noalloc */
#define DG_ERR_HOST_MEMORY (-7) /* host memory for a host-side pass could not be allocated */

/* bits OR-ed into *dev_status by device code */
#define DG_STATUS_CAPACITY 1u /* tile instances exceed `capacity`; ranges were emptied */

#define DG_MAX_BLOCKS 64      /* K, the number of block-local models in one batch */
#define DG_MAX_VIEWS 4096

/* ---- Gaussian parameter set ---------------------------------------------- */
/* One Gaussian x_i = {mean p, rotation q, scale s, SH features f, opacity o}
 * (Sec. 3.1, under Eq. 3; the same property split as the per-property ADMM of
 * Eq. 12).  Structure of arrays in one device buffer `data` of
 * dg_gaussian_floats(ld, sh_degree) floats:
 *   floats [0, 4 ld)        float4 per Gaussian: (p.x, p.y, p.z, opacity logit)
 *   floats [4 ld, 8 ld)     float4 per Gaussian: quaternion (w, x, y, z), any norm
 *   floats [8 ld, 12 ld)    float4 per Gaussian: (log s.x, log s.y, log s.z, 0)
 *   floats [12 ld + j ld)   SH plane j = 3 k + channel, k = l*l + l + m the real
 *                           SH index (Condon-Shortley phase), j < 3 (D+1)^2
 * ld >= n, ld % 4 == 0, data 16-byte aligned.  Gradients, Adam moments, duals
 * u and the penalty anchor use the same layout. */
typedef struct dg_gaussians {
    float* data;
    int64_t n;
    int64_t ld;
    int32_t sh_degree; /* 0..3 */
    int32_t reserved;
} dg_gaussians;

/* floats needed for a parameter set of leading dimension ld */
int64_t dg_gaussian_floats(int64_t ld, int sh_degree);

/* ---- cameras and the batch plan ------------------------------------------ */
/* Pinhole camera, OpenCV axes (x right, y down, z forward): a world point p
 * maps to R p + t; pixel (px, py) covers [px, px+1) x [py, py+1) and is
 * sampled at its centre.  View v renders the copies of block `block`.
 * The fields after `block` are filled by dg_plan_views. */
typedef struct dg_camera {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];       /* world -> camera rotation, row-major */
    float t[3];       /* world -> camera translation         */
    float campos[3];  /* camera centre (for the SH view direction) */
    float near_z;     /* copies with camera z <= near_z are culled */
    int32_t block;
    /* derived */
    int32_t tiles_x, tiles_y;
    int32_t tile_off;  /* first tile of this view in the batch numbering */
    int32_t reserved;
    int64_t rec_off;   /* first projected record of this view */
    int64_t pix_off;   /* first pixel of this view in the batch image buffers */
    int64_t gauss_begin, gauss_end; /* copy range of `block` */
} dg_camera;

/* Batch plan: K blocks of copies [blk_off[k], blk_off[k+1]) and the views of
 * each block [blk_view_off[k], blk_view_off[k+1]) (views grouped by block in
 * ascending order).  Record r of view v is copy gauss_begin + (r - rec_off). */
typedef struct dg_plan {
    int32_t n_views, n_blocks;
    int32_t tile_w, tile_h;
    int64_t n_rec;     /* sum over views of the copies of its block */
    int64_t n_tiles;   /* sum over views of tiles_x * tiles_y      */
    int64_t n_pixels;  /* sum over views of width * height         */
    int64_t blk_off[DG_MAX_BLOCKS + 1];
    int32_t blk_view_off[DG_MAX_BLOCKS + 1];
    int32_t max_width, max_height;  /* largest view in the batch */
    /* compositing variant (set to 4, 2 by dg_plan_views; a tuner may change
     * them): warps per tile in {1, 2, 4, 8} (8 / warps pixels per thread) and
     * instances staged per thread per round in {1, 2} */
    int32_t raster_warps, raster_stage;
    /* the backward's variant, same ranges; 0, 0 (the dg_plan_views default)
     * = the forward's */
    int32_t raster_warps_bwd, raster_stage_bwd;
} dg_plan;

/* Fill the derived camera fields (host array cams[n_views]) and the plan.
 * blk_off: host, n_blocks + 1 entries.  Tile shapes: tile_w * tile_h == 256
 * with tile_w in {8, 16, 32}.  Fails with DG_ERR_INVALID if views are not
 * grouped by ascending block, a size is non-positive, or a count overflows
 * 32-bit tile / record numbering. */
int dg_plan_views(dg_camera* cams, int n_views, const int64_t* blk_off, int n_blocks,
                  int tile_w, int tile_h, dg_plan* plan);

/* ---- projection (K1) ------------------------------------------------------ */
/* Projected record of (view, copy): three float4 per record at rec[3 r + i]:
 *   rec[3r+0] = (mean2d.x, mean2d.y, conic.a, conic.b)
 *   rec[3r+1] = (conic.c, opacity, colour.r, colour.g)
 *   rec[3r+2] = (colour.b, depth, 0, 0)
 * where conic = inverse of the 2D covariance J W Sigma W^T J^T + 0.3 I,
 * colour = max(0, sum_k f_k Y_k(d) + 0.5), d the unit view direction,
 * opacity = sigmoid(logit), depth = camera z.  rect[r] = (x0 | y0 << 16,
 * x1 | y1 << 16): the covered tiles [x0, x1) x [y0, y1), from the radius
 * ceil(3 sqrt(lambda_max)); x0 == x1 marks a culled record, whose `rec` is
 * left unwritten.  Culled: camera z <= near_z, |x/z| > 1.3 W / (2 fx),
 * |y/z| > 1.3 H / (2 fy), or no tile covered. */
int dg_project(const dg_gaussians* x, const dg_camera* dev_cams, const dg_plan* plan,
               float* rec, uint32_t* rect, void* stream);

/* ---- tile binning and the key sort (K2-K4) ------------------------------- */
/* One instance per (record, covered tile), key = (tile << 32) | bits(depth),
 * value = record index, sorted ascending by (key, value).  A tile of the
 * record's rectangle is covered when some pixel centre of it can reach
 * alpha >= 1/255: min over the tile's pixel-centre box of q(d) = a dx^2 +
 * 2 b dx dy + c dy^2 is at most 2 ln(255 o) (1 + 2^-10) + 2^-6 (a widened
 * form of Eq. 2's 1/255 skip; the compositing would skip every pair of the
 * other tiles, so no image or gradient depends on it).  Outputs: vals
 * (capacity entries), keys (optional, NULL to skip), ranges (device
 * uint32[3 n_tiles]): ranges[2 t], ranges[2 t + 1] = first and end index of
 * tile t (empty tiles: start == end), then ranges[2 n_tiles + i] = the i-th
 * tile of the compositing's work order (every tile once, by descending
 * instance count n in buckets set by n's leading one bit and the two bits
 * after it, empty tiles last; the order within a bucket is unspecified),
 * dev_count[0] = number of instances M.  If M > capacity the DG_STATUS_CAPACITY bit is set and
 * every range is emptied (nothing is rendered); retry with capacity >= M.
 * Workspace: dg_bin_sort_workspace_size bytes of device memory (it holds,
 * among the per-tile counters and the unsorted pairs, a list of the records
 * with a non-empty rectangle, 4 bytes per record, over which the expansion
 * runs).  A workspace of at least dg_bin_sort_workspace_min_size bytes but
 * less than that runs without the list (every record scanned; the same
 * output, slower in scenes where few records are visible); below the
 * minimum, DG_ERR_WORKSPACE. */
size_t dg_bin_sort_workspace_size(const dg_plan* plan, int64_t capacity);
size_t dg_bin_sort_workspace_min_size(const dg_plan* plan, int64_t capacity);
int dg_bin_sort(const float* rec, const uint32_t* rect, const dg_camera* dev_cams,
                const dg_plan* plan, int64_t capacity, uint64_t* keys, uint32_t* vals,
                uint32_t* ranges, uint32_t* dev_count, void* ws, size_t ws_bytes,
                uint32_t* dev_status, void* stream);

/* ---- binning without caller-provided scratch ------------------------------ */
/* The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory when they bin, e.g. a plugin inside an
 * application whose allocator owns the device's memory, or a latency-bound
 * loop that must not pay cudaMalloc's implicit synchronisation.  Same inputs,
 * outputs and results as dg_bin_sort, but the scratch comes from a static
 * device array of 40 MiB that the library reserves on every GPU that loads it,
 * for the life of the process.  Its arguments are checked as dg_bin_sort's are
 * (plan, capacity, null and misaligned pointers: DG_ERR_INVALID before any
 * launch).  Limits: plan->n_tiles <= DG_NOALLOC_MAX_TILES and
 * capacity <= DG_NOALLOC_MAX_INSTANCES, else DG_ERR_TOO_LARGE before any
 * launch.  The first call on a device looks up the array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.  Every call shares the array: calls whose work overlaps
 * on the GPU (unordered streams, concurrent host threads) race and give wrong
 * results; serialise them.  Allocates and frees nothing. */
#define DG_NOALLOC_MAX_TILES 262144
#define DG_NOALLOC_MAX_INSTANCES 4194304
int dg_bin_sort_noalloc(const float* rec, const uint32_t* rect, const dg_camera* dev_cams,
                        const dg_plan* plan, int64_t capacity, uint64_t* keys, uint32_t* vals,
                        uint32_t* ranges, uint32_t* dev_count, uint32_t* dev_status, void* stream);

/* ---- compositing (K5) ------------------------------------------------------ */
/* Eq. 2 front to back per pixel over its tile's instances: alpha =
 * min(0.99, opacity * G), G = exp(-0.5 d^T conic d); pairs with alpha < 1/255
 * are skipped; the pass stops before T (1 - alpha) < 1e-4; pixel = sum + T bg.
 * image: [3][H][W] per view at 3 * pix_off; T_final, last: [H][W] at pix_off
 * (last = list position + 1 of the last composited instance, 0 if none).
 * bg: host float[3].  ranges: as dg_bin_sort wrote them, work order
 * included (the tiles are composited in that order). */
int dg_rasterize_fwd(const float* rec, const uint32_t* vals, const uint32_t* ranges,
                     const dg_camera* dev_cams, const dg_plan* plan, const float* bg,
                     float* image, float* T_final, uint32_t* last, void* stream);

/* dg_rasterize_fwd with the same outputs, plus work counters for measuring:
 * counts (device uint64[2], 8-byte aligned, zeroed by the call, then
 * accumulated on the stream) receives [0] the (pixel, instance) pairs
 * examined while the pixel was still compositing and [1] the pairs that
 * contributed (alpha >= 1/255, before the stop).  The pairs the backward
 * visits are the sum of `last`; the ones it differentiates are counts[1]. */
int dg_rasterize_count(const float* rec, const uint32_t* vals, const uint32_t* ranges,
                       const dg_camera* dev_cams, const dg_plan* plan, const float* bg,
                       float* image, float* T_final, uint32_t* last, uint64_t* counts, void* stream);

/* ---- losses (K6, K11) ----------------------------------------------------- */
/* Per view v: loss[v] = w_l1 * mean |I - I*| + w_ssim * (1 - mean SSIM(I, I*))
 * (Eq. 3 with lambda = w_ssim and the L1 weight w_l1; SSIM with an 11x11
 * Gaussian window, sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, zero padding) and
 * dL_dimage = d loss[v] / d image.  loss: device double[n_views], overwritten.
 * dg_loss_l1 is the w_ssim = 0 case.  Workspace for SSIM:
 * dg_loss_workspace_size bytes. */
int dg_loss_l1(const float* image, const float* target, const dg_camera* dev_cams,
               const dg_plan* plan, float w_l1, double* loss, float* dL_dimage, void* stream);
size_t dg_loss_workspace_size(const dg_plan* plan);
int dg_loss_dssim(const float* image, const float* target, const dg_camera* dev_cams,
                  const dg_plan* plan, float w_l1, float w_ssim, double* loss,
                  float* dL_dimage, void* ws, size_t ws_bytes, void* stream);

/* ---- backward (K7 + K8) ---------------------------------------------------- */
/* Analytic adjoint of dg_project + dg_rasterize_fwd: each tile is walked
 * back to front from T_final and last.  drec: device scratch, 12 floats per
 * record (zeroed here, then dL/d(mean2d, conic, opacity, colour) accumulated).
 * grads: same layout as x, OVERWRITTEN with dL/dx for every copy (zero for
 * copies no view sees).  bg: host float[3]. */
int dg_rasterize_bwd(const float* rec, const uint32_t* rect, const uint32_t* vals,
                     const uint32_t* ranges, const dg_camera* dev_cams, const dg_plan* plan,
                     const float* bg, const float* T_final, const uint32_t* last,
                     const float* dL_dimage, const dg_gaussians* x, float* drec,
                     dg_gaussians* grads, void* stream);

/* The compositing adjoint alone (the first half of dg_rasterize_bwd): drec
 * (12 floats per record) zeroed, then dL/d(mean2d, conic, opacity, colour)
 * accumulated.  Feeds dg_xstep_from_records.  rect: the projection's
 * rectangles, or NULL.  Given, only the records with a non-empty rectangle
 * (the records the adjoint adds to and the projection adjoint reads) are
 * zeroed and the other entries of drec are left as they are; NULL zeroes
 * every record. */
int dg_rasterize_bwd_records(const float* rec, const uint32_t* rect, const uint32_t* vals, const uint32_t* ranges,
                             const dg_camera* dev_cams, const dg_plan* plan, const float* bg,
                             const float* T_final, const uint32_t* last, const float* dL_dimage,
                             float* drec, void* stream);

/* Deterministic form of dg_rasterize_bwd_records: the same adjoint with the
 * same tile walk, but the backward of each (record, tile) pair is stored in
 * its own slot of part (9 floats per slot) instead of being added to drec
 * by atomics, and drec[r] is then summed from record r's slots in tile
 * order; drec (12 floats per record, the last 3 zero) is therefore the same
 * bit for bit from run to run, which makes a resumed run repeat an
 * uninterrupted one exactly.  A record's slots are one per tile of its
 * rectangle: the slot offsets are the exclusive sum of the rectangle areas
 * (computed here into ws, size dg_rasterize_bwd_slots_workspace_size), and
 * the total is written to *dev_slots (device uint64).  part: device,
 * 9 * slot_capacity floats, zeroed here.  If the total exceeds
 * slot_capacity, DG_STATUS_CAPACITY is set in *dev_status and the records
 * whose slots fall beyond it get zero gradients (retry with a larger part).
 * Always one warp per tile (the plan's backward staging depth is kept). */
size_t dg_rasterize_bwd_slots_workspace_size(const dg_plan* plan);
int dg_rasterize_bwd_slots(const float* rec, const uint32_t* rect, const uint32_t* vals,
                           const uint32_t* ranges, const dg_camera* dev_cams, const dg_plan* plan,
                           const float* bg, const float* T_final, const uint32_t* last,
                           const float* dL_dimage, float* part, int64_t slot_capacity, void* ws,
                           size_t ws_bytes, uint64_t* dev_slots, uint32_t* dev_status, float* drec,
                           void* stream);

/* The projection adjoint (K8) and the x-step (K9, Eq. 8a / 12a) in one pass,
 * for batches whose blocks have at most one view each: every copy then has
 * at most one record, so each thread finishes its copy's dL/dx from drec
 * and takes the Adam + penalty step on it at once; the gradient never goes
 * to memory.  Same result as dg_rasterize_bwd's second half followed by
 * dg_adam_admm_step (x, m, v updated in place; the parameters before the
 * step are the ones differentiated).  rect: the forward's rectangles.
 * DG_ERR_INVALID if a block of the plan has more than one view (use those
 * two calls then). */
int dg_xstep_from_records(const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                          const float* drec, dg_gaussians* x, dg_gaussians* m, dg_gaussians* v,
                          const dg_gaussians* anchor, const uint8_t* copy_shared, const float* rho,
                          const float* lr, float beta1, float beta2, float eps, int step,
                          const int32_t* dev_step, void* stream);

/* dg_xstep_from_records in two parts that together take the same step
 * (bit for bit), by groups of 128 consecutive copies: part 1 steps the
 * groups none of whose copies has a kept record (zero rendering gradient:
 * Adam on the penalty alone; drec is not read and may be NULL), part 2 the
 * others (the fused adjoint + step).  Part 1 reads only the rectangles of
 * the projection, so it can run on another stream alongside binning,
 * compositing and the loss; `ctas` > 0 bounds its grid (a grid-stride loop
 * over the groups), so that it leaves most of each SM to the kernels beside
 * it; 0 = one CTA per group.  part 0 = the whole step.
 * z_unshared (may be NULL): the global model of an iteration whose
 * consensus follows; every copy with copy_shared[c] == 0 then also stores
 * its stepped value at z_unshared[copy_gid[c]] (int32, device) -- the
 * consensus's z = x for a global held by one block, taken in this pass, so
 * that dg_admm_consensus can be given the shared globals alone (a z whose n
 * counts them, when they come first in the global order).  copy_gid[c]
 * must be < z_unshared->n for those copies.
 * Same arguments and errors as dg_xstep_from_records; DG_ERR_INVALID for a
 * part outside 0..2, a negative ctas, or z_unshared with another SH degree
 * or without copy_gid / copy_shared. */
int dg_xstep_part(int part, int ctas, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                  const float* drec, dg_gaussians* x, dg_gaussians* m, dg_gaussians* v,
                  const dg_gaussians* anchor, const uint8_t* copy_shared, const float* rho,
                  const float* lr, float beta1, float beta2, float eps, int step,
                  const int32_t* dev_step, dg_gaussians* z_unshared, const int32_t* copy_gid,
                  void* stream);

/* Part 1 of dg_xstep_part (the groups of 128 copies without a kept record,
 * Eq. 8a / 12a with a zero rendering gradient), streamed: the same result
 * bit for bit, taken by `ctas` persistent CTAs (0 = one per SM) that move
 * each listed group's x, m, v and anchors through shared memory by
 * asynchronous copies.  A few CTAs then keep HBM busy in the registers and
 * shared memory that the compositing adjoint leaves free, so the call can
 * run on another stream beside dg_rasterize_bwd_records.  Two launches on
 * `stream`: the list of those groups (it reads the projection's rectangles),
 * then the step over it at the device's highest stream priority.
 * ws: device memory of dg_xstep_stream_workspace_size(x) bytes, 16-byte
 * aligned, owned by the caller and not used by another call in flight
 * (a counter pair, then the list).  Same arguments and errors as
 * dg_xstep_part with part 1; DG_ERR_INVALID for ctas outside 0..65535 or a
 * missing or misaligned ws, DG_ERR_WORKSPACE if ws_bytes is too small. */
size_t dg_xstep_stream_workspace_size(const dg_gaussians* x);
int dg_xstep_stream(int ctas, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                    dg_gaussians* x, dg_gaussians* m, dg_gaussians* v, const dg_gaussians* anchor,
                    const uint8_t* copy_shared, const float* rho, const float* lr, float beta1, float beta2,
                    float eps, int step, const int32_t* dev_step, dg_gaussians* z_unshared,
                    const int32_t* copy_gid, void* ws, size_t ws_bytes, void* stream);

/* dg_xstep_stream's two launches as separate calls, and part 2 over a list:
 * dg_xstep_groups lists, in ws (as for dg_xstep_stream), every group of 128
 * copies once: the groups without a kept record from the front, the others
 * from the back.  dg_xstep_listed then takes a part of dg_xstep_part's step
 * (Eq. 8a / 12a) over those lists: part 1 streamed as dg_xstep_stream does
 * (`ctas` as there), part 2 (the fused adjoint + step, after the compositing
 * adjoint; `ctas` unused) with the n-th CTA on the n-th listed group with a
 * kept record, so that the CTAs past the list, which find nothing to step,
 * all come after those that step.  The two parts together take
 * dg_xstep_part's step, bit for bit.  The caller
 * orders dg_xstep_groups before both parts (on another stream: by an event
 * recorded after it) and leaves ws alone until both have run.
 * dg_xstep_groups: arguments as dg_xstep_stream's (x gives the copy count);
 * DG_ERR_INVALID for a bad plan, a block with two views, a missing or
 * misaligned rect / dev_cams / ws, DG_ERR_WORKSPACE for a small ws_bytes.
 * dg_xstep_listed: arguments and errors as dg_xstep_part's, plus ws and
 * ws_bytes as dg_xstep_stream's; DG_ERR_INVALID for a part other than 1 or 2
 * or ctas outside 0..65535. */
int dg_xstep_groups(const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                    const dg_gaussians* x, void* ws, size_t ws_bytes, void* stream);
int dg_xstep_listed(int part, int ctas, const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                    const float* drec, dg_gaussians* x, dg_gaussians* m, dg_gaussians* v,
                    const dg_gaussians* anchor, const uint8_t* copy_shared, const float* rho,
                    const float* lr, float beta1, float beta2, float eps, int step,
                    const int32_t* dev_step, dg_gaussians* z_unshared, const int32_t* copy_gid,
                    void* ws, size_t ws_bytes, void* stream);

/* ---- ADMM (K9, K10) -------------------------------------------------------- */
/* x-step (Eq. 8a / 12a): one Adam step on every local copy with gradient
 * g + rho_grp (x - anchor) on shared copies (copy_shared[c] != 0), where the
 * anchor of a shared copy is z_{g(c)} - u_c, kept by dg_admm_consensus and
 * dg_admm_anchor.  Groups in the paper's order (Eq. 12): 0 p (mean),
 * 1 q (rotation), 2 s (scale), 3 f (SH), 4 o (opacity): rho[5], in host
 * memory (read at the call) or device memory (read when the kernels run,
 * e.g. as dg_admm_adapt leaves it).
 * lr[6] (host): p, q, s, SH DC, SH rest, o.  Moments m, v updated in place;
 * bias correction with the iteration number `step` >= 1, or, if dev_step is
 * not NULL, with the int32 it points to in device memory (read when the
 * kernel runs, so a captured graph can be replayed for successive steps).
 * anchor may be NULL (no penalty: plain Adam). */
int dg_adam_admm_step(dg_gaussians* x, const dg_gaussians* g, dg_gaussians* m,
                      dg_gaussians* v, const dg_gaussians* anchor, const uint8_t* copy_shared,
                      const float* rho, const float* lr, float beta1, float beta2, float eps,
                      int step, const int32_t* dev_step, void* stream);

/* Consensus (Eq. 8b-c / 12b-c) over the global model z (n_global Gaussians).
 * Sharing map as CSR: the copies of global i are g_copies[g_off[i] ..
 * g_off[i+1]) (device).  For a global held by n_i >= 2 blocks:
 *   xh_k = alpha x_k + (1 - alpha) z     (over-relaxation, Sec. 3.3)
 *   z    = (1/n_i) sum_k (xh_k + u_k)    (complete form of Eq. 8b)
 *   u_k += xh_k - z                      (Eq. 8c)
 *   anchor_k = z - u_k                   (for the next x-steps)
 * A global held by one block gets z = x.  The globals processed are the
 * first z->n of the CSR: a caller whose x-step already stored the unshared
 * globals (dg_xstep_part with z_unshared) and numbers the shared globals
 * first passes a z whose n counts the shared ones (the same memory).
 * residuals (device double[10], may be NULL, overwritten): per group the
 * squared primal residual sum ||x_k - z||^2 (0..4) and squared dual residual
 * rho^2 n_i ||z - z_prev||^2 (5..9), shared globals only (Eq. 9). */
int dg_admm_consensus(const dg_gaussians* x, dg_gaussians* u, dg_gaussians* z,
                      dg_gaussians* anchor, const int64_t* g_off, const int32_t* g_copies,
                      const float* rho, float alpha, double* residuals, void* stream);

/* Adds 1 to the device step counter *dev_step (int32, 4-byte aligned) on the
 * stream: the x-step calls read their Adam step from it, so an iteration
 * that advances it on the device before its x-step can be replayed from a
 * graph, back to back, with each replay seeing its own count. */
int dg_step_advance(int32_t* dev_step, void* stream);

/* ---- Densification under consensus (Sec. 4, 3DGS adaptive density control) ---
 * Decision codes of dg_densify_decide. */
#define DG_DENSIFY_KEEP 0
#define DG_DENSIFY_PRUNE 1
#define DG_DENSIFY_CLONE 2
#define DG_DENSIFY_SPLIT 3

/* Adds one iteration's densification statistic: for every record r of the
 * plan whose rectangle is non-empty, copy c of r (its view's gauss_begin +
 * r - rec_off) gets stats[2c] += |(drec[12r] W/2, drec[12r+1] H/2)| (the norm
 * of its projected mean's gradient in normalised device units, W x H its
 * view) and stats[2c+1] += 1.  stats: device float[2 n_copies], accumulated
 * (the caller zeroes it after each densification); rect / drec: the forward's
 * rectangles and dg_rasterize_bwd_records' gradients. */
int dg_densify_stats(const uint32_t* rect, const dg_camera* dev_cams, const dg_plan* plan,
                     const float* drec, float* stats, void* stream);

/* Bytes of workspace dg_densify_decide needs for n globals. */
size_t dg_densify_workspace_size(int64_t n_global);

/* The densification decision per global Gaussian of z, from the summed
 * statistics of its copies (CSR g_off / g_copies as for dg_admm_consensus,
 * summed in that order in FP32): DG_DENSIFY_PRUNE if the opacity logit is
 * below log(min_opacity / (1 - min_opacity)); else, if count > 0 and
 * sum >= grad_threshold * count, DG_DENSIFY_SPLIT when the largest
 * log-scale exceeds log(percent_dense * extent) and DG_DENSIFY_CLONE
 * otherwise; else DG_DENSIFY_KEEP.  codes: device int32[n]; counts: device
 * uint32[n] (outputs of each Gaussian: 0, 1, 2, 2); offsets: device
 * uint32[n + 1], their exclusive scan with the total at offsets[n] (n + 1
 * entries; must fit in 32 bits).  ws: dg_densify_workspace_size bytes. */
int dg_densify_decide(const dg_gaussians* z, const int64_t* g_off, const int32_t* g_copies,
                      const float* stats, float grad_threshold, float percent_dense, float extent,
                      float min_opacity, int32_t* codes, uint32_t* counts, uint32_t* offsets,
                      void* ws, size_t ws_bytes, void* stream);

/* The densified set: global i writes its outputs at out[offsets[i] ..]:
 * KEEP itself; CLONE itself and an exact copy; SPLIT two children with mean
 * mu + R(q) (S xi_h) (R of the normalised quaternion, S = exp(log-scale),
 * xi_h = normals[6i + 3h .. 6i + 3h + 2], standard normals drawn by the
 * caller) and log-scales reduced by ln 1.6, the other parameters copied;
 * PRUNE nothing.  src[o]: the parent of output o; original[o] = 1 where o is
 * the parent itself (KEEP, or the first output of CLONE), whose optimiser
 * state and duals carry over.  out: same SH degree, n >= offsets[n]. */
int dg_densify_emit(const dg_gaussians* z, const int32_t* codes, const uint32_t* offsets,
                    const float* normals, dg_gaussians* out, int32_t* src, uint8_t* original,
                    void* stream);

/* The copy layout of the densified set, built on the device in the old
 * layout's order: each Gaussian's outputs take its place.  From the old
 * layout (n_global globals with their sharing map g_off[n_global + 1] /
 * g_copies, and copy_gid[n_copies] listing the blocks' copies, blocks
 * concatenated) and dg_densify_decide's codes and offsets:
 *   copy_offsets[c] (uint32[n_copies + 1]): exclusive sum over the old
 *     copies of their Gaussian's output count, total last; old copy c of
 *     global p becomes the new copies copy_offsets[c] + h, h < outputs of p,
 *     in the same block (block k's new range starts at
 *     copy_offsets[old blk_off[k]]; its shared copies still come first);
 *   new_copy_gid[copy_offsets[c] + h] = offsets[p] + h;
 *   new_g_off / new_g_copies: the new sharing map (int64[n_new + 1] /
 *     int32), each new global's copies in ascending block;
 *   carry[new copy] = the old copy whose optimiser state and dual it takes
 *     over (the Gaussian is its parent itself: KEEP, or the first output of
 *     CLONE), else -1.
 * Shared globals stay numbered first (their outputs are shared, with the
 * parent's blocks).  new_g_copies, new_copy_gid and carry hold
 * copy_offsets[n_copies] entries (at most 2 n_copies).  ws:
 * dg_densify_layout_workspace_size bytes, 256-byte aligned.  Device
 * pointers; n_global and n_copies below 2^30. */
size_t dg_densify_layout_workspace_size(int64_t n_global, int64_t n_copies);
int dg_densify_layout(const int32_t* codes, const uint32_t* offsets, int64_t n_global, const int64_t* g_off,
                      const int32_t* g_copies, const int32_t* copy_gid, int64_t n_copies,
                      int64_t* new_g_off, int32_t* new_g_copies, int32_t* new_copy_gid, int32_t* carry,
                      uint32_t* copy_offsets, void* ws, size_t ws_bytes, void* stream);

/* counts[b] = #{i < n : v[i] == lo + b} for b < n_bins (1..64; device int32
 * v, device uint32 counts, overwritten); values outside the bins are not
 * counted.  The densification's tallies (codes per kind, carried copies). */
int dg_histogram_i32(const int32_t* v, int64_t n, int32_t lo, int n_bins, uint32_t* counts, void* stream);

/* ---- 8-bit images (training targets cross the host link as bytes) -------
 * dg_image_u8_to_f32: dst[i] = src[i] / 255 for i < n (device; src 4-byte
 * and dst 16-byte aligned).  dg_image_f32_to_u8:
 * dst[i] = round(clamp(src[i], 0, 1) * 255). */
int dg_image_u8_to_f32(const uint8_t* src, float* dst, int64_t n, void* stream);
int dg_image_f32_to_u8(const float* src, uint8_t* dst, int64_t n, void* stream);

/* The opacity reset of the density control: every opacity of g above `cap`
 * (0 < cap < 1) is brought down to it, i.e. the logit becomes
 * min(logit, log(cap / (1 - cap))) (formed in double, rounded once); where m
 * / v are given (Adam's moments in g's layout, may be NULL) their opacity
 * lanes are zeroed. */
int dg_reset_opacity(dg_gaussians* g, float cap, dg_gaussians* m, dg_gaussians* v, void* stream);

/* ---- Copy layout of a block membership (host, no GPU) ---------------------
 * member[i]: bit k set when point i belongs to block k (K <= DG_MAX_BLOCKS,
 * every point in at least one block).  dg_layout_copies returns the number
 * of copies (the set bits), -1 on bad arguments.  dg_layout numbers the
 * globals (order[g] = the point that becomes global g): those in two or more
 * blocks first (*n_shared of them), each part by (lowest block, Z-order of
 * (x, y) = xy[2i], xy[2i+1] quantised to 16 bits over their bounding box);
 * copy_gid lists block k's copies in [blk_off[k], blk_off[k+1]), its shared
 * globals in ascending id then its unshared ones (blk_nshared[k] shared);
 * g_off[n + 1] / g_copies: each global's copies in ascending block.  Arrays
 * are host memory sized n (order, g_off: n + 1), K + 1, K and the copy count.
 * DG_ERR_INVALID on bad sizes, null pointers or a point in no block. */
int64_t dg_layout_copies(const uint64_t* member, int64_t n);
int dg_layout(const double* xy, const uint64_t* member, int64_t n, int K, int32_t* order,
              int32_t* copy_gid, int64_t* blk_off, int64_t* blk_nshared, int64_t* g_off,
              int32_t* g_copies, int64_t* n_shared);

/* The block membership of a re-laid-out set: member[j] = the bitmask of the
 * blocks (bit k: block k) that hold a copy of old global parent[j], read
 * from the old block offsets (old_blk_off, K + 1) and sharing map
 * (old_g_off[n_old + 1] / old_g_copies).  parent, member: n_new entries.
 * Host memory; no GPU.  DG_ERR_INVALID on bad sizes, null pointers or an
 * id out of range (member then partly written). */
int dg_layout_membership(const int64_t* old_blk_off, const int64_t* old_g_off, const int32_t* old_g_copies,
                         int64_t n_old, int K, const int32_t* parent, int64_t n_new, uint64_t* member);

/* The state carried across a re-layout (densification, Sec. 4, under the
 * consensus): for every copy e of a new layout, carry[e] = the copy of the
 * old layout, in the same block, of old global parent[g] when original[g]
 * != 0 (g = the new global of e, a Gaussian that is its parent itself),
 * else -1.  Both layouts are given by their block offsets (old_blk_off,
 * new_blk_off: K + 1) and sharing maps (old_g_off[n_old + 1] /
 * old_g_copies, new_g_off[n_new + 1] / new_g_copies: each global's copies
 * in ascending block); parent, original: n_new entries; carry: the new
 * copy count.  Host memory; no GPU.  DG_ERR_INVALID on bad sizes, null
 * pointers or an id out of range (carry then partly written). */
int dg_layout_carry(const int64_t* old_blk_off, const int64_t* old_g_off, const int32_t* old_g_copies,
                    int64_t n_old, int K, const int64_t* new_blk_off, const int64_t* new_g_off,
                    const int32_t* new_g_copies, const int32_t* parent, const uint8_t* original,
                    int64_t n_new, int32_t* carry);

/* dst row r = src row idx[r] (all fields and SH planes) for r < dst->n;
 * rows with idx[r] < 0 are left unchanged.  The rows move between the
 * library layouts of the two sets (same SH degree, any ld); idx[r] must be
 * < src->n. */
int dg_gather_rows(const dg_gaussians* src, const int32_t* idx, dg_gaussians* dst, void* stream);

/* Adaptive penalty (Sec. 3.3, Eq. 10): when rho_grp changes to rho'_grp the
 * scaled duals u = y / rho follow as u_grp *= rho_grp / rho'_grp.  This call
 * multiplies each group of u on shared copies by factor[5] (host); rerun
 * dg_admm_anchor afterwards. */
int dg_admm_scale_duals(dg_gaussians* u, const uint8_t* copy_shared, const float* factor, void* stream);

/* Adaptive penalty on the device (Sec. 3.3, Eq. 10), for a loop that keeps
 * rho in device memory: rho (device, float[5]) may then be passed as the rho
 * of dg_adam_admm_step, dg_xstep_part and dg_admm_consensus, which read it
 * when their kernels run.  After a consensus that wrote `residuals` (device,
 * double[10]: squared primal per group, then squared dual), per group g
 * with r = sqrt(primal_g) and s = sqrt(dual_g): rho_g *= tau_inc when
 * r > mu s, rho_g /= tau_dec when s > mu r, unchanged otherwise -- only
 * while the iteration t = *dev_step - 1 is below freeze_after (dev_step:
 * the Adam step counter, advanced at the start of each iteration).  Writes
 * factor (device, float[5]) = old rho_g / new rho_g.  No host
 * synchronisation: the whole rule runs in one small kernel, so it can sit
 * inside a captured graph.  DG_ERR_INVALID on a null or misaligned pointer
 * or mu, tau_inc, tau_dec below 1. */
int dg_admm_adapt(const double* residuals, float* rho, float* factor, const int32_t* dev_step, float mu,
                  float tau_inc, float tau_dec, int freeze_after, void* stream);

/* The scaled duals and anchors after dg_admm_adapt: on every shared copy
 * u_grp *= factor[grp] (factor: device, float[5]) and anchor = z_{g(c)} - u,
 * in one pass; when every factor is 1 the kernel returns without touching
 * memory.  u, anchor: same layout; z: the global set (same SH degree). */
int dg_admm_rescale(dg_gaussians* u, const dg_gaussians* z, dg_gaussians* anchor, const int32_t* copy_gid,
                    const uint8_t* copy_shared, const float* factor, void* stream);

/* anchor_c = z_{copy_gid[c]} - u_c for every shared copy (initialisation). */
int dg_admm_anchor(const dg_gaussians* z, const dg_gaussians* u, const int32_t* copy_gid,
                   const uint8_t* copy_shared, dg_gaussians* anchor, void* stream);

/* ---- serving render (K12) ------------------------------------------------ */
/* Render n_views requests (any mix of resolutions) of the global model z:
 * dg_project + dg_bin_sort + dg_rasterize_fwd on one plan with a single
 * block holding all of z.  dg_render_plan fills host_cams' derived fields
 * and the plan (copy host_cams to dev_cams afterwards); buffers are sized
 * from the plan.  Workspace: dg_render_workspace_size. */
int dg_render_plan(dg_camera* host_cams, int n_views, int64_t n_gauss, int tile_w,
                   int tile_h, dg_plan* plan);
size_t dg_render_workspace_size(const dg_plan* plan, int64_t capacity);
int dg_render(const dg_gaussians* z, const dg_camera* dev_cams, const dg_plan* plan,
              const float* bg, int64_t capacity, float* image, void* ws, size_t ws_bytes,
              uint32_t* dev_count, uint32_t* dev_status, void* stream);

/* ---- scene splitting (host pre-processing; Sec. 3.2, Alg. 1) --------------- */
/* Recursive bipartite split of n ground-plane positions xy (host, double[2n],
 * x and y of point i at 2i, 2i+1; finite) into K cells, 1 <= K <= 64.
 * Starting from one cell holding every point with a budget of K leaves,
 * cells are processed level by level in first-in first-out order (Alg. 1);
 * a cell with budget k >= 2 is cut across the longer side of the tight box
 * of its points (ties: x), the lower child taking the first floor(n_c
 * floor(k/2) / k) of its n_c points in (coordinate, index) order and budget
 * floor(k/2), the upper child the rest and budget k - floor(k/2); cells with
 * budget 1 are kept.  For K a power of two this is the median bipartition of
 * Alg. 1, and every cell ends with floor(n/K) or ceil(n/K) points.
 * Outputs (host, caller-owned): cell[i] (int32[n]) the cell of point i in the
 * final order of the cell list; boxes (double[4K]) xmin, xmax, ymin, ymax of
 * each cell's tight box (an empty cell gets +inf, -inf, +inf, -inf).
 * DG_ERR_INVALID on a bad K, a null pointer with n > 0 or a non-finite
 * coordinate; nothing is written then.  No GPU work. */
int dg_scene_split(const double* xy, int64_t n, int K, int32_t* cell, double* boxes);

/* Overlap by a scale factor (Sec. 3.2): each box is expanded about its centre
 * by s >= 1 on both sides (centre c = (lo + hi) / 2, half side s (hi - lo) / 2,
 * evaluated in double in that order), and position i belongs to every block
 * whose expanded box contains it (closed intervals).  own (int32[n] or NULL)
 * adds each point's own cell; nearest != 0 gives a position covered by no
 * expanded box the block of the nearest one (ties: lowest index), as for
 * camera centres outside the point cloud's boxes.  member (host, uint64[n],
 * caller-owned) receives bit k set for block k.  Empty boxes contain nothing.
 * DG_ERR_INVALID on a bad K or s, an own[i] outside [0, K), a null pointer
 * with n > 0 or a non-finite coordinate.  No GPU work. */
int dg_scene_assign(const double* xy, int64_t n, const double* boxes, int K, double s,
                    const int32_t* own, int nearest, uint64_t* member);

/* ---- misc ------------------------------------------------------------------ */
const char* dg_version(void);
/* number of kernel launches this library has enqueued since load (monotone) */
uint64_t dg_launch_count(void);

/* ---- measurement helper (not part of the method) -------------------------- */
/* dg_probe_fma: launches blocks x 256 threads, each running 8 independent
 * chains of iters x 16 FP32 fused multiply-adds, and writes one float per
 * thread to out (device, blocks x 256 floats, caller-owned).  Returns the
 * FLOPs the launch performs (2 per multiply-add), or -1 on a bad argument or
 * launch error.  Timing the launch on `stream` gives the device's FP32 rate,
 * the denominator of the compositing kernels' roofline. */
int64_t dg_probe_fma(int iters, int blocks, float* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DOGS_H */
