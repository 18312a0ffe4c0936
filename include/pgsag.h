/*
 * pgsag.h -- C ABI of libpgsag.so: masked, tile-based differentiable
 * Gaussian-splat rasterisation (forward and backward) for PG-SAG's per-sub-region
 * optimisation (arXiv 2501.01677), hand-written CUDA for sm_103a (B300).
 *
 * What the library computes (paper passages):
 *   - Sec. 3.1, Eq. 1: each 3D Gaussian is projected to a 2D Gaussian (EWA,
 *     3DGS by citation), binned to image tiles, depth-sorted and alpha-blended
 *     front to back: C = sum_i c_i a_i T_i, T_i = prod_{j<i} (1 - a_j).
 *   - Sec. 3.1, Eq. 2-3: the same weights blend the camera-frame normal of each
 *     flattened Gaussian (N) and its camera-to-plane distance d_i (D).
 *   - Sec. 3.1, Eq. 4: unbiased depth Depth(p) = D / (-N(p) . K^-1 p~).
 *   - Sec. 4.1 / 4.2 / Sec. 5.3: only building-mask pixels are rendered and
 *     optimised, at the original image resolution.
 *   - Sec. 4.2, Eq. 8: boundary-aware normal loss (w = 0.1 on mask boundaries).
 *   - Sec. 4.3, Eq. 9: per-pixel / per-tile Gaussian counts for the
 *     gradient-constrained balance-load loss.
 *
 * Conventions (all entry points):
 *   - Every array argument is DEVICE memory owned by the caller, unless marked
 *     "host".  The library never allocates device memory and never synchronises
 *     the host inside a step call; work is enqueued on `stream`.
 *   - Floating-point arrays are float32, row-major, contiguous; float4 / uint2 /
 *     uint4 arrays must be 16-byte (uint2: 8-byte) aligned.
 *   - Return value: PGSAG_OK, or a negative status detected on the host
 *     (bad argument, launch failure).  Errors found on the device (capacity
 *     overflow, a bounded wait that ran out) are OR-ed as bit flags into the
 *     caller's `int32_t* status` (device); kernels that see a nonzero status
 *     return without work.  Nothing traps.
 *   - Views.  A step may render several views at once (sub-regions of uneven
 *     size, mixed resolutions).  Each view renders the Gaussian index range
 *     [g_begin, g_end) of the shared parameter arrays; a (view, Gaussian) pair has
 *     index pair_base + (g - g_begin).
 *   - Pixel arrays come in two layouts (Sec. 5.3: only mask pixels are
 *     rendered).  Dense arrays -- flags and the pixel-index map pidx, 5 bytes
 *     per image pixel -- concatenate the views' full images: pixel (x, y) of
 *     view v lives at pix_base + y * width + x.  Every other per-pixel array
 *     (targets, GC weights, rendered outputs, upstream gradients, scratch) is
 *     compact: indexed by the pixel's position q in px_list (the rendered set R
 *     of all views, grouped by active tile), so its size is |R| entries and
 *     consecutive threads touch consecutive entries.
 *     Per-tile arrays are concatenated with tile_base / sat_base; active tiles
 *     (tiles holding at least one rendered pixel) are numbered globally from
 *     act_base.
 *   - Pixel (x, y) has its centre at (x + 0.5, y + 0.5).  Camera axes follow
 *     OpenCV (x right, y down, z forward); x_cam = R x_world + t.
 */
#ifndef PGSAG_H
#define PGSAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* host-side status codes */
#define PGSAG_OK 0
#define PGSAG_ERR_ARG (-1)         /* null pointer, bad size, misalignment      */
#define PGSAG_ERR_CAPACITY (-2)    /* host-visible capacity/workspace too small */
#define PGSAG_ERR_CUDA (-3)        /* a CUDA launch or API call failed          */
#define PGSAG_ERR_TIMEOUT (-4)     /* reserved for bounded device waits         */
#define PGSAG_ERR_UNSUPPORTED (-5) /* parameter outside the supported range     */

/* device status bit flags (OR-ed into *status) */
#define PGSAG_DEV_CAPACITY 1u      /* duplicate count K exceeded the capacity   */
#define PGSAG_DEV_TIMEOUT 2u       /* a bounded spin-wait ran out               */
#define PGSAG_DEV_BOUNDS 4u        /* an index failed a bounds check            */

#define PGSAG_MAX_VIEWS 256
#define PGSAG_CHUNK 32             /* rendered pixels per warp work item        */
#define PGSAG_SH_COEFFS 16         /* SH degree 3, coefficient-major [N,16,3]   */
#define PGSAG_REC_FLOATS 16        /* projected record per (view, Gaussian)     */
#define PGSAG_GRAD2D_FLOATS 16     /* 2D gradient record per (view, Gaussian)   */

/* pixel flag bits (uint8 per pixel) */
#define PGSAG_PIX_MASK 1u          /* M: building mask pixel                     */
#define PGSAG_PIX_EDGE 2u          /* E: mask boundary (3x3 dilation - erosion)  */
#define PGSAG_PIX_RENDER 4u        /* R: rendered (3x3 dilation of M)            */

/*
 * One view.  Filled by the caller (host), uploaded as an array of
 * pgsag_view (device) for the step calls.  Fields marked (prep) are results of
 * pgsag_prep_flags / pgsag_prep_lists that the caller copies in.
 */
typedef struct pgsag_view {
  float R[9];                 /* world -> camera rotation, row-major            */
  float t[3];                 /* world -> camera translation                    */
  float fx, fy, cx, cy;       /* pinhole intrinsics (pixels)                    */
  float znear;                /* near plane; Gaussians with z <= znear culled   */
  float reserved0[3];         /* unused (the camera centre is computed from R, t) */
  int32_t width, height;      /* image size (pixels)                            */
  int32_t tile_w, tile_h;     /* tile size: each in {8,16,32}, tile_w*tile_h<=1024 */
  int32_t tiles_x, tiles_y;   /* ceil(width/tile_w), ceil(height/tile_h)        */
  uint32_t g_begin, g_end;    /* Gaussian index range rendered in this view     */
  uint32_t pair_base;         /* first (view, Gaussian) pair index              */
  uint32_t tile_base;         /* offset of this view in per-tile arrays         */
  uint32_t sat_base;          /* offset in the summed-area table of active tiles*/
  uint32_t act_base;          /* global index of this view's first active tile  */
  uint32_t n_active;          /* (prep) active tiles of this view               */
  uint32_t n_mask;            /* (prep) |M|, building-mask pixels               */
  uint32_t chunk_base;        /* (prep) global index of this view's first chunk */
  uint32_t n_chunks;          /* (prep) chunks of this view                     */
  uint64_t pix_base;          /* offset of this view in dense per-pixel arrays  */
} pgsag_view;

/* Optional work scheduling for the render kernels. */
typedef struct pgsag_sched {
  const uint32_t* order;      /* device, active-tile ids in processing order, or NULL */
  uint32_t* counter;          /* device uint32 work counter for a persistent launch, or NULL */
  int32_t ctas_per_sm;        /* persistent launch: CTAs per SM (used when counter != NULL);
                                 <= 0: as many as the kernel's occupancy allows          */
  int32_t reserved;
} pgsag_sched;

/* Human-readable name of a host status code. */
const char* pgsag_status_str(int status);

/* Library / build information string (architecture, version). */
const char* pgsag_build_info(void);

/* --------------------------------------------------------------------------
 * Mask preparation (once per view; not part of the timed step).
 * Sec. 4.1 (refined building masks RBM), Sec. 4.2 (mask boundaries MB).
 * ------------------------------------------------------------------------ */

/*
 * pgsag_prep_flags: per-pixel sets and per-tile counts of one view.
 *   view   host, one view (size, tiling, pix_base, tile_base are used)
 *   mask   device uint8 [height*width], nonzero = building pixel (M)
 *   flags  device uint8 [dense per-pixel array], written at pix_base:
 *          PGSAG_PIX_MASK (M), PGSAG_PIX_EDGE (E = 3x3 dilation minus 3x3
 *          erosion of M), PGSAG_PIX_RENDER (R = 3x3 dilation of M); neighbours
 *          outside the image are ignored.
 *   tile_npix  device uint32 [per-tile array], written at tile_base: number of R
 *          pixels in each tile.
 *   totals device uint32 [4], overwritten: {active tiles, |R|, chunks, |M|} of
 *          this view (chunks = sum over tiles of ceil(npix / 32)).
 * Errors: PGSAG_ERR_ARG on null pointers or a bad tiling.
 */
int pgsag_prep_flags(const pgsag_view* view, const uint8_t* mask, uint8_t* flags,
                     uint32_t* tile_npix, uint32_t* totals, void* stream);

/*
 * pgsag_prep_lists: active-tile numbering, compacted pixel lists and chunk list
 * of one view, given its tile counts.
 *   view        host; act_base, tile_base, sat_base, pix_base set
 *   view_index  index of this view in the step's view array
 *   flags, tile_npix   from pgsag_prep_flags
 *   px_base     global offset of this view's first rendered pixel in px_list
 *   chunk_base  global offset of this view's first chunk in chunks
 *   tile_act    device int32 [per-tile]: global active index of each tile, -1 if
 *               the tile renders no pixel
 *   sat         device uint32 [(tiles_y+1)*(tiles_x+1) at sat_base]: summed-area
 *               table of the active-tile indicator, S[y][x] = #active in [0,y)x[0,x)
 *   act_tiles   device uint4 [active tiles at act_base]: {view_index,
 *               tile_x | tile_y << 16, first px_list entry, pixel count}
 *   px_list     device uint32 [|R| at px_base]: linear pixel index y*width+x of
 *               every R pixel, grouped by active tile; inside a tile in 8x8-block
 *               order (blocks row-major over the tile, pixels row-major in a block)
 *   chunks      device uint4 [chunks at chunk_base] (16-byte aligned): {view_index,
 *               first px_list entry, pixel count (<= 32), global active tile}; a
 *               chunk covers up to 32 consecutive entries of one tile
 *   pidx        device uint32 [dense per-pixel array], written at pix_base for the
 *               whole image: the px_list position q of each R pixel, 0xFFFFFFFF
 *               for pixels outside R
 * Errors: PGSAG_ERR_ARG on null pointers or act_tiles / chunks not 16-byte
 * aligned; PGSAG_ERR_UNSUPPORTED for tiles of more than 1024 pixels.
 */
int pgsag_prep_lists(const pgsag_view* view, uint32_t view_index, const uint8_t* flags,
                     const uint32_t* tile_npix, uint32_t px_base, uint32_t chunk_base,
                     int32_t* tile_act, uint32_t* sat, void* act_tiles, uint32_t* px_list,
                     void* chunks, uint32_t* pidx, void* stream);

/*
 * pgsag_prep_neighbours: static neighbourhood of one view's rendered pixels, for
 * the loss (Eq. 8 needs each mask pixel's 4 neighbours) and its adjoint.
 *   px_list, pidx, flags  from pgsag_prep_lists / pgsag_prep_flags; this view's
 *             px_list entries are [px_base, px_base + n_px)
 *   nbr       device uint4 [1 per compact pixel] (16-byte aligned), written at
 *             px_base: px_list positions of the {up, down, left, right}
 *             neighbours, 0xFFFFFFFF outside the image or outside R
 *   flags_c   device uint8 [1 per compact pixel], written at px_base: the
 *             pixel's flags
 * n_px = 0 does nothing.  Errors: PGSAG_ERR_ARG on null pointers, nbr not
 * 16-byte aligned or an empty image.
 */
int pgsag_prep_neighbours(const pgsag_view* view, const uint32_t* px_list, uint32_t px_base, uint32_t n_px,
                          const uint8_t* flags, const uint32_t* pidx, void* nbr, uint8_t* flags_c, void* stream);

/*
 * pgsag_prep_gc_weight: w_i of Eq. 9 (Sec. 4.3), read as 1 + |Sobel(Y)| of the
 * target luminance Y = 0.299 R + 0.587 G + 0.114 B, replicated borders; also
 * gathers the target colours of the rendered pixels into the compact layout.
 *   view      host, one view (width, height)
 *   target    device float [height*width*3], this view's full image (RGB
 *             interleaved, row-major); only read, may be freed afterwards
 *   px_list   device, from pgsag_prep_lists; this view's entries are
 *             [px_base, px_base + n_px)
 *   target_c  device float [3 per compact pixel], written at 3*px_base
 *   weight    device float [1 per compact pixel], written at px_base
 * n_px = 0 does nothing.  Errors: PGSAG_ERR_ARG on null pointers or an empty image.
 */
int pgsag_prep_gc_weight(const pgsag_view* view, const float* target, const uint32_t* px_list,
                         uint32_t px_base, uint32_t n_px, float* target_c, float* weight, void* stream);

/* --------------------------------------------------------------------------
 * Step calls (the timed hot path).
 * ------------------------------------------------------------------------ */

/*
 * pgsag_preprocess (Sec. 3.1, Eq. 2-3; EWA projection and SH colour of 3DGS by
 * citation).  For every (view, Gaussian) pair:
 *   s = exp(log_scale), q^ = q/|q| (w,x,y,z), o = sigmoid(opacity_logit);
 *   mu_c = R mu + t; the pair is culled if any input is non-finite or the depth
 *   key z (camera z in float32, ((R20 x + R21 y) + R22 z) + t2 without FMA) is
 *   <= znear, or o < 1/255;
 *   Sigma = R(q^) diag(s^2) R(q^)^T; Sigma' = J R Sigma R^T J^T + 0.3 I with J the
 *   pinhole Jacobian at mu_c (x/z, y/z clamped to 1.3 x half-FOV);
 *   conic Q = Sigma'^-1 (stored as its Cholesky factor); mean2d = (fx x/z + cx, fy y/z + cy);
 *   rgb = max(0, SH3(normalize(mu - c)) + 0.5), c = -R^T t the camera centre;
 *   normal n_c = R * (column of R(q^) for the smallest log-scale, ties to the
 *   lowest axis), negated if n_c . mu_c > 0; d = -n_c . mu_c;
 *   tile rectangle = tiles overlapping the axis-aligned box of the alpha >= 1/255
 *   ellipse (half-extents sqrt(2 ln(255 o) Sigma'_xx), ... plus 1 px), and
 *   `touched` = number of ACTIVE tiles the pair is binned to: if the rectangle
 *   spans at most 64 tiles, the active tiles whose pixel centres the ellipse
 *   meets (exact ellipse-rectangle test, widened by its float32 error bound);
 *   otherwise every active tile of the rectangle (summed-area table).
 * Inputs: means [N,3], log_scales [N,3], quats [N,4], opacity_logit [N],
 *   sh [N,16,3]; views (device, n_views <= PGSAG_MAX_VIEWS); tile_act, sat.
 * Outputs per pair p:
 *   rec [p*16 .. p*16+15] float (16-byte aligned):
 *     {mi, ni, l11, l21, l22, o, r, g, b, d, nx, ny, nz, thr, mf, nf}
 *     (2D mean = (mi + mf, ni + nf): integer part + fraction of a compensated
 *     float32 evaluation of fx x/z + cx, fy y/z + cy, so that pixel offsets
 *     keep ~1e-7 px accuracy at any image size;
 *     l11, l21, l22: Cholesky factor of the conic, Q = L L^T with
 *     L = [[l11, 0], [l21, l22]], so -1/2 d^T Q d = -1/2((l11 dx + l21 dy)^2 +
 *     (l22 dy)^2); det Sigma' is evaluated as |V0 x V1|^2 + 0.3(|V0|^2 + |V1|^2)
 *     + 0.09 with Sigma' = V V^T + 0.3 I, free of cancellation for elongated
 *     Gaussians; thr = -ln(255 o): the pair enters a pixel iff the exponent is
 *     >= thr, i.e. alpha >= 1/255)
 *   depth_key [p]: float bits of z, 0xFFFFFFFF for culled pairs
 *   bininfo [p] uint4: {x0 | y0 << 16, x1 | y1 << 16 (inclusive tile rect),
 *     view index, touched}
 *   tile_mask [p] uint64 (8-byte aligned): for a rectangle of at most 64 tiles,
 *     bit (ty - y0) * (x1 - x0 + 1) + (tx - x0) set for each tile the pair is
 *     binned to (popcount = touched); 0 for larger rectangles
 *   rec and tile_mask are written for binned pairs (touched > 0) only; the
 *   other entries keep whatever they held.
 *   grad2d (nullable, 16-byte aligned) float [16 per pair]: when given, the row
 *   of every binned pair is zeroed, so that pgsag_render_bwd may be called with
 *   n_pairs = 0 (only binned rows are accumulated into or read later).
 * n_pairs = sum over views of (g_end - g_begin).
 * This call begins a step: it clears *status (its kernel, which sets no flag,
 * does it; with n_gauss = 0 a memset does), so every later call of the step
 * sees only the flags raised after it.
 */
int pgsag_preprocess(uint32_t n_gauss, const float* means, const float* log_scales,
                     const float* quats, const float* opacity_logit, const float* sh,
                     uint32_t n_views, const pgsag_view* views, const int32_t* tile_act,
                     const uint32_t* sat, float* rec, uint32_t* depth_key, void* bininfo,
                     uint64_t* tile_mask, float* grad2d, int32_t* status, void* stream);

/*
 * pgsag_bin (Sec. 3.1: the projected Gaussians are assigned to the tiles they
 * overlap and ordered by depth).  Duplicates every binned pair once per active
 * tile it is binned to (as pgsag_preprocess decided: the tiles of its tile_mask
 * for rectangles of up to 64 tiles, every active tile of larger rectangles) and
 * orders each tile's list by (depth key, pair index), i.e. by depth and then
 * ascending Gaussian index within a view:
 *   1. emission of (active tile, pair) for the binned pairs, counting per tile;
 *      K (*k_out) is the total;
 *   2. exclusive scan of the tile counts -> ranges, in active-tile order;
 *   3. scatter of the duplicates into their tiles' ranges;
 *   4. per tile, sort of the range by the 64-bit key (depth_key << 32 | pair):
 *      a warp in registers for lists of up to 256, else a block in shared
 *      memory (chunks of 2048 merged in global memory).
 * The result equals a sort of K keys (tile, depth, index) and is bit-exact and
 * deterministic (the sort key is unique).
 *   tile_mask, bininfo, depth_key  from pgsag_preprocess
 *   capacity   maximum K; if K > capacity, PGSAG_DEV_CAPACITY is set in *status,
 *              nothing is emitted, and later step kernels return without work.
 *   ws         device workspace of pgsag_bin_workspace_size(n_pairs,
 *              n_active_total, capacity) bytes
 *   dup_pairs  device uint32 [capacity]: pair index of each duplicate, sorted
 *   ranges     device uint2 [n_active_total]: {begin, end} per active tile
 *   k_out      device uint64 [1]: K
 */
size_t pgsag_bin_workspace_size(uint32_t n_pairs, uint32_t n_active_total, uint64_t capacity);
int pgsag_bin(uint32_t n_pairs, uint32_t n_views, const pgsag_view* views,
              uint32_t n_active_total, const int32_t* tile_act, const uint64_t* tile_mask, const void* bininfo,
              const uint32_t* depth_key, uint64_t capacity, void* ws, size_t ws_bytes,
              uint32_t* dup_pairs, void* ranges, uint64_t* k_out, int32_t* status,
              void* stream);

/*
 * pgsag_render_fwd (Sec. 3.1, Eq. 1-4).  One CTA of 4 warps per active tile
 * (more rounds for tiles of more than 256 rendered pixels), each lane owning 2
 * compacted rendered pixels; the tile's sorted Gaussians are staged through
 * shared memory in batches of 128 and each warp skips the Gaussians whose
 * alpha >= 1/255 ellipse misses the bounding box of its pixels.  Per pixel,
 * front to back:
 *   alpha = min(0.99, o exp(-1/2 d^T Q d)); skipped if alpha < 1/255 (tested as
 *   -1/2 d^T Q d < thr, identically in the forward and the adjoint); if
 *   T (1 - alpha) < 1e-4 the pixel stops before this Gaussian; otherwise
 *   w = alpha T, C += w c, N += w n_c, D += w d, T *= 1 - alpha.
 *   Depth = D / (-N . K^-1 (x+1/2, y+1/2, 1)) if something was blended,
 *   -N.r > 1e-8 and D > 0 (the pixel is then "valid"), else 0.
 * Outputs (compact per-pixel arrays, every px_list entry written):
 *   out8  float [8 per compact pixel]: {C_r, C_g, C_b, D, N_x, N_y, N_z, A = 1 - T}
 *   depth float [1 per compact pixel]
 *   aux   uint4 [1 per compact pixel]: {float bits of final T, index (into dup_pairs) of the
 *         last blended Gaussian, number blended n_contrib, float bits of the soft
 *         count g~ = sum of the blended alphas (PGSAG_RENDER_SOFT_COUNT), else of
 *         the ray-plane dot s = -N . K^-1 (x+1/2, y+1/2, 1) of Eq. 4}
 * sched may be NULL (one CTA per active tile in index order); with a counter the
 * launch is persistent (ctas_per_sm x SMs CTAs pulling tiles, in `order` if
 * given; ctas_per_sm <= 0: as many as the occupancy allows).
 * flags: 0, or PGSAG_RENDER_SOFT_COUNT (needed by the PGSAG_OBJ_EQ11 objective).
 */
#define PGSAG_RENDER_SOFT_COUNT 1u
int pgsag_render_fwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                     const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                     uint32_t n_active_total, const uint32_t* px_list, const pgsag_sched* sched, uint32_t flags,
                     float* out8, float* depth, void* aux, int32_t* status, void* stream);

/*
 * pgsag_loss_ban (Sec. 4.2, Eq. 8; photometric L1 term of Eq. 10).  Per view v:
 *   L_rgb = 1/(3|M|) sum_{i in M} |C_i - C*_i|_1
 *   L_ban = 1/|V| sum_{i in V} w_i || n_depth,i - N_i/|N_i| ||^2,
 *     n_depth = normalize((P[y+1]-P[y-1]) x (P[x+1]-P[x-1])), P = Depth r,
 *     w = 0.1 on E, 1 elsewhere; V = mask pixels off the image border that are
 *     valid, whose 4 neighbours are in R and valid, with a non-zero cross product.
 *   L = L_rgb + lambda_ban L_ban.
 * Writes dL/d(out8) for every R pixel (gradient through both n_depth -- into D
 * and N of the 4 neighbours via Eq. 4 -- and the rendered normal; dL/dA = 0).
 * Two passes: pass A evaluates the terms, the own-pixel gradient and, per mask
 * pixel, dL/da and dL/db of its two central differences (scratch); pass B
 * gathers those from each pixel's neighbours and maps them through Eq. 4.
 *   flags_c, nbr  the compact flags and neighbour table of pgsag_prep_neighbours
 *   chunks, px_list  from pgsag_prep_lists (act_tiles is not read)
 *   aux      pgsag_render_fwd's aux (read only when gc_weight is given)
 *   target   float [3 per compact pixel] (from pgsag_prep_gc_weight)
 *   gc_weight  nullable, float [1 per compact pixel] (pgsag_prep_gc_weight): when
 *            given, pass A also sums the Eq. 9 statistic (see pgsag_tile_stats)
 *            and gc_load [1 per view] receives the GC-load; both or neither
 *   gather   1: run pass B, dout8 is complete.  0: skip it; dout8 then holds
 *            pass A's values and pgsag_render_bwd must be given a
 *            pgsag_ban_gather built from the same scratch and acc
 *   scratch  float [6 per compact pixel] (written for every R pixel: zero off the mask)
 *   acc      double [8 per view]: {sum L1, sum w |n_depth - n|^2, |V|, 0,
 *            |R|, sum g/w, sum (g/w)^2, 0}, overwritten
 *   chunk_scratch  float [8 per chunk] scratch (per-chunk partial sums, reduced
 *            per view without contended atomics)
 *   loss     float [3 per view + 1]: {L_rgb, L_ban, L} per view, then sum_v L
 *   dout8    float [8 per compact pixel]
 *   objective  PGSAG_OBJ_PG: L = L_rgb + lambda_ban L_ban, dout8 = dL/d(out8); the
 *            GC-load (if gc_weight) uses the integer count n_contrib, value only.
 *            PGSAG_OBJ_EQ11 (Sec. 4.3, Eq. 10-11 over the locally defined terms):
 *            L = (1 - lambda) (L_rgb + lambda_3 L_s + lambda_4 L_ban)
 *                + lambda sum_v GC-load_v, lambda = 0.41, lambda_3 = 100,
 *            lambda_4 = lambda_ban; the GC-load uses the soft count g~ (aux.w,
 *            pgsag_render_fwd with PGSAG_RENDER_SOFT_COUNT) and is differentiated;
 *            L_s = mean over the n_gauss Gaussians of min(exp(log_scales)) (the
 *            flattening loss, PGSR by citation).  Requires gc_weight, gc_load
 *            and gather = 0; acc then holds 8 doubles per view + 8 (the L_s
 *            sum); loss per view {L_rgb, L_ban, view total under Eq. 11} and the
 *            last entry the full L.  dout8 stays d(L_rgb + lambda_4 L_ban); the
 *            (1 - lambda) factor, the GC-load gradient (its per-view
 *            coefficients are left in acc, slot 3) and the L_s gradient are
 *            applied by pgsag_render_bwd (pgsag_ban_gather.objective) and
 *            pgsag_preprocess_bwd (flatten_weight).
 *   n_gauss, log_scales  the Gaussians of L_s (objective EQ11; n_gauss may be 0)
 *   dssim    NULL, or the masked D-SSIM term of L_rgb (pgsag_dssim; act_tiles is
 *            then read, 16-byte aligned; acc slot 7 of each view receives the
 *            sum of the SSIM values)
 */
/*
 * Masked D-SSIM term of L_rgb (3DGS's photometric loss by citation, restricted
 * to the building mask): with dssim given, L_rgb = (1 - lambda) L1 +
 * lambda (1 - SSIM_M), SSIM_M = mean over the mask pixels and the 3 channels of
 * SSIM with the 11 x 11 Gaussian window (sigma 1.5) restricted to the rendered
 * set R and renormalised over it, C1 = 0.01^2, C2 = 0.03^2; its gradient is added
 * to dout8's colour.  The window sums are taken per active tile with a 5-pixel
 * halo gathered through the dense pixel map pidx.
 */
typedef struct pgsag_dssim {
  const uint32_t* pidx;     /* device, dense pixel -> compact index (pgsag_prep_lists) */
  float* scratch;           /* device float [9 per compact pixel] (gradient coefficients) */
  uint32_t n_active_total;  /* entries of act_tiles                                     */
  int32_t tile_w, tile_h;   /* the tile size every view uses                            */
  float lambda;             /* D-SSIM weight (3DGS: 0.2)                                */
} pgsag_dssim;              /* 32 bytes */

#define PGSAG_OBJ_PG 0u
#define PGSAG_OBJ_EQ11 1u
#define PGSAG_LAMBDA_GC 0.41f      /* Sec. 4.3, Eq. 11: lambda   */
#define PGSAG_LAMBDA_FLAT 100.0f   /* Sec. 4.3, Eq. 11: lambda_3 */
int pgsag_loss_ban(uint32_t n_views, const pgsag_view* views, uint32_t n_chunks,
                   const void* chunks, const void* act_tiles, const uint32_t* px_list,
                   const uint8_t* flags_c, const void* nbr, const float* out8, const float* depth,
                   const void* aux, const float* target, float lambda_ban, const float* gc_weight,
                   int gather, float* scratch, double* acc, float* chunk_scratch, float* loss,
                   float* gc_load, float* dout8, uint32_t objective, uint32_t n_gauss,
                   const float* log_scales, const pgsag_dssim* dssim, int32_t* status, void* stream);

/*
 * Deferred Eq. 8 adjoint for pgsag_render_bwd.  pgsag_loss_ban with gather = 0
 * leaves out its second pass (the neighbour gather of dL/dP, P = Depth r, and
 * the lambda / |V| scaling of the normal-loss gradient); pgsag_render_bwd given
 * this struct does that gather for each pixel as it loads the pixel's upstream
 * gradient, which saves one pass over the per-pixel arrays.
 */
typedef struct pgsag_ban_gather {
  const uint8_t* flags_c;  /* compact flags (pgsag_prep_neighbours); not read, nullable */
  const void* nbr;         /* device, compact neighbour table (pgsag_prep_neighbours)   */
  const float* scratch;    /* device, loss scratch from pgsag_loss_ban (6 per compact px) */
  const double* acc;       /* device, loss accumulators from pgsag_loss_ban (8 per view) */
  float lambda_ban;        /* the lambda given to pgsag_loss_ban                         */
  uint32_t objective;      /* the objective given to pgsag_loss_ban                      */
  const float* gc_weight;  /* device, Eq. 9 weights (objective PGSAG_OBJ_EQ11)           */
  float lambda_gc;         /* Eq. 11 lambda (objective PGSAG_OBJ_EQ11)                   */
  uint32_t reserved;       /* 0                                                         */
  const float* depth;      /* device, nullable: pgsag_render_fwd's depth output; the
                              adjoint then takes Eq. 4's chain rule from it and the
                              ray-plane dot (aux's fourth word under PGSAG_OBJ_PG, the
                              rendered normal under PGSAG_OBJ_EQ11) instead of
                              reloading all of out8                                    */
} pgsag_ban_gather;       /* 64 bytes */

/*
 * pgsag_render_bwd (Sec. 3.1: the Gaussians' parameters are fitted through the
 * differentiable renderer).
 * Adjoint of pgsag_render_fwd: each CTA re-traverses its tile's list back to
 * front from the last blended Gaussian, recovering T by division
 * (T_i = T_{i+1} / (1 - alpha_i)), and accumulates per pair
 *   grad2d[p*16 + {0..12}] = dL/d{mx, my, l11, l21, l22, o, r, g, b, d, nx, ny, nz}
 * (warp shuffle reduction, shared-memory sum over the CTA's warps, then one
 * float4 atomic add per 4 values per tile).  grad2d (16-byte aligned) is zeroed
 * by this call when n_pairs > 0; with n_pairs = 0 it is not cleared and the
 * rows of the binned pairs must already be zero (pgsag_preprocess given grad2d
 * clears them).  out8, aux, dout8 and ddepth are compact per-pixel arrays
 * (8, 1, 8, 1 entries per px_list position).  ddepth (nullable) adds a
 * gradient on the depth output, folded into dD and dN through Eq. 4.  ban
 * (nullable, host struct) adds the deferred Eq. 8 gather: dout8 is then the
 * output of pgsag_loss_ban with gather = 0.  dout_scale (nullable, device float[1])
 * multiplies the whole upstream gradient (chain rule from a scalar loss).
 * clear (nullable, host struct) names buffers that this call sets to zero on
 * the side: every CTA stores zeros over its share of them (streaming stores
 * that drain while it renders; the call is ALU-bound and leaves most of the
 * memory bandwidth unused).  It is meant for the raw-parameter gradients of
 * the step, so that pgsag_preprocess_bwd with accumulate = 2 writes only the
 * rows of the Gaussians that have a binned pair.  The cleared buffers must not
 * overlap any input or output of this call.
 */
#define PGSAG_CLEAR_MAX 5
typedef struct pgsag_clear {
  float* ptr[PGSAG_CLEAR_MAX];   /* device, 16-byte aligned; NULL where n is 0   */
  uint64_t n[PGSAG_CLEAR_MAX];   /* floats to set to zero from ptr[i]            */
} pgsag_clear;                   /* 80 bytes */
int pgsag_render_bwd(uint32_t n_views, const pgsag_view* views, const float* rec,
                     const uint32_t* dup_pairs, const void* ranges, const void* act_tiles,
                     uint32_t n_active_total, const uint32_t* px_list, const pgsag_sched* sched,
                     const float* out8, const void* aux, const float* dout8, const float* ddepth,
                     const pgsag_ban_gather* ban, const float* dout_scale, uint32_t n_pairs, float* grad2d,
                     const pgsag_clear* clear, int32_t* status, void* stream);

/*
 * pgsag_preprocess_bwd: chain rule from grad2d to the raw parameters (the
 * adjoint of pgsag_preprocess), summed over the views that render each Gaussian
 * (no atomics: one thread per Gaussian loops over its views; each warp lists
 * the Gaussians of its 64 that have a binned pair and runs the per-pair work
 * over that list).  The argmin axis, the normal flip, the Jacobian clamp and
 * the colour clamp are locally constant.  accumulate = 0 overwrites the
 * outputs, 1 adds to them (the outputs of a Gaussian with no binned pair and no
 * flattening term are then left as they are: its gradient is zero), 2 takes
 * outputs that already hold zeros (pgsag_render_bwd's clear): the rows of the
 * Gaussians with a binned pair are overwritten, the others are written only
 * where the flattening term is on.
 * flatten_weight != 0 adds the gradient of flatten_weight * L_s, L_s = mean over
 * the n_gauss Gaussians of min(exp(log_scales)) (Eq. 11's flattening term; its
 * weight there is (1 - lambda) lambda_3), scaled by *dout_scale if dout_scale is
 * given, to d_log_scales at each Gaussian's smallest axis (ties: lowest axis).
 * Outputs: d_means [N,3], d_log_scales [N,3], d_quats [N,4], d_opacity_logit [N],
 * d_sh [N,16,3].
 */
int pgsag_preprocess_bwd(uint32_t n_gauss, const float* means, const float* log_scales,
                         const float* quats, const float* opacity_logit, const float* sh,
                         uint32_t n_views, const pgsag_view* views, const void* bininfo,
                         const float* grad2d, int accumulate, float* d_means,
                         float* d_log_scales, float* d_quats, float* d_opacity_logit,
                         float* d_sh, const float* dout_scale, float flatten_weight,
                         int32_t* status, void* stream);

/*
 * pgsag_tile_stats (Sec. 4.3, Eq. 9).
 *   tile_counts [n_active_total] uint32: Gaussians binned to each active tile
 *     (length of its range);
 *   per view, GC-load = population std over R pixels of g_i / w_i with
 *     g_i = n_contrib (from aux) and w_i from pgsag_prep_gc_weight;
 *   acc   double [3 per view] scratch; chunk_scratch float [4 per chunk] scratch;
 *   gc_load float [1 per view]; NULL computes the tile counts only (acc,
 *     chunk_scratch, aux and gc_weight are then not used).
 */
int pgsag_tile_stats(uint32_t n_views, const pgsag_view* views, uint32_t n_active_total,
                     const void* ranges, uint32_t n_chunks, const void* chunks,
                     const void* act_tiles, const uint32_t* px_list, const void* aux,
                     const float* gc_weight, uint32_t* tile_counts, double* acc,
                     float* chunk_scratch, float* gc_load, int32_t* status, void* stream);

/*
 * pgsag_schedule_lpt (batched sub-regions, Sec. 4.1 / Sec. 5.1): order of the
 * active tiles for a persistent render launch, longest first.  cost_t =
 * rendered pixels x (list length + 1); tiles are emitted in descending
 * floor(log2(cost_t)) (counting sort; order inside a bucket unspecified).
 *   ws     device uint32 [33] scratch
 *   order  device uint32 [n_active_total]: a permutation of the active tiles;
 *          pass it as pgsag_sched.order together with a counter.
 * Run it after pgsag_bin (it reads the ranges).
 */
int pgsag_schedule_lpt(uint32_t n_active_total, const void* ranges, const void* act_tiles,
                       uint32_t* ws, uint32_t* order, int32_t* status, void* stream);

/*
 * pgsag_tile_stats_noalloc: pgsag_tile_stats without caller-provided scratch.
 * The paper has no counterpart; this is an interface for callers that cannot
 * allocate device memory (an application or plug-in that must take every
 * device buffer from its own memory manager, or a latency-critical loop where a
 * cudaMalloc, which can synchronise the device, is not acceptable).  The caller
 * still passes all inputs and outputs (same meaning as pgsag_tile_stats); the
 * scratch lives in a fixed device array inside the library (about 16 MiB, held
 * on every GPU that loads the library until the process exits).
 *   - At most PGSAG_NOALLOC_MAX_CHUNKS chunks (2^20, i.e. about 33.5M rendered
 *     pixels); larger inputs return PGSAG_ERR_CAPACITY and enqueue nothing.
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress (that device must be current); make this first call
 *     before any stream capture.  The address is kept for the process: after a
 *     cudaDeviceReset (or anything else that destroys and re-creates the
 *     device's primary context) it is stale, and this entry point must not be
 *     called again on that device.
 *   - Every view's chunk range [chunk_base, chunk_base + n_chunks) in the
 *     device view table must lie inside [0, n_chunks); a view table that does
 *     not agree sets PGSAG_DEV_BOUNDS in *status and the view is skipped.
 *   - Calls share the array: calls that overlap on the GPU (other streams or
 *     host threads on the same device) race and give wrong results.
 *   - Allocates nothing (no cudaMalloc / cudaFree, no allocating library call).
 */
#define PGSAG_NOALLOC_MAX_CHUNKS (1u << 20)
int pgsag_tile_stats_noalloc(uint32_t n_views, const pgsag_view* views, uint32_t n_active_total,
                             const void* ranges, uint32_t n_chunks, const void* chunks,
                             const void* act_tiles, const uint32_t* px_list, const void* aux,
                             const float* gc_weight, uint32_t* tile_counts, float* gc_load,
                             int32_t* status, void* stream);

/*
 * pgsag_adam: fused Adam update of n parameters (p, g, m, v float32):
 *   m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *   p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * The paper does not name its optimiser; this is the 3DGS convention.
 */
int pgsag_adam(uint64_t n, float* p, const float* g, float* m, float* v, float lr, float beta1,
               float beta2, float eps, int32_t step, void* stream);

/*
 * pgsag_adam_multi: the same update for up to PGSAG_ADAM_MAX_TENSORS tensors
 * (each with its own learning rate) in one launch, with the step count in device
 * memory, so a captured CUDA graph of a training iteration can be replayed as is.
 *   tensors: HOST array (copied into the launch); p, g, m, v device float32 [n].
 *   step: device int32 [4]: step[0] is the step count, advanced by one per call
 *         before the update (start it at 0); step[1], step[2] receive the bias
 *         corrections of the new step (float bits); step[3] unused.
 *   status: device status word (nonzero: nothing is updated).
 * Two launches (the step advance, then the update); capturable in a graph.
 * Errors: PGSAG_ERR_UNSUPPORTED for more than PGSAG_ADAM_MAX_TENSORS tensors,
 * PGSAG_ERR_ARG for missing pointers.
 */
typedef struct pgsag_adam_tensor {
  float* p;
  const float* g;
  float* m;
  float* v;
  uint64_t n;
  float lr;
  uint32_t reserved;       /* 0 */
} pgsag_adam_tensor;       /* 48 bytes */
#define PGSAG_ADAM_MAX_TENSORS 8
int pgsag_adam_multi(uint32_t n_tensors, const pgsag_adam_tensor* tensors, float beta1, float beta2, float eps,
                     int32_t* step, int32_t* status, void* stream);

/*
 * ---------------------------------------------------------------------------
 * Reliability-scored multi-view voting filter (Sec. 4.1, Eq. 5-7).  The step
 * before optimisation that refines coarse building masks: every sparse SfM point
 * is projected into every view; a point that lands inside the mask of at least
 * one view is a potential building point (Eq. 5 / 6); its unreliability score US
 * counts the views in which it lands inside the image but outside the mask
 * (Eq. 7); a potential point with US < tau is a reliable building point.
 *
 * Projection (pinhole, the camera model of the renderer): x_c = R x_w + t; the
 * point is in front iff z_c > znear; it lands on pixel (floor(u), floor(v)) with
 * u = fx (x_c (1 / z_c)) + cx, v = fy (y_c (1 / z_c)) + cy, and is inside the
 * image iff 0 <= u < width and 0 <= v < height.  Whether a point is in front, in
 * the image and in the mask is decided in float32 by this fixed sequence of
 * correctly rounded operations (no fused multiply-add; sums left to right:
 * x_c = ((R00 x + R01 y) + R02 z) + t0, ...), so the decision is reproducible
 * off the GPU.  The paper states no occlusion test: a point "appears" in every
 * view it projects into.
 * ---------------------------------------------------------------------------
 */
typedef struct pgsag_vote_view {
  float R[9];              /* world -> camera rotation, row-major: x_c = R x_w + t */
  float t[3];
  float fx, fy, cx, cy;    /* pixel (u, v) covers [u, u+1) x [v, v+1)               */
  float znear;             /* in front iff z_c > znear                              */
  int32_t width, height;   /* > 0                                                   */
  uint32_t words_per_row;  /* packed mask row stride in 32-bit words, >= ceil(width/32) */
  uint32_t reserved[2];    /* zero                                                  */
  uint64_t mask_offset;    /* first 32-bit word of this view's packed mask           */
} pgsag_vote_view;         /* 96 bytes */

#define PGSAG_VOTE_MAX_VIEWS 256  /* views per pgsag_vote_filter call */

/*
 * pgsag_vote_pack_mask: bit-pack one view's mask.  mask: uint8 [height, width]
 * (nonzero = building); bits: uint32 [height, words_per_row] (device), bit
 * (x & 31) of word y * words_per_row + (x >> 5) set iff mask[y * width + x] != 0;
 * bits past the row's end are zero.  words_per_row >= ceil(width / 32).  Masks
 * are fixed over training, so packing is preparation, done once per view.
 */
int pgsag_vote_pack_mask(int32_t width, int32_t height, const uint8_t* mask, uint32_t words_per_row,
                         uint32_t* bits, void* stream);

/*
 * pgsag_vote_filter: Eq. 5-7 for n_points points against n_views views.
 *   points:    float32 [n_points, 3] world coordinates (device, 4-byte aligned).
 *   views:     HOST array of n_views <= PGSAG_VOTE_MAX_VIEWS cameras (copied into
 *              the launch; the call validates them: width, height > 0,
 *              words_per_row >= ceil(width / 32)).
 *   mask_bits: packed masks (pgsag_vote_pack_mask), view v's at mask_offset.
 *   in_mask:   uint32 [n_points]: number of views whose mask holds the point's
 *              pixel (Eq. 5 / 6: potential iff > 0).
 *   us:        uint32 [n_points]: number of views where the point is inside the
 *              image but outside the mask (Eq. 7).
 *   reliable:  uint8 [n_points]: 1 iff in_mask > 0 and us < tau, else 0.
 *   accumulate: 0 = overwrite the counts; 1 = add to them (views in several
 *              calls of at most PGSAG_VOTE_MAX_VIEWS); reliable is recomputed
 *              from the summed counts on every call.
 * n_points == 0 enqueues nothing; n_views == 0 with accumulate == 0 writes zero
 * counts.  Bad pointers / views: PGSAG_ERR_ARG; n_views too large:
 * PGSAG_ERR_UNSUPPORTED.
 */
int pgsag_vote_filter(uint32_t n_points, const float* points, uint32_t n_views, const pgsag_vote_view* views,
                      const uint32_t* mask_bits, uint32_t tau, int accumulate, uint32_t* in_mask,
                      uint32_t* us, uint8_t* reliable, int32_t* status, void* stream);

/*
 * pgsag_vote_compact: indices of the reliable points in ascending order.
 *   reliable: uint8 [n_points] (nonzero = keep); idx: uint32 [n_points] (the
 *   first n_out entries are written); n_out: uint32 [1] (device).
 *   workspace: pgsag_vote_compact_workspace_size(n_points) bytes (device, 4-byte
 *   aligned), caller-owned.
 */
size_t pgsag_vote_compact_workspace_size(uint32_t n_points);
int pgsag_vote_compact(uint32_t n_points, const uint8_t* reliable, uint32_t* idx, uint32_t* n_out,
                       void* workspace, size_t workspace_bytes, int32_t* status, void* stream);

/*
 * ---------------------------------------------------------------------------
 * Depth-map fusion and TSDF integration (Sec. 4.4, "Mesh Extraction and Merge"):
 * the building and background depth maps of every view are fused by their mean
 * where they overlap, then integrated into a truncated signed distance function
 * on a regular voxel grid (the TSDF method, by citation), from which a mesher
 * extracts the surface (mesh extraction is not part of the library).
 *
 * Voxel (i, j, k) (x fastest, linear index i + nx (j + ny k)) has its centre at
 * origin + ((i, j, k) + 1/2) voxel.  Per view the centre is projected like a
 * voting-filter point (x_c = R c + t, in front iff z_c > znear, pixel
 * (floor u, floor v) inside the image); where that pixel holds a depth d (> 0,
 * finite), sdf = d - z_c; the view is integrated iff sdf >= -trunc, with value
 * min(1, sdf / trunc) and weight 1.  The TSDF is the weighted mean of the
 * integrated values; voxels with weight 0 hold 1.  The decisions (in front, inside,
 * which pixel, valid depth, sdf >= -trunc) are taken in float32 with one correctly
 * rounded operation per step in the order c = origin + ((i + 1/2) voxel),
 * x_c = ((R00 c_x + R01 c_y) + R02 c_z) + t0, iz = 1 / z_c, u = fx (x_c iz) + cx,
 * sdf = d - z_c, so they are reproducible off the GPU.
 * ---------------------------------------------------------------------------
 */
typedef struct pgsag_depth_view {
  float R[9];              /* world -> camera rotation, row-major: x_c = R x_w + t */
  float t[3];
  float fx, fy, cx, cy;
  float znear;
  int32_t width, height;   /* > 0                                                   */
  uint32_t reserved[3];    /* zero                                                  */
  uint64_t depth_offset;   /* first float of this view's depth map [height, width]  */
} pgsag_depth_view;        /* 96 bytes */

typedef struct pgsag_tsdf_grid {
  float origin[3];         /* world position of the grid's low corner               */
  float voxel;             /* voxel edge length (> 0)                               */
  uint32_t nx, ny, nz;     /* voxels per axis (nx * ny * nz < 2^32)                 */
  float trunc;             /* truncation distance (> 0)                             */
} pgsag_tsdf_grid;         /* 32 bytes */

#define PGSAG_TSDF_MAX_VIEWS 256  /* views per pgsag_tsdf_integrate call */

/*
 * pgsag_depth_fuse: out[p] = mean of maps[m * n_pix + p] over the maps whose
 * value there is > 0 and finite; 0 where none is.  maps: float32 [n_maps, n_pix]
 * (device), 1 <= n_maps <= 8; out: float32 [n_pix] (may not alias maps).
 */
int pgsag_depth_fuse(uint32_t n_maps, const float* maps, uint64_t n_pix, float* out, void* stream);

/*
 * pgsag_tsdf_integrate: integrate n_views <= PGSAG_TSDF_MAX_VIEWS depth maps
 * into the grid.
 *   grid, views: HOST structs (copied into the launch; validated: voxel, trunc,
 *     width, height > 0, grid size < 2^32).
 *   depth: float32 depth maps (device), view v's at views[v].depth_offset.
 *   tsdf, weight: float32 [nz, ny, nx] (device).  accumulate = 0: overwritten
 *     (weight = number of integrated views, tsdf = their mean value, 1 where the
 *     weight is 0); 1: the new views are merged into the running weighted mean
 *     (w' = w + n, t' = (t w + sum) / w'; voxels no new view reaches unchanged).
 * The views are integrated in chunks whose depth maps fit in L2 together (one
 * launch per chunk, later chunks merged into the running mean).
 * Errors: PGSAG_ERR_UNSUPPORTED for too many views or a grid of 2^32 voxels or
 * more; PGSAG_ERR_ARG for missing pointers or a bad grid / view.
 */
int pgsag_tsdf_integrate(const pgsag_tsdf_grid* grid, uint32_t n_views, const pgsag_depth_view* views,
                         const float* depth, int accumulate, float* tsdf, float* weight, int32_t* status,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PGSAG_H */
