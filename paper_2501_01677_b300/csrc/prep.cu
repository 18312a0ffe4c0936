// Mask preparation (once per view, outside the timed step): the building mask M
// (Sec. 4.1, refined masks), its boundary E (Sec. 4.2, "masked boundaries"),
// the rendered set R = 3x3 dilation of M (every mask pixel's 4 neighbours are
// rendered, which the depth-derived normal of Eq. 8 needs), active tiles, a
// summed-area table of the active-tile indicator and mask-compacted pixel lists.
#include "common.cuh"

namespace pgsag {

__global__ void k_prep_flags(int W, int H, int tw, int th, int tiles_x, const uint8_t* __restrict__ mask,
                             uint8_t* __restrict__ flags, uint32_t* __restrict__ tile_npix,
                             uint32_t* __restrict__ totals) {
  // one block per tile
  __shared__ uint32_t s_r, s_m;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  if (threadIdx.x == 0) {
    s_r = 0;
    s_m = 0;
  }
  __syncthreads();
  uint32_t nr = 0, nm = 0;
  for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
    const int x = tx * tw + i % tw, y = ty * th + i / tw;
    if (x >= W || y >= H) continue;
    bool any = false, all = true;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx, yy = y + dy;
        if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
        const bool m = mask[(size_t)yy * W + xx] != 0;
        any |= m;
        all &= m;
      }
    const bool m = mask[(size_t)y * W + x] != 0;
    uint8_t f = 0;
    if (m) f |= PGSAG_PIX_MASK;
    if (any && !all) f |= PGSAG_PIX_EDGE;
    if (any) f |= PGSAG_PIX_RENDER;
    flags[(size_t)y * W + x] = f;
    nr += any;
    nm += m;
  }
  atomicAdd(&s_r, nr);
  atomicAdd(&s_m, nm);
  __syncthreads();
  if (threadIdx.x == 0) {
    tile_npix[blockIdx.x] = s_r;
    if (s_r) {
      atomicAdd(totals + 0, 1u);
      atomicAdd(totals + 1, s_r);
      atomicAdd(totals + 2, (s_r + PGSAG_CHUNK - 1) / PGSAG_CHUNK);
    }
    if (s_m) atomicAdd(totals + 3, s_m);
  }
}

// Single block: scans over the view's tiles (active indicator, pixel counts, chunk
// counts), active-tile records and chunk records {view, first px_list entry,
// pixel count, active tile}.
__global__ void __launch_bounds__(1024) k_prep_tiles(uint32_t n_tiles, int tiles_x, uint32_t view_index,
                                                     const uint32_t* __restrict__ npix, uint32_t act_base,
                                                     uint32_t px_base, uint32_t chunk_base,
                                                     int32_t* __restrict__ tile_act, uint4* __restrict__ act_tiles,
                                                     uint4* __restrict__ chunks) {
  __shared__ uint32_t wa[32], wp[32], wc[32];
  __shared__ uint32_t carry[3];
  if (threadIdx.x == 0) carry[0] = carry[1] = carry[2] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t base = 0; base < n_tiles; base += 1024) {
    const uint32_t t = base + threadIdx.x;
    const uint32_t n = t < n_tiles ? npix[t] : 0u;
    const uint32_t a = n > 0, c = (n + PGSAG_CHUNK - 1) / PGSAG_CHUNK;
    uint32_t ia = a, ip = n, ic = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t ya = __shfl_up_sync(kFull, ia, o), yp = __shfl_up_sync(kFull, ip, o),
                     yc = __shfl_up_sync(kFull, ic, o);
      if (lane >= o) {
        ia += ya;
        ip += yp;
        ic += yc;
      }
    }
    if (lane == 31) {
      wa[warp] = ia;
      wp[warp] = ip;
      wc[warp] = ic;
    }
    __syncthreads();
    uint32_t pa = 0, pp = 0, pc = 0, ta = 0, tp = 0, tc = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) {
        pa += wa[w];
        pp += wp[w];
        pc += wc[w];
      }
      ta += wa[w];
      tp += wp[w];
      tc += wc[w];
    }
    const uint32_t ea = carry[0] + pa + ia - a, ep = carry[1] + pp + ip - n, ec = carry[2] + pc + ic - c;
    if (t < n_tiles) {
      if (a) {
        const uint32_t g = act_base + ea;
        tile_act[t] = (int32_t)g;
        const uint32_t tx = t % (uint32_t)tiles_x, ty = t / (uint32_t)tiles_x;
        act_tiles[g] = make_uint4(view_index, tx | (ty << 16), px_base + ep, n);
        for (uint32_t j = 0; j < c; ++j)
          chunks[chunk_base + ec + j] =
              make_uint4(view_index, px_base + ep + j * PGSAG_CHUNK, min((uint32_t)PGSAG_CHUNK, n - j * PGSAG_CHUNK), g);
      } else {
        tile_act[t] = -1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry[0] += ta;
      carry[1] += tp;
      carry[2] += tc;
    }
    __syncthreads();
  }
}

// Single block: summed-area table of the active indicator, S[y][x] = #active
// tiles in [0,y) x [0,x), (tiles_y+1) x (tiles_x+1).
__global__ void __launch_bounds__(1024) k_prep_sat(int tiles_x, int tiles_y, const int32_t* __restrict__ tile_act,
                                                   uint32_t* __restrict__ S) {
  const int sw = tiles_x + 1;
  for (int x = threadIdx.x; x < sw; x += blockDim.x) S[x] = 0;
  for (int y = threadIdx.x; y < tiles_y; y += blockDim.x) {
    uint32_t run = 0;
    S[(size_t)(y + 1) * sw] = 0;
    for (int x = 0; x < tiles_x; ++x) {
      run += tile_act[(size_t)y * tiles_x + x] >= 0;
      S[(size_t)(y + 1) * sw + x + 1] = run;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < sw; x += blockDim.x) {
    uint32_t run = 0;
    for (int y = 1; y <= tiles_y; ++y) {
      run += S[(size_t)y * sw + x];
      S[(size_t)y * sw + x] = run;
    }
  }
}

// One block per tile: the tile's rendered pixels in 8x8-block order (blocks
// row-major over the tile, pixels row-major inside a block), so that a render
// warp's 64 consecutive entries cover a square patch, which fewer Gaussians
// overlap than a 16x4 strip; the dense map pidx gets each rendered pixel's
// position in px_list.
__global__ void __launch_bounds__(256) k_prep_px(int W, int H, int tw, int th, int tiles_x,
                                                 const uint8_t* __restrict__ flags,
                                                 const int32_t* __restrict__ tile_act,
                                                 const uint4* __restrict__ act_tiles,
                                                 uint32_t* __restrict__ px_list, uint32_t* __restrict__ pidx) {
  __shared__ uint32_t ws[8];
  __shared__ uint32_t s_carry;
  const int32_t a = tile_act[blockIdx.x];
  if (a < 0) return;
  const uint32_t first = act_tiles[a].z;
  const int tx = blockIdx.x % tiles_x, ty = blockIdx.x / tiles_x;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int bw = tw / 8;  // 8x8 blocks per tile row (tile sides are multiples of 8)
  for (int base = 0; base < tw * th; base += 256) {
    const int i = base + threadIdx.x;
    const int blk = i / 64, j = i % 64;
    const int x = tx * tw + (blk % bw) * 8 + j % 8, y = ty * th + (blk / bw) * 8 + j / 8;
    const bool r = i < tw * th && x < W && y < H && (flags[(size_t)y * W + x] & PGSAG_PIX_RENDER);
    const uint32_t b = __ballot_sync(kFull, r);
    if (lane == 0) ws[warp] = __popc(b);
    __syncthreads();
    uint32_t pre = 0, tot = 0;
    for (int w = 0; w < 8; ++w) {
      if (w < warp) pre += ws[w];
      tot += ws[w];
    }
    const uint32_t rank = s_carry + pre + __popc(b & ((1u << lane) - 1u));
    if (r) {
      px_list[first + rank] = (uint32_t)y * (uint32_t)W + (uint32_t)x;
      pidx[(size_t)y * W + x] = first + rank;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
}

// Per rendered pixel of one view (compact index px_base + i): the compact
// indices of its up, down, left and right neighbours (0xFFFFFFFF outside the
// image or outside R) and its flags, so that the loss and its adjoint find a
// pixel's neighbours with coalesced loads.
__global__ void __launch_bounds__(256) k_prep_nbr(int W, int H, uint32_t n, const uint32_t* __restrict__ px,
                                                  const uint8_t* __restrict__ flags,
                                                  const uint32_t* __restrict__ pidx, uint4* __restrict__ nbr,
                                                  uint8_t* __restrict__ flags_c) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t pix = __ldg(px + i);
  const int y = (int)(pix / (uint32_t)W), x = (int)(pix - (uint32_t)y * (uint32_t)W);
  const size_t p = (size_t)y * W + x;
  const uint32_t none = 0xffffffffu;
  nbr[i] = make_uint4(y > 0 ? __ldg(pidx + p - W) : none, y + 1 < H ? __ldg(pidx + p + W) : none,
                      x > 0 ? __ldg(pidx + p - 1) : none, x + 1 < W ? __ldg(pidx + p + 1) : none);
  flags_c[i] = __ldg(flags + p);
}

}  // namespace pgsag

using namespace pgsag;

static int check_tiling(const pgsag_view* v) {
  if (v->width <= 0 || v->height <= 0) return PGSAG_ERR_ARG;
  const int tw = v->tile_w, th = v->tile_h;
  if (!((tw == 8 || tw == 16 || tw == 32) && (th == 8 || th == 16 || th == 32))) return PGSAG_ERR_UNSUPPORTED;
  if (tw * th > 1024) return PGSAG_ERR_UNSUPPORTED;
  if (v->tiles_x != (v->width + tw - 1) / tw || v->tiles_y != (v->height + th - 1) / th) return PGSAG_ERR_ARG;
  if (v->tiles_x >= 65536 || v->tiles_y >= 65536) return PGSAG_ERR_UNSUPPORTED;
  return PGSAG_OK;
}

extern "C" int pgsag_prep_flags(const pgsag_view* view, const uint8_t* mask, uint8_t* flags,
                                uint32_t* tile_npix, uint32_t* totals, void* stream) {
  if (!view || !mask || !flags || !tile_npix || !totals) return PGSAG_ERR_ARG;
  int r = check_tiling(view);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  PGSAG_CUDA(cudaMemsetAsync(totals, 0, 4 * sizeof(uint32_t), s));
  const unsigned n_tiles = (unsigned)view->tiles_x * (unsigned)view->tiles_y;
  k_prep_flags<<<n_tiles, 256, 0, s>>>(view->width, view->height, view->tile_w, view->tile_h, view->tiles_x, mask,
                                       flags + view->pix_base, tile_npix + view->tile_base, totals);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_prep_lists(const pgsag_view* view, uint32_t view_index, const uint8_t* flags,
                                const uint32_t* tile_npix, uint32_t px_base, uint32_t chunk_base,
                                int32_t* tile_act, uint32_t* sat, void* act_tiles, uint32_t* px_list,
                                void* chunks, uint32_t* pidx, void* stream) {
  if (!view || !flags || !tile_npix || !tile_act || !sat || !act_tiles || !px_list || !chunks || !pidx)
    return PGSAG_ERR_ARG;
  if (((uintptr_t)act_tiles & 15u) || ((uintptr_t)chunks & 15u)) return PGSAG_ERR_ARG;
  int r = check_tiling(view);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned n_tiles = (unsigned)view->tiles_x * (unsigned)view->tiles_y;
  k_prep_tiles<<<1, 1024, 0, s>>>(n_tiles, view->tiles_x, view_index, tile_npix + view->tile_base, view->act_base,
                                  px_base, chunk_base, tile_act + view->tile_base, (uint4*)act_tiles,
                                  (uint4*)chunks);
  PGSAG_CHECK_LAUNCH();
  k_prep_sat<<<1, 1024, 0, s>>>(view->tiles_x, view->tiles_y, tile_act + view->tile_base, sat + view->sat_base);
  PGSAG_CHECK_LAUNCH();
  PGSAG_CUDA(cudaMemsetAsync(pidx + view->pix_base, 0xff,
                             (size_t)view->width * (size_t)view->height * sizeof(uint32_t), s));
  k_prep_px<<<n_tiles, 256, 0, s>>>(view->width, view->height, view->tile_w, view->tile_h, view->tiles_x,
                                    flags + view->pix_base, tile_act + view->tile_base, (const uint4*)act_tiles,
                                    px_list, pidx + view->pix_base);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

extern "C" int pgsag_prep_neighbours(const pgsag_view* view, const uint32_t* px_list, uint32_t px_base, uint32_t n_px,
                                     const uint8_t* flags, const uint32_t* pidx, void* nbr, uint8_t* flags_c,
                                     void* stream) {
  if (!view || !px_list || !flags || !pidx || !nbr || !flags_c) return PGSAG_ERR_ARG;
  if ((uintptr_t)nbr & 15u) return PGSAG_ERR_ARG;
  if (view->width <= 0 || view->height <= 0) return PGSAG_ERR_ARG;
  if (n_px == 0) return PGSAG_OK;
  k_prep_nbr<<<pgsag_div_up(n_px, 256), 256, 0, (cudaStream_t)stream>>>(
      view->width, view->height, n_px, px_list + px_base, flags + view->pix_base, pidx + view->pix_base,
      (uint4*)nbr + px_base, flags_c + px_base);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
