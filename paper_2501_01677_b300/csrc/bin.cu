// Tile binning and ordering (Sec. 3.1: the projected Gaussians are assigned to
// the image tiles they overlap and ordered by depth).  Every binned
// (view, Gaussian) pair is duplicated once per active tile its alpha >= 1/255
// region meets (as pgsag_preprocess decided: its tile mask for rectangles of
// up to 64 tiles, every active tile of larger ones), and each tile's list
// is ordered by (depth key, pair index):
//   1. emission: each block gathers the binned pairs of its slice of the pair
//      array in shared memory (so every lane has work), reserves output room
//      with one atomic per block and writes (active tile, pair) per duplicate,
//      counting the duplicates of every tile; K = the total;
//   2. exclusive scan of the tile counts: the per-tile ranges, in tile order;
//   3. scatter of the duplicates into their tile's range (the position inside
//      a range comes from an atomic cursor, so it is in no particular order);
//   4. per tile, sort of its range by the 64-bit key (depth key << 32 | pair):
//      one warp per tile in registers for lists of up to kWarpSegMax entries,
//      one block per longer list (shared memory, chunks of kSegMax merged in
//      global memory).
// (depth key, pair) is unique, so step 4 fixes one total order whatever the
// atomics did: the result equals a sort of the K keys (tile, depth, pair).
// No kernel waits on another block.
#include "common.cuh"

namespace pgsag {

#ifndef PGSAG_SCAN_BLOCKS
#define PGSAG_SCAN_BLOCKS 592  // 4 blocks per SM on 148 SMs
#endif
constexpr int kScanBlocks = PGSAG_SCAN_BLOCKS;
// the emission and the scatter wait on dependent loads and atomics: 20 blocks
// per SM in flight (grid-stride beyond that; blocks without work exit at once)
constexpr int kWideBlocks = 148 * 20;
static_assert(kScanBlocks >= 1 && kScanBlocks <= 1024, "k_tile_ranges sums the block sums before its own");
constexpr int kScanThreads = 256;
constexpr int kEmitChunk = 1024;   // pairs gathered per block round in the emission
constexpr int kSortThreads = 256;
constexpr int kSegMax = 2048;      // keys sorted in shared memory at once by a block (16 KB)
constexpr int kWarpSegMax = 256;   // longest list a warp sorts on its own (8 keys per lane in registers)
constexpr int kWarpSortWarps = 8;  // warps per block of the per-warp sort
#ifndef PGSAG_SORT_MINB
#define PGSAG_SORT_MINB 6  // resident per-warp sort blocks per SM the register budget must allow
#endif

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void block_range(uint64_t n, uint32_t b, uint32_t nb, uint32_t& lo, uint32_t& hi) {
  const uint64_t per = (n + nb - 1) / nb;
  const uint64_t l = umin64(n, (uint64_t)b * per);
  lo = (uint32_t)l;
  hi = (uint32_t)umin64(n, l + per);
}

// Exclusive scan over the block (kScanThreads threads); `total` = block sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t& total, uint32_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  uint32_t pre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    const uint32_t t = sh[w];
    if (w < warp) pre += t;
    tot += t;
  }
  __syncthreads();
  total = tot;
  return pre + inc - x;
}

// Per-block sums of counts[i * stride] over block_range(n).
__global__ void __launch_bounds__(kScanThreads) k_block_sums(uint32_t n, const uint32_t* __restrict__ counts,
                                                             int stride, uint64_t* __restrict__ partial,
                                                             const int32_t* status) {
  __shared__ unsigned long long ws[kScanThreads / 32];
  if (status_bad(status)) return;
  uint32_t lo, hi;
  block_range(n, blockIdx.x, gridDim.x, lo, hi);
  unsigned long long s = 0;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += kScanThreads) s += __ldg(counts + (size_t)i * stride);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// The binning's counters: per-tile counts, the long-list count and K (one
// launch instead of three memsets).
__global__ void k_bin_clear(uint32_t n_active, uint32_t* __restrict__ tile_cnt, unsigned long long* __restrict__ n_long,
                            unsigned long long* __restrict__ k_total) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_active) tile_cnt[i] = 0u;
  if (i == 0) {
    *n_long = 0ull;
    *k_total = 0ull;
  }
}

// Step 1: emission.  Blocks stride over kEmitChunk-pair slices; the binned
// pairs of a slice are gathered in shared memory, each round of up to
// kScanThreads of them reserves its output with one atomic on *k_total, and
// every duplicate is written as (active tile, pair) and counted per tile.
// Duplicates beyond `capacity` are not written (the capacity flag is set).
__global__ void __launch_bounds__(kScanThreads) k_emit(uint32_t n, const uint4* __restrict__ bininfo,
                                                       const pgsag_view* __restrict__ views,
                                                       const int32_t* __restrict__ tile_act,
                                                       const unsigned long long* __restrict__ tmask,
                                                       uint32_t n_active, uint64_t capacity,
                                                       unsigned long long* __restrict__ k_total,
                                                       uint32_t* __restrict__ tile_keys,
                                                       uint32_t* __restrict__ pair_vals,
                                                       uint32_t* __restrict__ tile_cnt, int32_t* status) {
  __shared__ uint32_t s_list[kEmitChunk];
  __shared__ uint32_t s_n;
  __shared__ uint32_t sh[kScanThreads / 32];
  __shared__ unsigned long long s_base;
  if (status_bad(status)) return;
  for (uint32_t c0 = blockIdx.x * kEmitChunk; c0 < n; c0 += gridDim.x * kEmitChunk) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kEmitChunk; i += kScanThreads) {
      const uint32_t p = c0 + i;
      if (p < n && __ldg(&bininfo[p].w) != 0u) s_list[atomicAdd(&s_n, 1u)] = p;
    }
    __syncthreads();
    const uint32_t m = s_n;
    for (uint32_t r = 0; r < m; r += kScanThreads) {
      const uint32_t j = r + threadIdx.x;
      const uint32_t p = j < m ? s_list[j] : 0u;
      const uint4 bi = j < m ? __ldg(&bininfo[p]) : make_uint4(0, 0, 0, 0);
      // the tile mask and the view's tiling are requested before the block scan
      const unsigned long long mk0 = j < m ? __ldg(tmask + p) : 0ull;
      const pgsag_view* V = views + bi.z;
      const int tiles_x = j < m ? __ldg(&V->tiles_x) : 0;
      const uint32_t tbase = j < m ? __ldg(&V->tile_base) : 0u;
      uint32_t total;
      const uint32_t off = block_excl_scan(bi.w, total, sh);
      if (threadIdx.x == 0) s_base = atomicAdd(k_total, (unsigned long long)total);
      __syncthreads();
      const unsigned long long base = s_base;
      __syncthreads();
      if (threadIdx.x == 0 && base + total > capacity) status_set(status, PGSAG_DEV_CAPACITY);
      if (bi.w) {
        const int32_t* ta = tile_act + tbase;
        const uint32_t x0 = bi.x & 0xffffu, y0 = bi.x >> 16, x1 = bi.y & 0xffffu, y1 = bi.y >> 16;
        const uint32_t rw = x1 - x0 + 1;
        const bool exact = rw * (y1 - y0 + 1) <= (uint32_t)kExactTileMax;
        unsigned long long o = base + off;
        const unsigned long long oend = o + bi.w;
        auto put = [&](int32_t a) {
          if ((uint32_t)a >= n_active) {
            status_set(status, PGSAG_DEV_BOUNDS);
          } else if (o < oend && o < capacity) {
            tile_keys[o] = (uint32_t)a;
            pair_vals[o] = p;
            atomicAdd(tile_cnt + a, 1u);
          }
          ++o;
        };
        if (exact) {
          // the tiles the projection's exact test accepted, one bit each
          for (unsigned long long mk = mk0; mk; mk &= mk - 1) {
            const uint32_t b = (uint32_t)__ffsll((long long)mk) - 1u;
            const uint32_t ty = y0 + b / rw, tx = x0 + b % rw;
            put(__ldg(ta + (size_t)ty * tiles_x + tx));
          }
        } else {
          // large rectangles: every active tile of the rectangle
          for (uint32_t ty = y0; ty <= y1; ++ty) {
            const int32_t* row = ta + (size_t)ty * tiles_x;
            for (uint32_t tx = x0; tx <= x1; ++tx) {
              const int32_t a = __ldg(row + tx);
              if (a >= 0) put(a);
            }
          }
        }
        // the count and this enumeration describe the same tiles; a mismatch is a bug
        if (o != oend) status_set(status, PGSAG_DEV_BOUNDS);
      }
    }
    __syncthreads();
  }
}

// Step 2 (after the block sums of the counts): ranges[a] = {start, start + count}.
__global__ void __launch_bounds__(kScanThreads) k_tile_ranges(uint32_t n_active, const uint32_t* __restrict__ cnt,
                                                              const uint64_t* __restrict__ partial,
                                                              uint2* __restrict__ ranges, const int32_t* status) {
  __shared__ uint32_t sh[kScanThreads / 32];
  __shared__ unsigned long long s_pre[kScanThreads / 32];
  if (status_bad(status)) return;
  uint32_t lo, hi;
  block_range(n_active, blockIdx.x, gridDim.x, lo, hi);
  // this block's offset: the sum of the block sums before it (at most a few
  // hundred L2-resident values; no separate scan launch)
  unsigned long long pre = 0;
  for (uint32_t b = threadIdx.x; b < blockIdx.x; b += kScanThreads) pre += __ldg(partial + b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pre += __shfl_xor_sync(kFull, pre, o);
  if ((threadIdx.x & 31) == 0) s_pre[threadIdx.x >> 5] = pre;
  __syncthreads();
  pre = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) pre += s_pre[w];
  uint32_t carry = (uint32_t)pre;
  for (uint32_t base = lo; base < hi; base += kScanThreads) {
    const uint32_t a = base + threadIdx.x;
    const uint32_t c = a < hi ? __ldg(cnt + a) : 0u;
    uint32_t total;
    const uint32_t off = block_excl_scan(c, total, sh);
    if (a < hi) ranges[a] = make_uint2(carry + off, carry + off + c);
    carry += total;
  }
}

// Step 3: duplicate k goes to ranges[tile].x + (a distinct slot of its tile).
// The cursor counts each tile down from its count to 0.
__global__ void k_scatter(const uint64_t* __restrict__ k_dev, uint64_t cap, uint32_t n_active,
                          const uint32_t* __restrict__ tile_keys, const uint32_t* __restrict__ pair_vals,
                          const uint2* __restrict__ ranges, uint32_t* __restrict__ cursor, uint32_t* __restrict__ out,
                          int32_t* status) {
  if (status_bad(status)) return;
  const uint32_t n = (uint32_t)umin64(*k_dev, cap);
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t a = __ldg(tile_keys + k);
    const uint32_t pv = __ldg(pair_vals + k);  // requested with the key, not after the atomic
    if (a >= n_active) {
      status_set(status, PGSAG_DEV_BOUNDS);
      continue;
    }
    const uint2 r = __ldg(ranges + a);
    const uint32_t left = atomicSub(cursor + a, 1u);
    if (left == 0u || left > r.y - r.x) {
      status_set(status, PGSAG_DEV_BOUNDS);
      continue;
    }
    out[r.x + left - 1u] = pv;
  }
}

__device__ __forceinline__ unsigned long long sort_key(const uint32_t* __restrict__ dkey, uint32_t p) {
  return ((unsigned long long)__ldg(dkey + p) << 32) | p;
}

// Sort n <= kSegMax pair indices by sort_key in shared memory (bitonic network
// over the next power of two, padded with the largest key); `in` and `out` may
// be the same array.
__device__ void sort_chunk(const uint32_t* in, uint32_t n, uint32_t* out, const uint32_t* __restrict__ dkey,
                           unsigned long long* sk) {
  uint32_t m = 2;
  while (m < n) m <<= 1;
  for (uint32_t i = threadIdx.x; i < m; i += kSortThreads) sk[i] = i < n ? sort_key(dkey, in[i]) : ~0ull;
  __syncthreads();
  for (uint32_t k = 2; k <= m; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < m; i += kSortThreads) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long a = sk[i], b = sk[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            sk[i] = b;
            sk[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += kSortThreads) out[i] = (uint32_t)sk[i];
  __syncthreads();
}

// Merge the sorted runs src[0, na) and src[na, na + nb) into dst[0, na + nb):
// each thread finds where its output slice starts on both runs by a binary
// search along the merge path, then merges the slice sequentially.
__device__ void merge_runs(const uint32_t* src, uint32_t na, uint32_t nb, uint32_t* dst,
                           const uint32_t* __restrict__ dkey) {
  const uint32_t L = na + nb;
  const uint32_t per = (L + kSortThreads - 1) / kSortThreads;
  const uint32_t d0 = min(L, threadIdx.x * per), d1 = min(L, d0 + per);
  if (d0 < d1) {
    const uint32_t* A = src;
    const uint32_t* B = src + na;
    // i = number of A elements among the first d0 outputs: the largest i in
    // [max(0, d0 - nb), min(d0, na)] with A[i - 1] < B[d0 - i]
    uint32_t lo = d0 > nb ? d0 - nb : 0u, hi = min(d0, na);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sort_key(dkey, A[mid]) < sort_key(dkey, B[d0 - mid - 1])) lo = mid + 1;
      else hi = mid;
    }
    uint32_t i = lo, j = d0 - lo;
    for (uint32_t d = d0; d < d1; ++d) {
      bool take_a;
      if (i >= na) take_a = false;
      else if (j >= nb) take_a = true;
      else take_a = sort_key(dkey, A[i]) < sort_key(dkey, B[j]);
      dst[d] = take_a ? A[i++] : B[j++];
    }
  }
  __syncthreads();
}

// Bitonic sort of m = 32 E keys held by one warp in registers: element
// i = e * 32 + lane is x[e].  Compare-exchange partners at distance j >= 32
// sit in the same lane (register e ^ j/32), closer ones in lane ^ j (one
// 64-bit shuffle).
template <int E>
__device__ __forceinline__ void warp_bitonic(unsigned long long (&x)[E], int lane) {
  constexpr int m = 32 * E;
#pragma unroll
  for (int k = 2; k <= m; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int je = j >> 5;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int f = e ^ je;
          if (f > e) {
            const int i = e * 32 + lane;
            const bool up = (i & k) == 0;
            const unsigned long long a = x[e], b = x[f];
            if ((a > b) == up) {
              x[e] = b;
              x[f] = a;
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int i = e * 32 + lane;
          const unsigned long long y = __shfl_xor_sync(kFull, x[e], j);
          const bool up = (i & k) == 0, lower = (lane & j) == 0;
          x[e] = (up == lower) ? (x[e] < y ? x[e] : y) : (x[e] < y ? y : x[e]);
        }
      }
    }
  }
}

template <int E>
__device__ __forceinline__ void warp_sort_list(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ out,
                                               const uint32_t* __restrict__ dkey, int lane) {
  unsigned long long x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = (uint32_t)(e * 32 + lane);
    x[e] = i < n ? sort_key(dkey, __ldg(in + i)) : ~0ull;
  }
  warp_bitonic<E>(x, lane);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const uint32_t i = (uint32_t)(e * 32 + lane);
    if (i < n) out[i] = (uint32_t)x[e];
  }
}

// Step 4a: one warp per active tile sorts lists of up to kWarpSegMax entries
// in registers; longer lists are appended to `long_list` for k_sort_long.
__global__ void __launch_bounds__(kWarpSortWarps * 32, PGSAG_SORT_MINB) k_sort_warp(uint32_t n_active,
                                                                   const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ dkey,
                                                                   const uint32_t* __restrict__ buf,
                                                                   uint32_t* __restrict__ out,
                                                                   uint32_t* __restrict__ long_list,
                                                                   unsigned long long* __restrict__ n_long,
                                                                   const int32_t* status) {
  static_assert(kWarpSegMax == 32 * 8, "the register sort covers up to 8 keys per lane");
  if (status_bad(status)) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t a = blockIdx.x * kWarpSortWarps + warp; a < n_active; a += gridDim.x * kWarpSortWarps) {
    const uint2 r = __ldg(ranges + a);
    const uint32_t n = r.y - r.x;
    if (n <= 1) {
      if (n == 1 && lane == 0) out[r.x] = __ldg(buf + r.x);
      continue;
    }
    const uint32_t* in = buf + r.x;
    uint32_t* o = out + r.x;
    if (n <= 32) warp_sort_list<1>(in, n, o, dkey, lane);
    else if (n <= 64) warp_sort_list<2>(in, n, o, dkey, lane);
    else if (n <= 128) warp_sort_list<4>(in, n, o, dkey, lane);
    else if (n <= (uint32_t)kWarpSegMax) warp_sort_list<8>(in, n, o, dkey, lane);
    else if (lane == 0) long_list[atomicAdd(n_long, 1ull)] = a;
  }
}

// Step 4b: blocks stride over the long lists and sort each tile's range.
// buf holds the scattered lists; the sorted lists end in out.
__global__ void __launch_bounds__(kSortThreads) k_sort_long(const unsigned long long* __restrict__ n_long,
                                                            const uint32_t* __restrict__ long_list,
                                                            const uint2* __restrict__ ranges,
                                                            const uint32_t* __restrict__ dkey, uint32_t* buf,
                                                            uint32_t* out, const int32_t* status) {
  __shared__ unsigned long long sk[kSegMax];
  if (status_bad(status)) return;
  const uint32_t count = (uint32_t)*n_long;
  for (uint32_t e = blockIdx.x; e < count; e += gridDim.x) {
    const uint2 r = __ldg(ranges + __ldg(long_list + e));
    const uint32_t n = r.y - r.x;
    if (n <= (uint32_t)kSegMax) {
      sort_chunk(buf + r.x, n, out + r.x, dkey, sk);
      continue;
    }
    // sorted chunks, then rounds of pairwise merges between buf and out,
    // starting in whichever array makes the last round land in out
    const uint32_t chunks = (n + kSegMax - 1) / kSegMax;
    uint32_t rounds = 0;
    while ((1u << rounds) < chunks) ++rounds;
    uint32_t* src = (rounds & 1) ? buf + r.x : out + r.x;
    uint32_t* dst = (rounds & 1) ? out + r.x : buf + r.x;
    for (uint32_t c = 0; c < chunks; ++c) {
      const uint32_t s = c * kSegMax;
      sort_chunk(buf + r.x + s, min((uint32_t)kSegMax, n - s), src + s, dkey, sk);
    }
    for (uint32_t w = kSegMax; w < n; w <<= 1) {
      for (uint32_t s = 0; s < n; s += 2 * w) {
        const uint32_t na = min(w, n - s), nb = n - s > w ? min(w, n - s - w) : 0u;
        merge_runs(src + s, na, nb, dst + s, dkey);
      }
      uint32_t* t = src;
      src = dst;
      dst = t;
    }
  }
}

}  // namespace pgsag

using namespace pgsag;

namespace {
struct BinWs {
  uint64_t* tile_partial;        // kScanBlocks + 1
  unsigned long long* n_long;    // lists longer than kWarpSegMax
  uint32_t* tile_cnt;            // n_active: duplicates per tile, then the scatter cursor
  uint32_t* long_list;           // n_active: tiles with long lists
  uint32_t* tile_keys;           // capacity: emitted active tile
  uint32_t* pair_vals;           // capacity: emitted pair
  uint32_t* buf;                 // capacity: lists scattered into their tiles
  size_t bytes;
};
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
BinWs carve(void* base, uint32_t n_active, uint64_t cap) {
  BinWs w;
  size_t o = 0;
  char* b = (char*)base;
  auto take = [&](size_t bytes) {
    char* p = b ? b + o : nullptr;
    o += align256(bytes);
    return p;
  };
  const size_t capb = (size_t)(cap ? cap : 1) * 4, actb = (size_t)(n_active ? n_active : 1) * 4;
  w.tile_partial = (uint64_t*)take((size_t)(kScanBlocks + 1) * 8);
  w.n_long = (unsigned long long*)take(8);
  w.tile_cnt = (uint32_t*)take(actb);
  w.long_list = (uint32_t*)take(actb);
  w.tile_keys = (uint32_t*)take(capb);
  w.pair_vals = (uint32_t*)take(capb);
  w.buf = (uint32_t*)take(capb);
  w.bytes = o;
  return w;
}
}  // namespace

extern "C" size_t pgsag_bin_workspace_size(uint32_t n_pairs, uint32_t n_active_total, uint64_t capacity) {
  (void)n_pairs;
  return carve(nullptr, n_active_total, capacity).bytes;
}

extern "C" int pgsag_bin(uint32_t n_pairs, uint32_t n_views, const pgsag_view* views,
                         uint32_t n_active_total, const int32_t* tile_act, const uint64_t* tile_mask,
                         const void* bininfo,
                         const uint32_t* depth_key, uint64_t capacity, void* ws, size_t ws_bytes,
                         uint32_t* dup_pairs, void* ranges, uint64_t* k_out, int32_t* status,
                         void* stream) {
  if (n_views == 0 || n_views > PGSAG_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!views || !k_out || !status || !ws) return PGSAG_ERR_ARG;
  if (capacity > 0xffffffffull) return PGSAG_ERR_UNSUPPORTED;
  if (n_pairs && (!bininfo || !depth_key || !tile_act || !tile_mask)) return PGSAG_ERR_ARG;
  if (((uintptr_t)bininfo & 15u) || ((uintptr_t)tile_mask & 7u)) return PGSAG_ERR_ARG;
  if (n_active_total && !ranges) return PGSAG_ERR_ARG;
  if (capacity && !dup_pairs) return PGSAG_ERR_ARG;
  const BinWs w = carve(ws, n_active_total, capacity);
  if (ws_bytes < w.bytes) return PGSAG_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_pairs == 0 || n_active_total == 0) {
    PGSAG_CUDA(cudaMemsetAsync(k_out, 0, sizeof(uint64_t), s));
    // nothing is emitted: every tile's list is empty
    if (n_active_total) PGSAG_CUDA(cudaMemsetAsync(ranges, 0, (size_t)n_active_total * sizeof(uint2), s));
    return PGSAG_OK;
  }
  // (the ranges of every active tile are written by step 2)
  k_bin_clear<<<pgsag_div_up(n_active_total, 256u), 256, 0, s>>>(n_active_total, w.tile_cnt, w.n_long,
                                                                  (unsigned long long*)k_out);
  PGSAG_CHECK_LAUNCH();

  // 1. emission (K accumulates in *k_out)
  k_emit<<<kWideBlocks, kScanThreads, 0, s>>>(n_pairs, (const uint4*)bininfo, views, tile_act,
                                              (const unsigned long long*)tile_mask, n_active_total, capacity, (unsigned long long*)k_out, w.tile_keys,
                                              w.pair_vals, w.tile_cnt, status);
  PGSAG_CHECK_LAUNCH();
  // 2. per-tile ranges
  k_block_sums<<<kScanBlocks, kScanThreads, 0, s>>>(n_active_total, w.tile_cnt, 1, w.tile_partial, status);
  PGSAG_CHECK_LAUNCH();
  k_tile_ranges<<<kScanBlocks, kScanThreads, 0, s>>>(n_active_total, w.tile_cnt, w.tile_partial, (uint2*)ranges,
                                                     status);
  PGSAG_CHECK_LAUNCH();
  // 3. scatter into the tiles' ranges; 4. per-tile sort into dup_pairs
  k_scatter<<<kWideBlocks, 256, 0, s>>>(k_out, capacity, n_active_total, w.tile_keys, w.pair_vals,
                                        (const uint2*)ranges, w.tile_cnt, w.buf, status);
  PGSAG_CHECK_LAUNCH();
  const uint32_t warp_blocks = (n_active_total + kWarpSortWarps - 1) / kWarpSortWarps;
  k_sort_warp<<<warp_blocks < (1u << 20) ? warp_blocks : (1u << 20), kWarpSortWarps * 32, 0, s>>>(
      n_active_total, (const uint2*)ranges, depth_key, w.buf, dup_pairs, w.long_list, w.n_long, status);
  PGSAG_CHECK_LAUNCH();
  k_sort_long<<<296, kSortThreads, 0, s>>>(w.n_long, w.long_list, (const uint2*)ranges, depth_key, w.buf, dup_pairs,
                                           status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
