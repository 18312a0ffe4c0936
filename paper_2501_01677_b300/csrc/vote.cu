// Reliability-scored multi-view voting filter (Sec. 4.1, Eq. 5-7).
//
// Every sparse point is projected into every view; the counts of views whose
// mask holds the point's pixel (Eq. 5 / 6) and of views where it lands in the
// image but outside the mask (Eq. 7, the unreliability score US) decide whether
// it is a reliable building point (potential and US < tau).
//
// Layout and schedule.  Masks are bit-packed (one bit per pixel, 2.5 MB for a
// 5472x3648 view), so tens of views fit in L2 at once.  Each thread owns
// a few points (loaded once, counts kept in registers) and sweeps the views in
// order; every CTA of the grid walks the same view sequence at about the same
// time, so a view's mask is read from HBM about once and served from L2 to the
// rest.  The camera table is a __grid_constant__ kernel parameter (up to 256
// views, 96 bytes each): every lane reads the same camera, a constant-cache
// broadcast.  The projection is a fixed sequence of correctly rounded float32
// operations (no contraction), so the integer decisions it feeds are
// reproducible off the GPU.
#include "common.cuh"

namespace pgsag {

constexpr int kVoteThreads = 256;
constexpr int kCmpThreads = 256;
constexpr int kCmpPerThread = 16;
constexpr int kCmpPerBlock = kCmpThreads * kCmpPerThread;

template <int kMaxViews>
struct VoteTable {
  pgsag_vote_view v[kMaxViews];
};

// Pack one mask row chunk: each warp turns 32 mask bytes into one word.
__global__ void __launch_bounds__(256) k_vote_pack(int W, const uint8_t* __restrict__ mask, uint32_t wpr,
                                                   uint32_t* __restrict__ bits) {
  const uint32_t y = blockIdx.y;
  const uint32_t x = blockIdx.x * 256u + threadIdx.x;
  const bool b = x < (uint32_t)W && __ldg(mask + (size_t)y * (uint32_t)W + x) != 0;
  const uint32_t word = __ballot_sync(kFull, b);
  const uint32_t wi = x >> 5;
  if ((threadIdx.x & 31) == 0 && wi < wpr) bits[(size_t)y * wpr + wi] = word;
}

// kPPT points per thread; a CTA covers kVoteThreads * kPPT consecutive points per
// group and walks groups blockIdx.x, blockIdx.x + gridDim.x, ... (the host sizes
// the grid to one wave).  Per view, every point's projection is computed first,
// then all its mask words are loaded, then counted, so kPPT loads are in flight
// per thread.  The two counts of a point share one register (16 bits each; at
// most PGSAG_VOTE_MAX_VIEWS views per call).
#ifndef PGSAG_VOTE_MINB
#define PGSAG_VOTE_MINB 1
#endif
template <int kMaxViews, int kPPT>
__global__ void __launch_bounds__(kVoteThreads, PGSAG_VOTE_MINB) k_vote(uint32_t n, const float* __restrict__ pts, uint32_t n_views,
                                                       const __grid_constant__ VoteTable<kMaxViews> T,
                                                       const uint32_t* __restrict__ bits, uint32_t tau,
                                                       int accumulate, uint32_t* __restrict__ in_mask,
                                                       uint32_t* __restrict__ us, uint8_t* __restrict__ reliable,
                                                       const int32_t* status) {
  if (status_bad(status)) return;
  constexpr uint32_t kGroup = (uint32_t)(kVoteThreads * kPPT);
  const uint32_t n_groups = (n + kGroup - 1) / kGroup;
  for (uint32_t grp = blockIdx.x; grp < n_groups; grp += gridDim.x) {
    const uint32_t base = grp * kGroup + threadIdx.x;
    float X[kPPT], Y[kPPT], Z[kPPT];
    uint32_t cnt[kPPT];  // in-mask count | outside-mask count << 16
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
      const uint32_t i = base + (uint32_t)(k * kVoteThreads);
      const bool ok = i < n;
      // slots past n evaluate the origin and are never written
      X[k] = ok ? __ldg(pts + 3ull * i + 0) : 0.f;
      Y[k] = ok ? __ldg(pts + 3ull * i + 1) : 0.f;
      Z[k] = ok ? __ldg(pts + 3ull * i + 2) : 0.f;
      cnt[k] = 0u;
    }
    for (uint32_t v = 0; v < n_views; ++v) {
      const pgsag_vote_view& V = T.v[v];
      const float r0 = V.R[0], r1 = V.R[1], r2 = V.R[2], r3 = V.R[3], r4 = V.R[4], r5 = V.R[5];
      const float r6 = V.R[6], r7 = V.R[7], r8 = V.R[8];
      const float t0 = V.t[0], t1 = V.t[1], t2 = V.t[2];
      const float fx = V.fx, fy = V.fy, cx = V.cx, cy = V.cy, zn = V.znear;
      const float Wf = (float)V.width, Hf = (float)V.height;
      const uint32_t wpr = V.words_per_row;
      const uint32_t* mb = bits + V.mask_offset;
      bool in[kPPT];
      uint32_t word_i[kPPT], sh[kPPT];
#pragma unroll
      for (int k = 0; k < kPPT; ++k) {
        // x_c = R x + t, each row summed left to right
        const float xc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r0, X[k]), __fmul_rn(r1, Y[k])), __fmul_rn(r2, Z[k])), t0);
        const float yc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r3, X[k]), __fmul_rn(r4, Y[k])), __fmul_rn(r5, Z[k])), t1);
        const float zc = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r6, X[k]), __fmul_rn(r7, Y[k])), __fmul_rn(r8, Z[k])), t2);
        const float iz = __frcp_rn(zc);
        const float u = __fadd_rn(__fmul_rn(fx, __fmul_rn(xc, iz)), cx);
        const float w = __fadd_rn(__fmul_rn(fy, __fmul_rn(yc, iz)), cy);
        // in front of the near plane and inside the image (false for NaN)
        in[k] = zc > zn && u >= 0.f && u < Wf && w >= 0.f && w < Hf;
        const uint32_t px = in[k] ? (uint32_t)u : 0u, py = in[k] ? (uint32_t)w : 0u;  // floor: u, w >= 0
        word_i[k] = py * wpr + (px >> 5);
        sh[k] = px & 31u;
      }
      uint32_t word[kPPT];
#pragma unroll
      for (int k = 0; k < kPPT; ++k) word[k] = in[k] ? __ldg(mb + word_i[k]) : 0u;
#pragma unroll
      for (int k = 0; k < kPPT; ++k) {
        const uint32_t hit = (word[k] >> sh[k]) & 1u;
        cnt[k] += in[k] ? (hit ? 1u : 0x10000u) : 0u;
      }
    }
#pragma unroll
    for (int k = 0; k < kPPT; ++k) {
      const uint32_t i = base + (uint32_t)(k * kVoteThreads);
      if (i >= n) continue;
      uint32_t a = cnt[k] & 0xffffu, b = cnt[k] >> 16;
      if (accumulate) {
        a += in_mask[i];
        b += us[i];
      }
      in_mask[i] = a;
      us[i] = b;
      reliable[i] = (a > 0u && b < tau) ? 1 : 0;
    }
  }
}

// Compaction, pass 1: number of kept entries per block of kCmpPerBlock.
__global__ void __launch_bounds__(kCmpThreads) k_cmp_count(uint32_t n, const uint8_t* __restrict__ keep,
                                                           uint32_t* __restrict__ block_cnt) {
  __shared__ uint32_t s_w[kCmpThreads / 32];
  const uint32_t b0 = blockIdx.x * (uint32_t)kCmpPerBlock + threadIdx.x * (uint32_t)kCmpPerThread;
  uint32_t c = 0;
#pragma unroll
  for (int k = 0; k < kCmpPerThread; ++k) {
    const uint32_t i = b0 + (uint32_t)k;
    c += (i < n && __ldg(keep + i) != 0) ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kCmpThreads / 32; ++w) t += s_w[w];
    block_cnt[blockIdx.x] = t;
  }
}

// Pass 2 (one block): exclusive scan of the block counts in place; total -> n_out.
__global__ void __launch_bounds__(1024) k_cmp_scan(uint32_t nb, uint32_t* __restrict__ block_cnt,
                                                   uint32_t* __restrict__ n_out) {
  __shared__ uint32_t s[1024];
  const uint32_t per = (nb + 1023u) / 1024u;
  const uint32_t lo = min(nb, threadIdx.x * per), hi = min(nb, lo + per);
  uint32_t sum = 0;
  for (uint32_t i = lo; i < hi; ++i) sum += block_cnt[i];
  s[threadIdx.x] = sum;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 slice sums
  for (uint32_t o = 1; o < 1024u; o <<= 1) {
    const uint32_t add = threadIdx.x >= o ? s[threadIdx.x - o] : 0u;
    __syncthreads();
    s[threadIdx.x] += add;
    __syncthreads();
  }
  uint32_t run = s[threadIdx.x] - sum;
  for (uint32_t i = lo; i < hi; ++i) {
    const uint32_t c = block_cnt[i];
    block_cnt[i] = run;
    run += c;
  }
  if (threadIdx.x == 1023) *n_out = s[1023];
}

// Pass 3: each thread writes the indices of its kept entries at its offset
// (block offset + exclusive prefix over the block's threads), ascending.
__global__ void __launch_bounds__(kCmpThreads) k_cmp_scatter(uint32_t n, const uint8_t* __restrict__ keep,
                                                             const uint32_t* __restrict__ block_off,
                                                             uint32_t* __restrict__ idx) {
  __shared__ uint32_t s_w[kCmpThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t b0 = blockIdx.x * (uint32_t)kCmpPerBlock + threadIdx.x * (uint32_t)kCmpPerThread;
  uint32_t m = 0;
#pragma unroll
  for (int k = 0; k < kCmpPerThread; ++k) {
    const uint32_t i = b0 + (uint32_t)k;
    if (i < n && __ldg(keep + i) != 0) m |= 1u << k;
  }
  const uint32_t c = __popc(m);
  uint32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += s_w[w];
  uint32_t pos = block_off[blockIdx.x] + wbase + incl - c;
  while (m) {
    const int k = __ffs(m) - 1;
    m &= m - 1;
    idx[pos++] = b0 + (uint32_t)k;
  }
}

}  // namespace pgsag

using namespace pgsag;

extern "C" int pgsag_vote_pack_mask(int32_t width, int32_t height, const uint8_t* mask, uint32_t words_per_row,
                                    uint32_t* bits, void* stream) {
  if (width <= 0 || height <= 0 || !mask || !bits) return PGSAG_ERR_ARG;
  if ((uint64_t)words_per_row * 32ull < (uint64_t)width) return PGSAG_ERR_ARG;
  if (height > 65535) return PGSAG_ERR_UNSUPPORTED;
  const dim3 grid(pgsag_div_up((uint64_t)words_per_row * 32ull, 256), (unsigned)height);
  k_vote_pack<<<grid, 256, 0, (cudaStream_t)stream>>>(width, mask, words_per_row, bits);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

template <int kMaxViews, int kPPT>
static int launch_vote_ppt(uint32_t n, const float* pts, uint32_t nv, const VoteTable<kMaxViews>& T,
                           const uint32_t* bits, uint32_t tau, int acc, uint32_t* in_mask, uint32_t* us,
                           uint8_t* rel, int32_t* status, cudaStream_t s, unsigned max_blocks) {
  const unsigned groups = pgsag_div_up(n, (uint64_t)kVoteThreads * kPPT);
  const unsigned blocks = groups < max_blocks ? groups : max_blocks;
  k_vote<kMaxViews, kPPT><<<blocks, kVoteThreads, 0, s>>>(n, pts, nv, T, bits, tau, acc, in_mask, us, rel, status);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}

// Grid: at most one wave (as many CTAs as are resident at once); each CTA loops
// over groups of kVoteThreads * PGSAG_VOTE_PPT points.  4 points per thread (46
// registers, 5 CTAs per SM) measured fastest on B300 for 1M points x 32 views
// (85 us; 1 / 2 / 8 points per thread: 111 / 88 / 97 us).
#ifndef PGSAG_VOTE_PPT
#define PGSAG_VOTE_PPT 4
#endif
template <int kMaxViews>
static int launch_vote(uint32_t n, const float* pts, uint32_t nv, const pgsag_vote_view* views, const uint32_t* bits,
                       uint32_t tau, int acc, uint32_t* in_mask, uint32_t* us, uint8_t* rel, int32_t* status,
                       cudaStream_t s) {
  VoteTable<kMaxViews> T;
  for (uint32_t v = 0; v < nv; ++v) T.v[v] = views[v];
  for (uint32_t v = nv; v < (uint32_t)kMaxViews; ++v) T.v[v] = pgsag_vote_view{};
  static int occ = 0, sms = 0;
  if (occ <= 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PGSAG_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)k_vote<kMaxViews, PGSAG_VOTE_PPT>,
                                                      kVoteThreads, 0) != cudaSuccess)
      return PGSAG_ERR_CUDA;
    if (occ <= 0) occ = 1;
  }
  return launch_vote_ppt<kMaxViews, PGSAG_VOTE_PPT>(n, pts, nv, T, bits, tau, acc, in_mask, us, rel, status, s,
                                                    (unsigned)(sms * occ));
}

extern "C" int pgsag_vote_filter(uint32_t n_points, const float* points, uint32_t n_views,
                                 const pgsag_vote_view* views, const uint32_t* mask_bits, uint32_t tau,
                                 int accumulate, uint32_t* in_mask, uint32_t* us, uint8_t* reliable,
                                 int32_t* status, void* stream) {
  if (n_views > PGSAG_VOTE_MAX_VIEWS) return PGSAG_ERR_UNSUPPORTED;
  if (!status) return PGSAG_ERR_ARG;
  if (n_points == 0) return PGSAG_OK;
  if (!points || !in_mask || !us || !reliable || ((uintptr_t)points & 3u)) return PGSAG_ERR_ARG;
  if (n_views > 0 && (!views || !mask_bits)) return PGSAG_ERR_ARG;
  for (uint32_t v = 0; v < n_views; ++v) {
    const pgsag_vote_view& V = views[v];
    if (V.width <= 0 || V.height <= 0) return PGSAG_ERR_ARG;
    if ((uint64_t)V.words_per_row * 32ull < (uint64_t)V.width) return PGSAG_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (n_views <= 32)
    return launch_vote<32>(n_points, points, n_views, views, mask_bits, tau, accumulate, in_mask, us, reliable,
                           status, s);
  return launch_vote<PGSAG_VOTE_MAX_VIEWS>(n_points, points, n_views, views, mask_bits, tau, accumulate, in_mask,
                                           us, reliable, status, s);
}

extern "C" size_t pgsag_vote_compact_workspace_size(uint32_t n_points) {
  const uint64_t nb = n_points ? pgsag_div_up(n_points, kCmpPerBlock) : 1u;
  return (size_t)nb * sizeof(uint32_t);
}

extern "C" int pgsag_vote_compact(uint32_t n_points, const uint8_t* reliable, uint32_t* idx, uint32_t* n_out,
                                  void* workspace, size_t workspace_bytes, int32_t* status, void* stream) {
  if (!n_out || !status) return PGSAG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_points == 0) {
    PGSAG_CUDA(cudaMemsetAsync(n_out, 0, sizeof(uint32_t), s));
    return PGSAG_OK;
  }
  if (!reliable || !idx || !workspace || ((uintptr_t)workspace & 3u)) return PGSAG_ERR_ARG;
  if (workspace_bytes < pgsag_vote_compact_workspace_size(n_points)) return PGSAG_ERR_CAPACITY;
  const unsigned nb = pgsag_div_up(n_points, kCmpPerBlock);
  uint32_t* cnt = (uint32_t*)workspace;
  k_cmp_count<<<nb, kCmpThreads, 0, s>>>(n_points, reliable, cnt);
  PGSAG_CHECK_LAUNCH();
  k_cmp_scan<<<1, 1024, 0, s>>>(nb, cnt, n_out);
  PGSAG_CHECK_LAUNCH();
  k_cmp_scatter<<<nb, kCmpThreads, 0, s>>>(n_points, reliable, cnt, idx);
  PGSAG_CHECK_LAUNCH();
  return PGSAG_OK;
}
