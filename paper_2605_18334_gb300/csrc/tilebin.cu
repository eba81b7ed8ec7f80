// Tile-major binning: the second way sr_bin_sort builds the sorted key list
// (Preliminaries: each tile's Gaussians, in depth order).
//
//   1. the projection counts, per tile, the keys that land in it (one atomic
//      per key, from the same row spans it counts the keys with);
//   2. an exclusive scan over the tiles gives every tile its run of the list
//      (the ranges) and a cursor at the run's start;
//   3. tile_scatter_kernel enumerates each record's tiles (index order) and
//      places the record index in each tile's run at a cursor taken with an
//      atomic add: the runs are complete, their order arbitrary;
//   4. tile_segsort_kernel sorts each run by (FP32 depth bits, record index)
//      in shared memory (a bitonic network over 64-bit keys); runs longer
//      than one block holds are sorted in chunks and merged by
//      tile_bigsort_kernel.
//
// The result is the key list of the depth-sort-then-tile-sort path bit for
// bit: per tile, the records that touch it, ordered by depth bits with ties
// by record index.  It takes no global radix pass: the atomics replace the
// tile passes, and the per-tile sorts replace the depth passes.
#include <algorithm>

#include "kernels.cuh"

namespace sr {
namespace {

constexpr int kSegThreads = 256;
constexpr int kSegCap = 4096;  // keys one block sorts in shared memory (32 KB)

__device__ __forceinline__ int warp_owner_tb(uint32_t x, uint32_t q) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const uint32_t s = __shfl_sync(0xffffffffu, x, lo + step);
    if (s <= q) lo += step;
  }
  return lo;
}

__device__ __forceinline__ uint32_t span_cum_tb(uint32_t cum_lo, uint32_t cum_hi, int rr) {
  return ((rr < 4 ? cum_lo : cum_hi) >> (8 * (rr & 3))) & 0xffu;
}

__device__ __forceinline__ void place(uint32_t* __restrict__ cursor, uint32_t* __restrict__ vals,
                                      unsigned long long cap, uint32_t tile, uint32_t m) {
  const uint32_t pos = atomicAdd(cursor + tile, 1u);
  if (pos < cap) vals[pos] = m;
}

// Each warp takes 32 consecutive records (index order).  Records with packed
// row spans: the warp flattens their keys (an exclusive scan of the counts)
// and places 32 at a time, a lane finding its key's record by a binary
// search over the lanes' starts and its tile from the record's packed spans.
// Tall records: one at a time across the warp, a lane per tile row.
__global__ void __launch_bounds__(256) tile_scatter_kernel(int64_t n, int n_views, const ViewInfo* __restrict__ views,
                                                           const uint32_t* __restrict__ ntouch,
                                                           const uint2* __restrict__ rect,
                                                           const float4* __restrict__ rec,
                                                           const float4* __restrict__ foot,
                                                           uint32_t* __restrict__ cursor,
                                                           uint32_t* __restrict__ vals, unsigned long long cap) {
  pdl_entry();
  const int64_t m_total = n * n_views;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < m_total; w += warps) {
    const int64_t j = w * 32 + lane;
    uint32_t cnt = 0, rx = 0, ry = 0;
    uint4 sp = make_uint4(0u, 0u, 0u, 0u);
    if (j < m_total) {
      cnt = ntouch[j];
      if (cnt) {
        const uint2 r = rect[j];
        rx = r.x;
        ry = r.y;
        sp = reinterpret_cast<const uint4*>(foot)[4 * j + 1];
      }
    }
    const bool tall = cnt && sp.w == kSpansTall;
    const uint32_t m = (uint32_t)j;
    const uint32_t tx0 = rx & 0xffffu, ty0 = rx >> 16, ty1 = ry >> 16;
    uint32_t row0 = 0, tiles_x = 0;
    if (cnt) {
      const ViewInfo& vi = views[(int)((uint64_t)j / (uint64_t)n)];
      tiles_x = (uint32_t)vi.tiles_x;
      row0 = (uint32_t)(vi.tile_base + (int64_t)ty0 * vi.tiles_x);
    }
    // packed records: flattened keys, 32 at a time
    const uint32_t pc = tall ? 0u : cnt;
    uint32_t inc = pc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    const uint32_t excl = inc - pc;
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    for (uint32_t q0 = 0; q0 < total; q0 += 32) {
      const uint32_t q = q0 + lane;
      const int ow = warp_owner_tb(excl, q);
      const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, ow);
      const uint32_t o_m = __shfl_sync(0xffffffffu, m, ow);
      const uint32_t o_lo = __shfl_sync(0xffffffffu, sp.x, ow);
      const uint32_t o_hi = __shfl_sync(0xffffffffu, sp.y, ow);
      const uint32_t o_firsts = __shfl_sync(0xffffffffu, sp.z, ow);
      const uint32_t o_tx0 = __shfl_sync(0xffffffffu, tx0, ow);
      const uint32_t o_row0 = __shfl_sync(0xffffffffu, row0, ow);
      const uint32_t o_tx = __shfl_sync(0xffffffffu, tiles_x, ow);
      if (q < total) {
        const uint32_t k = q - o_excl;  // the key's index within its record
        const uint32_t kk = k * 0x01010101u;
        const uint32_t row = ((__popc(__vcmpgeu4(kk, o_lo)) + __popc(__vcmpgeu4(kk, o_hi))) >> 3) - 1u;
        const uint32_t first = (o_firsts >> (4 * row)) & 15u;
        const uint32_t tile = o_row0 + row * o_tx + o_tx0 + first + (k - span_cum_tb(o_lo, o_hi, (int)row));
        place(cursor, vals, cap, tile, o_m);
      }
    }
    // tall records, one at a time across the warp
    uint32_t pending = __ballot_sync(0xffffffffu, tall);
    while (pending) {
      const int src = __ffs(pending) - 1;
      pending &= pending - 1;
      const uint32_t tm = __shfl_sync(0xffffffffu, m, src);
      const uint32_t tcnt = __shfl_sync(0xffffffffu, cnt, src);
      const int t_ty0 = (int)__shfl_sync(0xffffffffu, ty0, src), t_ty1 = (int)__shfl_sync(0xffffffffu, ty1, src);
      const float4* ft = foot + 4 * (int64_t)tm;
      const float4 g0 = ft[0], g1 = ft[1], g2 = ft[2], g3 = ft[3];
      const float2 mu = reinterpret_cast<const float2*>(rec + 4 * (int64_t)tm)[0];
      const ViewInfo& vi = views[(int)(tm / (uint64_t)n)];
      uint32_t done = 0;
      for (int rb = t_ty0; rb < t_ty1; rb += 32) {
        const int ty = rb + lane;
        int tlo = 0, thi = -1;
        const bool ok = ty < t_ty1 && row_tile_span(g0, g1, g2, g3, mu.x, mu.y, ty, vi.width, vi.height, tlo, thi);
        const uint32_t num = ok ? (uint32_t)(thi - tlo + 1) : 0u;
        uint32_t rinc = num;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, rinc, o);
          if (lane >= o) rinc += y;
        }
        const uint32_t rexcl = rinc - num;
        const uint32_t rtotal = __shfl_sync(0xffffffffu, rinc, 31);
        const uint32_t first_tile = (uint32_t)(vi.tile_base + (int64_t)ty * vi.tiles_x) + (uint32_t)tlo;
        for (uint32_t c0 = 0; c0 < rtotal; c0 += 32) {
          const uint32_t q = c0 + lane;
          const int ow = warp_owner_tb(rexcl, q);
          const uint32_t o_excl = __shfl_sync(0xffffffffu, rexcl, ow);
          const uint32_t o_first = __shfl_sync(0xffffffffu, first_tile, ow);
          if (q < rtotal && done + q < tcnt) place(cursor, vals, cap, o_first + (q - o_excl), tm);
        }
        done += rtotal;
      }
    }
  }
}

__device__ __forceinline__ unsigned long long seg_key(const uint32_t* __restrict__ depth, uint32_t v) {
  return ((unsigned long long)depth[v] << 32) | v;
}

// Bitonic sort of s[0, P) ascending, P a power of two <= kSegCap.
__device__ __forceinline__ void bitonic_sort(unsigned long long* s, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = s[lo], b = s[hi];
        if ((a > b) == up) {
          s[lo] = b;
          s[hi] = a;
        }
      }
      __syncthreads();
    }
  }
}

// One block per tile: its run, sorted by (depth bits, record index).  Runs
// longer than kSegCap are listed for tile_bigsort_kernel.
__global__ void __launch_bounds__(kSegThreads) tile_segsort_kernel(const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ depth,
                                                                   uint32_t* __restrict__ vals,
                                                                   unsigned long long cap, uint32_t* __restrict__ big) {
  pdl_entry();
  __shared__ unsigned long long s[kSegCap];
  const int64_t tile = blockIdx.x;
  const uint2 r = tile_range(ranges, tile);
  const uint32_t n = r.y - r.x;
  if (n < 2 || r.y > cap) return;  // nothing to order, or the frame overflowed the key capacity
  if (n > (uint32_t)kSegCap) {
    if (threadIdx.x == 0) big[1 + atomicAdd(big, 1u)] = (uint32_t)tile;
    return;
  }
  int P = 2;
  while (P < (int)n) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < (int)n ? seg_key(depth, vals[r.x + i]) : ~0ull;
  __syncthreads();
  bitonic_sort(s, P);
  for (int i = threadIdx.x; i < (int)n; i += blockDim.x) vals[r.x + i] = (uint32_t)s[i];
}

// Number of elements of the sorted run src[0, len) whose key is below key.
__device__ __forceinline__ uint32_t rank_below(const uint32_t* __restrict__ src, uint32_t len,
                                               const uint32_t* __restrict__ depth, unsigned long long key) {
  uint32_t lo = 0, hi = len;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (seg_key(depth, src[mid]) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Runs longer than kSegCap (big[0] of them, tile ids at big[1..]): one block
// per run at a time sorts its chunks of kSegCap in shared memory, then merges
// neighbouring sorted pieces pairwise (each element's place in the merged
// piece is its index plus its rank in the other piece; keys are distinct),
// alternating between vals and tmp, and leaves the result in vals.
__global__ void __launch_bounds__(kSegThreads) tile_bigsort_kernel(const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ depth,
                                                                   uint32_t* __restrict__ vals,
                                                                   uint32_t* __restrict__ tmp,
                                                                   const uint32_t* __restrict__ big) {
  pdl_entry();
  __shared__ unsigned long long s[kSegCap];
  const uint32_t nbig = big[0];
  for (uint32_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const uint2 r = tile_range(ranges, big[1 + b]);
    const uint32_t n = r.y - r.x;
    uint32_t* src = vals + r.x;
    uint32_t* dst = tmp + r.x;
    for (uint32_t c = 0; c < n; c += kSegCap) {
      const uint32_t len = min((uint32_t)kSegCap, n - c);
      for (int i = threadIdx.x; i < kSegCap; i += blockDim.x)
        s[i] = i < (int)len ? seg_key(depth, src[c + i]) : ~0ull;
      __syncthreads();
      bitonic_sort(s, kSegCap);
      for (int i = threadIdx.x; i < (int)len; i += blockDim.x) src[c + i] = (uint32_t)s[i];
      __syncthreads();
    }
    for (uint32_t run = kSegCap; run < n; run <<= 1) {
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const uint32_t piece = i / (2 * run) * (2 * run);  // start of the pair of pieces
        const uint32_t a0 = piece, a1 = min(piece + run, n), b1 = min(piece + 2 * run, n);
        const unsigned long long key = seg_key(depth, src[i]);
        uint32_t out;
        if (i < a1) out = piece + (i - a0) + rank_below(src + a1, b1 - a1, depth, key);
        else out = piece + (i - a1) + rank_below(src + a0, a1 - a0, depth, key);
        dst[out] = src[i];
      }
      __syncthreads();
      uint32_t* t = src;
      src = dst;
      dst = t;
    }
    if (src != vals + r.x)
      for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) vals[r.x + i] = src[i];
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_tile_scatter(const BinArgs& a, cudaStream_t st, int sms) {
  const int64_t m = a.n * a.n_views;
  if (m == 0) return cudaSuccess;
  const int64_t want = (m + 255) / 256;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  launch_pdl(tile_scatter_kernel, dim3(grid), dim3(256), 0, st, a.n, a.n_views, (const ViewInfo*)a.ws.views,
             (const uint32_t*)a.ws.ntouch, (const uint2*)a.ws.rect, (const float4*)a.ws.rec,
             (const float4*)a.ws.foot, a.ws.tile_cur, a.ws.vals[0], a.cap);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tile_segsort(const BinArgs& a, cudaStream_t st, int sms) {
  if (a.total_tiles == 0) return cudaSuccess;
  launch_pdl(tile_segsort_kernel, dim3((unsigned)a.total_tiles), dim3(kSegThreads), 0, st,
             (const uint2*)a.ws.ranges, (const uint32_t*)a.ws.depth, a.ws.vals[0], a.cap, a.ws.tile_big);
  launch_pdl(tile_bigsort_kernel, dim3((unsigned)sms), dim3(kSegThreads), 0, st, (const uint2*)a.ws.ranges,
             (const uint32_t*)a.ws.depth, a.ws.vals[0], a.ws.vals[1], (const uint32_t*)a.ws.tile_big);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace sr
