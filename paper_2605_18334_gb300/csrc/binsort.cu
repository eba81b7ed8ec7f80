// Tile binning and depth sort (the tile-based, depth-sorted pipeline of the
// Preliminaries).  The result is the order of the key (global tile << 32 |
// FP32 depth bits) with ties broken by record index, obtained in two sorts:
//
//   depth sort   the M records by their 32-bit depth key (records that touch
//                no tile carry ~0 and sink to the end): 4 stable 8-bit passes
//                over M, not over the (much larger) number of tile keys; the
//                last pass writes the records' tile counts in depth order
//   scan         exclusive scan of the tile counts in depth order
//   duplicate    one 32-bit global tile id per touched tile, value = record
//                index, emitted in depth order (warp-cooperative, coalesced),
//                counting the tile sort's digit histograms on the way
//   tile sort    stable LSD passes over the tile-id bits only; stability
//                keeps the depth order (and index order of equal depths)
//                inside every tile; the last pass also reduces the tile ranges
//   order        the composites' tile order, longest key lists first
//
// Every radix pass is one onesweep launch: a block ranks a partition of 4096
// keys with warp match-any, stages them in shared memory in block-local
// order, resolves its global offsets by a decoupled look-back over the
// preceding partitions (each wait bounded), and scatters each digit's run
// contiguously.
#include <algorithm>
#include <cstddef>
#include <mutex>

#include "kernels.cuh"

namespace sr {

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// block-wide exclusive scan (NT threads), total in `total`
template <int NT>
__device__ __forceinline__ unsigned long long block_exclusive_u64(unsigned long long x, unsigned long long* s_warp,
                                                                  unsigned long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < NT / 32 ? s_warp[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < NT / 32) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[NT / 32 - 1];
  const unsigned long long before = warp > 0 ? s_warp[warp - 1] : 0ull;
  __syncthreads();
  return before + inc - x;
}

__device__ __forceinline__ unsigned long long element_count(const unsigned long long* count_dev,
                                                            unsigned long long count) {
  if (!count_dev) return count;
  const unsigned long long c = *count_dev;
  return c < count ? c : count;
}

// ---------------------------------------------------------------------------
// scan of the tile counts (in the order given by perm)
// ---------------------------------------------------------------------------
// the kScanItems counts of this thread, in order (16-byte loads when the
// thread's slice is whole; the counts array is 256-byte aligned)
__device__ __forceinline__ void scan_load(const uint32_t* __restrict__ cnt, int64_t base, int64_t m,
                                          uint32_t (&v)[kScanItems]) {
  if (base + kScanItems <= m) {
#pragma unroll
    for (int k = 0; k < kScanItems; k += 4) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(cnt + base + k));
      v[k] = q.x;
      v[k + 1] = q.y;
      v[k + 2] = q.z;
      v[k + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) v[k] = base + k < m ? cnt[base + k] : 0u;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ cnt, int64_t m,
                                                                   unsigned long long* __restrict__ part) {
  pdl_entry();
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  scan_load(cnt, base, m, v);
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) sum += v[k];
  unsigned long long total;
  block_exclusive_u64<kScanThreads>(sum, s_warp, total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_parts_kernel(unsigned long long* part, int nb, Status* st,
                                                          unsigned long long cap) {
  pdl_entry();
  __shared__ unsigned long long s_warp[32];
  unsigned long long carry = 0;
  for (int c0 = 0; c0 < nb; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const unsigned long long x = i < nb ? part[i] : 0ull;
    unsigned long long total;
    const unsigned long long ex = block_exclusive_u64<1024>(x, s_warp, total);
    if (i < nb) part[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) {
    part[nb] = carry;
    st->keys_needed = carry;
    if (carry > cap) raise_status(st, kStatusCapacity);
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const uint32_t* __restrict__ cnt, int64_t m,
                                                                 const unsigned long long* __restrict__ part,
                                                                 uint32_t* __restrict__ offsets) {
  pdl_entry();
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  scan_load(cnt, base, m, v);
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) sum += v[k];
  unsigned long long total;
  unsigned long long run = block_exclusive_u64<kScanThreads>(sum, s_warp, total) + part[blockIdx.x];
  uint32_t o[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    o[k] = run > 0xffffffffull ? 0xffffffffu : (uint32_t)run;
    run += v[k];
  }
  if (base + kScanItems <= m) {
#pragma unroll
    for (int k = 0; k < kScanItems; k += 4)
      *reinterpret_cast<uint4*>(offsets + base + k) = make_uint4(o[k], o[k + 1], o[k + 2], o[k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (base + k < m) offsets[base + k] = o[k];
  }
}

// ---------------------------------------------------------------------------
// key duplication, in depth order.  A warp takes 32 consecutive depth-sorted
// records and writes their keys as one contiguous run: each lane finds the
// record owning its output slot by a binary search over the lanes' starts
// and decodes the slot's tile from the owner's packed row spans (coalesced
// writes).  Records whose tile box is too large for packed spans are then
// taken one at a time by the whole warp: a lane per tile row computes the
// row's span (row_tile_span), a warp scan places the rows, and the keys go
// out 32 at a time by the same owner search.  The digit histograms of the
// tile sort are counted on the way (keys are written once and not re-read).
// ---------------------------------------------------------------------------
// Digit histograms of the tile sort, counted per span of consecutive tile ids
// [a, a + len) instead of per key.  Digit 0 runs through consecutive values:
// whole cycles of 256 go to one counter, the rest into a difference array
// (two or four adds); a higher digit p changes only at multiples of 256^p,
// so the span splits into a few constant-digit pieces.
struct TileHist {
  int diff0[257];            // difference array of digit 0 (partial cycles)
  uint32_t cycles0;          // whole cycles of digit 0 (each adds 1 to every bin)
  uint32_t h[kMaxPasses][256];  // digits 1.. (row 0 unused)
};

__device__ __forceinline__ void tile_hist_span(TileHist& th, int passes, uint32_t a, uint32_t len) {
  if (len == 0) return;
  const uint32_t full = len >> 8, rem = len & 0xffu;
  if (full) atomicAdd(&th.cycles0, full);
  if (rem) {
    const uint32_t a0 = a & 0xffu, e0 = a0 + rem;
    atomicAdd(&th.diff0[a0], 1);
    if (e0 <= 256u) {
      atomicAdd(&th.diff0[e0], -1);
    } else {
      atomicAdd(&th.diff0[256], -1);
      atomicAdd(&th.diff0[0], 1);
      atomicAdd(&th.diff0[e0 - 256u], -1);
    }
  }
  const uint32_t b = a + len - 1;
  for (int p = 1; p < passes; ++p) {
    const int sh = 8 * p;
    const uint32_t unit_mask = sh >= 32 ? 0xffffffffu : ((1u << sh) - 1u);
    for (uint32_t t = a;;) {
      const uint32_t seg_end = min(b, t | unit_mask);
      atomicAdd(&th.h[p][(t >> sh) & 0xffu], seg_end - t + 1u);
      if (seg_end == b) break;
      t = seg_end + 1u;
    }
  }
}

// index of the last lane whose (non-decreasing) x is <= q
__device__ __forceinline__ int warp_owner(uint32_t x, uint32_t q) {
  int lo = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const uint32_t s = __shfl_sync(0xffffffffu, x, lo + step);
    if (s <= q) lo += step;
  }
  return lo;
}

// prefix count of packed row rr (one byte per row)
__device__ __forceinline__ uint32_t span_cum(uint32_t cum_lo, uint32_t cum_hi, int rr) {
  return ((rr < 4 ? cum_lo : cum_hi) >> (8 * (rr & 3))) & 0xffu;
}

// one lane's record in the duplication pipeline
struct DupFields {
  uint32_t m, start, cnt, rx, ry;
  uint4 sp;  // the footprint's second float4, as bits (packed row spans or kSpansTall)
};

__device__ __forceinline__ void dup_load_index(const uint32_t* __restrict__ perm,
                                               const uint32_t* __restrict__ offsets, int64_t m_total, int64_t w,
                                               int lane, uint32_t& m, uint32_t& start) {
  const int64_t j = w * 32 + lane;
  if (j < m_total) {
    m = perm[j];
    start = offsets[j];
  } else {
    m = 0;
    start = 0xffffffffu;
  }
}

__device__ __forceinline__ void dup_load_fields(const uint32_t* __restrict__ cnt_sorted,
                                                const uint2* __restrict__ rect, const float4* __restrict__ foot,
                                                int64_t m_total, int64_t w, int lane, DupFields& f) {
  f.cnt = 0;
  f.rx = f.ry = 0;
  f.sp = make_uint4(0u, 0u, 0u, 0u);
  const int64_t j = w * 32 + lane;
  if (j < m_total) {
    f.cnt = cnt_sorted[j];
    const uint2 r = rect[f.m];
    f.sp = reinterpret_cast<const uint4*>(foot)[4 * (int64_t)f.m + 1];
    f.rx = r.x;
    f.ry = r.y;
  }
}

__global__ void __launch_bounds__(256, 4) duplicate_kernel(int64_t n, int n_views, const ViewInfo* __restrict__ views,
                                                        const uint32_t* __restrict__ perm,
                                                        const uint32_t* __restrict__ cnt_sorted,
                                                        const uint32_t* __restrict__ offsets,
                                                        const uint2* __restrict__ rect,
                                                        const float4* __restrict__ rec,
                                                        const float4* __restrict__ foot,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        unsigned long long cap, uint32_t* __restrict__ tile_hist,
                                                        int passes) {
  pdl_entry();
  __shared__ TileHist th;
  for (int i = threadIdx.x; i < 257; i += blockDim.x) th.diff0[i] = 0;
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) (&th.h[0][0])[i] = 0u;
  if (threadIdx.x == 0) th.cycles0 = 0u;
  __syncthreads();
  const int64_t m_total = n * n_views;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  // Three-stage software pipeline over the warp's groups of 32 records: the
  // sorted index and key offset of group i+2, then the record fields of
  // group i+1 (which depend on the index), are in flight while group i is
  // written.
  const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  DupFields cur, nxt;
  uint32_t nn_m = 0, nn_start = 0xffffffffu;
  dup_load_index(perm, offsets, m_total, w0, lane, cur.m, cur.start);
  dup_load_fields(cnt_sorted, rect, foot, m_total, w0, lane, cur);
  dup_load_index(perm, offsets, m_total, w0 + warps, lane, nxt.m, nxt.start);
  for (int64_t w = w0; w * 32 < m_total; w += warps) {
    dup_load_fields(cnt_sorted, rect, foot, m_total, w + warps, lane, nxt);
    dup_load_index(perm, offsets, m_total, w + 2 * warps, lane, nn_m, nn_start);
    const uint32_t m = cur.m, cnt = cur.cnt, start = cur.start;
    const uint32_t cum_lo = cur.sp.x, cum_hi = cur.sp.y, firsts = cur.sp.z;
    const uint32_t tx0 = cur.rx & 0xffffu, ty0 = cur.rx >> 16, ty1 = cur.ry >> 16;
    const bool tall = cnt && cur.sp.w == kSpansTall;
    uint32_t row0 = 0, tiles_x = 0;  // global tile id of (0, ty0) and the view's tiles per row
    if (cnt) {
      const ViewInfo& vi = views[(int)(m / (uint64_t)n)];
      tiles_x = (uint32_t)vi.tiles_x;
      row0 = (uint32_t)(vi.tile_base + (int64_t)ty0 * vi.tiles_x);
      if (!tall) {
        // histogram of this record's keys, one call per packed row span
#pragma unroll
        for (int rr = 0; rr < kSpanRows; ++rr) {
          const uint32_t c0 = span_cum(cum_lo, cum_hi, rr);
          if (c0 < cnt) {
            const uint32_t c1 = rr + 1 < kSpanRows ? min(span_cum(cum_lo, cum_hi, rr + 1), cnt) : cnt;
            tile_hist_span(th, passes, row0 + (uint32_t)rr * tiles_x + tx0 + ((firsts >> (4 * rr)) & 15u), c1 - c0);
          }
        }
      }
    }
    cur = nxt;
    nxt.m = nn_m;
    nxt.start = nn_start;
    // the run of this warp: [start of lane 0, end of the last valid lane)
    const uint32_t base = __shfl_sync(0xffffffffu, start, 0);
    const uint32_t end = __reduce_max_sync(0xffffffffu, cnt ? start + cnt : 0u);
    const uint32_t rel = start - base;  // non-decreasing over lanes; huge past the last record
    // warp-uniform loop: every lane takes part in the shuffles
    for (uint32_t p0 = base; p0 < end; p0 += 32) {
      const uint32_t p = p0 + lane;
      const uint32_t q_rel = p - base;
      // owner: the last lane whose start <= q_rel (lanes without tiles share
      // their start with the next lane, whose range then covers q_rel)
      const int lo = warp_owner(rel, q_rel);
      const uint32_t o_rel = __shfl_sync(0xffffffffu, rel, lo);
      const uint32_t o_m = __shfl_sync(0xffffffffu, m, lo);
      const uint32_t o_cum_lo = __shfl_sync(0xffffffffu, cum_lo, lo);
      const uint32_t o_cum_hi = __shfl_sync(0xffffffffu, cum_hi, lo);
      const uint32_t o_firsts = __shfl_sync(0xffffffffu, firsts, lo);
      const bool o_tall = __shfl_sync(0xffffffffu, (uint32_t)tall, lo) != 0u;
      const uint32_t o_tx0 = __shfl_sync(0xffffffffu, tx0, lo);
      const uint32_t o_row0 = __shfl_sync(0xffffffffu, row0, lo);
      const uint32_t o_tx = __shfl_sync(0xffffffffu, tiles_x, lo);
      bool on = false;
      uint32_t key = 0;
      if (p < end && !o_tall) {
        // the q-th key's row: the last row whose prefix count is <= q (a
        // byte-wise compare of q against the eight prefixes, then a popcount)
        const uint32_t q = q_rel - o_rel;
        const uint32_t qq = q * 0x01010101u;
        const uint32_t row = ((__popc(__vcmpgeu4(qq, o_cum_lo)) + __popc(__vcmpgeu4(qq, o_cum_hi))) >> 3) - 1u;
        const uint32_t first = (o_firsts >> (4 * row)) & 15u;
        key = o_row0 + row * o_tx + o_tx0 + first + (q - span_cum(o_cum_lo, o_cum_hi, (int)row));
        on = p < cap;
      }
      if (on) {
        keys[p] = key;
        vals[p] = o_m;
      }
    }
    // tall records, one at a time across the warp
    uint32_t pending = __ballot_sync(0xffffffffu, tall);
    while (pending) {
      const int src = __ffs(pending) - 1;
      pending &= pending - 1;
      const uint32_t tm = __shfl_sync(0xffffffffu, m, src);
      const uint32_t tstart = __shfl_sync(0xffffffffu, start, src);
      const uint32_t tcnt = __shfl_sync(0xffffffffu, cnt, src);
      const int t_ty0 = (int)__shfl_sync(0xffffffffu, ty0, src), t_ty1 = (int)__shfl_sync(0xffffffffu, ty1, src);
      // the record's footprint constants (one address for the whole warp)
      const float4* ft = foot + 4 * (int64_t)tm;
      const float4 g0 = ft[0], g1 = ft[1], g2 = ft[2], g3 = ft[3];
      const float2 mu = reinterpret_cast<const float2*>(rec + 4 * (int64_t)tm)[0];
      const float mx = mu.x, my = mu.y;
      const ViewInfo& vi = views[(int)(tm / (uint64_t)n)];
      uint32_t done = 0;  // keys of this record placed by earlier row groups
      for (int rb = t_ty0; rb < t_ty1; rb += 32) {
        const int ty = rb + lane;
        int tlo = 0, thi = -1;
        const bool ok = ty < t_ty1 && row_tile_span(g0, g1, g2, g3, mx, my, ty, vi.width, vi.height, tlo, thi);
        const uint32_t num = ok ? (uint32_t)(thi - tlo + 1) : 0u;
        uint32_t inc = num;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += y;
        }
        const uint32_t excl = inc - num;
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        const uint32_t first_key = (uint32_t)(vi.tile_base + (int64_t)ty * vi.tiles_x) + (uint32_t)tlo;
        // histogram: this lane's row span, up to the record's count
        tile_hist_span(th, passes, first_key, done + excl >= tcnt ? 0u : min(num, tcnt - done - excl));
        for (uint32_t c0 = 0; c0 < total; c0 += 32) {
          const uint32_t q = c0 + lane;
          const int ow = warp_owner(excl, q);
          const uint32_t o_excl = __shfl_sync(0xffffffffu, excl, ow);
          const uint32_t o_key = __shfl_sync(0xffffffffu, first_key, ow);
          const unsigned long long pos = (unsigned long long)tstart + done + q;
          const bool on = q < total && done + q < tcnt && pos < cap;
          const uint32_t key = o_key + (q - o_excl);
          if (on) {
            keys[pos] = key;
            vals[pos] = tm;
          }
        }
        done += total;
      }
    }
  }
  __syncthreads();
  // digit 0: prefix sum of the difference array (one warp), plus whole cycles
  if (threadIdx.x < 32) {
    int run = 0;
    for (int c = 0; c < 8; ++c) {
      const int v = th.diff0[c * 32 + threadIdx.x];
      int inc = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)threadIdx.x >= o) inc += y;
      }
      const uint32_t cnt0 = (uint32_t)(run + inc) + th.cycles0;
      if (cnt0) atomicAdd(tile_hist + c * 32 + threadIdx.x, cnt0);
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  for (int i = 256 + threadIdx.x; i < passes * 256; i += blockDim.x) {
    const uint32_t c = (&th.h[0][0])[i];
    if (c) atomicAdd(tile_hist + i, c);
  }
}

// ---------------------------------------------------------------------------
// digit histograms of `passes` 8-bit digits
// ---------------------------------------------------------------------------
template <class KEY>
__global__ void __launch_bounds__(256) histogram_kernel(const KEY* __restrict__ keys,
                                                        const unsigned long long* count_dev,
                                                        unsigned long long count, int passes,
                                                        uint32_t* __restrict__ hist) {
  pdl_entry();
  __shared__ uint32_t s_h[kMaxPasses][256];
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) (&s_h[0][0])[i] = 0u;
  __syncthreads();
  const unsigned long long kn = element_count(count_dev, count);
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  // four keys of a thread in flight at a time
  for (unsigned long long k0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k0 < kn; k0 += 4 * stride) {
    unsigned long long key[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) key[u] = k0 + u * stride < kn ? (unsigned long long)keys[k0 + u * stride] : 0ull;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (k0 + u * stride < kn)
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(key[u] >> (8 * p)) & 0xffu], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) {
    const uint32_t c = (&s_h[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// per pass: exclusive digit offsets in place, and whether one digit holds every key
__global__ void __launch_bounds__(256) hist_scan_kernel(uint32_t* __restrict__ hist, uint32_t* trivial,
                                                        const unsigned long long* count_dev,
                                                        unsigned long long count) {
  pdl_entry();
  __shared__ unsigned long long s_warp[8];
  const int p = blockIdx.x;
  const unsigned long long kn = element_count(count_dev, count);
  const uint32_t c = hist[p * 256 + threadIdx.x];
  unsigned long long total;
  const unsigned long long ex = block_exclusive_u64<256>(c, s_warp, total);
  hist[p * 256 + threadIdx.x] = (uint32_t)ex;
  const int full = __syncthreads_or(kn > 0 && c == kn);
  if (threadIdx.x == 0) trivial[p] = full ? 1u : 0u;
}

// ---------------------------------------------------------------------------
// one onesweep radix pass
// ---------------------------------------------------------------------------
// Look-back word of (partition, pass, digit): a flag in bits 62-63 (0: not
// published, kFlagAgg: the partition's count of the digit, kFlagInc: the
// inclusive prefix of the digit up to and including the partition) and the
// value below it.
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

template <class KEY>
struct PassArgs {
  const KEY* keys_in;
  const uint32_t* vals_in;        // nullptr: the value is the element's input index
  KEY* keys_out;
  uint32_t* vals_out;
  const uint32_t* digit_base;     // exclusive digit offsets of this pass
  unsigned long long* lookback;   // [parts][passes][256] look-back words, zeroed per frame
  uint32_t* part_counter;         // partition tickets of this pass (zeroed)
  const unsigned long long* count_dev;  // element count on the device, or nullptr
  unsigned long long count;       // element count (count_dev == nullptr) or the capacity bound
  Status* st;                     // status flags (timeouts)
  uint2* ranges;                  // last pass of the tile sort: tile ranges to reduce into, else nullptr
  unsigned long long n_tiles;     // number of tiles (bounds the range writes)
  int sorted_buf;                 // last pass of the tile sort: index of the output buffer
  const uint32_t* out_gather;     // last pass of the depth sort: keys_out receives out_gather[value]
                                  // (the sorted keys are not needed afterwards), else nullptr
  int passes;
  int pass;
  int shift;
  int bits;                       // digit width of this pass (8, less on the last pass of a narrower key)
  int spin_limit;
};

// shared memory of one onesweep block: the partition's keys and values in
// their block-local sorted order, per-warp digit counts, digit starts
template <class KEY>
struct SortSmem {
  KEY key[kSortPart];
  uint32_t val[kSortPart];
  uint32_t whist[kSortThreads / 32][256];
  uint32_t lstart[256];
  uint32_t gofs[256];  // modulo 2^32: positions stay below 2^32
  unsigned long long warp_tot[kSortThreads / 32];
  uint32_t part;
};

constexpr int kLookbackWindow = 4;  // look-back words in flight per digit

template <class KEY>
__global__ void __launch_bounds__(kSortThreads, 4) onesweep_kernel(PassArgs<KEY> a) {
  pdl_entry();
  constexpr int NW = kSortThreads / 32;
  extern __shared__ __align__(16) unsigned char s_raw[];
  SortSmem<KEY>& sm = *reinterpret_cast<SortSmem<KEY>*>(s_raw);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t dmask = (1u << a.bits) - 1u;  // this pass's digit: bits [shift, shift + bits)
  const unsigned long long kn = element_count(a.count_dev, a.count);
  const unsigned long long nparts = (kn + kSortPart - 1) / kSortPart;
  if (tid == 0) sm.part = atomicAdd(a.part_counter, 1u);
  for (int i = tid; i < NW * 256; i += kSortThreads) (&sm.whist[0][0])[i] = 0u;
  __syncthreads();
  const unsigned long long part = sm.part;
  if (part >= nparts) return;
  const unsigned long long base = part * kSortPart;
  // warp-blocked: warp w owns elements [w*512, (w+1)*512) of the partition;
  // element j of this thread is wbase + 32 j, valid while 32 j < rem
  const unsigned long long wbase = base + (unsigned long long)warp * (32 * kSortItems) + lane;
  const int rem = wbase >= kn ? 0 : (kn - wbase < 32ull * kSortItems ? (int)(kn - wbase) : 32 * kSortItems);

  // all key and value loads first, so a thread's 32 reads are in flight together
  KEY key[kSortItems];
  uint32_t val[kSortItems];
  const KEY* kp = a.keys_in + wbase;
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) key[j] = 32 * j < rem ? kp[32 * j] : (KEY)~(KEY)0;
  if (a.vals_in) {
    const uint32_t* vp = a.vals_in + wbase;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) val[j] = 32 * j < rem ? vp[32 * j] : 0u;
  } else {
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) val[j] = (uint32_t)wbase + 32 * j;
  }

  // rank inside the warp (lanes holding the same digit are peers); ranks are
  // below 512, two to a register
  uint32_t rank2[kSortItems / 2];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const bool valid = 32 * j < rem;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const uint32_t d = (uint32_t)(key[j] >> a.shift) & dmask;
      const uint32_t peers = __match_any_sync(vmask, d);
      const uint32_t prev = sm.whist[warp][d];
      __syncwarp(vmask);
      if ((peers & lt) == 0) sm.whist[warp][d] = prev + __popc(peers);
      __syncwarp(vmask);
      const uint32_t r = prev + __popc(peers & lt);
      rank2[j >> 1] = (j & 1) ? (rank2[j >> 1] | (r << 16)) : r;
    } else if (!(j & 1)) {
      rank2[j >> 1] = 0u;
    }
    __syncwarp();
  }
  __syncthreads();

  // per digit (thread d): counts across warps -> warp offsets; publish the
  // partition's count of digit d
  const int d = tid;  // kSortThreads == 256 digits
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t c = sm.whist[w][d];
    sm.whist[w][d] = tot;
    tot += c;
  }
  unsigned long long* lb = a.lookback + (part * a.passes + a.pass) * 256;
  st_relaxed_u64(lb + d, (part == 0 ? kFlagInc : kFlagAgg) | tot);

  // block-local order: digit starts, then keys and values into shared memory
  unsigned long long total;
  sm.lstart[d] = (uint32_t)block_exclusive_u64<kSortThreads>(tot, sm.warp_tot, total);
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    if (32 * j < rem) {
      const uint32_t dg = (uint32_t)(key[j] >> a.shift) & dmask;
      const uint32_t lpos = sm.lstart[dg] + sm.whist[warp][dg] + ((rank2[j >> 1] >> (16 * (j & 1))) & 0xffffu);
      sm.key[lpos] = key[j];
      sm.val[lpos] = val[j];
    }
  }

  // decoupled look-back over the predecessors' words of digit d, a window of
  // kLookbackWindow loads in flight: aggregates are summed, an inclusive
  // prefix ends the walk, a word not yet published is polled again (at most
  // spin_limit times)
  unsigned long long excl = 0;
  if (part > 0) {
    const unsigned long long stride = (unsigned long long)a.passes * 256;
    const unsigned long long* col = a.lookback + (unsigned long long)a.pass * 256 + d;
    long long q = (long long)part - 1;
    int spins = 0;
    bool walking = true;
    while (walking) {
      unsigned long long w[kLookbackWindow];
#pragma unroll
      for (int k = 0; k < kLookbackWindow; ++k)
        w[k] = q - k >= 0 ? ld_relaxed_u64(col + (unsigned long long)(q - k) * stride) : 0ull;
      bool stalled = false;
#pragma unroll
      for (int k = 0; k < kLookbackWindow; ++k) {
        if (!walking || stalled || q < 0) continue;
        const unsigned long long v = w[k];
        if (v & kFlagInc) {
          excl += v & kValMask;
          walking = false;
        } else if (v & kFlagAgg) {
          excl += v & kValMask;
          --q;
          walking = q >= 0;
        } else {
          stalled = true;  // not published yet: poll from q again
        }
      }
      if (walking && stalled) {
        if (++spins > a.spin_limit) {  // bounded wait: report and go on
          raise_status(a.st, kStatusTimeout);
          atomicCAS(&a.st->timeout_where, 0u, (uint32_t)(a.pass * 1000000 + (part % 1000000)) + 1u);
          walking = false;
        } else {
          __nanosleep(32);
        }
      }
    }
    st_relaxed_u64(lb + d, kFlagInc | (excl + tot));
  }
  // global position of local element i of digit dg: gofs[dg] + i
  sm.gofs[d] = (uint32_t)((unsigned long long)a.digit_base[d] + excl - sm.lstart[d]);
  __syncthreads();

  // scatter in block-local order, so each digit's run goes out contiguously
  const uint32_t count = (uint32_t)((kn - base) < (unsigned long long)kSortPart ? (kn - base) : kSortPart);
#pragma unroll 4
  for (uint32_t i = tid; i < count; i += kSortThreads) {
    const KEY k = sm.key[i];
    const uint32_t dg = (uint32_t)(k >> a.shift) & dmask;
    const uint32_t g = sm.gofs[dg] + i;
    if (g < kn) {  // always true unless a look-back gave up
      const uint32_t v = sm.val[i];
      a.keys_out[g] = a.out_gather ? (KEY)a.out_gather[v] : k;
      a.vals_out[g] = v;
      // after the last pass the keys are sorted, and the equal keys of this
      // partition are one run in block-local order: its ends bound the tile's
      // range (partitions combine by atomicMax on (~start, end))
      if (a.ranges && (unsigned long long)k < a.n_tiles) {
        if (i == 0 || sm.key[i - 1] != k) atomicMax(&a.ranges[k].x, ~(uint32_t)g);
        if (i + 1 == count || sm.key[i + 1] != k) atomicMax(&a.ranges[k].y, (uint32_t)(g + 1));
      }
    }
  }
  if (a.ranges && part == 0 && tid == 0) a.st->sorted_buf = (uint32_t)a.sorted_buf;
}

// ---------------------------------------------------------------------------
// tile ranges
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ keys, Status* st,
                                                     unsigned long long cap, uint2* __restrict__ ranges,
                                                     int sorted_buf) {
  pdl_entry();
  const unsigned long long kn = element_count(&st->keys_needed, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->sorted_buf = (uint32_t)sorted_buf;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < kn;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t t = keys[k];
    if (k == 0 || keys[k - 1] != t) ranges[t].x = ~(uint32_t)k;
    if (k + 1 == kn || keys[k + 1] != t) ranges[t].y = (uint32_t)(k + 1);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int clamp_grid(unsigned long long blocks, int sms, int per_sm) {
  const unsigned long long cap = (unsigned long long)sms * per_sm;
  if (blocks < 1) blocks = 1;
  return (int)(blocks < cap ? blocks : cap);
}

// Runs `passes` onesweep passes (those with run[p] != 0, or all if run is
// null) from (keys_in, vals_in) through the ping-pong buffers kbuf/vbuf;
// returns the index of the buffer holding the result, or -1 if no pass ran.
template <class KEY>
static int run_passes(const KEY* keys_in, const uint32_t* vals_in, KEY* const* kbuf, uint32_t* const* vbuf,
                      const uint32_t* hist, unsigned long long* lookback, uint32_t* part_counter,
                      const unsigned long long* count_dev, unsigned long long count, unsigned long long parts,
                      int passes, int key_bits, const int* run, Status* status, int spin_limit,
                      cudaStream_t st, uint2* ranges = nullptr, unsigned long long n_tiles = 0,
                      const int* buf_ids = nullptr, const uint32_t* last_gather = nullptr,
                      cudaError_t* first_error = nullptr) {
  int cur = -1;  // -1: still the input
  int last = -1;
  for (int p = 0; p < passes; ++p)
    if (!run || run[p]) last = p;
  // above the 48 KB default; a host-side attribute, no stream work
  cudaFuncSetAttribute(onesweep_kernel<KEY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem<KEY>));
  for (int p = 0; p < passes; ++p) {
    if (run && !run[p]) continue;
    const int out = cur == 0 ? 1 : 0;
    PassArgs<KEY> pa;
    pa.keys_in = cur < 0 ? keys_in : kbuf[cur];
    pa.vals_in = cur < 0 ? vals_in : vbuf[cur];
    pa.keys_out = kbuf[out];
    pa.vals_out = vbuf[out];
    pa.digit_base = hist + p * 256;
    pa.lookback = lookback;
    pa.part_counter = part_counter + p;
    pa.count_dev = count_dev;
    pa.count = count;
    pa.st = status;
    pa.passes = passes;
    pa.pass = p;
    pa.shift = 8 * p;
    pa.bits = std::max(1, std::min(8, key_bits - 8 * p));
    pa.spin_limit = spin_limit;
    pa.ranges = p == last ? ranges : nullptr;
    pa.n_tiles = n_tiles;
    pa.sorted_buf = (p == last && buf_ids) ? buf_ids[out] : 0;
    pa.out_gather = p == last ? last_gather : nullptr;
    const cudaError_t e =
        launch_pdl(onesweep_kernel<KEY>, dim3((unsigned)parts), dim3(kSortThreads), sizeof(SortSmem<KEY>), st, pa);
    if (first_error && *first_error == cudaSuccess) *first_error = e;
    count_launches(1);
    cur = out;
  }
  return cur;
}

// Phase 1: depth sort of the records, scan, key duplication (with the tile
// sort's digit histograms).
cudaError_t launch_bin_phase1(const BinArgs& a, cudaStream_t st, int sms) {
  const int64_t m = a.n * a.n_views;
  cudaError_t e;
  // status word, histograms, look-back words of both sorts and ranges start
  // at zero every frame; the last four are consecutive workspace slots, so
  // one memset clears them all
  if ((e = cudaMemsetAsync(a.ws.status, 0, offsetof(Status, d2_fresh), st)) != cudaSuccess) return e;
  {
    char* lo = reinterpret_cast<char*>(a.ws.hist);
    char* hi = reinterpret_cast<char*>(a.ws.ranges + a.total_tiles);
    if ((e = cudaMemsetAsync(lo, 0, (size_t)(hi - lo), st)) != cudaSuccess) return e;
  }
  const unsigned long long um = (unsigned long long)m;
  const unsigned long long dparts = (um + kSortPart - 1) / kSortPart;
  const uint32_t* perm = a.ws.perm[0];
  const uint32_t* cnt_sorted = a.ws.dkey[0];
  if (m > 0) {
    // depth sort of the records (values: record indices)
    // two blocks per SM (one measured slower): each bin's count goes to global
    // memory from few blocks
    launch_pdl(histogram_kernel<uint32_t>, dim3(clamp_grid((um + 255) / 256, sms, 2)), dim3(256), 0, st,
               (const uint32_t*)a.ws.dkey[0], (const unsigned long long*)nullptr, um, (int)kDepthPasses, a.ws.hist);
    launch_pdl(hist_scan_kernel, dim3(kDepthPasses), dim3(256), 0, st, a.ws.hist, a.ws.status->pass_trivial,
               (const unsigned long long*)nullptr, um);
    count_launches(2);
    uint32_t* const kb[2] = {a.ws.dkey[1], a.ws.dkey[0]};
    uint32_t* const vb[2] = {a.ws.perm[1], a.ws.perm[0]};
    // the last pass writes, in place of the sorted depth keys, the records'
    // tile counts in depth order (what the scan and the key emission read)
    const int r = run_passes<uint32_t>(a.ws.dkey[0], nullptr, kb, vb, a.ws.hist, a.ws.lookback_d,
                                       a.ws.status->part_counter, nullptr, um, dparts, kDepthPasses, 32, nullptr,
                                       a.ws.status, a.spin_limit, st, nullptr, 0, nullptr, a.ws.ntouch);
    perm = vb[r];
    cnt_sorted = kb[r];
  }
  const int nb = (int)((m + kScanBlock - 1) / kScanBlock);
  if (m > 0) {
    launch_pdl(scan_reduce_kernel, dim3(nb), dim3(kScanThreads), 0, st, cnt_sorted, m, a.ws.scan_part);
    count_launches(1);
  }
  launch_pdl(scan_parts_kernel, dim3(1), dim3(1024), 0, st, a.ws.scan_part, nb, a.ws.status, a.cap);
  count_launches(1);
  if (m > 0) {
    launch_pdl(scan_down_kernel, dim3(nb), dim3(kScanThreads), 0, st, cnt_sorted, m,
               (const unsigned long long*)a.ws.scan_part, a.ws.offsets);
    // keys and the tile sort's digit histograms
    launch_pdl(duplicate_kernel, dim3(clamp_grid((m + 255) / 256, sms, 4)), dim3(256), 0, st, a.n, a.n_views,
               (const ViewInfo*)a.ws.views, perm, cnt_sorted, (const uint32_t*)a.ws.offsets, (const uint2*)a.ws.rect,
               (const float4*)a.ws.rec, (const float4*)a.ws.foot, a.ws.keys[0], a.ws.vals[0], a.cap,
               a.ws.hist + kMaxPasses * 256, a.passes);
    count_launches(2);
  }
  if (a.passes > 0) {
    launch_pdl(hist_scan_kernel, dim3(a.passes), dim3(256), 0, st, a.ws.hist + kMaxPasses * 256,
               a.ws.status->pass_trivial + kMaxPasses, (const unsigned long long*)&a.ws.status->keys_needed, a.cap);
    count_launches(1);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Composite order: tiles by descending length of their key lists, in
// buckets of 1/2^kOrderSubBits of a power of two (empty tiles last), so the
// heaviest tiles start first and the last wave of the composites holds light
// ones.  Counters (cnt[kOrderBuckets], cursor[kOrderBuckets]) follow the
// order array and start at zero.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tile_bucket(const uint2* ranges, int64_t t) {
  const uint2 r = tile_range(ranges, t);
  const uint32_t len = r.y - r.x;
  if (!len) return kOrderBuckets - 1;
  constexpr int S = 1 << kOrderSubBits;
  const int e = 31 - __clz(len);  // floor(log2(len))
  // the kOrderSubBits bits below the leading one (zero-filled below 2^kOrderSubBits)
  const uint32_t frac = e >= kOrderSubBits ? (len >> (e - kOrderSubBits)) & (S - 1u)
                                           : (len << (kOrderSubBits - e)) & (S - 1u);
  return S * (31 - e) + S - 1 - (int)frac;  // 0 for the longest lists
}

// exclusive offsets base[b] of the bucket counts cnt[b], by a block of NT threads
template <int NT>
__device__ __forceinline__ void bucket_offsets(const uint32_t* cnt, uint32_t* base, unsigned long long* s_warp) {
  constexpr int K = (kOrderBuckets + NT - 1) / NT;
  uint32_t c[K];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int b = (int)threadIdx.x * K + k;
    c[k] = b < kOrderBuckets ? cnt[b] : 0u;
    sum += c[k];
  }
  unsigned long long total;
  unsigned long long run = block_exclusive_u64<NT>(sum, s_warp, total);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int b = (int)threadIdx.x * K + k;
    if (b < kOrderBuckets) base[b] = (uint32_t)run;
    run += c[k];
  }
}

// one block for up to kOrderOneBlock tiles: count, scan and scatter in
// shared memory
constexpr int64_t kOrderOneBlock = 16384;
__global__ void __launch_bounds__(1024) tile_order_block_kernel(const uint2* __restrict__ ranges, int64_t tiles,
                                                                uint32_t* __restrict__ order) {
  pdl_entry();
  __shared__ uint32_t s_cnt[kOrderBuckets], s_cur[kOrderBuckets];
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_cnt[b] = 0u;
  __syncthreads();
  __shared__ unsigned long long s_warp[32];
  for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) atomicAdd(&s_cnt[tile_bucket(ranges, t)], 1u);
  __syncthreads();
  bucket_offsets<1024>(s_cnt, s_cur, s_warp);
  __syncthreads();
  for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x)
    order[atomicAdd(&s_cur[tile_bucket(ranges, t)], 1u)] = (uint32_t)t;
}

__global__ void __launch_bounds__(256) tile_order_count_kernel(const uint2* __restrict__ ranges, int64_t tiles,
                                                               uint32_t* __restrict__ cnt) {
  pdl_entry();
  __shared__ uint32_t s_cnt[kOrderBuckets];
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) s_cnt[b] = 0u;
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&s_cnt[tile_bucket(ranges, t)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x)
    if (s_cnt[b]) atomicAdd(&cnt[b], s_cnt[b]);
}

__global__ void __launch_bounds__(256) tile_order_scatter_kernel(const uint2* __restrict__ ranges, int64_t tiles,
                                                                 const uint32_t* __restrict__ cnt,
                                                                 uint32_t* __restrict__ cursor,
                                                                 uint32_t* __restrict__ order) {
  pdl_entry();
  __shared__ uint32_t s_base[kOrderBuckets];
  __shared__ unsigned long long s_warp[8];
  bucket_offsets<256>(cnt, s_base, s_warp);
  __syncthreads();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = tile_bucket(ranges, t);
    order[s_base[b] + atomicAdd(&cursor[b], 1u)] = (uint32_t)t;
  }
}

// Phase 2: tile passes (run[p] != 0) and ranges.  keys_known: exact key
// count (sizes the grids), or -1 to size them for the capacity.
cudaError_t launch_bin_phase2(const BinArgs& a, const int* run, long long keys_known, cudaStream_t st) {
  const unsigned long long kn = keys_known >= 0 ? (unsigned long long)keys_known : a.cap;
  const unsigned long long parts = (kn + kSortPart - 1) / kSortPart;
  cudaError_t e;
  int r = -1;  // buffer of kb/vb holding the sorted result, -1: no pass ran
  if (parts > 0 && a.passes > 0) {  // look-back words zeroed by phase 1
    uint32_t* const kb[2] = {a.ws.keys[1], a.ws.keys[0]};
    uint32_t* const vb[2] = {a.ws.vals[1], a.ws.vals[0]};
    const int ws_index[2] = {1, 0};  // kb[i] is ws.keys[ws_index[i]]
    // the last pass also reduces the tile ranges and records the buffer
    r = run_passes<uint32_t>(a.ws.keys[0], a.ws.vals[0], kb, vb, a.ws.hist + kMaxPasses * 256, a.ws.lookback,
                             a.ws.status->part_counter + kMaxPasses, &a.ws.status->keys_needed, a.cap, parts,
                             a.passes, a.tile_bits, run, a.ws.status, a.spin_limit, st, a.ws.ranges,
                             (unsigned long long)a.total_tiles, ws_index);
  }
  if (r < 0) {  // no pass ran (one tile, or every pass trivial): ranges from the unsorted-equals-sorted keys
    const unsigned grid = (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>((kn + 255) / 256,
                                                                                                 1ull << 20));
    ranges_kernel<<<grid, 256, 0, st>>>(a.ws.keys[0], a.ws.status, a.cap, a.ws.ranges, 0);
    count_launches(1);
  }
  // composite order of the tiles
  if (a.total_tiles <= kOrderOneBlock) {
    launch_pdl(tile_order_block_kernel, dim3(1), dim3(1024), 0, st, (const uint2*)a.ws.ranges, a.total_tiles,
               a.ws.tile_order);
    count_launches(1);
  } else {
    uint32_t* counters = a.ws.tile_order + a.total_tiles;
    if ((e = cudaMemsetAsync(counters, 0, sizeof(uint32_t) * 2 * kOrderBuckets, st)) != cudaSuccess) return e;
    const unsigned tgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((a.total_tiles + 255) / 256, 1024));
    launch_pdl(tile_order_count_kernel, dim3(tgrid), dim3(256), 0, st, (const uint2*)a.ws.ranges, a.total_tiles,
               counters);
    launch_pdl(tile_order_scatter_kernel, dim3(tgrid), dim3(256), 0, st, (const uint2*)a.ws.ranges, a.total_tiles,
               (const uint32_t*)counters, counters + kOrderBuckets, a.ws.tile_order);
    count_launches(2);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The status word into mapped host memory (the synchronous key-count readback)
// ---------------------------------------------------------------------------
__global__ void status_export_kernel(const Status* __restrict__ src, Status* dst) {
  pdl_entry();
  constexpr int kWords = (int)(sizeof(Status) / sizeof(uint32_t));
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < kWords; i += blockDim.x) d[i] = s[i];
  __threadfence_system();
}

cudaError_t launch_status_export(const Status* src, Status* dst_mapped, cudaStream_t st) {
  static_assert(sizeof(Status) % sizeof(uint32_t) == 0, "status word size");
  launch_pdl(status_export_kernel, dim3(1), dim3(32), 0, st, src, dst_mapped);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bounded-wait self-test: one onesweep pass over zero keys in which partition
// ticket 0 is skipped, so partition 1 waits for a look-back word that nothing
// writes.  The wait must give up after spin_limit polls, raise the timeout
// flag and still publish, so the pass ends and the context stays usable.
// ---------------------------------------------------------------------------
__global__ void selftest_setup_kernel(Status* st, unsigned long long n, uint32_t* digit_base) {
  if (threadIdx.x == 0) {
    st->keys_needed = n;
    st->part_counter[kMaxPasses] = 1u;  // nobody takes partition 0
  }
  for (int d = threadIdx.x; d < 256; d += blockDim.x) digit_base[d] = d == 0 ? 0u : (uint32_t)n;
}

cudaError_t launch_selftest_bounded_wait(const Ws& ws, unsigned long long cap, int spin_limit, cudaStream_t st) {
  const unsigned long long n = 4ull * kSortPart < cap ? 4ull * kSortPart : cap;
  const unsigned long long parts = (n + kSortPart - 1) / kSortPart;
  cudaError_t e;
  if ((e = cudaMemsetAsync(ws.status, 0, sizeof(Status), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.keys[0], 0, sizeof(uint32_t) * n, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ws.lookback, 0, sizeof(unsigned long long) * 256 * parts, st)) != cudaSuccess) return e;
  uint32_t* th = ws.hist + kMaxPasses * 256;
  selftest_setup_kernel<<<1, 256, 0, st>>>(ws.status, n, th);
  uint32_t* const kb[2] = {ws.keys[1], ws.keys[0]};
  uint32_t* const vb[2] = {ws.vals[1], ws.vals[0]};
  count_launches(1);
  run_passes<uint32_t>(ws.keys[0], nullptr, kb, vb, th, ws.lookback, ws.status->part_counter + kMaxPasses, nullptr,
                       n, parts, 1, 8, nullptr, ws.status, spin_limit, st);
  return cudaGetLastError();
}

}  // namespace sr

// ---------------------------------------------------------------------------
// Sort without caller-provided scratch (sr_sort_keys_noalloc)
//
// For callers that cannot allocate device memory at all (a host-side runtime
// that owns a fixed memory pool, a plugin that only receives its input and
// output buffers, code running where a cudaMalloc would break a frame-time
// budget or an allocation-free guarantee).  All scratch of the radix sort
// (one ping-pong key/value buffer, the digit histograms, the look-back state
// and the status word) lives in one file-scope device array of fixed size,
// so the call allocates nothing; every GPU that loads this library holds the
// array (about 16 MiB) until the process exits.
// ---------------------------------------------------------------------------
namespace sr {

constexpr unsigned long long kNoallocKeys = 1ull << 20;  // == SR_NOALLOC_MAX_KEYS
constexpr unsigned long long kNoallocParts = kNoallocKeys / kSortPart;
constexpr size_t kNoallocStatusBytes = 256;
constexpr size_t kNoallocHistBytes = sizeof(uint32_t) * kMaxPasses * 256;
constexpr size_t kNoallocLookbackBytes = sizeof(unsigned long long) * 256 * kMaxPasses * kNoallocParts;
constexpr size_t kNoallocKeyBytes = sizeof(unsigned long long) * kNoallocKeys;
constexpr size_t kNoallocValBytes = sizeof(uint32_t) * kNoallocKeys;
constexpr size_t kNoallocBytes =
    kNoallocStatusBytes + kNoallocHistBytes + kNoallocLookbackBytes + kNoallocKeyBytes + kNoallocValBytes;
static_assert(sizeof(Status) <= kNoallocStatusBytes, "status word does not fit");

// Host code must not use this name as a device address; it receives the
// address from cudaGetSymbolAddress (see noalloc_scratch_address below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Clears what the sort expects at zero and records the key count.
__global__ void noalloc_reset_kernel(unsigned char* scratch, unsigned long long n, int passes) {
  Status* st = reinterpret_cast<Status*>(scratch);
  uint32_t* hist = reinterpret_cast<uint32_t*>(scratch + kNoallocStatusBytes);
  unsigned long long* lb =
      reinterpret_cast<unsigned long long*>(scratch + kNoallocStatusBytes + kNoallocHistBytes);
  const unsigned long long parts = (n + kSortPart - 1) / kSortPart;
  const unsigned long long lb_words = parts * (unsigned long long)passes * 256ull;
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = tid; i < lb_words; i += stride) lb[i] = 0ull;
  for (unsigned long long i = tid; i < (unsigned long long)kMaxPasses * 256; i += stride) hist[i] = 0u;
  if (tid == 0) {
    st->flags = 0u;
    st->sorted_buf = 0u;
    st->keys_needed = n;
    for (int p = 0; p < 2 * kMaxPasses; ++p) {
      st->part_counter[p] = 0u;
      st->pass_trivial[p] = 0u;
    }
    st->timeout_where = 0u;
  }
}

// Device address of the scratch array on the current device, looked up on
// every call (a cudaDeviceReset reloads the module, which can move it).
static unsigned char* noalloc_scratch_address(cudaError_t* err) {
  void* p = nullptr;
  *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  return *err == cudaSuccess ? static_cast<unsigned char*>(p) : nullptr;
}

}  // namespace sr

extern "C" sr_status sr_sort_keys_noalloc(const uint64_t* keys_in, const uint32_t* vals_in, int64_t n,
                                          int32_t sort_bits, uint64_t* keys_out, uint32_t* vals_out,
                                          void* stream) {
  using namespace sr;
  typedef unsigned long long u64;
  if (n < 0 || sort_bits < 1 || sort_bits > 64) return SR_ERR_INVALID;
  if ((u64)n > kNoallocKeys) return SR_ERR_CAPACITY;
  if (n == 0) return SR_OK;
  if (!keys_in || !vals_in || !keys_out || !vals_out) return SR_ERR_INVALID;
  if ((const void*)keys_in == (const void*)keys_out || vals_in == vals_out) return SR_ERR_INVALID;
  cudaError_t e;
  unsigned char* base = noalloc_scratch_address(&e);
  if (!base) return SR_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int passes = (sort_bits + 7) / 8;
  const u64 un = (u64)n;
  Status* status = reinterpret_cast<Status*>(base);
  uint32_t* hist = reinterpret_cast<uint32_t*>(base + kNoallocStatusBytes);
  u64* lookback = reinterpret_cast<u64*>(base + kNoallocStatusBytes + kNoallocHistBytes);
  u64* tmp_keys = reinterpret_cast<u64*>(base + kNoallocStatusBytes + kNoallocHistBytes + kNoallocLookbackBytes);
  uint32_t* tmp_vals = reinterpret_cast<uint32_t*>(base + kNoallocStatusBytes + kNoallocHistBytes +
                                                   kNoallocLookbackBytes + kNoallocKeyBytes);
  // each launch's own result decides SR_ERR_CUDA (no cudaGetLastError, which
  // would report, and clear, an error some earlier call left behind)
  e = launch_plain(noalloc_reset_kernel, dim3(clamp_grid((un * passes + 255) / 256, sms, 4)), dim3(256), 0, st, base,
                   un, passes);
  if (e == cudaSuccess)
    e = launch_pdl(histogram_kernel<u64>, dim3(clamp_grid((un + 255) / 256, sms, 4)), dim3(256), 0, st,
                   reinterpret_cast<const u64*>(keys_in), (const unsigned long long*)nullptr, un, passes, hist);
  if (e == cudaSuccess)
    e = launch_pdl(hist_scan_kernel, dim3(passes), dim3(256), 0, st, hist, status->pass_trivial,
                   (const unsigned long long*)nullptr, un);
  count_launches(3);
  if (e != cudaSuccess) return SR_ERR_CUDA;
  // ping-pong between the scratch buffer and the output so that the last pass
  // writes the output: an odd pass count starts into the output
  u64* const kb[2] = {(passes & 1) ? reinterpret_cast<u64*>(keys_out) : tmp_keys,
                      (passes & 1) ? tmp_keys : reinterpret_cast<u64*>(keys_out)};
  uint32_t* const vb[2] = {(passes & 1) ? vals_out : tmp_vals, (passes & 1) ? tmp_vals : vals_out};
  const u64 parts = (un + kSortPart - 1) / kSortPart;
  run_passes<u64>(reinterpret_cast<const u64*>(keys_in), vals_in, kb, vb, hist, lookback, status->part_counter,
                  nullptr, un, parts, passes, 8 * passes, nullptr, status, 1 << 20, st, nullptr, 0, nullptr, nullptr,
                  &e);
  if (e != cudaSuccess) return SR_ERR_CUDA;
  // the status word: a look-back wait that gave up leaves the output unsorted
  uint32_t flags = 0u;
  if (cudaMemcpyAsync(&flags, &status->flags, sizeof(flags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SR_ERR_CUDA;
  if (flags & kStatusTimeout) return SR_ERR_TIMEOUT;
  return SR_OK;
}
