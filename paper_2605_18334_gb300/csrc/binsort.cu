// Tile binning and depth sort (the tile-based, depth-sorted pipeline of the
// Preliminaries).  The result is the order of the key (global tile << 32 |
// FP32 depth bits) with ties broken by record index, obtained in two sorts:
//
//   depth sort   the M records by their 32-bit depth key (records that touch
//                no tile carry ~0 and sink to the end): 4 stable 8-bit passes
//                over M, not over the (much larger) number of tile keys
//   scan         exclusive scan of the tile counts in depth order
//   duplicate    one 32-bit global tile id per touched tile, value = record
//                index, emitted in depth order (warp-cooperative, coalesced)
//   tile sort    stable LSD passes over the tile-id bits only; stability
//                keeps the depth order (and index order of equal depths)
//                inside every tile
//   ranges       [start, end) of each tile in the sorted list
//
// Every radix pass is one onesweep launch: a block ranks a partition of 4096
// keys with warp match-any, publishes its digit counts, resolves its global
// offsets by a decoupled look-back over the preceding partitions (each wait
// bounded), and scatters through shared memory so writes go out in runs.
#include <algorithm>
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
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t* __restrict__ cnt,
                                                                   const uint32_t* __restrict__ perm, int64_t m,
                                                                   unsigned long long* __restrict__ part) {
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < m) sum += cnt[perm[base + k]];
  unsigned long long total;
  block_exclusive_u64<kScanThreads>(sum, s_warp, total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_parts_kernel(unsigned long long* part, int nb, Status* st,
                                                          unsigned long long cap) {
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

__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const uint32_t* __restrict__ cnt,
                                                                 const uint32_t* __restrict__ perm, int64_t m,
                                                                 const unsigned long long* __restrict__ part,
                                                                 uint32_t* __restrict__ offsets) {
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < m ? cnt[perm[base + k]] : 0u;
    sum += v[k];
  }
  unsigned long long total;
  unsigned long long run = block_exclusive_u64<kScanThreads>(sum, s_warp, total) + part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < m) offsets[base + k] = run > 0xffffffffull ? 0xffffffffu : (uint32_t)run;
    run += v[k];
  }
}

// ---------------------------------------------------------------------------
// key duplication, in depth order.  A warp takes 32 consecutive depth-sorted
// records and writes their keys as one contiguous run: each lane finds the
// record owning its output slot by a binary search over the lanes' starts
// and decodes the slot's tile from the owner's packed row spans (coalesced
// writes).  Records whose tile box is too large for packed spans are written
// afterwards by their own lane, row by row (row_tile_span).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) duplicate_kernel(int64_t n, int n_views, const ViewInfo* __restrict__ views,
                                                        const uint32_t* __restrict__ perm,
                                                        const uint32_t* __restrict__ ntouch,
                                                        const uint32_t* __restrict__ offsets,
                                                        const uint2* __restrict__ rect,
                                                        const float4* __restrict__ rec,
                                                        const float4* __restrict__ foot,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        unsigned long long cap) {
  const int64_t m_total = n * n_views;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w * 32 < m_total; w += warps) {
    const int64_t j = w * 32 + lane;
    uint32_t m = 0, cnt = 0, start = 0xffffffffu, tx0 = 0, ty0 = 0, sp0 = 0, sp1 = 0;
    uint32_t row0 = 0, tiles_x = 0;  // global tile id of (0, ty0) and the view's tiles per row
    bool tall = false;
    ViewInfo vi;
    if (j < m_total) {
      m = perm[j];
      cnt = ntouch[m];
      start = offsets[j];
      if (cnt) {
        const uint2 r = rect[m];
        tx0 = r.x & 0xffffu;
        ty0 = r.x >> 16;
        const float4 f1 = foot[2 * (int64_t)m + 1];
        sp0 = __float_as_uint(f1.z);
        sp1 = __float_as_uint(f1.w);
        tall = sp0 == kSpansTall;
        vi = views[(int)(m / (uint64_t)n)];
        tiles_x = (uint32_t)vi.tiles_x;
        row0 = (uint32_t)(vi.tile_base + (int64_t)ty0 * vi.tiles_x);
      }
    }
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
      int lo = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t s_rel = __shfl_sync(0xffffffffu, rel, lo + step);
        if (s_rel <= q_rel) lo += step;
      }
      const uint32_t o_rel = __shfl_sync(0xffffffffu, rel, lo);
      const uint32_t o_m = __shfl_sync(0xffffffffu, m, lo);
      const uint32_t o_sp0 = __shfl_sync(0xffffffffu, sp0, lo);
      const uint32_t o_sp1 = __shfl_sync(0xffffffffu, sp1, lo);
      const uint32_t o_tx0 = __shfl_sync(0xffffffffu, tx0, lo);
      const uint32_t o_row0 = __shfl_sync(0xffffffffu, row0, lo);
      const uint32_t o_tx = __shfl_sync(0xffffffffu, tiles_x, lo);
      if (p >= end || o_sp0 == kSpansTall) continue;
      // decode the row of the q-th key from the packed spans
      uint32_t q = q_rel - o_rel, key = 0;
      bool found = false;
#pragma unroll
      for (int rr = 0; rr < kSpanRows; ++rr) {
        const uint32_t word = (rr < 2 ? o_sp0 : o_sp1) >> (16 * (rr & 1));
        const uint32_t first = word & 0xffu, num = (word >> 8) & 0xffu;
        if (!found && q < num) {
          key = o_row0 + (uint32_t)rr * o_tx + o_tx0 + first + q;
          found = true;
        }
        if (!found) q -= num;
      }
      if (found && p < cap) {
        keys[p] = key;
        vals[p] = o_m;
      }
    }
    if (tall && cnt) {
      const uint2 r = rect[m];
      const int ty1 = (int)(r.y >> 16);
      const float4 f0 = foot[2 * (int64_t)m], f1 = foot[2 * (int64_t)m + 1];
      const float4 r0 = rec[4 * (int64_t)m];
      unsigned long long pos = start;
      const unsigned long long stop = pos + cnt;
      for (int ty = (int)ty0; ty < ty1; ++ty) {
        int lo, hi;
        if (!row_tile_span(f0, f1, r0.x, r0.y, ty, vi.width, vi.height, lo, hi)) continue;
        const uint32_t row = (uint32_t)(vi.tile_base + (int64_t)ty * vi.tiles_x);
        for (int tx = lo; tx <= hi; ++tx, ++pos)
          if (pos < stop && pos < cap) {
            keys[pos] = row + (uint32_t)tx;
            vals[pos] = m;
          }
      }
    }
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
  __shared__ uint32_t s_h[kMaxPasses][256];
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += blockDim.x) (&s_h[0][0])[i] = 0u;
  __syncthreads();
  const unsigned long long kn = element_count(count_dev, count);
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < kn;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[k];
    for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][(key >> (8 * p)) & 0xffu], 1u);
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
  unsigned long long* lookback;   // [parts][passes][256], zeroed per frame
  uint32_t* part_counter;         // partition tickets of this pass (zeroed)
  const unsigned long long* count_dev;  // element count on the device, or nullptr
  unsigned long long count;       // element count (count_dev == nullptr) or the capacity bound
  Status* st;                     // status flags (timeouts)
  int passes;
  int pass;
  int shift;
  int spin_limit;
};

template <class KEY>
__global__ void __launch_bounds__(kSortThreads, 4) onesweep_kernel(PassArgs<KEY> a) {
  constexpr int NW = kSortThreads / 32;
  __shared__ KEY s_buf[kSortPart];  // keys, then values (as u32) in the scatter phase
  __shared__ uint32_t s_whist[NW][256];
  __shared__ uint32_t s_lstart[256];
  __shared__ unsigned long long s_gbase[256];
  __shared__ unsigned long long s_warp[NW];
  __shared__ uint8_t s_dig[kSortPart];
  __shared__ uint32_t s_part;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long kn = element_count(a.count_dev, a.count);
  const unsigned long long nparts = (kn + kSortPart - 1) / kSortPart;
  if (tid == 0) s_part = atomicAdd(a.part_counter, 1u);
  for (int i = tid; i < NW * 256; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
  __syncthreads();
  const unsigned long long part = s_part;
  if (part >= nparts) return;
  const unsigned long long base = part * kSortPart;

  // load, warp-blocked: warp w owns keys [w*512, (w+1)*512) of the partition
  KEY key[kSortItems];
  uint32_t rank[kSortItems];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const unsigned long long idx = base + (unsigned long long)warp * (32 * kSortItems) + j * 32 + lane;
    const bool valid = idx < kn;
    key[j] = valid ? a.keys_in[idx] : (KEY)~(KEY)0;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const uint32_t d = (uint32_t)(key[j] >> a.shift) & 0xffu;
      const uint32_t peers = __match_any_sync(vmask, d);
      const uint32_t prev = s_whist[warp][d];
      __syncwarp(vmask);
      if ((peers & lt) == 0) s_whist[warp][d] = prev + __popc(peers);
      __syncwarp(vmask);
      rank[j] = prev + __popc(peers & lt);
    } else {
      rank[j] = 0u;
    }
    __syncwarp();
  }
  __syncthreads();

  // per digit: counts across warps -> warp offsets; publish and look back
  const int d = tid;  // kSortThreads == 256 digits
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const uint32_t c = s_whist[w][d];
    s_whist[w][d] = tot;
    tot += c;
  }
  unsigned long long* lb = a.lookback + (part * a.passes + a.pass) * 256;
  st_relaxed_u64(lb + d, (part == 0 ? kFlagInc : kFlagAgg) | tot);
  unsigned long long excl = 0;
  if (part > 0) {
    // walk back over the predecessors' words of this digit, four loads in
    // flight at a time: aggregates are summed, an inclusive prefix ends the
    // walk, a word not yet published is polled again (at most spin_limit times)
    constexpr int kWin = 4;
    const unsigned long long stride = (unsigned long long)a.passes * 256;
    const unsigned long long* col = a.lookback + (unsigned long long)a.pass * 256 + d;
    long long q = (long long)part - 1;
    int spins = 0;
    bool walking = true;
    while (walking) {
      unsigned long long w[kWin];
#pragma unroll
      for (int k = 0; k < kWin; ++k) w[k] = q - k >= 0 ? ld_relaxed_u64(col + (unsigned long long)(q - k) * stride) : 0ull;
      bool stalled = false;
#pragma unroll
      for (int k = 0; k < kWin; ++k) {
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
  s_gbase[d] = (unsigned long long)a.digit_base[d] + excl;

  // local digit starts (exclusive scan of tot over digits)
  unsigned long long total;
  s_lstart[d] = (uint32_t)block_exclusive_u64<kSortThreads>(tot, s_warp, total);
  __syncthreads();

  // local positions, keys through shared memory
  uint32_t lpos[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const unsigned long long idx = base + (unsigned long long)warp * (32 * kSortItems) + j * 32 + lane;
    if (idx < kn) {
      const uint32_t dg = (uint32_t)(key[j] >> a.shift) & 0xffu;
      lpos[j] = s_lstart[dg] + s_whist[warp][dg] + rank[j];
      s_buf[lpos[j]] = key[j];
    }
  }
  __syncthreads();
  const uint32_t count = (uint32_t)((kn - base) < (unsigned long long)kSortPart ? (kn - base) : kSortPart);
  for (uint32_t i = tid; i < count; i += kSortThreads) {
    const KEY k = s_buf[i];
    const uint32_t dg = (uint32_t)(k >> a.shift) & 0xffu;
    s_dig[i] = (uint8_t)dg;
    const unsigned long long g = s_gbase[dg] + (i - s_lstart[dg]);
    if (g < kn) a.keys_out[g] = k;  // always true unless a look-back gave up
  }
  __syncthreads();
  uint32_t* s_val = reinterpret_cast<uint32_t*>(s_buf);
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    const unsigned long long idx = base + (unsigned long long)warp * (32 * kSortItems) + j * 32 + lane;
    if (idx < kn) s_val[lpos[j]] = a.vals_in ? a.vals_in[idx] : (uint32_t)idx;
  }
  __syncthreads();
  for (uint32_t i = tid; i < count; i += kSortThreads) {
    const uint32_t dg = s_dig[i];
    const unsigned long long g = s_gbase[dg] + (i - s_lstart[dg]);
    if (g < kn) a.vals_out[g] = s_val[i];
  }
}

// ---------------------------------------------------------------------------
// tile ranges
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ranges_kernel(const uint32_t* __restrict__ keys, Status* st,
                                                     unsigned long long cap, uint2* __restrict__ ranges,
                                                     int sorted_buf) {
  const unsigned long long kn = element_count(&st->keys_needed, cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->sorted_buf = (uint32_t)sorted_buf;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < kn;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t t = keys[k];
    if (k == 0 || keys[k - 1] != t) ranges[t].x = (uint32_t)k;
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
                      int passes, const int* run, Status* status, int spin_limit, cudaStream_t st) {
  int cur = -1;  // -1: still the input
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
    pa.spin_limit = spin_limit;
    onesweep_kernel<KEY><<<(unsigned)parts, kSortThreads, 0, st>>>(pa);
    count_launches(1);
    cur = out;
  }
  return cur;
}

// Phase 1: depth sort of the records, scan, duplicate, tile histograms.
cudaError_t launch_bin_phase1(const BinArgs& a, cudaStream_t st, int sms) {
  const int64_t m = a.n * a.n_views;
  cudaError_t e;
  // status word, histograms and ranges start at zero every frame
  if ((e = cudaMemsetAsync(a.ws.status, 0, sizeof(Status), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.ws.hist, 0, sizeof(uint32_t) * 2 * kMaxPasses * 256, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.ws.ranges, 0, sizeof(uint2) * a.total_tiles, st)) != cudaSuccess) return e;
  const unsigned long long um = (unsigned long long)m;
  const unsigned long long dparts = (um + kSortPart - 1) / kSortPart;
  const uint32_t* perm = a.ws.perm[0];
  if (m > 0) {
    if ((e = cudaMemsetAsync(a.ws.lookback_d, 0, sizeof(unsigned long long) * 256 * kDepthPasses * dparts, st)) !=
        cudaSuccess)
      return e;
    // depth sort of the records (values: record indices)
    histogram_kernel<uint32_t><<<clamp_grid((um + 255) / 256, sms, 4), 256, 0, st>>>(a.ws.dkey[0], nullptr, um,
                                                                                      kDepthPasses, a.ws.hist);
    hist_scan_kernel<<<kDepthPasses, 256, 0, st>>>(a.ws.hist, a.ws.status->pass_trivial, nullptr, um);
    count_launches(2);
    uint32_t* const kb[2] = {a.ws.dkey[1], a.ws.dkey[0]};
    uint32_t* const vb[2] = {a.ws.perm[1], a.ws.perm[0]};
    const int r = run_passes<uint32_t>(a.ws.dkey[0], nullptr, kb, vb, a.ws.hist, a.ws.lookback_d,
                                       a.ws.status->part_counter, nullptr, um, dparts, kDepthPasses, nullptr,
                                       a.ws.status, a.spin_limit, st);
    perm = vb[r];
  }
  const int nb = (int)((m + kScanBlock - 1) / kScanBlock);
  if (m > 0) {
    scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(a.ws.ntouch, perm, m, a.ws.scan_part);
    count_launches(1);
  }
  scan_parts_kernel<<<1, 1024, 0, st>>>(a.ws.scan_part, nb, a.ws.status, a.cap);
  count_launches(1);
  if (m > 0) {
    scan_down_kernel<<<nb, kScanThreads, 0, st>>>(a.ws.ntouch, perm, m, a.ws.scan_part, a.ws.offsets);
    duplicate_kernel<<<clamp_grid((m + 255) / 256, sms, 8), 256, 0, st>>>(
        a.n, a.n_views, a.ws.views, perm, a.ws.ntouch, a.ws.offsets, a.ws.rect, a.ws.rec, a.ws.foot, a.ws.keys[0],
        a.ws.vals[0], a.cap);
    count_launches(2);
  }
  if (a.passes > 0) {
    uint32_t* th = a.ws.hist + kMaxPasses * 256;
    histogram_kernel<uint32_t><<<clamp_grid((a.cap + 255) / 256, sms, 4), 256, 0, st>>>(
        a.ws.keys[0], &a.ws.status->keys_needed, a.cap, a.passes, th);
    hist_scan_kernel<<<a.passes, 256, 0, st>>>(th, a.ws.status->pass_trivial + kMaxPasses,
                                               &a.ws.status->keys_needed, a.cap);
    count_launches(2);
  }
  return cudaGetLastError();
}

// Phase 2: tile passes (run[p] != 0) and ranges.  keys_known: exact key
// count (sizes the grids), or -1 to size them for the capacity.
cudaError_t launch_bin_phase2(const BinArgs& a, const int* run, long long keys_known, cudaStream_t st) {
  const unsigned long long kn = keys_known >= 0 ? (unsigned long long)keys_known : a.cap;
  const unsigned long long parts = (kn + kSortPart - 1) / kSortPart;
  cudaError_t e;
  int cur = 0;  // index into ws.keys / ws.vals of the sorted result
  if (parts > 0 && a.passes > 0) {
    if ((e = cudaMemsetAsync(a.ws.lookback, 0, sizeof(unsigned long long) * 256 * a.passes * parts, st)) !=
        cudaSuccess)
      return e;
    uint32_t* const kb[2] = {a.ws.keys[1], a.ws.keys[0]};
    uint32_t* const vb[2] = {a.ws.vals[1], a.ws.vals[0]};
    const int r = run_passes<uint32_t>(a.ws.keys[0], a.ws.vals[0], kb, vb, a.ws.hist + kMaxPasses * 256,
                                       a.ws.lookback, a.ws.status->part_counter + kMaxPasses,
                                       &a.ws.status->keys_needed, a.cap, parts, a.passes, run, a.ws.status,
                                       a.spin_limit, st);
    cur = r < 0 ? 0 : (r == 0 ? 1 : 0);  // kb[0] is ws.keys[1]
  }
  const unsigned grid = (unsigned)std::max<unsigned long long>(1, std::min<unsigned long long>((kn + 255) / 256,
                                                                                               1ull << 20));
  ranges_kernel<<<grid, 256, 0, st>>>(a.ws.keys[cur], a.ws.status, a.cap, a.ws.ranges, cur);
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
                       n, parts, 1, nullptr, ws.status, spin_limit, st);
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
// array (about 16.2 MiB) until the process exits.
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

// Device address of the scratch array for the current device, looked up once
// per device (the first call on a device does it).
static unsigned char* noalloc_scratch_address(cudaError_t* err) {
  static std::mutex mu;
  static unsigned char* addr[64] = {nullptr};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    addr[dev] = static_cast<unsigned char*>(p);
  }
  return addr[dev];
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
  noalloc_reset_kernel<<<clamp_grid((un * passes + 255) / 256, sms, 4), 256, 0, st>>>(base, un, passes);
  histogram_kernel<u64><<<clamp_grid((un + 255) / 256, sms, 4), 256, 0, st>>>(
      reinterpret_cast<const u64*>(keys_in), nullptr, un, passes, hist);
  hist_scan_kernel<<<passes, 256, 0, st>>>(hist, status->pass_trivial, nullptr, un);
  // ping-pong between the scratch buffer and the output so that the last pass
  // writes the output: an odd pass count starts into the output
  u64* const kb[2] = {(passes & 1) ? reinterpret_cast<u64*>(keys_out) : tmp_keys,
                      (passes & 1) ? tmp_keys : reinterpret_cast<u64*>(keys_out)};
  uint32_t* const vb[2] = {(passes & 1) ? vals_out : tmp_vals, (passes & 1) ? tmp_vals : vals_out};
  const u64 parts = (un + kSortPart - 1) / kSortPart;
  run_passes<u64>(reinterpret_cast<const u64*>(keys_in), vals_in, kb, vb, hist, lookback, status->part_counter,
                  nullptr, un, parts, passes, nullptr, status, 1 << 20, st);
  count_launches(3);
  return cudaGetLastError() == cudaSuccess ? SR_OK : SR_ERR_CUDA;
}
