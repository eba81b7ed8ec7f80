// Per-tile compositing of skew Gaussians: forward (Alg. 1, Eq. color) and
// the reverse replay that differentiates it (Alg. 2).
//
// One block per 16x16 tile (or, in persistent launches, blocks that take
// tile after tile from a counter); each thread owns PX vertically adjacent pixels
// of one column, so a warp covers an 8-wide block of 4*PX rows.  The tile's
// depth-sorted records are staged into shared memory in batches (128, 256 or
// 512 gathered 64-byte records), then every pixel walks the batch:
//   alpha = min(alpha_max, o G' (1 + erf z)),  skip if alpha < alpha_min,
//   stop before the Gaussian whose T' = T (1 - alpha) would fall below t_stop,
//   C += c alpha T, T = T'.
// A block leaves as soon as every pixel has stopped (__syncthreads_count).
// With an even PX a thread takes its rows two at a time: they share dx, and
// the packed FP32x2 instructions of sm_100+ evaluate and blend both in one
// instruction stream, with results equal to the scalar path bit for bit.
//
// Backward per pixel from its last blended Gaussian down: T_k = T_{k+1} /
// (1 - alpha_k), R_{k+1} = colour behind k normalised by T_{k+1} (the
// background included), dL/dalpha_k = T_k sum_c g_c (c_k,c - R_{k+1},c).
// A thread first sums its PX pixels' contributions to a Gaussian, the warp
// then sums its lanes with a transposing butterfly, warps add into padded
// shared-memory accumulators, and each block issues one set of vector atomics
// per Gaussian per batch.  Which positions a pixel blended comes from the
// forward's blend masks, or, in plans that keep none, from re-evaluating
// the alpha gate at every position below the pixel's n_contrib (the stop
// cannot occur there), as Alg. 2 does.
#include <algorithm>

#include "kernels.cuh"

namespace sr {


struct TileCoord {
  ViewInfo vi;
  int tx, ty;
};

__device__ __forceinline__ TileCoord tile_coord(const RenderArgs& a, int64_t tile) {
  TileCoord t;
  const int v = view_of_tile(a.views, a.n_views, tile);
  t.vi = a.views[v];
  const int lt = (int)(tile - t.vi.tile_base);
  t.tx = lt % t.vi.tiles_x;
  t.ty = lt / t.vi.tiles_x;
  return t;
}

// Pixels of a thread: PX vertically adjacent pixels of one column.  A warp
// covers an 8-wide block of 4*PX rows (2 warps across the tile), more compact
// than a 16-wide strip, so fewer of its lanes sit outside a Gaussian that
// touches it.  pi0: index in the tile of the thread's first pixel (row-major).
struct PixelMap {
  int px, py0, pi0;
};
template <int PX>
__device__ __forceinline__ PixelMap pixel_map(const TileCoord& tc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = (warp & 1) * 8 + (lane & 7);
  const int ly = (warp >> 1) * 4 * PX + (lane >> 3) * PX;
  PixelMap m;
  m.px = tc.tx * kTile + lx;
  m.py0 = tc.ty * kTile + ly;
  m.pi0 = ly * kTile + lx;
  return m;
}

template <int MODE, int BATCH>
__device__ __forceinline__ void stage_batch(const RenderArgs& a, const uint32_t* vals, uint32_t start, uint32_t end,
                                            int nt, float4* s_r0, float4* s_r1, float4* s_r2, float4* s_r3,
                                            uint32_t* s_id) {
  for (int q = threadIdx.x; q < BATCH; q += nt) {
    const uint32_t idx = start + q;
    if (idx < end) {
      const uint32_t id = vals[idx];
      const float4* r = a.rec + 4 * (int64_t)id;
      if (s_id) s_id[q] = id;
      s_r0[q] = r[0];
      s_r1[q] = r[1];
      if (MODE != MODE_PLAIN) s_r2[q] = r[2];
      s_r3[q] = r[3];
    }
  }
}

// Blend masks.  For the backward pass the forward records, per pixel, which
// positions of its tile's sorted list it blended: one bit per position, a
// 32-bit word per 32 positions (chunk c covers positions range.x + 32c ..).
// Tile t's words start at chunk floor(range.x / 32) + t, which never overlaps
// the next tile's, and the 256 pixels' words of one chunk are consecutive,
// so the stores of a warp are coalesced.  A pixel writes every word up to the
// one holding its stop; the backward reads only words below its last blend.
__device__ __forceinline__ uint32_t* mask_tile_base(uint32_t* mask, uint2 range, int64_t tile) {
  return mask + ((int64_t)(range.x >> 5) + tile) * 256;
}

// Persistent launches: a block takes tile after tile of the composite order
// from a counter (zeroed before the launch) until none is left.
__device__ __forceinline__ uint32_t next_work(uint32_t* counter, uint32_t* s_next) {
  __syncthreads();  // the block is done with the previous tile and with *s_next
  if (threadIdx.x == 0) *s_next = atomicAdd(counter, 1u);
  __syncthreads();
  return *s_next;
}

// a finished 32-position blend word: its blends are counted and its highest
// bit is the pixel's last contributor so far (list position + 1)
__device__ __forceinline__ void credit(uint32_t w, uint32_t cbase, uint32_t& blended, uint32_t& last) {
  if (w) {
    blended += __popc(w);
    last = cbase + 32u - __clz(w);
  }
}

// occupancy target of the forward composite: 5 blocks of 256 threads per SM
// for one pixel per thread (<= 51 registers), the compiler's choice otherwise
template <int PX>
struct FwdMinBlocks {
  static constexpr int value = PX == 1 ? 5 : 1;
};

template <int MODE, int PX, bool REC, int BATCH, bool PERSIST>
__global__ void __launch_bounds__(256 / PX, FwdMinBlocks<PX>::value) render_fwd_kernel(RenderArgs a) {
  pdl_entry();
  constexpr int NT = 256 / PX;
  __shared__ float4 s_r0[BATCH], s_r1[BATCH], s_r2[MODE == MODE_PLAIN ? 1 : BATCH], s_r3[BATCH];
  __shared__ uint32_t s_next;
  // one tile of the composite order; a persistent block takes tile after tile
  auto tile_body = [&](uint32_t it) {
    const int64_t tile = a.tile_order[it];
    const TileCoord tc = tile_coord(a, tile);
    const PixelMap pm = pixel_map<PX>(tc);
    const int px = pm.px, py0 = pm.py0, pi0 = pm.pi0;
    const float fx = (float)px + 0.5f;
    const uint2 range = tile_range(a.ranges, tile);
    const uint32_t* vals = a.status->sorted_buf ? a.vals1 : a.vals0;
    const float amin = a.cfg.alpha_min, amax = a.cfg.alpha_max, tstop = a.cfg.t_stop;
    uint32_t* mbase = REC ? mask_tile_base(a.mask, range, tile) : nullptr;

    // colour state: scalar, or (even PX) packed per pair of rows for FP32x2 arithmetic
    constexpr bool PACKED = PX % 2 == 0;
    constexpr int Q = (PX + 1) / 2;
    float T[PX], C0[PX], C1[PX], C2[PX];
    float2 T2[Q], D0[Q], D1[Q], D2[Q];
    // mw: the pixel's blend bits in the current chunk of 32 list positions (the
    // blend mask word when recorded); the blend count and the last contributor
    // are taken from each finished word, not per blend
    uint32_t last[PX], stop[PX], mw[PX];
    bool done[PX];
    int active = 0;  // pixels of this thread still compositing
  #pragma unroll
    for (int q = 0; q < Q; ++q) {
      T2[q] = f2(1.0f);
      D0[q] = D1[q] = D2[q] = f2(0.0f);
    }
  #pragma unroll
    for (int p = 0; p < PX; ++p) {
      T[p] = 1.0f;
      C0[p] = C1[p] = C2[p] = 0.0f;
      last[p] = 0;
      stop[p] = range.y;
      mw[p] = 0u;
      done[p] = !(px < tc.vi.width && py0 + p < tc.vi.height);
      active += done[p] ? 0 : 1;
    }
    uint32_t blended = 0;
    for (uint32_t start = range.x; start < range.y; start += BATCH) {
      if (__syncthreads_count(active == 0) == NT) break;
      stage_batch<MODE, BATCH>(a, vals, start, range.y, NT, s_r0, s_r1, s_r2, s_r3, nullptr);
      __syncthreads();
      const int cnt = (int)min((uint32_t)BATCH, range.y - start);
      if (active) {
        for (int jc = 0; jc < cnt; jc += 32) {  // chunks of 32 positions (one mask word)
          const int jend = min(cnt, jc + 32);
          const uint32_t cbase = start - range.x + jc;  // list position of the chunk's bit 0
          const uint32_t chunk = cbase >> 5;
          for (int j = jc; j < jend; ++j) {
            const float4 r0 = s_r0[j], r1 = s_r1[j], r3 = s_r3[j];
            const float4 r2 = MODE == MODE_PLAIN ? r0 : s_r2[j];
            if constexpr (PACKED) {
              // rows 2q and 2q + 1 together; a row that fails the gate, the
              // alpha_min test or has stopped takes alpha = 0 in the packed
              // blend, which leaves its T and colour unchanged exactly
  #pragma unroll
              for (int q = 0; q < Q; ++q) {
                if (done[2 * q] && done[2 * q + 1]) continue;
                PairEval2 e;
                const float2 p2 = pair2_exponent(r0, r1, fx, (float)(py0 + 2 * q) + 0.5f, e);
                const bool g0 = !done[2 * q] && p2.x >= r3.w, g1 = !done[2 * q + 1] && p2.y >= r3.w;
                if (!(g0 || g1)) continue;
                pair2_alpha<MODE>(r1, r2, p2, e);
                const float al0 = fminf(e.alpha.x, amax), al1 = fminf(e.alpha.y, amax);
                const bool b0 = g0 && al0 >= amin, b1 = g1 && al1 >= amin;
                if (!(b0 || b1)) continue;
                float2 al = make_float2(b0 ? al0 : 0.0f, b1 ? al1 : 0.0f);
                float2 Tn = fma2(neg2(T2[q]), al, T2[q]);
                const bool s0 = b0 && Tn.x < tstop, s1 = b1 && Tn.y < tstop;
                if (s0 || s1) {
                  if (s0) {
                    done[2 * q] = true;
                    stop[2 * q] = start + j + 1;
                    credit(mw[2 * q], cbase, blended, last[2 * q]);
                    if (REC) mbase[chunk * 256 + pi0 + 2 * q * kTile] = mw[2 * q];
                    al.x = 0.0f;
                    Tn.x = T2[q].x;
                    --active;
                  }
                  if (s1) {
                    done[2 * q + 1] = true;
                    stop[2 * q + 1] = start + j + 1;
                    credit(mw[2 * q + 1], cbase, blended, last[2 * q + 1]);
                    if (REC) mbase[chunk * 256 + pi0 + (2 * q + 1) * kTile] = mw[2 * q + 1];
                    al.y = 0.0f;
                    Tn.y = T2[q].y;
                    --active;
                  }
                  if (active == 0) goto batch_done;
                }
                const bool c0 = b0 && !s0, c1 = b1 && !s1;
                const float2 w = mul2(al, T2[q]);
                D0[q] = fma2(f2(r3.x), w, D0[q]);
                D1[q] = fma2(f2(r3.y), w, D1[q]);
                D2[q] = fma2(f2(r3.z), w, D2[q]);
                T2[q] = Tn;
                mw[2 * q] |= (uint32_t)c0 << (j & 31);
                mw[2 * q + 1] |= (uint32_t)c1 << (j & 31);
              }
            } else {
  #pragma unroll
              for (int p = 0; p < PX; ++p) {
                if (PX > 1 && done[p]) continue;
                PairEval e;
                if (!eval_pair<MODE>(r0, r1, r2, r3.w, fx, (float)(py0 + p) + 0.5f, e)) continue;
                const float alpha = fminf(e.alpha, amax);
                if (alpha < amin) continue;
                const float Tn = __fmaf_rn(-T[p], alpha, T[p]);
                if (Tn < tstop) {
                  done[p] = true;
                  stop[p] = start + j + 1;
                  credit(mw[p], cbase, blended, last[p]);
                  if (REC) mbase[chunk * 256 + pi0 + p * kTile] = mw[p];
                  if (--active == 0) goto batch_done;  // the only exit test, off the hot path
                  continue;
                }
                mw[p] |= 1u << (j & 31);
                const float w = __fmul_rn(alpha, T[p]);
                C0[p] = __fmaf_rn(r3.x, w, C0[p]);
                C1[p] = __fmaf_rn(r3.y, w, C1[p]);
                C2[p] = __fmaf_rn(r3.z, w, C2[p]);
                T[p] = Tn;
              }
            }
          }
  #pragma unroll
          for (int p = 0; p < PX; ++p)
            if (!done[p]) {
              credit(mw[p], cbase, blended, last[p]);
              if (REC) mbase[chunk * 256 + pi0 + p * kTile] = mw[p];
              mw[p] = 0u;
            }
        }
      }
    batch_done:;
    }
    // work counters: pairs each pixel evaluated (up to its stop) and blended
    unsigned long long tested = 0;
  #pragma unroll
    for (int p = 0; p < PX; ++p)
      if (px < tc.vi.width && py0 + p < tc.vi.height) tested += stop[p] - range.x;
    unsigned long long b64 = blended;
  #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tested += __shfl_xor_sync(0xffffffffu, tested, o);
      b64 += __shfl_xor_sync(0xffffffffu, b64, o);
    }
    if ((threadIdx.x & 31) == 0 && tested) {
      atomicAdd(&a.status->pairs_tested, tested);
      atomicAdd(&a.status->pairs_blended, b64);
    }
    const int64_t plane = (int64_t)tc.vi.width * tc.vi.height;
    float* img = a.images + tc.vi.image_offset;
    if constexpr (PACKED) {
  #pragma unroll
      for (int p = 0; p < PX; ++p) {
        const bool hi = p & 1;
        T[p] = hi ? T2[p >> 1].y : T2[p >> 1].x;
        C0[p] = hi ? D0[p >> 1].y : D0[p >> 1].x;
        C1[p] = hi ? D1[p >> 1].y : D1[p >> 1].x;
        C2[p] = hi ? D2[p >> 1].y : D2[p >> 1].x;
      }
    }
  #pragma unroll
    for (int p = 0; p < PX; ++p) {
      const int py = py0 + p;
      if (px < tc.vi.width && py < tc.vi.height) {
        const int64_t pix = (int64_t)py * tc.vi.width + px;
        img[pix] = __fmaf_rn(T[p], a.cfg.bg[0], C0[p]);
        img[plane + pix] = __fmaf_rn(T[p], a.cfg.bg[1], C1[p]);
        img[2 * plane + pix] = __fmaf_rn(T[p], a.cfg.bg[2], C2[p]);
        a.t_final[tc.vi.pixel_offset + pix] = T[p];
        a.n_contrib[tc.vi.pixel_offset + pix] = last[p];
      }
    }
  };
  if (PERSIST) {
    for (uint32_t it = next_work(a.work, &s_next); it < a.n_order; it = next_work(a.work, &s_next)) tile_body(it);
  } else {
    tile_body(blockIdx.x);
  }
}

// Sum 16 per-lane values over the warp with a transposing butterfly: at each
// step a lane keeps half of its values and sends the other half to its
// partner, so 8 + 4 + 2 + 1 + 1 shuffles replace 16 x 5.  Returns, in every
// lane, the warp total of value index (lane >> 1) & 15.
// ZERO3: slots 3 and 11 are zero in every lane (one opacity); slots 7 and 15
// always are, so their exchanges are skipped.
static_assert(G_ABS == 7 && G_PAD == 15 && G_UX == 3 && G_UY == 11, "reduction pairs of zero slots");
template <bool ZERO3>
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i == 7 || (ZERO3 && i == 3)) continue;  // v[i] and v[i + 8] are zero: so is the sum
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 8];
    const float keep = hi ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (ZERO3 && i == 3) continue;  // positions 3 and 7 hold slots 3, 11, 7 and 15: zero
    const bool hi = lane & 8;
    const float send = hi ? v[i] : v[i + 4];
    const float keep = hi ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 4;
    const float send = hi ? v[i] : v[i + 2];
    const float keep = hi ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    const float send = hi ? v[0] : v[1];
    const float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Per-thread pixel state of the backward composite and the contribution of
// one record to the thread's pixels.  Scalar form: any PX.
template <int MODE, int PX, bool PACKED = (PX % 2 == 0)>
struct BwdPixels {
  float T[PX], g0[PX], g1[PX], g2[PX], R0[PX], R1[PX], R2[PX];

  __device__ __forceinline__ void init(int p, const float* bg) {
    T[p] = 1.0f;
    g0[p] = g1[p] = g2[p] = 0.0f;
    R0[p] = bg[0];
    R1[p] = bg[1];
    R2[p] = bg[2];
  }
  __device__ __forceinline__ void load(int p, float t, float c0, float c1, float c2) {
    T[p] = t;
    g0[p] = c0;
    g1[p] = c1;
    g2[p] = c2;
  }
  // Adds to gr the record's gradient components over the pixels whose mask
  // word has `bit` set; returns whether there was one.
  __device__ __forceinline__ bool visit(const uint32_t (&bw)[PX], uint32_t bit, const float4& r0, const float4& r1,
                                        const float4& r2, const float4& r3, float fx, int py0, float amax,
                                        float (&gr)[16]) {
    const float a_ = -2.0f * kLn2 * r0.z, b_ = -kLn2 * r0.w, c_ = -2.0f * kLn2 * r1.x;
    bool contrib = false;
#pragma unroll
    for (int k = 0; k < 16; ++k) gr[k] = 0.0f;
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      if (!((bw[p] >> bit) & 1u)) continue;  // not blended in the forward pass
      PairEval e;
      // blended in the forward pass: the same arithmetic passes the alpha gate again
      eval_pair<MODE, false>(r0, r1, r2, r3.w, fx, (float)(py0 + p) + 0.5f, e);
      const float alpha = fminf(e.alpha, amax);
      contrib = true;
      const float one_m = 1.0f - alpha;
      T[p] = __fdividef(T[p], one_m);  // T_k (alpha <= alpha_max < 1)
      const float w = alpha * T[p];
      gr[G_R] += w * g0[p];
      gr[G_G] += w * g1[p];
      gr[G_BL] += w * g2[p];
      const float dLda = T[p] * (g0[p] * (r3.x - R0[p]) + g1[p] * (r3.y - R1[p]) + g2[p] * (r3.z - R2[p]));
      R0[p] = alpha * r3.x + one_m * R0[p];
      R1[p] = alpha * r3.y + one_m * R1[p];
      R2[p] = alpha * r3.z + one_m * R2[p];
      if (e.alpha <= amax) {  // the clamp has zero derivative
        const float S = e.G * e.E;           // skew kernel G' (1 + erf z)
        const float gS = dLda * e.o * S;
        const float gz = dLda * e.o * e.G * kTwoOverSqrtPi * e.ez;  // dL/dz
        float gdx = -gS * (a_ * e.dx + b_ * e.dy) + gz * r1.y;
        float gdy = -gS * (b_ * e.dx + c_ * e.dy) + gz * r1.z;
        gr[G_M] += dLda * S;
        gr[G_A] += -0.5f * gS * e.dx * e.dx;
        gr[G_B] += -gS * e.dx * e.dy;
        gr[G_C] += -0.5f * gS * e.dy * e.dy;
        gr[G_BX] += gz * e.dx * kInvSqrt2;
        gr[G_BY] += gz * e.dy * kInvSqrt2;
        if (MODE != MODE_PLAIN) {
          gr[G_H] += dLda * e.eu * S;
          const float gzu = dLda * r2.x * S * kTwoOverSqrtPi * e.ezu;
          gdx += gzu * r2.y;
          gdy += gzu * r2.z;
          gr[G_UX] += gzu * e.dx * kInvSqrt2;
          gr[G_UY] += gzu * e.dy * kInvSqrt2;
        }
        gr[G_MX] -= gdx;
        gr[G_MY] -= gdy;
      }
    }
    return contrib;
  }
  // The same for plans without blend masks: the bits mark candidate
  // positions (below the pixel's n_contrib) rather than blends, and a pair
  // counts only if it passes the forward's alpha gate, evaluated with the same
  // arithmetic (Alg. 2's replay without stored decisions).
  __device__ __forceinline__ bool visit_gated(const uint32_t (&bw)[PX], uint32_t bit, const float4& r0, const float4& r1,
                                        const float4& r2, const float4& r3, float fx, int py0, float amin, float amax,
                                        float (&gr)[16]) {
    const float a_ = -2.0f * kLn2 * r0.z, b_ = -kLn2 * r0.w, c_ = -2.0f * kLn2 * r1.x;
    bool contrib = false;
#pragma unroll
    for (int k = 0; k < 16; ++k) gr[k] = 0.0f;
#pragma unroll
    for (int p = 0; p < PX; ++p) {
      if (!((bw[p] >> bit) & 1u)) continue;  // not blended (not reached) in the forward pass
      PairEval e;
      if (!eval_pair<MODE, true>(r0, r1, r2, r3.w, fx, (float)(py0 + p) + 0.5f, e)) continue;
      if (fminf(e.alpha, amax) < amin) continue;
      const float alpha = fminf(e.alpha, amax);
      contrib = true;
      const float one_m = 1.0f - alpha;
      T[p] = __fdividef(T[p], one_m);  // T_k (alpha <= alpha_max < 1)
      const float w = alpha * T[p];
      gr[G_R] += w * g0[p];
      gr[G_G] += w * g1[p];
      gr[G_BL] += w * g2[p];
      const float dLda = T[p] * (g0[p] * (r3.x - R0[p]) + g1[p] * (r3.y - R1[p]) + g2[p] * (r3.z - R2[p]));
      R0[p] = alpha * r3.x + one_m * R0[p];
      R1[p] = alpha * r3.y + one_m * R1[p];
      R2[p] = alpha * r3.z + one_m * R2[p];
      if (e.alpha <= amax) {  // the clamp has zero derivative
        const float S = e.G * e.E;           // skew kernel G' (1 + erf z)
        const float gS = dLda * e.o * S;
        const float gz = dLda * e.o * e.G * kTwoOverSqrtPi * e.ez;  // dL/dz
        float gdx = -gS * (a_ * e.dx + b_ * e.dy) + gz * r1.y;
        float gdy = -gS * (b_ * e.dx + c_ * e.dy) + gz * r1.z;
        gr[G_M] += dLda * S;
        gr[G_A] += -0.5f * gS * e.dx * e.dx;
        gr[G_B] += -gS * e.dx * e.dy;
        gr[G_C] += -0.5f * gS * e.dy * e.dy;
        gr[G_BX] += gz * e.dx * kInvSqrt2;
        gr[G_BY] += gz * e.dy * kInvSqrt2;
        if (MODE != MODE_PLAIN) {
          gr[G_H] += dLda * e.eu * S;
          const float gzu = dLda * r2.x * S * kTwoOverSqrtPi * e.ezu;
          gdx += gzu * r2.y;
          gdy += gzu * r2.z;
          gr[G_UX] += gzu * e.dx * kInvSqrt2;
          gr[G_UY] += gzu * e.dy * kInvSqrt2;
        }
        gr[G_MX] -= gdx;
        gr[G_MY] -= gdy;
      }
    }
    return contrib;
  }
};

// Packed form (even PX): pixels 2q and 2q + 1 of the thread's column share
// dx and every operation runs on both at once (FP32x2).  A pixel whose bit is
// clear takes alpha = 0 (its colour state is unchanged exactly) and a zero
// dL/dalpha, so it adds nothing.  Every lane evaluates the pair, bits set or
// not: the warp issues the same instructions as with the clear lanes idle in
// a branch, and no zero-fill or reconvergence follows (every factor is
// finite, so the products with the zero alpha and dL/dalpha are zeros).
template <int MODE, int PX>
struct BwdPixels<MODE, PX, true> {
  static constexpr int Q = PX / 2;
  float2 T[Q], g0[Q], g1[Q], g2[Q], R0[Q], R1[Q], R2[Q];

  __device__ __forceinline__ static void put(float2& v, int p, float x) {
    if (p & 1) v.y = x;
    else v.x = x;
  }
  __device__ __forceinline__ void init(int p, const float* bg) {
    put(T[p >> 1], p, 1.0f);
    put(g0[p >> 1], p, 0.0f);
    put(g1[p >> 1], p, 0.0f);
    put(g2[p >> 1], p, 0.0f);
    put(R0[p >> 1], p, bg[0]);
    put(R1[p >> 1], p, bg[1]);
    put(R2[p >> 1], p, bg[2]);
  }
  __device__ __forceinline__ void load(int p, float t, float c0, float c1, float c2) {
    put(T[p >> 1], p, t);
    put(g0[p >> 1], p, c0);
    put(g1[p >> 1], p, c1);
    put(g2[p >> 1], p, c2);
  }
  __device__ __forceinline__ bool visit(const uint32_t (&bw)[PX], uint32_t bit, const float4& r0, const float4& r1,
                                        const float4& r2, const float4& r3, float fx, int py0, float amax,
                                        float (&gr)[16]) {
    const float a_ = -2.0f * kLn2 * r0.z, b_ = -kLn2 * r0.w, c_ = -2.0f * kLn2 * r1.x;
    float2 acc[16];
    bool any = false;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const bool m0 = (bw[2 * q] >> bit) & 1u, m1 = (bw[2 * q + 1] >> bit) & 1u;
      float2 t[16];
      any |= m0 || m1;
      PairEval2 e;
      eval_pair2<MODE>(r0, r1, r2, fx, (float)(py0 + 2 * q) + 0.5f, e);
      const float2 alpha = make_float2(m0 ? fminf(e.alpha.x, amax) : 0.0f, m1 ? fminf(e.alpha.y, amax) : 0.0f);
      const float2 one_m = add2(f2(1.0f), neg2(alpha));
      // T_k = T_{k+1} / (1 - alpha) as a product with the reciprocal (rcp.approx)
      const float2 Tn = mul2(T[q], make_float2(rcp_approx(one_m.x), rcp_approx(one_m.y)));
      T[q] = make_float2(m0 ? Tn.x : T[q].x, m1 ? Tn.y : T[q].y);
      const float2 w = mul2(alpha, T[q]);
      t[G_R] = mul2(w, g0[q]);
      t[G_G] = mul2(w, g1[q]);
      t[G_BL] = mul2(w, g2[q]);
      const float2 c0 = f2(r3.x), c1 = f2(r3.y), c2 = f2(r3.z);
      float2 s = mul2(g0[q], add2(c0, neg2(R0[q])));
      s = fma2(g1[q], add2(c1, neg2(R1[q])), s);
      s = fma2(g2[q], add2(c2, neg2(R2[q])), s);
      const float2 dl = mul2(T[q], s);
      R0[q] = fma2(alpha, c0, mul2(one_m, R0[q]));
      R1[q] = fma2(alpha, c1, mul2(one_m, R1[q]));
      R2[q] = fma2(alpha, c2, mul2(one_m, R2[q]));
      // dL/dalpha through the unclamped alpha (the clamp has zero derivative)
      const float2 dLda = make_float2(m0 && e.alpha.x <= amax ? dl.x : 0.0f, m1 && e.alpha.y <= amax ? dl.y : 0.0f);
      const float2 S = mul2(e.G, e.E);  // skew kernel G' (1 + erf z)
      const float2 dlo = mul2(dLda, e.o);
      const float2 gS = mul2(dlo, S);
      const float2 gz = mul2(mul2(mul2(dlo, e.G), f2(kTwoOverSqrtPi)), e.ez);  // dL/dz
      float2 gdx = fma2(neg2(gS), fma2(f2(b_), e.dy, f2(a_ * e.dx)), mul2(gz, f2(r1.y)));
      float2 gdy = fma2(neg2(gS), fma2(f2(c_), e.dy, f2(b_ * e.dx)), mul2(gz, f2(r1.z)));
      const float2 dx = f2(e.dx);
      t[G_M] = mul2(dLda, S);
      t[G_A] = mul2(gS, f2(-0.5f * e.dx * e.dx));
      t[G_B] = mul2(mul2(neg2(gS), dx), e.dy);
      t[G_C] = mul2(mul2(gS, f2(-0.5f)), mul2(e.dy, e.dy));
      t[G_BX] = mul2(gz, f2(e.dx * kInvSqrt2));
      t[G_BY] = mul2(mul2(gz, e.dy), f2(kInvSqrt2));
      if (MODE != MODE_PLAIN) {
        t[G_H] = mul2(mul2(dLda, e.eu), S);
        const float2 gzu = mul2(mul2(mul2(mul2(dLda, f2(r2.x)), S), f2(kTwoOverSqrtPi)), e.ezu);
        gdx = fma2(gzu, f2(r2.y), gdx);
        gdy = fma2(gzu, f2(r2.z), gdy);
        t[G_UX] = mul2(gzu, f2(e.dx * kInvSqrt2));
        t[G_UY] = mul2(mul2(gzu, e.dy), f2(kInvSqrt2));
      } else {
        t[G_H] = t[G_UX] = t[G_UY] = f2(0.0f);
      }
      t[G_MX] = neg2(gdx);
      t[G_MY] = neg2(gdy);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k == G_ABS || k == G_PAD) continue;
        acc[k] = q == 0 ? t[k] : add2(acc[k], t[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) gr[k] = (k == G_ABS || k == G_PAD) ? 0.0f : acc[k].x + acc[k].y;
    return any;
  }
  // visit for plans without blend masks: the bits mark candidates, the gate decides
  __device__ __forceinline__ bool visit_gated(const uint32_t (&bw)[PX], uint32_t bit, const float4& r0, const float4& r1,
                                        const float4& r2, const float4& r3, float fx, int py0, float amin, float amax,
                                        float (&gr)[16]) {
    const float a_ = -2.0f * kLn2 * r0.z, b_ = -kLn2 * r0.w, c_ = -2.0f * kLn2 * r1.x;
    float2 acc[16];
    bool any = false;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      bool m0 = (bw[2 * q] >> bit) & 1u, m1 = (bw[2 * q + 1] >> bit) & 1u;
      float2 t[16];
      PairEval2 e;
      const float2 p2 = pair2_exponent(r0, r1, fx, (float)(py0 + 2 * q) + 0.5f, e);
      pair2_alpha<MODE>(r1, r2, p2, e);
      // the forward's gate, with its arithmetic
      m0 = m0 && p2.x >= r3.w && fminf(e.alpha.x, amax) >= amin;
      m1 = m1 && p2.y >= r3.w && fminf(e.alpha.y, amax) >= amin;
      any |= m0 || m1;
      const float2 alpha = make_float2(m0 ? fminf(e.alpha.x, amax) : 0.0f, m1 ? fminf(e.alpha.y, amax) : 0.0f);
      const float2 one_m = add2(f2(1.0f), neg2(alpha));
      // T_k = T_{k+1} / (1 - alpha) as a product with the reciprocal (rcp.approx)
      const float2 Tn = mul2(T[q], make_float2(rcp_approx(one_m.x), rcp_approx(one_m.y)));
      T[q] = make_float2(m0 ? Tn.x : T[q].x, m1 ? Tn.y : T[q].y);
      const float2 w = mul2(alpha, T[q]);
      t[G_R] = mul2(w, g0[q]);
      t[G_G] = mul2(w, g1[q]);
      t[G_BL] = mul2(w, g2[q]);
      const float2 c0 = f2(r3.x), c1 = f2(r3.y), c2 = f2(r3.z);
      float2 s = mul2(g0[q], add2(c0, neg2(R0[q])));
      s = fma2(g1[q], add2(c1, neg2(R1[q])), s);
      s = fma2(g2[q], add2(c2, neg2(R2[q])), s);
      const float2 dl = mul2(T[q], s);
      R0[q] = fma2(alpha, c0, mul2(one_m, R0[q]));
      R1[q] = fma2(alpha, c1, mul2(one_m, R1[q]));
      R2[q] = fma2(alpha, c2, mul2(one_m, R2[q]));
      // dL/dalpha through the unclamped alpha (the clamp has zero derivative)
      const float2 dLda = make_float2(m0 && e.alpha.x <= amax ? dl.x : 0.0f, m1 && e.alpha.y <= amax ? dl.y : 0.0f);
      const float2 S = mul2(e.G, e.E);  // skew kernel G' (1 + erf z)
      const float2 dlo = mul2(dLda, e.o);
      const float2 gS = mul2(dlo, S);
      const float2 gz = mul2(mul2(mul2(dlo, e.G), f2(kTwoOverSqrtPi)), e.ez);  // dL/dz
      float2 gdx = fma2(neg2(gS), fma2(f2(b_), e.dy, f2(a_ * e.dx)), mul2(gz, f2(r1.y)));
      float2 gdy = fma2(neg2(gS), fma2(f2(c_), e.dy, f2(b_ * e.dx)), mul2(gz, f2(r1.z)));
      const float2 dx = f2(e.dx);
      t[G_M] = mul2(dLda, S);
      t[G_A] = mul2(gS, f2(-0.5f * e.dx * e.dx));
      t[G_B] = mul2(mul2(neg2(gS), dx), e.dy);
      t[G_C] = mul2(mul2(gS, f2(-0.5f)), mul2(e.dy, e.dy));
      t[G_BX] = mul2(gz, f2(e.dx * kInvSqrt2));
      t[G_BY] = mul2(mul2(gz, e.dy), f2(kInvSqrt2));
      if (MODE != MODE_PLAIN) {
        t[G_H] = mul2(mul2(dLda, e.eu), S);
        const float2 gzu = mul2(mul2(mul2(mul2(dLda, f2(r2.x)), S), f2(kTwoOverSqrtPi)), e.ezu);
        gdx = fma2(gzu, f2(r2.y), gdx);
        gdy = fma2(gzu, f2(r2.z), gdy);
        t[G_UX] = mul2(gzu, f2(e.dx * kInvSqrt2));
        t[G_UY] = mul2(mul2(gzu, e.dy), f2(kInvSqrt2));
      } else {
        t[G_H] = t[G_UX] = t[G_UY] = f2(0.0f);
      }
      t[G_MX] = neg2(gdx);
      t[G_MY] = neg2(gdy);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k == G_ABS || k == G_PAD) continue;
        acc[k] = q == 0 ? t[k] : add2(acc[k], t[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) gr[k] = (k == G_ABS || k == G_PAD) ? 0.0f : acc[k].x + acc[k].y;
    return any;
  }
};

// Zero the 2D-gradient records unless the projection zeroed this frame's
// touched records and no backward composite has used them since (the
// backward composite that follows marks them used).
__global__ void __launch_bounds__(256) d2_clear_kernel(Status* status, float4* d2, int64_t n4) {
  pdl_entry();
  if (status->d2_fresh) return;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x)
    d2[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

cudaError_t launch_d2_clear(Status* status, float4* d2, int64_t n4, int sms, cudaStream_t st) {
  const int64_t want = (n4 + 255) / 256;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  launch_pdl(d2_clear_kernel, dim3(grid), dim3(256), 0, st, status, d2, n4);
  count_launches(1);
  return cudaGetLastError();
}

// GATED: no blend masks (recompute_keys plans); every position below a
// pixel's n_contrib is a candidate and the pair's own gate decides.
template <int MODE, int PX, int BATCH, bool GATED, bool PERSIST>
__global__ void __launch_bounds__(256 / PX) render_bwd_kernel(RenderArgs a) {
  pdl_entry();
  if (blockIdx.x == 0 && threadIdx.x == 0) a.status->d2_fresh = 0u;  // read by the next d2_clear_kernel only
  constexpr int NT = 256 / PX;
  __shared__ float4 s_r0[BATCH], s_r1[BATCH], s_r2[MODE == MODE_PLAIN ? 1 : BATCH], s_r3[BATCH];
  __shared__ uint32_t s_id[BATCH];
  // per-batch gradient accumulators, component-major with a padded row so
  // both the warps' adds (16 components of one Gaussian) and the flush (one
  // Gaussian per thread) are free of bank conflicts
  __shared__ float s_acc[16][BATCH + 1];
  __shared__ uint32_t s_max;
  __shared__ uint32_t s_next;
  // one tile of the composite order; a persistent block takes tile after tile
  auto tile_body = [&](uint32_t it) {
    const int64_t tile = a.tile_order[it];
    const TileCoord tc = tile_coord(a, tile);
    const PixelMap pm = pixel_map<PX>(tc);
    const int px = pm.px, py0 = pm.py0;
    const float fx = (float)px + 0.5f;
    const uint2 range = tile_range(a.ranges, tile);
    const uint32_t* vals = a.status->sorted_buf ? a.vals1 : a.vals0;
    const float amin = a.cfg.alpha_min, amax = a.cfg.alpha_max;
    const int lane = threadIdx.x & 31;
    const int64_t plane = (int64_t)tc.vi.width * tc.vi.height;
    const float* gimg = a.d_images + tc.vi.image_offset;

    BwdPixels<MODE, PX> pix;
    uint32_t my_end[PX], bw[PX];
    const int pi0 = pm.pi0;
    const uint32_t* mbase = GATED ? nullptr : mask_tile_base(a.mask, range, tile);
    uint32_t my_max = 0;
  #pragma unroll
    for (int p = 0; p < PX; ++p) {
      const int py = py0 + p;
      pix.init(p, a.cfg.bg);
      my_end[p] = range.x;
      if (px < tc.vi.width && py < tc.vi.height) {
        const int64_t pix_i = (int64_t)py * tc.vi.width + px;
        pix.load(p, a.t_final[tc.vi.pixel_offset + pix_i], gimg[pix_i], gimg[plane + pix_i], gimg[2 * plane + pix_i]);
        const uint32_t nc = a.n_contrib[tc.vi.pixel_offset + pix_i];
        my_end[p] = min(range.y, range.x + nc);
        my_max = max(my_max, nc);
      }
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    if (my_max) atomicMax(&s_max, my_max);
    __syncthreads();
    const uint32_t end = min(range.y, range.x + s_max);

    for (uint32_t bend = end; bend > range.x;) {
      const uint32_t bstart = bend - range.x > (uint32_t)BATCH ? bend - BATCH : range.x;
      __syncthreads();  // previous batch fully consumed
      stage_batch<MODE, BATCH>(a, vals, bstart, bend, NT, s_r0, s_r1, s_r2, s_r3, s_id);
      for (int q = threadIdx.x; q < BATCH; q += NT) {
  #pragma unroll
        for (int k = 0; k < 16; ++k) s_acc[k][q] = 0.0f;
      }
      __syncthreads();
      // walk the batch from the top, one 32-position mask chunk at a time; the
      // warp visits only the positions one of its lanes blended, in descending
      // order (the replay recovers T and the colour behind from the top down)
      for (int jhi = (int)(bend - bstart) - 1; jhi >= 0;) {
        const uint32_t lp_hi = bstart + (uint32_t)jhi - range.x;
        const uint32_t chunk = lp_hi >> 5;
        const uint32_t chunk_first = range.x + (chunk << 5);  // position of bit 0
        const int jlo = chunk_first > bstart ? (int)(chunk_first - bstart) : 0;
  #pragma unroll
        for (int p = 0; p < PX; ++p) {
          if (GATED)  // the positions below the pixel's end
            bw[p] = chunk_first < my_end[p]
                        ? (my_end[p] - chunk_first >= 32u ? 0xffffffffu : (1u << (my_end[p] - chunk_first)) - 1u)
                        : 0u;
          else
            bw[p] = chunk_first < my_end[p] ? mbase[chunk * 256 + pi0 + p * kTile] : 0u;
        }
        uint32_t mine = 0u;
  #pragma unroll
        for (int p = 0; p < PX; ++p) mine |= bw[p];
        const uint32_t hi_bit = (uint32_t)jhi + bstart - chunk_first, lo_bit = (uint32_t)jlo + bstart - chunk_first;
        uint32_t todo = __reduce_or_sync(0xffffffffu, mine) & ((2u << hi_bit) - 1u) & ~((1u << lo_bit) - 1u);
        while (todo) {
          const uint32_t bit = 31u - __clz(todo);
          todo &= ~(1u << bit);
          const int j = (int)(chunk_first + bit - bstart);
          const float4 r0 = s_r0[j], r1 = s_r1[j], r3 = s_r3[j];
          const float4 r2 = MODE == MODE_PLAIN ? r0 : s_r2[j];
          float gr[16];
          const bool contrib = GATED ? pix.visit_gated(bw, bit, r0, r1, r2, r3, fx, py0, amin, amax, gr)
                                   : pix.visit(bw, bit, r0, r1, r2, r3, fx, py0, amax, gr);
          // true whenever the position is reached (it is a bit of the warp's
          // OR); the vote stays as the point where the warp meets before the
          // shuffles, which measured faster than leaving it out
          if (__any_sync(0xffffffffu, contrib)) {
            const float sum = warp_transpose_sum16<MODE == MODE_PLAIN>(gr, lane);
            if ((lane & 1) == 0 && sum != 0.0f) atomicAdd(&s_acc[lane >> 1][j], sum);
          }
        }
        jhi = jlo - 1;
      }
      __syncthreads();
      // one set of vector atomics per Gaussian per batch
      const int cnt = (int)(bend - bstart);
      for (int q = threadIdx.x; q < cnt; q += NT) {
        float c[16];
  #pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = s_acc[k][q];
        float* dst = a.d2 + kD2Stride * (int64_t)s_id[q];
  #pragma unroll
        for (int k = 0; k < 4; ++k)
          if (c[4 * k] != 0.0f || c[4 * k + 1] != 0.0f || c[4 * k + 2] != 0.0f || c[4 * k + 3] != 0.0f)
            red_add_v4(dst + 4 * k, c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]);
      }
      bend = bstart;
    }
  };
  if (PERSIST) {
    for (uint32_t it = next_work(a.work, &s_next); it < a.n_order; it = next_work(a.work, &s_next)) tile_body(it);
  } else {
    tile_body(blockIdx.x);
  }
}

// ---------------------------------------------------------------------------
// Dynamic shared memory (unused by the kernel) that caps the blocks resident
// on an SM at `blocks` (0: no cap): with it, blocks + 1 blocks no longer fit
// in the SM's shared memory, and `blocks` still do.
template <typename K>
static size_t occupancy_pad(K kernel, int blocks) {
  if (blocks <= 0) return 0;
  int dev = 0, per_sm = 0, reserved = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kernel) != cudaSuccess)
    return 0;
  const long dyn = (long)per_sm / (blocks + 1) - reserved - (long)fa.sharedSizeBytes + 1;
  if (dyn <= 0) return 0;  // shared memory already holds fewer than blocks + 1
  // above 48 KB of shared memory per block (static + dynamic) a kernel must opt in
  if (dyn + (long)fa.sharedSizeBytes > 48 * 1024)
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  return (size_t)dyn;
}

// Grid of a composite launch: one block per tile, or for a persistent launch
// as many blocks as fit on the GPU at once (at most one per tile).
template <typename K>
static unsigned composite_grid(K kernel, int threads, size_t dyn_smem, const RenderArgs& a, unsigned tiles) {
  if (!a.persistent) return tiles;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, dyn_smem) != cudaSuccess || occ < 1)
    occ = 1;
  return std::min<unsigned>(tiles, (unsigned)occ * (unsigned)std::max(1, a.sms));
}

template <int PX, bool REC, int BATCH, bool PERSIST>
static void launch_fwd_kernel(const RenderArgs& a, int mode, unsigned grid, cudaStream_t st) {
  auto k = mode == MODE_PLAIN ? render_fwd_kernel<MODE_PLAIN, PX, REC, BATCH, PERSIST>
           : mode == MODE_TWO ? render_fwd_kernel<MODE_TWO, PX, REC, BATCH, PERSIST>
                              : render_fwd_kernel<MODE_SPLIT, PX, REC, BATCH, PERSIST>;
  const size_t dyn = occupancy_pad(k, a.blocks_fwd);
  launch_pdl(k, dim3(composite_grid(k, 256 / PX, dyn, a, grid)), dim3(256 / PX), dyn, st, a);
}

template <int PX, bool REC, int BATCH>
static void launch_fwd_px(const RenderArgs& a, int mode, unsigned grid, cudaStream_t st) {
  if (a.persistent) launch_fwd_kernel<PX, REC, BATCH, true>(a, mode, grid, st);
  else launch_fwd_kernel<PX, REC, BATCH, false>(a, mode, grid, st);
}

template <bool REC, int BATCH>
static void launch_fwd_batch(const RenderArgs& a, int mode, unsigned grid, cudaStream_t st) {
  switch (a.px_fwd) {
    case 1: launch_fwd_px<1, REC, BATCH>(a, mode, grid, st); break;
    case 4: launch_fwd_px<4, REC, BATCH>(a, mode, grid, st); break;
    default: launch_fwd_px<2, REC, BATCH>(a, mode, grid, st); break;
  }
}

template <bool REC>
static void launch_fwd_rec(const RenderArgs& a, int mode, unsigned grid, cudaStream_t st) {
  switch (a.batch_fwd) {
    case 128: launch_fwd_batch<REC, 128>(a, mode, grid, st); break;
    case 512: launch_fwd_batch<REC, 512>(a, mode, grid, st); break;
    default: launch_fwd_batch<REC, 256>(a, mode, grid, st); break;
  }
}

template <int PX, int BATCH, bool GATED, bool PERSIST>
static void launch_bwd_kernel(const RenderArgs& a, int mode, unsigned grid, cudaStream_t st) {
  auto k = mode == MODE_PLAIN ? render_bwd_kernel<MODE_PLAIN, PX, BATCH, GATED, PERSIST>
           : mode == MODE_TWO ? render_bwd_kernel<MODE_TWO, PX, BATCH, GATED, PERSIST>
                              : render_bwd_kernel<MODE_SPLIT, PX, BATCH, GATED, PERSIST>;
  const size_t dyn = occupancy_pad(k, a.blocks_bwd);
  launch_pdl(k, dim3(composite_grid(k, 256 / PX, dyn, a, grid)), dim3(256 / PX), dyn, st, a);
}

template <int PX, int BATCH, bool GATED>
static void launch_bwd_px(const RenderArgs& a, int mode, unsigned grid, cudaStream_t st) {
  if (a.persistent) launch_bwd_kernel<PX, BATCH, GATED, true>(a, mode, grid, st);
  else launch_bwd_kernel<PX, BATCH, GATED, false>(a, mode, grid, st);
}

template <int BATCH, bool GATED>
static void launch_bwd_batch(const RenderArgs& a, int mode, unsigned grid, cudaStream_t st) {
  switch (a.px_bwd) {
    case 1: launch_bwd_px<1, BATCH, GATED>(a, mode, grid, st); break;
    case 4: launch_bwd_px<4, BATCH, GATED>(a, mode, grid, st); break;
    default: launch_bwd_px<2, BATCH, GATED>(a, mode, grid, st); break;
  }
}

cudaError_t launch_render_fwd(const RenderArgs& a, int mode, int64_t total_tiles, cudaStream_t st) {
  if (total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)total_tiles;
  if (a.persistent && cudaMemsetAsync(a.work, 0, sizeof(uint32_t), st) != cudaSuccess) return cudaGetLastError();
  if (a.mask) launch_fwd_rec<true>(a, mode, grid, st);
  else launch_fwd_rec<false>(a, mode, grid, st);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const RenderArgs& a, int mode, int64_t total_tiles, cudaStream_t st) {
  if (total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)total_tiles;
  if (a.persistent && cudaMemsetAsync(a.work, 0, sizeof(uint32_t), st) != cudaSuccess) return cudaGetLastError();
  const bool gated = a.mask == nullptr;  // no blend masks: replay with the gate
  if (a.batch_bwd == 128) {
    if (gated) launch_bwd_batch<128, true>(a, mode, grid, st);
    else launch_bwd_batch<128, false>(a, mode, grid, st);
  } else {
    if (gated) launch_bwd_batch<256, true>(a, mode, grid, st);
    else launch_bwd_batch<256, false>(a, mode, grid, st);
  }
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace sr
