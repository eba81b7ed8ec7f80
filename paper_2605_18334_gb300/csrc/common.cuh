// Shared device-side definitions of the skew-Gaussian rasterizer (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "skewraster.h"

namespace sr {

// ---------------------------------------------------------------------------
// Workspace layout.  sr_plan_init fills plan->off[] with these slots, each
// 256-byte aligned; kernels receive raw pointers derived from them.
// ---------------------------------------------------------------------------
enum WsSlot {
  WS_STATUS = 0,   // Status
  WS_VIEWS,        // ViewInfo[SR_MAX_VIEWS]
  WS_REC,          // float4[M][4] render records
  WS_DEPTH,        // uint32_t[M] FP32 depth bits
  WS_DKEY0,        // uint32_t[M] depth sort key: depth bits, or ~0 if the record touches no tile
  WS_DKEY1,        //   ping-pong
  WS_PERM0,        // uint32_t[M] record indices in depth order (after the depth sort)
  WS_PERM1,        //   ping-pong
  WS_RECT,         // uint2[M]   tile rectangle (tx0 | ty0 << 16, tx1 | ty1 << 16), tx1/ty1 exclusive
  WS_NTOUCH,       // uint32_t[M] tiles touched
  WS_OFFSETS,      // uint32_t[M] exclusive scan of the tile counts, in depth order
  WS_SCAN_PART,    // uint64_t[scan blocks + 1]
  WS_KEYS0, WS_KEYS1,  // uint32_t[cap] global tile ids, ping-pong
  WS_VALS0, WS_VALS1,  // uint32_t[cap] record indices, ping-pong
  // WS_HIST .. WS_RANGES are cleared together every frame: keep them adjacent
  WS_HIST,         // uint32_t[2 * kMaxPasses][256] digit counts -> exclusive offsets (depth, tile)
  WS_LOOKBACK_D,   // uint64_t[parts(M)][kDepthPasses][256] look-back words of the depth sort
  WS_LOOKBACK,     // uint64_t[parts(cap)][tile passes][256] look-back words of the tile sort
  WS_RANGES,       // uint2[total_tiles] [start, end) of each tile's sorted keys
  WS_D2,           // float[M][16] per-(view, Gaussian) 2D gradients
  WS_FOOT,         // float4[M][4] footprint constants or packed row spans (row_tile_span)
  WS_MASK,         // uint32_t[(cap/32 + tiles + 1) * 256] per-pixel blend masks (see render.cu)
  WS_TILE_ORDER,   // uint32_t[tiles] composite order (longest key lists first) + uint32_t[kOrderWords] counters
                   // of the ordering + the tile counters of persistent forward and backward composites
  WS_SHJAC,        // float4[M][3] d colour / d view direction (3x3) and the colour clamp bits (backward only)
  WS_NUM_SLOTS
};
static_assert(WS_LOOKBACK_D == WS_HIST + 1 && WS_LOOKBACK == WS_HIST + 2 && WS_RANGES == WS_HIST + 3,
              "the per-frame cleared slots must be adjacent");

constexpr int kMaxPasses = 8;          // per sort: 8-bit digits of at most 64-bit keys
constexpr int kDepthPasses = 4;        // 32-bit depth keys
constexpr int kSortThreads = 256;      // threads per onesweep partition block
constexpr int kSortItems = 16;         // keys per thread
constexpr int kSortPart = kSortThreads * kSortItems;  // keys per partition
constexpr int kScanThreads = 512;
constexpr int kScanItems = 16;
constexpr int kScanBlock = kScanThreads * kScanItems;
constexpr int kTile = 16;              // tile edge in pixels
constexpr int kD2Stride = 16;          // floats per 2D-gradient record
constexpr int kOrderSubBits = 4;       // composite-order buckets per power of two: 2^kOrderSubBits
constexpr int kOrderBuckets = 32 * (1 << kOrderSubBits) + 1;  // over 32 bits, + empty
constexpr int kOrderWords = 2 * kOrderBuckets + 2;  // order counters, then the composites' work counters

// status word flags
constexpr uint32_t kStatusCapacity = 1u;
constexpr uint32_t kStatusTimeout = 2u;

struct Status {
  uint32_t flags;
  uint32_t sorted_buf;                // which ping-pong buffer holds the sorted keys
  unsigned long long keys_needed;     // total keys of the last frame
  uint32_t part_counter[2 * kMaxPasses];  // onesweep partition tickets per pass (depth sort, tile sort)
  uint32_t pass_trivial[2 * kMaxPasses];  // 1 if one digit holds every key of that pass
  uint32_t timeout_where;             // pass * 1e6 + partition of the first timed-out wait
  uint32_t pad1;
  unsigned long long pairs_tested;    // render_fwd: (pixel, Gaussian) pairs evaluated
  unsigned long long pairs_blended;   // render_fwd: pairs composited
  // last, kept across bin_sort's per-frame clear: 1 once the projection has
  // zeroed this frame's 2D-gradient records and no backward composite has
  // added into them since
  uint32_t d2_fresh;
  uint32_t pad2;
};

// host-side launch counter (diagnostics; defined in api.cu)
void count_launches(int k);

struct ViewInfo {
  int32_t width, height, tiles_x, tiles_y;
  int64_t tile_base;     // first global tile id
  int64_t image_offset;  // float offset of the [3][H][W] image
  int64_t pixel_offset;  // element offset of the [H][W] state
  int64_t pad;
};

// 2D-gradient record slots (float[16] per (view, Gaussian))
// The order puts the slots that are always zero (G_ABS, G_PAD) at 7 and 15
// and those zero with one opacity (G_UX, G_UY) at 3 and 11: the backward's
// transposing warp reduction pairs slot i with i + 8, then i with i + 4, and
// skips pairs that are zero in every lane.  (Mirrored by D2_SLOTS in the
// Python binding.)
enum D2Slot {
  G_MX = 0, G_MY = 1, G_A = 2, G_UX = 3, G_B = 4, G_C = 5, G_BX = 6, G_ABS = 7,
  G_BY = 8, G_M = 9, G_H = 10, G_UY = 11, G_R = 12, G_G = 13, G_BL = 14, G_PAD = 15
};
static_assert(G_G == G_R + 1 && G_BL == G_R + 2, "colour slots are read as G_R + channel");

// Render record: four float4 per (view, Gaussian).
//  r0 = (mx, my, A2, B2)     exponent in log2 units: P2 = A2 dx^2 + B2 dx dy + C2 dy^2
//  r1 = (C2, bxs, bys, m)    bxs = beta_x / sqrt 2, ...; m = comp (o1 + o2) / 2
//  r2 = (h, uxs, uys, 0)     h = comp (o1 - o2) / 2, u_2 / sqrt 2 (enhanced opacity)
//  r3 = (r, g, b, thr)       colour; thr: P2 < thr implies alpha < alpha_min
// with A2 = -a log2(e) / 2, B2 = -b log2(e), C2 = -c log2(e) / 2.

// Render modes, fixed per plan: what the opacity term needs.
enum RenderMode {
  MODE_PLAIN = 0,    // one opacity: o = m
  MODE_TWO = 1,      // two opacities, no split direction: u_2 = beta_2, erf shared
  MODE_SPLIT = 2     // two opacities and a split direction: a second erf
};

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kInvSqrt2 = 0.7071067811865476f;
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

// Abramowitz & Stegun (1964), formula 7.1.26 (after Hastings 1955):
//   erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-x^2),
//   t = 1 / (1 + p x), x >= 0, |error| <= 1.5e-7.
constexpr float kAsP = 0.3275911f;
constexpr float kAsA1 = 0.254829592f;
constexpr float kAsA2 = -0.284496736f;
constexpr float kAsA3 = 1.421413741f;
constexpr float kAsA4 = -1.453152027f;
constexpr float kAsA5 = 1.061405429f;

// Programmatic dependent launch (sm_90+).  A kernel launched with
// launch_pdl may be scheduled while its predecessor in the stream drains:
// it waits here for the predecessor to complete (its memory included)
// before anything else, so it may read and write what the predecessor did;
// and it lets its own dependents be scheduled once all its blocks run.
// Launched without the attribute, both instructions do nothing.
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1 + erf(z) and exp(-z^2) together.  For z < 0, 1 + erf(z) = erfc(|z|)
// is evaluated directly (no cancellation); for z >= 0 it is 2 - erfc(z).
struct OnePlusErf {
  float E;   // 1 + erf(z)
  float ez;  // exp(-z^2)
};

__device__ __forceinline__ OnePlusErf one_plus_erf(float z) {
  const float x = fabsf(z);
  const float t = rcp_approx(__fmaf_rn(kAsP, x, 1.0f));
  float p = __fmaf_rn(t, kAsA5, kAsA4);
  p = __fmaf_rn(t, p, kAsA3);
  p = __fmaf_rn(t, p, kAsA2);
  p = __fmaf_rn(t, p, kAsA1);
  const float ez = ex2_approx(__fmul_rn(__fmul_rn(-x, x), kLog2e));
  const float y = __fmul_rn(__fmul_rn(t, p), ez);  // erfc(|z|)
  OnePlusErf r;
  r.E = z >= 0.0f ? __fadd_rn(2.0f, -y) : y;
  r.ez = ez;
  return r;
}

// Per-pair evaluation shared by the forward and the backward kernels, with
// explicit rounding intrinsics so both take bit-identical decisions.
struct PairEval {
  float dx, dy;
  float G;       // exp(-1/2 d^T A d)
  float E;       // 1 + erf(z)
  float ez;      // exp(-z^2)
  float o;       // opacity term m + h erf(u^T d / sqrt 2)
  float eu;      // erf(u^T d / sqrt 2)  (MODE_TWO, MODE_SPLIT)
  float ezu;     // exp(-zu^2)           (MODE_SPLIT; = ez in MODE_TWO)
  float alpha;   // o G E, before the clamp
};

// GATE = false skips the early rejection, for pairs known to pass it (the
// backward replays only pairs the forward blended).
template <int MODE, bool GATE = true>
__device__ __forceinline__ bool eval_pair(const float4& r0, const float4& r1, const float4& r2, float thr, float px,
                                          float py, PairEval& e) {
  e.dx = __fadd_rn(px, -r0.x);
  e.dy = __fadd_rn(py, -r0.y);
  const float lin = __fmaf_rn(r0.z, e.dx, __fmul_rn(r0.w, e.dy));
  const float p2 = __fmaf_rn(lin, e.dx, __fmul_rn(__fmul_rn(r1.x, e.dy), e.dy));
  if (GATE && !(p2 >= thr)) return false;  // alpha < alpha_min guaranteed (and NaN-safe)
  e.G = ex2_approx(p2);
  if (r1.y == 0.0f && r1.z == 0.0f) {  // zero skew: 1 + erf(0) = 1 exactly
    e.E = 1.0f;
    e.ez = 1.0f;
  } else {
    const OnePlusErf s = one_plus_erf(__fmaf_rn(r1.y, e.dx, __fmul_rn(r1.z, e.dy)));
    e.E = s.E;
    e.ez = s.ez;
  }
  if (MODE == MODE_PLAIN) {
    e.o = r1.w;
    e.eu = 0.0f;
    e.ezu = 0.0f;
  } else if (MODE == MODE_TWO) {
    e.eu = __fadd_rn(e.E, -1.0f);
    e.ezu = e.ez;
    e.o = __fmaf_rn(r2.x, e.eu, r1.w);
  } else {
    if (r2.y == 0.0f && r2.z == 0.0f) {
      e.eu = 0.0f;
      e.ezu = 1.0f;
    } else {
      const OnePlusErf s = one_plus_erf(__fmaf_rn(r2.y, e.dx, __fmul_rn(r2.z, e.dy)));
      e.eu = __fadd_rn(s.E, -1.0f);
      e.ezu = s.ez;
    }
    e.o = __fmaf_rn(r2.x, e.eu, r1.w);
  }
  e.alpha = __fmul_rn(__fmul_rn(e.o, e.G), e.E);
  return true;
}

// Two pixels of one column (rows py and py + 1) against one record with the
// packed FP32x2 instructions of sm_100+ (__ffma2_rn and friends round each
// component like the scalar intrinsic): the same operations in the same order
// as eval_pair, so every component equals eval_pair's result bit for bit,
// in about half the issued instructions.  No gate: the backward evaluates
// only pairs the forward blended (and discards the other component).
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void one_plus_erf2(float2 z, float2& E, float2& ez) {
  const float2 x = make_float2(fabsf(z.x), fabsf(z.y));
  const float2 d = fma2(f2(kAsP), x, f2(1.0f));
  const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  float2 p = fma2(t, f2(kAsA5), f2(kAsA4));
  p = fma2(t, p, f2(kAsA3));
  p = fma2(t, p, f2(kAsA2));
  p = fma2(t, p, f2(kAsA1));
  const float2 q = mul2(mul2(neg2(x), x), f2(kLog2e));
  ez = make_float2(ex2_approx(q.x), ex2_approx(q.y));
  const float2 y = mul2(mul2(t, p), ez);  // erfc(|z|)
  const float2 two_m = add2(f2(2.0f), neg2(y));
  E = make_float2(z.x >= 0.0f ? two_m.x : y.x, z.y >= 0.0f ? two_m.y : y.y);
}

struct PairEval2 {
  float dx;  // shared by the two pixels
  float2 dy, G, E, ez, o, eu, ezu, alpha;
};

// The exponent P2 of both pixels (what the alpha gate tests).
__device__ __forceinline__ float2 pair2_exponent(const float4& r0, const float4& r1, float px, float py,
                                                 PairEval2& e) {
  e.dx = __fadd_rn(px, -r0.x);
  e.dy = add2(make_float2(py, py + 1.0f), f2(-r0.y));
  const float2 dx = f2(e.dx);
  const float2 lin = fma2(f2(r0.z), dx, mul2(f2(r0.w), e.dy));
  return fma2(lin, dx, mul2(mul2(f2(r1.x), e.dy), e.dy));
}

// The rest of the evaluation from the exponent: kernel, erf terms, opacity, alpha.
template <int MODE>
__device__ __forceinline__ void pair2_alpha(const float4& r1, const float4& r2, float2 p2, PairEval2& e) {
  const float2 dx = f2(e.dx);
  e.G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
  if (r1.y == 0.0f && r1.z == 0.0f) {
    e.E = f2(1.0f);
    e.ez = f2(1.0f);
  } else {
    one_plus_erf2(fma2(f2(r1.y), dx, mul2(f2(r1.z), e.dy)), e.E, e.ez);
  }
  if (MODE == MODE_PLAIN) {
    e.o = f2(r1.w);
    e.eu = f2(0.0f);
    e.ezu = f2(0.0f);
  } else if (MODE == MODE_TWO) {
    e.eu = add2(e.E, f2(-1.0f));
    e.ezu = e.ez;
    e.o = fma2(f2(r2.x), e.eu, f2(r1.w));
  } else {
    if (r2.y == 0.0f && r2.z == 0.0f) {
      e.eu = f2(0.0f);
      e.ezu = f2(1.0f);
    } else {
      float2 Eu;
      one_plus_erf2(fma2(f2(r2.y), dx, mul2(f2(r2.z), e.dy)), Eu, e.ezu);
      e.eu = add2(Eu, f2(-1.0f));
    }
    e.o = fma2(f2(r2.x), e.eu, f2(r1.w));
  }
  e.alpha = mul2(mul2(e.o, e.G), e.E);
}

template <int MODE>
__device__ __forceinline__ void eval_pair2(const float4& r0, const float4& r1, const float4& r2, float px, float py,
                                           PairEval2& e) {
  pair2_alpha<MODE>(r1, r2, pair2_exponent(r0, r1, px, py, e), e);
}

// Footprint of a record: the region
//   S = (E1 and beta^T d >= 0)  union  (E2 and beta^T d < 0)
// around mu_2, with E1 = {d^T Sigma_d^-1 d <= rho^2} (the conservative
// ellipse: alpha >= tau implies d in E1) and, on the side where
// z = beta^T d / sqrt 2 < 0, the smaller ellipse
// E2 = {d^T (Sigma_d^-1 + beta beta^T) d <= rho_-^2}, rho_-^2 =
// 2 ln(o_max comp / tau)(1 + 2^-10): there 1 + erf z = erfc|z| <= e^{-z^2},
// so alpha <= o_max comp exp(-d^T (Sigma_d^-1 + beta beta^T) d / 2).
// An ellipse with covariance Sigma is stored as e = (slope, wdet, ystar,
// ymax) and (rho2, inv_syy): slope = Sxy/Syy, wdet = det(Sigma)/Syy,
// ystar = rho Sxy / sqrt(Sxx) (height of its rightmost point), ymax =
// rho sqrt(Syy), inv_syy = 1/Syy; at height y (relative to mu_y) it spans
//   x = slope y -+ sqrt(wdet (rho2 - y^2 / Syy)).
// Record layout: f0 = E1's e; f1 = (rho2, inv_syy) of E1 (or the packed row
// spans, see below); f2 = E2's e; f3 = (rho_-^2, inv_syy of E2, slope,
// side) with the half-plane's boundary x = slope y (slope = -beta_y /
// beta_x) and side = +1 / -1 for beta_x > 0 / < 0 (the half-plane is to the
// right / left of the line), +2 / -2 for beta_x = 0 and beta_y > 0 / < 0
// (above / below mu), 0 for beta = 0 (the footprint is E1 alone).
//
// x-extent (relative to mu_x) of an ellipse within the band of heights
// [y0, y1] (relative to mu_y): the right edge is largest at y =
// clamp(ystar, band), the left edge smallest at y = clamp(-ystar, band)
// (concave / convex in y).  False if they do not meet.
__device__ __forceinline__ bool ellipse_band(const float4& e, float rho2, float inv_syy, float y0, float y1,
                                             float& xl, float& xr) {
  y0 = fmaxf(y0, -e.w);
  y1 = fminf(y1, e.w);
  if (!(y0 <= y1)) return false;
  const float yh = fminf(fmaxf(e.z, y0), y1);
  const float yl = fminf(fmaxf(-e.z, y0), y1);
  const float hh = __fsqrt_rn(__fmul_rn(e.y, fmaxf(0.0f, __fadd_rn(rho2, -__fmul_rn(__fmul_rn(yh, yh), inv_syy)))));
  const float hl = __fsqrt_rn(__fmul_rn(e.y, fmaxf(0.0f, __fadd_rn(rho2, -__fmul_rn(__fmul_rn(yl, yl), inv_syy)))));
  xr = __fadd_rn(__fmul_rn(e.x, yh), hh);
  xl = __fadd_rn(__fmul_rn(e.x, yl), -hl);
  return true;
}

// Tile row ty is touched in the tile columns that hold a pixel centre inside
// the x-extent of the footprint within the row's band of pixel-centre
// heights, taken as E1's extent cut by the hull of the half-plane's extent
// and E2's (a superset of S's extent).  The counting (preprocess) and
// emitting (duplicate) kernels call this with the stored constants and
// explicitly rounded operations, so they agree bit for bit.  Returns false
// if the row touches no tile.
__device__ __forceinline__ bool row_tile_span(const float4& f0, const float4& f1, const float4& f2,
                                              const float4& f3, float mx, float my, int ty, int width, int height,
                                              int& tlo, int& thi) {
  const float y0 = __fadd_rn((float)(ty * kTile) + 0.5f, -my);
  const float y1 = __fadd_rn((float)min(ty * kTile + kTile - 1, height - 1) + 0.5f, -my);
  float xl, xr;
  if (!ellipse_band(f0, f1.x, f1.y, y0, y1, xl, xr)) return false;
  const float side = f3.w;
  if (side != 0.0f) {
    // the half-plane beta^T d >= 0 within the band (clipped to E1's heights)
    const float c0 = fmaxf(y0, -f0.w), c1 = fminf(y1, f0.w);
    bool hon = true;
    float hl = -INFINITY, hr = INFINITY;
    if (side == 1.0f) {
      hl = fminf(__fmul_rn(f3.z, c0), __fmul_rn(f3.z, c1));
    } else if (side == -1.0f) {
      hr = fmaxf(__fmul_rn(f3.z, c0), __fmul_rn(f3.z, c1));
    } else {
      hon = side > 0.0f ? c1 >= 0.0f : c0 <= 0.0f;
    }
    float l2 = 0.0f, r2 = 0.0f;
    const bool e2on = ellipse_band(f2, f3.x, f3.y, y0, y1, l2, r2);
    if (!hon && !e2on) return false;
    const float ul = hon ? (e2on ? fminf(hl, l2) : hl) : l2;
    const float ur = hon ? (e2on ? fmaxf(hr, r2) : hr) : r2;
    xl = fmaxf(xl, ul);
    xr = fminf(xr, ur);
  }
  float lo = ceilf(__fadd_rn(__fadd_rn(mx, xl), -0.5f));
  float hi = floorf(__fadd_rn(__fadd_rn(mx, xr), -0.5f));
  lo = fmaxf(lo, 0.0f);
  hi = fminf(hi, (float)(width - 1));
  if (!(lo <= hi)) return false;
  tlo = (int)lo / kTile;
  thi = (int)hi / kTile;
  return true;
}

// Tile ranges: [start, end) of each tile's run in the sorted key list, stored
// as (~start, end) so that both ends can be reduced with atomicMax into a
// zero-initialised array; end == 0 marks an empty tile.
__device__ __forceinline__ uint2 tile_range(const uint2* ranges, int64_t tile) {
  const uint2 v = ranges[tile];
  return v.y ? make_uint2(~v.x, v.y) : make_uint2(0u, 0u);
}

// Row spans of a record's touched tiles, packed for the key emission when the
// tile box has at most kSpanRows rows, every row's first touched column lies
// within 15 of the box's first column and the record touches at most 255
// tiles: the footprint's second float4 then holds, as bits,
//   x, y  the exclusive prefix count of each row, one byte per row (rows
//         0-3 in x, 4-7 in y; 255 for rows below the box),
//   z     the first column of each row relative to the box, 4 bits per row,
//   w     kSpansPacked.
// Other records keep (rho2, 1/Syy, 0, kSpansTall) there and are enumerated
// with row_tile_span again (from f0..f3).
constexpr int kSpanRows = 8;
constexpr uint32_t kSpansTall = 0xffffffffu;
constexpr uint32_t kSpansPacked = 0u;

// Storage loads (FP32 arithmetic whatever the storage type).
template <int DT>
__device__ __forceinline__ float ld(const void* p, int64_t i) {
  if (DT == SR_F32) return __ldg(static_cast<const float*>(p) + i);
  if (DT == SR_BF16) return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
  return __half2float(static_cast<const __half*>(p)[i]);
}

__device__ __forceinline__ float ld_dyn(const void* p, int dt, int64_t i) {
  if (dt == SR_F32) return ld<SR_F32>(p, i);
  if (dt == SR_BF16) return ld<SR_BF16>(p, i);
  return ld<SR_F16>(p, i);
}

// Record a status flag (first writer wins on timeout_where).
__device__ __forceinline__ void raise_status(Status* st, uint32_t flag) { atomicOr(&st->flags, flag); }

// Global tile id -> view by binary search over the tile bases.
__device__ __forceinline__ int view_of_tile(const ViewInfo* views, int n_views, int64_t tile) {
  int lo = 0, hi = n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct CfgDev {
  float alpha_min, alpha_max, t_stop, dilation, fov_clamp, near_z;
  float bg[3];
  int antialias;
};

inline CfgDev to_dev(const sr_config& c) {
  CfgDev d;
  d.alpha_min = c.alpha_min;
  d.alpha_max = c.alpha_max;
  d.t_stop = c.t_stop;
  d.dilation = c.dilation;
  d.fov_clamp = c.fov_clamp;
  d.near_z = c.near_z;
  d.bg[0] = c.bg[0];
  d.bg[1] = c.bg[1];
  d.bg[2] = c.bg[2];
  d.antialias = c.antialias_comp;
  return d;
}

// Pointers into the workspace.
struct Ws {
  Status* status;
  ViewInfo* views;
  float4* rec;
  uint32_t* depth;
  uint32_t* dkey[2];
  uint32_t* perm[2];
  uint2* rect;
  uint32_t* ntouch;
  uint32_t* offsets;
  unsigned long long* scan_part;
  uint32_t* keys[2];
  uint32_t* vals[2];
  uint32_t* hist;
  unsigned long long* lookback_d;
  unsigned long long* lookback;
  uint2* ranges;
  float* d2;
  float4* foot;
  uint32_t* mask;   // null when the plan is forward-only
  uint32_t* tile_order;
  float4* shjac;    // null when the plan is forward-only
};

inline Ws ws_ptrs(const sr_plan& p, void* base) {
  char* b = static_cast<char*>(base);
  auto at = [&](int slot) { return b + p.off[slot]; };
  Ws w;
  w.status = reinterpret_cast<Status*>(at(WS_STATUS));
  w.views = reinterpret_cast<ViewInfo*>(at(WS_VIEWS));
  w.rec = reinterpret_cast<float4*>(at(WS_REC));
  w.depth = reinterpret_cast<uint32_t*>(at(WS_DEPTH));
  w.dkey[0] = reinterpret_cast<uint32_t*>(at(WS_DKEY0));
  w.dkey[1] = reinterpret_cast<uint32_t*>(at(WS_DKEY1));
  w.perm[0] = reinterpret_cast<uint32_t*>(at(WS_PERM0));
  w.perm[1] = reinterpret_cast<uint32_t*>(at(WS_PERM1));
  w.rect = reinterpret_cast<uint2*>(at(WS_RECT));
  w.ntouch = reinterpret_cast<uint32_t*>(at(WS_NTOUCH));
  w.offsets = reinterpret_cast<uint32_t*>(at(WS_OFFSETS));
  w.scan_part = reinterpret_cast<unsigned long long*>(at(WS_SCAN_PART));
  w.keys[0] = reinterpret_cast<uint32_t*>(at(WS_KEYS0));
  w.keys[1] = reinterpret_cast<uint32_t*>(at(WS_KEYS1));
  w.vals[0] = reinterpret_cast<uint32_t*>(at(WS_VALS0));
  w.vals[1] = reinterpret_cast<uint32_t*>(at(WS_VALS1));
  w.hist = reinterpret_cast<uint32_t*>(at(WS_HIST));
  w.lookback_d = reinterpret_cast<unsigned long long*>(at(WS_LOOKBACK_D));
  w.lookback = reinterpret_cast<unsigned long long*>(at(WS_LOOKBACK));
  w.ranges = reinterpret_cast<uint2*>(at(WS_RANGES));
  w.d2 = reinterpret_cast<float*>(at(WS_D2));
  w.foot = reinterpret_cast<float4*>(at(WS_FOOT));
  w.mask = (p.forward_only || p.recompute_keys) ? nullptr : reinterpret_cast<uint32_t*>(at(WS_MASK));
  w.tile_order = reinterpret_cast<uint32_t*>(at(WS_TILE_ORDER));
  w.shjac = p.forward_only ? nullptr : reinterpret_cast<float4*>(at(WS_SHJAC));
  return w;
}

}  // namespace sr
