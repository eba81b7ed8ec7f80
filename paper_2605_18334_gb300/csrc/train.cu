// The training step around the rasterizer: the photometric loss and its
// gradient, and a fused Adam update.  The paper trains its skew Gaussians
// inside the 3DGS framework (Preliminaries: "driven by photometric loss";
// Appendix "Implementation": the 3DGS protocol, learning rate 1e-4 for the
// skew parameters), so the objective is 3DGS's
//   L = (1 - lambda) mean |C - T| + lambda (1 - mean SSIM(C, T)),
// SSIM per channel with an 11 x 11 Gaussian window (sigma 1.5, normalised,
// zero padding), C1 = 0.01^2, C2 = 0.03^2, means over the 3 channels and
// all pixels of all views.
//
// SSIM at pixel q, from windowed moments mu_x, mu_y, s_x = E[x^2] - mu_x^2,
// s_y, s_xy = E[xy] - mu_x mu_y:
//   S = A1 A2 / (B1 B2),  A1 = 2 mu_x mu_y + C1, A2 = 2 s_xy + C2,
//                         B1 = mu_x^2 + mu_y^2 + C1, B2 = s_x + s_y + C2.
// With a = dS/dmu_x = 2 A2 (mu_y B1 - mu_x A1) / (B1^2 B2),
//      b = dS/ds_x = -A1 A2 / (B1 B2^2), c = dS/ds_xy = 2 A1 / (B1 B2),
// and dmu_x(q)/dx_p = w(p - q), ds_x/dx_p = 2 w (x_p - mu_x), ds_xy/dx_p =
// w (y_p - mu_y), the gradient of sum_q g S(q) is
//   dx_p = (w * u)(p) + 2 x_p (w * v)(p) + y_p (w * k)(p),
//   u = g (a - 2 mu_x b - mu_y c), v = g b, k = g c
// (w symmetric, so the adjoint correlation is the same filter).  One kernel
// computes the moments and u, v, k per 16 x 16 tile (a 26 x 26 halo in
// shared memory, separable passes), a second filters u, v, k the same way.
#include <cmath>

#include "kernels.cuh"

namespace sr {

constexpr int kWin = 11, kHalf = 5, kHalo = kTile + 2 * kHalf;  // 26
constexpr float kC1 = 0.0001f, kC2 = 0.0009f;                  // (0.01)^2, (0.03)^2

struct LossArgs {
  const float* images;
  const float* targets;
  float* d_images;
  float* loss;          // [1]
  float* ssim_l1;       // [2] or nullptr: mean SSIM, mean |C - T|
  float* maps;          // u, v, k: [3][3 * total pixels] (channel-major per view like the images)
  float* partial;       // [2][blocks]: per-block sums of S and |C - T|
  const ViewInfo* views;
  int n_views;
  int64_t total_tiles;
  int64_t total_values;  // 3 * total pixels
  float lambda;
  float win[kWin];       // normalised Gaussian window (kernel parameters: no separate upload)
};

struct TileRef {
  ViewInfo vi;
  int x0, y0;       // first pixel of the tile
  int64_t plane;    // offset of this channel's [H][W] plane
};

__device__ __forceinline__ TileRef loss_tile(const LossArgs& a, uint32_t b) {
  TileRef t;
  const uint32_t tt = (uint32_t)a.total_tiles;  // < 2^31 tiles per plan
  const uint32_t ch = b / tt;
  const uint32_t tile = b - ch * tt;
  const int v = view_of_tile(a.views, a.n_views, tile);
  t.vi = a.views[v];
  const int lt = (int)(tile - (uint32_t)t.vi.tile_base);
  t.x0 = (lt % t.vi.tiles_x) * kTile;
  t.y0 = (lt / t.vi.tiles_x) * kTile;
  t.plane = t.vi.image_offset + (int64_t)ch * t.vi.width * t.vi.height;
  return t;
}

// Separable window sums over a 16 x 16 tile with a 5-pixel halo (26 x 26),
// in shared memory.  Two values that are filtered alike travel as one float2
// (x and y; x^2 and y^2; u and v) so each tap is one packed FP32x2 FMA.  The
// horizontal pass gives each of 208 threads one halo row and two adjacent
// output columns (12 inputs, 11 taps); its results are stored transposed
// (column-major), so the vertical pass reads a column's 12 inputs as
// contiguous 16-byte vectors; a vertical-pass thread owns one tile column and
// two adjacent rows and finishes its two pixels itself.
constexpr int kHp = kHalo + 2;  // padded row length (even: 8-byte aligned pairs)

struct WinWeights {
  float w[kWin];
  __device__ __forceinline__ explicit WinWeights(const LossArgs& a) {
#pragma unroll
    for (int k = 0; k < kWin; ++k) w[k] = a.win[k];
  }
};

// sum_k w_k v[k + o] for o = 0, 1 (two adjacent outputs of a 12-input run)
__device__ __forceinline__ void taps2(const WinWeights& W, const float2 (&v)[kWin + 1], float2& o0, float2& o1) {
  o0 = o1 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    o0 = fma2(f2(W.w[k]), v[k], o0);
    o1 = fma2(f2(W.w[k]), v[k + 1], o1);
  }
}
__device__ __forceinline__ void taps1(const WinWeights& W, const float (&v)[kWin + 1], float& o0, float& o1) {
  o0 = o1 = 0.0f;
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    o0 = __fmaf_rn(W.w[k], v[k], o0);
    o1 = __fmaf_rn(W.w[k], v[k + 1], o1);
  }
}

__device__ __forceinline__ void block_sum2(float a, float b, float* s_red, float* out_a, float* out_b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s_red[2 * warp] = a;
    s_red[2 * warp + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float sa = 0.0f, sb = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += s_red[2 * w];
      sb += s_red[2 * w + 1];
    }
    *out_a = sa;
    *out_b = sb;
  }
}

// moments, SSIM and the maps u, v, k of one channel of one tile
__global__ void __launch_bounds__(256) ssim_fwd_kernel(LossArgs a) {
  pdl_entry();
  __shared__ __align__(16) float2 s_xy[kHalo][kHp];    // (x, y) of the tile and its halo
  __shared__ __align__(16) float2 s_a[kTile][kHp];     // horizontal sums of (x, y), [column][row]
  __shared__ __align__(16) float2 s_b[kTile][kHp];     // ... of (x^2, y^2)
  __shared__ __align__(16) float s_c[kTile][kHp];      // ... of x y
  __shared__ float s_red[16];
  const TileRef t = loss_tile(a, blockIdx.x);
  const int W = t.vi.width, H = t.vi.height;
  // the tile and its halo: every load of the thread issued before the stores
  constexpr int kPer = (kHalo * kHalo + 255) / 256;
  float2 xy[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + 256 * j, r = i / kHalo, c = i - r * kHalo;
    const int px = t.x0 - kHalf + c, py = t.y0 - kHalf + r;
    xy[j] = make_float2(0.0f, 0.0f);
    if (i < kHalo * kHalo && px >= 0 && px < W && py >= 0 && py < H) {
      const int64_t o = t.plane + (int64_t)py * W + px;
      xy[j] = make_float2(a.images[o], a.targets[o]);
    }
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + 256 * j, r = i / kHalo, c = i - r * kHalo;
    if (i < kHalo * kHalo) s_xy[r][c] = xy[j];
  }
  __syncthreads();
  const WinWeights Wt(a);
  if (threadIdx.x < kHalo * (kTile / 2)) {  // horizontal: halo row r, output columns c0, c0 + 1
    const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 2;
    float2 p[kWin + 1], q[kWin + 1];
    float m[kWin + 1];
#pragma unroll
    for (int j = 0; j <= kWin; ++j) {
      p[j] = s_xy[r][c0 + j];
      q[j] = mul2(p[j], p[j]);
      m[j] = p[j].x * p[j].y;
    }
    float2 a0, a1, b0, b1;
    float e0, e1;
    taps2(Wt, p, a0, a1);
    taps2(Wt, q, b0, b1);
    taps1(Wt, m, e0, e1);
    s_a[c0][r] = a0;
    s_a[c0 + 1][r] = a1;
    s_b[c0][r] = b0;
    s_b[c0 + 1][r] = b1;
    s_c[c0][r] = e0;
    s_c[c0 + 1][r] = e1;
  }
  __syncthreads();
  float s_val = 0.0f, l1 = 0.0f;
  if (threadIdx.x < kTile * (kTile / 2)) {  // vertical: column c, rows r0, r0 + 1
    const int c = threadIdx.x >> 3, r0 = (threadIdx.x & 7) * 2;
    float2 p[kWin + 1], q[kWin + 1];
    float m[kWin + 1];
#pragma unroll
    for (int j = 0; j <= kWin; ++j) {
      p[j] = s_a[c][r0 + j];
      q[j] = s_b[c][r0 + j];
      m[j] = s_c[c][r0 + j];
    }
    float2 mu[2], sq[2];
    float cr[2];
    taps2(Wt, p, mu[0], mu[1]);
    taps2(Wt, q, sq[0], sq[1]);
    taps1(Wt, m, cr[0], cr[1]);
    const float g = -a.lambda / (float)a.total_values;  // dL/dS
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int px = t.x0 + c, py = t.y0 + r0 + h;
      if (px < W && py < H) {
        const float mx = mu[h].x, my = mu[h].y;
        const float sx = sq[h].x - mx * mx, sy = sq[h].y - my * my, sxy = cr[h] - mx * my;
        const float A1 = 2.0f * mx * my + kC1, A2 = 2.0f * sxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = sx + sy + kC2;
        const float inv = 1.0f / (B1 * B2);
        const float S = A1 * A2 * inv;
        const float da = 2.0f * A2 * (my * B1 - mx * A1) * inv / B1;
        const float db = -S / B2;
        const float dc = 2.0f * A1 * inv;
        const int64_t o = t.plane + (int64_t)py * W + px;
        a.maps[o] = g * (da - 2.0f * mx * db - my * dc);
        a.maps[a.total_values + o] = g * db;
        a.maps[2 * a.total_values + o] = g * dc;
        const float2 v = s_xy[r0 + h + kHalf][c + kHalf];
        s_val += S;
        l1 += fabsf(v.x - v.y);
      }
    }
  }
  block_sum2(s_val, l1, s_red, &a.partial[blockIdx.x], &a.partial[gridDim.x + blockIdx.x]);
}

// dL/dC = (w * u) + 2 x (w * v) + y (w * k) + (1 - lambda) sign(x - y) / N
__global__ void __launch_bounds__(256) ssim_bwd_kernel(LossArgs a) {
  pdl_entry();
  __shared__ __align__(16) float2 s_uv[kHalo][kHp];
  __shared__ __align__(16) float s_k[kHalo][kHp];
  __shared__ __align__(16) float2 s_a[kTile][kHp];  // horizontal sums of (u, v), [column][row]
  __shared__ __align__(16) float s_c[kTile][kHp];   // ... of k
  const TileRef t = loss_tile(a, blockIdx.x);
  const int W = t.vi.width, H = t.vi.height;
  constexpr int kPer = (kHalo * kHalo + 255) / 256;
  float2 uv[kPer];
  float ks[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + 256 * j, r = i / kHalo, c = i - r * kHalo;
    const int px = t.x0 - kHalf + c, py = t.y0 - kHalf + r;
    uv[j] = make_float2(0.0f, 0.0f);
    ks[j] = 0.0f;
    if (i < kHalo * kHalo && px >= 0 && px < W && py >= 0 && py < H) {
      const int64_t o = t.plane + (int64_t)py * W + px;
      uv[j] = make_float2(a.maps[o], a.maps[a.total_values + o]);
      ks[j] = a.maps[2 * a.total_values + o];
    }
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int i = threadIdx.x + 256 * j, r = i / kHalo, c = i - r * kHalo;
    if (i < kHalo * kHalo) {
      s_uv[r][c] = uv[j];
      s_k[r][c] = ks[j];
    }
  }
  __syncthreads();
  const WinWeights Wt(a);
  if (threadIdx.x < kHalo * (kTile / 2)) {
    const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 2;
    float2 p[kWin + 1];
    float m[kWin + 1];
#pragma unroll
    for (int j = 0; j <= kWin; ++j) {
      p[j] = s_uv[r][c0 + j];
      m[j] = s_k[r][c0 + j];
    }
    float2 a0, a1;
    float e0, e1;
    taps2(Wt, p, a0, a1);
    taps1(Wt, m, e0, e1);
    s_a[c0][r] = a0;
    s_a[c0 + 1][r] = a1;
    s_c[c0][r] = e0;
    s_c[c0 + 1][r] = e1;
  }
  __syncthreads();
  if (threadIdx.x < kTile * (kTile / 2)) {
    const int c = threadIdx.x >> 3, r0 = (threadIdx.x & 7) * 2;
    float2 p[kWin + 1];
    float m[kWin + 1];
#pragma unroll
    for (int j = 0; j <= kWin; ++j) {
      p[j] = s_a[c][r0 + j];
      m[j] = s_c[c][r0 + j];
    }
    float2 f[2];
    float fk[2];
    taps2(Wt, p, f[0], f[1]);
    taps1(Wt, m, fk[0], fk[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int px = t.x0 + c, py = t.y0 + r0 + h;
      if (px < W && py < H) {
        const int64_t o = t.plane + (int64_t)py * W + px;
        const float x = a.images[o], y = a.targets[o];
        const float d = x - y;
        const float sgn = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
        a.d_images[o] = f[h].x + 2.0f * x * f[h].y + y * fk[h] + (1.0f - a.lambda) * sgn / (float)a.total_values;
      }
    }
  }
}

// L from the per-block sums (one block, fixed order: deterministic); eight
// loads of a thread in flight at a time, not one
constexpr int kReduceThreads = 1024;
__global__ void __launch_bounds__(kReduceThreads) loss_reduce_kernel(LossArgs a, int blocks) {
  pdl_entry();
  __shared__ float s_red[2 * kReduceThreads / 32];
  float s = 0.0f, l = 0.0f;
  for (int i0 = threadIdx.x; i0 < blocks; i0 += 8 * kReduceThreads) {
    float vs[8], vl[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * kReduceThreads;
      vs[u] = i < blocks ? a.partial[i] : 0.0f;
      vl[u] = i < blocks ? a.partial[blocks + i] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s += vs[u];
      l += vl[u];
    }
  }
  float ts = 0.0f, tl = 0.0f;
  block_sum2(s, l, s_red, &ts, &tl);
  if (threadIdx.x == 0) {
    const float n = (float)a.total_values;
    const float ms = ts / n, ml = tl / n;
    a.loss[0] = (1.0f - a.lambda) * ml + a.lambda * (1.0f - ms);
    if (a.ssim_l1) {
      a.ssim_l1[0] = ms;
      a.ssim_l1[1] = ml;
    }
  }
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba 2015), the update of torch.optim.Adam:
//   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//   p -= (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// over several parameter groups in one launch (blockIdx.y = group); within
// a group, elements whose index modulo `period` is at least `split_at` use
// lr_rest (the higher-order SH coefficients of an [N][K][3] array).
// ---------------------------------------------------------------------------
struct AdamGroupDev {
  float* p;
  const float* g;
  float* m;
  float* v;
  int64_t n;
  float step_size, step_size_rest;  // lr / (1 - b1^t) for the two learning rates
  int32_t period, split_at;
};

struct AdamArgs {
  AdamGroupDev grp[SR_ADAM_MAX_GROUPS];
  float b1, b2, eps, inv_sqrt_bc2;  // inv_sqrt_bc2 = 1 / sqrt(1 - b2^t)
};

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float step_size, const AdamArgs& a) {
  m = __fmaf_rn(a.b1, m, (1.0f - a.b1) * g);
  v = __fmaf_rn(a.b2, v, (1.0f - a.b2) * g * g);
  const float denom = __fmaf_rn(__fsqrt_rn(v), a.inv_sqrt_bc2, a.eps);
  p -= step_size * __fdiv_rn(m, denom);
}

__global__ void __launch_bounds__(256) adam_kernel(AdamArgs a) {
  pdl_entry();
  const AdamGroupDev& G = a.grp[blockIdx.y];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // 16-byte vectors when the arrays are aligned and a period (if any) is a
  // multiple of 4, so the 4 elements of a vector sit in one period
  const bool vec = (G.period % 4) == 0 &&
                   (((uintptr_t)G.p | (uintptr_t)G.g | (uintptr_t)G.m | (uintptr_t)G.v) & 15) == 0;
  if (vec) {
    const int64_t n4 = G.n / 4;
    const int32_t p4 = G.period / 4;
    for (int64_t i = tid; i < n4; i += stride) {
      float4 p = reinterpret_cast<float4*>(G.p)[i];
      const float4 g = reinterpret_cast<const float4*>(G.g)[i];
      float4 m = reinterpret_cast<float4*>(G.m)[i];
      float4 v = reinterpret_cast<float4*>(G.v)[i];
      const int32_t pos = p4 ? (int32_t)(i % p4) * 4 : 0;  // index of .x within its period
      const float s0 = p4 && pos >= G.split_at ? G.step_size_rest : G.step_size;
      const float s1 = p4 && pos + 1 >= G.split_at ? G.step_size_rest : G.step_size;
      const float s2 = p4 && pos + 2 >= G.split_at ? G.step_size_rest : G.step_size;
      const float s3 = p4 && pos + 3 >= G.split_at ? G.step_size_rest : G.step_size;
      adam_one(p.x, g.x, m.x, v.x, s0, a);
      adam_one(p.y, g.y, m.y, v.y, s1, a);
      adam_one(p.z, g.z, m.z, v.z, s2, a);
      adam_one(p.w, g.w, m.w, v.w, s3, a);
      reinterpret_cast<float4*>(G.p)[i] = p;
      reinterpret_cast<float4*>(G.m)[i] = m;
      reinterpret_cast<float4*>(G.v)[i] = v;
    }
    for (int64_t i = 4 * n4 + tid; i < G.n; i += stride) {
      const bool rest = G.period > 0 && (int32_t)(i % G.period) >= G.split_at;
      adam_one(G.p[i], G.g[i], G.m[i], G.v[i], rest ? G.step_size_rest : G.step_size, a);
    }
  } else {
    for (int64_t i = tid; i < G.n; i += stride) {
      const bool rest = G.period > 0 && (int32_t)(i % G.period) >= G.split_at;
      adam_one(G.p[i], G.g[i], G.m[i], G.v[i], rest ? G.step_size_rest : G.step_size, a);
    }
  }
}

// ---------------------------------------------------------------------------
// Densification statistics over iterations (Sec. "Depth-Aware Densification
// Strategy"): the 2D positional gradient norm g^(uv) accumulated with the
// number of steps a Gaussian was seen in, and g^(z) = max over iterations of
// |dL/dz| of its centre.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) densify_stats_kernel(const float* __restrict__ g_uv,
                                                            const float* __restrict__ g_z, int64_t n,
                                                            float* __restrict__ uv_sum, int32_t* __restrict__ seen,
                                                            float* __restrict__ z_max) {
  pdl_entry();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float u = g_uv[i];
    if (u > 0.0f) {
      uv_sum[i] += u;
      seen[i] += 1;
    }
    z_max[i] = fmaxf(z_max[i], fabsf(g_z[i]));
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// w_k = exp(-(k - 5)^2 / (2 * 1.5^2)), normalised to sum 1, in FP64, rounded once
static void window_weights(float* w) {
  double sum = 0.0, e[kWin];
  for (int k = 0; k < kWin; ++k) {
    const double d = k - kHalf;
    e[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += e[k];
  }
  for (int k = 0; k < kWin; ++k) w[k] = (float)(e[k] / sum);
}

size_t loss_scratch_bytes(int64_t total_pixels, int64_t total_tiles) {
  const size_t maps = sizeof(float) * 9 * (size_t)total_pixels;
  const size_t part = sizeof(float) * 2 * 3 * (size_t)total_tiles;
  return (maps + 255) / 256 * 256 + (part + 255) / 256 * 256;
}

cudaError_t launch_loss(const float* images, const float* targets, float lambda, float* d_images, float* loss,
                        float* ssim_l1, void* scratch, const ViewInfo* views, int n_views, int64_t total_tiles,
                        int64_t total_pixels, cudaStream_t st) {
  LossArgs a;
  window_weights(a.win);
  a.images = images;
  a.targets = targets;
  a.d_images = d_images;
  a.loss = loss;
  a.ssim_l1 = ssim_l1;
  a.maps = static_cast<float*>(scratch);
  a.partial = reinterpret_cast<float*>(static_cast<char*>(scratch) +
                                       (sizeof(float) * 9 * (size_t)total_pixels + 255) / 256 * 256);
  a.views = views;
  a.n_views = n_views;
  a.total_tiles = total_tiles;
  a.total_values = 3 * total_pixels;
  a.lambda = lambda;
  const int64_t blocks = 3 * total_tiles;
  launch_pdl(ssim_fwd_kernel, dim3((unsigned)blocks), dim3(256), 0, st, a);
  launch_pdl(ssim_bwd_kernel, dim3((unsigned)blocks), dim3(256), 0, st, a);
  launch_pdl(loss_reduce_kernel, dim3(1), dim3(kReduceThreads), 0, st, a, (int)blocks);
  count_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_adam(const sr_adam_group* groups, int n_groups, int64_t step, float b1, float b2, float eps,
                        int sms, cudaStream_t st) {
  AdamArgs a;
  const double bc1 = 1.0 - std::pow((double)b1, (double)step);
  const double bc2 = 1.0 - std::pow((double)b2, (double)step);
  int64_t max_n = 0;
  for (int i = 0; i < n_groups; ++i) {
    const sr_adam_group& g = groups[i];
    AdamGroupDev& d = a.grp[i];
    d.p = g.param;
    d.g = g.grad;
    d.m = g.m;
    d.v = g.v;
    d.n = g.n;
    d.step_size = (float)(g.lr / bc1);
    d.step_size_rest = (float)(g.lr_rest / bc1);
    d.period = g.period;
    d.split_at = g.split_at;
    max_n = std::max<int64_t>(max_n, g.n);
  }
  a.b1 = b1;
  a.b2 = b2;
  a.eps = eps;
  a.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(bc2));
  const int64_t want = (max_n / 4 + 255) / 256;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  launch_pdl(adam_kernel, dim3(gx, (unsigned)n_groups), dim3(256), 0, st, a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_densify_stats(const float* g_uv, const float* g_z, int64_t n, float* uv_sum, int32_t* seen,
                                 float* z_max, int sms, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
  launch_pdl(densify_stats_kernel, dim3(grid), dim3(256), 0, st, g_uv, g_z, n, uv_sum, seen, z_max);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace sr
