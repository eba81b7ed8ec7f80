// Per-tile compositing of skew Gaussians: forward (Alg. 1, Eq. color) and
// the reverse replay that differentiates it (Alg. 2).
//
// One 16x16 block per tile, one thread per pixel.  The tile's depth-sorted
// records are staged into shared memory in batches of 256 (one gathered
// 64-byte record per thread), then every pixel walks the batch:
//   alpha = min(alpha_max, o G' (1 + erf z)),  skip if alpha < alpha_min,
//   stop before the Gaussian whose T' = T (1 - alpha) would fall below t_stop,
//   C += c alpha T, T = T'.
// A block leaves as soon as every pixel has stopped (__syncthreads_count).
//
// Backward per pixel from its last blended Gaussian down: T_k = T_{k+1} /
// (1 - alpha_k), R_{k+1} = colour behind k normalised by T_{k+1} (the
// background included), dL/dalpha_k = T_k sum_c g_c (c_k,c - R_{k+1},c);
// per-pair 2D gradients are summed over the warp with shuffles and added to
// the Gaussian's record with one vector atomic per 4 components.
#include "kernels.cuh"

namespace sr {


template <int MODE>
__global__ void __launch_bounds__(256) render_fwd_kernel(RenderArgs a) {
  __shared__ float4 s_r0[256], s_r1[256], s_r2[MODE == MODE_PLAIN ? 1 : 256], s_r3[256];
  const int64_t tile = blockIdx.x;
  const int v = view_of_tile(a.views, a.n_views, tile);
  const ViewInfo vi = a.views[v];
  const int lt = (int)(tile - vi.tile_base);
  const int tx = lt % vi.tiles_x, ty = lt / vi.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < vi.width && py < vi.height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 range = a.ranges[tile];
  const uint32_t* vals = a.status->sorted_buf ? a.vals1 : a.vals0;
  const float amin = a.cfg.alpha_min, amax = a.cfg.alpha_max, tstop = a.cfg.t_stop;

  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
  uint32_t last = 0, tested = 0, blended = 0;
  bool done = !inside;
  for (uint32_t start = range.x; start < range.y; start += 256) {
    if (__syncthreads_count(done) == 256) break;
    const uint32_t idx = start + threadIdx.x;
    if (idx < range.y) {
      const float4* r = a.rec + 4 * (int64_t)vals[idx];
      s_r0[threadIdx.x] = r[0];
      s_r1[threadIdx.x] = r[1];
      if (MODE != MODE_PLAIN) s_r2[threadIdx.x] = r[2];
      s_r3[threadIdx.x] = r[3];
    }
    __syncthreads();
    const int cnt = (int)min(256u, range.y - start);
    if (!done) {
      int j = 0;
      for (; j < cnt; ++j) {
        const float4 r3 = s_r3[j];
        PairEval e;
        if (!eval_pair<MODE>(s_r0[j], s_r1[j], MODE == MODE_PLAIN ? s_r0[j] : s_r2[j], r3.w, fx, fy, e)) continue;
        const float alpha = fminf(e.alpha, amax);
        if (alpha < amin) continue;
        const float Tn = __fmaf_rn(-T, alpha, T);
        if (Tn < tstop) {
          done = true;
          ++j;
          break;
        }
        ++blended;
        const float w = __fmul_rn(alpha, T);
        C0 = __fmaf_rn(r3.x, w, C0);
        C1 = __fmaf_rn(r3.y, w, C1);
        C2 = __fmaf_rn(r3.z, w, C2);
        T = Tn;
        last = start + j + 1 - range.x;
      }
      tested += j;
    }
  }
  // work counters: one atomic per warp
  unsigned long long t64 = tested, b64 = blended;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t64 += __shfl_xor_sync(0xffffffffu, t64, o);
    b64 += __shfl_xor_sync(0xffffffffu, b64, o);
  }
  if ((threadIdx.x & 31) == 0 && t64) {
    atomicAdd(&a.status->pairs_tested, t64);
    atomicAdd(&a.status->pairs_blended, b64);
  }
  if (inside) {
    const int64_t plane = (int64_t)vi.width * vi.height;
    const int64_t pix = (int64_t)py * vi.width + px;
    float* img = a.images + vi.image_offset;
    img[pix] = __fmaf_rn(T, a.cfg.bg[0], C0);
    img[plane + pix] = __fmaf_rn(T, a.cfg.bg[1], C1);
    img[2 * plane + pix] = __fmaf_rn(T, a.cfg.bg[2], C2);
    a.t_final[vi.pixel_offset + pix] = T;
    a.n_contrib[vi.pixel_offset + pix] = last;
  }
}

// Sum 16 per-lane values over the warp with a transposing butterfly: at each
// step a lane keeps half of its values and sends the other half to its
// partner, so 8 + 4 + 2 + 1 + 1 shuffles replace 16 x 5.  Returns, in every
// lane, the warp total of value index (lane >> 1) & 15.
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 8];
    const float keep = hi ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
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

template <int MODE>
__global__ void __launch_bounds__(256) render_bwd_kernel(RenderArgs a) {
  __shared__ float4 s_r0[256], s_r1[256], s_r2[MODE == MODE_PLAIN ? 1 : 256], s_r3[256];
  __shared__ uint32_t s_id[256];
  // per-batch gradient accumulators, component-major with a padded row so
  // both the warps' adds (16 components of one Gaussian) and the flush (one
  // Gaussian per thread) are free of bank conflicts
  __shared__ float s_acc[16][257];
  __shared__ uint32_t s_max;
  const int64_t tile = blockIdx.x;
  const int v = view_of_tile(a.views, a.n_views, tile);
  const ViewInfo vi = a.views[v];
  const int lt = (int)(tile - vi.tile_base);
  const int tx = lt % vi.tiles_x, ty = lt / vi.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x >> 4);
  const bool inside = px < vi.width && py < vi.height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 range = a.ranges[tile];
  const uint32_t* vals = a.status->sorted_buf ? a.vals1 : a.vals0;
  const float amin = a.cfg.alpha_min, amax = a.cfg.alpha_max;
  const int lane = threadIdx.x & 31;

  float T = 1.0f, g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
  uint32_t my_last = 0;
  if (inside) {
    const int64_t plane = (int64_t)vi.width * vi.height;
    const int64_t pix = (int64_t)py * vi.width + px;
    const float* gi = a.d_images + vi.image_offset;
    g0 = gi[pix];
    g1 = gi[plane + pix];
    g2 = gi[2 * plane + pix];
    T = a.t_final[vi.pixel_offset + pix];
    my_last = a.n_contrib[vi.pixel_offset + pix];
  }
  float R0 = a.cfg.bg[0], R1 = a.cfg.bg[1], R2 = a.cfg.bg[2];
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  if (my_last) atomicMax(&s_max, my_last);
  __syncthreads();
  const uint32_t end = min(range.y, range.x + s_max);
  const uint32_t my_end = min(range.y, range.x + my_last);

  for (uint32_t bend = end; bend > range.x;) {
    const uint32_t bstart = bend - range.x > 256u ? bend - 256u : range.x;
    const uint32_t idx = bstart + threadIdx.x;
    __syncthreads();  // previous batch fully consumed
    if (idx < bend) {
      const uint32_t id = vals[idx];
      const float4* r = a.rec + 4 * (int64_t)id;
      s_id[threadIdx.x] = id;
      s_r0[threadIdx.x] = r[0];
      s_r1[threadIdx.x] = r[1];
      if (MODE != MODE_PLAIN) s_r2[threadIdx.x] = r[2];
      s_r3[threadIdx.x] = r[3];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) s_acc[k][threadIdx.x] = 0.0f;
    __syncthreads();
    for (int j = (int)(bend - bstart) - 1; j >= 0; --j) {
      const uint32_t pos = bstart + j;
      float gr[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) gr[k] = 0.0f;
      bool contrib = false;
      if (pos < my_end) {
        const float4 r0 = s_r0[j], r1 = s_r1[j], r3 = s_r3[j];
        const float4 r2 = MODE == MODE_PLAIN ? r0 : s_r2[j];
        PairEval e;
        if (eval_pair<MODE>(r0, r1, r2, r3.w, fx, fy, e)) {
          const float alpha = fminf(e.alpha, amax);
          if (alpha >= amin) {
            contrib = true;
            const float one_m = 1.0f - alpha;
            T = T / one_m;  // T_k
            const float w = alpha * T;
            gr[G_R] = w * g0;
            gr[G_G] = w * g1;
            gr[G_BL] = w * g2;
            const float dLda = T * (g0 * (r3.x - R0) + g1 * (r3.y - R1) + g2 * (r3.z - R2));
            R0 = alpha * r3.x + one_m * R0;
            R1 = alpha * r3.y + one_m * R1;
            R2 = alpha * r3.z + one_m * R2;
            if (e.alpha <= amax) {
              // alpha = o G E;  natural-unit conic a = -2 ln2 A2, b = -ln2 B2, c = -2 ln2 C2
              const float a_ = -2.0f * kLn2 * r0.z, b_ = -kLn2 * r0.w, c_ = -2.0f * kLn2 * r1.x;
              const float S = e.G * e.E;           // skew kernel G' (1 + erf z)
              const float gS = dLda * e.o * S;     // dL/dlog(G) path factor
              const float gz = dLda * e.o * e.G * kTwoOverSqrtPi * e.ez;  // dL/dz
              float gdx = -gS * (a_ * e.dx + b_ * e.dy) + gz * r1.y;
              float gdy = -gS * (b_ * e.dx + c_ * e.dy) + gz * r1.z;
              gr[G_M] = dLda * S;
              gr[G_A] = -0.5f * gS * e.dx * e.dx;
              gr[G_B] = -gS * e.dx * e.dy;
              gr[G_C] = -0.5f * gS * e.dy * e.dy;
              gr[G_BX] = gz * e.dx * kInvSqrt2;
              gr[G_BY] = gz * e.dy * kInvSqrt2;
              if (MODE != MODE_PLAIN) {
                gr[G_H] = dLda * e.eu * S;
                const float gzu = dLda * r2.x * S * kTwoOverSqrtPi * e.ezu;
                gdx += gzu * r2.y;
                gdy += gzu * r2.z;
                gr[G_UX] = gzu * e.dx * kInvSqrt2;
                gr[G_UY] = gzu * e.dy * kInvSqrt2;
              }
              gr[G_MX] = -gdx;
              gr[G_MY] = -gdy;
            }
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        const float sum = warp_transpose_sum16(gr, lane);
        if ((lane & 1) == 0 && sum != 0.0f) atomicAdd(&s_acc[lane >> 1][j], sum);
      }
    }
    __syncthreads();
    // one set of vector atomics per Gaussian per batch
    const int cnt = (int)(bend - bstart);
    if ((int)threadIdx.x < cnt) {
      float c[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) c[k] = s_acc[k][threadIdx.x];
      float* dst = a.d2 + kD2Stride * (int64_t)s_id[threadIdx.x];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c[4 * q] != 0.0f || c[4 * q + 1] != 0.0f || c[4 * q + 2] != 0.0f || c[4 * q + 3] != 0.0f)
          red_add_v4(dst + 4 * q, c[4 * q], c[4 * q + 1], c[4 * q + 2], c[4 * q + 3]);
    }
    bend = bstart;
  }
}

// ---------------------------------------------------------------------------
cudaError_t launch_render_fwd(const RenderArgs& a, int mode, int64_t total_tiles, cudaStream_t st) {
  if (total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)total_tiles;
  if (mode == MODE_PLAIN) render_fwd_kernel<MODE_PLAIN><<<grid, 256, 0, st>>>(a);
  else if (mode == MODE_TWO) render_fwd_kernel<MODE_TWO><<<grid, 256, 0, st>>>(a);
  else render_fwd_kernel<MODE_SPLIT><<<grid, 256, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_render_bwd(const RenderArgs& a, int mode, int64_t total_tiles, cudaStream_t st) {
  if (total_tiles == 0) return cudaSuccess;
  const unsigned grid = (unsigned)total_tiles;
  if (mode == MODE_PLAIN) render_bwd_kernel<MODE_PLAIN><<<grid, 256, 0, st>>>(a);
  else if (mode == MODE_TWO) render_bwd_kernel<MODE_TWO><<<grid, 256, 0, st>>>(a);
  else render_bwd_kernel<MODE_SPLIT><<<grid, 256, 0, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace sr
