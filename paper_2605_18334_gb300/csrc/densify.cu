// Densification (Sec. "Depth-Aware Densification Strategy"; the split of
// Fig. "split"): each Gaussian is removed, kept, cloned or split in two from
// the statistics collected over the iterations, and the new scene is written
// in one pass.
//
//   classify  per block of 1024 Gaussians: the action of each, and the
//             block's counts of kept, cloned and split Gaussians
//   scan      one block: exclusive offsets of the blocks, totals
//   scatter   per block: the Gaussians' output slots (block offset + block
//             scan), attributes copied or split
//
// Decision (FP32): removed if the largest opacity logit < logit_prune; else
// densified if uv_sum / seen >= grad_uv (g^(uv)) or z_max >= grad_z (g^(z),
// Eq. depth_grad): split if the largest log-scale > log_scale_split, cloned
// otherwise.
//
// Split along the largest axis k.  In the Gaussian's standardised frame the
// skew normal is Z ~ SN_3(0, I, eta) and its marginal along k is
// SN(0, 1, alpha_k), delta_k = eta_k / sqrt(1 + |eta|^2).  With
// phi = atan2(sqrt(1 + sum_{j != k} eta_j^2), -+eta_k) for the half Z_k >= 0
// (+) or < 0 (-) (phi / pi is the half's mass; phi = pi/2 +- asin(delta_k)),
// the half's mean and variance along k are
//   m = +-pi g(phi) / phi,  g(phi) = 2 sin^2(phi / 2) / sqrt(2 pi),
//   v = pi f(phi) / phi - m^2,  f(phi) = (2 phi - sin 2 phi) / (2 pi),
// forms without cancellation as a half's mass goes to zero (x - sin x by its
// Taylor series for small x).  A child moves by s_k m along the axis, takes
// log-scale log s_k + log(v) / 2 on it, skew eta_k = 0 and, on the other
// axes, eta_j / sqrt(1 + eta_k^2), which keeps the parent's marginal skew
// delta_j there.  Other attributes are copied.
#include <algorithm>

#include "kernels.cuh"

namespace sr {

constexpr int kDenThreads = 256;
constexpr int kDenItems = 4;
constexpr int kDenBlock = kDenThreads * kDenItems;
constexpr int kDenScanThreads = 1024;

enum DensifyAction { ACT_REMOVE = 0, ACT_KEEP = 1, ACT_CLONE = 2, ACT_SPLIT = 3 };

__device__ __forceinline__ int densify_action(const DensifyArgs& a, int64_t i) {
  float op = a.two ? fmaxf(a.opacity[2 * i], a.opacity[2 * i + 1]) : a.opacity[i];
  if (op < a.logit_prune) return ACT_REMOVE;
  const int32_t c = a.seen[i];
  const float guv = c > 0 ? a.uv_sum[i] / (float)c : 0.0f;
  if (guv >= a.grad_uv || a.z_max[i] >= a.grad_z) {
    const float* ls = a.log_scales + 3 * i;
    const float lmax = fmaxf(fmaxf(ls[0], ls[1]), ls[2]);
    return lmax > a.log_scale_split ? ACT_SPLIT : ACT_CLONE;
  }
  return ACT_KEEP;
}

// kept / cloned / split counts, 21 bits each in one word
__device__ __forceinline__ unsigned long long action_word(int act) {
  return act == ACT_KEEP ? 1ull : act == ACT_CLONE ? (1ull | (1ull << 21)) : act == ACT_SPLIT ? (1ull << 42) : 0ull;
}
constexpr unsigned long long kField = (1ull << 21) - 1ull;

template <class T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* s_warp, T& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? s_warp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[nw - 1];
  const T base = warp > 0 ? s_warp[warp - 1] : T(0);
  __syncthreads();
  return base + x - v;
}

__global__ void __launch_bounds__(kDenThreads) densify_classify_kernel(DensifyArgs a) {
  __shared__ unsigned long long s_warp[32];
  const int64_t base = (int64_t)blockIdx.x * kDenBlock + (int64_t)threadIdx.x * kDenItems;
  unsigned long long w = 0;
#pragma unroll
  for (int j = 0; j < kDenItems; ++j)
    if (base + j < a.n) w += action_word(densify_action(a, base + j));
  unsigned long long total;
  block_exclusive_sum(w, s_warp, total);
  if (threadIdx.x == 0) {
    uint32_t* bs = a.block_sums + 4 * (int64_t)blockIdx.x;
    bs[0] = (uint32_t)(total & kField);
    bs[1] = (uint32_t)((total >> 21) & kField);
    bs[2] = (uint32_t)((total >> 42) & kField);
  }
}

// exclusive offsets of the blocks' counts (in place) and the totals
__global__ void __launch_bounds__(kDenScanThreads) densify_scan_kernel(uint32_t* block_sums, int64_t nb,
                                                                       int64_t* counts) {
  __shared__ unsigned long long s_warp[32];
  unsigned long long carry[3] = {0, 0, 0};
  for (int64_t b0 = 0; b0 < nb; b0 += kDenScanThreads) {
    const int64_t b = b0 + threadIdx.x;
    uint32_t* bs = block_sums + 4 * b;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const unsigned long long v = b < nb ? bs[c] : 0ull;
      unsigned long long total;
      const unsigned long long ex = block_exclusive_sum(v, s_warp, total);
      if (b < nb) bs[c] = (uint32_t)(carry[c] + ex);
      carry[c] += total;
    }
  }
  if (threadIdx.x == 0) {
    counts[0] = (int64_t)carry[0];
    counts[1] = (int64_t)carry[1];
    counts[2] = (int64_t)carry[2];
    counts[3] = (int64_t)(carry[0] + carry[1] + 2 * carry[2]);
  }
}

__device__ __forceinline__ void copy3(const float* s, float* d) {
  d[0] = s[0];
  d[1] = s[1];
  d[2] = s[2];
}

// one output Gaussian but its SH row: a copy of Gaussian i, or (side = +1 /
// -1) one of its split children
__device__ __forceinline__ void write_gaussian(const DensifyArgs& a, int64_t i, int64_t p, int side) {
  const float* mu = a.means + 3 * i;
  const float* ls = a.log_scales + 3 * i;
  const float* eta = a.skew + 3 * i;
  const float4 q = reinterpret_cast<const float4*>(a.quats)[i];
  reinterpret_cast<float4*>(a.o_quats)[p] = q;
  if (a.two) {
    a.o_opacity[2 * p] = a.opacity[2 * i];
    a.o_opacity[2 * p + 1] = a.opacity[2 * i + 1];
  } else {
    a.o_opacity[p] = a.opacity[i];
  }
  if (a.split_dir) copy3(a.split_dir + 3 * i, a.o_split_dir + 3 * p);
  if (side == 0) {
    copy3(mu, a.o_means + 3 * p);
    copy3(ls, a.o_log_scales + 3 * p);
    copy3(eta, a.o_skew + 3 * p);
  } else {
    const int k = ls[1] > ls[0] ? (ls[2] > ls[1] ? 2 : 1) : (ls[2] > ls[0] ? 2 : 0);  // first largest
    // axis k of R(q / |q|) (w, x, y, z)
    const float inv = 1.0f / sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    float ax[3];
    if (k == 0) {
      ax[0] = 1.0f - 2.0f * (y * y + z * z); ax[1] = 2.0f * (x * y + w * z); ax[2] = 2.0f * (x * z - w * y);
    } else if (k == 1) {
      ax[0] = 2.0f * (x * y - w * z); ax[1] = 1.0f - 2.0f * (x * x + z * z); ax[2] = 2.0f * (y * z + w * x);
    } else {
      ax[0] = 2.0f * (x * z + w * y); ax[1] = 2.0f * (y * z - w * x); ax[2] = 1.0f - 2.0f * (x * x + y * y);
    }
    float r2 = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) r2 += j == k ? 0.0f : eta[j] * eta[j];
    const float ek = eta[k];
    const float phi = atan2f(sqrtf(1.0f + r2), side > 0 ? -ek : ek);  // pi x the half's mass
    const float sh = sinf(0.5f * phi);
    const float g = 2.0f * sh * sh * 0.3989422804014327f;  // 2 sin^2(phi/2) / sqrt(2 pi)
    const float x2 = 2.0f * phi;
    float xs;  // x - sin x
    if (x2 < 1.0f) {
      const float t = x2 * x2;
      xs = x2 * t *
           (1.0f / 6.0f - t * (1.0f / 120.0f - t * (1.0f / 5040.0f - t * (1.0f / 362880.0f - t * (1.0f / 39916800.0f)))));
    } else {
      xs = x2 - sinf(x2);
    }
    const float f = xs * 0.15915494309189535f;  // / (2 pi)
    const float pi = 3.14159265358979324f;
    const float m = (side > 0 ? pi : -pi) * g / phi;
    const float v = pi * f / phi - m * m;
    const float sk = expf(ls[k]);
    float* om = a.o_means + 3 * p;
    float* ol = a.o_log_scales + 3 * p;
    float* oe = a.o_skew + 3 * p;
    const float rk = 1.0f / sqrtf(1.0f + ek * ek);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      om[j] = mu[j] + sk * m * ax[j];
      ol[j] = j == k ? ls[k] + 0.5f * logf(v) : ls[j];
      oe[j] = j == k ? 0.0f : eta[j] * rk;
    }
  }
}

// The SH rows (most of the bytes) are copied by the whole block once every
// output of its 1024 Gaussians is placed: consecutive threads take
// consecutive floats (float4s) of consecutive outputs, so reads and writes
// are coalesced.
__global__ void __launch_bounds__(kDenThreads) densify_scatter_kernel(DensifyArgs a) {
  __shared__ unsigned long long s_warp[32];
  __shared__ uint32_t s_src[2 * kDenBlock], s_dst[2 * kDenBlock];
  const int64_t base = (int64_t)blockIdx.x * kDenBlock + (int64_t)threadIdx.x * kDenItems;
  int act[kDenItems];
  unsigned long long w = 0;
#pragma unroll
  for (int j = 0; j < kDenItems; ++j) {
    act[j] = base + j < a.n ? densify_action(a, base + j) : ACT_REMOVE;
    w += action_word(act[j]);
  }
  unsigned long long total;
  const unsigned long long ex = block_exclusive_sum(w, s_warp, total);
  const uint32_t* bo = a.block_sums + 4 * (int64_t)blockIdx.x;
  int64_t keep = bo[0] + (int64_t)(ex & kField);
  int64_t clone = a.counts[0] + bo[1] + (int64_t)((ex >> 21) & kField);
  int64_t split = a.counts[0] + a.counts[1] + 2 * (bo[2] + (int64_t)((ex >> 42) & kField));
  // this thread's first slot in the block's list of (source, output) rows
  int slot = (int)((ex & kField) + ((ex >> 21) & kField) + 2 * ((ex >> 42) & kField));
  const int n_rows = (int)((total & kField) + ((total >> 21) & kField) + 2 * ((total >> 42) & kField));
#pragma unroll
  for (int j = 0; j < kDenItems; ++j) {
    const int64_t i = base + j;
    if (act[j] == ACT_KEEP || act[j] == ACT_CLONE) {
      write_gaussian(a, i, keep, 0);
      if (a.src_map) a.src_map[keep] = (uint32_t)i;
      s_src[slot] = (uint32_t)i;
      s_dst[slot++] = (uint32_t)keep;
      ++keep;
    }
    if (act[j] == ACT_CLONE) {
      write_gaussian(a, i, clone, 0);
      if (a.src_map) a.src_map[clone] = (uint32_t)i | (1u << 30);
      s_src[slot] = (uint32_t)i;
      s_dst[slot++] = (uint32_t)clone;
      ++clone;
    }
    if (act[j] == ACT_SPLIT) {
      write_gaussian(a, i, split, +1);
      write_gaussian(a, i, split + 1, -1);
      if (a.src_map) {
        a.src_map[split] = (uint32_t)i | (2u << 30);
        a.src_map[split + 1] = (uint32_t)i | (3u << 30);
      }
      s_src[slot] = (uint32_t)i;
      s_dst[slot++] = (uint32_t)split;
      s_src[slot] = (uint32_t)i;
      s_dst[slot++] = (uint32_t)(split + 1);
      split += 2;
    }
  }
  __syncthreads();
  if (a.sh_vec4) {
    const int w = a.k3 / 4;
    const float4* s = reinterpret_cast<const float4*>(a.sh);
    float4* d = reinterpret_cast<float4*>(a.o_sh);
    for (int e = threadIdx.x; e < n_rows * w; e += kDenThreads) {
      const int r = e / w, c = e - r * w;
      d[(int64_t)s_dst[r] * w + c] = s[(int64_t)s_src[r] * w + c];
    }
  } else {
    const int w = a.k3;
    for (int e = threadIdx.x; e < n_rows * w; e += kDenThreads) {
      const int r = e / w, c = e - r * w;
      a.o_sh[(int64_t)s_dst[r] * w + c] = a.sh[(int64_t)s_src[r] * w + c];
    }
  }
}

// per-Gaussian state after densification: kept outputs take their source's
// values, new ones (clone copies, children) start at zero
__global__ void __launch_bounds__(256) densify_remap_kernel(const float* __restrict__ in, int width,
                                                            const uint32_t* __restrict__ src_map,
                                                            const int64_t* __restrict__ counts, int64_t cap,
                                                            float* __restrict__ out) {
  const int64_t n_out = counts[3] < cap ? counts[3] : cap;
  const int64_t total = n_out * width;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / width;
    const uint32_t s = src_map[p];
    out[e] = (s >> 30) == 0 ? in[(int64_t)(s & 0x3fffffffu) * width + (e - p * width)] : 0.0f;
  }
}

size_t densify_scratch_bytes(int64_t n) {
  const int64_t nb = (n + kDenBlock - 1) / kDenBlock;
  return (size_t)(nb > 0 ? nb : 1) * 4 * sizeof(uint32_t);
}

cudaError_t launch_densify(const DensifyArgs& a, cudaStream_t st) {
  const int64_t nb = (a.n + kDenBlock - 1) / kDenBlock;
  if (nb > 0) densify_classify_kernel<<<(unsigned)nb, kDenThreads, 0, st>>>(a);
  densify_scan_kernel<<<1, kDenScanThreads, 0, st>>>(a.block_sums, nb, a.counts);
  if (nb > 0) densify_scatter_kernel<<<(unsigned)nb, kDenThreads, 0, st>>>(a);
  count_launches(nb > 0 ? 3 : 1);
  return cudaGetLastError();
}

cudaError_t launch_densify_remap(const float* in, int width, const uint32_t* src_map, const int64_t* counts,
                                 int64_t cap, float* out, int sms, cudaStream_t st) {
  if (cap == 0 || width == 0) return cudaSuccess;
  const int64_t total = cap * width;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)sms * 8));
  densify_remap_kernel<<<grid, 256, 0, st>>>(in, width, src_map, counts, cap, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace sr
