// Per-Gaussian projection (forward) and its chain rule (backward).
//
// Forward, per (view, Gaussian), FP32 (Preliminaries, Eq. 1; Appendix
// "Forward Pass"):
//   t = W mu + t_w (camera z in a fixed FP32 operation order, no FMA: it is
//   the depth sort key), R from q/|q|, M = R diag(exp(log_s)),
//   J = local-affine Jacobian at t with x/z, y/z limited to fov_clamp*tan(fov/2),
//   T = J W M, Sigma' = T T^T, Sigma_d = Sigma' + sI,
//   det Sigma' as a sum of squared 2x2 minors of T (Cauchy-Binet, no
//   cancellation), comp = sqrt(det Sigma' / det Sigma_d), conic = Sigma_d^-1,
//   skew: delta_2 = T eta / sqrt(1+|eta|^2), beta_2 = Sigma_d^-1 delta_2 /
//   sqrt(1 - delta_2^T Sigma_d^-1 delta_2) (skew-normal marginal under the
//   local-affine map), u_2 = beta_2 + P(d) for the split direction,
//   o1, o2 = sigmoid, m = comp (o1+o2)/2, h = comp (o1-o2)/2 (Eq. alpha),
//   rgb = max(0, SH(dir) + 0.5), mu_2 = K t / t_z,
//   conservative footprint: rho0^2 = 2 ln(2 o_max comp / tau),
//   kappa = 1 + erf(rho0 sqrt(beta^T Sigma_d beta) / sqrt 2),
//   rho^2 = 2 ln(kappa o_max comp / tau) (1 + 2^-10),
//   half extents rho sqrt(Sigma_d,xx), rho sqrt(Sigma_d,yy) -> tile range.
// Backward: the adjoint of each of those steps, written out by hand.
#include <algorithm>

#include "kernels.cuh"

namespace sr {

// Real spherical-harmonic normalisation constants (degree <= 3), values of
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the real-form factor.
constexpr float kSH0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kSH1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kSH2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float kSH3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
constexpr float kSH3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float kSH3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
constexpr float kSH3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kSH3e = 1.445305721320277f;    // sqrt(105/pi)/4

template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
  Y[0] = kSH0;
  if (DEG < 1) return;
  Y[1] = -kSH1 * y;
  Y[2] = kSH1 * z;
  Y[3] = -kSH1 * x;
  if (DEG < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kSH2a * x * y;
  Y[5] = -kSH2a * y * z;
  Y[6] = kSH2b * (2.0f * zz - xx - yy);
  Y[7] = -kSH2a * x * z;
  Y[8] = kSH2c * (xx - yy);
  if (DEG < 3) return;
  Y[9] = -kSH3a * y * (3.0f * xx - yy);
  Y[10] = kSH3b * x * y * z;
  Y[11] = -kSH3c * y * (4.0f * zz - xx - yy);
  Y[12] = kSH3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
  Y[13] = -kSH3c * x * (4.0f * zz - xx - yy);
  Y[14] = kSH3e * z * (xx - yy);
  Y[15] = -kSH3a * x * (xx - 3.0f * yy);
}

// d/d(x,y,z) of sum_k gY[k] Y_k, the polynomials above.
// d colour / d direction of all three channels at once: J[ch][d] = sum_k
// sh[3 k + ch] dY_k / d dir_d (sh_grad with the three channels sharing the
// basis derivatives)
template <int DEG>
__device__ __forceinline__ void sh_grad3(float x, float y, float z, const float* sh, float (&J)[3][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) J[c][0] = J[c][1] = J[c][2] = 0.0f;
  if (DEG < 1) return;
  { const float e = -kSH1; J[0][1] += e * sh[3]; J[1][1] += e * sh[4]; J[2][1] += e * sh[5]; }
  { const float e = kSH1; J[0][2] += e * sh[6]; J[1][2] += e * sh[7]; J[2][2] += e * sh[8]; }
  { const float e = -kSH1; J[0][0] += e * sh[9]; J[1][0] += e * sh[10]; J[2][0] += e * sh[11]; }
  if (DEG < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  { const float e = kSH2a * y; J[0][0] += e * sh[12]; J[1][0] += e * sh[13]; J[2][0] += e * sh[14]; }
  { const float e = kSH2a * x; J[0][1] += e * sh[12]; J[1][1] += e * sh[13]; J[2][1] += e * sh[14]; }
  { const float e = -kSH2a * z; J[0][1] += e * sh[15]; J[1][1] += e * sh[16]; J[2][1] += e * sh[17]; }
  { const float e = -kSH2a * y; J[0][2] += e * sh[15]; J[1][2] += e * sh[16]; J[2][2] += e * sh[17]; }
  { const float e = -2.0f * kSH2b * x; J[0][0] += e * sh[18]; J[1][0] += e * sh[19]; J[2][0] += e * sh[20]; }
  { const float e = -2.0f * kSH2b * y; J[0][1] += e * sh[18]; J[1][1] += e * sh[19]; J[2][1] += e * sh[20]; }
  { const float e = 4.0f * kSH2b * z; J[0][2] += e * sh[18]; J[1][2] += e * sh[19]; J[2][2] += e * sh[20]; }
  { const float e = -kSH2a * z; J[0][0] += e * sh[21]; J[1][0] += e * sh[22]; J[2][0] += e * sh[23]; }
  { const float e = -kSH2a * x; J[0][2] += e * sh[21]; J[1][2] += e * sh[22]; J[2][2] += e * sh[23]; }
  { const float e = 2.0f * kSH2c * x; J[0][0] += e * sh[24]; J[1][0] += e * sh[25]; J[2][0] += e * sh[26]; }
  { const float e = -2.0f * kSH2c * y; J[0][1] += e * sh[24]; J[1][1] += e * sh[25]; J[2][1] += e * sh[26]; }
  if (DEG < 3) return;
  { const float e = -6.0f * kSH3a * x * y; J[0][0] += e * sh[27]; J[1][0] += e * sh[28]; J[2][0] += e * sh[29]; }
  { const float e = -kSH3a * (3.0f * xx - 3.0f * yy); J[0][1] += e * sh[27]; J[1][1] += e * sh[28]; J[2][1] += e * sh[29]; }
  { const float e = kSH3b * y * z; J[0][0] += e * sh[30]; J[1][0] += e * sh[31]; J[2][0] += e * sh[32]; }
  { const float e = kSH3b * x * z; J[0][1] += e * sh[30]; J[1][1] += e * sh[31]; J[2][1] += e * sh[32]; }
  { const float e = kSH3b * x * y; J[0][2] += e * sh[30]; J[1][2] += e * sh[31]; J[2][2] += e * sh[32]; }
  { const float e = 2.0f * kSH3c * x * y; J[0][0] += e * sh[33]; J[1][0] += e * sh[34]; J[2][0] += e * sh[35]; }
  { const float e = -kSH3c * (4.0f * zz - xx - 3.0f * yy); J[0][1] += e * sh[33]; J[1][1] += e * sh[34]; J[2][1] += e * sh[35]; }
  { const float e = -8.0f * kSH3c * y * z; J[0][2] += e * sh[33]; J[1][2] += e * sh[34]; J[2][2] += e * sh[35]; }
  { const float e = -6.0f * kSH3d * x * z; J[0][0] += e * sh[36]; J[1][0] += e * sh[37]; J[2][0] += e * sh[38]; }
  { const float e = -6.0f * kSH3d * y * z; J[0][1] += e * sh[36]; J[1][1] += e * sh[37]; J[2][1] += e * sh[38]; }
  { const float e = kSH3d * (6.0f * zz - 3.0f * xx - 3.0f * yy); J[0][2] += e * sh[36]; J[1][2] += e * sh[37]; J[2][2] += e * sh[38]; }
  { const float e = -kSH3c * (4.0f * zz - 3.0f * xx - yy); J[0][0] += e * sh[39]; J[1][0] += e * sh[40]; J[2][0] += e * sh[41]; }
  { const float e = 2.0f * kSH3c * x * y; J[0][1] += e * sh[39]; J[1][1] += e * sh[40]; J[2][1] += e * sh[41]; }
  { const float e = -8.0f * kSH3c * x * z; J[0][2] += e * sh[39]; J[1][2] += e * sh[40]; J[2][2] += e * sh[41]; }
  { const float e = 2.0f * kSH3e * x * z; J[0][0] += e * sh[42]; J[1][0] += e * sh[43]; J[2][0] += e * sh[44]; }
  { const float e = -2.0f * kSH3e * y * z; J[0][1] += e * sh[42]; J[1][1] += e * sh[43]; J[2][1] += e * sh[44]; }
  { const float e = kSH3e * (xx - yy); J[0][2] += e * sh[42]; J[1][2] += e * sh[43]; J[2][2] += e * sh[44]; }
  { const float e = -kSH3a * (3.0f * xx - 3.0f * yy); J[0][0] += e * sh[45]; J[1][0] += e * sh[46]; J[2][0] += e * sh[47]; }
  { const float e = 6.0f * kSH3a * x * y; J[0][1] += e * sh[45]; J[1][1] += e * sh[46]; J[2][1] += e * sh[47]; }
}


struct Attr {
  float mu[3], ls[3], qr[4], eta[3], dsp[3];
  float l1, l2;
};

// Everything the forward computes for one (view, Gaussian); the backward
// recomputes it rather than storing it.
struct Proj {
  float t[3];
  float inv_qn, q[4];
  float R[3][3];
  float s[3];
  float WM[3][3];
  float txz, tyz;
  bool clx, cly;
  float J00, J02, J11, J12;
  float T[2][3];
  float sxx, sxy, syy;
  float m01, m02, m12;
  float detS, detD, comp;
  float a, b, c;
  // skew and split projections
  float nrm_e, v_e[3], del_e[2], w_e[2], r_e;
  float nrm_d, v_d[3], del_d[2], w_d[2], r_d;
  float beta[2], ud[2];
  float o1, o2;
  float dir[3], dlen;
  float mx, my;
};

__device__ __forceinline__ float depth_key_f32(const sr_camera& c, const float* mu) {
  // ((w20 x + w21 y) + w22 z) + w23, each operation rounded, no contraction
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.w2c[8], mu[0]), __fmul_rn(c.w2c[9], mu[1])),
                             __fmul_rn(c.w2c[10], mu[2])),
                   c.w2c[11]);
}

__device__ __forceinline__ float sigmoidf(float x) { return 1.0f / (1.0f + expf(-x)); }

// skew-normal marginal of a local-frame skew vector e (see file header)
__device__ __forceinline__ void skew_project(const Proj& P, const float* e, float& nrm, float* v, float* del, float* w,
                                             float& r, float* out) {
  nrm = 1.0f / sqrtf(1.0f + e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  v[0] = e[0] * nrm;
  v[1] = e[1] * nrm;
  v[2] = e[2] * nrm;
  del[0] = P.T[0][0] * v[0] + P.T[0][1] * v[1] + P.T[0][2] * v[2];
  del[1] = P.T[1][0] * v[0] + P.T[1][1] * v[1] + P.T[1][2] * v[2];
  w[0] = P.a * del[0] + P.b * del[1];
  w[1] = P.b * del[0] + P.c * del[1];
  const float q = del[0] * w[0] + del[1] * w[1];
  r = 1.0f / sqrtf(fmaxf(1.0f - q, 1e-12f));
  out[0] = w[0] * r;
  out[1] = w[1] * r;
}

__device__ __forceinline__ void project(const Attr& A, const sr_camera& c, const CfgDev& cfg, bool two_opac,
                                        bool has_split, Proj& P) {
  const float* W = c.w2c;
  P.t[0] = W[0] * A.mu[0] + W[1] * A.mu[1] + W[2] * A.mu[2] + W[3];
  P.t[1] = W[4] * A.mu[0] + W[5] * A.mu[1] + W[6] * A.mu[2] + W[7];
  P.t[2] = depth_key_f32(c, A.mu);

  const float qn2 = A.qr[0] * A.qr[0] + A.qr[1] * A.qr[1] + A.qr[2] * A.qr[2] + A.qr[3] * A.qr[3];
  P.inv_qn = 1.0f / sqrtf(qn2);
  for (int k = 0; k < 4; ++k) P.q[k] = A.qr[k] * P.inv_qn;
  const float w = P.q[0], x = P.q[1], y = P.q[2], z = P.q[3];
  P.R[0][0] = 1.0f - 2.0f * (y * y + z * z);
  P.R[0][1] = 2.0f * (x * y - w * z);
  P.R[0][2] = 2.0f * (x * z + w * y);
  P.R[1][0] = 2.0f * (x * y + w * z);
  P.R[1][1] = 1.0f - 2.0f * (x * x + z * z);
  P.R[1][2] = 2.0f * (y * z - w * x);
  P.R[2][0] = 2.0f * (x * z - w * y);
  P.R[2][1] = 2.0f * (y * z + w * x);
  P.R[2][2] = 1.0f - 2.0f * (x * x + y * y);
  for (int j = 0; j < 3; ++j) P.s[j] = expf(A.ls[j]);
  // WM = W_rot (R diag(s))
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      P.WM[i][j] = (W[4 * i + 0] * P.R[0][j] + W[4 * i + 1] * P.R[1][j] + W[4 * i + 2] * P.R[2][j]) * P.s[j];

  const float tz = P.t[2];
  const float limx = cfg.fov_clamp * c.tan_fovx, limy = cfg.fov_clamp * c.tan_fovy;
  const float rx = P.t[0] / tz, ry = P.t[1] / tz;
  P.clx = !(fabsf(rx) <= limx);
  P.cly = !(fabsf(ry) <= limy);
  P.txz = fminf(fmaxf(rx, -limx), limx);
  P.tyz = fminf(fmaxf(ry, -limy), limy);
  P.J00 = c.fx / tz;
  P.J02 = -c.fx * P.txz / tz;
  P.J11 = c.fy / tz;
  P.J12 = -c.fy * P.tyz / tz;
  for (int j = 0; j < 3; ++j) {
    P.T[0][j] = P.J00 * P.WM[0][j] + P.J02 * P.WM[2][j];
    P.T[1][j] = P.J11 * P.WM[1][j] + P.J12 * P.WM[2][j];
  }
  P.sxx = P.T[0][0] * P.T[0][0] + P.T[0][1] * P.T[0][1] + P.T[0][2] * P.T[0][2];
  P.sxy = P.T[0][0] * P.T[1][0] + P.T[0][1] * P.T[1][1] + P.T[0][2] * P.T[1][2];
  P.syy = P.T[1][0] * P.T[1][0] + P.T[1][1] * P.T[1][1] + P.T[1][2] * P.T[1][2];
  P.m01 = P.T[0][0] * P.T[1][1] - P.T[0][1] * P.T[1][0];
  P.m02 = P.T[0][0] * P.T[1][2] - P.T[0][2] * P.T[1][0];
  P.m12 = P.T[0][1] * P.T[1][2] - P.T[0][2] * P.T[1][1];
  P.detS = P.m01 * P.m01 + P.m02 * P.m02 + P.m12 * P.m12;
  const float sd = cfg.dilation;
  P.detD = P.detS + sd * (P.sxx + P.syy) + sd * sd;
  P.comp = cfg.antialias ? sqrtf(P.detS / P.detD) : 1.0f;
  const float inv = 1.0f / P.detD;
  P.a = (P.syy + sd) * inv;
  P.b = -P.sxy * inv;
  P.c = (P.sxx + sd) * inv;

  skew_project(P, A.eta, P.nrm_e, P.v_e, P.del_e, P.w_e, P.r_e, P.beta);
  if (has_split) {
    skew_project(P, A.dsp, P.nrm_d, P.v_d, P.del_d, P.w_d, P.r_d, P.ud);
  } else {
    P.ud[0] = P.ud[1] = 0.0f;
  }
  P.o1 = sigmoidf(A.l1);
  P.o2 = two_opac ? sigmoidf(A.l2) : P.o1;

  const float d0 = A.mu[0] - c.campos[0], d1 = A.mu[1] - c.campos[1], d2 = A.mu[2] - c.campos[2];
  P.dlen = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  const float il = 1.0f / P.dlen;
  P.dir[0] = d0 * il;
  P.dir[1] = d1 * il;
  P.dir[2] = d2 * il;
  P.mx = c.fx * P.t[0] / tz + c.cx;
  P.my = c.fy * P.t[1] / tz + c.cy;
}

// three consecutive elements of a storage-typed array, the three loads in
// one branch of the (warp-uniform) type switch so they issue back to back
__device__ __forceinline__ void ld3_dyn(const void* p, int dt, int64_t i, float* out) {
  if (dt == SR_F32) {
    const float* f = static_cast<const float*>(p) + i;
    const float x = __ldg(f), y = __ldg(f + 1), z = __ldg(f + 2);
    out[0] = x; out[1] = y; out[2] = z;
  } else if (dt == SR_BF16) {
    const __nv_bfloat16* h = static_cast<const __nv_bfloat16*>(p) + i;
    const __nv_bfloat16 x = h[0], y = h[1], z = h[2];
    out[0] = __bfloat162float(x); out[1] = __bfloat162float(y); out[2] = __bfloat162float(z);
  } else {
    const __half* h = static_cast<const __half*>(p) + i;
    const __half x = h[0], y = h[1], z = h[2];
    out[0] = __half2float(x); out[1] = __half2float(y); out[2] = __half2float(z);
  }
}

__device__ __forceinline__ void load_attr(const sr_gaussians& g, int64_t i, bool has_split, Attr& A) {
  const float* means = static_cast<const float*>(g.means);
  A.mu[0] = __ldg(means + 3 * i);
  A.mu[1] = __ldg(means + 3 * i + 1);
  A.mu[2] = __ldg(means + 3 * i + 2);
  ld3_dyn(g.log_scales, g.dt_scale, 3 * i, A.ls);
  const float4 q = __ldg(reinterpret_cast<const float4*>(g.quats) + i);
  A.qr[0] = q.x;
  A.qr[1] = q.y;
  A.qr[2] = q.z;
  A.qr[3] = q.w;
  const float* op = static_cast<const float*>(g.opacity_logits);
  if (g.two_opacities) {
    A.l1 = __ldg(op + 2 * i);
    A.l2 = __ldg(op + 2 * i + 1);
  } else {
    A.l1 = __ldg(op + i);
    A.l2 = A.l1;
  }
  ld3_dyn(g.skew, g.dt_skew, 3 * i, A.eta);
  if (has_split) {
    ld3_dyn(g.split_dir, g.dt_skew, 3 * i, A.dsp);
  } else {
    A.dsp[0] = A.dsp[1] = A.dsp[2] = 0.0f;
  }
}


// View table from the cameras (one thread); same layout rule as sr_plan_init.
__device__ void write_view_table(const sr_camera* cams, int n_views, ViewInfo* views) {
  int64_t tb = 0, io = 0, po = 0;
  for (int v = 0; v < n_views; ++v) {
    ViewInfo vi;
    vi.width = cams[v].width;
    vi.height = cams[v].height;
    vi.tiles_x = (vi.width + kTile - 1) / kTile;
    vi.tiles_y = (vi.height + kTile - 1) / kTile;
    vi.tile_base = tb;
    vi.image_offset = io;
    vi.pixel_offset = po;
    vi.pad = 0;
    views[v] = vi;
    tb += (int64_t)vi.tiles_x * vi.tiles_y;
    io += 3 * (int64_t)vi.width * vi.height;
    po += (int64_t)vi.width * vi.height;
  }
}

// only for frames without Gaussians (the projection writes the table otherwise)
__global__ void view_table_kernel(const sr_camera* cams, int n_views, ViewInfo* views) {
  pdl_entry();
  if (threadIdx.x == 0 && blockIdx.x == 0) write_view_table(cams, n_views, views);
}

// Block shape of the per-Gaussian kernels: 4 warps; each warp takes 32
// consecutive Gaussians at a time and stages their SH coefficients through a
// padded shared-memory tile (row = 3K + 1 floats, so lane l reading its own
// row is conflict-free), which turns the per-thread 3K-float strided loads
// into coalesced ones.
constexpr int kPreThreads = 128;
constexpr int kPreWarps = kPreThreads / 32;

__host__ __device__ constexpr size_t cams_bytes(int n_views) { return (sizeof(sr_camera) * n_views + 15) & ~size_t(15); }

template <int K3, int DT_SH>
__device__ __forceinline__ void stage_sh(const void* sh, int64_t base, int cnt, float* s, int lane) {
  const int64_t off = base * K3;
  if (cnt == 32) {
    // a full group: every load is issued before the first store, so the
    // group's K3 coalesced loads wait on one memory latency, not K3
    float v[K3];
#pragma unroll
    for (int i = 0; i < K3; ++i) v[i] = ld<DT_SH>(sh, off + lane + 32 * i);
#pragma unroll
    for (int i = 0; i < K3; ++i) {
      const int w = lane + 32 * i, g = w / K3, k = w - g * K3;
      s[g * (K3 + 1) + k] = v[i];
    }
    return;
  }
  for (int w = lane; w < cnt * K3; w += 32) {
    const int g = w / K3, k = w - g * K3;
    s[g * (K3 + 1) + k] = ld<DT_SH>(sh, off + w);
  }
}

// 4 blocks per SM (up to 128 registers): room to hold the attributes while the
// SH tile's loads are in flight, without spills (5 blocks at 96 registers spill
// and wait on the two loads one after the other)
template <int DEG, int DT_SH>
__global__ void __launch_bounds__(kPreThreads, 4) preprocess_fwd_kernel(PreArgs a) {
  pdl_entry();
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int K3 = 3 * K, ROW = K3 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sr_camera* s_cams = reinterpret_cast<sr_camera*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_sh = reinterpret_cast<float*>(smem_raw + cams_bytes(a.n_views)) + warp * 32 * ROW;
  for (int v = threadIdx.x; v < a.n_views; v += blockDim.x) s_cams[v] = a.cams[v];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    write_view_table(a.cams, a.n_views, a.ws.views);
    a.ws.status->d2_fresh = a.d2 ? 1u : 0u;
  }
  __syncthreads();
  const int64_t n = a.g.n;
  const bool has_split = a.g.split_dir != nullptr;
  const bool two = a.g.two_opacities != 0;
  const float tau = a.cfg.alpha_min;
  for (int64_t base = ((int64_t)blockIdx.x * kPreWarps + warp) * 32; base < n;
       base += (int64_t)gridDim.x * kPreWarps * 32) {
    const int cnt = (int)(n - base < 32 ? n - base : 32);
    const int64_t i = base + lane;
    // the attribute loads go out before the SH loads, so both wait on one
    // memory latency (the SH tile's stores and the warp barrier come after)
    Attr A;
    if (lane < cnt) load_attr(a.g, i, has_split, A);
    stage_sh<K3, DT_SH>(a.g.sh, base, cnt, s_sh, lane);
    __syncwarp();
    const float* sh = s_sh + lane * ROW;
    if (lane < cnt) {

    for (int v = 0; v < a.n_views; ++v) {
      const sr_camera& c = s_cams[v];
      const int64_t m = (int64_t)v * n + i;
      const float tz = depth_key_f32(c, A.mu);
      a.ws.depth[m] = __float_as_uint(tz);
      uint32_t ntouch = 0;
      uint2 rect = make_uint2(0u, 0u);
      if (tz > a.cfg.near_z) {
        Proj P;
        project(A, c, a.cfg, two, has_split, P);
        const float omax = P.comp * fmaxf(P.o1, P.o2);
        bool on = 2.0f * omax >= tau;
        float kappa = 1.0f;
        if (on) {
          const float rho0sq = 2.0f * logf(2.0f * omax / tau);
          const float bx = P.beta[0], by = P.beta[1];
          const float dxx = P.sxx + a.cfg.dilation, dyy = P.syy + a.cfg.dilation;
          const float bsb = fmaxf(bx * (bx * dxx + 2.0f * by * P.sxy) + by * by * dyy, 0.0f);
          kappa = 1.0f + erff(sqrtf(rho0sq * bsb) * kInvSqrt2);
          on = kappa * omax >= tau;
          if (on) {
            const float rho2 = 2.0f * logf(kappa * omax / tau) * (1.0f + 1.0f / 1024.0f);
            const float ex = sqrtf(rho2 * dxx), ey = sqrtf(rho2 * dyy);
            float xlo = ceilf(P.mx - ex - 0.5f), xhi = floorf(P.mx + ex - 0.5f);
            float ylo = ceilf(P.my - ey - 0.5f), yhi = floorf(P.my + ey - 0.5f);
            xlo = fmaxf(xlo, 0.0f);
            ylo = fmaxf(ylo, 0.0f);
            xhi = fminf(xhi, (float)(c.width - 1));
            yhi = fminf(yhi, (float)(c.height - 1));
            if (xlo <= xhi && ylo <= yhi) {
              const uint32_t tx0 = (uint32_t)xlo / kTile, tx1 = (uint32_t)xhi / kTile + 1;
              const uint32_t ty0 = (uint32_t)ylo / kTile, ty1 = (uint32_t)yhi / kTile + 1;
              rect = make_uint2(tx0 | (ty0 << 16), tx1 | (ty1 << 16));
              // exact footprint / tile test, row by row (row_tile_span): E1 ...
              const float4 f0 = make_float4(P.sxy / dyy, P.detD / dyy, sqrtf(rho2) * P.sxy / sqrtf(dxx), ey);
              float4 f1 = make_float4(rho2, 1.0f / dyy, 0.0f, 0.0f);
              // ... and E2, the smaller ellipse on the side beta^T d < 0, with
              // conic Sigma_d^-1 + beta beta^T (determinant (1 + bsb) / det Sigma_d)
              const float rho2m = 2.0f * logf(omax / tau) * (1.0f + 1.0f / 1024.0f);
              float4 f2 = make_float4(0.0f, 0.0f, 0.0f, -1.0f);  // ymax < 0: empty
              const float side = bx > 0.0f ? 1.0f : bx < 0.0f ? -1.0f : by > 0.0f ? 2.0f : by < 0.0f ? -2.0f : 0.0f;
              // the slope stays finite (a huge slope and a zero height must not make a NaN)
              float4 f3 = make_float4(0.0f, 0.0f, bx != 0.0f ? fminf(fmaxf(-by / bx, -1e30f), 1e30f) : 0.0f, side);
              if (rho2m > 0.0f && (bx != 0.0f || by != 0.0f)) {
                const float a2 = P.a + bx * bx, b2 = P.b + bx * by, c2 = P.c + by * by;
                const float det2 = (1.0f + bsb) / P.detD;
                f2 = make_float4(-b2 / a2, 1.0f / a2, -sqrtf(rho2m) * b2 / sqrtf(c2 * det2), sqrtf(rho2m * a2 / det2));
                f3.x = rho2m;
                f3.y = det2 / a2;
              }
              const uint32_t nrows = ty1 - ty0;
              bool packed = nrows <= (uint32_t)kSpanRows;
              uint32_t cum_lo = 0u, cum_hi = 0u, firsts = 0u;
              for (uint32_t ty = ty0; ty < ty1; ++ty) {
                const uint32_t rr = ty - ty0;
                if (packed) {  // this row's exclusive prefix (checked <= 255 below)
                  const uint32_t c8 = min(ntouch, 255u) << (8 * (rr & 3));
                  if (rr < 4) cum_lo |= c8; else cum_hi |= c8;
                }
                int lo, hi;
                if (row_tile_span(f0, f1, f2, f3, P.mx, P.my, (int)ty, c.width, c.height, lo, hi)) {
                  ntouch += (uint32_t)(hi - lo + 1);
                  const uint32_t first = (uint32_t)(lo - (int)tx0);
                  packed = packed && first <= 15u;
                  if (packed) firsts |= first << (4 * rr);
                }
              }
              packed = packed && ntouch <= 255u;
              if (packed) {  // rows below the box never own a key
                if (nrows < 4) {
                  cum_lo |= 0xffffffffu << (8 * nrows);
                  cum_hi = 0xffffffffu;
                } else if (nrows < 8) {
                  cum_hi |= 0xffffffffu << (8 * (nrows - 4));
                }
              }
              a.ws.foot[4 * m + 1] =
                  packed ? make_float4(__uint_as_float(cum_lo), __uint_as_float(cum_hi), __uint_as_float(firsts),
                                       __uint_as_float(kSpansPacked))
                         : make_float4(f1.x, f1.y, 0.0f, __uint_as_float(kSpansTall));
              if (!packed) {  // the emission enumerates the rows again
                a.ws.foot[4 * m] = f0;
                a.ws.foot[4 * m + 2] = f2;
                a.ws.foot[4 * m + 3] = f3;
              }
            }
          }
        }
        if (ntouch) {
          float Y[16];
          sh_eval<DEG>(P.dir[0], P.dir[1], P.dir[2], Y);
          float rgb[3];
          uint32_t clamped = 0u;
#pragma unroll
          for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) acc += Y[k] * sh[3 * k + ch];
            rgb[ch] = fmaxf(acc, 0.0f);
            clamped |= (acc < 0.0f ? 1u : 0u) << ch;
          }
          if (a.ws.shjac) {
            // per channel: d colour / d direction (the backward's view-direction
            // term, so it need not read the SH coefficients) and the clamp flag
            float4* jp = a.ws.shjac + 3 * m;
            float J[3][3];
            sh_grad3<DEG>(P.dir[0], P.dir[1], P.dir[2], sh, J);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch)
              jp[ch] = make_float4(J[ch][0], J[ch][1], J[ch][2], (clamped >> ch) & 1u ? 1.0f : 0.0f);
          }
          const float m_ = P.comp * (P.o1 + P.o2) * 0.5f;
          const float h_ = P.comp * (P.o1 - P.o2) * 0.5f;
          // alpha >= tau implies P2 >= log2(tau / (kappa o_max)); a small margin
          // keeps the early rejection strictly inside the exact bound
          const float thr = log2f(tau / (kappa * omax)) - 0.01f;
          float4* r = a.ws.rec + 4 * m;
          r[0] = make_float4(P.mx, P.my, -0.5f * kLog2e * P.a, -kLog2e * P.b);
          r[1] = make_float4(-0.5f * kLog2e * P.c, P.beta[0] * kInvSqrt2, P.beta[1] * kInvSqrt2, m_);
          r[2] = make_float4(h_, (P.beta[0] + P.ud[0]) * kInvSqrt2, (P.beta[1] + P.ud[1]) * kInvSqrt2, 0.0f);
          r[3] = make_float4(rgb[0], rgb[1], rgb[2], thr);
          if (a.d2) {  // the record's 2D gradients start at zero for the backward
            float4* z = a.d2 + 4 * m;
            z[0] = z[1] = z[2] = z[3] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          }
        }
      }
      a.ws.ntouch[m] = ntouch;
      a.ws.rect[m] = rect;
      a.ws.dkey[0][m] = ntouch ? __float_as_uint(tz) : 0xffffffffu;
    }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------

// adjoint of skew_project: given g_out = dL/d(out), accumulate dL/d(conic)
// into (ga, gb, gc), dL/dT into gT, and return dL/de in ge.
__device__ __forceinline__ void skew_project_bwd(const Proj& P, const float* e, float nrm, const float* v,
                                                 const float* del, const float* w, float r, const float* g_out,
                                                 float& ga, float& gb, float& gc, float gT[2][3], float* ge) {
  // out = r w, r = (1 - q)^(-1/2), q = del . w, w = A del, del = T v, v = e nrm
  float gw0 = r * g_out[0], gw1 = r * g_out[1];
  const float gr = g_out[0] * w[0] + g_out[1] * w[1];
  const float gq = gr * 0.5f * r * r * r;
  float gd0 = gq * w[0], gd1 = gq * w[1];
  gw0 += gq * del[0];
  gw1 += gq * del[1];
  ga += gw0 * del[0];
  gb += gw0 * del[1] + gw1 * del[0];
  gc += gw1 * del[1];
  gd0 += P.a * gw0 + P.b * gw1;
  gd1 += P.b * gw0 + P.c * gw1;
  float gv[3];
  for (int j = 0; j < 3; ++j) {
    gT[0][j] += gd0 * v[j];
    gT[1][j] += gd1 * v[j];
    gv[j] = P.T[0][j] * gd0 + P.T[1][j] * gd1;
  }
  const float ev = e[0] * gv[0] + e[1] * gv[1] + e[2] * gv[2];
  const float n3 = nrm * nrm * nrm;
  for (int j = 0; j < 3; ++j) ge[j] = nrm * gv[j] - n3 * ev * e[j];
}

template <int DEG, int DT_SH>
__global__ void __launch_bounds__(kPreThreads, 4) preprocess_bwd_kernel(BwdArgs a) {
  pdl_entry();
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int K3 = 3 * K, ROW = K3 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sr_camera* s_cams = reinterpret_cast<sr_camera*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* s_gsh = reinterpret_cast<float*>(smem_raw + cams_bytes(a.n_views)) + warp * 32 * ROW;
  for (int v = threadIdx.x; v < a.n_views; v += blockDim.x) s_cams[v] = a.cams[v];
  __syncthreads();
  const int64_t n = a.g.n;
  const bool has_split = a.g.split_dir != nullptr;
  const bool two = a.g.two_opacities != 0;
  for (int64_t base = ((int64_t)blockIdx.x * kPreWarps + warp) * 32; base < n;
       base += (int64_t)gridDim.x * kPreWarps * 32) {
    const int cnt = (int)(n - base < 32 ? n - base : 32);
    float* gsh = s_gsh + lane * ROW;
#pragma unroll
    for (int k = 0; k < K3; ++k) gsh[k] = 0.0f;
    __syncwarp();
    const int64_t i = base + lane;
    if (lane < cnt) {
    float g_mu[3] = {0, 0, 0}, g_ls[3] = {0, 0, 0}, g_q[4] = {0, 0, 0, 0}, g_eta[3] = {0, 0, 0},
          g_dsp[3] = {0, 0, 0}, g_l1 = 0.0f, g_l2 = 0.0f, g_abs = 0.0f, g_depth = 0.0f;
    // the attributes, and each view's tile count, 2D gradients and colour
    // Jacobian, are loaded together (one memory latency; what a record that
    // touches no tile loads is dropped)
    Attr A;
    load_attr(a.g, i, has_split, A);
    for (int v = 0; v < a.n_views; ++v) {
      const int64_t m = (int64_t)v * n + i;
      const float4* d2p = reinterpret_cast<const float4*>(a.ws.d2 + kD2Stride * m);
      const uint32_t nt = a.ws.ntouch[m];
      const float4 q0 = d2p[0], q1 = d2p[1], q2 = d2p[2], q3 = d2p[3];
      const float4* jp = a.ws.shjac + 3 * m;
      const float4 J3[3] = {jp[0], jp[1], jp[2]};  // d colour_ch / d direction, clamp flag
      if (nt == 0) continue;
      const float gd[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                            q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
      const sr_camera& c = s_cams[v];
      Proj P;
      project(A, c, a.cfg, two, has_split, P);
      g_abs += sqrtf(gd[G_MX] * gd[G_MX] + gd[G_MY] * gd[G_MY]);
      float gmu_v[3];  // this view's dL/dmu

      // colour -> SH coefficients and view direction: with the forward's
      // d colour / d direction J and clamp bits, the SH coefficients
      // themselves are not needed (d colour / d coefficient is Y)
      float Y[16];
      sh_eval<DEG>(P.dir[0], P.dir[1], P.dir[2], Y);
      float gdir[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float4 J = J3[ch];
        const float gc_ = J.w != 0.0f ? 0.0f : gd[G_R + ch];
#pragma unroll
        for (int k = 0; k < K; ++k) gsh[3 * k + ch] += Y[k] * gc_;
        gdir[0] += gc_ * J.x;
        gdir[1] += gc_ * J.y;
        gdir[2] += gc_ * J.z;
      }
      {
        const float dd = P.dir[0] * gdir[0] + P.dir[1] * gdir[1] + P.dir[2] * gdir[2];
        const float il = 1.0f / P.dlen;
        for (int k = 0; k < 3; ++k) gmu_v[k] = (gdir[k] - P.dir[k] * dd) * il;
      }

      // opacities
      const float gcomp = gd[G_M] * (P.o1 + P.o2) * 0.5f + gd[G_H] * (P.o1 - P.o2) * 0.5f;
      const float go1 = 0.5f * P.comp * (gd[G_M] + gd[G_H]);
      const float go2 = 0.5f * P.comp * (gd[G_M] - gd[G_H]);
      if (two) {
        g_l1 += go1 * P.o1 * (1.0f - P.o1);
        g_l2 += go2 * P.o2 * (1.0f - P.o2);
      } else {
        g_l1 += (go1 + go2) * P.o1 * (1.0f - P.o1);
      }

      // skew vectors: u_2 = beta_2 + P(d)
      float ga = gd[G_A], gb = gd[G_B], gcn = gd[G_C];
      float gT[2][3] = {{0, 0, 0}, {0, 0, 0}};
      const float gbeta[2] = {gd[G_BX] + gd[G_UX], gd[G_BY] + gd[G_UY]};
      float ge[3];
      skew_project_bwd(P, A.eta, P.nrm_e, P.v_e, P.del_e, P.w_e, P.r_e, gbeta, ga, gb, gcn, gT, ge);
      for (int k = 0; k < 3; ++k) g_eta[k] += ge[k];
      if (has_split) {
        const float gu[2] = {gd[G_UX], gd[G_UY]};
        skew_project_bwd(P, A.dsp, P.nrm_d, P.v_d, P.del_d, P.w_d, P.r_d, gu, ga, gb, gcn, gT, ge);
        for (int k = 0; k < 3; ++k) g_dsp[k] += ge[k];
      }

      // conic = Sigma_d^-1: dL/dSigma_d = -A G A with G = [[ga, gb/2], [gb/2, gc]]
      const float hb = 0.5f * gb;
      const float AG00 = P.a * ga + P.b * hb, AG01 = P.a * hb + P.b * gcn;
      const float AG10 = P.b * ga + P.c * hb, AG11 = P.b * hb + P.c * gcn;
      float gsxx = -(AG00 * P.a + AG01 * P.b);
      float gsxy = -2.0f * (AG00 * P.b + AG01 * P.c);
      float gsyy = -(AG10 * P.b + AG11 * P.c);
      // comp = sqrt(detS / detD), detD = detS + s (sxx + syy) + s^2
      if (a.cfg.antialias && P.detS > 0.0f) {
        const float gdetD = -gcomp * P.comp / (2.0f * P.detD);
        const float gdetS = gcomp * P.comp / (2.0f * P.detS) + gdetD;
        gsxx += gdetD * a.cfg.dilation;
        gsyy += gdetD * a.cfg.dilation;
        const float gm01 = 2.0f * P.m01 * gdetS, gm02 = 2.0f * P.m02 * gdetS, gm12 = 2.0f * P.m12 * gdetS;
        gT[0][0] += gm01 * P.T[1][1] + gm02 * P.T[1][2];
        gT[1][1] += gm01 * P.T[0][0] - gm12 * P.T[0][2];
        gT[0][1] += -gm01 * P.T[1][0] + gm12 * P.T[1][2];
        gT[1][0] += -gm01 * P.T[0][1] - gm02 * P.T[0][2];
        gT[1][2] += gm02 * P.T[0][0] + gm12 * P.T[0][1];
        gT[0][2] += -gm02 * P.T[1][0] - gm12 * P.T[1][1];
      }
      // Sigma' = T T^T
      for (int j = 0; j < 3; ++j) {
        const float t0 = P.T[0][j], t1 = P.T[1][j];
        gT[0][j] += 2.0f * gsxx * t0 + gsxy * t1;
        gT[1][j] += 2.0f * gsyy * t1 + gsxy * t0;
      }
      // T = J WM
      float gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0, gWM[3][3];
      for (int j = 0; j < 3; ++j) {
        gJ00 += gT[0][j] * P.WM[0][j];
        gJ02 += gT[0][j] * P.WM[2][j];
        gJ11 += gT[1][j] * P.WM[1][j];
        gJ12 += gT[1][j] * P.WM[2][j];
        gWM[0][j] = gT[0][j] * P.J00;
        gWM[1][j] = gT[1][j] * P.J11;
        gWM[2][j] = gT[0][j] * P.J02 + gT[1][j] * P.J12;
      }
      // WM = W_rot R diag(s)
      const float* W = c.w2c;
      float gR[3][3];
      for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) {
          const float gM = W[0 + k] * gWM[0][j] + W[4 + k] * gWM[1][j] + W[8 + k] * gWM[2][j];
          gR[k][j] = gM * P.s[j];
          g_ls[j] += gM * P.R[k][j] * P.s[j];
        }
      {
        const float w = P.q[0], x = P.q[1], y = P.q[2], z = P.q[3];
        float gq[4];
        gq[0] = 2.0f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
        gq[1] = 2.0f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - 2.0f * x * gR[1][1] - w * gR[1][2] +
                        z * gR[2][0] + w * gR[2][1] - 2.0f * x * gR[2][2]);
        gq[2] = 2.0f * (-2.0f * y * gR[0][0] + x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] -
                        w * gR[2][0] + z * gR[2][1] - 2.0f * y * gR[2][2]);
        gq[3] = 2.0f * (-2.0f * z * gR[0][0] - w * gR[0][1] + x * gR[0][2] + w * gR[1][0] - 2.0f * z * gR[1][1] +
                        y * gR[1][2] + x * gR[2][0] + y * gR[2][1]);
        const float qd = P.q[0] * gq[0] + P.q[1] * gq[1] + P.q[2] * gq[2] + P.q[3] * gq[3];
        for (int k = 0; k < 4; ++k) g_q[k] += (gq[k] - P.q[k] * qd) * P.inv_qn;
      }
      // J(t) and mu_2(t)
      const float tx = P.t[0], ty = P.t[1], tz = P.t[2];
      const float itz = 1.0f / tz, itz2 = itz * itz;
      float gtx = gd[G_MX] * c.fx * itz;
      float gty = gd[G_MY] * c.fy * itz;
      float gtz = -(gd[G_MX] * c.fx * tx + gd[G_MY] * c.fy * ty) * itz2;
      gtz += -gJ00 * c.fx * itz2 - gJ11 * c.fy * itz2;
      gtz += gJ02 * c.fx * P.txz * itz2 + gJ12 * c.fy * P.tyz * itz2;
      const float gtxz = -gJ02 * c.fx * itz, gtyz = -gJ12 * c.fy * itz;
      if (!P.clx) {
        gtx += gtxz * itz;
        gtz -= gtxz * tx * itz2;
      }
      if (!P.cly) {
        gty += gtyz * itz;
        gtz -= gtyz * ty * itz2;
      }
      for (int k = 0; k < 3; ++k) gmu_v[k] += W[0 + k] * gtx + W[4 + k] * gty + W[8 + k] * gtz;
      for (int k = 0; k < 3; ++k) g_mu[k] += gmu_v[k];
      // dL/dz of the centre along this camera's axis: (W dL/dmu)_z (Eq. depth_grad)
      g_depth += W[8] * gmu_v[0] + W[9] * gmu_v[1] + W[10] * gmu_v[2];
    }
    // write (zeros for Gaussians no view touched)
    float* o;
    o = a.out.means + 3 * i;
    o[0] = g_mu[0]; o[1] = g_mu[1]; o[2] = g_mu[2];
    o = a.out.log_scales + 3 * i;
    o[0] = g_ls[0]; o[1] = g_ls[1]; o[2] = g_ls[2];
    reinterpret_cast<float4*>(a.out.quats)[i] = make_float4(g_q[0], g_q[1], g_q[2], g_q[3]);
    if (two) {
      a.out.opacity_logits[2 * i] = g_l1;
      a.out.opacity_logits[2 * i + 1] = g_l2;
    } else {
      a.out.opacity_logits[i] = g_l1;
    }
    o = a.out.skew + 3 * i;
    o[0] = g_eta[0]; o[1] = g_eta[1]; o[2] = g_eta[2];
    if (has_split && a.out.split_dir) {
      o = a.out.split_dir + 3 * i;
      o[0] = g_dsp[0]; o[1] = g_dsp[1]; o[2] = g_dsp[2];
    }
    if (a.out.means2d_abs) a.out.means2d_abs[i] = g_abs;
    if (a.out.depth_grad) a.out.depth_grad[i] = g_depth;
    }
    __syncwarp();
    // SH gradients out of the padded tile with coalesced stores
    const int64_t off = base * K3;
    for (int w = lane; w < cnt * K3; w += 32) {
      const int g = w / K3, k = w - g * K3;
      a.out.sh[off + w] = s_gsh[g * ROW + k];
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class Args>
static cudaError_t launch_sized(void (*fn)(Args), const Args& a, int grid, size_t smem, cudaStream_t st) {
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  launch_pdl(fn, dim3(grid), dim3(kPreThreads), smem, st, a);
  count_launches(1);
  return cudaGetLastError();
}

static int grid_for(int64_t n, int sms) {
  const int64_t blocks = (n + kPreThreads - 1) / kPreThreads;
  const int64_t cap = (int64_t)sms * 16;
  return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

static size_t sh_stage_bytes(int deg, int tiles_per_warp) {
  const int row = 3 * (deg + 1) * (deg + 1) + 1;
  return sizeof(float) * (size_t)kPreWarps * 32 * row * tiles_per_warp;
}

cudaError_t launch_preprocess_fwd(const PreArgs& a, cudaStream_t st, int sms) {
  if (a.g.n == 0) {
    launch_pdl(view_table_kernel, dim3(1), dim3(32), 0, st, a.cams, a.n_views, a.ws.views);
    count_launches(1);
    return cudaGetLastError();
  }
  const int grid = grid_for(a.g.n, sms);
  const size_t smem = cams_bytes(a.n_views) + sh_stage_bytes(a.g.sh_degree, 1);
#define SR_DEG_CASE(D)                                                                              \
  case D:                                                                                           \
    if (a.g.dt_sh == SR_F32) return launch_sized(preprocess_fwd_kernel<D, SR_F32>, a, grid, smem, st);   \
    if (a.g.dt_sh == SR_BF16) return launch_sized(preprocess_fwd_kernel<D, SR_BF16>, a, grid, smem, st); \
    return launch_sized(preprocess_fwd_kernel<D, SR_F16>, a, grid, smem, st);
  switch (a.g.sh_degree) {
    SR_DEG_CASE(0)
    SR_DEG_CASE(1)
    SR_DEG_CASE(2)
    SR_DEG_CASE(3)
  }
#undef SR_DEG_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_preprocess_bwd(const BwdArgs& a, cudaStream_t st, int sms) {
  if (a.g.n == 0) return cudaSuccess;
  const int grid = grid_for(a.g.n, sms);
  const size_t smem = cams_bytes(a.n_views) + sh_stage_bytes(a.g.sh_degree, 1);
#define SR_DEG_CASE(D)                                                                              \
  case D:                                                                                           \
    if (a.g.dt_sh == SR_F32) return launch_sized(preprocess_bwd_kernel<D, SR_F32>, a, grid, smem, st);   \
    if (a.g.dt_sh == SR_BF16) return launch_sized(preprocess_bwd_kernel<D, SR_BF16>, a, grid, smem, st); \
    return launch_sized(preprocess_bwd_kernel<D, SR_F16>, a, grid, smem, st);
  switch (a.g.sh_degree) {
    SR_DEG_CASE(0)
    SR_DEG_CASE(1)
    SR_DEG_CASE(2)
    SR_DEG_CASE(3)
  }
#undef SR_DEG_CASE
  return cudaErrorInvalidValue;
}

}  // namespace sr
