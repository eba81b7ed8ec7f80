// FP64 CPU oracle for the skew-Gaussian tile rasterizer.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only the tests, the smoke check and the CPU-baseline leg of
// the benchmark do.  It shares no code, header, table or constant with the
// CUDA library: every formula below is written out again from the paper.
//
// What it computes, and where the paper defines it:
//   * camera set-up: OpenGL->OpenCV alignment M_cv = M_gl * diag(1,-1,-1,1)
//     (Eq. coord_transform, Alg. 3) and the intrinsics K from W, H and the
//     field of view (the K matrix of Sec. "Decoupled Interactive Visual
//     Analytics Engine");
//   * per-Gaussian projection: Sigma = R S S^T R^T from quaternion and scale
//     (Preliminaries, Eq. 1), local-affine (EWA) projection to Sigma'
//     (Preliminaries), dilation Sigma'+sI with the compensation
//     sqrt(det Sigma' / det(Sigma'+sI)) and the conic (a,b,c)
//     (Appendix "Forward Pass", the alpha expansion and the (a,b,c,d)
//     definitions), the projected skew vector (beta_x, beta_y) (Alg. 1
//     inputs; the 3D->2D rule is the skew-normal marginal, see below), the
//     enhanced opacity o(x) (Eq. alpha, second form) and the SH colour
//     (Preliminaries);
//   * the per-pixel skew kernel alpha = d * G'(x) * (1 + erf(z)) (Alg. 1,
//     Appendix alpha expansion) and front-to-back compositing
//     C = sum_i c_i alpha_i prod_{j<i}(1-alpha_j) (Eq. 2, Eq. color);
//   * gradients: the plain derivative of that composite, dC/dalpha_k
//     (Appendix "Backward Pass", dL/dalpha_k), and of alpha and of the
//     projection with respect to every attribute, obtained by forward-mode
//     dual numbers applied to the same definitions (the paper defers the
//     projection backward to 3DGS: Appendix "Backward Pass").
//
// Readings where the paper is silent or ambiguous (kept identical on the
// CUDA side, and pinned by tests against mathematics rather than code):
//   * skew projection: with the stored skew eta in the Gaussian's standardised
//     local frame, the 3D skew normal has delta_3 = R S eta / sqrt(1+|eta|^2);
//     under the local-affine camera delta_2 = T eta / sqrt(1+|eta|^2) with
//     T = J W R S, and beta_2 = Sd^-1 delta_2 / sqrt(1 - delta_2^T Sd^-1 delta_2)
//     (closure of the skew-normal family under linear maps, Azzalini &
//     Capitanio 1999).  Dilation adds independent N(0, sI).
//   * factor 2: alpha uses (1 + erf z) = 2 Phi, as in Alg. 1.
//   * footprint: conservative ellipse rho^2 = 2 ln(kappa o_max comp / tau)
//     with kappa = 1 + erf(rho0 sqrt(beta^T Sd beta) / sqrt 2),
//     rho0^2 = 2 ln(2 o_max comp / tau), enlarged by (1 + 2^-10).
//   * depth order key: FP32 camera z computed as ((w20 x + w21 y) + w22 z) + w23
//     with every operation rounded to FP32 and no fused multiply-add; ties
//     broken by Gaussian index.
//   * alpha is clamped to alpha_max, gated by alpha_min, and the Gaussian whose
//     transmittance would fall below T_stop is not blended (stop before it).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

struct OrCamera {            // values are the FP32-rounded camera, held in FP64
  double w2c[12];            // row-major 3x4 world-to-camera (OpenCV: +Z forward, +Y down)
  double fx, fy, cx, cy;     // intrinsics K
  double tan_fovx, tan_fovy; // tan(FoV/2)
  double campos[3];          // camera centre in world space
  int32_t width, height;
};

struct OrConfig {
  int32_t tile_w, tile_h;
  double alpha_min, alpha_max, t_stop, dilation, fov_clamp, near_z;
  double bg[3];
  int32_t antialias_comp;
  int32_t pad_;
};

struct OrScene {
  int64_t n;
  const double* means;       // [n,3]
  const double* log_scales;  // [n,3]
  const double* quats;       // [n,4] (w,x,y,z), not normalised
  const double* opac;        // [n] or [n,2] logits
  const double* skew;        // [n,3] eta
  const double* split;       // [n,3] or null
  const double* sh;          // [n,K,3]
  int32_t two_opac;
  int32_t sh_degree;
};

}  // extern "C"

namespace {

// ---------------------------------------------------------------------------
// Forward-mode dual numbers.  Used only to differentiate the definitions
// below; D is the number of seeded input directions.
// ---------------------------------------------------------------------------
template <int D>
struct Dual {
  double v;
  double d[D];
  Dual() : v(0.0) { std::fill(d, d + D, 0.0); }
  Dual(double x) : v(x) { std::fill(d, d + D, 0.0); }  // NOLINT: implicit constant
};

template <int D> Dual<D> operator+(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r(a.v + b.v); for (int i = 0; i < D; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int D> Dual<D> operator-(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r(a.v - b.v); for (int i = 0; i < D; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int D> Dual<D> operator-(const Dual<D>& a) {
  Dual<D> r(-a.v); for (int i = 0; i < D; ++i) r.d[i] = -a.d[i]; return r; }
template <int D> Dual<D> operator*(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r(a.v * b.v); for (int i = 0; i < D; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int D> Dual<D> operator/(const Dual<D>& a, const Dual<D>& b) {
  Dual<D> r(a.v / b.v);
  for (int i = 0; i < D; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int D> Dual<D> operator+(const Dual<D>& a, double b) { return a + Dual<D>(b); }
template <int D> Dual<D> operator+(double a, const Dual<D>& b) { return Dual<D>(a) + b; }
template <int D> Dual<D> operator-(const Dual<D>& a, double b) { return a - Dual<D>(b); }
template <int D> Dual<D> operator-(double a, const Dual<D>& b) { return Dual<D>(a) - b; }
template <int D> Dual<D> operator*(const Dual<D>& a, double b) { return a * Dual<D>(b); }
template <int D> Dual<D> operator*(double a, const Dual<D>& b) { return Dual<D>(a) * b; }
template <int D> Dual<D> operator/(const Dual<D>& a, double b) { return a / Dual<D>(b); }
template <int D> Dual<D> operator/(double a, const Dual<D>& b) { return Dual<D>(a) / b; }

// chain rule for a scalar function f with value fv and derivative fp at a.v
template <int D> Dual<D> apply(const Dual<D>& a, double fv, double fp) {
  Dual<D> r(fv); for (int i = 0; i < D; ++i) r.d[i] = fp * a.d[i]; return r; }
template <int D> Dual<D> exp(const Dual<D>& a) { double e = std::exp(a.v); return apply(a, e, e); }
template <int D> Dual<D> log(const Dual<D>& a) { return apply(a, std::log(a.v), 1.0 / a.v); }
template <int D> Dual<D> sqrt(const Dual<D>& a) { double s = std::sqrt(a.v); return apply(a, s, 0.5 / s); }
// d/dx erf(x) = 2/sqrt(pi) exp(-x^2)  (Appendix, derivative of erf)
template <int D> Dual<D> erf(const Dual<D>& a) {
  return apply(a, std::erf(a.v), 2.0 / std::sqrt(M_PI) * std::exp(-a.v * a.v)); }

inline double value(double x) { return x; }
template <int D> double value(const Dual<D>& x) { return x.v; }

using std::erf;
using std::exp;
using std::log;
using std::sqrt;

// clamp / max with the derivative of the branch that is taken
template <class S> S clamp_to(const S& x, double lo, double hi) {
  if (value(x) < lo) return S(lo);
  if (value(x) > hi) return S(hi);
  return x;
}
template <class S> S relu(const S& x) { return value(x) < 0.0 ? S(0.0) : x; }
template <class S> S sigmoid(const S& x) { return 1.0 / (1.0 + exp(-x)); }

// ---------------------------------------------------------------------------
// Real spherical harmonics up to degree 3, evaluated on a unit direction.
// Normalisation N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), real form
// sqrt(2) N_lm P_l^|m|(cos th) {cos, sin}(|m| phi) with the Condon-Shortley
// phase, ordered m = -l..l.  Written as polynomials in (x, y, z).
// ---------------------------------------------------------------------------
template <class S>
void sh_basis(int deg, const S& x, const S& y, const S& z, S* Y) {
  const double pi = M_PI;
  Y[0] = S(std::sqrt(1.0 / (4.0 * pi)));
  if (deg < 1) return;
  const double c1 = std::sqrt(3.0 / (4.0 * pi));
  Y[1] = -c1 * y;
  Y[2] = c1 * z;
  Y[3] = -c1 * x;
  if (deg < 2) return;
  const double c2a = 0.5 * std::sqrt(15.0 / pi);
  const double c2b = 0.25 * std::sqrt(5.0 / pi);
  const double c2c = 0.25 * std::sqrt(15.0 / pi);
  Y[4] = c2a * x * y;
  Y[5] = -c2a * y * z;
  Y[6] = c2b * (2.0 * z * z - x * x - y * y);
  Y[7] = -c2a * x * z;
  Y[8] = c2c * (x * x - y * y);
  if (deg < 3) return;
  const double c3a = 0.25 * std::sqrt(35.0 / (2.0 * pi));
  const double c3b = 0.5 * std::sqrt(105.0 / pi);
  const double c3c = 0.25 * std::sqrt(21.0 / (2.0 * pi));
  const double c3d = 0.25 * std::sqrt(7.0 / pi);
  const double c3e = 0.25 * std::sqrt(105.0 / pi);
  Y[9] = -c3a * y * (3.0 * x * x - y * y);
  Y[10] = c3b * x * y * z;
  Y[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
  Y[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
  Y[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
  Y[14] = c3e * z * (x * x - y * y);
  Y[15] = -c3a * x * (x * x - 3.0 * y * y);
}

// Record of one projected Gaussian.  The first NDIFF entries are the 2D
// quantities the per-pixel kernel consumes (and that gradients flow through).
enum {
  R_MX, R_MY,           // projected centre mu_2 (pixels)
  R_A, R_B, R_C,        // conic (Sigma' + sI)^-1 = [[a,b],[b,c]]
  R_BX, R_BY,           // projected skew vector beta_2
  R_M, R_H,             // enhanced opacity o(delta) = m + h erf(u_2^T delta / sqrt 2)
  R_UX, R_UY,           // u_2 = beta_2 + P(d)
  R_CR, R_CG, R_CB,     // colour
  NDIFF,
  R_COMP = NDIFF,       // sqrt(det Sigma' / det(Sigma'+sI))
  R_O1, R_O2,           // base opacities
  R_TZ,                 // FP64 camera z
  R_DXX, R_DXY, R_DYY,  // Sigma' + sI
  NREC
};

constexpr int NPARAM = 18;  // mu 3, log_s 3, quat 4, logits 2, eta 3, d 3
enum { P_MU = 0, P_LS = 3, P_Q = 6, P_L = 10, P_ETA = 12, P_D = 15 };

// FP32 depth key, exactly as specified: every product and sum rounded to
// FP32, no fused multiply-add (this file is compiled with -ffp-contract=off).
inline float depth_f32(const OrCamera& c, const double* mu) {
  volatile float w0 = (float)c.w2c[8], w1 = (float)c.w2c[9], w2 = (float)c.w2c[10], w3 = (float)c.w2c[11];
  volatile float x = (float)mu[0], y = (float)mu[1], z = (float)mu[2];
  volatile float p0 = w0 * x;
  volatile float p1 = w1 * y;
  volatile float s0 = p0 + p1;
  volatile float p2 = w2 * z;
  volatile float s1 = s0 + p2;
  volatile float s2 = s1 + w3;
  return s2;
}

// Projection of one Gaussian (Preliminaries; Appendix "Forward Pass").
// theta holds the NPARAM differentiable attributes; sh the (deg+1)^2 x 3
// colour coefficients (colour is linear in them).  Writes NREC entries.
template <class S>
void project(const S* theta, bool two_opac, bool has_split, const double* sh, int deg,
             const OrCamera& c, const OrConfig& cfg, S* rec, bool colour_clamp = true) {
  const S* mu = theta + P_MU;
  // world -> camera
  S t[3];
  for (int r = 0; r < 3; ++r)
    t[r] = c.w2c[4 * r + 0] * mu[0] + c.w2c[4 * r + 1] * mu[1] + c.w2c[4 * r + 2] * mu[2] + c.w2c[4 * r + 3];

  // rotation from the normalised quaternion (w, x, y, z)
  const S* qq = theta + P_Q;
  S qn = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
  S w = qq[0] / qn, x = qq[1] / qn, y = qq[2] / qn, z = qq[3] / qn;
  S R[3][3] = {
      {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)},
      {2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)},
      {2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)}};
  // M = R S, so Sigma = M M^T = R S S^T R^T (Eq. 1)
  S M[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i][j] = R[i][j] * exp(theta[P_LS + j]);

  // Jacobian of the pinhole projection at t; x/z and y/z limited to the
  // widened frustum (the local-affine approximation of the Preliminaries)
  S txz = clamp_to(t[0] / t[2], -cfg.fov_clamp * c.tan_fovx, cfg.fov_clamp * c.tan_fovx);
  S tyz = clamp_to(t[1] / t[2], -cfg.fov_clamp * c.tan_fovy, cfg.fov_clamp * c.tan_fovy);
  S J[2][3] = {{c.fx / t[2], S(0.0), -c.fx * txz / t[2]},
               {S(0.0), c.fy / t[2], -c.fy * tyz / t[2]}};
  S T[2][3];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      S acc(0.0);
      for (int k = 0; k < 3; ++k) {
        S jw = J[i][0] * c.w2c[0 + k] + J[i][1] * c.w2c[4 + k] + J[i][2] * c.w2c[8 + k];
        acc = acc + jw * M[k][j];
      }
      T[i][j] = acc;
    }
  // Sigma' = T T^T
  S sxx = T[0][0] * T[0][0] + T[0][1] * T[0][1] + T[0][2] * T[0][2];
  S sxy = T[0][0] * T[1][0] + T[0][1] * T[1][1] + T[0][2] * T[1][2];
  S syy = T[1][0] * T[1][0] + T[1][1] * T[1][1] + T[1][2] * T[1][2];
  // dilation, compensation and conic (Appendix alpha expansion)
  S dxx = sxx + cfg.dilation, dxy = sxy, dyy = syy + cfg.dilation;
  S det_s = sxx * syy - sxy * sxy;
  S det_d = dxx * dyy - dxy * dxy;
  S comp = cfg.antialias_comp ? sqrt(relu(det_s) / det_d) : S(1.0);
  S a = dyy / det_d, b = -dxy / det_d, cc = dxx / det_d;

  // projected skew vector of a local-frame skew eta (skew-normal marginal)
  auto skew2d = [&](const S* e, S* out) {
    S nrm = 1.0 / sqrt(1.0 + e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    S d0 = (T[0][0] * e[0] + T[0][1] * e[1] + T[0][2] * e[2]) * nrm;
    S d1 = (T[1][0] * e[0] + T[1][1] * e[1] + T[1][2] * e[2]) * nrm;
    S w0 = a * d0 + b * d1, w1 = b * d0 + cc * d1;
    S q = d0 * w0 + d1 * w1;
    S r = 1.0 / sqrt(1.0 - q);
    out[0] = w0 * r;
    out[1] = w1 * r;
  };
  S beta[2], ud[2] = {S(0.0), S(0.0)};
  skew2d(theta + P_ETA, beta);
  if (has_split) skew2d(theta + P_D, ud);

  // enhanced opacity (Eq. alpha, second form), compensation on both halves
  S o1 = sigmoid(theta[P_L + 0]);
  S o2 = two_opac ? sigmoid(theta[P_L + 1]) : o1;

  // colour from SH at the viewing direction
  S dv[3] = {mu[0] - c.campos[0], mu[1] - c.campos[1], mu[2] - c.campos[2]};
  S dl = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  S Y[16];
  sh_basis(deg, dv[0] / dl, dv[1] / dl, dv[2] / dl, Y);
  const int K = (deg + 1) * (deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    S acc(0.5);
    for (int k = 0; k < K; ++k) acc = acc + sh[3 * k + ch] * Y[k];
    rec[R_CR + ch] = colour_clamp ? relu(acc) : acc;
  }

  rec[R_MX] = c.fx * t[0] / t[2] + c.cx;
  rec[R_MY] = c.fy * t[1] / t[2] + c.cy;
  rec[R_A] = a;
  rec[R_B] = b;
  rec[R_C] = cc;
  rec[R_BX] = beta[0];
  rec[R_BY] = beta[1];
  rec[R_M] = comp * (o1 + o2) * 0.5;
  rec[R_H] = comp * (o1 - o2) * 0.5;
  rec[R_UX] = beta[0] + ud[0];
  rec[R_UY] = beta[1] + ud[1];
  rec[R_COMP] = comp;
  rec[R_O1] = o1;
  rec[R_O2] = o2;
  rec[R_TZ] = t[2];
  rec[R_DXX] = dxx;
  rec[R_DXY] = dxy;
  rec[R_DYY] = dyy;
}

// Skew kernel times opacity at pixel centre (px, py) (Alg. 1 with the
// enhanced opacity): alpha = o(delta) * exp(-1/2(a dx^2 + c dy^2) - b dx dy)
//                             * (1 + erf((bx dx + by dy)/sqrt 2)), unclamped.
template <class S>
S alpha_raw(const S* r, double px, double py) {
  S dx = px - r[R_MX], dy = py - r[R_MY];
  S g = exp(-0.5 * (r[R_A] * dx * dx + r[R_C] * dy * dy) - r[R_B] * dx * dy);
  S zs = (r[R_BX] * dx + r[R_BY] * dy) / std::sqrt(2.0);
  S zu = (r[R_UX] * dx + r[R_UY] * dy) / std::sqrt(2.0);
  S o = r[R_M] + r[R_H] * erf(zu);
  return o * g * (1.0 + erf(zs));
}

void load_theta(const OrScene& s, int64_t i, double* th) {
  for (int k = 0; k < 3; ++k) th[P_MU + k] = s.means[3 * i + k];
  for (int k = 0; k < 3; ++k) th[P_LS + k] = s.log_scales[3 * i + k];
  for (int k = 0; k < 4; ++k) th[P_Q + k] = s.quats[4 * i + k];
  th[P_L + 0] = s.two_opac ? s.opac[2 * i] : s.opac[i];
  th[P_L + 1] = s.two_opac ? s.opac[2 * i + 1] : 0.0;
  for (int k = 0; k < 3; ++k) th[P_ETA + k] = s.skew[3 * i + k];
  for (int k = 0; k < 3; ++k) th[P_D + k] = s.split ? s.split[3 * i + k] : 0.0;
}

inline int sh_count(int deg) { return (deg + 1) * (deg + 1); }

// Conservative footprint and tile rectangle.  Returns false if the Gaussian
// can reach alpha >= alpha_min nowhere.  ext = (ex, ey, rho2).
bool footprint(const double* rec, const OrConfig& cfg, double* ext, double* cull_margin) {
  const double tau = cfg.alpha_min;
  const double omax = rec[R_COMP] * std::max(rec[R_O1], rec[R_O2]);
  *cull_margin = std::fabs(2.0 * omax - tau) / tau;
  if (2.0 * omax < tau) return false;
  const double rho0sq = 2.0 * std::log(2.0 * omax / tau);
  const double bx = rec[R_BX], by = rec[R_BY];
  const double bsb = bx * bx * rec[R_DXX] + 2.0 * bx * by * rec[R_DXY] + by * by * rec[R_DYY];
  const double kappa = 1.0 + std::erf(std::sqrt(rho0sq * bsb) / std::sqrt(2.0));
  *cull_margin = std::min(*cull_margin, std::fabs(kappa * omax - tau) / tau);
  if (kappa * omax < tau) return false;
  const double rho2 = 2.0 * std::log(kappa * omax / tau) * (1.0 + 1.0 / 1024.0);
  ext[0] = std::sqrt(rho2 * rec[R_DXX]);
  ext[1] = std::sqrt(rho2 * rec[R_DYY]);
  ext[2] = rho2;
  return true;
}

// Pixels whose centre (p + 0.5) lies in [m - e, m + e], as a tile range.
void tile_range_1d(double m, double e, int size, int tile, int* t0, int* t1) {
  double lo = std::ceil(m - e - 0.5), hi = std::floor(m + e - 0.5);
  lo = std::max(lo, 0.0);
  hi = std::min(hi, (double)size - 1.0);
  if (lo > hi) { *t0 = 0; *t1 = 0; return; }
  *t0 = (int)lo / tile;
  *t1 = (int)hi / tile + 1;
}

// x-extent, relative to mu_x, of the ellipse {d : d^T [[a, b], [b, c]] d <=
// rho2} within the heights [y0, y1] (relative to mu_y); false if they do not
// meet.  The boundary is x(y) = (-b y +- sqrt(a rho2 - D y^2)) / a with
// D = ac - b^2; its rightmost point is at y = -b rho / sqrt(D c) (leftmost at
// the opposite height), the right end is concave in y and the left end
// convex, so their extremes over the band sit at those heights clamped to the
// band.  *ymax receives the ellipse's half height.
bool ellipse_band(double a, double b, double c, double rho2, double y0, double y1, double* xl, double* xr,
                  double* ymax) {
  const double D = a * c - b * b;
  *ymax = rho2 > 0.0 ? std::sqrt(a * rho2 / D) : -1.0;
  y0 = std::max(y0, -*ymax);
  y1 = std::min(y1, *ymax);
  if (!(y0 <= y1)) return false;
  const double ys = -b * std::sqrt(rho2) / std::sqrt(D * c);
  const double yh = std::min(std::max(ys, y0), y1);
  const double yl = std::min(std::max(-ys, y0), y1);
  *xr = (-b * yh + std::sqrt(std::max(0.0, a * rho2 - D * yh * yh))) / a;
  *xl = (-b * yl - std::sqrt(std::max(0.0, a * rho2 - D * yl * yl))) / a;
  return true;
}

// Tile columns of tile row ty touched by the footprint of a record (the
// Gaussian's conic A = [[a, b], [b, c]], skew beta, E1 radius rho2):
//   S = (E1 and beta^T d >= 0) union (E2 and beta^T d < 0),
//   E1 = {d^T A d <= rho2},
//   E2 = {d^T (A + beta beta^T) d <= rho_-^2}, rho_-^2 = 2 ln(o_max comp / tau)(1 + 2^-10),
// E2 bounding the side z = beta^T d / sqrt 2 < 0, where 1 + erf z = erfc|z| <= e^{-z^2}.
// The row touches the tile columns holding a pixel centre in the x-extent of
// the footprint within the row's band of pixel-centre heights, taken as
// E1's extent cut by the hull of the half-plane's extent (the band clipped
// to E1's heights) and E2's; with beta = 0, E1's extent alone.  edge_shift
// perturbs both x ends (ambiguity checks).  Returns false if the row touches
// no tile; *near_edge is set when the band's edge lies within tol of a height
// where the rule changes discontinuously (the top or bottom of E1 or E2, or
// a horizontal half-plane boundary).
bool row_span(const double* r, double rho2, double tau, int ty, int width, int height, int tile, double edge_shift,
              double tol, int* t0, int* t1, bool* near_edge) {
  const double a = r[R_A], b = r[R_B], c = r[R_C];
  const double y0 = ty * (double)tile + 0.5 - r[R_MY];
  const double y1 = std::min(ty * tile + tile - 1, height - 1) + 0.5 - r[R_MY];
  double xl, xr, ymax1;
  const bool on1 = ellipse_band(a, b, c, rho2, y0, y1, &xl, &xr, &ymax1);
  bool near = std::fabs(y0 - ymax1) < tol || std::fabs(y1 + ymax1) < tol;
  bool on = on1;
  const double bx = r[R_BX], by = r[R_BY];
  if (on && (bx != 0.0 || by != 0.0)) {
    const double c0 = std::max(y0, -ymax1), c1 = std::min(y1, ymax1);
    bool hon = true;
    double hl = -INFINITY, hr = INFINITY;
    if (bx > 0.0) {
      hl = std::min(-by * c0 / bx, -by * c1 / bx);
    } else if (bx < 0.0) {
      hr = std::max(-by * c0 / bx, -by * c1 / bx);
    } else {
      hon = by > 0.0 ? c1 >= 0.0 : c0 <= 0.0;
      near = near || std::fabs(c0) < tol || std::fabs(c1) < tol;
    }
    const double omax = r[R_COMP] * std::max(r[R_O1], r[R_O2]);
    const double rho2m = 2.0 * std::log(omax / tau) * (1.0 + 1.0 / 1024.0);
    double l2 = 0.0, r2 = 0.0, ymax2 = -1.0;
    const bool e2on = rho2m > 0.0 && ellipse_band(a + bx * bx, b + bx * by, c + by * by, rho2m, y0, y1, &l2, &r2,
                                                  &ymax2);
    if (ymax2 > 0.0) near = near || std::fabs(y0 - ymax2) < tol || std::fabs(y1 + ymax2) < tol;
    if (!hon && !e2on) {
      on = false;
    } else {
      xl = std::max(xl, hon ? (e2on ? std::min(hl, l2) : hl) : l2);
      xr = std::min(xr, hon ? (e2on ? std::max(hr, r2) : hr) : r2);
    }
  }
  if (near_edge) *near_edge = near;
  if (!on) return false;
  double lo = std::ceil(r[R_MX] + xl - 0.5 - edge_shift), hi = std::floor(r[R_MX] + xr - 0.5 + edge_shift);
  lo = std::max(lo, 0.0);
  hi = std::min(hi, (double)width - 1.0);
  if (lo > hi) return false;
  *t0 = (int)lo / tile;
  *t1 = (int)hi / tile;
  return true;
}

}  // namespace

extern "C" {

int or_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Threads the oracle's parallel loops use from now on (timing runs only;
// results do not depend on it beyond the summation order of gradients).
void or_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// Alg. 3: M_cv = M_gl diag(1,-1,-1,1); W2C = M_cv^-1; K from (W, H, FoV).
// c2w_gl is row-major 4x4.  All fields are rounded to FP32 once.
void or_camera_from_gl(const double* c2w_gl, int32_t width, int32_t height, double fovx, double fovy,
                       OrCamera* out) {
  double m[4][4];
  const double flip[4] = {1.0, -1.0, -1.0, 1.0};
  for (int r = 0; r < 4; ++r)
    for (int k = 0; k < 4; ++k) m[r][k] = c2w_gl[4 * r + k] * flip[k];  // right-multiply by diag
  // inverse of a rigid transform [R t; 0 1] is [R^T, -R^T t]
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) out->w2c[4 * r + k] = (float)m[k][r];
    double tr = -(m[0][r] * m[0][3] + m[1][r] * m[1][3] + m[2][r] * m[2][3]);
    out->w2c[4 * r + 3] = (float)tr;
  }
  const double tx = std::tan(0.5 * fovx), ty = std::tan(0.5 * fovy);
  out->fx = (float)(width / (2.0 * tx));
  out->fy = (float)(height / (2.0 * ty));
  out->cx = (float)(0.5 * width);
  out->cy = (float)(0.5 * height);
  out->tan_fovx = (float)tx;
  out->tan_fovy = (float)ty;
  for (int k = 0; k < 3; ++k) out->campos[k] = (float)m[k][3];
  out->width = width;
  out->height = height;
}

// Project every Gaussian.  Outputs per Gaussian: rec[NREC] (FP64), the FP32
// depth key bits, visible (0 if culled by the near plane), rect[4] tile
// range (tx0, ty0, tx1, ty1) with tx1/ty1 exclusive, ext[3] = (ex, ey, rho2),
// rect_ambig = 1 where an FP32 evaluation of the rectangle or of the opacity
// cull could differ (an edge within tol_px of a pixel-centre boundary that
// changes the tile range, or the cull test within rel 1e-5 of alpha_min).
int or_nrec() { return NREC; }
int or_ndiff() { return NDIFF; }

void or_preprocess(const OrScene* s, const OrCamera* c, const OrConfig* cfg, double tol_px,
                   double* rec, uint32_t* depth_bits, int32_t* visible, int32_t* rect,
                   double* ext, int32_t* rect_ambig, int32_t* ntouch) {
  const int K = sh_count(s->sh_degree);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < s->n; ++i) {
    double th[NPARAM];
    load_theta(*s, i, th);
    float dz = depth_f32(*c, s->means + 3 * i);
    uint32_t bits;
    std::memcpy(&bits, &dz, 4);
    depth_bits[i] = bits;
    double* r = rec + NREC * i;
    int32_t* rc = rect + 4 * i;
    rc[0] = rc[1] = rc[2] = rc[3] = 0;
    ext[3 * i] = ext[3 * i + 1] = ext[3 * i + 2] = 0.0;
    rect_ambig[i] = 0;
    ntouch[i] = 0;
    visible[i] = dz > (float)cfg->near_z;
    if (!visible[i]) {
      std::fill(r, r + NREC, 0.0);
      continue;
    }
    project<double>(th, s->two_opac, s->split != nullptr, s->sh + (size_t)3 * K * i, s->sh_degree, *c, *cfg, r);
    double e[3], margin;
    bool on = footprint(r, *cfg, e, &margin);
    if (margin < 1e-5) rect_ambig[i] = 1;
    if (!on) continue;
    ext[3 * i] = e[0]; ext[3 * i + 1] = e[1]; ext[3 * i + 2] = e[2];
    tile_range_1d(r[R_MX], e[0], c->width, cfg->tile_w, &rc[0], &rc[2]);
    tile_range_1d(r[R_MY], e[1], c->height, cfg->tile_h, &rc[1], &rc[3]);
    // perturb each edge by +-tol_px: a different tile range means ambiguous
    for (int sgn = -1; sgn <= 1; sgn += 2) {
      int a0, a1, b0, b1;
      tile_range_1d(r[R_MX], e[0] + sgn * tol_px, c->width, cfg->tile_w, &a0, &a1);
      tile_range_1d(r[R_MY], e[1] + sgn * tol_px, c->height, cfg->tile_h, &b0, &b1);
      int empty0 = (rc[0] == rc[2]) || (rc[1] == rc[3]);
      int empty1 = (a0 == a1) || (b0 == b1);
      if (empty0 != empty1 || (!empty0 && (a0 != rc[0] || a1 != rc[2] || b0 != rc[1] || b1 != rc[3])))
        rect_ambig[i] = 1;
      tile_range_1d(r[R_MX] + sgn * tol_px, e[0], c->width, cfg->tile_w, &a0, &a1);
      tile_range_1d(r[R_MY] + sgn * tol_px, e[1], c->height, cfg->tile_h, &b0, &b1);
      empty1 = (a0 == a1) || (b0 == b1);
      if (empty0 != empty1 || (!empty0 && (a0 != rc[0] || a1 != rc[2] || b0 != rc[1] || b1 != rc[3])))
        rect_ambig[i] = 1;
    }
    // exact ellipse / tile test per row of the box
    for (int ty = rc[1]; ty < rc[3]; ++ty) {
      int t0, t1, u0, u1, v0, v1;
      bool near = false;
      const double tau = cfg->alpha_min;
      const bool on0 = row_span(r, e[2], tau, ty, c->width, c->height, cfg->tile_w, 0.0, tol_px, &t0, &t1, &near);
      const bool onm =
          row_span(r, e[2], tau, ty, c->width, c->height, cfg->tile_w, -tol_px, tol_px, &u0, &u1, nullptr);
      const bool onp =
          row_span(r, e[2], tau, ty, c->width, c->height, cfg->tile_w, tol_px, tol_px, &v0, &v1, nullptr);
      if (on0) ntouch[i] += t1 - t0 + 1;
      if (near || on0 != onm || on0 != onp || (on0 && (t0 != u0 || t1 != u1 || t0 != v0 || t1 != v1)))
        rect_ambig[i] = 1;
    }
  }
}

}  // extern "C"

namespace {

int or_num_threads_impl() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Depth order of the visible Gaussians: by (FP32 depth bits, index).
static std::vector<int32_t> depth_order(int64_t n, const uint32_t* depth_bits, const int32_t* visible) {
  std::vector<int32_t> order;
  for (int64_t i = 0; i < n; ++i)
    if (visible[i]) order.push_back((int32_t)i);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return depth_bits[a] < depth_bits[b]; });
  return order;
}

// One blended pair of a pixel: its alpha, the transmittance in front of it,
// whether alpha_max clamped it and whether that clamp decision lies within
// the tolerance of alpha_max (its derivative is then ambiguous).
struct Blend { int32_t id; double alpha; double T; int clamped; int clamp_near; };

// What a pixel's decisions looked like.  ambiguous: some pair lies within
// the tolerance of the gate or of the stop.  For a replay of another
// renderer's decisions: status 0 if every decision it took is admissible,
// else the kind of the first inadmissible one (1: blended a pair below the
// gate, 2: blended a pair past the stop, 3: skipped a pair it should have
// stopped at, 4: skipped a pair it should have blended, 5: blended a pair
// this pixel's list does not hold, or out of order); flips counts the
// decisions that differ from the FP64 ones, margin the largest relative
// distance of such a decision's alpha (gate) or T' (stop) to its threshold.
struct PixelDecisions {
  int ambiguous = 0;
  int status = 0;
  int flips_gate = 0, flips_stop = 0;
  double margin_gate = 0.0, margin_stop = 0.0;
};

// Front-to-back compositing of one pixel over a depth-ordered candidate list
// ids[0..m) (Alg. 1, Eq. color): alpha = min(alpha_max, alpha_raw); a pair
// with alpha < alpha_min is skipped; the stop comes before the Gaussian whose
// T' = T (1 - alpha) falls below t_stop; C = sum c alpha T + T_final bg.
// Decisions are FP64's own, or, when gpu is non-null, those of another
// renderer that blended exactly gpu[0..ng) (in order): each of its decisions
// must then either agree with FP64 or lie within the tolerance (tol_a
// relative to alpha_min, tol_t relative to t_stop) of its threshold.
// Candidates missing from ids must have alpha < alpha_min (1 - tol_a).
static void composite_list(const int32_t* ids, int64_t m, const int32_t* gpu, int64_t ng, const double* rec,
                           const OrConfig& cfg, int px, int py, double tol_a, double tol_t, double* C,
                           double* T_out, std::vector<Blend>* blended, PixelDecisions* dec,
                           uint64_t* signature = nullptr) {
  double T = 1.0, acc[3] = {0.0, 0.0, 0.0};
  uint64_t sig = 1469598103934665603ull;  // FNV-1a over the discrete decisions
  const double x = px + 0.5, y = py + 0.5;
  const double amin = cfg.alpha_min, amax = cfg.alpha_max, tstop = cfg.t_stop;
  int64_t k = 0;  // next pair the other renderer blended
  for (int64_t j = 0; j < m; ++j) {
    const int32_t id = ids[j];
    const double* r = rec + (size_t)NREC * id;
    const double a_raw = alpha_raw<double>(r, x, y);
    const double a = std::min(amax, a_raw);
    const bool pass = a >= amin;
    const bool near_gate = std::fabs(a - amin) < tol_a * amin;
    if (near_gate) dec->ambiguous = 1;
    if (!pass && !gpu) continue;
    const double Tn = T * (1.0 - a);
    const bool stop = Tn < tstop;
    const bool near_stop = std::fabs(Tn - tstop) < tol_t * tstop;
    if (pass && near_stop) dec->ambiguous = 1;
    bool take;
    if (!gpu) {
      sig = (sig ^ (uint64_t)(2 * (int64_t)id + (a_raw > amax))) * 1099511628211ull;
      if (stop) { sig = (sig ^ 0xffffull) * 1099511628211ull; break; }
      take = true;
    } else if (k < ng && gpu[k] == id) {
      // blended by the other renderer
      if (!pass) {
        if (!near_gate) { dec->status = 1; break; }
        ++dec->flips_gate;
        dec->margin_gate = std::max(dec->margin_gate, std::fabs(a - amin) / amin);
      }
      if (stop) {
        if (!near_stop) { dec->status = 2; break; }
        ++dec->flips_stop;
        dec->margin_stop = std::max(dec->margin_stop, std::fabs(Tn - tstop) / tstop);
      }
      take = true;
      ++k;
    } else {
      // not blended by the other renderer
      if (!pass) continue;
      if (k == ng && (stop || near_stop)) {  // it stopped here
        if (!stop) {
          ++dec->flips_stop;
          dec->margin_stop = std::max(dec->margin_stop, std::fabs(Tn - tstop) / tstop);
        }
        break;
      }
      if (near_gate) {  // it saw alpha below the gate
        ++dec->flips_gate;
        dec->margin_gate = std::max(dec->margin_gate, std::fabs(a - amin) / amin);
        continue;
      }
      dec->status = stop ? 3 : 4;
      break;
    }
    if (!take) continue;
    for (int ch = 0; ch < 3; ++ch) acc[ch] += r[R_CR + ch] * a * T;
    if (blended)
      blended->push_back({id, a, T, a_raw > amax, std::fabs(a_raw - amax) < tol_a * amax ? 1 : 0});
    T = Tn;
  }
  if (gpu && dec->status == 0 && k < ng) dec->status = 5;
  for (int ch = 0; ch < 3; ++ch) C[ch] = acc[ch] + T * cfg.bg[ch];
  *T_out = T;
  if (signature) *signature = sig;
}

// ---------------------------------------------------------------------------
// Mode B: the same composite, with each pixel's candidate list restricted to
// the Gaussians whose footprint reaches it.  A Gaussian can have
// alpha >= tau_s = alpha_min (1 - kScatterSlack) only inside the ellipse
// d^T A d <= rho_s^2 with rho_s^2 = 2 ln(kappa o_max comp / tau_s) (the
// conservative footprint, whose bound holds for any threshold), so every
// pair left out has alpha < tau_s: mode A skips it and flags nothing
// (tol_a < kScatterSlack), and mode B's result equals mode A's bit for bit.
// ---------------------------------------------------------------------------
constexpr double kScatterSlack = 1e-2;

struct Scatter {
  int width = 0, height = 0;
  std::vector<int64_t> row_off;  // [height + 1]
  std::vector<int32_t> id;       // per row, the Gaussians reaching it, in depth order
  std::vector<int32_t> x0, x1;   // columns of their pixel centres in the row (inclusive)
};

// Rows and columns of pixel centres inside a Gaussian's scatter ellipse.
struct Ellipse { double a, b, c, rho2, mx, my; bool on; };

static Ellipse scatter_ellipse(const double* r, const OrConfig& cfg) {
  Ellipse e{r[R_A], r[R_B], r[R_C], 0.0, r[R_MX], r[R_MY], false};
  const double tau = cfg.alpha_min * (1.0 - kScatterSlack);
  const double omax = r[R_COMP] * std::max(r[R_O1], r[R_O2]);
  if (2.0 * omax < tau) return e;
  const double rho0sq = 2.0 * std::log(2.0 * omax / tau);
  const double bx = r[R_BX], by = r[R_BY];
  const double bsb = bx * bx * r[R_DXX] + 2.0 * bx * by * r[R_DXY] + by * by * r[R_DYY];
  const double kappa = 1.0 + std::erf(std::sqrt(rho0sq * bsb) / std::sqrt(2.0));
  if (kappa * omax < tau) return e;
  e.rho2 = 2.0 * std::log(kappa * omax / tau) * (1.0 + 1e-9);
  e.on = true;
  return e;
}

static void ellipse_rows(const Ellipse& e, int height, int* y0, int* y1) {
  const double D = e.a * e.c - e.b * e.b;
  const double h = std::sqrt(e.a * e.rho2 / D) + 1e-7;
  *y0 = (int)std::max(0.0, std::ceil(e.my - h - 0.5));
  *y1 = (int)std::min((double)height - 1.0, std::floor(e.my + h - 0.5));
}

static bool ellipse_cols(const Ellipse& e, int py, int width, int* x0, int* x1) {
  const double D = e.a * e.c - e.b * e.b;
  const double dy = py + 0.5 - e.my;
  const double disc = e.a * e.rho2 - D * dy * dy;
  if (disc < 0.0) return false;
  const double s = std::sqrt(disc);
  const double lo = (-e.b * dy - s) / e.a - 1e-7, hi = (-e.b * dy + s) / e.a + 1e-7;
  const double c0 = std::max(0.0, std::ceil(e.mx + lo - 0.5));
  const double c1 = std::min((double)width - 1.0, std::floor(e.mx + hi - 0.5));
  if (c0 > c1) return false;
  *x0 = (int)c0;
  *x1 = (int)c1;
  return true;
}

// Row lists in depth order: the Gaussians are split into contiguous chunks of
// the depth order, each thread counts and then fills its chunk's entries at
// offsets that keep the chunks in order.
static void build_scatter(const std::vector<int32_t>& order, const double* rec, const OrConfig& cfg, int width,
                          int height, Scatter* s) {
  s->width = width;
  s->height = height;
  const int64_t m = (int64_t)order.size();
  const int nt = std::max(1, or_num_threads_impl());
  std::vector<int64_t> cnt((size_t)nt * (height + 1), 0);
#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    const int64_t lo = m * t / nt, hi = m * (t + 1) / nt;
    int64_t* c = cnt.data() + (size_t)t * (height + 1);
    for (int64_t j = lo; j < hi; ++j) {
      const Ellipse e = scatter_ellipse(rec + (size_t)NREC * order[j], cfg);
      if (!e.on) continue;
      int y0, y1, a, b;
      ellipse_rows(e, height, &y0, &y1);
      for (int y = y0; y <= y1; ++y)
        if (ellipse_cols(e, y, width, &a, &b)) ++c[y];
    }
  }
  s->row_off.assign(height + 1, 0);
  std::vector<int64_t> start((size_t)nt * (height + 1), 0);
  int64_t tot = 0;
  for (int y = 0; y < height; ++y) {
    s->row_off[y] = tot;
    for (int t = 0; t < nt; ++t) {
      start[(size_t)t * (height + 1) + y] = tot;
      tot += cnt[(size_t)t * (height + 1) + y];
    }
  }
  s->row_off[height] = tot;
  s->id.resize(tot);
  s->x0.resize(tot);
  s->x1.resize(tot);
#pragma omp parallel num_threads(nt)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    const int64_t lo = m * t / nt, hi = m * (t + 1) / nt;
    int64_t* w = start.data() + (size_t)t * (height + 1);
    for (int64_t j = lo; j < hi; ++j) {
      const Ellipse e = scatter_ellipse(rec + (size_t)NREC * order[j], cfg);
      if (!e.on) continue;
      int y0, y1, a, b;
      ellipse_rows(e, height, &y0, &y1);
      for (int y = y0; y <= y1; ++y)
        if (ellipse_cols(e, y, width, &a, &b)) {
          const int64_t q = w[y]++;
          s->id[q] = order[j];
          s->x0[q] = a;
          s->x1[q] = b;
        }
    }
  }
}

// Per-pixel candidate lists of one row (a counting sort of the row's entries
// by column keeps their depth order).
struct RowLists {
  std::vector<int64_t> off;  // [width + 1]
  std::vector<int32_t> id;
};

static void row_lists(const Scatter& s, int y, RowLists* L) {
  const int W = s.width;
  L->off.assign(W + 1, 0);
  const int64_t b = s.row_off[y], e = s.row_off[y + 1];
  for (int64_t q = b; q < e; ++q)
    for (int x = s.x0[q]; x <= s.x1[q]; ++x) ++L->off[x + 1];
  for (int x = 0; x < W; ++x) L->off[x + 1] += L->off[x];
  L->id.resize(L->off[W]);
  std::vector<int64_t> w(L->off.begin(), L->off.end() - 1);
  for (int64_t q = b; q < e; ++q)
    for (int x = s.x0[q]; x <= s.x1[q]; ++x) L->id[w[x]++] = s.id[q];
}

// ---------------------------------------------------------------------------
// Backward of one pixel (Appendix "Backward Pass"): for the blended list bl,
// dC/dalpha_k = c_k T_k - (sum_{i>k} c_i alpha_i T_i + T_N bg) / (1 - alpha_k),
// the plain derivative of C = sum_i c_i alpha_i T_i + T_N bg, zero where
// alpha_max clamped alpha; dalpha/d(record) by dual numbers.  Adds into
// grad[n, NDIFF]; scale (optional) receives, per record entry, the sum over
// pairs of the magnitudes of the terms a rounding error in any factor
// scales with; slack (optional), per entry, the magnitude of the
// alpha-path term of every pair whose clamp decision lies within tolerance.
// ---------------------------------------------------------------------------
static void backward_pixel(const std::vector<Blend>& bl, double T_final, const double* g, const double* rec,
                           const OrConfig& cfg, int px, int py, double* grad, double* scale, double* slack) {
  const int nb = (int)bl.size();
  std::vector<double> suffix(3 * (nb + 1), 0.0);  // sum_{i>k} c_i alpha_i T_i + T_N bg
  std::vector<double> sabs(3 * (nb + 1), 0.0);    // the same with magnitudes
  for (int ch = 0; ch < 3; ++ch) {
    suffix[3 * nb + ch] = T_final * cfg.bg[ch];
    sabs[3 * nb + ch] = std::fabs(T_final * cfg.bg[ch]);
  }
  for (int k = nb - 1; k >= 0; --k) {
    const double* r = rec + (size_t)NREC * bl[k].id;
    for (int ch = 0; ch < 3; ++ch) {
      const double t = r[R_CR + ch] * bl[k].alpha * bl[k].T;
      suffix[3 * k + ch] = suffix[3 * (k + 1) + ch] + t;
      sabs[3 * k + ch] = sabs[3 * (k + 1) + ch] + std::fabs(t);
    }
  }
  const double x = px + 0.5, y = py + 0.5;
  for (int k = 0; k < nb; ++k) {
    const int32_t id = bl[k].id;
    const double* r = rec + (size_t)NREC * id;
    double* out = grad + (size_t)NDIFF * id;
    for (int ch = 0; ch < 3; ++ch) {
      out[R_CR + ch] += g[ch] * bl[k].alpha * bl[k].T;
      if (scale) scale[(size_t)NDIFF * id + R_CR + ch] += std::fabs(g[ch] * bl[k].alpha * bl[k].T);
    }
    if (bl[k].clamped && !(bl[k].clamp_near && slack)) continue;
    double dLda = 0.0, wabs = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      dLda += g[ch] * (r[R_CR + ch] * bl[k].T - suffix[3 * (k + 1) + ch] / (1.0 - bl[k].alpha));
      wabs += std::fabs(g[ch]) * (std::fabs(r[R_CR + ch]) * bl[k].T + sabs[3 * (k + 1) + ch] / (1.0 - bl[k].alpha));
    }
    Dual<11> rr[NDIFF];
    for (int q = 0; q < NDIFF; ++q) rr[q] = Dual<11>(r[q]);
    for (int q = 0; q < 11; ++q) rr[q].d[q] = 1.0;  // R_MX..R_UY are entries 0..10
    Dual<11> a = alpha_raw<Dual<11>>(rr, x, y);
    if (bl[k].clamp_near && slack)
      for (int q = 0; q < 11; ++q) slack[(size_t)NDIFF * id + q] += std::fabs(dLda * a.d[q]);
    if (bl[k].clamped) continue;
    for (int q = 0; q < 11; ++q) out[q] += dLda * a.d[q];
    if (scale)
      for (int q = 0; q < 11; ++q) scale[(size_t)NDIFF * id + q] += wabs * std::fabs(a.d[q]);
  }
}

// Attribute-gradient outputs (same layouts as the scene; split may be null).
struct OrGradsOut {
  double* means;
  double* log_scales;
  double* quats;
  double* opac;
  double* skew;
  double* split;
  double* sh;
};

// Chain rule from the record gradients d2[n, NDIFF] to every attribute, by
// dual numbers through the projection; colour is linear in the SH
// coefficients.  With d2_scale / d2_slack, the same map applied to their
// magnitudes (|Jacobian| times the entry) goes to scale / slack; a colour
// channel whose pre-activation lies within 1e-5 of the clamp at zero adds
// its whole term to slack (the other renderer's clamp may differ).
static void chain_to_attributes(const OrScene& s, const OrCamera& cam, const OrConfig& cfg, const int32_t* visible,
                                const double* d2, const double* d2_scale, const double* d2_slack,
                                const OrGradsOut& G, const OrGradsOut* S, const OrGradsOut* L) {
  const int64_t n = s.n;
  const int K = sh_count(s.sh_degree);
  const int nop = s.two_opac ? 2 : 1;
  auto zero = [&](const OrGradsOut& o, int64_t i) {
    for (int k = 0; k < 3; ++k) { o.means[3 * i + k] = 0; o.log_scales[3 * i + k] = 0; o.skew[3 * i + k] = 0; }
    for (int k = 0; k < 4; ++k) o.quats[4 * i + k] = 0;
    for (int k = 0; k < nop; ++k) o.opac[nop * i + k] = 0;
    if (o.split) for (int k = 0; k < 3; ++k) o.split[3 * i + k] = 0;
    for (int k = 0; k < 3 * K; ++k) o.sh[(size_t)3 * K * i + k] = 0;
  };
  auto store = [&](const OrGradsOut& o, int64_t i, const double* gth) {
    for (int k = 0; k < 3; ++k) o.means[3 * i + k] = gth[P_MU + k];
    for (int k = 0; k < 3; ++k) o.log_scales[3 * i + k] = gth[P_LS + k];
    for (int k = 0; k < 4; ++k) o.quats[4 * i + k] = gth[P_Q + k];
    for (int k = 0; k < nop; ++k) o.opac[nop * i + k] = gth[P_L + k];
    for (int k = 0; k < 3; ++k) o.skew[3 * i + k] = gth[P_ETA + k];
    if (o.split) for (int k = 0; k < 3; ++k) o.split[3 * i + k] = gth[P_D + k];
  };
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    zero(G, i);
    if (S) zero(*S, i);
    if (L) zero(*L, i);
    const double* gi = d2 + (size_t)NDIFF * i;
    bool any = false;
    for (int q = 0; q < NDIFF; ++q) any |= gi[q] != 0.0;
    if (d2_slack)
      for (int q = 0; q < NDIFF; ++q) any |= d2_slack[(size_t)NDIFF * i + q] != 0.0;
    if (!any || !visible[i]) continue;
    double th[NPARAM];
    load_theta(s, i, th);
    Dual<NPARAM> thd[NPARAM];
    for (int q = 0; q < NPARAM; ++q) { thd[q] = Dual<NPARAM>(th[q]); thd[q].d[q] = 1.0; }
    Dual<NPARAM> r[NREC];
    const double* shi = s.sh + (size_t)3 * K * i;
    project<Dual<NPARAM>>(thd, s.two_opac, s.split != nullptr, shi, s.sh_degree, cam, cfg, r);
    double gth[NPARAM] = {0}, sth[NPARAM] = {0}, lth[NPARAM] = {0};
    for (int q = 0; q < NDIFF; ++q)
      for (int p = 0; p < NPARAM; ++p) {
        gth[p] += gi[q] * r[q].d[p];
        if (S) sth[p] += d2_scale[(size_t)NDIFF * i + q] * std::fabs(r[q].d[p]);
        if (L) lth[p] += d2_slack[(size_t)NDIFF * i + q] * std::fabs(r[q].d[p]);
      }
    // colour channels near the clamp at zero: the pre-activation's derivative
    double dv[3] = {th[0] - cam.campos[0], th[1] - cam.campos[1], th[2] - cam.campos[2]};
    double dl = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    double Y[16];
    sh_basis<double>(s.sh_degree, dv[0] / dl, dv[1] / dl, dv[2] / dl, Y);
    double pre[3];
    for (int ch = 0; ch < 3; ++ch) {
      pre[ch] = 0.5;
      for (int k = 0; k < K; ++k) pre[ch] += shi[3 * k + ch] * Y[k];
    }
    const bool near0 = std::fabs(pre[0]) < 1e-5 || std::fabs(pre[1]) < 1e-5 || std::fabs(pre[2]) < 1e-5;
    if (L && near0) {
      Dual<NPARAM> u[NREC];
      project<Dual<NPARAM>>(thd, s.two_opac, s.split != nullptr, shi, s.sh_degree, cam, cfg, u, false);
      for (int ch = 0; ch < 3; ++ch)
        if (std::fabs(pre[ch]) < 1e-5)
          for (int p = 0; p < NPARAM; ++p) lth[p] += std::fabs(gi[R_CR + ch] * u[R_CR + ch].d[p]);
    }
    store(G, i, gth);
    if (S) store(*S, i, sth);
    if (L) store(*L, i, lth);
    for (int ch = 0; ch < 3; ++ch) {
      const bool amb = std::fabs(pre[ch]) < 1e-5;
      for (int k = 0; k < K; ++k) {
        const size_t o = (size_t)3 * K * i + 3 * k + ch;
        if (pre[ch] >= 0.0) G.sh[o] = Y[k] * gi[R_CR + ch];
        if (S) S->sh[o] = std::fabs(Y[k]) * d2_scale[(size_t)NDIFF * i + R_CR + ch];
        if (L && amb) L->sh[o] = std::fabs(Y[k] * gi[R_CR + ch]);
      }
    }
  }
}

// Pixel-parallel accumulation of record gradients: one [n, NDIFF] array per
// thread for each requested output, summed at the end.
struct Accum {
  int64_t n;
  bool want_scale, want_slack;
  std::vector<std::vector<double>> g, s, l;
  Accum(int64_t n_, int nt, bool ws, bool wl) : n(n_), want_scale(ws), want_slack(wl), g(nt), s(nt), l(nt) {}
  void init(int t) {
    g[t].assign((size_t)n * NDIFF, 0.0);
    if (want_scale) s[t].assign((size_t)n * NDIFF, 0.0);
    if (want_slack) l[t].assign((size_t)n * NDIFF, 0.0);
  }
  void reduce(double* d2, double* d2s, double* d2l) {
    std::fill(d2, d2 + (size_t)n * NDIFF, 0.0);
    if (d2s) std::fill(d2s, d2s + (size_t)n * NDIFF, 0.0);
    if (d2l) std::fill(d2l, d2l + (size_t)n * NDIFF, 0.0);
    for (size_t t = 0; t < g.size(); ++t) {
      if (g[t].empty()) continue;
#pragma omp parallel for schedule(static)
      for (int64_t q = 0; q < n * NDIFF; ++q) {
        d2[q] += g[t][q];
        if (d2s) d2s[q] += s[t][q];
        if (d2l) d2l[q] += l[t][q];
      }
    }
  }
};

}  // namespace

extern "C" {

// Render a list of pixels (pix[2*j] = px, pix[2*j+1] = py) by brute force
// over every visible Gaussian in depth order (mode A).  out_rgb [n_pix,3],
// out_T [n_pix], out_last [n_pix] (id of the last blended Gaussian or -1),
// out_count [n_pix] (number blended), out_amb [n_pix] (a pair within tol_a
// (relative to alpha_min) of the gate or within tol_t (relative to t_stop)
// of the stop), out_sig [n_pix] (a hash of which Gaussians were blended,
// which were clamped and whether the transmittance stop fired; may be null).
void or_render_pixels(const OrCamera* cam, const OrConfig* cfg, int64_t n, const double* rec,
                      const uint32_t* depth_bits, const int32_t* visible, int64_t n_pix, const int32_t* pix,
                      double tol_a, double tol_t, double* out_rgb, double* out_T, int64_t* out_last,
                      int32_t* out_count, int32_t* out_amb, uint64_t* out_sig) {
  (void)cam;
  const std::vector<int32_t> order = depth_order(n, depth_bits, visible);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < n_pix; ++j) {
    std::vector<Blend> bl;
    PixelDecisions dec;
    composite_list(order.data(), (int64_t)order.size(), nullptr, 0, rec, *cfg, pix[2 * j], pix[2 * j + 1], tol_a,
                   tol_t, out_rgb + 3 * j, out_T + j, &bl, &dec, out_sig ? out_sig + j : nullptr);
    out_amb[j] = dec.ambiguous;
    out_count[j] = (int32_t)bl.size();
    out_last[j] = bl.empty() ? -1 : bl.back().id;
  }
}

// Whole frame, row-major pixels (mode B: per-pixel lists of the Gaussians
// whose footprint reaches the pixel, in depth order).  Outputs as
// or_render_pixels, [H*W] per pixel.  With gpu_off non-null, the gate and
// stop decisions are those of another renderer that blended, at pixel p,
// gpu_ids[gpu_off[p] .. gpu_off[p+1]) in order: out_status [H*W] (null
// allowed otherwise) receives each pixel's PixelDecisions status, and stats
// (null allowed) [8] = pixels with a flipped decision, flipped gate
// decisions, flipped stop decisions, largest gate margin, largest stop
// margin, inadmissible pixels, candidate pairs, pixels with an ambiguous pair.
// With list_off non-null (the prefix sums of an earlier call's out_count),
// the ids of the Gaussians each pixel blended go to list_ids[list_off[p]..).
void or_render_frame(const OrCamera* cam, const OrConfig* cfg, int64_t n, const double* rec,
                     const uint32_t* depth_bits, const int32_t* visible, double tol_a, double tol_t,
                     const int64_t* gpu_off, const int32_t* gpu_ids, double* out_rgb, double* out_T,
                     int64_t* out_last, int32_t* out_count, int32_t* out_amb, int32_t* out_status,
                     double* stats, const int64_t* list_off, int32_t* list_ids) {
  const int W = cam->width, H = cam->height;
  const std::vector<int32_t> order = depth_order(n, depth_bits, visible);
  Scatter sc;
  build_scatter(order, rec, *cfg, W, H, &sc);
  double st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma omp parallel
  {
    double mine[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    RowLists L;
    std::vector<Blend> bl;
#pragma omp for schedule(dynamic, 1)
    for (int y = 0; y < H; ++y) {
      row_lists(sc, y, &L);
      mine[6] += (double)L.id.size();
      for (int x = 0; x < W; ++x) {
        const int64_t p = (int64_t)y * W + x;
        bl.clear();
        PixelDecisions dec;
        const int32_t* gp = gpu_off ? gpu_ids + gpu_off[p] : nullptr;
        const int64_t ng = gpu_off ? gpu_off[p + 1] - gpu_off[p] : 0;
        composite_list(L.id.data() + L.off[x], L.off[x + 1] - L.off[x], gp, ng, rec, *cfg, x, y, tol_a, tol_t,
                       out_rgb + 3 * p, out_T + p, &bl, &dec);
        out_amb[p] = dec.ambiguous;
        out_count[p] = (int32_t)bl.size();
        out_last[p] = bl.empty() ? -1 : bl.back().id;
        if (list_off)
          for (size_t k = 0; k < bl.size(); ++k) list_ids[list_off[p] + (int64_t)k] = bl[k].id;
        if (out_status) out_status[p] = dec.status;
        mine[0] += (dec.flips_gate + dec.flips_stop) > 0;
        mine[1] += dec.flips_gate;
        mine[2] += dec.flips_stop;
        mine[3] = std::max(mine[3], dec.margin_gate);
        mine[4] = std::max(mine[4], dec.margin_stop);
        mine[5] += dec.status != 0;
        mine[7] += dec.ambiguous;
      }
    }
#pragma omp critical
    {
      for (int k : {0, 1, 2, 5, 6, 7}) st[k] += mine[k];
      st[3] = std::max(st[3], mine[3]);
      st[4] = std::max(st[4], mine[4]);
    }
  }
  if (stats) std::copy(st, st + 8, stats);
}

// Gradients of L = sum_pixels sum_ch dL_dC[pixel, ch] * C[pixel, ch].
//  * mode A (pix non-null): over the listed pixels, dL_dC [n_pix, 3], brute
//    force over every visible Gaussian; mode B (pix null): every pixel of the
//    frame, row-major, dL_dC [H*W, 3], per-pixel footprint lists;
//  * gpu_off / gpu_ids (optional, indexed like dL_dC's rows): the gate and
//    stop decisions of another renderer, replayed as in or_render_frame
//    (inadmissible pixels are counted in *n_bad and contribute nothing);
//  * d2 [n, NDIFF]: dL/d(record), the 2D quantities of Alg. 2; d2_scale and
//    d2_slack (optional): see backward_pixel;
//  * G: the attribute gradients; S, L (optional): scale and slack mapped
//    through the projection (see chain_to_attributes).
// tol_a: the relative tolerance of the alpha_max clamp (slack) and, with a
// replay, of the gate; tol_t: of the stop (replay only).
void or_render_backward(const OrScene* s, const OrCamera* cam, const OrConfig* cfg, const double* rec,
                        const uint32_t* depth_bits, const int32_t* visible, int64_t n_pix, const int32_t* pix,
                        const double* dL_dC, const int64_t* gpu_off, const int32_t* gpu_ids, double tol_a,
                        double tol_t, double* d2, double* d2_scale, double* d2_slack, const OrGradsOut* G,
                        const OrGradsOut* S, const OrGradsOut* L, int64_t* n_bad) {
  const int64_t n = s->n;
  const int W = cam->width, H = cam->height;
  const std::vector<int32_t> order = depth_order(n, depth_bits, visible);
  const bool frame = pix == nullptr;
  Scatter sc;
  if (frame) build_scatter(order, rec, *cfg, W, H, &sc);
  const int nt = or_num_threads_impl();
  Accum acc(n, nt, d2_scale != nullptr, d2_slack != nullptr);
  int64_t bad = 0;
#pragma omp parallel num_threads(nt) reduction(+ : bad)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    acc.init(t);
    double* ga = acc.g[t].data();
    double* sa = acc.want_scale ? acc.s[t].data() : nullptr;
    double* la = acc.want_slack ? acc.l[t].data() : nullptr;
    std::vector<Blend> bl;
    RowLists Lr;
    auto one = [&](int64_t p, int px, int py, const int32_t* ids, int64_t m) {
      const double* g = dL_dC + 3 * p;
      if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) return;
      bl.clear();
      PixelDecisions dec;
      double C[3], T_final;
      const int32_t* gp = gpu_off ? gpu_ids + gpu_off[p] : nullptr;
      const int64_t ng = gpu_off ? gpu_off[p + 1] - gpu_off[p] : 0;
      composite_list(ids, m, gp, ng, rec, *cfg, px, py, tol_a, tol_t, C, &T_final, &bl, &dec);
      if (dec.status != 0) { ++bad; return; }
      backward_pixel(bl, T_final, g, rec, *cfg, px, py, ga, sa, la);
    };
    if (frame) {
#pragma omp for schedule(dynamic, 1)
      for (int y = 0; y < H; ++y) {
        row_lists(sc, y, &Lr);
        for (int x = 0; x < W; ++x)
          one((int64_t)y * W + x, x, y, Lr.id.data() + Lr.off[x], Lr.off[x + 1] - Lr.off[x]);
      }
    } else {
#pragma omp for schedule(dynamic, 8)
      for (int64_t j = 0; j < n_pix; ++j)
        one(j, pix[2 * j], pix[2 * j + 1], order.data(), (int64_t)order.size());
    }
  }
  acc.reduce(d2, d2_scale, d2_slack);
  if (n_bad) *n_bad = bad;
  chain_to_attributes(*s, *cam, *cfg, visible, d2, d2_scale, d2_slack, *G, S, L);
}

// Tile keys of one view: for each visible Gaussian, in index order, one
// (tile | depth) key per tile its footprint touches (row_span,
// row-major), then a stable sort.  tile_base / val_base offset the tile id
// and the value.
// Returns the number of keys; writes at most cap of them.
int64_t or_bin(int64_t n, const double* rec, const double* ext, const uint32_t* depth_bits, const int32_t* visible,
               const int32_t* rect, int32_t width, int32_t height, int32_t tile_size, double tau, int64_t tile_base,
               int64_t val_base, int64_t cap, uint64_t* keys, int64_t* vals) {
  const int32_t tiles_x = (width + tile_size - 1) / tile_size;
  std::vector<std::pair<uint64_t, int64_t>> kv;
  for (int64_t i = 0; i < n; ++i) {
    if (!visible[i]) continue;
    const int32_t* r = rect + 4 * i;
    for (int ty = r[1]; ty < r[3]; ++ty) {
      int t0, t1;
      if (!row_span(rec + (size_t)NREC * i, ext[3 * i + 2], tau, ty, width, height, tile_size, 0.0, 0.0, &t0, &t1,
                    nullptr))
        continue;
      for (int tx = t0; tx <= t1; ++tx) {
        uint64_t tile = (uint64_t)(tile_base + (int64_t)ty * tiles_x + tx);
        kv.push_back({(tile << 32) | depth_bits[i], val_base + i});
      }
    }
  }
  std::stable_sort(kv.begin(), kv.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  int64_t m = (int64_t)kv.size();
  for (int64_t j = 0; j < std::min(m, cap); ++j) { keys[j] = kv[j].first; vals[j] = kv[j].second; }
  return m;
}

// Skew kernel (with o = 1, no clamp) at arbitrary offsets, for quadrature and
// Monte-Carlo checks: out[j] = exp(-1/2 d^T A d) (1 + erf(beta^T d / sqrt 2)).
void or_kernel_at(const double* abc, const double* beta, int64_t m, const double* dxy, double* out) {
  double r[NREC] = {0};
  r[R_A] = abc[0]; r[R_B] = abc[1]; r[R_C] = abc[2];
  r[R_BX] = beta[0]; r[R_BY] = beta[1];
  r[R_M] = 1.0;
  for (int64_t j = 0; j < m; ++j) out[j] = alpha_raw<double>(r, dxy[2 * j] + 0.0, dxy[2 * j + 1] + 0.0);
}

// Alpha of one record at pixel centres (for footprint checks).
void or_alpha_at(const double* rec1, int64_t m, const int32_t* pix, double* out) {
  for (int64_t j = 0; j < m; ++j) out[j] = alpha_raw<double>(rec1, pix[2 * j] + 0.5, pix[2 * j + 1] + 0.5);
}

// SH basis (for pinning against an independent library routine).
void or_sh_basis(int deg, int64_t m, const double* dirs, double* out) {
  const int K = sh_count(deg);
  for (int64_t j = 0; j < m; ++j) sh_basis<double>(deg, dirs[3 * j], dirs[3 * j + 1], dirs[3 * j + 2], out + K * j);
}

}  // extern "C"
