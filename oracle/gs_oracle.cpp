// CPU oracle for differentiable tile-based Gaussian splatting.
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product path may load, call or link
// this file: it exists so that tests/, the smoke check and the CPU-baseline leg
// of bench.py can compare the CUDA library against a plain, slow, obviously
// correct restatement of the method. It shares no code, header, table or
// constant with the CUDA library.
//
// What it computes. The paper (arXiv 2606.11390, §4 "Distributed Gaussian
// Splatting") names the operators of a Gaussian-splatting training step (SH
// colour evaluation, projection, per-camera depth sort, tile rasterisation and
// their backward passes with gradient accumulation) and defers their
// mathematics to 3D Gaussian Splatting (Kerbl et al. 2023, cited in §1). The
// steps below restate that published formulation:
//   project   : activations, view transform, EWA covariance Σ2 = J W Σ Wᵀ Jᵀ + eps,
//               conic, 2D mean, 3-sigma radius, tile rectangle, SH colour.
//   bin_sort  : one (tile | depth) key per (view, Gaussian, tile) pair, stable sort.
//   raster    : per-pixel front-to-back alpha compositing with alpha cap,
//               alpha cutoff and transmittance early stop.
//   backward  : the exact derivative of all of the above, with the set of
//               composited (pixel, splat) pairs held fixed.
//
// Precision policy. Every decision that produces an integer or selects a
// branch (visibility, tile rectangle, alpha cutoff / cap, early stop, clamp
// flags) is taken in the precision R of the instantiation. For R = float the
// rectangle path is evaluated in a fixed, documented operation order with no
// contraction (build flag -ffp-contract=off), so that a float GPU kernel that
// follows the same order produces identical integers. All gradient arithmetic
// is carried out in double, given those decisions.
//
// Pins (tests/test_oracle_*.py): brute force tile enumeration, closed form for
// an isotropic splat, sum(alpha*T) + T_final = 1, SH orthonormality by
// quadrature and agreement with scipy's spherical harmonics, an independent
// untiled renderer, python's sort on (tile, depth, index), central finite
// differences in double for every parameter gradient, textbook Adam.

#ifdef _OPENMP
#include <omp.h>
#endif
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

// ------------------------------------------------------------------------
// Configuration and camera records (oracle-private layouts).
// ------------------------------------------------------------------------
struct OConfig {
  int32_t tile_w, tile_h, sh_degree, pad;
  float near_plane, far_plane, eps2d, alpha_cap, alpha_min, t_stop;
  float bg[3];
};

// Camera as passed from Python: viewmat row-major 4x4 (world -> camera,
// OpenCV axes: +x right, +y down, +z forward), then fx, fy, cx, cy.
struct OCam {
  double Wd[9], tvd[3];
  float Wf[9], tvf[3];
  double fx, fy, cx, cy;
  float fxf, fyf, cxf, cyf;
  int width, height;
};

template <class R> struct CamView;
template <> struct CamView<float> {
  static const float* W(const OCam& c) { return c.Wf; }
  static const float* tv(const OCam& c) { return c.tvf; }
  static float fx(const OCam& c) { return c.fxf; }
  static float fy(const OCam& c) { return c.fyf; }
  static float cx(const OCam& c) { return c.cxf; }
  static float cy(const OCam& c) { return c.cyf; }
};
template <> struct CamView<double> {
  static const double* W(const OCam& c) { return c.Wd; }
  static const double* tv(const OCam& c) { return c.tvd; }
  static double fx(const OCam& c) { return c.fx; }
  static double fy(const OCam& c) { return c.fy; }
  static double cx(const OCam& c) { return c.cx; }
  static double cy(const OCam& c) { return c.cy; }
};

std::vector<OCam> load_cams(const float* cams, const int32_t* sizes, int V) {
  std::vector<OCam> out(V);
  for (int v = 0; v < V; ++v) {
    const float* m = cams + 20 * v;
    OCam& c = out[v];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) {
        c.Wf[3 * i + j] = m[4 * i + j];
        c.Wd[3 * i + j] = m[4 * i + j];
      }
      c.tvf[i] = m[4 * i + 3];
      c.tvd[i] = m[4 * i + 3];
    }
    c.fxf = m[16]; c.fyf = m[17]; c.cxf = m[18]; c.cyf = m[19];
    c.fx = m[16]; c.fy = m[17]; c.cx = m[18]; c.cy = m[19];
    c.width = sizes[2 * v];
    c.height = sizes[2 * v + 1];
  }
  return out;
}

struct TileLayout {
  std::vector<int64_t> ntx, nty, tile_base, pix_base;
  int64_t n_tiles = 0, n_pix = 0;
};

TileLayout make_layout(const std::vector<OCam>& cams, const OConfig& cfg) {
  TileLayout L;
  int V = (int)cams.size();
  L.ntx.resize(V); L.nty.resize(V); L.tile_base.resize(V + 1); L.pix_base.resize(V + 1);
  L.tile_base[0] = 0; L.pix_base[0] = 0;
  for (int v = 0; v < V; ++v) {
    L.ntx[v] = (cams[v].width + cfg.tile_w - 1) / cfg.tile_w;
    L.nty[v] = (cams[v].height + cfg.tile_h - 1) / cfg.tile_h;
    L.tile_base[v + 1] = L.tile_base[v] + L.ntx[v] * L.nty[v];
    L.pix_base[v + 1] = L.pix_base[v] + (int64_t)cams[v].width * cams[v].height;
  }
  L.n_tiles = L.tile_base[V];
  L.n_pix = L.pix_base[V];
  return L;
}

// ------------------------------------------------------------------------
// Exponential used for the scale activation s = exp(log_scale).
//
// The scale feeds the tile rectangle, an integer result, so both sides of the
// parity check must round it identically; neither libm's expf nor CUDA's expf
// is specified to the last bit. This routine follows Cody & Waite (1980):
// reduce x = k ln2 + r with |r| <= ln2/2 using a two-part ln2 (the high part
// has 16 significant bits so k*ln2_hi is exact for |k| < 256), evaluate the
// Taylor series of e^r to degree 7 by Horner's rule, and scale by 2^k built
// from the exponent bits. The input is clamped to [-87, 88] so that 2^k stays
// a normal float. Every step is a single IEEE operation (no fused multiply-add).
// Error versus exp in double: at most 2 ulp (tests/test_oracle_math.py).
// ------------------------------------------------------------------------
float exp_cody_waite(float x) {
  if (!(x > -87.0f)) x = -87.0f;  // NaN also lands here
  if (x > 88.0f) x = 88.0f;
  const float log2e = 1.44269502f;            // 1/ln 2 rounded to float
  const float ln2_hi = 0.693145751953125f;    // 45426 / 65536
  const float ln2_lo = 1.42860677e-6f;        // ln 2 - ln2_hi, rounded to float
  float k = std::nearbyint(x * log2e);
  float r = x - k * ln2_hi;
  r = r - k * ln2_lo;
  // 1/n! for n = 2..7, each rounded to float
  const float c7 = 1.0f / 5040.0f, c6 = 1.0f / 720.0f, c5 = 1.0f / 120.0f;
  const float c4 = 1.0f / 24.0f, c3 = 1.0f / 6.0f, c2 = 0.5f;
  float p = c7;
  p = p * r + c6;
  p = p * r + c5;
  p = p * r + c4;
  p = p * r + c3;
  p = p * r + c2;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  int32_t ki = (int32_t)k;
  uint32_t bits = (uint32_t)(ki + 127) << 23;
  float scale;
  std::memcpy(&scale, &bits, 4);
  return p * scale;
}

inline float scale_exp(float x) { return exp_cody_waite(x); }
inline double scale_exp(double x) { return std::exp(x); }

template <class R> inline R clamp_to(R x, R lo, R hi) { return x < lo ? lo : (x > hi ? hi : x); }

// Tile index bound from a float coordinate: NaN -> 0, otherwise clamp to [0, n].
template <class R> inline int tile_clamp(R f, int n) {
  if (f >= R(0)) {
    if (f <= R(n)) return (int)f;
    return n;
  }
  return 0;
}

// ------------------------------------------------------------------------
// Real spherical harmonics up to degree 3, in the coefficient order used by
// 3D Gaussian Splatting: index l*l + l + m, m = -l..l. Each basis function is
// a normalisation K times a Cartesian polynomial in the unit direction. The
// normalisations are computed here from the definition
//   K_l^m = sqrt((2l+1)/(4 pi) * (l-|m|)! / (l+|m|)!),
// times sqrt(2) for m != 0, times the integer factor that the associated
// Legendre function P_l^|m| (Condon-Shortley phase included) contributes when
// it is written as a polynomial in (x, y, z).
// ------------------------------------------------------------------------
struct SHBasis {
  double c[16];
  SHBasis() {
    auto fact = [](int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; };
    auto K = [&](int l, int m) {
      m = std::abs(m);
      return std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - m) / fact(l + m));
    };
    const double s2 = std::sqrt(2.0);
    c[0] = K(0, 0);
    c[1] = -s2 * K(1, 1);          // P_1^1 = -sin(theta)            -> y
    c[2] = K(1, 0);                //                                 -> z
    c[3] = -s2 * K(1, 1);          //                                 -> x
    c[4] = 6.0 * s2 * K(2, 2);     // P_2^2 = 3 sin^2, sin(2phi)=2xy  -> xy
    c[5] = -3.0 * s2 * K(2, 1);    // P_2^1 = -3 z sin                -> yz
    c[6] = 0.5 * K(2, 0);          // P_2^0 = (3z^2-1)/2              -> 2z^2-x^2-y^2
    c[7] = -3.0 * s2 * K(2, 1);    //                                 -> xz
    c[8] = 3.0 * s2 * K(2, 2);     // cos(2phi) sin^2 = x^2-y^2       -> x^2-y^2
    c[9] = -15.0 * s2 * K(3, 3);   // P_3^3 = -15 sin^3               -> y(3x^2-y^2)
    c[10] = 30.0 * s2 * K(3, 2);   // P_3^2 = 15 z sin^2, 2xy         -> xyz
    c[11] = -1.5 * s2 * K(3, 1);   // P_3^1 = -1.5 (5z^2-1) sin       -> y(4z^2-x^2-y^2)
    c[12] = 0.5 * K(3, 0);         // P_3^0 = (5z^3-3z)/2             -> z(2z^2-3x^2-3y^2)
    c[13] = -1.5 * s2 * K(3, 1);   //                                 -> x(4z^2-x^2-y^2)
    c[14] = 15.0 * s2 * K(3, 2);   //                                 -> z(x^2-y^2)
    c[15] = -15.0 * s2 * K(3, 3);  //                                 -> x(x^2-3y^2)
  }
  // Polynomial parts p_i and their gradients; Y_i = c[i] * p_i.
  template <class R>
  static void poly(const R d[3], R p[16]) {
    R x = d[0], y = d[1], z = d[2];
    R xx = x * x, yy = y * y, zz = z * z;
    p[0] = R(1);
    p[1] = y; p[2] = z; p[3] = x;
    p[4] = x * y; p[5] = y * z; p[6] = R(2) * zz - xx - yy; p[7] = x * z; p[8] = xx - yy;
    p[9] = y * (R(3) * xx - yy);
    p[10] = x * y * z;
    p[11] = y * (R(4) * zz - xx - yy);
    p[12] = z * (R(2) * zz - R(3) * xx - R(3) * yy);
    p[13] = x * (R(4) * zz - xx - yy);
    p[14] = z * (xx - yy);
    p[15] = x * (xx - R(3) * yy);
  }
  static void poly_grad(const double d[3], double g[16][3]) {
    double x = d[0], y = d[1], z = d[2];
    double xx = x * x, yy = y * y, zz = z * z;
    auto set = [&](int i, double a, double b, double c) { g[i][0] = a; g[i][1] = b; g[i][2] = c; };
    set(0, 0, 0, 0);
    set(1, 0, 1, 0); set(2, 0, 0, 1); set(3, 1, 0, 0);
    set(4, y, x, 0); set(5, 0, z, y); set(6, -2 * x, -2 * y, 4 * z); set(7, z, 0, x); set(8, 2 * x, -2 * y, 0);
    set(9, 6 * x * y, 3 * xx - 3 * yy, 0);
    set(10, y * z, x * z, x * y);
    set(11, -2 * x * y, 4 * zz - xx - 3 * yy, 8 * y * z);
    set(12, -6 * x * z, -6 * y * z, 6 * zz - 3 * xx - 3 * yy);
    set(13, 4 * zz - 3 * xx - yy, -2 * x * y, 8 * x * z);
    set(14, 2 * x * z, -2 * y * z, xx - yy);
    set(15, 3 * xx - 3 * yy, -6 * x * y, 0);
  }
};
const SHBasis& sh_basis() { static SHBasis b; return b; }

inline int sh_count(int degree) { return (degree + 1) * (degree + 1); }

// ------------------------------------------------------------------------
// Forward projection of one (view, Gaussian) pair.
// ------------------------------------------------------------------------
template <class R> struct Proj {
  bool visible = false;
  bool clamp_x = false, clamp_y = false;   // frustum clamp active -> zero gradient
  bool rgb_clamped[3] = {false, false, false};
  R s[3], qn[4], Rm[9], M[9], Sig[9];
  R t[3], u, w, uc, wc;
  R J00, J02, J11, J12;
  R T[6];        // J * W, 2x3 row-major
  R U[6];        // T * Sigma, 2x3
  R a, b, c;     // Sigma2 entries 00, 01, 11 (eps included)
  R det, A, B, C, mx, my, radius;
  R o;
  R dvec[3], dnorm, dir[3];
  R rgb_raw[3], rgb[3];
  int rect[4] = {0, 0, 0, 0};
  uint32_t count = 0;
};

// Forward decisions that the double-precision gradient pass reuses.
struct ProjDecision {
  bool visible, clamp_x, clamp_y, rgb_clamped[3];
};

// One (view, Gaussian) projection. The rectangle path (steps 1-8) is written
// in the operation order that the float GPU kernel follows; with no
// contraction both produce identical rectangles. `forced` (may be null)
// overrides the branch decisions with those of another precision.
template <class R>
void project_one(const R* mean, const R* log_scale, const R* quat, R opac_logit, const R* sh, int sh_degree,
                 const OCam& cam, const OConfig& cfg, Proj<R>& P, const ProjDecision* forced) {
  using CV = CamView<R>;
  const R* W = CV::W(cam);
  const R* tv = CV::tv(cam);
  const R fx = CV::fx(cam), fy = CV::fy(cam), cx = CV::cx(cam), cy = CV::cy(cam);
  // 1. activations
  for (int i = 0; i < 3; ++i) P.s[i] = scale_exp(log_scale[i]);
  R n2 = quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3];
  R nrm = std::sqrt(n2);
  for (int i = 0; i < 4; ++i) P.qn[i] = quat[i] / nrm;
  P.o = R(1) / (R(1) + std::exp(-opac_logit));
  // 3. rotation matrix of the unit quaternion (w, x, y, z), M = R diag(s), Sigma = M M^T
  {
    R qw = P.qn[0], qx = P.qn[1], qy = P.qn[2], qz = P.qn[3];
    R xx = qx * qx, yy = qy * qy, zz = qz * qz;
    R xy = qx * qy, xz = qx * qz, yz = qy * qz;
    R wx = qw * qx, wy = qw * qy, wz = qw * qz;
    R* Rm = P.Rm;
    Rm[0] = R(1) - R(2) * (yy + zz);
    Rm[1] = R(2) * (xy - wz);
    Rm[2] = R(2) * (xz + wy);
    Rm[3] = R(2) * (xy + wz);
    Rm[4] = R(1) - R(2) * (xx + zz);
    Rm[5] = R(2) * (yz - wx);
    Rm[6] = R(2) * (xz - wy);
    Rm[7] = R(2) * (yz + wx);
    Rm[8] = R(1) - R(2) * (xx + yy);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) P.M[3 * i + j] = Rm[3 * i + j] * P.s[j];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        P.Sig[3 * i + j] = P.M[3 * i] * P.M[3 * j] + P.M[3 * i + 1] * P.M[3 * j + 1] + P.M[3 * i + 2] * P.M[3 * j + 2];
  }
  // 2. view transform
  for (int i = 0; i < 3; ++i) P.t[i] = W[3 * i] * mean[0] + W[3 * i + 1] * mean[1] + W[3 * i + 2] * mean[2] + tv[i];
  const R tz = P.t[2];
  bool visible = (tz > R(cfg.near_plane)) && (tz < R(cfg.far_plane));
  // 4. Jacobian of the pinhole projection, with the frustum clamp
  const R Wf = R(cam.width), Hf = R(cam.height);
  P.u = P.t[0] / tz;
  P.w = P.t[1] / tz;
  const R lox = (R(-0.15) * Wf - cx) / fx, hix = (R(1.15) * Wf - cx) / fx;
  const R loy = (R(-0.15) * Hf - cy) / fy, hiy = (R(1.15) * Hf - cy) / fy;
  P.uc = clamp_to(P.u, lox, hix);
  P.wc = clamp_to(P.w, loy, hiy);
  P.clamp_x = !(P.u > lox && P.u < hix);
  P.clamp_y = !(P.w > loy && P.w < hiy);
  P.J00 = fx / tz;
  P.J02 = (-fx * P.uc) / tz;
  P.J11 = fy / tz;
  P.J12 = (-fy * P.wc) / tz;
  for (int j = 0; j < 3; ++j) {
    P.T[j] = P.J00 * W[j] + P.J02 * W[6 + j];
    P.T[3 + j] = P.J11 * W[3 + j] + P.J12 * W[6 + j];
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j)
      P.U[3 * i + j] = P.T[3 * i] * P.Sig[j] + P.T[3 * i + 1] * P.Sig[3 + j] + P.T[3 * i + 2] * P.Sig[6 + j];
  const R eps = R(cfg.eps2d);
  P.a = P.U[0] * P.T[0] + P.U[1] * P.T[1] + P.U[2] * P.T[2] + eps;
  P.b = P.U[0] * P.T[3] + P.U[1] * P.T[4] + P.U[2] * P.T[5];
  P.c = P.U[3] * P.T[3] + P.U[4] * P.T[4] + P.U[5] * P.T[5] + eps;
  // 5. determinant and conic
  P.det = P.a * P.c - P.b * P.b;
  visible = visible && (P.det > R(0));
  P.A = P.c / P.det;
  P.B = -P.b / P.det;
  P.C = P.a / P.det;
  // 6. 2D mean (unclamped)
  P.mx = fx * P.u + cx;
  P.my = fy * P.w + cy;
  // 7. radius: 3 sigma of the larger eigenvalue of Sigma2
  const R half = R(0.5) * (P.a + P.c);
  const R disc = half * half - P.det;
  const R lam = half + std::sqrt(std::max(R(0.1), disc));
  P.radius = std::ceil(R(3) * std::sqrt(lam));
  // 8. tile rectangle
  const int ntx = (cam.width + cfg.tile_w - 1) / cfg.tile_w;
  const int nty = (cam.height + cfg.tile_h - 1) / cfg.tile_h;
  const R tw = R(cfg.tile_w), th = R(cfg.tile_h);
  int x0 = tile_clamp(std::floor((P.mx - P.radius) / tw), ntx);
  int x1 = tile_clamp(std::ceil((P.mx + P.radius) / tw), ntx);
  int y0 = tile_clamp(std::floor((P.my - P.radius) / th), nty);
  int y1 = tile_clamp(std::ceil((P.my + P.radius) / th), nty);
  uint32_t count = 0;
  if (visible && x1 > x0 && y1 > y0) count = (uint32_t)((x1 - x0) * (y1 - y0));
  visible = visible && count > 0;
  if (visible) {
    P.rect[0] = x0; P.rect[1] = y0; P.rect[2] = x1; P.rect[3] = y1;
  }
  P.count = visible ? count : 0;
  // 9. view-dependent colour from the SH coefficients
  {
    const R* Wm = W;
    // camera centre c = -W^T tv
    R cc[3];
    for (int j = 0; j < 3; ++j) cc[j] = -(Wm[j] * tv[0] + Wm[3 + j] * tv[1] + Wm[6 + j] * tv[2]);
    for (int j = 0; j < 3; ++j) P.dvec[j] = mean[j] - cc[j];
    P.dnorm = std::sqrt(P.dvec[0] * P.dvec[0] + P.dvec[1] * P.dvec[1] + P.dvec[2] * P.dvec[2]);
    for (int j = 0; j < 3; ++j) P.dir[j] = P.dvec[j] / P.dnorm;
    R p[16];
    SHBasis::poly(P.dir, p);
    const SHBasis& B = sh_basis();
    const int nb = sh_count(sh_degree);
    for (int ch = 0; ch < 3; ++ch) {
      R acc = R(0);
      for (int i = 0; i < nb; ++i) acc += R(B.c[i]) * p[i] * sh[3 * i + ch];
      P.rgb_raw[ch] = acc + R(0.5);
      P.rgb_clamped[ch] = !(P.rgb_raw[ch] > R(0));
      P.rgb[ch] = P.rgb_clamped[ch] ? R(0) : P.rgb_raw[ch];
    }
  }
  P.visible = visible;
  if (forced) {
    P.visible = forced->visible;
    P.clamp_x = forced->clamp_x;
    P.clamp_y = forced->clamp_y;
    if (P.clamp_x) P.uc = P.u < lox ? lox : hix;
    else P.uc = P.u;
    if (P.clamp_y) P.wc = P.w < loy ? loy : hiy;
    else P.wc = P.w;
    for (int ch = 0; ch < 3; ++ch) {
      P.rgb_clamped[ch] = forced->rgb_clamped[ch];
      P.rgb[ch] = P.rgb_clamped[ch] ? R(0) : P.rgb_raw[ch];
    }
    // recompute the clamp-dependent quantities with the forced decision
    P.J02 = (-fx * P.uc) / tz;
    P.J12 = (-fy * P.wc) / tz;
    for (int j = 0; j < 3; ++j) {
      P.T[j] = P.J00 * W[j] + P.J02 * W[6 + j];
      P.T[3 + j] = P.J11 * W[3 + j] + P.J12 * W[6 + j];
    }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j)
        P.U[3 * i + j] = P.T[3 * i] * P.Sig[j] + P.T[3 * i + 1] * P.Sig[3 + j] + P.T[3 * i + 2] * P.Sig[6 + j];
    P.a = P.U[0] * P.T[0] + P.U[1] * P.T[1] + P.U[2] * P.T[2] + eps;
    P.b = P.U[0] * P.T[3] + P.U[1] * P.T[4] + P.U[2] * P.T[5];
    P.c = P.U[3] * P.T[3] + P.U[4] * P.T[4] + P.U[5] * P.T[5] + eps;
    P.det = P.a * P.c - P.b * P.b;
    P.A = P.c / P.det;
    P.B = -P.b / P.det;
    P.C = P.a / P.det;
  }
}

// Projected record layout (12 values per (view, Gaussian)):
//   0 mean2d.x  1 mean2d.y  2 conic A  3 conic B  4 conic C  5 opacity
//   6 depth     7 radius    8 r        9 g       10 b       11 0
template <class R> void write_record(const Proj<R>& P, R* rec) {
  rec[0] = P.mx; rec[1] = P.my; rec[2] = P.A; rec[3] = P.B; rec[4] = P.C; rec[5] = P.o;
  rec[6] = P.t[2]; rec[7] = P.radius; rec[8] = P.rgb[0]; rec[9] = P.rgb[1]; rec[10] = P.rgb[2]; rec[11] = R(0);
}

template <class R>
void project_all(const R* means, const R* log_scales, const R* quats, const R* opac, const R* sh, int64_t N,
                 const std::vector<OCam>& cams, const OConfig& cfg, R* projected, int16_t* rects, uint32_t* counts) {
  const int V = (int)cams.size();
  for (int v = 0; v < V; ++v) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t g = 0; g < N; ++g) {
      Proj<R> P;
      project_one<R>(means + 3 * g, log_scales + 3 * g, quats + 4 * g, opac[g], sh + 48 * g, cfg.sh_degree, cams[v], cfg,
                     P, nullptr);
      const int64_t vg = (int64_t)v * N + g;
      R* rec = projected + 12 * vg;
      if (P.visible) write_record(P, rec);
      else for (int i = 0; i < 12; ++i) rec[i] = R(0);
      for (int i = 0; i < 4; ++i) rects[4 * vg + i] = (int16_t)P.rect[i];
      counts[vg] = P.count;
    }
  }
}

// ------------------------------------------------------------------------
// Key emission and stable sort: key = (global tile id << 32) | bits(depth).
// Emission order: views ascending, Gaussians ascending, rectangle row-major.
// ------------------------------------------------------------------------
inline uint32_t float_bits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

template <class R>
int64_t bin_sort(const R* projected, const int16_t* rects, const uint32_t* counts, int64_t N, const std::vector<OCam>& cams,
                 const OConfig& cfg, uint64_t* keys, uint32_t* vals, int64_t capacity, uint32_t* ranges) {
  const TileLayout L = make_layout(cams, cfg);
  const int V = (int)cams.size();
  std::vector<std::pair<uint64_t, uint32_t>> list;
  for (int v = 0; v < V; ++v) {
    for (int64_t g = 0; g < N; ++g) {
      const int64_t vg = (int64_t)v * N + g;
      if (counts[vg] == 0) continue;
      const float depth = (float)projected[12 * vg + 6];
      const int16_t* r = rects + 4 * vg;
      for (int ty = r[1]; ty < r[3]; ++ty)
        for (int tx = r[0]; tx < r[2]; ++tx) {
          uint64_t tile = (uint64_t)(L.tile_base[v] + (int64_t)ty * L.ntx[v] + tx);
          list.push_back({(tile << 32) | float_bits(depth), (uint32_t)vg});
        }
    }
  }
  std::stable_sort(list.begin(), list.end(),
                   [](const std::pair<uint64_t, uint32_t>& x, const std::pair<uint64_t, uint32_t>& y) { return x.first < y.first; });
  const int64_t I = (int64_t)list.size();
  for (int64_t t = 0; t < L.n_tiles; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
  if (I > capacity) return I;
  for (int64_t i = 0; i < I; ++i) {
    keys[i] = list[i].first;
    vals[i] = list[i].second;
    const uint64_t tile = list[i].first >> 32;
    if (i == 0 || (list[i - 1].first >> 32) != tile) ranges[2 * tile] = (uint32_t)i;
    if (i == I - 1 || (list[i + 1].first >> 32) != tile) ranges[2 * tile + 1] = (uint32_t)(i + 1);
  }
  return I;
}

// ------------------------------------------------------------------------
// Compositing.
// ------------------------------------------------------------------------
// Relative distance of a computed value from a decision threshold; a small
// value means the decision could go either way under a different rounding.
inline double rel_margin(double value, double threshold) {
  double s = std::max(std::fabs(threshold), 1e-30);
  return std::fabs(value - threshold) / s;
}
const double kMarginal = 1e-4;

// Writes shared between pixels: a flag set to 1 and a gradient sum. In the
// OpenMP build (used only to time the oracle on all host cores) pixels run
// in parallel, so these become atomic; the serial build does plain stores and
// adds in the same order as always.
inline void flag_set(uint8_t* p) { __atomic_store_n(p, (uint8_t)1, __ATOMIC_RELAXED); }
inline void acc(double* p, double v) {
#ifdef _OPENMP
#pragma omp atomic
#endif
  *p += v;
}

// Composite one pixel. `hits` (may be null) receives, for each composited
// entry, 2*k + (1 if the alpha cap was active).
// Optionally flags marginal decisions per (view, Gaussian) and per pixel.
// `sig` (may be null) receives a signature of the composited set (used by the
// finite-difference tests to detect a perturbation that changed the set).
template <class R>
void composite_pixel(const R* projected, const uint32_t* vals, uint32_t start, uint32_t end, R px, R py, const OConfig& cfg,
                     R out[3], R& T_final, uint32_t& last, std::vector<int64_t>* hits, uint8_t* marg_vg, bool* marg_pix,
                     uint64_t* sig = nullptr, uint32_t* ncomp = nullptr) {
  if (sig) *sig = 0;
  if (ncomp) *ncomp = 0;
  R T = R(1);
  R Cacc[3] = {R(0), R(0), R(0)};
  last = 0;
  const R cap = R(cfg.alpha_cap), amin = R(cfg.alpha_min), tstop = R(cfg.t_stop);
  for (uint32_t k = start; k < end; ++k) {
    const uint32_t vg = vals[k];
    const R* rec = projected + 12 * (int64_t)vg;
    const R dx = px - rec[0], dy = py - rec[1];
    const R power = R(0.5) * (rec[2] * dx * dx + rec[4] * dy * dy) + rec[3] * dx * dy;
    bool marg = false;
    if (power < R(0)) {
      if (std::fabs((double)power) < 1e-5) marg = true;
      if (marg && marg_vg) { flag_set(marg_vg + vg); if (marg_pix) *marg_pix = true; }
      continue;
    }
    const R G = std::exp(-power);
    const R oG = rec[5] * G;
    const R alpha = std::min(cap, oG);
    if (rel_margin((double)oG, (double)cap) < kMarginal) marg = true;
    if (rel_margin((double)alpha, (double)amin) < kMarginal) marg = true;
    if (marg && marg_vg) { flag_set(marg_vg + vg); if (marg_pix) *marg_pix = true; }
    if (alpha < amin) continue;
    const R Tn = T * (R(1) - alpha);
    if (rel_margin((double)Tn, (double)tstop) < kMarginal) {
      if (marg_vg) flag_set(marg_vg + vg);
      if (marg_pix) *marg_pix = true;
    }
    if (Tn < tstop) break;
    for (int ch = 0; ch < 3; ++ch) Cacc[ch] += rec[8 + ch] * alpha * T;
    T = Tn;
    last = k - start + 1;
    if (hits) hits->push_back(2 * (int64_t)k + (oG > cap ? 1 : 0));
    if (sig) *sig += ((uint64_t)(k - start) + 1) * 0x9E3779B97F4A7C15ull + (oG > cap ? 1 : 0);
    if (ncomp) ++*ncomp;
  }
  for (int ch = 0; ch < 3; ++ch) out[ch] = Cacc[ch] + T * R(cfg.bg[ch]);
  T_final = T;
}

// Locate (view, tile, pixel) coordinates of a global tile id.
inline int view_of_tile(const TileLayout& L, int64_t tile) {
  int v = 0;
  while (tile >= L.tile_base[v + 1]) ++v;
  return v;
}

template <class R>
void raster_fwd(const R* projected, const uint32_t* vals, const uint32_t* ranges, const std::vector<OCam>& cams,
                const OConfig& cfg, const int64_t* tiles, int64_t n_sel, R* image, R* final_T, uint32_t* last,
                uint8_t* marg_vg, uint8_t* marg_pix, uint64_t* hitsig, uint32_t* ncomp) {
  const TileLayout L = make_layout(cams, cfg);
  const int64_t nt = tiles ? n_sel : L.n_tiles;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t ti = 0; ti < nt; ++ti) {
    const int64_t tile = tiles ? tiles[ti] : ti;
    const int v = view_of_tile(L, tile);
    const int64_t local = tile - L.tile_base[v];
    const int tx = (int)(local % L.ntx[v]), ty = (int)(local / L.ntx[v]);
    const int Wv = cams[v].width, Hv = cams[v].height;
    for (int j = ty * cfg.tile_h; j < std::min((ty + 1) * cfg.tile_h, Hv); ++j)
      for (int i = tx * cfg.tile_w; i < std::min((tx + 1) * cfg.tile_w, Wv); ++i) {
        const int64_t p = L.pix_base[v] + (int64_t)j * Wv + i;
        R out[3];
        bool mp = false;
        composite_pixel<R>(projected, vals, ranges[2 * tile], ranges[2 * tile + 1], R(i) + R(0.5), R(j) + R(0.5), cfg, out,
                           final_T[p], last[p], nullptr, marg_vg, &mp, hitsig ? hitsig + p : nullptr,
                           ncomp ? ncomp + p : nullptr);
        for (int ch = 0; ch < 3; ++ch) image[3 * p + ch] = out[ch];
        if (marg_pix) marg_pix[p] = mp ? 1 : 0;
      }
  }
}

// Backward of compositing for one pixel, in double, with the composited set
// taken from the forward pass in precision R. Accumulates into d_proj (9 per
// record: mean2d x/y, conic A/B/C, r/g/b, opacity).
template <class R>
void composite_pixel_bwd(const R* projected, const uint32_t* vals, uint32_t start, uint32_t end, int px_i, int py_i,
                         const OConfig& cfg, const double* dout, double* d_proj) {
  std::vector<int64_t> hits;
  R out[3], Tf;
  uint32_t last;
  const R px = R(px_i) + R(0.5), py = R(py_i) + R(0.5);
  composite_pixel<R>(projected, vals, start, end, px, py, cfg, out, Tf, last, &hits, nullptr, nullptr);
  const size_t n = hits.size();
  if (n == 0) return;
  const double cap = cfg.alpha_cap;
  const double pxd = (double)px_i + 0.5, pyd = (double)py_i + 0.5;
  std::vector<double> alpha(n), G(n), Tk(n + 1), dx(n), dy(n);
  std::vector<char> capped(n);
  Tk[0] = 1.0;
  for (size_t i = 0; i < n; ++i) {
    const R* rec = projected + 12 * (int64_t)vals[hits[i] >> 1];
    dx[i] = pxd - (double)rec[0];
    dy[i] = pyd - (double)rec[1];
    const double power = 0.5 * ((double)rec[2] * dx[i] * dx[i] + (double)rec[4] * dy[i] * dy[i]) + (double)rec[3] * dx[i] * dy[i];
    G[i] = std::exp(-power);
    capped[i] = (char)(hits[i] & 1);  // cap decision as taken by the forward in R
    alpha[i] = capped[i] ? cap : (double)rec[5] * G[i];
    Tk[i + 1] = Tk[i] * (1.0 - alpha[i]);
  }
  const double Tfin = Tk[n];
  // suffix sums S_k = sum_{j>k} c_j alpha_j T_j
  double S[3] = {0, 0, 0};
  for (size_t ii = n; ii-- > 0;) {
    const int64_t vg = vals[hits[ii] >> 1];
    const R* rec = projected + 12 * vg;
    double* g = d_proj + 9 * vg;
    const double w = alpha[ii] * Tk[ii];
    double dalpha = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      const double c = (double)rec[8 + ch];
      acc(g + 5 + ch, w * dout[ch]);
      dalpha += dout[ch] * (c * Tk[ii] - S[ch] / (1.0 - alpha[ii]) - Tfin * (double)cfg.bg[ch] / (1.0 - alpha[ii]));
    }
    for (int ch = 0; ch < 3; ++ch) S[ch] += (double)rec[8 + ch] * w;
    if (!capped[ii]) {
      // alpha = o * exp(-power)
      acc(g + 8, dalpha * G[ii]);
      const double dpower = -dalpha * alpha[ii];
      const double A = rec[2], B = rec[3], C = rec[4];
      // power = 0.5 (A dx^2 + C dy^2) + B dx dy, dx = px - mean.x
      acc(g + 0, dpower * (-(A * dx[ii] + B * dy[ii])));
      acc(g + 1, dpower * (-(B * dx[ii] + C * dy[ii])));
      acc(g + 2, dpower * 0.5 * dx[ii] * dx[ii]);
      acc(g + 3, dpower * dx[ii] * dy[ii]);
      acc(g + 4, dpower * 0.5 * dy[ii] * dy[ii]);
    }
  }
}

template <class R>
void raster_bwd(const R* projected, const uint32_t* vals, const uint32_t* ranges, const std::vector<OCam>& cams,
                const OConfig& cfg, const int64_t* tiles, int64_t n_sel, const double* dL_dimage, double* d_proj) {
  const TileLayout L = make_layout(cams, cfg);
  const int64_t nt = tiles ? n_sel : L.n_tiles;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int64_t ti = 0; ti < nt; ++ti) {
    const int64_t tile = tiles ? tiles[ti] : ti;
    const int v = view_of_tile(L, tile);
    const int64_t local = tile - L.tile_base[v];
    const int tx = (int)(local % L.ntx[v]), ty = (int)(local / L.ntx[v]);
    const int Wv = cams[v].width, Hv = cams[v].height;
    for (int j = ty * cfg.tile_h; j < std::min((ty + 1) * cfg.tile_h, Hv); ++j)
      for (int i = tx * cfg.tile_w; i < std::min((tx + 1) * cfg.tile_w, Wv); ++i) {
        const int64_t p = L.pix_base[v] + (int64_t)j * Wv + i;
        composite_pixel_bwd<R>(projected, vals, ranges[2 * tile], ranges[2 * tile + 1], i, j, cfg, dL_dimage + 3 * p, d_proj);
      }
  }
}

// ------------------------------------------------------------------------
// Backward of the projection for one Gaussian, summed over views, in double.
// Decisions (visibility, clamps) come from the precision-R forward.
// ------------------------------------------------------------------------
template <class R>
void project_bwd_one(const R* means, const R* log_scales, const R* quats, const R* opac, const R* sh, int64_t N, int64_t g,
                     const std::vector<OCam>& cams, const OConfig& cfg, const double* d_proj, double* gm, double* gls,
                     double* gq, double* go, double* gsh) {
  const int V = (int)cams.size();
  double mean[3], ls[3], q[4], sh_d[48];
  for (int i = 0; i < 3; ++i) { mean[i] = means[3 * g + i]; ls[i] = log_scales[3 * g + i]; }
  for (int i = 0; i < 4; ++i) q[i] = quats[4 * g + i];
  for (int i = 0; i < 48; ++i) sh_d[i] = sh[48 * g + i];
  const double ol = opac[g];
  for (int i = 0; i < 3; ++i) { gm[i] = 0; gls[i] = 0; }
  for (int i = 0; i < 4; ++i) gq[i] = 0;
  *go = 0;
  for (int i = 0; i < 48; ++i) gsh[i] = 0;
  const int nb = sh_count(cfg.sh_degree);
  const SHBasis& SB = sh_basis();
  for (int v = 0; v < V; ++v) {
    const int64_t vg = (int64_t)v * N + g;
    Proj<R> PR;
    project_one<R>(means + 3 * g, log_scales + 3 * g, quats + 4 * g, opac[g], sh + 48 * g, cfg.sh_degree, cams[v], cfg, PR,
                   nullptr);
    if (!PR.visible) continue;
    ProjDecision dec;
    dec.visible = true;
    dec.clamp_x = PR.clamp_x;
    dec.clamp_y = PR.clamp_y;
    for (int ch = 0; ch < 3; ++ch) dec.rgb_clamped[ch] = PR.rgb_clamped[ch];
    Proj<double> P;
    project_one<double>(mean, ls, q, ol, sh_d, cfg.sh_degree, cams[v], cfg, P, &dec);
    const double* W = cams[v].Wd;
    const double fx = cams[v].fx, fy = cams[v].fy;
    const double* dp = d_proj + 9 * vg;
    // opacity
    *go += dp[8] * P.o * (1.0 - P.o);
    // colour -> SH coefficients and view direction
    double graw[3];
    for (int ch = 0; ch < 3; ++ch) graw[ch] = P.rgb_clamped[ch] ? 0.0 : dp[5 + ch];
    double pol[16], pg[16][3];
    SHBasis::poly(P.dir, pol);
    SHBasis::poly_grad(P.dir, pg);
    double gdir[3] = {0, 0, 0};
    for (int i = 0; i < nb; ++i) {
      double acc = 0;
      for (int ch = 0; ch < 3; ++ch) {
        gsh[3 * i + ch] += SB.c[i] * pol[i] * graw[ch];
        acc += sh_d[3 * i + ch] * graw[ch];
      }
      for (int k = 0; k < 3; ++k) gdir[k] += acc * SB.c[i] * pg[i][k];
    }
    // dir = dvec / |dvec|
    {
      double dd = P.dir[0] * gdir[0] + P.dir[1] * gdir[1] + P.dir[2] * gdir[2];
      for (int k = 0; k < 3; ++k) gm[k] += (gdir[k] - P.dir[k] * dd) / P.dnorm;
    }
    // conic (A, B, C) -> Sigma2 entries (a, b, c), with A = c/det, B = -b/det, C = a/det
    const double gA = dp[2], gB = dp[3], gC = dp[4];
    const double det = P.det;
    const double gdet = -(gA * P.c - gB * P.b + gC * P.a) / (det * det);
    const double ga = gC / det + gdet * P.c;
    const double gc = gA / det + gdet * P.a;
    const double gb = -gB / det - 2.0 * P.b * gdet;
    // Sigma2 = T Sigma T^T (+eps): symmetric gradient Gs
    const double Gs[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
    // gT = 2 Gs T Sigma = 2 Gs U ; gSigma = T^T Gs T
    double gT[6];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) gT[3 * i + j] = 2.0 * (Gs[2 * i] * P.U[j] + Gs[2 * i + 1] * P.U[3 + j]);
    double gSig[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int r = 0; r < 2; ++r)
          for (int s = 0; s < 2; ++s) acc += P.T[3 * r + i] * Gs[2 * r + s] * P.T[3 * s + j];
        gSig[3 * i + j] = acc;
      }
    // T = J W: rows T0 = J00 W0 + J02 W2, T1 = J11 W1 + J12 W2
    double gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
    for (int j = 0; j < 3; ++j) {
      gJ00 += gT[j] * W[j];
      gJ02 += gT[j] * W[6 + j];
      gJ11 += gT[3 + j] * W[3 + j];
      gJ12 += gT[3 + j] * W[6 + j];
    }
    const double tz = P.t[2];
    double gt[3] = {0, 0, 0};
    gt[2] += gJ00 * (-fx / (tz * tz)) + gJ11 * (-fy / (tz * tz));
    gt[2] += gJ02 * (fx * P.uc / (tz * tz)) + gJ12 * (fy * P.wc / (tz * tz));
    double gu = 0, gw = 0;
    if (!P.clamp_x) gu += gJ02 * (-fx / tz);
    if (!P.clamp_y) gw += gJ12 * (-fy / tz);
    // mean2d = (fx u + cx, fy w + cy)
    gu += dp[0] * fx;
    gw += dp[1] * fy;
    // u = tx / tz, w = ty / tz
    gt[0] += gu / tz;
    gt[1] += gw / tz;
    gt[2] += -gu * P.t[0] / (tz * tz) - gw * P.t[1] / (tz * tz);
    // t = W mean + tv
    for (int k = 0; k < 3; ++k) gm[k] += W[k] * gt[0] + W[3 + k] * gt[1] + W[6 + k] * gt[2];
    // Sigma = M M^T -> gM = (gSig + gSig^T) M
    double gM[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int k = 0; k < 3; ++k) acc += (gSig[3 * i + k] + gSig[3 * k + i]) * P.M[3 * k + j];
        gM[3 * i + j] = acc;
      }
    // M = Rm diag(s)
    double gR[9], gs[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        gR[3 * i + j] = gM[3 * i + j] * P.s[j];
        gs[j] += gM[3 * i + j] * P.Rm[3 * i + j];
      }
    for (int j = 0; j < 3; ++j) gls[j] += gs[j] * P.s[j];
    // Rm(qn), qn = (w, x, y, z)
    const double w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    double gqn[4];
    gqn[0] = 2.0 * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gqn[1] = 2.0 * (y * gR[1] + z * gR[2] + y * gR[3] - 2 * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] - 2 * x * gR[8]);
    gqn[2] = 2.0 * (-2 * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] - 2 * y * gR[8]);
    gqn[3] = 2.0 * (-2 * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2 * z * gR[4] + y * gR[5] + x * gR[6] + y * gR[7]);
    // qn = q / |q|
    const double qnorm = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double dotp = gqn[0] * P.qn[0] + gqn[1] * P.qn[1] + gqn[2] * P.qn[2] + gqn[3] * P.qn[3];
    for (int k = 0; k < 4; ++k) gq[k] += (gqn[k] - P.qn[k] * dotp) / qnorm;
  }
}

template <class R>
void project_bwd(const R* means, const R* log_scales, const R* quats, const R* opac, const R* sh, int64_t N,
                 const std::vector<OCam>& cams, const OConfig& cfg, const double* d_proj, const int64_t* gsel, int64_t n_sel,
                 double* gm, double* gls, double* gq, double* go, double* gsh) {
  const int64_t n = gsel ? n_sel : N;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) {
    const int64_t g = gsel ? gsel[i] : i;
    project_bwd_one<R>(means, log_scales, quats, opac, sh, N, g, cams, cfg, d_proj, gm + 3 * i, gls + 3 * i, gq + 4 * i,
                       go + i, gsh + 48 * i);
  }
}

// Untiled brute-force renderer: each pixel composites every visible record of
// its view whose tile rectangle contains the pixel's tile, in (depth, index)
// order. It does not use the key list or the tile ranges.
template <class R>
void render_bruteforce(const R* projected, const int16_t* rects, const uint32_t* counts, int64_t N,
                       const std::vector<OCam>& cams, const OConfig& cfg, R* image, R* final_T) {
  const TileLayout L = make_layout(cams, cfg);
  const int V = (int)cams.size();
  for (int v = 0; v < V; ++v) {
    std::vector<int64_t> order;
    for (int64_t g = 0; g < N; ++g)
      if (counts[(int64_t)v * N + g]) order.push_back((int64_t)v * N + g);
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      const float da = (float)projected[12 * a + 6], db = (float)projected[12 * b + 6];
      if (da != db) return da < db;
      return a < b;
    });
    const int Wv = cams[v].width, Hv = cams[v].height;
    for (int j = 0; j < Hv; ++j)
      for (int i = 0; i < Wv; ++i) {
        const int tx = i / cfg.tile_w, ty = j / cfg.tile_h;
        std::vector<uint32_t> lst;
        for (int64_t vg : order) {
          const int16_t* r = rects + 4 * vg;
          if (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) lst.push_back((uint32_t)vg);
        }
        R out[3], Tf;
        uint32_t last;
        composite_pixel<R>(projected, lst.data(), 0, (uint32_t)lst.size(), R(i) + R(0.5), R(j) + R(0.5), cfg, out, Tf, last,
                           nullptr, nullptr, nullptr);
        const int64_t p = L.pix_base[v] + (int64_t)j * Wv + i;
        for (int ch = 0; ch < 3; ++ch) image[3 * p + ch] = out[ch];
        final_T[p] = Tf;
      }
  }
}

}  // namespace

// ------------------------------------------------------------------------
// C entry points (ctypes). Suffix _f32 / _f64 selects the precision R.
// ------------------------------------------------------------------------
extern "C" {

float oracle_exp_cody_waite(float x) { return exp_cody_waite(x); }

void oracle_sh_basis(const double* dirs, int64_t n, double* out /*[n][16]*/) {
  const SHBasis& B = sh_basis();
  for (int64_t i = 0; i < n; ++i) {
    double p[16];
    SHBasis::poly(dirs + 3 * i, p);
    for (int k = 0; k < 16; ++k) out[16 * i + k] = B.c[k] * p[k];
  }
}

int64_t oracle_num_tiles(const int32_t* sizes, int32_t V, const OConfig* cfg) {
  int64_t n = 0;
  for (int v = 0; v < V; ++v)
    n += (int64_t)((sizes[2 * v] + cfg->tile_w - 1) / cfg->tile_w) * ((sizes[2 * v + 1] + cfg->tile_h - 1) / cfg->tile_h);
  return n;
}

#define ORACLE_INSTANTIATE(R, SUF)                                                                                         \
  void oracle_project_##SUF(const R* means, const R* log_scales, const R* quats, const R* opac, const R* sh, int64_t N,     \
                            const float* cams, const int32_t* sizes, int32_t V, const OConfig* cfg, R* projected,          \
                            int16_t* rects, uint32_t* counts) {                                                            \
    project_all<R>(means, log_scales, quats, opac, sh, N, load_cams(cams, sizes, V), *cfg, projected, rects, counts);      \
  }                                                                                                                        \
  int64_t oracle_bin_sort_##SUF(const R* projected, const int16_t* rects, const uint32_t* counts, int64_t N,               \
                                const float* cams, const int32_t* sizes, int32_t V, const OConfig* cfg, uint64_t* keys,    \
                                uint32_t* vals, int64_t capacity, uint32_t* ranges) {                                      \
    return bin_sort<R>(projected, rects, counts, N, load_cams(cams, sizes, V), *cfg, keys, vals, capacity, ranges);        \
  }                                                                                                                        \
  void oracle_raster_fwd_##SUF(const R* projected, const uint32_t* vals, const uint32_t* ranges, const float* cams,         \
                               const int32_t* sizes, int32_t V, const OConfig* cfg, const int64_t* tiles, int64_t n_sel,   \
                               R* image, R* final_T, uint32_t* last, uint8_t* marg_vg, uint8_t* marg_pix,                  \
                               uint64_t* hitsig, uint32_t* ncomp) {                                                        \
    raster_fwd<R>(projected, vals, ranges, load_cams(cams, sizes, V), *cfg, tiles, n_sel, image, final_T, last, marg_vg,    \
                  marg_pix, hitsig, ncomp);                                                                                \
  }                                                                                                                        \
  void oracle_raster_bwd_##SUF(const R* projected, const uint32_t* vals, const uint32_t* ranges, const float* cams,         \
                               const int32_t* sizes, int32_t V, const OConfig* cfg, const int64_t* tiles, int64_t n_sel,   \
                               const double* dL_dimage, double* d_proj) {                                                  \
    raster_bwd<R>(projected, vals, ranges, load_cams(cams, sizes, V), *cfg, tiles, n_sel, dL_dimage, d_proj);              \
  }                                                                                                                        \
  void oracle_project_bwd_##SUF(const R* means, const R* log_scales, const R* quats, const R* opac, const R* sh, int64_t N, \
                                const float* cams, const int32_t* sizes, int32_t V, const OConfig* cfg,                    \
                                const double* d_proj, const int64_t* gsel, int64_t n_sel, double* gm, double* gls,         \
                                double* gq, double* go, double* gsh) {                                                     \
    project_bwd<R>(means, log_scales, quats, opac, sh, N, load_cams(cams, sizes, V), *cfg, d_proj, gsel, n_sel, gm, gls,   \
                   gq, go, gsh);                                                                                           \
  }                                                                                                                        \
  void oracle_render_bruteforce_##SUF(const R* projected, const int16_t* rects, const uint32_t* counts, int64_t N,         \
                                      const float* cams, const int32_t* sizes, int32_t V, const OConfig* cfg, R* image,    \
                                      R* final_T) {                                                                        \
    render_bruteforce<R>(projected, rects, counts, N, load_cams(cams, sizes, V), *cfg, image, final_T);                    \
  }

ORACLE_INSTANTIATE(float, f32)
ORACLE_INSTANTIATE(double, f64)

// Loss on the rendered image: L = w1 * mean|r| + w2 * mean(r^2), r = image - target,
// means over all n values. Writes dL/dimage; returns L. (In double.)
double oracle_loss(const float* image, const float* target, int64_t n, double w1, double w2, double* dL_dimage) {
  double L = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double r = (double)image[i] - (double)target[i];
    L += w1 * std::fabs(r) + w2 * r * r;
    const double sgn = r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0);
    dL_dimage[i] = (w1 * sgn + 2.0 * w2 * r) / (double)n;
  }
  return L / (double)n;
}

// Adam (Kingma & Ba 2015, Algorithm 1) for step t >= 1, in double.
// Host threads the OpenMP build uses (1 in the serial build).
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void oracle_adam(double* param, const double* grad, double* m, double* v, int64_t n, double lr, double beta1, double beta2,
                 double eps, int32_t t) {
  const double bc1 = 1.0 - std::pow(beta1, t), bc2 = 1.0 - std::pow(beta2, t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
    v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
    const double mh = m[i] / bc1, vh = v[i] / bc2;
    param[i] -= lr * mh / (std::sqrt(vh) + eps);
  }
}

}  // extern "C"
