// Device-side kernel functions of the 2-D Stokes boundary integral
// equation (Sec. 3.1), in FP64 and in FP32.
//
// FP32 entries (the mixed-precision form) keep the coordinate differences
// accurate: every node position is also stored as a pair of floats
// x = xh + xl, and r = (xh_t - xh_s) + (xl_t - xl_s) is formed in float, so
// the difference of two nearby nodes keeps ~1e-7 relative accuracy instead
// of losing digits to cancellation.  The rest of the entry is plain float.
#pragma once

#include "skel_internal.h"

namespace skel {

// ---------------------------------------------------------------------------
// FP64

// Stresslet double layer of Eq. (stokesbie) times the source weight:
//   D(t,s) w_s = (1/pi) ((t-s).n_s) (t-s)(t-s)^T / |t-s|^4 w_s
// The 2x2 block is symmetric: returns (d00, d01, d11).
__device__ __forceinline__ void dl_block(double tx, double ty, double sx,
                                         double sy, double snx, double sny,
                                         double sw, double &d00, double &d01,
                                         double &d11) {
  double rx = tx - sx, ry = ty - sy;
  double r2 = rx * rx + ry * ry;
  double rn = rx * snx + ry * sny;
  double c = rn / (kPi * r2 * r2) * sw;
  d00 = c * rx * rx;
  d01 = c * rx * ry;
  d11 = c * ry * ry;
}

// Smooth limit of the same block as s -> t along the curve:
//   (gamma''.n)/(2 pi |gamma'|^2) t t^T w,   t = (-n_y, n_x)
__device__ __forceinline__ void dl_diag(double nx, double ny, double kap,
                                        double w, double &d00, double &d01,
                                        double &d11) {
  double c = kap / (2.0 * kPi) * w;
  double tx = -ny, ty = nx;
  d00 = c * tx * tx;
  d01 = c * tx * ty;
  d11 = c * ty * ty;
}

// Stokeslet of Sec. 3.1: (1/4pi)(ln(1/|r|) I + r r^T/|r|^2), r = x - c.
__device__ __forceinline__ void stokeslet(double rx, double ry, double &s00,
                                          double &s01, double &s11) {
  double r2 = rx * rx + ry * ry;
  double lg = -0.5 * log(r2);
  double inv = 1.0 / r2;
  const double f = 1.0 / (4.0 * kPi);
  s00 = (lg + rx * rx * inv) * f;
  s01 = (rx * ry * inv) * f;
  s11 = (lg + ry * ry * inv) * f;
}

// 1/a for a normal positive double: the approximate FP64 reciprocal of
// PTX (rcp.approx.ftz.f64) refined by one cubic Newton-Raphson step,
// y (1 + e + e^2) with e = 1 - a y (the truncated series of 1/(1 - e)),
// whose own error is O(e^3).  Within an ulp or two of the correctly rounded
// reciprocal at three FMAs, where the double-layer sums spend most of their
// FP64 issue slots.
__device__ __forceinline__ double recip_nr3(double a) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(a));
  const double e = fma(-a, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

template <class T>
__device__ __forceinline__ T pick(T d00, T d01, T d11, int a, int b) {
  return (a == b) ? (a == 0 ? d00 : d11) : d01;
}

// Entry of the discretised double layer K for DOFs (2i+a, 2j+b).
__device__ __forceinline__ double k_entry(const DevGeom &g, int di, int dj) {
  int i = di >> 1, a = di & 1, j = dj >> 1, b = dj & 1;
  double d00, d01, d11;
  if (i == j)
    dl_diag(g.nx[j], g.ny[j], g.kap[j], g.w[j], d00, d01, d11);
  else
    dl_block(g.x[i], g.y[i], g.x[j], g.y[j], g.nx[j], g.ny[j], g.w[j], d00,
             d01, d11);
  return pick(d00, d01, d11, a, b);
}

// Entry of -1/2 I + D + N (Eq. completedback) with the rank-one completion
// (N mu)(x) = n(x) int n(y).mu(y) dy of Eq. (null-spaceop).
__device__ __forceinline__ double a11_entry(const DevGeom &g, int di, int dj) {
  int i = di >> 1, a = di & 1, j = dj >> 1, b = dj & 1;
  double v = k_entry(g, di, dj);
  double ni = a ? g.ny[i] : g.nx[i];
  double nj = b ? g.ny[j] : g.nx[j];
  v += ni * nj * g.w[j];
  if (di == dj) v -= 0.5;
  return v;
}

// ---------------------------------------------------------------------------
// FP32 (mixed-precision form)

constexpr float kPif = 3.14159265358979323846f;

__device__ __forceinline__ void dl_block_f(float rx, float ry, float snx,
                                           float sny, float sw, float &d00,
                                           float &d01, float &d11) {
  const float r2 = rx * rx + ry * ry;
  const float rn = rx * snx + ry * sny;
  const float inv = 1.0f / r2;
  const float c = rn * inv * inv * (sw * (1.0f / kPif));
  d00 = c * rx * rx;
  d01 = c * rx * ry;
  d11 = c * ry * ry;
}

__device__ __forceinline__ void stokeslet_f(float rx, float ry, float &s00,
                                            float &s01, float &s11) {
  const float r2 = rx * rx + ry * ry;
  const float lg = -0.5f * logf(r2);
  const float inv = 1.0f / r2;
  const float f = 1.0f / (4.0f * kPif);
  s00 = (lg + rx * rx * inv) * f;
  s01 = (rx * ry * inv) * f;
  s11 = (lg + ry * ry * inv) * f;
}

// r = x_i - x_j from the float pairs
__device__ __forceinline__ void diff_f(const DevGeom &g, int i, int j,
                                       float &rx, float &ry) {
  rx = (g.xh[i] - g.xh[j]) + (g.xl[i] - g.xl[j]);
  ry = (g.yh[i] - g.yh[j]) + (g.yl[i] - g.yl[j]);
}

__device__ __forceinline__ float k_entry_f(const DevGeom &g, int di, int dj) {
  const int i = di >> 1, a = di & 1, j = dj >> 1, b = dj & 1;
  float d00, d01, d11;
  if (i == j) {
    const float c = g.kapf[j] * (1.0f / (2.0f * kPif)) * g.wf[j];
    const float tx = -g.nyf[j], ty = g.nxf[j];
    d00 = c * tx * tx;
    d01 = c * tx * ty;
    d11 = c * ty * ty;
  } else {
    float rx, ry;
    diff_f(g, i, j, rx, ry);
    dl_block_f(rx, ry, g.nxf[j], g.nyf[j], g.wf[j], d00, d01, d11);
  }
  return pick(d00, d01, d11, a, b);
}

__device__ __forceinline__ float a11_entry_f(const DevGeom &g, int di,
                                             int dj) {
  const int i = di >> 1, a = di & 1, j = dj >> 1, b = dj & 1;
  float v = k_entry_f(g, di, dj);
  const float ni = a ? g.nyf[i] : g.nxf[i];
  const float nj = b ? g.nyf[j] : g.nxf[j];
  v += ni * nj * g.wf[j];
  if (di == dj) v -= 0.5f;
  return v;
}

// ---------------------------------------------------------------------------
// Laplace Neumann form (the paper's Sec. 4.4.1 experiment): one DOF per
// node.  D[i, j] w_j with D mu(x) = -(1/2pi) int (x - y).n(x)/|x - y|^2
// mu(y) dy, the normal derivative of the single layer at the target; its
// diagonal is the smooth limit (gamma''.n)/(4 pi |gamma'|^2).  The operator
// is 1/2 I + D + N with N = 1 w^T (rank one; it completes the interior
// Neumann null space), always in FP64.

__device__ __forceinline__ double lap_d_entry(const DevGeom &g, int i, int j) {
  if (i == j) return g.kap[i] * (0.25 / kPi) * g.w[i];
  const double rx = g.x[i] - g.x[j], ry = g.y[i] - g.y[j];
  const double rn = rx * g.nx[i] + ry * g.ny[i];
  return -rn / (2.0 * kPi * (rx * rx + ry * ry)) * g.w[j];
}

__device__ __forceinline__ double lap_a_entry(const DevGeom &g, int i, int j) {
  return lap_d_entry(g, i, j) + g.w[j] + (i == j ? 0.5 : 0.0);
}

// precision dispatch for the assembly kernels (the Laplace form is FP64
// only; its float instantiation exists for uniformity and is not used)
template <class Real>
__device__ __forceinline__ Real k_entry_r(const DevGeom &g, int di, int dj);
template <>
__device__ __forceinline__ double k_entry_r<double>(const DevGeom &g, int di,
                                                    int dj) {
  return g.lap ? lap_d_entry(g, di, dj) : k_entry(g, di, dj);
}
template <>
__device__ __forceinline__ float k_entry_r<float>(const DevGeom &g, int di,
                                                  int dj) {
  return g.lap ? (float)lap_d_entry(g, di, dj) : k_entry_f(g, di, dj);
}
template <class Real>
__device__ __forceinline__ Real a11_entry_r(const DevGeom &g, int di, int dj);
template <>
__device__ __forceinline__ double a11_entry_r<double>(const DevGeom &g,
                                                      int di, int dj) {
  return g.lap ? lap_a_entry(g, di, dj) : a11_entry(g, di, dj);
}
template <>
__device__ __forceinline__ float a11_entry_r<float>(const DevGeom &g, int di,
                                                    int dj) {
  return g.lap ? (float)lap_a_entry(g, di, dj) : a11_entry_f(g, di, dj);
}

}  // namespace skel
