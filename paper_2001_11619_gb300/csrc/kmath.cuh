// Device-side kernel functions of the 2-D Stokes boundary integral
// equation (Sec. 3.1).  All in IEEE double.
#pragma once

#include "skel_internal.h"

namespace skel {

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

__device__ __forceinline__ double pick(double d00, double d01, double d11,
                                       int a, int b) {
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

}  // namespace skel
