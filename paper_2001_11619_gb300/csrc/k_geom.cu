// Geometry, boundary data and evaluation kernels: trapezoid quadrature
// (Sec. 4 opening), the bordering columns H and Psi (Sec. 3.1, Eq.
// null-space), point-force boundary data, the interior velocity of
// Eq. (completed) and the FP64 operator A x of Eq. (backwardeq).
#include "kmath.cuh"

namespace skel {

__global__ void k_quadrature(const double *x, const double *y,
                             const double *dx, const double *dy,
                             const double *ddx, const double *ddy,
                             const double *dt, int64_t N, double *nx,
                             double *ny, double *w, double *kap) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  double sp = sqrt(dx[j] * dx[j] + dy[j] * dy[j]);
  double vx = dy[j] / sp, vy = -dx[j] / sp;  // outward from Omega
  nx[j] = vx;
  ny[j] = vy;
  w[j] = sp * dt[j];
  kap[j] = (ddx[j] * vx + ddy[j] * vy) / (sp * sp);
}

void launch_quadrature(const double *x, const double *y, const double *dx,
                       const double *dy, const double *ddx, const double *ddy,
                       const double *dt, int64_t N, double *nx, double *ny,
                       double *w, double *kap, cudaStream_t s) {
  int th = 256;
  int64_t nb = (N + th - 1) / th;
  k_quadrature<<<(unsigned)nb, th, 0, s>>>(x, y, dx, dy, ddx, ddy, dt, N, nx,
                                           ny, w, kap);
  note_launches(1);
}

// H column 3i+a at DOF (j, c): Stokeslet (a<2) or rotlet (a=2) at c_i.
__global__ void k_h_columns(DevGeom g, double *H, int64_t ld) {
  int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (d >= 2 * g.N) return;
  int64_t j = d >> 1;
  int c = (int)(d & 1);
  double rx = g.x[j] - g.centers[2 * i], ry = g.y[j] - g.centers[2 * i + 1];
  double s00, s01, s11;
  stokeslet(rx, ry, s00, s01, s11);
  double r2 = rx * rx + ry * ry;
  double rot = (c == 0 ? -ry : rx) / (4.0 * kPi * r2);
  H[d + ld * (3 * i + 0)] = c == 0 ? s00 : s01;
  H[d + ld * (3 * i + 1)] = c == 0 ? s01 : s11;
  H[d + ld * (3 * i + 2)] = rot;
}

void launch_h_columns(const DevGeom &g, double *H, int64_t ld,
                      cudaStream_t s) {
  if (g.p == 0) return;
  int th = 256;
  dim3 grid((unsigned)((2 * g.N + th - 1) / th), g.p);
  k_h_columns<<<grid, th, 0, s>>>(g, H, ld);
  note_launches(1);
}

// Psi column 3i+a at DOF (j,c): w_j psi_i^(a)(x_j)_c with psi^(1)=e1,
// psi^(2)=e2, psi^(3)=x^perp=(-y,x), zero off hole i.
__global__ void k_psi_columns(DevGeom g, double *P, int64_t ld) {
  int64_t d = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int i = blockIdx.y;
  if (d >= 2 * g.N) return;
  int64_t j = d >> 1;
  int c = (int)(d & 1);
  bool on = g.comp[j] == i + 1;
  double wj = g.w[j];
  P[d + ld * (3 * i + 0)] = (on && c == 0) ? wj : 0.0;
  P[d + ld * (3 * i + 1)] = (on && c == 1) ? wj : 0.0;
  P[d + ld * (3 * i + 2)] = on ? wj * (c == 0 ? -g.y[j] : g.x[j]) : 0.0;
}

void launch_psi_columns(const DevGeom &g, double *P, int64_t ld,
                        cudaStream_t s) {
  if (g.p == 0) return;
  int th = 256;
  dim3 grid((unsigned)((2 * g.N + th - 1) / th), g.p);
  k_psi_columns<<<grid, th, 0, s>>>(g, P, ld);
  note_launches(1);
}

__global__ void k_point_force_rhs(DevGeom g, int ns, const double *sxy,
                                  const double *sf, int holes_zero, double *f,
                                  int64_t ld) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  int64_t n2 = 2 * g.N;
  if (j < g.N) {
    double ux = 0.0, uy = 0.0;
    if (!(holes_zero && g.comp[j] != 0)) {
      for (int q = 0; q < ns; ++q) {
        const double *p = sxy + 2 * ((int64_t)r * ns + q);
        const double *F = sf + 2 * ((int64_t)r * ns + q);
        double s00, s01, s11;
        stokeslet(g.x[j] - p[0], g.y[j] - p[1], s00, s01, s11);
        ux += s00 * F[0] + s01 * F[1];
        uy += s01 * F[0] + s11 * F[1];
      }
    }
    f[2 * j + ld * r] = ux;
    f[2 * j + 1 + ld * r] = uy;
  }
  if (j < 3 * (int64_t)g.p) f[n2 + j + ld * r] = 0.0;
}

void launch_point_force_rhs(const DevGeom &g, int nrhs, int ns,
                            const double *sxy, const double *sf,
                            int holes_zero, double *f, int64_t ld,
                            cudaStream_t s) {
  int th = 256;
  int64_t n = g.N > 3 * g.p ? g.N : 3 * g.p;
  dim3 grid((unsigned)((n + th - 1) / th), nrhs);
  k_point_force_rhs<<<grid, th, 0, s>>>(g, ns, sxy, sf, holes_zero, f, ld);
  note_launches(1);
}

// u(t) = sum_j D(t, x_j) w_j mu_j + sum_i S_i alpha_i + R_i beta_i.
// One thread per (target, rhs); sources staged through shared memory.
__global__ void k_eval_velocity(DevGeom g, const double *sol, int64_t ld,
                                int nrhs, int64_t nt, const double *tx,
                                const double *ty, double *u) {
  __shared__ double sh[6][128];
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  double px = t < nt ? tx[t] : 0.0, py = t < nt ? ty[t] : 0.0;
  double ux = 0.0, uy = 0.0;
  const double *mu = sol + ld * r;
  for (int64_t base = 0; base < g.N; base += 128) {
    int64_t j = base + threadIdx.x;
    __syncthreads();
    if (threadIdx.x < 128) {
      bool ok = j < g.N;
      sh[0][threadIdx.x] = ok ? g.x[j] : 0.0;
      sh[1][threadIdx.x] = ok ? g.y[j] : 0.0;
      sh[2][threadIdx.x] = ok ? g.nx[j] : 0.0;
      sh[3][threadIdx.x] = ok ? g.ny[j] : 0.0;
      sh[4][threadIdx.x] = ok ? g.w[j] * mu[2 * j] : 0.0;
      sh[5][threadIdx.x] = ok ? g.w[j] * mu[2 * j + 1] : 0.0;
    }
    __syncthreads();
    int cnt = (int)((g.N - base) < 128 ? (g.N - base) : 128);
    if (t < nt) {
      for (int q = 0; q < cnt; ++q) {
        double d00, d01, d11;
        dl_block(px, py, sh[0][q], sh[1][q], sh[2][q], sh[3][q], 1.0, d00, d01,
                 d11);
        ux += d00 * sh[4][q] + d01 * sh[5][q];
        uy += d01 * sh[4][q] + d11 * sh[5][q];
      }
    }
  }
  if (t >= nt) return;
  const double *lam = mu + 2 * g.N;
  for (int i = 0; i < g.p; ++i) {
    double rx = px - g.centers[2 * i], ry = py - g.centers[2 * i + 1];
    double s00, s01, s11;
    stokeslet(rx, ry, s00, s01, s11);
    double r2 = rx * rx + ry * ry;
    double a0 = lam[3 * i], a1 = lam[3 * i + 1], b = lam[3 * i + 2];
    ux += s00 * a0 + s01 * a1 - ry / (4.0 * kPi * r2) * b;
    uy += s01 * a0 + s11 * a1 + rx / (4.0 * kPi * r2) * b;
  }
  u[2 * t + 2 * nt * r] = ux;
  u[2 * t + 1 + 2 * nt * r] = uy;
}

void launch_eval_velocity(const DevGeom &g, int nrhs, const double *sol,
                          int64_t ld, int64_t nt, const double *tx,
                          const double *ty, double *u, cudaStream_t s) {
  if (nt == 0) return;
  int th = 128;
  dim3 grid((unsigned)((nt + th - 1) / th), nrhs);
  k_eval_velocity<<<grid, th, 0, s>>>(g, sol, ld, nrhs, nt, tx, ty, u);
  note_launches(1);
}

// y = A x for the bordered matrix, one thread per (node, rhs), FP64,
// sources staged through shared memory.
__global__ void k_matvec(DevGeom g, const double *x, double *y, int64_t ld) {
  __shared__ double sh[6][128];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  const double *xr = x + ld * r;
  double *yr = y + ld * r;
  int64_t n2 = 2 * g.N;
  double px = i < g.N ? g.x[i] : 0.0, py = i < g.N ? g.y[i] : 0.0;
  double acc0 = 0.0, acc1 = 0.0, flux = 0.0;
  for (int64_t base = 0; base < g.N; base += 128) {
    int64_t j = base + threadIdx.x;
    __syncthreads();
    if (threadIdx.x < 128) {
      bool ok = j < g.N;
      sh[0][threadIdx.x] = ok ? g.x[j] : 0.0;
      sh[1][threadIdx.x] = ok ? g.y[j] : 0.0;
      sh[2][threadIdx.x] = ok ? g.nx[j] : 0.0;
      sh[3][threadIdx.x] = ok ? g.ny[j] : 0.0;
      sh[4][threadIdx.x] = ok ? g.w[j] * xr[2 * j] : 0.0;
      sh[5][threadIdx.x] = ok ? g.w[j] * xr[2 * j + 1] : 0.0;
    }
    __syncthreads();
    int cnt = (int)((g.N - base) < 128 ? (g.N - base) : 128);
    if (i < g.N) {
      for (int q = 0; q < cnt; ++q) {
        flux += sh[2][q] * sh[4][q] + sh[3][q] * sh[5][q];
        if (base + q == i) continue;
        double d00, d01, d11;
        dl_block(px, py, sh[0][q], sh[1][q], sh[2][q], sh[3][q], 1.0, d00,
                 d01, d11);
        acc0 += d00 * sh[4][q] + d01 * sh[5][q];
        acc1 += d01 * sh[4][q] + d11 * sh[5][q];
      }
    }
  }
  if (i < g.N) {
    double d00, d01, d11;
    dl_diag(g.nx[i], g.ny[i], g.kap[i], g.w[i], d00, d01, d11);
    double m0 = xr[2 * i], m1 = xr[2 * i + 1];
    acc0 += d00 * m0 + d01 * m1 - 0.5 * m0 + g.nx[i] * flux;
    acc1 += d01 * m0 + d11 * m1 - 0.5 * m1 + g.ny[i] * flux;
    const double *lam = xr + n2;
    for (int h = 0; h < g.p; ++h) {
      double rx = px - g.centers[2 * h], ry = py - g.centers[2 * h + 1];
      double s00, s01, s11;
      stokeslet(rx, ry, s00, s01, s11);
      double r2 = rx * rx + ry * ry;
      double a0 = lam[3 * h], a1 = lam[3 * h + 1], b = lam[3 * h + 2];
      acc0 += s00 * a0 + s01 * a1 - ry / (4.0 * kPi * r2) * b;
      acc1 += s01 * a0 + s11 * a1 + rx / (4.0 * kPi * r2) * b;
    }
    yr[2 * i] = acc0;
    yr[2 * i + 1] = acc1;
  }
}

// Psi^T mu - lambda rows: one block per (hole, rhs), deterministic tree
// reduction over the hole's nodes.
__global__ void k_matvec_psi(DevGeom g, const double *x, double *y,
                             int64_t ld) {
  __shared__ double red[3][256];
  int h = blockIdx.x, r = blockIdx.y;
  const double *xr = x + ld * r;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t j = threadIdx.x; j < g.N; j += blockDim.x) {
    if (g.comp[j] != h + 1) continue;
    double m0 = xr[2 * j], m1 = xr[2 * j + 1], wj = g.w[j];
    a0 += wj * m0;
    a1 += wj * m1;
    a2 += wj * (-g.y[j] * m0 + g.x[j] * m1);
  }
  red[0][threadIdx.x] = a0;
  red[1][threadIdx.x] = a1;
  red[2][threadIdx.x] = a2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 3) {
    int64_t row = 2 * g.N + 3 * h + threadIdx.x;
    y[row + ld * r] = red[threadIdx.x][0] - xr[row];
  }
}

void launch_matvec(const DevGeom &g, int nrhs, const double *x, double *y,
                   int64_t ld, cudaStream_t s) {
  int th = 128;
  dim3 grid((unsigned)((g.N + th - 1) / th), nrhs);
  k_matvec<<<grid, th, 0, s>>>(g, x, y, ld);
  note_launches(1);
  if (g.p) k_matvec_psi<<<dim3(g.p, nrhs), 256, 0, s>>>(g, x, y, ld);
  note_launches(1);
}

}  // namespace skel
