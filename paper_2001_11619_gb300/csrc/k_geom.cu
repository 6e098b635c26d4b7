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
                             double *ny, double *w, double *kap, float *f32) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  double sp = sqrt(dx[j] * dx[j] + dy[j] * dy[j]);
  double vx = dy[j] / sp, vy = -dx[j] / sp;  // outward from Omega
  nx[j] = vx;
  ny[j] = vy;
  w[j] = sp * dt[j];
  kap[j] = (ddx[j] * vx + ddy[j] * vy) / (sp * sp);
  const float xh = (float)x[j], yh = (float)y[j];
  f32[j] = xh;
  f32[N + j] = (float)(x[j] - (double)xh);
  f32[2 * N + j] = yh;
  f32[3 * N + j] = (float)(y[j] - (double)yh);
  f32[4 * N + j] = (float)vx;
  f32[5 * N + j] = (float)vy;
  f32[6 * N + j] = (float)w[j];
  f32[7 * N + j] = (float)kap[j];
}

void launch_quadrature(const double *x, const double *y, const double *dx,
                       const double *dy, const double *ddx, const double *ddy,
                       const double *dt, int64_t N, double *nx, double *ny,
                       double *w, double *kap, float *f32, cudaStream_t s) {
  int th = 256;
  int64_t nb = (N + th - 1) / th;
  k_quadrature<<<(unsigned)nb, th, 0, s>>>(x, y, dx, dy, ddx, ddy, dt, N, nx,
                                           ny, w, kap, f32);
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

// ---------------------------------------------------------------------------
// Double-layer sums over all nodes, sum_j D(t, x_j) w_j mu_j (Eq. stokesbie),
// for interior targets (the velocity of Eq. completed) or for the nodes
// themselves (the operator apply, j = t excluded).  Sources are split in
// chunks over the grid's z dimension; each CTA writes its chunk's partial
// sums and a second kernel adds the chunks in a fixed order, so results do
// not depend on scheduling.  Per pair: r = t - x_j,
//   D(t,x_j) w_j mu_j = (1/pi) (r.n_j) (r.(w_j mu_j)) r / |r|^4.

constexpr int kDlThreads = 128;
constexpr int kDlStage = 256;

// Source chunks for the pair-sum kernels.  Their grids are units x nch
// CTAs of (nearly) equal work, so the time is that of the SM with the most
// CTAs: with T CTAs on 152 SMs it carries ceil(T / 152), against T / 152
// on average (768 CTAs: 6 against 5.05, 16 % of the machine idle at the
// end).  Takes the fewest chunks (at least min_per_sm CTAs per SM where
// possible, at most maxc) whose quantisation loss is within 3 %, else the
// best one below 64 CTAs per SM.  A larger maxc never gives fewer chunks.
int balanced_chunks(int64_t units, int64_t maxc, int min_per_sm) {
  const int64_t sms = 152;
  if (units < 1) units = 1;
  if (maxc < 1) maxc = 1;
  int64_t lo = (min_per_sm * sms + units - 1) / units;
  lo = lo < 1 ? 1 : (lo > maxc ? maxc : lo);
  int64_t hi = (64 * sms + units - 1) / units;
  hi = hi < lo ? lo : (hi > maxc ? maxc : hi);
  int64_t best = lo;
  double bq = 1e300;
  for (int64_t c = lo; c <= hi; ++c) {
    const int64_t T = units * c;
    const double q = (double)((T + sms - 1) / sms * sms) / (double)T;
    if (q <= 1.03) return (int)c;
    if (q < bq) {
      bq = q;
      best = c;
    }
  }
  return (int)best;
}

int dl_chunks(int64_t nt, int nrhs, int64_t N) {
  const int64_t tb = (nt + kDlThreads - 1) / kDlThreads;
  return balanced_chunks(tb * nrhs, (N + kDlStage - 1) / kDlStage, 4);
}

// Symmetric pair sums of the double layer on the nodes (the FP64 operator).
// The product of a pair, (r.n_j)(r.m_j) r / |r|^4 with m_j = w_j mu_j, is
// written as the quadratic form a_j rx^2 + b_j rx ry + c_j ry^2 (a = nx mx,
// b = nx my + ny mx, c = ny my, formed once per source) over |r|^4.  The two
// directions of a pair, j -> i and i -> j, share r = x_i - x_j, its squares,
// |r|^2 and the reciprocal: 23 FP64 operations give both products, against
// 17 for one in k_dl_partial.  The nodes are cut into R ranges of S points
// (S a multiple of kSymB).  CTA (A, B), A <= B, takes the pairs with i in
// range A and j in range B (i < j when A == B); its i sums go to slot B + 1
// and its j sums to slot A of the partial array.  A point of range X thus
// receives slots 0..X from the j side and X+1..R from the i side: every
// one of the R + 1 slots once, summed in slot order (deterministic).
constexpr int kSymB = 128;      // points per block (4 warps x 32)
constexpr int kSymMaxS = 4096;  // largest range (its j sums sit in shared)

void sym_ranges(int64_t N, int &S, int &R) {
  // about 128 ranges (8256 CTAs per column): finer than 64 ranges, whose
  // last CTAs left SMs idle at the end (22.8 against 21.6 ms at 32768 nodes)
  int64_t s = (N + 127) / 128;
  s = (s + kSymB - 1) / kSymB * kSymB;
  s = s < kSymB ? kSymB : (s > kSymMaxS ? kSymMaxS : s);
  S = (int)s;
  R = (int)((N + s - 1) / s);
}

size_t dl_scratch(int64_t nt, int nrhs, int64_t N) {
  size_t a = (size_t)dl_chunks(nt, nrhs, N) * nrhs * nt * 2;
  if (nt == N) {
    int S, R;
    sym_ranges(N, S, R);
    const size_t b = (size_t)(R + 1) * nrhs * N * 2;
    a = a > b ? a : b;
  }
  return a + (size_t)nrhs + 8;
}

__global__ void __launch_bounds__(kDlThreads)
k_dl_partial(DevGeom g, const double *sol, int64_t ld, int64_t nt,
             const double *tx, const double *ty, int self, int nchunk,
             double *partial) {
  __shared__ double sh[6][kDlStage];
  const int64_t t = blockIdx.x * (int64_t)kDlThreads + threadIdx.x;
  const int r = blockIdx.y, c = blockIdx.z;
  const double *mu = sol + ld * r;
  const int64_t per = (g.N + nchunk - 1) / nchunk;
  const int64_t j0 = c * per, j1 = j0 + per < g.N ? j0 + per : g.N;
  const bool on = t < nt;
  const double px = on ? (self ? g.x[t] : tx[t]) : 0.0;
  const double py = on ? (self ? g.y[t] : ty[t]) : 0.0;
  double a0 = 0.0, a1 = 0.0;
  for (int64_t base = j0; base < j1; base += kDlStage) {
    __syncthreads();
    for (int q = threadIdx.x; q < kDlStage; q += kDlThreads) {
      const int64_t j = base + q;
      const bool ok = j < j1;
      const double w = ok ? g.w[j] : 0.0;
      sh[0][q] = ok ? g.x[j] : 0.0;
      sh[1][q] = ok ? g.y[j] : 0.0;
      sh[2][q] = ok ? g.nx[j] : 0.0;
      sh[3][q] = ok ? g.ny[j] : 0.0;
      sh[4][q] = ok ? w * mu[2 * j] : 0.0;
      sh[5][q] = ok ? w * mu[2 * j + 1] : 0.0;
    }
    __syncthreads();
    const int cnt = (int)(j1 - base < kDlStage ? j1 - base : kDlStage);
    for (int q = 0; q < cnt; ++q) {
      const double rx = px - sh[0][q], ry = py - sh[1][q];
      const bool skip = self && (base + q == t);
      const double r2 = skip ? 1.0 : rx * rx + ry * ry;
      const double inv = recip_nr3(r2);
      const double rn = rx * sh[2][q] + ry * sh[3][q];
      const double tm = rx * sh[4][q] + ry * sh[5][q];
      const double s = skip ? 0.0 : rn * tm * inv * inv;
      a0 += s * rx;
      a1 += s * ry;
    }
  }
  if (!on) return;
  double *out = partial + (((int64_t)c * gridDim.y + r) * nt + t) * 2;
  out[0] = a0 / kPi;
  out[1] = a1 / kPi;
}

// Within a CTA, warp w holds targets i = 32 w + lane of the current block
// of range A in registers and takes the j-blocks of range B 32 sources at a
// time, the four warps on four different chunks per round.  At step t lane
// l takes source (l + t) mod 32 of the chunk; the source's running sum
// moves one lane down after each step (shuffle), so no two lanes touch one
// source at once, and after the chunk it is added to the range's j sums in
// shared memory.  In the diagonal chunk of a diagonal block the steps
// t = 1..16 (the second half of t = 16 dropped) give each pair once.
__global__ void __launch_bounds__(kSymB)
k_dl_sym(DevGeom g, const double *sol, int64_t ld, int S, int R,
         double *part) {
  extern __shared__ double sm[];
  double *jd = sm;                // sources of one block: [5][kSymB]
  double *jsum = sm + 5 * kSymB;  // j sums of range B: [S][2]
  int x = blockIdx.x, A = 0;
  while (x >= R - A) {
    x -= R - A;
    ++A;
  }
  const int B = A + x;
  const int r = blockIdx.y;
  const int64_t N = g.N;
  const double *mu = sol + ld * r;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a0 = (int64_t)A * S, b0 = (int64_t)B * S;
  const int la = (int)(N - a0 < S ? N - a0 : S);
  const int lb = (int)(N - b0 < S ? N - b0 : S);
  const int nbi = (la + kSymB - 1) / kSymB, nbj = (lb + kSymB - 1) / kSymB;
  for (int k = threadIdx.x; k < 2 * S; k += kSymB) jsum[k] = 0.0;
  for (int ib = 0; ib < nbi; ++ib) {
    const int64_t i = a0 + (int64_t)ib * kSymB + threadIdx.x;
    const bool oki = i < a0 + la;
    double px = 0.0, py = 0.0, pa = 0.0, pb = 0.0, pc = 0.0;
    if (oki) {
      const double mx = g.w[i] * mu[2 * i], my = g.w[i] * mu[2 * i + 1];
      px = g.x[i];
      py = g.y[i];
      pa = g.nx[i] * mx;
      pb = g.nx[i] * my + g.ny[i] * mx;
      pc = g.ny[i] * my;
    }
    double ax = 0.0, ay = 0.0;
    for (int jb = (A == B ? ib : 0); jb < nbj; ++jb) {
      const int64_t jbase = b0 + (int64_t)jb * kSymB;
      __syncthreads();  // the previous block's sources are consumed
      {
        const int64_t j = jbase + threadIdx.x;
        double sx = 0.0, sy = 0.0, sa = 0.0, sb = 0.0, sc = 0.0;
        if (j < b0 + lb) {
          const double mx = g.w[j] * mu[2 * j], my = g.w[j] * mu[2 * j + 1];
          sx = g.x[j];
          sy = g.y[j];
          sa = g.nx[j] * mx;
          sb = g.nx[j] * my + g.ny[j] * mx;
          sc = g.ny[j] * my;
        }
        jd[threadIdx.x] = sx;
        jd[kSymB + threadIdx.x] = sy;
        jd[2 * kSymB + threadIdx.x] = sa;
        jd[3 * kSymB + threadIdx.x] = sb;
        jd[4 * kSymB + threadIdx.x] = sc;
      }
      __syncthreads();
      const bool dblk = A == B && jb == ib;
      for (int round = 0; round < 4; ++round) {
        const int c = (round + w) & 3;
        if (round) __syncthreads();  // one warp per chunk of j sums
        if (dblk && c < w) continue;
        const bool half = dblk && c == w;
        const int t0 = half ? 1 : 0, t1 = half ? 17 : 32;
        const int64_t cbase = jbase + c * 32;
        const double *d = jd + c * 32;
        double jx = 0.0, jy = 0.0;
        for (int t = t0; t < t1; ++t) {
          const int q = (lane + t) & 31;
          const double rx = px - d[q], ry = py - d[kSymB + q];
          const double xx = rx * rx, yy = ry * ry, xy = rx * ry;
          const double inv = recip_nr3(xx + yy);
          const double inv2 = inv * inv;
          const double sf =
              fma(d[2 * kSymB + q], xx,
                  fma(d[3 * kSymB + q], xy, d[4 * kSymB + q] * yy)) *
              inv2;
          const double sr = fma(pa, xx, fma(pb, xy, pc * yy)) * inv2;
          const bool act = oki && cbase + q < b0 + lb &&
                           !(half && t == 16 && lane >= 16);
          const double f = act ? sf : 0.0, b = act ? sr : 0.0;
          ax += f * rx;
          ay += f * ry;
          jx -= b * rx;
          jy -= b * ry;
          jx = __shfl_sync(0xffffffffu, jx, (lane + 1) & 31);
          jy = __shfl_sync(0xffffffffu, jy, (lane + 1) & 31);
        }
        const int k = jb * kSymB + c * 32 + ((lane + t1) & 31);
        jsum[2 * k] += jx;
        jsum[2 * k + 1] += jy;
      }
    }
    if (oki) {
      double *o = part + (((int64_t)(B + 1) * gridDim.y + r) * N + i) * 2;
      o[0] = ax / kPi;
      o[1] = ay / kPi;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < lb; k += kSymB) {
    double *o = part + (((int64_t)A * gridDim.y + r) * N + b0 + k) * 2;
    o[0] = jsum[2 * k] / kPi;
    o[1] = jsum[2 * k + 1] / kPi;
  }
}

// flux[r] = sum_j n_j . (w_j mu_j), the integral in (N mu) (Eq. null-spaceop)
__global__ void k_flux(DevGeom g, const double *x, int64_t ld, double *flux) {
  __shared__ double red[32];
  const double *xr = x + ld * blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < g.N; j += blockDim.x)
    s += g.w[j] * (g.nx[j] * xr[2 * j] + g.ny[j] * xr[2 * j + 1]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    flux[blockIdx.x] = t;
  }
}

// Stokeslet and rotlet contributions at (px, py): sum_i S_i alpha_i + R_i beta_i
__device__ __forceinline__ void add_point_sources(const DevGeom &g,
                                                  const double *lam, double px,
                                                  double py, double &u0,
                                                  double &u1) {
  for (int i = 0; i < g.p; ++i) {
    const double rx = px - g.centers[2 * i], ry = py - g.centers[2 * i + 1];
    double s00, s01, s11;
    stokeslet(rx, ry, s00, s01, s11);
    const double r2 = rx * rx + ry * ry;
    const double a0 = lam[3 * i], a1 = lam[3 * i + 1], b = lam[3 * i + 2];
    u0 += s00 * a0 + s01 * a1 - ry / (4.0 * kPi * r2) * b;
    u1 += s01 * a0 + s11 * a1 + rx / (4.0 * kPi * r2) * b;
  }
}

__global__ void k_eval_finish(DevGeom g, const double *sol, int64_t ld,
                              int64_t nt, const double *tx, const double *ty,
                              int nchunk, const double *partial, double *u) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (t >= nt) return;
  double u0 = 0.0, u1 = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double *p = partial + (((int64_t)c * gridDim.y + r) * nt + t) * 2;
    u0 += p[0];
    u1 += p[1];
  }
  add_point_sources(g, sol + ld * r + 2 * g.N, tx[t], ty[t], u0, u1);
  u[2 * t + 2 * nt * r] = u0;
  u[2 * t + 1 + 2 * nt * r] = u1;
}

void launch_eval_velocity(const DevGeom &g, int nrhs, const double *sol,
                          int64_t ld, int64_t nt, const double *tx,
                          const double *ty, double *u, double *scratch,
                          cudaStream_t s) {
  if (nt == 0 || nrhs == 0) return;
  const int nch = dl_chunks(nt, nrhs, g.N);
  dim3 grid((unsigned)((nt + kDlThreads - 1) / kDlThreads), nrhs, nch);
  k_dl_partial<<<grid, kDlThreads, 0, s>>>(g, sol, ld, nt, tx, ty, 0, nch,
                                           scratch);
  note_launches(1);
  dim3 g2((unsigned)((nt + 127) / 128), nrhs);
  k_eval_finish<<<g2, 128, 0, s>>>(g, sol, ld, nt, tx, ty, nch, scratch, u);
  note_launches(1);
}

// The same two kernels with the partial sums in caller-provided scratch of
// cap doubles: the source-chunk count is lowered until the partials
// (nchunk x nrhs x nt x 2 doubles) fit.  Returns false, launching nothing,
// when even a single chunk does not fit.
bool launch_eval_velocity_capped(const DevGeom &g, int nrhs, const double *sol,
                                 int64_t ld, int64_t nt, const double *tx,
                                 const double *ty, double *u, double *scratch,
                                 int64_t cap, cudaStream_t s) {
  if (nt == 0 || nrhs == 0) return true;
  const int64_t per_chunk = (int64_t)nrhs * nt * 2;
  if (per_chunk > cap) return false;
  int nch = dl_chunks(nt, nrhs, g.N);
  if ((int64_t)nch * per_chunk > cap) nch = (int)(cap / per_chunk);
  dim3 grid((unsigned)((nt + kDlThreads - 1) / kDlThreads), nrhs, nch);
  k_dl_partial<<<grid, kDlThreads, 0, s>>>(g, sol, ld, nt, tx, ty, 0, nch,
                                           scratch);
  note_launches(1);
  dim3 g2((unsigned)((nt + 127) / 128), nrhs);
  k_eval_finish<<<g2, 128, 0, s>>>(g, sol, ld, nt, tx, ty, nch, scratch, u);
  note_launches(1);
  return true;
}

// y = A x for the bordered matrix: double layer (above) + smooth diagonal
// limit - x/2 + n (flux) + Stokeslet/rotlet columns, then the Psi^T rows.
__global__ void k_matvec_finish(DevGeom g, const double *x, double *y,
                                int64_t ld, int nchunk, const double *partial,
                                const double *flux) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (i >= g.N) return;
  const double *xr = x + ld * r;
  double u0 = 0.0, u1 = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double *p = partial + (((int64_t)c * gridDim.y + r) * g.N + i) * 2;
    u0 += p[0];
    u1 += p[1];
  }
  double d00, d01, d11;
  dl_diag(g.nx[i], g.ny[i], g.kap[i], g.w[i], d00, d01, d11);
  const double m0 = xr[2 * i], m1 = xr[2 * i + 1];
  u0 += d00 * m0 + d01 * m1 - 0.5 * m0 + g.nx[i] * flux[r];
  u1 += d01 * m0 + d11 * m1 - 0.5 * m1 + g.ny[i] * flux[r];
  add_point_sources(g, xr + 2 * g.N, g.x[i], g.y[i], u0, u1);
  y[2 * i + ld * r] = u0;
  y[2 * i + 1 + ld * r] = u1;
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

// ---------------------------------------------------------------------------
// Transposed operator A^T z for A = [[-1/2 I + K + N, H], [Psi^T, -I]]:
//   (A^T z)_mu   = -z/2 + K^T z_mu + w n (sum_i n_i . z_i) + Psi z_lambda
//   (A^T z)_lam  = H^T z_mu - z_lambda
// K_ij = D(x_i, x_j) w_j is symmetric per 2x2 block, so
//   (K^T z)_j = (w_j/pi) sum_{i != j} ((x_i-x_j).n_j) ((x_i-x_j).z_i)
//               (x_i - x_j) / |x_i - x_j|^4  +  K_jj z_j.

// The transposed double-layer sums on the nodes, symmetric as k_dl_sym:
// the output of node t is (w_t / pi) sum_i (r.n_t)(r.z_i) r / |r|^4 with
// r = x_i - x_t.  For a pair (i, j), r = x_i - x_j, node j gets
// (r.n_j)(r.z_i) r / |r|^4 and node i gets -(r.n_i)(r.z_j) r / |r|^4; the
// two share r, |r|^2 and its reciprocal (25 FP64 operations per pair
// against 34).  The partials carry the factor w_t / pi of their node.
__global__ void __launch_bounds__(kSymB)
k_dlT_sym(DevGeom g, const double *z, int64_t ld, int S, int R, double *part) {
  extern __shared__ double sm[];
  double *jd = sm;                // partners of one block: [6][kSymB]
  double *jsum = sm + 6 * kSymB;  // their sums over range B: [S][2]
  int x = blockIdx.x, A = 0;
  while (x >= R - A) {
    x -= R - A;
    ++A;
  }
  const int B = A + x;
  const int r = blockIdx.y;
  const int64_t N = g.N;
  const double *zr = z + ld * r;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a0 = (int64_t)A * S, b0 = (int64_t)B * S;
  const int la = (int)(N - a0 < S ? N - a0 : S);
  const int lb = (int)(N - b0 < S ? N - b0 : S);
  const int nbi = (la + kSymB - 1) / kSymB, nbj = (lb + kSymB - 1) / kSymB;
  for (int k = threadIdx.x; k < 2 * S; k += kSymB) jsum[k] = 0.0;
  for (int ib = 0; ib < nbi; ++ib) {
    const int64_t i = a0 + (int64_t)ib * kSymB + threadIdx.x;
    const bool oki = i < a0 + la;
    double px = 0, py = 0, nix = 0, niy = 0, zix = 0, ziy = 0;
    if (oki) {
      px = g.x[i];
      py = g.y[i];
      nix = g.nx[i];
      niy = g.ny[i];
      zix = zr[2 * i];
      ziy = zr[2 * i + 1];
    }
    double ax = 0.0, ay = 0.0;
    for (int jb = (A == B ? ib : 0); jb < nbj; ++jb) {
      const int64_t jbase = b0 + (int64_t)jb * kSymB;
      __syncthreads();  // the previous block's partners are consumed
      {
        const int64_t j = jbase + threadIdx.x;
        const bool ok = j < b0 + lb;
        jd[threadIdx.x] = ok ? g.x[j] : 0.0;
        jd[kSymB + threadIdx.x] = ok ? g.y[j] : 0.0;
        jd[2 * kSymB + threadIdx.x] = ok ? g.nx[j] : 0.0;
        jd[3 * kSymB + threadIdx.x] = ok ? g.ny[j] : 0.0;
        jd[4 * kSymB + threadIdx.x] = ok ? zr[2 * j] : 0.0;
        jd[5 * kSymB + threadIdx.x] = ok ? zr[2 * j + 1] : 0.0;
      }
      __syncthreads();
      const bool dblk = A == B && jb == ib;
      for (int round = 0; round < 4; ++round) {
        const int c = (round + w) & 3;
        if (round) __syncthreads();  // one warp per chunk of partner sums
        if (dblk && c < w) continue;
        const bool half = dblk && c == w;
        const int t0 = half ? 1 : 0, t1 = half ? 17 : 32;
        const int64_t cbase = jbase + c * 32;
        const double *d = jd + c * 32;
        double jx = 0.0, jy = 0.0;
        for (int t = t0; t < t1; ++t) {
          const int q = (lane + t) & 31;
          const double rx = px - d[q], ry = py - d[kSymB + q];
          const double inv = recip_nr3(rx * rx + ry * ry);
          const double inv2 = inv * inv;
          const double sj = (rx * d[2 * kSymB + q] + ry * d[3 * kSymB + q]) *
                            (rx * zix + ry * ziy) * inv2;
          const double si = (rx * nix + ry * niy) *
                            (rx * d[4 * kSymB + q] + ry * d[5 * kSymB + q]) *
                            inv2;
          const bool act = oki && cbase + q < b0 + lb &&
                           !(half && t == 16 && lane >= 16);
          const double fj = act ? sj : 0.0, fi = act ? si : 0.0;
          ax -= fi * rx;
          ay -= fi * ry;
          jx += fj * rx;
          jy += fj * ry;
          jx = __shfl_sync(0xffffffffu, jx, (lane + 1) & 31);
          jy = __shfl_sync(0xffffffffu, jy, (lane + 1) & 31);
        }
        const int k = jb * kSymB + c * 32 + ((lane + t1) & 31);
        jsum[2 * k] += jx;
        jsum[2 * k + 1] += jy;
      }
    }
    if (oki) {
      double *o = part + (((int64_t)(B + 1) * gridDim.y + r) * N + i) * 2;
      const double f = g.w[i] / kPi;
      o[0] = ax * f;
      o[1] = ay * f;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < lb; k += kSymB) {
    double *o = part + (((int64_t)A * gridDim.y + r) * N + b0 + k) * 2;
    const double f = g.w[b0 + k] / kPi;
    o[0] = jsum[2 * k] * f;
    o[1] = jsum[2 * k + 1] * f;
  }
}

// sum_i n_i . z_i (the integral of the transposed completion)
__global__ void k_fluxT(DevGeom g, const double *z, int64_t ld, double *flux) {
  __shared__ double red[32];
  const double *zr = z + ld * blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < g.N; j += blockDim.x)
    s += g.nx[j] * zr[2 * j] + g.ny[j] * zr[2 * j + 1];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    flux[blockIdx.x] = t;
  }
}

__global__ void k_matvecT_finish(DevGeom g, const double *z, double *y,
                                 int64_t ld, int nchunk, const double *partial,
                                 const double *flux) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (j >= g.N) return;
  const double *zr = z + ld * r;
  double u0 = 0.0, u1 = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double *p = partial + (((int64_t)c * gridDim.y + r) * g.N + j) * 2;
    u0 += p[0];
    u1 += p[1];
  }
  double d00, d01, d11;
  dl_diag(g.nx[j], g.ny[j], g.kap[j], g.w[j], d00, d01, d11);
  const double m0 = zr[2 * j], m1 = zr[2 * j + 1];
  u0 += d00 * m0 + d01 * m1 - 0.5 * m0 + g.w[j] * g.nx[j] * flux[r];
  u1 += d01 * m0 + d11 * m1 - 0.5 * m1 + g.w[j] * g.ny[j] * flux[r];
  const int h = g.comp[j] - 1;  // Psi z_lambda on hole h
  if (h >= 0) {
    const double *zl = zr + 2 * g.N + 3 * h;
    u0 += g.w[j] * (zl[0] - g.y[j] * zl[2]);
    u1 += g.w[j] * (zl[1] + g.x[j] * zl[2]);
  }
  y[2 * j + ld * r] = u0;
  y[2 * j + 1 + ld * r] = u1;
}

// H^T z_mu - z_lambda: one block per (hole, rhs), fixed-order reduction
__global__ void k_matvecT_h(DevGeom g, const double *z, double *y,
                            int64_t ld) {
  __shared__ double red[3][256];
  const int h = blockIdx.x, r = blockIdx.y;
  const double *zr = z + ld * r;
  double a0 = 0, a1 = 0, a2 = 0;
  for (int64_t j = threadIdx.x; j < g.N; j += blockDim.x) {
    const double rx = g.x[j] - g.centers[2 * h];
    const double ry = g.y[j] - g.centers[2 * h + 1];
    double s00, s01, s11;
    stokeslet(rx, ry, s00, s01, s11);
    const double r2 = rx * rx + ry * ry;
    const double z0 = zr[2 * j], z1 = zr[2 * j + 1];
    a0 += s00 * z0 + s01 * z1;
    a1 += s01 * z0 + s11 * z1;
    a2 += (-ry * z0 + rx * z1) / (4.0 * kPi * r2);
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
    const int64_t row = 2 * g.N + 3 * h + threadIdx.x;
    y[row + ld * r] = red[threadIdx.x][0] - zr[row];
  }
}

void launch_matvec_adjoint(const DevGeom &g, int nrhs, const double *z,
                           double *y, int64_t ld, double *scratch,
                           cudaStream_t s) {
  if (nrhs == 0) return;
  int S, R;
  sym_ranges(g.N, S, R);
  const int nch = R + 1;
  double *flux = scratch + (size_t)nch * nrhs * g.N * 2;
  const size_t sm = (size_t)(6 * kSymB + 2 * S) * sizeof(double);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute((const void *)k_dlT_sym,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid((unsigned)((int64_t)R * (R + 1) / 2), nrhs);
  k_dlT_sym<<<grid, kSymB, sm, s>>>(g, z, ld, S, R, scratch);
  note_launches(1);
  k_fluxT<<<nrhs, 1024, 0, s>>>(g, z, ld, flux);
  note_launches(1);
  dim3 g2((unsigned)((g.N + 127) / 128), nrhs);
  k_matvecT_finish<<<g2, 128, 0, s>>>(g, z, y, ld, nch, scratch, flux);
  note_launches(1);
  if (g.p) {
    k_matvecT_h<<<dim3(g.p, nrhs), 256, 0, s>>>(g, z, y, ld);
    note_launches(1);
  }
}

// y = A x (one column) with the double-layer sums in double-float
// arithmetic (k_dlf.cu) and every O(N) term in FP64, as in launch_matvec.
void launch_matvec_fast(const DevGeom &g, const double *x, double *y,
                        const int32_t *blk, int nblk, double *scratch,
                        cudaStream_t s) {
  const int nch = launch_dlf_sym(g, x, blk, nblk, scratch, s);
  double *flux = scratch + (size_t)nch * g.N * 2;
  k_flux<<<1, 1024, 0, s>>>(g, x, 0, flux);
  note_launches(1);
  dim3 g2((unsigned)((g.N + 127) / 128), 1);
  k_matvec_finish<<<g2, 128, 0, s>>>(g, x, y, 0, nch, scratch, flux);
  note_launches(1);
  if (g.p) {
    k_matvec_psi<<<dim3(g.p, 1), 256, 0, s>>>(g, x, y, 0);
    note_launches(1);
  }
}

// A^T z (one column) with the transposed double-layer sums in double-float
// arithmetic (k_dlf.cu) and every O(N) term in FP64, as in
// launch_matvec_adjoint.
void launch_matvec_fast_adjoint(const DevGeom &g, const double *z, double *y,
                                const int32_t *blk, int nblk, double *scratch,
                                cudaStream_t s) {
  const int nch = launch_dlfT_sym(g, z, blk, nblk, scratch, s);
  double *flux = scratch + (size_t)nch * g.N * 2;
  k_fluxT<<<1, 1024, 0, s>>>(g, z, 0, flux);
  note_launches(1);
  dim3 g2((unsigned)((g.N + 127) / 128), 1);
  k_matvecT_finish<<<g2, 128, 0, s>>>(g, z, y, 0, nch, scratch, flux);
  note_launches(1);
  if (g.p) {
    k_matvecT_h<<<dim3(g.p, 1), 256, 0, s>>>(g, z, y, 0);
    note_launches(1);
  }
}

// ---------------------------------------------------------------------------
// Laplace Neumann form (one DOF per node, FP64): the operator
// y = (1/2 I + D + N) mu and the single-layer potential
// u(t) = -(1/2pi) sum_j log|t - x_j| w_j mu_j at targets.  One thread per
// target, the sources staged in shared memory; N mu = sum_j w_j mu_j is
// the per-column flux sum of k_lap_wsum (fixed-order reduction).

__global__ void k_lap_wsum(DevGeom g, const double *x, int64_t ld,
                           double *out) {
  __shared__ double red[32];
  const double *xr = x + ld * blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < g.N; j += blockDim.x) s += g.w[j] * xr[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

// mode 0: y = (1/2 I + D + N) mu at the nodes; mode 1: u = S mu at targets
__global__ void __launch_bounds__(kDlThreads)
k_lap_apply(DevGeom g, const double *mu, int64_t ld, int64_t nt,
            const double *tx, const double *ty, const double *wsum, int mode,
            double *y, int64_t ldy) {
  __shared__ double sh[3][kDlStage];
  const int64_t t = blockIdx.x * (int64_t)kDlThreads + threadIdx.x;
  const int r = blockIdx.y;
  const double *m = mu + ld * r;
  const bool on = t < nt;
  const double px = on ? (mode ? tx[t] : g.x[t]) : 0.0;
  const double py = on ? (mode ? ty[t] : g.y[t]) : 0.0;
  const double pnx = (on && !mode) ? g.nx[t] : 0.0;
  const double pny = (on && !mode) ? g.ny[t] : 0.0;
  double acc = 0.0;
  for (int64_t base = 0; base < g.N; base += kDlStage) {
    __syncthreads();
    for (int q = threadIdx.x; q < kDlStage; q += kDlThreads) {
      const int64_t j = base + q;
      const bool ok = j < g.N;
      sh[0][q] = ok ? g.x[j] : 0.0;
      sh[1][q] = ok ? g.y[j] : 0.0;
      sh[2][q] = ok ? g.w[j] * m[j] : 0.0;
    }
    __syncthreads();
    const int cnt = (int)(g.N - base < kDlStage ? g.N - base : kDlStage);
    for (int q = 0; q < cnt; ++q) {
      const double rx = px - sh[0][q], ry = py - sh[1][q];
      const double r2 = rx * rx + ry * ry;
      if (mode) {
        acc += log(r2) * sh[2][q];
      } else if (base + q != t) {
        acc += (rx * pnx + ry * pny) / r2 * sh[2][q];
      }
    }
  }
  if (!on) return;
  if (mode) {
    y[t + ldy * r] = -acc / (4.0 * kPi);  // log r^2 = 2 log r
  } else {
    const double mt = m[t];
    y[t + ldy * r] = 0.5 * mt - acc / (2.0 * kPi) +
                     g.kap[t] * (0.25 / kPi) * g.w[t] * mt + wsum[r];
  }
}

void launch_lap_matvec(const DevGeom &g, int nrhs, const double *x, double *y,
                       int64_t ld, double *scratch, cudaStream_t s) {
  if (nrhs == 0) return;
  k_lap_wsum<<<nrhs, 1024, 0, s>>>(g, x, ld, scratch);
  dim3 grid((unsigned)((g.N + kDlThreads - 1) / kDlThreads), nrhs);
  k_lap_apply<<<grid, kDlThreads, 0, s>>>(g, x, ld, g.N, nullptr, nullptr,
                                          scratch, 0, y, ld);
  note_launches(2);
}

void launch_lap_potential(const DevGeom &g, int nrhs, const double *sol,
                          int64_t ld, int64_t nt, const double *tx,
                          const double *ty, double *u, cudaStream_t s) {
  if (nrhs == 0 || nt == 0) return;
  dim3 grid((unsigned)((nt + kDlThreads - 1) / kDlThreads), nrhs);
  k_lap_apply<<<grid, kDlThreads, 0, s>>>(g, sol, ld, nt, tx, ty, nullptr, 1,
                                          u, nt);
  note_launches(1);
}

void launch_matvec(const DevGeom &g, int nrhs, const double *x, double *y,
                   int64_t ld, double *scratch, cudaStream_t s) {
  if (nrhs == 0) return;
  int S, R;
  sym_ranges(g.N, S, R);
  const int nch = R + 1;
  double *flux = scratch + (size_t)nch * nrhs * g.N * 2;
  const size_t sm = (size_t)(5 * kSymB + 2 * S) * sizeof(double);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute((const void *)k_dl_sym,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  dim3 grid((unsigned)((int64_t)R * (R + 1) / 2), nrhs);
  k_dl_sym<<<grid, kSymB, sm, s>>>(g, x, ld, S, R, scratch);
  note_launches(1);
  k_flux<<<nrhs, 1024, 0, s>>>(g, x, ld, flux);
  note_launches(1);
  dim3 g2((unsigned)((g.N + 127) / 128), nrhs);
  k_matvec_finish<<<g2, 128, 0, s>>>(g, x, y, ld, nch, scratch, flux);
  note_launches(1);
  if (g.p) {
    k_matvec_psi<<<dim3(g.p, nrhs), 256, 0, s>>>(g, x, y, ld);
    note_launches(1);
  }
}

}  // namespace skel
