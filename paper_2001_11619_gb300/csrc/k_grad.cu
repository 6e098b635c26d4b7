// Shape derivatives of the bordered system for the differentiation path:
//   L = z^T A(geom) s            (skel_grad_bilinear)
//   ubar . E(geom) s, E^T ubar   (skel_grad_velocity)
// with respect to every node's curve samples (gamma, gamma', gamma'') and
// the hole centres, for fixed vectors.  With A^T z = dJ/ds they give the
// adjoint shape gradient of an objective J of the interior velocity.
//
// Stresslet pairs (Eq. stokesbie, r = x_t - x_j, q_j = w_j mu_j):
//   F = (1/pi) (r.n_j)(r.q_j)(r.z_t) / |r|^4 = (1/pi) a b c / rho^2
//   dF/dr   = [(n_j b c + q_j a c + z_t a b) - 4 a b c r / rho] / (pi rho^2)
//   dF/dn_j = r b c / (pi rho^2),   dF/dq_j = r a c / (pi rho^2)
// summed over sources for each target and over targets for each source.
// For the bilinear form (targets = nodes) one symmetric pass takes both
// orders of each pair of nodes at once (k_gpair_sym); the velocity form
// (interior targets) runs the source pass.  Partial sums are deterministic.
// The
// diagonal limit, the rank-one N, the Stokeslet/rotlet columns H and the
// Psi rows (Sec. 3.1) are per-node or per-hole terms.  Chain rules for
// n = J t, t = gamma'/|gamma'|, w = |gamma'| dt:
//   dL/dgamma' += (J^T dL/dn - t (n . dL/dn)) / |gamma'| + dL/dw dt t.
#include "kmath.cuh"

namespace skel {

namespace {

constexpr int kGT = 128;      // threads per CTA of the pair passes
constexpr int kGStage = 128;  // staged partners per round

__device__ __forceinline__ double gk_rcp(double v) { return recip_nr3(v); }

}  // namespace

// Source pass: for every source node j, partial[(c * N + j) * 6 + ...] =
// sum over targets t of chunk c of (-dF/dr, dF/dn_j, dF/dq_j).  Targets are
// the nodes (tx == nullptr; weights zt, the pair t == j skipped) or nt
// interior points (tx, ty; weights zt).
__global__ void __launch_bounds__(kGT)
k_gpair_src(DevGeom g, const double *mu, int64_t nt, const double *tx,
            const double *ty, const double *zt, int nchunk, double *partial) {
  __shared__ double sh[4][kGStage];
  const int64_t j = blockIdx.x * (int64_t)kGT + threadIdx.x;
  const int c = blockIdx.z;
  const int64_t per = (nt + nchunk - 1) / nchunk;
  const int64_t t0 = c * per, t1 = t0 + per < nt ? t0 + per : nt;
  const bool on = j < g.N;
  const bool self = tx == nullptr;
  double sx = 0, sy = 0, nx = 0, ny = 0, qx = 0, qy = 0;
  if (on) {
    const double w = g.w[j];
    sx = g.x[j];
    sy = g.y[j];
    nx = g.nx[j];
    ny = g.ny[j];
    qx = w * mu[2 * j];
    qy = w * mu[2 * j + 1];
  }
  double o0 = 0, o1 = 0, o2 = 0, o3 = 0, o4 = 0, o5 = 0;
  for (int64_t base = t0; base < t1; base += kGStage) {
    __syncthreads();
    for (int q = threadIdx.x; q < kGStage; q += kGT) {
      const int64_t t = base + q;
      const bool ok = t < t1;
      sh[0][q] = ok ? (self ? g.x[t] : tx[t]) : 0.0;
      sh[1][q] = ok ? (self ? g.y[t] : ty[t]) : 0.0;
      sh[2][q] = ok ? zt[2 * t] : 0.0;
      sh[3][q] = ok ? zt[2 * t + 1] : 0.0;
    }
    __syncthreads();
    const int cnt = (int)(t1 - base < kGStage ? t1 - base : kGStage);
    for (int q = 0; q < cnt; ++q) {
      if (self && base + q == j) continue;
      const double rx = sh[0][q] - sx, ry = sh[1][q] - sy;
      const double zx = sh[2][q], zy = sh[3][q];
      const double rho = rx * rx + ry * ry;
      const double a = rx * nx + ry * ny;
      const double b = rx * qx + ry * qy;
      const double cc = rx * zx + ry * zy;
      const double i2 = gk_rcp(kPi * rho * rho);
      const double abc4 = 4.0 * a * b * cc * gk_rcp(rho);
      o0 -= (nx * b * cc + qx * a * cc + zx * a * b - abc4 * rx) * i2;
      o1 -= (ny * b * cc + qy * a * cc + zy * a * b - abc4 * ry) * i2;
      const double bc = b * cc * i2, ac = a * cc * i2;
      o2 += rx * bc;
      o3 += ry * bc;
      o4 += rx * ac;
      o5 += ry * ac;
    }
  }
  if (!on) return;
  double *out = partial + ((int64_t)c * g.N + j) * 6;
  out[0] = o0;
  out[1] = o1;
  out[2] = o2;
  out[3] = o3;
  out[4] = o4;
  out[5] = o5;
}

// Symmetric pass of the bilinear form over the nodes.  For a pair (i, j),
// r = x_i - x_j, both orders share r, |r|^2 and its reciprocal:
//   order A (target i, source j): a = r.n_j, b = r.q_j, c = r.z_i,
//   order B (target j, source i): a = r.n_i, b = r.q_i, c = r.z_j
// (order B written with r instead of x_j - x_i: its dF/dr keeps the same
// form, its source derivatives change sign).  Per node the pass sums the
// position derivative P (target minus source side), dF/dn and dF/dq, into
// part[(slot * N + node) * 6 + (Px, Py, nx, ny, qx, qy)].  Ranges, slots and
// the in-warp rotation of the partners' sums as in k_dl_sym (k_geom.cu).
__global__ void __launch_bounds__(kGT)
k_gpair_sym(DevGeom g, const double *zt, const double *mu, int S, int R,
            double *part) {
  extern __shared__ double sm[];
  double *jd = sm;                // partners of one block: [8][kGT]
  double *jsum = sm + 8 * kGT;    // their sums over range B: [S][6]
  int x = blockIdx.x, A = 0;
  while (x >= R - A) {
    x -= R - A;
    ++A;
  }
  const int B = A + x;
  const int64_t N = g.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t a0 = (int64_t)A * S, b0 = (int64_t)B * S;
  const int la = (int)(N - a0 < S ? N - a0 : S);
  const int lb = (int)(N - b0 < S ? N - b0 : S);
  const int nbi = (la + kGT - 1) / kGT, nbj = (lb + kGT - 1) / kGT;
  constexpr double kInvPi = 1.0 / kPi;
  for (int k = threadIdx.x; k < 6 * S; k += kGT) jsum[k] = 0.0;
  for (int ib = 0; ib < nbi; ++ib) {
    const int64_t i = a0 + (int64_t)ib * kGT + threadIdx.x;
    const bool oki = i < a0 + la;
    double px = 0, py = 0, nix = 0, niy = 0, qix = 0, qiy = 0, zix = 0,
           ziy = 0;
    if (oki) {
      px = g.x[i];
      py = g.y[i];
      nix = g.nx[i];
      niy = g.ny[i];
      qix = g.w[i] * mu[2 * i];
      qiy = g.w[i] * mu[2 * i + 1];
      zix = zt[2 * i];
      ziy = zt[2 * i + 1];
    }
    double o[6] = {0, 0, 0, 0, 0, 0};
    for (int jb = (A == B ? ib : 0); jb < nbj; ++jb) {
      const int64_t jbase = b0 + (int64_t)jb * kGT;
      __syncthreads();  // the previous block's partners are consumed
      {
        const int64_t j = jbase + threadIdx.x;
        const bool ok = j < b0 + lb;
        jd[threadIdx.x] = ok ? g.x[j] : 0.0;
        jd[kGT + threadIdx.x] = ok ? g.y[j] : 0.0;
        jd[2 * kGT + threadIdx.x] = ok ? g.nx[j] : 0.0;
        jd[3 * kGT + threadIdx.x] = ok ? g.ny[j] : 0.0;
        jd[4 * kGT + threadIdx.x] = ok ? g.w[j] * mu[2 * j] : 0.0;
        jd[5 * kGT + threadIdx.x] = ok ? g.w[j] * mu[2 * j + 1] : 0.0;
        jd[6 * kGT + threadIdx.x] = ok ? zt[2 * j] : 0.0;
        jd[7 * kGT + threadIdx.x] = ok ? zt[2 * j + 1] : 0.0;
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
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int t = t0; t < t1; ++t) {
          const int q = (lane + t) & 31;
          const double rx = px - d[q], ry = py - d[kGT + q];
          const double nxj = d[2 * kGT + q], nyj = d[3 * kGT + q];
          const double qxj = d[4 * kGT + q], qyj = d[5 * kGT + q];
          const double zxj = d[6 * kGT + q], zyj = d[7 * kGT + q];
          const double rho = rx * rx + ry * ry;
          const double inv = gk_rcp(rho);
          const double i2 = inv * inv * kInvPi;
          // order A: target i, source j
          const double aA = rx * nxj + ry * nyj, bA = rx * qxj + ry * qyj,
                       cA = rx * zix + ry * ziy;
          const double abA = aA * bA, bcA = bA * cA, acA = aA * cA;
          const double eA = 4.0 * abA * cA * inv;
          // order B: target j, source i
          const double aB = rx * nix + ry * niy, bB = rx * qix + ry * qiy,
                       cB = rx * zxj + ry * zyj;
          const double abB = aB * bB, bcB = bB * cB, acB = aB * cB;
          const double eB = 4.0 * abB * cB * inv;
          double dPx = ((nxj * bcA + qxj * acA + zix * abA - eA * rx) -
                        (nix * bcB + qix * acB + zxj * abB - eB * rx)) * i2;
          double dPy = ((nyj * bcA + qyj * acA + ziy * abA - eA * ry) -
                        (niy * bcB + qiy * acB + zyj * abB - eB * ry)) * i2;
          double fA = bcA * i2, gA = acA * i2, fB = bcB * i2, gB = acB * i2;
          const bool act = oki && cbase + q < b0 + lb &&
                           !(half && t == 16 && lane >= 16);
          if (!act) dPx = dPy = fA = gA = fB = gB = 0.0;
          o[0] += dPx;
          o[1] += dPy;
          o[2] -= fB * rx;
          o[3] -= fB * ry;
          o[4] -= gB * rx;
          o[5] -= gB * ry;
          s[0] -= dPx;
          s[1] -= dPy;
          s[2] += fA * rx;
          s[3] += fA * ry;
          s[4] += gA * rx;
          s[5] += gA * ry;
          const int src = (lane + 1) & 31;
#pragma unroll
          for (int e = 0; e < 6; ++e) s[e] = __shfl_sync(0xffffffffu, s[e], src);
        }
        const int jl = c * 32 + ((lane + t1) & 31);
        const int k = jb * kGT + jl;
#pragma unroll
        for (int e = 0; e < 6; ++e) jsum[6 * k + e] += s[e];
      }
    }
    if (oki) {
      double *out = part + ((int64_t)(B + 1) * N + i) * 6;
#pragma unroll
      for (int e = 0; e < 6; ++e) out[e] = o[e];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < lb; k += kGT) {
    double *out = part + ((int64_t)A * N + b0 + k) * 6;
#pragma unroll
    for (int e = 0; e < 6; ++e) out[e] = jsum[6 * k + e];
  }
}

// d/dr of z.S(r) alpha + z.R(r) beta (Stokeslet (1/4pi)(-ln|r| I +
// r r^T/|r|^2), rotlet r_perp / (4 pi |r|^2))
__device__ __forceinline__ void point_grad(double rx, double ry, double zx,
                                           double zy, double ax, double ay,
                                           double be, double &gx, double &gy) {
  const double rho = rx * rx + ry * ry;
  const double ir = 1.0 / rho;
  const double za = zx * ax + zy * ay;
  const double zr = zx * rx + zy * ry;
  const double ra = rx * ax + ry * ay;
  const double f = 1.0 / (4.0 * kPi);
  gx = f * (-za * rx * ir + (zx * ra + ax * zr) * ir - 2.0 * zr * ra * rx * ir * ir);
  gy = f * (-za * ry * ir + (zy * ra + ay * zr) * ir - 2.0 * zr * ra * ry * ir * ir);
  const double zp = zy * rx - zx * ry;
  gx += f * be * (zy * ir - 2.0 * zp * rx * ir * ir);
  gy += f * be * (-zx * ir - 2.0 * zp * ry * ir * ir);
}

// sums[0] = sum_i z_i . n_i, sums[1] = sum_j w_j n_j . mu_j (one CTA,
// fixed order)
__global__ void k_gsums(DevGeom g, const double *z, const double *mu,
                        double *sums) {
  __shared__ double sa[32], sb[32];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < g.N; i += blockDim.x) {
    a += z[2 * i] * g.nx[i] + z[2 * i + 1] * g.ny[i];
    b += g.w[i] * (g.nx[i] * mu[2 * i] + g.ny[i] * mu[2 * i + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sa[warp] = a;
    sb[warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += sa[w];
      tb += sb[w];
    }
    sums[0] = ta;
    sums[1] = tb;
  }
}

// Per node: combine the pair passes with the per-node terms and chain to
// the samples.  full != 0: the bilinear form of A (diagonal limit, N, H at
// the nodes, Psi rows, target pass); full == 0: the velocity form (source
// pass only).  g: 6N outputs (d/dx, d/dy, d/dgamma'_x, d/dgamma'_y,
// d/dgamma''_x, d/dgamma''_y).
__global__ void k_gnode(DevGeom g, const double *dx, const double *dy,
                        const double *ddx, const double *ddy, const double *dt,
                        const double *z, const double *s, int full,
                        const double *ptgt, int ntc, const double *psrc,
                        int nsc, const double *sums, double *out) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= g.N) return;
  const int64_t N = g.N;
  const double mx = s[2 * k], my = s[2 * k + 1];
  double gPx = 0, gPy = 0, gnx = 0, gny = 0, gqx = 0, gqy = 0;
  for (int c = 0; c < nsc; ++c) {
    const double *p = psrc + ((int64_t)c * N + k) * 6;
    gPx += p[0];
    gPy += p[1];
    gnx += p[2];
    gny += p[3];
    gqx += p[4];
    gqy += p[5];
  }
  double gw = gqx * mx + gqy * my;
  const double G1x = dx[k], G1y = dy[k];
  const double sp = sqrt(G1x * G1x + G1y * G1y);
  const double tX = G1x / sp, tY = G1y / sp;
  const double nX = g.nx[k], nY = g.ny[k];
  double gG1x = 0, gG1y = 0, gG2x = 0, gG2y = 0;
  if (full) {
    for (int c = 0; c < ntc; ++c) {
      const double *p = ptgt + ((int64_t)c * N + k) * 2;
      gPx += p[0];
      gPy += p[1];
    }
    const double zx = z[2 * k], zy = z[2 * k + 1];
    // diagonal limit: L2 = -(dt/2pi) cross (z.g1)(mu.g1) / |g1|^4
    const double G2x = ddx[k], G2y = ddy[k];
    const double cr = G1x * G2y - G1y * G2x;
    const double A = zx * G1x + zy * G1y, B = mx * G1x + my * G1y;
    const double g2 = G1x * G1x + G1y * G1y;
    const double kk = -dt[k] / (2.0 * kPi);
    const double ig4 = 1.0 / (g2 * g2);
    gG1x = kk * (G2y * A * B * ig4 + cr * (zx * B + mx * A) * ig4 -
                 4.0 * cr * A * B * ig4 / g2 * G1x);
    gG1y = kk * (-G2x * A * B * ig4 + cr * (zy * B + my * A) * ig4 -
                 4.0 * cr * A * B * ig4 / g2 * G1y);
    gG2x = kk * (-G1y) * A * B * ig4;
    gG2y = kk * G1x * A * B * ig4;
    // rank-one N: (sum z.n)(sum w n.mu)
    const double Zn = sums[0], Sn = sums[1];
    const double w = g.w[k];
    gnx += zx * Sn + Zn * w * mx;
    gny += zy * Sn + Zn * w * my;
    gw += Zn * (nX * mx + nY * my);
    // H lambda at this node, and the Psi rows of its hole
    const double *lam = s + 2 * N;
    const double *zl = z + 2 * N;
    for (int c = 0; c < g.p; ++c) {
      double hx, hy;
      point_grad(g.x[k] - g.centers[2 * c], g.y[k] - g.centers[2 * c + 1], zx,
                 zy, lam[3 * c], lam[3 * c + 1], lam[3 * c + 2], hx, hy);
      gPx += hx;
      gPy += hy;
    }
    const int hc = g.comp[k];
    if (hc > 0) {
      const double *zc = zl + 3 * (hc - 1);
      gw += zc[0] * mx + zc[1] * my + zc[2] * (-g.y[k] * mx + g.x[k] * my);
      gPx += w * zc[2] * my;
      gPy -= w * zc[2] * mx;
    }
  }
  const double gnn = gnx * nX + gny * nY;
  gG1x += (-gny - tX * gnn) / sp + gw * dt[k] * tX;
  gG1y += (gnx - tY * gnn) / sp + gw * dt[k] * tY;
  out[k] = gPx;
  out[N + k] = gPy;
  out[2 * N + k] = gG1x;
  out[3 * N + k] = gG1y;
  out[4 * N + k] = gG2x;
  out[5 * N + k] = gG2y;
}

// One CTA per hole c: the centre derivative -sum_points d/dr[z.(S a + R b)]
// over the nodes (tx == nullptr, weights z) or the interior points (weights
// ubar); for interior points also the lambda part of E^T ubar:
// gs[2N+3c..] = (sum_t S(x_t - c) ubar_t, sum_t ubar_t . R(x_t - c)).
__global__ void k_gcent(DevGeom g, int64_t np, const double *tx,
                        const double *ty, const double *zt, const double *s,
                        double *gc, double *gs) {
  __shared__ double red[5][32];
  const int c = blockIdx.x;
  const double cx = g.centers[2 * c], cy = g.centers[2 * c + 1];
  const double *lam = s + 2 * g.N;
  const double ax = lam[3 * c], ay = lam[3 * c + 1], be = lam[3 * c + 2];
  double v[5] = {0, 0, 0, 0, 0};
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) {
    const double px = tx ? tx[i] : g.x[i], py = ty ? ty[i] : g.y[i];
    const double zx = zt[2 * i], zy = zt[2 * i + 1];
    const double rx = px - cx, ry = py - cy;
    double hx, hy;
    point_grad(rx, ry, zx, zy, ax, ay, be, hx, hy);
    v[0] -= hx;
    v[1] -= hy;
    if (tx) {
      double s00, s01, s11;
      stokeslet(rx, ry, s00, s01, s11);
      const double r2 = rx * rx + ry * ry;
      v[2] += s00 * zx + s01 * zy;
      v[3] += s01 * zx + s11 * zy;
      v[4] += (-ry * zx + rx * zy) / (4.0 * kPi * r2);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 5; ++q) {
    double t = v[q];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[q][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[5] = {0, 0, 0, 0, 0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      for (int q = 0; q < 5; ++q) tot[q] += red[q][w];
    gc[2 * c] = tot[0];
    gc[2 * c + 1] = tot[1];
    if (tx) {
      gs[2 * g.N + 3 * c] = tot[2];
      gs[2 * g.N + 3 * c + 1] = tot[3];
      gs[2 * g.N + 3 * c + 2] = tot[4];
    }
  }
}

// mu part of E^T ubar from the source pass: gs[2j+a] = w_j dF/dq_j,a
__global__ void k_gs_mu(DevGeom g, const double *psrc, int nsc, double *gs) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= g.N) return;
  double qx = 0, qy = 0;
  for (int c = 0; c < nsc; ++c) {
    const double *p = psrc + ((int64_t)c * g.N + j) * 6;
    qx += p[4];
    qy += p[5];
  }
  gs[2 * j] = g.w[j] * qx;
  gs[2 * j + 1] = g.w[j] * qy;
}

static int grad_chunks(int64_t n_out, int64_t n_in) {
  const int64_t blocks = (n_out + kGT - 1) / kGT;
  return balanced_chunks(blocks, (n_in + kGStage - 1) / kGStage, 8);
}

size_t grad_scratch(int64_t N, int64_t nt) {
  const int64_t m = nt > N ? nt : N;
  size_t a = (size_t)grad_chunks(N, m) * N * 8;
  int S, R;
  sym_ranges(N, S, R);
  const size_t b = (size_t)(R + 1) * N * 6;
  return (a > b ? a : b) + 8;
}

void launch_grad_bilinear(const DevGeom &g, const double *dx, const double *dy,
                          const double *ddx, const double *ddy,
                          const double *dt, const double *z, const double *s,
                          double *scratch, double *out, cudaStream_t st) {
  int S, R;
  sym_ranges(g.N, S, R);
  const int ncs = R + 1;
  double *psrc = scratch;
  double *sums = psrc + (size_t)ncs * g.N * 6;
  const size_t sm = (size_t)(8 * kGT + 6 * S) * sizeof(double);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute((const void *)k_gpair_sym,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gpair_sym<<<(unsigned)((int64_t)R * (R + 1) / 2), kGT, sm, st>>>(
      g, z, s, S, R, psrc);
  note_launches(1);
  k_gsums<<<1, 1024, 0, st>>>(g, z, s, sums);
  note_launches(1);
  k_gnode<<<(unsigned)((g.N + 127) / 128), 128, 0, st>>>(
      g, dx, dy, ddx, ddy, dt, z, s, 1, nullptr, 0, psrc, ncs, sums, out);
  note_launches(1);
  if (g.p) {
    k_gcent<<<g.p, 256, 0, st>>>(g, g.N, nullptr, nullptr, z, s,
                                 out + 6 * g.N, nullptr);
    note_launches(1);
  }
}

void launch_grad_velocity(const DevGeom &g, const double *dx,
                          const double *dy, const double *dt, const double *s,
                          int64_t nt, const double *tx, const double *ty,
                          const double *ubar, double *scratch, double *gs,
                          double *out, cudaStream_t st) {
  const int ncs = grad_chunks(g.N, nt);
  double *psrc = scratch;
  const unsigned nb = (unsigned)((g.N + kGT - 1) / kGT);
  k_gpair_src<<<dim3(nb, 1, ncs), kGT, 0, st>>>(g, s, nt, tx, ty, ubar, ncs,
                                                psrc);
  note_launches(1);
  k_gnode<<<(unsigned)((g.N + 127) / 128), 128, 0, st>>>(
      g, dx, dy, nullptr, nullptr, dt, nullptr, s, 0, nullptr, 0, psrc, ncs,
      nullptr, out);
  note_launches(1);
  k_gs_mu<<<(unsigned)((g.N + 127) / 128), 128, 0, st>>>(g, psrc, ncs, gs);
  note_launches(1);
  if (g.p) {
    k_gcent<<<g.p, 256, 0, st>>>(g, nt, tx, ty, ubar, s, out + 6 * g.N, gs);
    note_launches(1);
  }
}

}  // namespace skel
