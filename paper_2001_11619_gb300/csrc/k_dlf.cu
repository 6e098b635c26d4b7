// The double-layer sums of the operator apply (Eq. stokesbie, j != i) in
// double-float arithmetic: every value is an unevaluated sum of two floats
// (h + l, about 48 significant bits) and is combined with the error-free
// transformations of Knuth (TwoSum), Dekker (FastTwoSum) and an FMA-based
// exact product.  GB300 runs FP32 about sixty times faster than FP64, so
// these sums cost a fraction of the FP64 ones at ~1e-14 relative accuracy
// per term.  They serve as the operator inside the GMRES iterations of the
// mixed form; the residual that decides convergence is the FP64 one.
//
// Coordinates: the nodes come in blocks of at most kThreads consecutive
// nodes of one curve (blk[2b] = first node, blk[2b+1] = count).  While a
// CTA works on a block of targets it shifts targets and sources to an
// origin at the block's first node (in FP64) before splitting them into
// float pairs, so the difference r = t - s of two nearby nodes keeps
// ~2^-48 relative accuracy with respect to the block's arc rather than to
// |x|.
#include "kmath.cuh"

namespace skel {

namespace {

struct f2 {
  float h, l;
};

// a + b = s + e exactly (Knuth)
__device__ __forceinline__ f2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// a + b = s + e exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ f2 df_add(f2 a, f2 b) {
  const f2 s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ f2 df_neg(f2 a) { return {-a.h, -a.l}; }

// product: the exact product of the high parts by FMA, plus cross terms
__device__ __forceinline__ f2 df_mul(f2 a, f2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ f2 df_sqr(f2 a) {
  const float p = a.h * a.h;
  float e = fmaf(a.h, a.h, -p);
  e = fmaf(a.h + a.h, a.l, e);
  return fast_two_sum(p, e);
}

// 1/a for a > 0: approximate float reciprocal y, e = 1 - a y formed with
// FMAs (the first one exact), then y (1 + e + e^2), the truncated series of
// 1/(1 - e)
__device__ __forceinline__ f2 df_rcp(f2 a) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a.h));
  float e = fmaf(-a.h, y, 1.0f);
  e = fmaf(-a.l, y, e);
  return fast_two_sum(y, y * fmaf(e, e, e));
}

// Unnormalised forms for intermediate values: the pair (h, l) is left
// without the final FastTwoSum, so |l| may reach a few units in the last
// place of h instead of half of one.  Every consumer below (TwoSum of the
// high parts, FMA products with the low parts folded in) stays accurate
// for such inputs; sums (df_add) renormalise.  This saves 3 FP32
// operations per product.
__device__ __forceinline__ f2 df_mul_u(f2 a, f2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return {p, e};
}

__device__ __forceinline__ f2 df_sqr_u(f2 a) {
  const float p = a.h * a.h;
  float e = fmaf(a.h, a.h, -p);
  e = fmaf(a.h + a.h, a.l, e);
  return {p, e};
}

__device__ __forceinline__ f2 split(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}

__device__ __forceinline__ double join(f2 a) {
  return (double)a.h + (double)a.l;
}

constexpr int kThreads = 128;
constexpr int kStage = 256;

}  // namespace

// Symmetric pair sums, as k_dl_sym (k_geom.cu) does them in FP64: the
// product of a pair is the quadratic form a rx^2 + b rx ry + c ry^2 over
// |r|^4 (a = nx mx, b = nx my + ny mx, c = ny my, m = w mu), and the two
// directions of a pair share r, its squares, |r|^2 and the reciprocal.
// Ranges of G consecutive blocks; CTA (A, B), A <= B, takes the targets of
// range A against the sources of range B (block jb >= ib, and i < j inside
// one block, when A == B).  The i sums go to slot B + 1, the j sums to slot
// A: a node of range X receives the R + 1 slots 0..R once each, summed in
// slot order (deterministic).  Output layout partial[(slot * N + t) * 2 + a]
// of (1/pi) sum_j (r.n_j)(r.(w_j mu_j)) r / |r|^4, r = x_t - x_j, j != t.
// Inside a CTA, warp w holds targets 32 w + lane of the current target
// block; the four warps take four different chunks of 32 sources per
// round, lane l taking source (l + t) mod 32 at step t, and the sources'
// running sums move one lane down per step (shuffle).
__global__ void __launch_bounds__(kThreads)
k_dlf_sym(DevGeom g, const double *mu, const int32_t *blk, int nblk, int G,
          int R, double *partial) {
  extern __shared__ double dsm[];
  f2 *jd = reinterpret_cast<f2 *>(dsm);  // sources of one block: [5][kThreads]
  double *jsum = dsm + 5 * kThreads;     // j sums of range B: [G * kThreads][2]
  int x = blockIdx.x, A = 0;
  while (x >= R - A) {
    x -= R - A;
    ++A;
  }
  const int B = A + x;
  const int64_t N = g.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ba0 = A * G, ba1 = ba0 + G < nblk ? ba0 + G : nblk;
  const int bb0 = B * G, bb1 = bb0 + G < nblk ? bb0 + G : nblk;
  const int64_t jr0 = blk[2 * bb0];
  const int lbn = (int)(blk[2 * (bb1 - 1)] + blk[2 * (bb1 - 1) + 1] - jr0);
  for (int k = threadIdx.x; k < 2 * lbn; k += kThreads) jsum[k] = 0.0;
  for (int ib = ba0; ib < ba1; ++ib) {
    const int64_t i0 = blk[2 * ib];
    const int icnt = blk[2 * ib + 1];
    const double ox = g.x[i0], oy = g.y[i0];  // the target block's origin
    const int64_t i = i0 + threadIdx.x;
    const bool oki = threadIdx.x < icnt;
    f2 px{0.f, 0.f}, py{0.f, 0.f}, pa{0.f, 0.f}, pb{0.f, 0.f}, pc{0.f, 0.f};
    if (oki) {
      const double mx = g.w[i] * mu[2 * i], my = g.w[i] * mu[2 * i + 1];
      px = split(g.x[i] - ox);
      py = split(g.y[i] - oy);
      pa = split(g.nx[i] * mx);
      pb = split(g.nx[i] * my + g.ny[i] * mx);
      pc = split(g.ny[i] * my);
    }
    f2 ax{0.f, 0.f}, ay{0.f, 0.f};
    for (int jb = (A == B ? ib : bb0); jb < bb1; ++jb) {
      const int64_t j0 = blk[2 * jb];
      const int jcnt = blk[2 * jb + 1];
      __syncthreads();  // the previous block's sources are consumed
      {
        f2 sx{0.f, 0.f}, sy{0.f, 0.f}, sa{0.f, 0.f}, sb{0.f, 0.f},
            sc{0.f, 0.f};
        if ((int)threadIdx.x < jcnt) {
          const int64_t j = j0 + threadIdx.x;
          const double mx = g.w[j] * mu[2 * j], my = g.w[j] * mu[2 * j + 1];
          sx = split(g.x[j] - ox);
          sy = split(g.y[j] - oy);
          sa = split(g.nx[j] * mx);
          sb = split(g.nx[j] * my + g.ny[j] * mx);
          sc = split(g.ny[j] * my);
        }
        jd[threadIdx.x] = sx;
        jd[kThreads + threadIdx.x] = sy;
        jd[2 * kThreads + threadIdx.x] = sa;
        jd[3 * kThreads + threadIdx.x] = sb;
        jd[4 * kThreads + threadIdx.x] = sc;
      }
      __syncthreads();
      const bool dblk = A == B && jb == ib;
      for (int round = 0; round < 4; ++round) {
        const int c = (round + w) & 3;
        if (round) __syncthreads();  // one warp per chunk of j sums
        if ((dblk && c < w) || c * 32 >= jcnt || w * 32 >= icnt) continue;
        const bool half = dblk && c == w;
        const int t0 = half ? 1 : 0, t1 = half ? 17 : 32;
        const f2 *d = jd + c * 32;
        f2 jx{0.f, 0.f}, jy{0.f, 0.f};
        for (int t = t0; t < t1; ++t) {
          const int q = (lane + t) & 31;
          // normalised differences: for nearby nodes the low parts of the
          // coordinates exceed the difference's own rounding, and an
          // unnormalised r would lose its low part squared in |r|^2
          const f2 rx = df_add(px, df_neg(d[q]));
          const f2 ry = df_add(py, df_neg(d[kThreads + q]));
          const f2 xx = df_sqr_u(rx), yy = df_sqr_u(ry), xy = df_mul_u(rx, ry);
          const f2 inv = df_rcp(df_add(xx, yy));
          const f2 inv2 = df_sqr_u(inv);
          const f2 qf = df_add(df_mul_u(d[2 * kThreads + q], xx),
                               df_add(df_mul_u(d[3 * kThreads + q], xy),
                                      df_mul_u(d[4 * kThreads + q], yy)));
          const f2 qr = df_add(df_mul_u(pa, xx),
                               df_add(df_mul_u(pb, xy), df_mul_u(pc, yy)));
          const bool act = oki && c * 32 + q < jcnt &&
                           !(half && t == 16 && lane >= 16);
          const f2 z{0.f, 0.f};
          const f2 sf = act ? df_mul_u(qf, inv2) : z;
          const f2 sr = act ? df_mul_u(qr, inv2) : z;
          // the accumulators stay normalised
          ax = df_add(ax, df_mul_u(sf, rx));
          ay = df_add(ay, df_mul_u(sf, ry));
          jx = df_add(jx, df_neg(df_mul_u(sr, rx)));
          jy = df_add(jy, df_neg(df_mul_u(sr, ry)));
          const int src = (lane + 1) & 31;
          jx.h = __shfl_sync(0xffffffffu, jx.h, src);
          jx.l = __shfl_sync(0xffffffffu, jx.l, src);
          jy.h = __shfl_sync(0xffffffffu, jy.h, src);
          jy.l = __shfl_sync(0xffffffffu, jy.l, src);
        }
        const int jl = c * 32 + ((lane + t1) & 31);
        if (jl < jcnt) {
          const int k = (int)(j0 - jr0) + jl;
          jsum[2 * k] += join(jx);
          jsum[2 * k + 1] += join(jy);
        }
      }
    }
    if (oki) {
      double *o = partial + ((int64_t)(B + 1) * N + i) * 2;
      o[0] = join(ax) / kPi;
      o[1] = join(ay) / kPi;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < lbn; k += kThreads) {
    double *o = partial + ((int64_t)A * N + jr0 + k) * 2;
    o[0] = jsum[2 * k] / kPi;
    o[1] = jsum[2 * k + 1] / kPi;
  }
}

// The transposed sums in double-float arithmetic, with the ranges, slots,
// origins and rotation of k_dlf_sym: node t receives
// (w_t / pi) sum_i (r.n_t)(r.z_i) r / |r|^4, r = x_i - x_t.  For a pair
// (i, j), r = x_i - x_j, node j gets (r.n_j)(r.z_i) r / |r|^4 and node i
// gets -(r.n_i)(r.z_j) r / |r|^4; the partials carry w_t / pi.
__global__ void __launch_bounds__(kThreads)
k_dlfT_sym(DevGeom g, const double *z, const int32_t *blk, int nblk, int G,
           int R, double *partial) {
  extern __shared__ double dsm[];
  f2 *jd = reinterpret_cast<f2 *>(dsm);  // partners of one block: [6][kThreads]
  double *jsum = dsm + 6 * kThreads;     // their sums over range B
  int x = blockIdx.x, A = 0;
  while (x >= R - A) {
    x -= R - A;
    ++A;
  }
  const int B = A + x;
  const int64_t N = g.N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ba0 = A * G, ba1 = ba0 + G < nblk ? ba0 + G : nblk;
  const int bb0 = B * G, bb1 = bb0 + G < nblk ? bb0 + G : nblk;
  const int64_t jr0 = blk[2 * bb0];
  const int lbn = (int)(blk[2 * (bb1 - 1)] + blk[2 * (bb1 - 1) + 1] - jr0);
  for (int k = threadIdx.x; k < 2 * lbn; k += kThreads) jsum[k] = 0.0;
  for (int ib = ba0; ib < ba1; ++ib) {
    const int64_t i0 = blk[2 * ib];
    const int icnt = blk[2 * ib + 1];
    const double ox = g.x[i0], oy = g.y[i0];  // the block's origin
    const int64_t i = i0 + threadIdx.x;
    const bool oki = threadIdx.x < icnt;
    f2 px{0.f, 0.f}, py{0.f, 0.f}, pnx{0.f, 0.f}, pny{0.f, 0.f},
        pzx{0.f, 0.f}, pzy{0.f, 0.f};
    if (oki) {
      px = split(g.x[i] - ox);
      py = split(g.y[i] - oy);
      pnx = split(g.nx[i]);
      pny = split(g.ny[i]);
      pzx = split(z[2 * i]);
      pzy = split(z[2 * i + 1]);
    }
    f2 ax{0.f, 0.f}, ay{0.f, 0.f};
    for (int jb = (A == B ? ib : bb0); jb < bb1; ++jb) {
      const int64_t j0 = blk[2 * jb];
      const int jcnt = blk[2 * jb + 1];
      __syncthreads();  // the previous block's partners are consumed
      {
        f2 v[6] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f},
                   {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if ((int)threadIdx.x < jcnt) {
          const int64_t j = j0 + threadIdx.x;
          v[0] = split(g.x[j] - ox);
          v[1] = split(g.y[j] - oy);
          v[2] = split(g.nx[j]);
          v[3] = split(g.ny[j]);
          v[4] = split(z[2 * j]);
          v[5] = split(z[2 * j + 1]);
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) jd[e * kThreads + threadIdx.x] = v[e];
      }
      __syncthreads();
      const bool dblk = A == B && jb == ib;
      for (int round = 0; round < 4; ++round) {
        const int c = (round + w) & 3;
        if (round) __syncthreads();  // one warp per chunk of partner sums
        if ((dblk && c < w) || c * 32 >= jcnt || w * 32 >= icnt) continue;
        const bool half = dblk && c == w;
        const int t0 = half ? 1 : 0, t1 = half ? 17 : 32;
        const f2 *d = jd + c * 32;
        f2 jx{0.f, 0.f}, jy{0.f, 0.f};
        for (int t = t0; t < t1; ++t) {
          const int q = (lane + t) & 31;
          // normalised differences (see k_dlf_sym)
          const f2 rx = df_add(px, df_neg(d[q]));
          const f2 ry = df_add(py, df_neg(d[kThreads + q]));
          const f2 inv = df_rcp(df_add(df_sqr_u(rx), df_sqr_u(ry)));
          const f2 inv2 = df_sqr_u(inv);
          // node j: (r.n_j)(r.z_i); node i: (r.n_i)(r.z_j)
          const f2 nj = df_add(df_mul_u(rx, d[2 * kThreads + q]),
                               df_mul_u(ry, d[3 * kThreads + q]));
          const f2 zi = df_add(df_mul_u(rx, pzx), df_mul_u(ry, pzy));
          const f2 ni = df_add(df_mul_u(rx, pnx), df_mul_u(ry, pny));
          const f2 zj = df_add(df_mul_u(rx, d[4 * kThreads + q]),
                               df_mul_u(ry, d[5 * kThreads + q]));
          const bool act = oki && c * 32 + q < jcnt &&
                           !(half && t == 16 && lane >= 16);
          const f2 zr{0.f, 0.f};
          const f2 sj = act ? df_mul_u(df_mul_u(nj, zi), inv2) : zr;
          const f2 si = act ? df_mul_u(df_mul_u(ni, zj), inv2) : zr;
          ax = df_add(ax, df_neg(df_mul_u(si, rx)));
          ay = df_add(ay, df_neg(df_mul_u(si, ry)));
          jx = df_add(jx, df_mul_u(sj, rx));
          jy = df_add(jy, df_mul_u(sj, ry));
          const int src = (lane + 1) & 31;
          jx.h = __shfl_sync(0xffffffffu, jx.h, src);
          jx.l = __shfl_sync(0xffffffffu, jx.l, src);
          jy.h = __shfl_sync(0xffffffffu, jy.h, src);
          jy.l = __shfl_sync(0xffffffffu, jy.l, src);
        }
        const int jl = c * 32 + ((lane + t1) & 31);
        if (jl < jcnt) {
          const int k = (int)(j0 - jr0) + jl;
          jsum[2 * k] += join(jx);
          jsum[2 * k + 1] += join(jy);
        }
      }
    }
    if (oki) {
      double *o = partial + ((int64_t)(B + 1) * N + i) * 2;
      const double f = g.w[i] / kPi;
      o[0] = join(ax) * f;
      o[1] = join(ay) * f;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < lbn; k += kThreads) {
    double *o = partial + ((int64_t)A * N + jr0 + k) * 2;
    const double f = g.w[jr0 + k] / kPi;
    o[0] = jsum[2 * k] * f;
    o[1] = jsum[2 * k + 1] * f;
  }
}

int dlf_block_size() { return kThreads; }

// Blocks per range: about 128 ranges (8256 CTAs), at most 32 blocks.
static int dlf_group(int nblk) {
  int G = (nblk + 127) / 128;
  return G < 1 ? 1 : (G > 32 ? 32 : G);
}

size_t dlf_scratch(int64_t N, int nblk) {
  const int G = dlf_group(nblk);
  const int R = (nblk + G - 1) / G;
  return (size_t)(R + 1) * N * 2 + 8;
}

int launch_dlfT_sym(const DevGeom &g, const double *z, const int32_t *blk,
                    int nblk, double *partial, cudaStream_t s) {
  const int G = dlf_group(nblk);
  const int R = (nblk + G - 1) / G;
  const size_t sm = (size_t)(6 * kThreads + 2 * G * kThreads) * sizeof(double);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute((const void *)k_dlfT_sym,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_dlfT_sym<<<(unsigned)((int64_t)R * (R + 1) / 2), kThreads, sm, s>>>(
      g, z, blk, nblk, G, R, partial);
  note_launches(1);
  return R + 1;
}

int launch_dlf_sym(const DevGeom &g, const double *mu, const int32_t *blk,
                   int nblk, double *partial, cudaStream_t s) {
  const int G = dlf_group(nblk);
  const int R = (nblk + G - 1) / G;
  const size_t sm = (size_t)(5 * kThreads + 2 * G * kThreads) * sizeof(double);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute((const void *)k_dlf_sym,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_dlf_sym<<<(unsigned)((int64_t)R * (R + 1) / 2), kThreads, sm, s>>>(
      g, mu, blk, nblk, G, R, partial);
  note_launches(1);
  return R + 1;
}

}  // namespace skel
