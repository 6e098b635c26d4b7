// The double-layer sums of the operator apply (Eq. stokesbie, j != i) in
// double-float arithmetic: every value is an unevaluated sum of two floats
// (h + l, about 48 significant bits) and is combined with the error-free
// transformations of Knuth (TwoSum), Dekker (FastTwoSum) and an FMA-based
// exact product.  GB300 runs FP32 about sixty times faster than FP64, so
// these sums cost a fraction of the FP64 ones at ~1e-14 relative accuracy
// per term.  They serve as the operator inside the GMRES iterations of the
// mixed form; the residual that decides convergence is the FP64 one.
//
// Coordinates: every CTA takes at most kThreads consecutive targets of one
// curve (blk[2b] = first node, blk[2b+1] = count) and shifts its sources and
// targets to an origin at its first target (in FP64) before splitting them
// into float pairs, so the difference r = t - s of two nearby nodes keeps
// ~2^-48 relative accuracy with respect to the arc the CTA covers rather
// than to |x|.
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

// Same output layout as the FP64 partial sums (one RHS, targets = nodes):
// partial[(c * N + t) * 2 + a] holds source chunk c's sum
//   (1/pi) sum_j (r.n_j)(r.(w_j mu_j)) r / |r|^4,   r = x_t - x_j, j != t,
// rounded to FP64 (the 1/pi is applied there).
__global__ void __launch_bounds__(kThreads)
k_dlf_partial(DevGeom g, const double *mu, const int32_t *blk, int nchunk,
              double *partial) {
  __shared__ f2 sh[6][kStage];
  const int64_t t0 = blk[2 * blockIdx.x];
  const int64_t t = t0 + threadIdx.x;
  const int c = blockIdx.z;
  const int64_t per = (g.N + nchunk - 1) / nchunk;
  const int64_t j0 = c * per, j1 = j0 + per < g.N ? j0 + per : g.N;
  const double ox = g.x[t0], oy = g.y[t0];  // the tile's origin
  const bool on = threadIdx.x < blk[2 * blockIdx.x + 1];
  const f2 px = on ? split(g.x[t] - ox) : f2{0.f, 0.f};
  const f2 py = on ? split(g.y[t] - oy) : f2{0.f, 0.f};
  f2 a0 = {0.f, 0.f}, a1 = {0.f, 0.f};
  for (int64_t base = j0; base < j1; base += kStage) {
    __syncthreads();
    for (int q = threadIdx.x; q < kStage; q += kThreads) {
      const int64_t j = base + q;
      if (j < j1) {
        const double w = g.w[j];
        sh[0][q] = split(g.x[j] - ox);
        sh[1][q] = split(g.y[j] - oy);
        sh[2][q] = split(g.nx[j]);
        sh[3][q] = split(g.ny[j]);
        sh[4][q] = split(w * mu[2 * j]);
        sh[5][q] = split(w * mu[2 * j + 1]);
      }
    }
    __syncthreads();
    const int cnt = (int)(j1 - base < kStage ? j1 - base : kStage);
    for (int q = 0; q < cnt; ++q) {
      // normalised differences: for nearby nodes the low parts of the
      // coordinates exceed the difference's own rounding, and an
      // unnormalised r would lose its low part squared in |r|^2
      const f2 rx = df_add(px, df_neg(sh[0][q]));
      const f2 ry = df_add(py, df_neg(sh[1][q]));
      const bool skip = base + q == t;
      f2 r2 = df_add(df_sqr_u(rx), df_sqr_u(ry));  // normalised: rcp input
      if (skip) r2 = {1.f, 0.f};
      const f2 inv = df_rcp(r2);
      const f2 rn = df_add(df_mul_u(rx, sh[2][q]), df_mul_u(ry, sh[3][q]));
      const f2 tm = df_add(df_mul_u(rx, sh[4][q]), df_mul_u(ry, sh[5][q]));
      f2 s = df_mul_u(df_mul_u(rn, tm), df_sqr_u(inv));
      if (skip) s = {0.f, 0.f};
      // the accumulators stay normalised (a low part of a few units in the
      // last place, summed over thousands of terms, would cost accuracy)
      a0 = df_add(a0, df_mul_u(s, rx));
      a1 = df_add(a1, df_mul_u(s, ry));
    }
  }
  if (!on) return;
  double *out = partial + ((int64_t)c * g.N + t) * 2;
  out[0] = join(a0) / kPi;
  out[1] = join(a1) / kPi;
}

int dlf_block_size() { return kThreads; }

void launch_dlf_partial(const DevGeom &g, const double *mu,
                        const int32_t *blk, int nblk, int nchunk,
                        double *partial, cudaStream_t s) {
  dim3 grid((unsigned)nblk, 1, nchunk);
  k_dlf_partial<<<grid, kThreads, 0, s>>>(g, mu, blk, nchunk, partial);
  note_launches(1);
}

}  // namespace skel
