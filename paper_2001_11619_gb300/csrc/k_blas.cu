// FP64 vector kernels for the refinement loop of the mixed-precision form
// (GMRES on the FP64 operator, preconditioned by the low-precision
// factorization; the factorization-as-preconditioner use of Eq. kinv's
// remark).  Reductions are two-stage in a fixed order, so results do not
// depend on scheduling.
#include "skel_internal.h"

namespace skel {

constexpr int kDotThreads = 256;
constexpr int kDotBlocks = 256;

// out[c] = sum_i x[i] * Y[i + ld c] for c < ncol (ncol <= 64), partials
// per block in part[block * ncol + c]
__global__ void k_multidot_partial(const double *x, const double *Y,
                                   int64_t ld, int ncol, int64_t n,
                                   double *part) {
  __shared__ double red[kDotThreads / 32][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < ncol; ++c) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kDotThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kDotThreads)
      s += x[i] * Y[i + ld * c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[warp][c] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += kDotThreads) {
    double s = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) s += red[w][c];
    part[blockIdx.x * ncol + c] = s;
  }
}

__global__ void k_multidot_final(const double *part, int nblk, int ncol,
                                 double *out) {
  const int c = threadIdx.x;
  if (c >= ncol) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[b * ncol + c];
  out[c] = s;
}

void launch_multidot(const double *x, const double *Y, int64_t ld, int ncol,
                     int64_t n, double *part, double *out, cudaStream_t s) {
  k_multidot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(x, Y, ld, ncol, n,
                                                        part);
  note_launches(1);
  k_multidot_final<<<1, 64, 0, s>>>(part, kDotBlocks, ncol, out);
  note_launches(1);
}

size_t multidot_scratch() { return (size_t)kDotBlocks * 64; }

// y <- a * y + sum_c coef[c] * X[:, c]   (coef on the device)
__global__ void k_combine(double *y, double a, const double *X, int64_t ld,
                          const double *coef, double csign, int ncol,
                          int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = a * y[i];
    for (int c = 0; c < ncol; ++c) v += csign * coef[c] * X[i + ld * c];
    y[i] = v;
  }
}

void launch_combine(double *y, double a, const double *X, int64_t ld,
                    const double *coef, double csign, int ncol, int64_t n,
                    cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4 * 152) blocks = 4 * 152;
  k_combine<<<blocks, 256, 0, s>>>(y, a, X, ld, coef, csign, ncol, n);
  note_launches(1);
}

// y <- alpha * x + beta * y  (y is not read when beta == 0)
__global__ void k_axpby(double alpha, const double *x, double beta, double *y,
                        int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = beta == 0.0 ? alpha * x[i] : alpha * x[i] + beta * y[i];
}

void launch_axpby(double alpha, const double *x, double beta, double *y,
                  int64_t n, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4 * 152) blocks = 4 * 152;
  k_axpby<<<blocks, 256, 0, s>>>(alpha, x, beta, y, n);
  note_launches(1);
}

}  // namespace skel
