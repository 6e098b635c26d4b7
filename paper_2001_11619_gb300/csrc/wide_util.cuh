// FP64 tiles for the whole-GPU kernels of large boxes (k_wide.cu,
// k_wide_qr.cu): strided matrix views and a 32 x 32 output tile of
// C = C0 + sign A B computed by one CTA of 256 threads.
#pragma once

#include <cstdint>

namespace skel {
namespace wide {

constexpr int kWT = 32;    // GEMM output tile (kWT x kWT), K slab kWT
constexpr int kWNB = 32;   // LU panel / TRSM block width (one warp of rows)

// strided matrix view: element (i, j) at p[i rs + j cs]
struct MV {
  double *p;
  int64_t rs, cs;
  __device__ double &at(int64_t i, int64_t j) const { return p[i * rs + j * cs]; }
  __device__ MV sub(int64_t i, int64_t j) const { return {p + i * rs + j * cs, rs, cs}; }
};

__device__ inline MV colmajor(double *p, int64_t ld) { return {p, 1, ld}; }
__device__ inline MV transposed(double *p, int64_t ld) { return {p, ld, 1}; }

// C(0:M, 0:N) tile at (r0, c0) = C0 + sign * A(0:M, 0:K) B(0:K, 0:N).
// 256 threads, 2 x 2 outputs each; slabs of kWT staged in shared memory
// along the operand's contiguous direction.  C may alias C0.
__device__ inline void tile_gemm(MV C, MV C0, MV A, MV B, int M, int N, int K,
                          double sign, int r0, int c0) {
  __shared__ double As[kWT][kWT + 1];
  __shared__ double Bs[kWT][kWT + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < K; k0 += kWT) {
    const int kw = K - k0 < kWT ? K - k0 : kWT;
    for (int idx = tid; idx < kWT * kWT; idx += 256) {
      int i, kk;
      if (A.rs == 1) {
        i = idx % kWT;
        kk = idx / kWT;
      } else {
        kk = idx % kWT;
        i = idx / kWT;
      }
      As[kk][i] = (r0 + i < M && kk < kw) ? A.at(r0 + i, k0 + kk) : 0.0;
      int j;
      if (B.rs == 1) {
        kk = idx % kWT;
        j = idx / kWT;
      } else {
        j = idx % kWT;
        kk = idx / kWT;
      }
      Bs[kk][j] = (c0 + j < N && kk < kw) ? B.at(k0 + kk, c0 + j) : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < kw; ++kk) {
      const double a0 = As[kk][tx], a1 = As[kk][tx + 16];
      const double b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = r0 + tx + 16 * u, j = c0 + ty + 16 * v;
      if (i < M && j < N) C.at(i, j) = C0.at(i, j) + sign * acc[u][v];
    }
}

}  // namespace wide
}  // namespace skel
