// Arithmetic peaks of the device, measured: the denominators of the
// roofline fractions that the ALU-bound kernels (pair sums, CPQR,
// elimination) report.  A kernel keeps every SM busy with independent FMA
// chains (8 per thread, 8 CTAs of 256 threads per SM) and is timed with
// CUDA events after a warm-up launch.  Not part of the method.
#include "skel_internal.h"

namespace skel {

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_fma_chains(T *out, int iters, T b,
                                                    T c, int sink) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (sink == 12345) out[threadIdx.x] = s;  // never true; keeps the chains
}

// FMA throughput in TFLOP/s (2 flops per FMA)
template <class T>
double measure(int sms, int iters, T *dummy, cudaError_t &err) {
  const int blocks = sms * 8;
  const T b = (T)0.999999, c = (T)1e-7;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  double tf = 0.0;
  if (err == cudaSuccess) {
    k_fma_chains<T><<<blocks, 256>>>(dummy, iters / 8, b, c, 0);  // warm-up
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, 256>>>(dummy, iters, b, c, 0);
    cudaEventRecord(e1);
    note_launches(2);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    const double fmas = (double)blocks * 256 * 8 * 16 * (double)iters;
    if (err == cudaSuccess && ms > 0.f) tf = 2.0 * fmas / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return tf;
}

}  // namespace

}  // namespace skel

extern "C" int skel_measure_alu_peaks(double *out) {
  if (!out) return SKEL_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
          cudaSuccess)
    return SKEL_ECUDA;
  void *dummy = nullptr;
  if (skel::dev_alloc(&dummy, 256 * sizeof(double)) != cudaSuccess)
    return SKEL_ENOMEM;
  cudaError_t err = cudaSuccess;
  // about 50 ms each on a GB300 (FP64 ~1.2, FP32 ~70 TFLOP/s)
  out[0] = skel::measure<double>(sms, 1500, static_cast<double *>(dummy), err);
  if (err == cudaSuccess)
    out[1] = skel::measure<float>(sms, 90000, static_cast<float *>(dummy), err);
  skel::dev_free(dummy);
  return err == cudaSuccess ? SKEL_OK : SKEL_ECUDA;
}
