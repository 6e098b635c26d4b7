// Split-precision (3xTF32) GEMM on the 5th-generation tensor cores.
//
// C = C0 + sign * A B for FP64 operands given as strided views: every
// operand entry is rounded to FP32 and split into a TF32 head and a TF32
// tail (a = a_hi + a_lo); the products a_hi b_hi + a_hi b_lo + a_lo b_hi
// are accumulated in FP32 by tcgen05.mma kind::tf32 into tensor memory,
// which gives about FP32 accuracy (the a_lo b_lo term is below FP32
// rounding) at tensor-core rate.  Used for the Schur-complement and
// interpolation products of Eq. (tmat) / Eq. (schurmat) of large boxes in
// the mixed-precision form, where the factorization is a preconditioner
// at ID tolerance 1e-6.
//
// One CTA of 128 threads per 128 x 128 output tile (UMMA M = 128,
// N = 128).  Per K slab of 32: all threads load the FP64 slab of A (128 x
// 32) and of B (32 x 128), split it and store the four TF32 tiles in
// shared memory in the canonical K-major layout without swizzle (core
// matrices of 8 rows x 16 bytes); then one thread issues 3 x 4 MMAs of
// K = 8 and commits them to an mbarrier that every thread waits on before
// the slab's shared memory is reused.  The epilogue reads the FP32
// accumulators from tensor memory (warp w: lanes 32w..32w+31 = rows) with
// tcgen05.ld and writes C in FP64.  Every wait has an iteration limit:
// on timeout the kernel records an error, waits once more (bounded) for
// its MMAs, frees its tensor memory and returns.
#include <cstdint>

#include "skel_internal.h"

namespace skel {

namespace {

constexpr int kTM = 128, kTN = 128, kTK = 32;  // tile and K slab
constexpr int kTThreads = 128;
// bytes of one TF32 tile of 128 rows x 32 k: 16 row groups x 8 k groups
// of core matrices (8 rows x 16 bytes)
constexpr uint32_t kTileBytes = kTM * kTK * 4;
constexpr uint32_t kLBO = 128;               // next core matrix along K
constexpr uint32_t kSBO = (kTK / 4) * 128;   // next 8-row group
// a wait gives up after this many nanoseconds of the global timer
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// canonical K-major, no-swizzle position of (row, k) in a tile (bytes)
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(row >> 3) * kSBO + (uint32_t)(k >> 2) * kLBO +
         (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

// shared-memory matrix descriptor (Blackwell): start address, leading and
// stride byte offsets (all >> 4), version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B,
// both K-major, N = 128, M = 128
__host__ __device__ constexpr uint32_t tf32_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
         ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ float tf32_head(float x) {
  // round to the 10-bit mantissa of TF32 (nearest, ties away from zero)
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// wait for the mbarrier phase to complete; each try_wait suspends for at
// most 100 us, and the whole wait for at most kWaitLimitNs
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(100000u)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}

}  // namespace

__global__ void __launch_bounds__(kTThreads)
k_tc_gemm(const TcJob *job_p, int *err) {
  const TcJob job = *job_p;
  const int r0 = blockIdx.x * kTM, c0 = blockIdx.y * kTN;
  if (r0 >= job.M || c0 >= job.N || job.M <= 0 || job.N <= 0) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned start for the tiles
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) &
                                          ~(uintptr_t)1023);
  unsigned char *a_hi = smem, *a_lo = smem + kTileBytes,
                *b_hi = smem + 2 * kTileBytes, *b_lo = smem + 3 * kTileBytes;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t bar = smem_u32(&mbar);
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
        :
        : "r"(smem_u32(&tmem_slot)), "r"(kTN)
        : "memory");
    asm volatile(
        "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::
            : "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tf32_idesc();
  uint32_t phase = 0;
  bool ok = true;
  const int nslab = (job.K + kTK - 1) / kTK;
  for (int sl = 0; sl < nslab && ok; ++sl) {
    const int k0 = sl * kTK;
    // A slab: 128 rows x 32 k; B slab: 32 k x 128 columns, stored N x K
    for (int idx = tid; idx < kTM * kTK; idx += kTThreads) {
      int row, k;
      if (job.A.rs == 1) {
        row = idx % kTM;
        k = idx / kTM;
      } else {
        k = idx % kTK;
        row = idx / kTK;
      }
      double v = 0.0;
      if (r0 + row < job.M && k0 + k < job.K)
        v = job.A.p[(int64_t)(r0 + row) * job.A.rs +
                    (int64_t)(k0 + k) * job.A.cs];
      const float f = (float)v, h = tf32_head(f);
      const uint32_t o = tile_off(row, k);
      *(float *)(a_hi + o) = h;
      *(float *)(a_lo + o) = f - h;
      int col;
      if (job.B.rs == 1) {
        k = idx % kTK;
        col = idx / kTK;
      } else {
        col = idx % kTN;
        k = idx / kTN;
      }
      double w = 0.0;
      if (c0 + col < job.N && k0 + k < job.K)
        w = job.B.p[(int64_t)(k0 + k) * job.B.rs +
                    (int64_t)(c0 + col) * job.B.cs];
      const float g = (float)w, gh = tf32_head(g);
      const uint32_t ob = tile_off(col, k);
      *(float *)(b_hi + ob) = gh;
      *(float *)(b_lo + ob) = g - gh;
    }
    // the generic-proxy stores become visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo),
                     bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const uint32_t a = t == 2 ? al : ah, b = t == 1 ? bl : bh;
#pragma unroll
        for (int kk = 0; kk < kTK / 8; ++kk) {
          // K = 8 per instruction: two core matrices along K
          const uint64_t ad = smem_desc(a + kk * 2 * kLBO);
          const uint64_t bd = smem_desc(b + kk * 2 * kLBO);
          const uint32_t acc = (sl > 0 || t > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
              "}\n"
              :
              : "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster"
          ".b64 [%0];\n" ::"r"(bar)
          : "memory");
    }
    if (!mbar_wait(bar, phase)) {
      ok = false;
      if (tid == 0) atomicMin(err, SKEL_ETIMEOUT);
    }
    phase ^= 1u;
  }
  if (!ok) {
    // give the MMAs in flight one more bounded wait before freeing
    (void)mbar_wait(bar, phase ^ 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok) {
    // epilogue: warp w reads rows 32w..32w+31, 32 columns at a time
    const int row = r0 + 32 * warp + lane;
    for (int cc = 0; cc < kTN; cc += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, "
          "%6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, "
          "%20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
          "[%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]),
            "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]),
            "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
            "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
            "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < job.M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = c0 + cc + j;
          if (col < job.N) {
            const double acc = (double)__uint_as_float(v[j]);
            const double base =
                job.C0.p[(int64_t)row * job.C0.rs + (int64_t)col * job.C0.cs];
            job.C[(int64_t)row * job.c_rs + (int64_t)col * job.c_cs] =
                base + job.sign * acc;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile(
        "tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
        "r"(kTN)
        : "memory");
}

static size_t tc_gemm_smem() { return 4 * (size_t)kTileBytes + 1024; }

cudaError_t launch_tc_gemm(const TcJob *job, int max_m, int max_n, int *err,
                           cudaStream_t s) {
  if (max_m <= 0 || max_n <= 0) return cudaSuccess;
  const size_t sm = tc_gemm_smem();
  cudaError_t e = cudaFuncSetAttribute(
      k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((max_m + kTM - 1) / kTM),
            (unsigned)((max_n + kTN - 1) / kTN));
  k_tc_gemm<<<grid, kTThreads, sm, s>>>(job, err);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace skel

// C = C - A B (column-major FP64, lda >= M, ldb >= K, ldc >= M) on the
// tensor cores in 3xTF32; the building block of the mixed form's
// large-box products, exposed for its parity test.
extern "C" int skel_gemm_tf32x3(int32_t M, int32_t N, int32_t K,
                                const double *A, int64_t lda,
                                const double *B, int64_t ldb, double *C,
                                int64_t ldc, void *stream) {
  if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!C || ldc < M)) ||
      (M > 0 && N > 0 && K > 0 && (!A || !B || lda < M || ldb < K)))
    return SKEL_EINVAL;
  if (M == 0 || N == 0) return SKEL_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  skel::TcJob job{};
  job.A = {A, 1, lda};
  job.B = {B, 1, ldb};
  job.C0 = {C, 1, ldc};
  job.C = C;
  job.c_rs = 1;
  job.c_cs = ldc;
  job.M = M;
  job.N = N;
  job.K = K;
  job.sign = -1.0;
  void *mem = nullptr;
  if (skel::dev_alloc(&mem, sizeof(skel::TcJob) + 16) != cudaSuccess)
    return SKEL_ENOMEM;
  skel::TcJob *dj = static_cast<skel::TcJob *>(mem);
  int *derr = reinterpret_cast<int *>(dj + 1);
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(dj, &job, sizeof job,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), s);
  if (e == cudaSuccess) e = skel::launch_tc_gemm(dj, M, N, derr, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  skel::dev_free(mem);
  if (e != cudaSuccess) return SKEL_ECUDA;
  return herr != 0 ? herr : SKEL_OK;
}
