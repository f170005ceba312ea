// qfs_int_peaks: measured issue rates of the integer multiply-add paths that bound the height kernels -- the
// denominators of their rooflines.  Each rate comes from a kernel of independent chains of one instruction kind
// (IMAD, IDP4A, mma.sync m16n8k32 s8), 8 CTAs of 256 threads per SM, timed with CUDA events after a warm-up.
#include <cuda_runtime.h>

#include "../../include/qfs.h"

namespace qfs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakIters = 4096;

// eight independent IMAD chains per thread: 8 x 16 MACs per iteration
__global__ void __launch_bounds__(kPeakThreads) peak_imad(int *out, int a, int b, int iters) {
  int x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (int)threadIdx.x + k;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  int s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// eight independent IDP4A chains per thread: 8 x 16 x 4 MACs per iteration
__global__ void __launch_bounds__(kPeakThreads) peak_dp4a(int *out, int a, int b, int iters) {
  int x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (int)threadIdx.x + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 16; ++j)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = __dp4a(a, b, x[k]);
    a ^= x[0];
  }
  int s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// four independent accumulator tiles per warp: 16 mma.sync m16n8k32 (4096 MACs each) per iteration
__global__ void __launch_bounds__(kPeakThreads) peak_mma_s8(int *out, int a, int b, int iters) {
  int c[4][4] = {};
  const int a0 = a ^ (int)threadIdx.x, a1 = a + 1, a2 = a + 2, a3 = a + 3, b0 = b ^ (int)threadIdx.x, b1 = b + 1;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        asm volatile(
            "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+r"(c[q][0]), "+r"(c[q][1]), "+r"(c[q][2]), "+r"(c[q][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  int s = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) s ^= c[q][0] ^ c[q][1] ^ c[q][2] ^ c[q][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace qfs

using namespace qfs;

extern "C" int qfs_int_peaks(double *macs_per_s, int *sms, int *max_clock_khz) {
  if (!macs_per_s) return QFS_ERR_NULL;
  int dev = 0, n_sm = 0, clk = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QFS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev) != cudaSuccess)
    return QFS_ERR_CUDA;
  if (sms) *sms = n_sm;
  if (max_clock_khz) *max_clock_khz = clk;
  const int blocks = 8 * n_sm;
  int *out = nullptr;
  if (cudaMalloc(&out, sizeof(int) * (size_t)blocks * kPeakThreads) != cudaSuccess) return QFS_ERR_NO_MEMORY;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = QFS_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = QFS_ERR_CUDA;
  using Kernel = void (*)(int *, int, int, int);
  const Kernel kernels[3] = {peak_imad, peak_dp4a, peak_mma_s8};
  // MACs one thread issues per loop iteration (an mma's 4096 MACs are shared by the warp's 32 threads)
  const double macs_per_thread_iter[3] = {8.0 * 16, 8.0 * 16 * 4, 16.0 * 4096 / 32};
  for (int k = 0; k < 3 && rc == QFS_OK; ++k) {
    double best = 0;
    for (int rep = 0; rep < 3 && rc == QFS_OK; ++rep) {
      kernels[k]<<<blocks, kPeakThreads>>>(out, 3, 5, kPeakIters / 16);   // warm-up
      if (cudaEventRecord(e0) != cudaSuccess) { rc = QFS_ERR_CUDA; break; }
      kernels[k]<<<blocks, kPeakThreads>>>(out, 3, 5, kPeakIters);
      if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess) {
        rc = QFS_ERR_CUDA;
        break;
      }
      float ms = 0;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0) { rc = QFS_ERR_CUDA; break; }
      const double rate = (double)blocks * kPeakThreads * kPeakIters * macs_per_thread_iter[k] / (ms * 1e-3);
      if (rate > best) best = rate;
    }
    macs_per_s[k] = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (cudaFree(out) != cudaSuccess && rc == QFS_OK) rc = QFS_ERR_CUDA;
  return rc;
}
