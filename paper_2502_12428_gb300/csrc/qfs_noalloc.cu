// qfs_heights_noalloc: the fused height launch with its scratch memory in a fixed, library-owned device array,
// for callers that cannot allocate device memory at call time.
//
// Who needs it: code that runs while a stream is being captured in global capture mode (cudaMalloc is then an
// illegal call that invalidates the capture), code whose device memory is handed out up front by another
// allocator (a framework's caching pool that owns the device), and code that must not stall the device
// (cudaFree synchronises it).  qfs_heights may grow its workspace with cudaMalloc/cudaFree on a call; this entry
// point never does.  It only uses the array below, which the CUDA runtime sets aside for every GPU that loads
// the library and keeps until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/qfs.h"
#include "qfs_kernels.cuh"

namespace qfs {
namespace {

// Fixed scratch per device: 64 MiB.  Bytes [0, 256) are the control block: the work-queue counter at 0 (cleared
// by every call), the device check word at 8 and the two work counters at 16 (both accumulate across calls until
// qfs_read_status / qfs_read_stats take and clear them); the rest holds the two ping-pong buffers of every
// persistent CTA.
constexpr size_t kScratchBytes = size_t(64) << 20;
constexpr size_t kControlBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The fused persistent kernel (dp4a form), given its workspace in the fixed array instead of a cudaMalloc'd one.
__global__ void __launch_bounds__(kThreads, 2) noalloc_fused_kernel(FusedParams prm) { fused_body<1, false>(prm); }

constexpr int kMaxDev = 64;
void *g_scratch_addr[kMaxDev];   // device address of g_noalloc_scratch on each device, set once
std::mutex g_noalloc_mu;

// The device address of the array for the current device.  The array's name in host code is only a host-side
// stand-in, so the real address comes from cudaGetSymbolAddress, once per device, with that device current.
// *fresh is set on the call that looked the address up (the first on this device).
int scratch_for_current_device(void **out, int *sms, bool *fresh) {
  *fresh = false;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return QFS_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDev) return QFS_ERR_DEVICE;
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return QFS_ERR_CUDA;
  if (major != 10 || minor != 3) return QFS_ERR_DEVICE;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return QFS_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
    *fresh = true;
  }
  *out = g_scratch_addr[dev];
  return QFS_OK;
}

}  // namespace

// Reads and clears the check word (status != nullptr) or the two work counters (stats != nullptr) that calls of
// qfs_heights_noalloc on the current device have accumulated; reports zeros if no call has set the array up on
// this device.  qfs_read_status and qfs_read_stats add these to their own words.  Synchronous (the caller has
// synchronised the device).
int noalloc_take_counters(uint32_t *status, unsigned long long *stats) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return QFS_ERR_CUDA;
  if (status) *status = 0;
  if (stats) stats[0] = stats[1] = 0;
  if (dev < 0 || dev >= kMaxDev) return QFS_OK;
  void *ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    ptr = g_scratch_addr[dev];
  }
  if (!ptr) return QFS_OK;
  unsigned char *base = static_cast<unsigned char *>(ptr);
  if (status) {
    if (cudaMemcpy(status, base + 8, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return QFS_ERR_CUDA;
    if (cudaMemset(base + 8, 0, 4) != cudaSuccess) return QFS_ERR_CUDA;
  }
  if (stats) {
    if (cudaMemcpy(stats, base + 16, 16, cudaMemcpyDeviceToHost) != cudaSuccess) return QFS_ERR_CUDA;
    if (cudaMemset(base + 16, 0, 16) != cudaSuccess) return QFS_ERR_CUDA;
  }
  // the clears are complete before a later call on any stream can add to the words
  return cudaDeviceSynchronize() == cudaSuccess ? QFS_OK : QFS_ERR_CUDA;
}

}  // namespace qfs

using namespace qfs;

extern "C" int qfs_heights_noalloc(int p, int64_t n, const uint8_t *coeffs, int max_h, int8_t *heights_out,
                                   cudaStream_t stream) {
  if (!(p == 3 || p == 5 || p == 7 || p == 11 || p == 13)) return QFS_ERR_INVALID_P;
  if (max_h < 1 || max_h > 10) return QFS_ERR_INVALID_MAX_H;
  if (n < 0) return QFS_ERR_INVALID_N;
  if (n > 0 && (!coeffs || !heights_out)) return QFS_ERR_NULL;
  if (n == 0) return QFS_OK;

  // Size check first: one persistent CTA needs two buffers that hold a form of degree 4p(p-1).
  const size_t ws_words = workspace_stride_words(p);
  const size_t per_cta = 2 * ws_words * sizeof(uint32_t);
  const size_t fit = (kScratchBytes - kControlBytes - kGuardWords * sizeof(uint32_t)) / per_cta;
  if (fit < 1) return QFS_ERR_NO_MEMORY;  // p = 13 needs more than the fixed 64 MiB for a single CTA

  void *scratch = nullptr;
  int sms = 0;
  bool fresh = false;
  int rc = scratch_for_current_device(&scratch, &sms, &fresh);
  if (rc) return rc;

  const size_t smem = smem_bytes_for(p, uses_ring_chain(QFS_FORM_DP4A, p));
  cudaError_t e = cudaFuncSetAttribute(noalloc_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return QFS_ERR_CUDA;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_fused_kernel, kThreads, smem);
  if (e != cudaSuccess) return QFS_ERR_CUDA;
  int64_t grid = (int64_t)sms * std::max(1, per_sm);
  grid = std::min<int64_t>(grid, (int64_t)fit);
  grid = std::min<int64_t>(grid, n);

  unsigned char *base = static_cast<unsigned char *>(scratch);
  FusedParams prm;
  memset(&prm, 0, sizeof(prm));
  prm.g[0].p = p;
  prm.g[0].n = n;
  prm.g[0].coeffs = coeffs;
  prm.g[0].heights = heights_out;
  prm.g[0].item_begin = 0;
  prm.g[0].tile_round = default_tile(p).round_chunks;
  prm.g[0].tile_ring = default_tile(p).ring_words;
  prm.g[0].dense_min = kDefaultDenseMin;
  prm.n_groups = 1;
  prm.n_items = n;
  prm.max_h = max_h;
  prm.sw_len = 4 * p * (p - 1) + 2;
  prm.counter = reinterpret_cast<unsigned long long *>(base);
  prm.status = reinterpret_cast<uint32_t *>(base + 8);
  prm.stats = reinterpret_cast<unsigned long long *>(base + 16);
  prm.ws = reinterpret_cast<uint32_t *>(base + kControlBytes);
  prm.ws_words = ws_words;
  prm.power_mode = QFS_POWER_CHAIN;
  // The array keeps whatever the previous call left.  Only the work-queue counter must start at zero; the check
  // word and the work counters accumulate until qfs_read_status / qfs_read_stats take them.  The chain buffers
  // need no clearing: every word a CTA reads is written earlier in the same quartic.
  // (the first call on a device clears the whole control block)
  e = cudaMemsetAsync(base, 0, fresh ? kControlBytes : 8, stream);
  if (e != cudaSuccess) return QFS_ERR_CUDA;
  noalloc_fused_kernel<<<(int)grid, kThreads, smem, stream>>>(prm);
  e = cudaGetLastError();
  return e == cudaSuccess ? QFS_OK : QFS_ERR_CUDA;
}
