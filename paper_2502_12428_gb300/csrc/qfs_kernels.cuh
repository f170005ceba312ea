// Kernel entry points of one arithmetic form (instantiated once per form in its own translation unit).
#pragma once
#include <cuda_runtime.h>
#include "qfs_engine.cuh"

namespace qfs {

// Resident CTAs per SM the register allocation is bounded for: the swept chain (dp4a and int32 forms) keeps five
// accumulator sets per lane and gets 128 registers (2 CTAs of 256 threads); the int8 tensor form gets 85 (3 CTAs).
template <int FORM>
constexpr int min_ctas_per_sm() { return FORM == 2 ? 3 : 2; }
// Persistent launch: every CTA pulls quartics from a global atomic queue until the queue is empty.
template <int FORM>
__global__ void __launch_bounds__(kThreads, min_ctas_per_sm<FORM>()) fused_kernel(FusedParams prm) {
  fused_body<FORM, false>(prm);
}
// The same for int8 tensor form launches whose primes are all <= 5: 85 registers, three CTAs per SM.
template <int FORM>
__global__ void __launch_bounds__(kThreads, 3) fused_kernel_small(FusedParams prm) {
  fused_body<FORM, true>(prm);
}

// One quartic with every intermediate array written out (kernel-level parity hook).
template <int P, int FORM>
__global__ void __launch_bounds__(kThreads) debug_kernel(const uint8_t *f, int max_h, int8_t *h_out, uint32_t *bufA,
                                                         uint32_t *bufB, uint32_t *status, DebugPtrs dbg,
                                                         int power_mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  uint8_t *gs = smem_raw + sizeof(Smem);
  uint8_t *gn = gs + Prime<P>::ld;
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem_raw + ring_offset_for(Prime<P>::ld));
  build_sw(sm.SW, Prime<P>::D + 2);
  init_task_queue(sm);
  if (threadIdx.x == 0) {
    sm.tile_round = default_tile(P).round_chunks;
    sm.tile_ring = default_tile(P).ring_words;
    sm.dense_min = kDefaultDenseMin;
  }
  __syncthreads();
  int steps = 0;
  const int h = process_quartic<P, FORM, true>(f, max_h, sm, gs, gn, ring, bufA, bufB, status, dbg, steps, power_mode);
  if (threadIdx.x == 0) *h_out = (int8_t)h;
}

// Host-side launchers (defined in qfs_form_<name>.cu).
template <int FORM>
struct FormLauncher {
  static cudaError_t fused(const FusedParams &prm, int grid, size_t smem, cudaStream_t st, bool small);
  static cudaError_t occupancy(int *blocks_per_sm, size_t smem, bool small);
  static cudaError_t debug(int p, const uint8_t *f, int max_h, int8_t *h_out, uint32_t *bufA, uint32_t *bufB,
                           uint32_t *status, DebugPtrs dbg, cudaStream_t st, int power_mode);
};

#define QFS_DEBUG_LAUNCH(PP, FORM)                                                                            \
  e = cudaFuncSetAttribute(debug_kernel<PP, FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
  if (e == cudaSuccess) debug_kernel<PP, FORM><<<1, kThreads, smem, st>>>(f, max_h, h_out, bufA, bufB, status, dbg, power_mode)

#define QFS_DEFINE_FORM_LAUNCHER(FORM)                                                                        \
  template <>                                                                                                 \
  cudaError_t FormLauncher<FORM>::fused(const FusedParams &prm, int grid, size_t smem, cudaStream_t st,      \
                                        bool small) {                                                         \
    auto k = small ? fused_kernel_small<FORM> : fused_kernel<FORM>;                                           \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
    if (e != cudaSuccess) return e;                                                                           \
    k<<<grid, kThreads, smem, st>>>(prm);                                                                     \
    return cudaGetLastError();                                                                                \
  }                                                                                                           \
  template <>                                                                                                 \
  cudaError_t FormLauncher<FORM>::occupancy(int *blocks_per_sm, size_t smem, bool small) {                    \
    auto k = small ? fused_kernel_small<FORM> : fused_kernel<FORM>;                                           \
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);          \
    if (e != cudaSuccess) return e;                                                                           \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, kThreads, smem);                   \
  }

#define QFS_DEFINE_DEBUG_LAUNCHER(FORM)                                                                       \
  template <>                                                                                                 \
  cudaError_t FormLauncher<FORM>::debug(int p, const uint8_t *f, int max_h, int8_t *h_out, uint32_t *bufA,    \
                                        uint32_t *bufB, uint32_t *status, DebugPtrs dbg, cudaStream_t st,     \
                                        int power_mode) {                                                     \
    const size_t smem = smem_bytes_for(p, uses_ring_chain(FORM, p));                                         \
    cudaError_t e = cudaSuccess;                                                                              \
    switch (p) {                                                                                              \
      case 3: QFS_DEBUG_LAUNCH(3, FORM); break;                                                               \
      case 5: QFS_DEBUG_LAUNCH(5, FORM); break;                                                               \
      case 7: QFS_DEBUG_LAUNCH(7, FORM); break;                                                               \
      case 11: QFS_DEBUG_LAUNCH(11, FORM); break;                                                             \
      default: QFS_DEBUG_LAUNCH(13, FORM); break;                                                             \
    }                                                                                                         \
    if (e != cudaSuccess) return e;                                                                           \
    return cudaGetLastError();                                                                                \
  }

}  // namespace qfs
