// Definitions shared by the per-quartic pipeline (qfs_engine.cuh) and the swept chain product (qfs_sweep.cuh):
// block size, device status bits, debug outputs and the static part of the shared memory.
#pragma once
#include <cstddef>
#include <cstdint>
#include "qfs_layout.cuh"

namespace qfs {

constexpr int kThreads = 256;
constexpr int kMaxUparDecl = 8;

// Workspace buffers.  Every buffer a chain product reads from is preceded by kGuardWords zero words (the swept
// product reads columns that do not exist from there).  A launch's workspace holds, per CTA, two buffers of
// workspace_stride_words(p) words each, and starts with one guard: buffer k of CTA b begins at word
// kGuardWords + (2b + k) * stride, and its guard is the last kGuardWords words of the stride before it, which
// nothing in the buffer reaches (its contents use at most stride - kGuardWords words).  Each CTA clears
// its two guards when it starts, since an earlier launch with another stride may have left data there.  A buffer
// holds either a padded form of degree up to 4p(p-1) or theta's guarded copy of Delta, which is larger.
constexpr int kGuardWords = 4;
size_t workspace_stride_words(int p);   // qfs_engine.cuh: the larger of a padded degree-D form and theta's copy
inline size_t workspace_words(int64_t ctas, size_t stride) { return kGuardWords + 2 * (size_t)ctas * stride; }

#if defined(__CUDACC__)
__device__ __forceinline__ void cta_buffers(uint32_t *ws, size_t stride, uint32_t *&bufA, uint32_t *&bufB) {
  bufA = ws + kGuardWords + (size_t)blockIdx.x * 2 * stride;
  bufB = bufA + stride;
  if (threadIdx.x < 2 * kGuardWords)
    (threadIdx.x < kGuardWords ? bufA : bufB)[(int)(threadIdx.x % kGuardWords) - kGuardWords] = 0u;
}
#endif

// Status bits (atomicOr into the device status word).
constexpr uint32_t kStatusInexactDivision = 1u;
constexpr uint32_t kStatusTheta = 2u;

struct DebugPtrs {
  uint32_t *G;        // padded, degree D: raw G (mod p^2) before the Delta_1 epilogue
  uint32_t *delta;    // padded, degree D: Delta (mod p)
  int32_t *g;         // packed, ld values
  int32_t *iters;     // packed, (max_h-1) x ld
};

struct Smem {
  int SW[kSWLen];
  int taps[35];           // coefficients of f, packed order (index tet(uI) + tri(sI) + tI)
  uint32_t tapword[15];   // dp4a tap words per (uI, sI) pair: byte k = a(uI, sI, 3-k)
  uint32_t pair_mask;     // bit tri(uI)+sI set iff that pair has a nonzero tap
  int dense_min;          // nonzero tap pairs from which the swept chain runs every pair (the two-slice loop)
  int powp[kMaxP];        // c^p mod p^2
  int slot_tab[2][kMaxUparDecl + 4];  // ring word offsets of the slices a chain round reads (double buffered)
  uint16_t chunk_tab[32 * 40];        // chain block: flat chunk index -> (column - s0) << 8 | chunk
  int tile_round, tile_ring;          // chain tile configuration of the current quartic's prime
  int64_t item;
  int flag;
  int task_next;   // swept chain: next task of the current product (work queue shared by the CTA's warps)
  int task_done;   // swept chain: warps that found the queue empty; the last one resets both counters
  // followed in dynamic shared memory by two byte arrays of ld entries: g (current iterate) and g_next
};

// Dynamic shared memory layout: [Smem][g: ld][g_next: ld][pad to 16 B][chain ring].
__host__ __device__ constexpr size_t ring_offset_for(int max_ld) {
  return (sizeof(Smem) + 2 * (size_t)max_ld + 15) & ~(size_t)15;
}

}  // namespace qfs
