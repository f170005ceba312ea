// Staged engine interface (kernels in qfs_staged.cu, plan and buffers owned by qfs_api.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace qfs {

struct StagedPlan {
  int grid;                 // persistent CTAs of the fedder, power and theta stages
  int sms;
  int64_t chunk;            // quartics per chunk (= the survivor capacity of the buffers)
  unsigned *counters;       // [0] survivors of the chunk, [1] work-queue head
  int *rows;                // chunk survivors -> row
  uint8_t *active;
  uint32_t *G;              // chunk x padded words of degree 4p(p-1)
  uint8_t *gA, *gB;         // chunk x C(4p-1,3) bytes each
  uint32_t *ws;             // grid x 2 x ws_words (chain ping-pong)
  size_t ws_words;
  unsigned long long *stats;
  uint32_t *status;
};

// Device bytes one survivor slot needs at prime p.
size_t staged_survivor_bytes(int p);
// Enqueues the stage sequence for n quartics over F_p on `st`.
cudaError_t staged_run(const StagedPlan &pl, int p, const uint8_t *coeffs, int8_t *heights, int64_t n, int max_h,
                       cudaStream_t st);
// Resident CTAs per SM of the heaviest stage at prime p.
cudaError_t staged_occupancy(int p, int *blocks);

}  // namespace qfs
