// Launcher of the height-1 screen (qfs_screen.cu), called by the C ABI in qfs_api.cu before the persistent launch.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "qfs_engine.cuh"

namespace qfs {

// Every row of every group of prm: heights = -1 where a coefficient is >= p, 1 where the height-1 test holds;
// the other rows are appended (as launch items) to list, with their count in *n_list (zeroed by the caller).
// grid_ctas: CTAs of kScreenThreads threads (one warp per row at a time).
constexpr int kScreenThreads = 256;
cudaError_t screen_launch(const FusedParams &prm, int max_p, int64_t *list, unsigned long long *n_list,
                          int grid_ctas, cudaStream_t st);

// Dynamic shared memory of one screen CTA for primes up to max_p.
size_t screen_smem_bytes(int max_p);

}  // namespace qfs
