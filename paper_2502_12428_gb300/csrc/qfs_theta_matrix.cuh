// Launcher of the theta-matrix export (qfs_theta_matrix.cu), called by the C ABI in qfs_api.cu.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace qfs {

// n quartics (device, n x 35) -> n matrices M (device, n x ld x ld bytes).  ws: a workspace of
// workspace_words(n, stride) words; which: n device ints (scratch); status: the device status word.
cudaError_t theta_matrix_launch(int p, const uint8_t *coeffs, int n, uint8_t *M, uint32_t *ws, size_t stride,
                                int *which, uint32_t *status, cudaStream_t st);

}  // namespace qfs
