// Launcher of the mod-p matrix multiplication (qfs_matmul.cu), called by the C ABI in qfs_api.cu.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace qfs {

// scratch bytes qfs_matmul_mod needs for an (n x k) by (k x m) product
size_t matmul_scratch_bytes(int n, int m, int k);
// C = A B mod p (uint8 row-major, values in [0, p), 2 <= p <= 256); scratch: matmul_scratch_bytes(n, m, k) bytes
cudaError_t matmul_mod_launch(int p, int n, int m, int k, const uint8_t *A, const uint8_t *B, uint8_t *C,
                              uint8_t *scratch, cudaStream_t st);

}  // namespace qfs
