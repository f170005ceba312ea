// Launcher of the exact polynomial powering (qfs_polypow.cu), called by the C ABI in qfs_api.cu.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace qfs {

constexpr int kPolyPowMaxPrimes = 7;   // word-size NTT primes available (their product exceeds 2^215)
constexpr int kPolyPowLimbs = 8;       // 256-bit output coefficients

// primes needed to reconstruct coefficients up to sum^n exactly (sum = the sum of the input coefficients); 0 if
// sum^n does not fit the 256-bit output or needs more than kPolyPowMaxPrimes primes
int polypow_primes(uint64_t sum, int n);
// scratch words for powering a degree-d form to the n-th power with nprimes primes (d n <= 255)
size_t polypow_scratch_words(int d, int n, int nprimes);
// transform length and algorithmic device-memory bytes (reads + writes of every kernel) of one powering call
void polypow_plan(int d, int n, int nprimes, uint64_t *transform_len, uint64_t *bytes);
// out: C(d n + 3, 3) x kPolyPowLimbs words; coeffs_dev: C(d + 3, 3) words in device memory
cudaError_t polypow_launch(int d, int n, int nprimes, const uint32_t *coeffs_dev, uint32_t *out, uint32_t *scratch,
                           cudaStream_t st);

}  // namespace qfs
