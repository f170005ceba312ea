// Exact powering of a homogeneous integer form in 4 variables (the paper's Sec. 4 polynomial-powering workload: a
// degree-16 form with coefficients in {0..4} raised to the powers 5 .. 15).
//
// Method (multimodular NTT, CRT):
//   1. Dehomogenise (x1 = 1) and pack by Kronecker substitution: the monomial x2^e2 x3^e3 x4^e4 goes to index
//      e2 + B e3 + B^2 e4 with B = d n + 1, so the product of packed vectors is the packed product (no digit of the
//      result exceeds d n < B).  The transform length N is the power of two >= B^3 (at most 2^24).
//   2. For each of P word-size primes q = c 2^24 + 1: reduce the coefficients mod q, forward transform
//      (Gentleman-Sande, natural order in, bit-reversed order out), raise every entry to the n-th power, inverse
//      transform (Cooley-Tukey, bit-reversed in, natural out), and gather the coefficients of the degree-d n output
//      monomials (times N^-1).
//   3. Chinese remaindering (Garner's mixed-radix form) of the P residues of every coefficient into a 256-bit
//      unsigned integer.  P is the smallest number of primes whose product exceeds the coefficient bound
//      (sum of |coefficients|)^n, so the result is exact.
// Modular products use Barrett reduction with mu = floor(2^64 / q).
#include <cuda_runtime.h>

#include <cstdint>

#include "qfs_layout.cuh"
#include "qfs_polypow.cuh"

namespace qfs {
namespace {

__device__ __forceinline__ uint32_t mulmod(uint32_t a, uint32_t b, uint32_t q, uint64_t mu) {
  const uint64_t x = (uint64_t)a * b;
  const uint64_t qh = __umul64hi(x, mu);
  uint64_t r = x - qh * q;
  if (r >= q) r -= q;
  return (uint32_t)r;
}
__device__ __forceinline__ uint32_t addmod(uint32_t a, uint32_t b, uint32_t q) {
  const uint32_t s = a + b;   // a, b < q < 2^31: no overflow
  return s >= q ? s - q : s;
}
__device__ __forceinline__ uint32_t submod(uint32_t a, uint32_t b, uint32_t q) { return a >= b ? a - b : a + q - b; }
__device__ __forceinline__ uint32_t powmod(uint32_t a, uint32_t e, uint32_t q, uint64_t mu) {
  uint32_t r = 1;
  while (e) {
    if (e & 1u) r = mulmod(r, a, q, mu);
    a = mulmod(a, a, q, mu);
    e >>= 1;
  }
  return r;
}

struct PrimeQ {
  uint32_t q;
  uint64_t mu;
};

// tw[k] = w^k, itw[k] = w^-k for k < N/2, with w a primitive N-th root of unity mod q
__global__ void twiddle_kernel(uint32_t *tw, uint32_t *itw, uint32_t half, uint32_t w, uint32_t wi, PrimeQ P) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < half; k += gridDim.x * blockDim.x) {
    tw[k] = powmod(w, k, P.q, P.mu);
    itw[k] = powmod(wi, k, P.q, P.mu);
  }
}

// a = 0, then the packed input reduced mod q
__global__ void zero_kernel(uint32_t *a, uint32_t N) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) a[i] = 0;
}
__global__ void scatter_kernel(const uint32_t *coeffs, int d, int B, uint32_t *a, PrimeQ P) {
  const int n_in = tet(d + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_in; i += gridDim.x * blockDim.x) {
    int u, s, t;
    decode_packed(i, u, s, t);
    // coefficient i belongs to the monomial with (u, s, t) = (e2+e3+e4, e3+e4, e4) in degree d
    const int e2 = u - s, e3 = s - t, e4 = t;
    a[(size_t)e2 + (size_t)B * e3 + (size_t)B * B * e4] = coeffs[i] % P.q;
  }
}

// one Gentleman-Sande stage (block length len, twiddle stride N / len): a[i0], a[i1] -> a[i0] + a[i1], (a[i0] - a[i1]) w^j
__global__ void dif_stage(uint32_t *a, uint32_t N, uint32_t half, uint32_t tstride, const uint32_t *tw, PrimeQ P) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < N / 2; t += gridDim.x * blockDim.x) {
    const uint32_t j = t & (half - 1), i0 = ((t - j) << 1) + j, i1 = i0 + half;
    const uint32_t u = a[i0], v = a[i1];
    a[i0] = addmod(u, v, P.q);
    a[i1] = mulmod(submod(u, v, P.q), tw[j * tstride], P.q, P.mu);
  }
}
// one Cooley-Tukey stage: a[i0], a[i1] -> a[i0] + a[i1] w^j, a[i0] - a[i1] w^j
__global__ void dit_stage(uint32_t *a, uint32_t N, uint32_t half, uint32_t tstride, const uint32_t *tw, PrimeQ P) {
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < N / 2; t += gridDim.x * blockDim.x) {
    const uint32_t j = t & (half - 1), i0 = ((t - j) << 1) + j, i1 = i0 + half;
    const uint32_t u = a[i0], v = mulmod(a[i1], tw[j * tstride], P.q, P.mu);
    a[i0] = addmod(u, v, P.q);
    a[i1] = submod(u, v, P.q);
  }
}
__global__ void pow_kernel(uint32_t *a, uint32_t N, uint32_t n, PrimeQ P) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    a[i] = powmod(a[i], n, P.q, P.mu);
}
// residue of every output coefficient (packed descending lex, degree D = d n), times N^-1
__global__ void gather_kernel(const uint32_t *a, int D, int B, uint32_t ninv, uint32_t *res, PrimeQ P) {
  const int n_out = tet(D + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_out; i += gridDim.x * blockDim.x) {
    int u, s, t;
    decode_packed(i, u, s, t);
    const size_t idx = (size_t)(u - s) + (size_t)B * (s - t) + (size_t)B * B * t;
    res[i] = mulmod(a[idx], ninv, P.q, P.mu);
  }
}

struct CrtParams {
  uint32_t q[kPolyPowMaxPrimes];
  uint64_t mu[kPolyPowMaxPrimes];
  uint32_t inv[kPolyPowMaxPrimes][kPolyPowMaxPrimes];   // inv[j][k] = q_k^-1 mod q_j (k < j)
  int nprimes;
};

// Garner: v_j = (...((r_j - v_0) q_0^-1 - v_1) q_1^-1 ... - v_{j-1}) q_{j-1}^-1 mod q_j; then
// X = v_0 + q_0 (v_1 + q_1 (v_2 + ...)) in 8 little-endian 32-bit limbs
__global__ void crt_kernel(const uint32_t *res, int n_out, CrtParams C, uint32_t *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_out; i += gridDim.x * blockDim.x) {
    uint32_t v[kPolyPowMaxPrimes];
    for (int j = 0; j < C.nprimes; ++j) {
      uint32_t t = res[(size_t)j * n_out + i];
      for (int k = 0; k < j; ++k) t = mulmod(submod(t, v[k] % C.q[j], C.q[j]), C.inv[j][k], C.q[j], C.mu[j]);
      v[j] = t;
    }
    uint32_t x[kPolyPowLimbs];
    for (int l = 0; l < kPolyPowLimbs; ++l) x[l] = 0;
    for (int j = C.nprimes - 1; j >= 0; --j) {
      // x = x * q_j + v_j
      uint64_t carry = v[j];
      for (int l = 0; l < kPolyPowLimbs; ++l) {
        const uint64_t y = (uint64_t)x[l] * C.q[j] + carry;
        x[l] = (uint32_t)y;
        carry = y >> 32;
      }
    }
    for (int l = 0; l < kPolyPowLimbs; ++l) out[(size_t)i * kPolyPowLimbs + l] = x[l];
  }
}

// primes q = c 2^24 + 1 below 2^31 (largest first) and a primitive root of each
constexpr uint32_t kQ[kPolyPowMaxPrimes] = {2130706433u, 2113929217u, 2013265921u, 1811939329u,
                                            1711276033u, 1224736769u, 1107296257u};
constexpr uint32_t kRoot[kPolyPowMaxPrimes] = {3u, 5u, 31u, 13u, 29u, 3u, 10u};

uint64_t host_mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((unsigned __int128)a * b % q); }
uint64_t host_powmod(uint64_t a, uint64_t e, uint64_t q) {
  uint64_t r = 1;
  a %= q;
  while (e) {
    if (e & 1) r = host_mulmod(r, a, q);
    a = host_mulmod(a, a, q);
    e >>= 1;
  }
  return r;
}
// floor(2^64 / q) for 2 <= q < 2^32
uint64_t barrett_mu(uint32_t q) { return (uint64_t)(((unsigned __int128)1 << 64) / q); }

}  // namespace

int polypow_primes(double log2_bound) {
  double acc = 0;
  for (int j = 0; j < kPolyPowMaxPrimes; ++j) {
    acc += 30.0;   // every prime exceeds 2^30
    if (acc > log2_bound + 1.0) return j + 1;
  }
  return 0;
}

size_t polypow_scratch_words(int d, int n, int nprimes) {
  const int B = d * n + 1;
  uint32_t N = 1;
  while ((uint64_t)N < (uint64_t)B * B * B) N <<= 1;
  return (size_t)N + (size_t)N + (size_t)nprimes * tet(d * n + 1) + tet(d + 1) + 64;
}

cudaError_t polypow_launch(int d, int n, int nprimes, const uint32_t *coeffs_dev, uint32_t *out, uint32_t *scratch,
                           cudaStream_t st) {
  const int B = d * n + 1, D = d * n;
  uint32_t N = 1;
  while ((uint64_t)N < (uint64_t)B * B * B) N <<= 1;
  const int n_out = tet(D + 1);
  uint32_t *a = scratch;
  uint32_t *tw = a + N, *itw = tw + N / 2;
  uint32_t *res = itw + N / 2;
  const int grid = 152 * 8, block = 256;
  CrtParams C;
  C.nprimes = nprimes;
  for (int j = 0; j < nprimes; ++j) {
    const uint32_t q = kQ[j];
    PrimeQ P{q, barrett_mu(q)};
    C.q[j] = q;
    C.mu[j] = P.mu;
    for (int k = 0; k < kPolyPowMaxPrimes; ++k) C.inv[j][k] = k < j ? (uint32_t)host_powmod(kQ[k] % q, q - 2, q) : 0u;
    const uint32_t w = (uint32_t)host_powmod(kRoot[j], (q - 1) / N, q);   // primitive N-th root
    const uint32_t wi = (uint32_t)host_powmod(w, q - 2, q);
    const uint32_t ninv = (uint32_t)host_powmod(N, q - 2, q);
    twiddle_kernel<<<grid, block, 0, st>>>(tw, itw, N / 2, w, wi, P);
    zero_kernel<<<grid, block, 0, st>>>(a, N);
    scatter_kernel<<<64, block, 0, st>>>(coeffs_dev, d, B, a, P);
    for (uint32_t len = N; len >= 2; len >>= 1) dif_stage<<<grid, block, 0, st>>>(a, N, len / 2, N / len, tw, P);
    pow_kernel<<<grid, block, 0, st>>>(a, N, (uint32_t)n, P);
    for (uint32_t len = 2; len <= N; len <<= 1) dit_stage<<<grid, block, 0, st>>>(a, N, len / 2, N / len, itw, P);
    gather_kernel<<<grid, block, 0, st>>>(a, D, B, ninv, res + (size_t)j * n_out, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  crt_kernel<<<grid, block, 0, st>>>(res, n_out, C, out);
  return cudaGetLastError();
}

}  // namespace qfs
