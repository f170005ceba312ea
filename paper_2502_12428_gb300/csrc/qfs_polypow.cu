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
//      monomials (times N^-1).  The transforms run in passes of up to 8 radix-2 stages (the four-step split of a
//      length-M transform into R-point transforms over columns of stride M / R, twiddles w_M^(c k) between
//      passes); inside a pass the stages run in registers in two groups with one exchange through shared memory
//      between them.  The last forward pass, the n-th powers and the first inverse pass share one kernel, so a
//      length-2^24 transform pair costs five round trips through device memory instead of 48.  Only the leading
//      rows of the first pass can hold input, so only they are cleared and read.
//   3. Chinese remaindering (Garner's mixed-radix form) of the P residues of every coefficient into a 256-bit
//      unsigned integer.  P is the smallest number of primes whose product exceeds the coefficient bound
//      (sum of |coefficients|)^n, so the result is exact.  The residues are gathered and recombined by rows of the
//      transform (contiguous reads), and each coefficient is written as one 32-byte record at its packed index.
// Modular products: Shoup's method (a precomputed floor(w 2^32 / q) for each fixed multiplier w) for the roots
// inside a pass, Montgomery products for the twiddles between passes and for the powers, Barrett reduction with
// mu = floor(2^64 / q) in the gather and the remaindering.  Every correction of a value below 2q is an unsigned
// minimum, min(x, x - q).
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
// Corrections as an unsigned minimum: for x < 2q, min(x, x - q) is x mod q (x - q wraps above x when x < q).
__device__ __forceinline__ uint32_t addmod(uint32_t a, uint32_t b, uint32_t q) {
  const uint32_t s = a + b;   // a, b < q < 2^31: no overflow
  return min(s, s - q);
}
// a - b mod q: d = a - b wraps to d + 2^32 when a < b, and then d + q (mod 2^32) = a - b + q is the smaller one
__device__ __forceinline__ uint32_t submod(uint32_t a, uint32_t b, uint32_t q) {
  const uint32_t d = a - b;
  return min(d, d + q);
}
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
  uint32_t qneg;   // -q^-1 mod 2^32 (Montgomery reduction)
  uint32_t rmod;   // 2^32 mod q: 1 in Montgomery form
  uint32_t r2;     // 2^64 mod q: converts into Montgomery form
};

// Montgomery product a b 2^-32 mod q for a, b < q < 2^31 (Montgomery's REDC): t + m q is divisible by 2^32 with
// m = t (-q^-1) mod 2^32, and (t + m q) / 2^32 < 2q
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, const PrimeQ &P) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t m = (uint32_t)t * P.qneg;
  const uint32_t u = (uint32_t)((t + (uint64_t)m * P.q) >> 32);
  return min(u, u - P.q);
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

// a w mod q for a < 2^32, w < q < 2^31, given ws = floor(w 2^32 / q) (Shoup): the quotient estimate
// floor(a ws / 2^32) is at most one below floor(a w / q), so a w - est q lies in [0, 2q)
__device__ __forceinline__ uint32_t shoup_mul(uint32_t a, uint32_t w, uint32_t ws, uint32_t q) {
  const uint32_t est = __umulhi(a, ws);
  const uint32_t r = a * w - est * q;
  return min(r, r - q);
}

// One power table of a batch: table[j] = base^(j step) for j < n, in Montgomery form (mont) or with Shoup
// companions comp[j].
struct TableJob {
  uint32_t *table, *comp;
  uint32_t n, base, step;
  int mont;
  PrimeQ P;
};
constexpr int kMaxTableJobs = 3 * 2 * kPolyPowMaxPrimes;
struct TableJobs {
  TableJob job[kMaxTableJobs];
};
// Every power table of every prime and direction in one launch: blockIdx.y selects the table.
__global__ void power_tables_kernel(TableJobs J) {
  const TableJob &T = J.job[blockIdx.y];
  const uint32_t b = powmod(T.base, T.step, T.P.q, T.P.mu);
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < T.n; j += gridDim.x * blockDim.x) {
    const uint32_t v = powmod(b, j, T.P.q, T.P.mu);
    if (T.mont) {
      T.table[j] = mulmod(v, T.P.rmod, T.P.q, T.P.mu);
    } else {
      T.table[j] = v;
      T.comp[j] = (uint32_t)(((uint64_t)v << 32) / T.P.q);
    }
  }
}

// Twiddle tables of one prime and direction: lo[j] = w^j (j < 4096), hi[j] = w^(4096 j) (j < max(1, N / 4096)),
// each with its Shoup companion, so that w^e = lo[e mod 4096] hi[e / 4096]; rt[j] = w_R^j (j < R / 2) for the
// R-point transforms inside a pass, R = min(256, N), also with companions.
struct TwTab {
  const uint32_t *lo, *los, *hi, *his, *rt, *rts;
};
constexpr int kTwLoBits = 12;
constexpr int kPassMaxStages = 8;
constexpr int kPassR = 1 << kPassMaxStages;   // longest column of a pass
constexpr int kPassCols = 32;                 // columns per block in the column passes
constexpr int kTileWords = kPassR * (kPassCols + 1);

// w^e in Montgomery form from the two-level tables (lo and hi hold Montgomery forms)
__device__ __forceinline__ uint32_t twiddle_mont(uint32_t e, const TwTab &T, const PrimeQ &P) {
  return mont_mul(__ldg(T.lo + (e & ((1u << kTwLoBits) - 1))), __ldg(T.hi + (e >> kTwLoBits)), P);
}

// The twiddles of a column pass's 32 columns in shared memory: for column cc with b = w_M^(c0 + cc),
// p1[cc][j] = b^j and p2[cc][j] = b^(16 j) (j < 16, Montgomery form), so that b^k = p1[k mod 16] p2[k / 16] for
// every frequency k < 256 of the column's R-point transform.  Threads 0 .. 63 build them; the caller synchronises.
__device__ __forceinline__ void column_twiddles(uint32_t (*p1)[16], uint32_t (*p2)[16], uint32_t c0, int lgs,
                                                const TwTab &T, const PrimeQ &P) {
  const int t = threadIdx.x;
  if (t < 2 * kPassCols) {
    const int cc = t & (kPassCols - 1);
    uint32_t b = twiddle_mont((c0 + cc) << lgs, T, P);   // w^((c0 + cc) N / M) = w_M^(c0 + cc)
    uint32_t (*dst)[16] = t < kPassCols ? p1 : p2;
    if (t >= kPassCols)
#pragma unroll
      for (int i = 0; i < 4; ++i) b = mont_mul(b, b, P);   // b^16
    uint32_t v = P.rmod;
    for (int j = 0; j < 16; ++j) {
      dst[cc][j] = v;
      v = mont_mul(v, b, P);
    }
  }
}

__device__ __forceinline__ uint32_t bitrev(uint32_t x, int bits) { return __brev(x) >> (32 - bits); }

// R-point DIF (natural in, bit-reversed out) on the columns of a shared tile: element m of column cc at
// tile[m * ld + cc], 2^lgcol columns, R = 2^kp; twiddles w_R^j from rt (a stage of length len uses w_R^(j R / len)).
// Stages run two at a time (radix 4: four elements j, j + L/4, j + L/2, j + 3L/4 of a block of length L through
// the stages of lengths L and L/2, in registers); an odd stage count starts with one radix-2 stage.  Index
// arithmetic by shifts and masks (every extent is a power of two).
__device__ __forceinline__ void tile_dif(uint32_t *tile, int ld, int lgcol, int kp, const uint32_t *rt,
                                         const uint32_t *rts, uint32_t q) {
  const int cmask = (1 << lgcol) - 1;
  int lglen = kp;
  if (kp & 1) {
    const int h = 1 << (lglen - 1), lgts = kp - lglen;
    for (int t = threadIdx.x; t < (1 << (lgcol + kp - 1)); t += blockDim.x) {
      const int cc = t & cmask, b = t >> lgcol, j = b & (h - 1), i0 = ((b - j) << 1) + j, i1 = i0 + h;
      const uint32_t u = tile[i0 * ld + cc], v = tile[i1 * ld + cc];
      tile[i0 * ld + cc] = addmod(u, v, q);
      tile[i1 * ld + cc] = shoup_mul(submod(u, v, q), rt[j << lgts], rts[j << lgts], q);
    }
    __syncthreads();
    --lglen;
  }
  for (; lglen >= 2; lglen -= 2) {
    const int L4 = 1 << (lglen - 2), lgts = kp - lglen;
    for (int t = threadIdx.x; t < (1 << (lgcol + kp - 2)); t += blockDim.x) {
      const int cc = t & cmask, u = t >> lgcol, j = u & (L4 - 1), base = ((u - j) << 2) + j;
      uint32_t *x0 = tile + base * ld + cc, *x1 = x0 + L4 * ld, *x2 = x1 + L4 * ld, *x3 = x2 + L4 * ld;
      const uint32_t a0 = *x0, a1 = *x1, a2 = *x2, a3 = *x3;
      const int k1 = j << lgts, k2 = (j + L4) << lgts, k3 = j << (lgts + 1);
      const uint32_t b0 = addmod(a0, a2, q), b2 = shoup_mul(submod(a0, a2, q), rt[k1], rts[k1], q);
      const uint32_t b1 = addmod(a1, a3, q), b3 = shoup_mul(submod(a1, a3, q), rt[k2], rts[k2], q);
      *x0 = addmod(b0, b1, q);
      *x1 = shoup_mul(submod(b0, b1, q), rt[k3], rts[k3], q);
      *x2 = addmod(b2, b3, q);
      *x3 = shoup_mul(submod(b2, b3, q), rt[k3], rts[k3], q);
    }
    __syncthreads();
  }
}
// R-point inverse DIT (bit-reversed in, natural out), twiddles w_R^-j: stages of lengths 2, 4, .., R, two at a time
// (lengths L/2 and L on the four elements j, j + L/4, j + L/2, j + 3L/4), an odd count ending with one radix-2 stage
__device__ __forceinline__ void tile_dit(uint32_t *tile, int ld, int lgcol, int kp, const uint32_t *rt,
                                         const uint32_t *rts, uint32_t q) {
  const int cmask = (1 << lgcol) - 1;
  int lglen = 2;
  for (; lglen <= kp; lglen += 2) {
    const int L4 = 1 << (lglen - 2), lgts = kp - lglen;
    for (int t = threadIdx.x; t < (1 << (lgcol + kp - 2)); t += blockDim.x) {
      const int cc = t & cmask, u = t >> lgcol, j = u & (L4 - 1), base = ((u - j) << 2) + j;
      uint32_t *x0 = tile + base * ld + cc, *x1 = x0 + L4 * ld, *x2 = x1 + L4 * ld, *x3 = x2 + L4 * ld;
      const int k1 = j << lgts, k2 = (j + L4) << lgts, k3 = j << (lgts + 1);
      const uint32_t a0 = *x0, a1 = shoup_mul(*x1, rt[k3], rts[k3], q);
      const uint32_t a2 = *x2, a3 = shoup_mul(*x3, rt[k3], rts[k3], q);
      const uint32_t u0 = addmod(a0, a1, q), u1 = submod(a0, a1, q);
      const uint32_t u2 = shoup_mul(addmod(a2, a3, q), rt[k1], rts[k1], q);
      const uint32_t u3 = shoup_mul(submod(a2, a3, q), rt[k2], rts[k2], q);
      *x0 = addmod(u0, u2, q);
      *x2 = submod(u0, u2, q);
      *x1 = addmod(u1, u3, q);
      *x3 = submod(u1, u3, q);
    }
    __syncthreads();
  }
  if (kp & 1) {
    lglen = kp;
    const int h = 1 << (lglen - 1), lgts = kp - lglen;
    for (int t = threadIdx.x; t < (1 << (lgcol + kp - 1)); t += blockDim.x) {
      const int cc = t & cmask, b = t >> lgcol, j = b & (h - 1), i0 = ((b - j) << 1) + j, i1 = i0 + h;
      const uint32_t u = tile[i0 * ld + cc], v = shoup_mul(tile[i1 * ld + cc], rt[j << lgts], rts[j << lgts], q);
      tile[i0 * ld + cc] = addmod(u, v, q);
      tile[i1 * ld + cc] = submod(u, v, q);
    }
    __syncthreads();
  }
}

// The R-point roots of a pass, from the table of Rmax-point roots (Rmax = min(kPassR, N)): w_R^j = w_Rmax^(j Rmax / R).
__device__ __forceinline__ void load_root_table(uint32_t *rt, uint32_t *rts, const TwTab &T, int R, int logN) {
  const int rmax = 1 << (logN < kPassMaxStages ? logN : kPassMaxStages);
  for (int j = threadIdx.x; j < (R >> 1); j += blockDim.x) {
    rt[j] = T.rt[j * (rmax / R)];
    rts[j] = T.rts[j * (rmax / R)];
  }
}

// A column pass of the length-N transform on blocks of M = R Nc elements (Nc >= kPassCols): column q = (block bb,
// offset c) holds a[bb M + c + m Nc], m < R.  Forward (INV = false): R-point DIF of every column, then element m of
// column c times w_M^(c k), k = bitrev(m) (its frequency index).  Inverse: the twiddle w_M^(-c k) first, then the
// R-point inverse DIT.  Each block takes kPassCols consecutive columns of one block of M.
template <bool INV>
__global__ void __launch_bounds__(256) ntt_column_pass(uint32_t *a, int logN, int logM, int kp, TwTab T,
                                                       TwTab TR, PrimeQ P) {
  __shared__ uint32_t tile[kTileWords];
  __shared__ uint32_t rt[kPassR / 2], rts[kPassR / 2];
  __shared__ uint32_t p1[kPassCols][16], p2[kPassCols][16];
  const int R = 1 << kp, logNc = logM - kp;
  const uint32_t Nc = 1u << logNc, M = 1u << logM;
  const uint32_t q0 = blockIdx.x * kPassCols;            // first column of this block
  const uint32_t bb = q0 >> logNc, c0 = q0 & (Nc - 1);
  const size_t base = (size_t)bb * M + c0;
  constexpr int ld = kPassCols + 1;
  load_root_table(rt, rts, TR, R, logN);
  column_twiddles(p1, p2, c0, logN - logM, T, P);
  if (INV) __syncthreads();
  for (int i = threadIdx.x; i < R * kPassCols; i += blockDim.x) {
    const int m = i / kPassCols, cc = i % kPassCols;
    uint32_t x = a[base + cc + (size_t)m * Nc];
    if (INV) {
      // the inverse twiddle w_M^(-(c0 + cc) k) (T holds the inverse root's powers)
      const uint32_t k = bitrev(m, kp);
      x = mont_mul(mont_mul(x, p1[cc][k & 15], P), p2[cc][k >> 4], P);
    }
    tile[m * ld + cc] = x;
  }
  __syncthreads();
  constexpr int lgcols = 5;
  static_assert((1 << lgcols) == kPassCols, "columns per block");
  if (INV) tile_dit(tile, ld, lgcols, kp, rt, rts, P.q);
  else tile_dif(tile, ld, lgcols, kp, rt, rts, P.q);
  for (int i = threadIdx.x; i < R * kPassCols; i += blockDim.x) {
    const int m = i / kPassCols, cc = i % kPassCols;
    uint32_t x = tile[m * ld + cc];
    if (!INV) {
      const uint32_t k = bitrev(m, kp);   // the frequency this position holds: times w_M^((c0 + cc) k)
      x = mont_mul(mont_mul(x, p1[cc][k & 15], P), p2[cc][k >> 4], P);
    }
    a[base + cc + (size_t)m * Nc] = x;
  }
}

// The innermost pass on contiguous runs of R = 2^kp elements: forward R-point DIF, every entry to the n-th power,
// inverse R-point DIT.  A block takes G = min(N, kPassR kPassCols) / R runs.
__global__ void __launch_bounds__(256) ntt_inner_pow(uint32_t *a, int logN, int kp, uint32_t n, TwTab TF,
                                                     TwTab TI, PrimeQ P) {
  __shared__ uint32_t tile[kTileWords];
  __shared__ uint32_t rf[kPassR / 2], rfs[kPassR / 2], ri[kPassR / 2], ris[kPassR / 2];
  const int R = 1 << kp;
  const int lgw = logN < kPassMaxStages + 5 ? logN : kPassMaxStages + 5;   // words = min(kPassR kPassCols, N)
  const int words = 1 << lgw, lgg = lgw - kp;
  const int ld = (1 << lgg) + 1;   // row stride G + 1: both the run-wise copies and the butterflies
  const size_t base = (size_t)blockIdx.x * words;   // are free of shared-memory bank conflicts
  load_root_table(rf, rfs, TF, R, logN);
  load_root_table(ri, ris, TI, R, logN);
  // tile[m * ld + g] = a[base + g R + m]: run g is a column of the tile
  for (int i = threadIdx.x; i < words; i += blockDim.x) {
    const int g = i >> kp, m = i & (R - 1);
    tile[m * ld + g] = a[base + i];
  }
  __syncthreads();
  tile_dif(tile, ld, lgg, kp, rf, rfs, P.q);
  for (int i = threadIdx.x; i < words; i += blockDim.x) {
    const int g = i >> kp, m = i & (R - 1);
    // x^n by squaring and multiplying in Montgomery form
    const uint32_t xm = mont_mul(tile[m * ld + g], P.r2, P);
    uint32_t y = P.rmod, sq = xm;
    for (uint32_t e = n; e; e >>= 1) {
      if (e & 1u) y = mont_mul(y, sq, P);
      sq = mont_mul(sq, sq, P);
    }
    tile[m * ld + g] = mont_mul(y, 1u, P);
  }
  __syncthreads();
  tile_dit(tile, ld, lgg, kp, ri, ris, P.q);
  for (int i = threadIdx.x; i < words; i += blockDim.x) {
    const int g = i >> kp, m = i & (R - 1);
    a[base + i] = tile[m * ld + g];
  }
}

// ------------------------------------------------------------------------------------ register-resident passes
// A pass of KP <= 8 stages in two register phases with one exchange through shared memory between them.  With
// K1 = KP / 2 and K2 = KP - K1, the element m of an R-point column (R = 2^KP) is written m = m0 + (k << K2)
// (m0 < 2^K2, k < 2^K1) or m = (g << K2) + r (g < 2^K1, r < 2^K2).  In the DIF, the stages of lengths R .. 2^(K2+1)
// pair elements with the same m0 (a 2^K1-point sub-transform per m0, in registers), and the stages of lengths
// 2^K2 .. 2 stay inside one block g of 2^K2 consecutive elements (a 2^K2-point sub-transform per g).  The inverse
// DIT takes the same two groups in the opposite order.  Every element is loaded and stored once per pass and goes
// through shared memory once, against one shared-memory round trip per stage pair in tile_dif / tile_dit.
constexpr int kNttThreads = 256;

__host__ __device__ constexpr uint32_t bitrev_c(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
  return r;
}

// In-register DIF stages on x[k] = X[m0 + (k << S)], k < 2^K, of an R-point transform (R = 2^KP): the stages of
// lengths 2^(S+K) .. 2^(S+1).  The stage of half-length h = 2^t in k pairs (k, k + h) for k mod 2h < h, with the
// twiddle w_R^(j R / len) = rt[j << (KP - S - t - 1)], j = m0 + ((k mod h) << S) (rt[e] = w_R^e, Shoup companions
// in rts).  M0ZERO: m0 is 0, so the pairs with k mod h = 0 take w^0 and skip the product.
template <int KP, int K, int S, bool M0ZERO>
__device__ __forceinline__ void reg_dif(uint32_t (&x)[1 << K], int m0, const uint32_t *rt, const uint32_t *rts,
                                        uint32_t q) {
#pragma unroll
  for (int t = K - 1; t >= 0; --t) {
    const int h = 1 << t, sh = KP - S - t - 1;
#pragma unroll
    for (int k = 0; k < (1 << K); ++k) {
      if (k & h) continue;
      const uint32_t u = x[k], v = x[k + h];
      x[k] = addmod(u, v, q);
      if (M0ZERO && (k & (h - 1)) == 0) {
        x[k + h] = submod(u, v, q);
      } else {
        const int e = (m0 + ((k & (h - 1)) << S)) << sh;
        x[k + h] = shoup_mul(submod(u, v, q), rt[e], rts[e], q);
      }
    }
  }
}

// In-register inverse DIT stages on x[k] = X[m0 + (k << S)]: lengths 2^(S+1) .. 2^(S+K), twiddles as in reg_dif
// (rt holds the inverse root's powers).
template <int KP, int K, int S, bool M0ZERO>
__device__ __forceinline__ void reg_dit(uint32_t (&x)[1 << K], int m0, const uint32_t *rt, const uint32_t *rts,
                                        uint32_t q) {
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const int h = 1 << t, sh = KP - S - t - 1;
#pragma unroll
    for (int k = 0; k < (1 << K); ++k) {
      if (k & h) continue;
      uint32_t v = x[k + h];
      if (!(M0ZERO && (k & (h - 1)) == 0)) {
        const int e = (m0 + ((k & (h - 1)) << S)) << sh;
        v = shoup_mul(v, rt[e], rts[e], q);
      }
      const uint32_t u = x[k];
      x[k] = addmod(u, v, q);
      x[k + h] = submod(u, v, q);
    }
  }
}

// Element m of column cc (frequency k = bitrev(m)) times w_M^(+-(c0 + cc) k) from the column's p1 / p2 tables.
__device__ __forceinline__ uint32_t column_twiddle(uint32_t x, const uint32_t *p1c, const uint32_t *p2c, uint32_t k,
                                                   const PrimeQ &P) {
  return mont_mul(mont_mul(x, p1c[k & 15], P), p2c[k >> 4], P);
}

// A column pass of KP stages (2 <= KP <= 8) with the layout of ntt_column_pass: column q = (block bb, offset c)
// holds a[bb M + c + m Nc], m < R = 2^KP; each block takes kPassCols consecutive columns.  A task (cc, m0) holds
// rows m0 + (k << K2) of column cc, a task (cc, g) rows (g << K2) + r; the lanes of a warp are 32 consecutive
// columns, so every global access is one 128-byte row segment and every shared-memory access is free of conflicts
// (row stride kPassCols + 1).
// nz_rows (forward): rows m >= nz_rows of every column are zero and are not read (the first pass of a transform
// whose input fills only its leading rows).
template <int KP, bool INV>
__global__ void __launch_bounds__(kNttThreads) ntt_column_regs(uint32_t *a, int logN, int logM, TwTab T, TwTab TR,
                                                               PrimeQ P, int nz_rows) {
  static_assert(KP >= 2 && KP <= kPassMaxStages, "two register phases");
  constexpr int K1 = KP / 2, K2 = KP - K1, ld = kPassCols + 1;
  constexpr int NT1 = kPassCols << K2, NT2 = kPassCols << K1;   // tasks of the strided and the contiguous phase
  __shared__ uint32_t tile[(1 << KP) * ld];
  __shared__ uint32_t rt[kPassR / 2], rts[kPassR / 2];
  __shared__ uint32_t p1[kPassCols][16], p2[kPassCols][16];
  const int logNc = logM - KP;
  const uint32_t Nc = 1u << logNc;
  const uint32_t q0 = blockIdx.x * kPassCols;
  const uint32_t bb = q0 >> logNc, c0 = q0 & (Nc - 1);
  uint32_t *col = a + ((size_t)bb << logM) + c0;
  load_root_table(rt, rts, TR, 1 << KP, logN);
  column_twiddles(p1, p2, c0, logN - logM, T, P);
  __syncthreads();
  if (!INV) {
#pragma unroll
    for (int it = 0; it < (NT1 + kNttThreads - 1) / kNttThreads; ++it) {
      const int task = threadIdx.x + it * kNttThreads;
      if (task < NT1) {
        const int cc = task & (kPassCols - 1), m0 = task >> 5;
        uint32_t x[1 << K1];
#pragma unroll
        for (int k = 0; k < (1 << K1); ++k) {
          const int m = m0 + (k << K2);
          x[k] = m < nz_rows ? col[cc + (size_t)m * Nc] : 0u;
        }
        reg_dif<KP, K1, K2, false>(x, m0, rt, rts, P.q);
#pragma unroll
        for (int k = 0; k < (1 << K1); ++k) tile[(m0 + (k << K2)) * ld + cc] = x[k];
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < (NT2 + kNttThreads - 1) / kNttThreads; ++it) {
      const int task = threadIdx.x + it * kNttThreads;
      if (task < NT2) {
        const int cc = task & (kPassCols - 1), g = task >> 5;
        uint32_t x[1 << K2];
#pragma unroll
        for (int r = 0; r < (1 << K2); ++r) x[r] = tile[((g << K2) + r) * ld + cc];
        reg_dif<KP, K2, 0, true>(x, 0, rt, rts, P.q);
        const uint32_t bg = bitrev(g, K1);
#pragma unroll
        for (int r = 0; r < (1 << K2); ++r) {
          // position (g << K2) + r holds frequency bitrev_KP = (bitrev_K2(r) << K1) | bitrev_K1(g)
          const uint32_t k = (bitrev_c(r, K2) << K1) | bg;
          col[cc + (size_t)((g << K2) + r) * Nc] = column_twiddle(x[r], p1[cc], p2[cc], k, P);
        }
      }
    }
  } else {
#pragma unroll
    for (int it = 0; it < (NT2 + kNttThreads - 1) / kNttThreads; ++it) {
      const int task = threadIdx.x + it * kNttThreads;
      if (task < NT2) {
        const int cc = task & (kPassCols - 1), g = task >> 5;
        const uint32_t bg = bitrev(g, K1);
        uint32_t x[1 << K2];
#pragma unroll
        for (int r = 0; r < (1 << K2); ++r) {
          // the inverse twiddle w_M^(-(c0 + cc) k) (T holds the inverse root's powers)
          const uint32_t k = (bitrev_c(r, K2) << K1) | bg;
          x[r] = column_twiddle(col[cc + (size_t)((g << K2) + r) * Nc], p1[cc], p2[cc], k, P);
        }
        reg_dit<KP, K2, 0, true>(x, 0, rt, rts, P.q);
#pragma unroll
        for (int r = 0; r < (1 << K2); ++r) tile[((g << K2) + r) * ld + cc] = x[r];
      }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < (NT1 + kNttThreads - 1) / kNttThreads; ++it) {
      const int task = threadIdx.x + it * kNttThreads;
      if (task < NT1) {
        const int cc = task & (kPassCols - 1), m0 = task >> 5;
        uint32_t x[1 << K1];
#pragma unroll
        for (int k = 0; k < (1 << K1); ++k) x[k] = tile[(m0 + (k << K2)) * ld + cc];
        reg_dit<KP, K1, K2, false>(x, m0, rt, rts, P.q);
#pragma unroll
        for (int k = 0; k < (1 << K1); ++k) col[cc + (size_t)(m0 + (k << K2)) * Nc] = x[k];
      }
    }
  }
}

// x^n for x < q (normal form) by Montgomery products on normal-form operands: every product carries a factor
// 2^-32, so the square-and-multiply chain gives x^n 2^(-32(n-1)), and one product with c = 2^(32 n) mod q restores
// x^n.  n >= 1.
__device__ __forceinline__ uint32_t pow_mont(uint32_t x, uint32_t n, uint32_t c, const PrimeQ &P) {
  uint32_t sq = x, e = n;
  while (!(e & 1u)) {
    sq = mont_mul(sq, sq, P);
    e >>= 1;
  }
  uint32_t y = sq;
  for (e >>= 1; e; e >>= 1) {
    sq = mont_mul(sq, sq, P);
    if (e & 1u) y = mont_mul(y, sq, P);
  }
  return mont_mul(y, c, P);
}

// The innermost pass for N >= kPassR kPassCols: a block takes kPassCols runs of R = kPassR contiguous elements
// (element m of run g at a[blk + g R + m]).  Strided phase of the forward DIF (task (g, m0)), then per block of 2^K2
// consecutive elements (task (g, b)) the contiguous phase, the n-th powers and the contiguous phase of the inverse
// DIT without leaving registers, then the strided phase of the inverse.  Shared tile: run g, element m at
// g RW + (m >> K2) BW + (m mod 2^K2) with blocks padded to BW = 2^K2 + 1 words, so that both phases' accesses
// (16 lanes per run, two runs per warp) are free of bank conflicts.  cn = 2^(32 n) mod q (pow_mont).
__global__ void __launch_bounds__(kNttThreads) ntt_inner_regs(uint32_t *a, int logN, uint32_t n, uint32_t cn,
                                                              TwTab TF, TwTab TI, PrimeQ P) {
  constexpr int KP = kPassMaxStages, K1 = KP / 2, K2 = KP - K1, G = kPassCols;
  constexpr int BW = (1 << K2) + 1, RW = (1 << K1) * BW;
  constexpr int NT1 = G << K2, NT2 = G << K1;
  __shared__ uint32_t tile[G * RW];
  __shared__ uint32_t rf[kPassR / 2], rfs[kPassR / 2], ri[kPassR / 2], ris[kPassR / 2];
  uint32_t *blk = a + ((size_t)blockIdx.x << (KP + 5));
  static_assert(G == 32, "32 runs per block");
  load_root_table(rf, rfs, TF, 1 << KP, logN);
  load_root_table(ri, ris, TI, 1 << KP, logN);
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NT1 / kNttThreads; ++it) {
    const int task = threadIdx.x + it * kNttThreads;
    const int m0 = task & ((1 << K2) - 1), g = task >> K2;
    uint32_t x[1 << K1];
#pragma unroll
    for (int k = 0; k < (1 << K1); ++k) x[k] = blk[(g << KP) + m0 + (k << K2)];
    reg_dif<KP, K1, K2, false>(x, m0, rf, rfs, P.q);
#pragma unroll
    for (int k = 0; k < (1 << K1); ++k) tile[g * RW + k * BW + m0] = x[k];
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NT2 / kNttThreads; ++it) {
    const int task = threadIdx.x + it * kNttThreads;
    const int b = task & ((1 << K1) - 1), g = task >> K1;
    uint32_t x[1 << K2];
#pragma unroll
    for (int r = 0; r < (1 << K2); ++r) x[r] = tile[g * RW + b * BW + r];
    reg_dif<KP, K2, 0, true>(x, 0, rf, rfs, P.q);
#pragma unroll
    for (int r = 0; r < (1 << K2); ++r) x[r] = pow_mont(x[r], n, cn, P);
    reg_dit<KP, K2, 0, true>(x, 0, ri, ris, P.q);
#pragma unroll
    for (int r = 0; r < (1 << K2); ++r) tile[g * RW + b * BW + r] = x[r];
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NT1 / kNttThreads; ++it) {
    const int task = threadIdx.x + it * kNttThreads;
    const int m0 = task & ((1 << K2) - 1), g = task >> K2;
    uint32_t x[1 << K1];
#pragma unroll
    for (int k = 0; k < (1 << K1); ++k) x[k] = tile[g * RW + k * BW + m0];
    reg_dit<KP, K1, K2, false>(x, m0, ri, ris, P.q);
#pragma unroll
    for (int k = 0; k < (1 << K1); ++k) blk[(g << KP) + m0 + (k << K2)] = x[k];
  }
}

// The output monomials x2^e2 x3^e3 x4^e4 (e2 + e3 + e4 <= D) in transform order: e4, then e3, then e2, which is
// contiguous in the packed transform (index e2 + B e3 + B^2 e4).  Row (e4, e3) holds D - e4 - e3 + 1 monomials and
// starts at toff(D, e4, e3); rows are numbered e4-major, PB(e4) = e4 (D + 1) - tri(e4 - 1) of them before slice e4.
__host__ __device__ __forceinline__ int toff(int D, int e4, int e3) {
  const int n = D - e4;
  return tet(D + 1) - tet(n + 1) + e3 * (n + 1) - tri(e3 - 1);
}
__device__ __forceinline__ int rows_before(int D, int e4) { return e4 * (D + 1) - tri(e4 - 1); }
// row index -> (e4, e3): PB(e) = e (2D + 3 - e) / 2 <= r gives e from an integer square root, then corrections
__device__ __forceinline__ void decode_row(int r, int D, int &e4, int &e3) {
  const int b = 2 * D + 3;
  int e = (b - isqrt(b * b - 8 * r)) >> 1;
  while (e > 0 && rows_before(D, e) > r) --e;
  while (rows_before(D, e + 1) <= r) ++e;
  e4 = e;
  e3 = r - rows_before(D, e);
}

// residue of every output coefficient, times N^-1, in transform order: one warp per row (e4, e3), lanes over e2,
// so the reads of the transform and the writes of the residues are contiguous
__global__ void gather_kernel(const uint32_t *a, int D, int B, uint32_t ninv, uint32_t *res, PrimeQ P) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= tri(D + 1)) return;
  int e4, e3;
  decode_row(r, D, e4, e3);
  const int o = toff(D, e4, e3), len = D - e4 - e3 + 1;
  const uint32_t *row = a + (size_t)B * e3 + (size_t)B * B * e4;
  for (int e2 = lane; e2 < len; e2 += 32) res[o + e2] = mulmod(row[e2], ninv, P.q, P.mu);
}

struct CrtParams {
  uint32_t q[kPolyPowMaxPrimes];
  uint64_t mu[kPolyPowMaxPrimes];
  uint32_t inv[kPolyPowMaxPrimes][kPolyPowMaxPrimes];   // inv[j][k] = q_k^-1 mod q_j (k < j)
  int nprimes;
};

// Garner: v_j = (...((r_j - v_0) q_0^-1 - v_1) q_1^-1 ... - v_{j-1}) q_{j-1}^-1 mod q_j; then
// X = v_0 + q_0 (v_1 + q_1 (v_2 + ...)) in 8 little-endian 32-bit limbs.  v_k mod q_j for k < j is one conditional
// subtraction: the primes are taken largest first and the largest is below twice the smallest, so v_k < 2 q_j.
// The residues are read in transform order (one warp per row, as the gather wrote them) and each coefficient is
// written at its packed (descending lex) index tet(u) + tri(s) + t, (u, s, t) = (e2 + e3 + e4, e3 + e4, e4): one
// 32-byte record per lane.
__global__ void crt_kernel(const uint32_t *res, int n_out, int D, CrtParams C, uint32_t *out) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (r >= tri(D + 1)) return;
  int e4, e3;
  decode_row(r, D, e4, e3);
  const int o = toff(D, e4, e3), len = D - e4 - e3 + 1;
  for (int e2 = lane; e2 < len; e2 += 32) {
    const size_t i = (size_t)tet(e2 + e3 + e4) + tri(e3 + e4) + e4;
    uint32_t v[kPolyPowMaxPrimes];
    for (int j = 0; j < C.nprimes; ++j) {
      uint32_t t = res[(size_t)j * n_out + o + e2];
      for (int k = 0; k < j; ++k) {
        const uint32_t vk = v[k] >= C.q[j] ? v[k] - C.q[j] : v[k];
        t = mulmod(submod(t, vk, C.q[j]), C.inv[j][k], C.q[j], C.mu[j]);
      }
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
    uint32_t *rec = out + i * kPolyPowLimbs;
    if ((reinterpret_cast<uintptr_t>(out) & 15) == 0) {   // the record as two 16-byte stores
      reinterpret_cast<uint4 *>(rec)[0] = make_uint4(x[0], x[1], x[2], x[3]);
      reinterpret_cast<uint4 *>(rec)[1] = make_uint4(x[4], x[5], x[6], x[7]);
    } else {
      for (int l = 0; l < kPolyPowLimbs; ++l) rec[l] = x[l];
    }
  }
}

// primes q = c 2^24 + 1 below 2^31 (largest first) and a primitive root of each
constexpr uint32_t kQ[kPolyPowMaxPrimes] = {2130706433u, 2113929217u, 2013265921u, 1811939329u,
                                            1711276033u, 1224736769u, 1107296257u};
constexpr uint32_t kRoot[kPolyPowMaxPrimes] = {3u, 5u, 31u, 13u, 29u, 3u, 10u};
static_assert(kQ[0] < 2ull * kQ[kPolyPowMaxPrimes - 1], "a residue mod an earlier prime reduces mod a later one by one subtraction");
static_assert(kPolyPowLimbs == 8, "a coefficient record is two 16-byte stores");

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

// Big unsigned integers on the host as little-endian 64-bit limbs, for exact bounds (kBigLimbs x 64 bits).
namespace {
constexpr int kBigLimbs = 6;
// x *= v; returns false if the product does not fit
bool big_mul(uint64_t (&x)[kBigLimbs], uint64_t v) {
  unsigned __int128 carry = 0;
  for (int l = 0; l < kBigLimbs; ++l) {
    const unsigned __int128 y = (unsigned __int128)x[l] * v + carry;
    x[l] = (uint64_t)y;
    carry = y >> 64;
  }
  return carry == 0;
}
// a > b
bool big_gt(const uint64_t (&a)[kBigLimbs], const uint64_t (&b)[kBigLimbs]) {
  for (int l = kBigLimbs - 1; l >= 0; --l)
    if (a[l] != b[l]) return a[l] > b[l];
  return false;
}
}  // namespace

int polypow_primes(uint64_t sum, int n) {
  // every coefficient of f^n is at most sum^n; the output holds 32 kPolyPowLimbs bits, and the product of the
  // primes (largest first) must exceed the bound for the Chinese remaindering to be exact
  uint64_t bound[kBigLimbs] = {1, 0, 0, 0, 0, 0};
  for (int i = 0; i < n; ++i)
    if (!big_mul(bound, sum < 1 ? 1 : sum)) return 0;
  for (int l = 32 * kPolyPowLimbs / 64; l < kBigLimbs; ++l)
    if (bound[l]) return 0;
  uint64_t prod[kBigLimbs] = {1, 0, 0, 0, 0, 0};
  for (int j = 0; j < kPolyPowMaxPrimes; ++j) {
    big_mul(prod, kQ[j]);   // at most 7 x 31 bits: fits
    if (big_gt(prod, bound)) return j + 1;
  }
  return 0;
}

// Twiddle table words of one prime and direction: lo and hi tables of 2^12 entries and the R-point roots, each with
// its companion.
constexpr size_t kTwWords = 2 * (4096 + 4096 + kPassR / 2);

size_t polypow_scratch_words(int d, int n, int nprimes) {
  const int B = d * n + 1;
  uint32_t N = 1;
  while ((uint64_t)N < (uint64_t)B * B * B) N <<= 1;
  return (size_t)N + 2 * kTwWords * (size_t)nprimes + (size_t)nprimes * tet(d * n + 1) + tet(d + 1) + 64;
}

// Rows of the first forward column pass (kp0 stages; 0: no column pass) that can hold input, and the words cleared
// before the input is scattered: the input's indices are < d B^2 + 1, and the pass takes columns of stride
// N / 2^kp0.  The shared-memory stage loop (kp0 = 1) reads every row, so the whole buffer is cleared then.
struct PassRows {
  int rows;
  uint32_t cleared;
};
PassRows first_pass_rows(int d, int B, int logN, int kp0) {
  const uint64_t N = 1ull << logN, bound = (uint64_t)d * B * B + 1;
  if (kp0 < 2) return PassRows{1 << kp0, (uint32_t)N};
  const uint64_t stride = N >> kp0;
  const uint64_t rows = (bound + stride - 1) / stride;
  return PassRows{(int)rows, (uint32_t)(rows * stride)};
}

void polypow_plan(int d, int n, int nprimes, uint64_t *transform_len, uint64_t *bytes) {
  const int B = d * n + 1;
  uint64_t N = 1;
  int logN = 0;
  while (N < (uint64_t)B * B * B) { N <<= 1; ++logN; }
  const int inner = logN < kPassMaxStages ? logN : kPassMaxStages;
  const int n_outer = (logN - inner + kPassMaxStages - 1) / kPassMaxStages;
  const uint64_t n_in = tet(d + 1), n_out = tet(d * n + 1);
  const uint64_t R = N < (uint64_t)kPassR ? N : (uint64_t)kPassR;
  const uint64_t nlo = N < 4096 ? N : 4096, nhi = N >> kTwLoBits ? N >> kTwLoBits : 1;
  // per prime and direction: the lo and hi tables (one word each) and the R / 2 roots with their companions
  const uint64_t tables = 2 * 4 * (nlo + nhi + R);
  // the first (outermost) pass takes min(8, logN - inner) stages, as polypow_launch splits them
  const int outer0 = logN - inner < kPassMaxStages ? logN - inner : kPassMaxStages;
  const PassRows PR = first_pass_rows(d, B, logN, outer0);
  // every pass reads and writes the buffer, except that the first forward pass reads only its leading rows
  const uint64_t passes = n_outer ? 4 * (uint64_t)PR.cleared + 4 * N + (uint64_t)(2 * n_outer) * 8 * N : 8 * N;
  const uint64_t per_prime = tables + 4 * (uint64_t)PR.cleared   // clear the leading rows
                             + 4 * 2 * n_in                       // read the input, write it into the buffer
                             + passes
                             + 8 * n_out;                         // gather: read a residue, write it
  if (transform_len) *transform_len = N;
  if (bytes) *bytes = (uint64_t)nprimes * per_prime + n_out * (4ull * nprimes + 4ull * kPolyPowLimbs);
}

namespace {

// Tables of w (forward) or w^-1 (inverse) for a length-N transform in tab (kTwWords words): fills the pointers and
// appends the three table jobs to J (built later by one power_tables_kernel launch).
TwTab plan_tables(uint32_t *tab, uint32_t w, uint32_t N, const PrimeQ &P, TableJobs &J, int &njobs) {
  TwTab T;
  uint32_t *p = tab;
  T.lo = p; T.los = p + 4096; p += 8192;
  T.hi = p; T.his = p + 4096; p += 8192;
  T.rt = p; T.rts = p + kPassR / 2;
  const uint32_t R = N < (uint32_t)kPassR ? N : (uint32_t)kPassR;
  const uint32_t nhi = N >> kTwLoBits ? N >> kTwLoBits : 1;
  const uint32_t nlo = N < 4096u ? N : 4096u;
  J.job[njobs++] = TableJob{const_cast<uint32_t *>(T.lo), nullptr, nlo, w, 1, 1, P};
  J.job[njobs++] = TableJob{const_cast<uint32_t *>(T.hi), nullptr, nhi, w, 4096, 1, P};
  // w_R^j for j < R / 2 with Shoup companions: the R-point roots of every pass are rt[j * (kPassR / R)]
  J.job[njobs++] = TableJob{const_cast<uint32_t *>(T.rt), const_cast<uint32_t *>(T.rts), R / 2, w, N / R, 0, P};
  return T;
}

// One column pass of kp stages: the register-phase kernel for kp >= 2, the shared-memory stage loop for kp = 1.
// nz_rows: rows of every column the forward pass reads (the rest are zero); the stage loop reads them all.
void column_pass(bool inv, int kp, uint32_t blocks, uint32_t *a, int logN, int logM, const TwTab &T, const PrimeQ &P,
                 cudaStream_t st, int nz_rows) {
#define QFS_COLUMN_PASS(KP)                                                                               \
  case KP:                                                                                                \
    if (inv) ntt_column_regs<KP, true><<<blocks, kNttThreads, 0, st>>>(a, logN, logM, T, T, P, 1 << KP);  \
    else ntt_column_regs<KP, false><<<blocks, kNttThreads, 0, st>>>(a, logN, logM, T, T, P, nz_rows);     \
    break;
  switch (kp) {
    QFS_COLUMN_PASS(2)
    QFS_COLUMN_PASS(3)
    QFS_COLUMN_PASS(4)
    QFS_COLUMN_PASS(5)
    QFS_COLUMN_PASS(6)
    QFS_COLUMN_PASS(7)
    QFS_COLUMN_PASS(8)
    default:
      if (inv) ntt_column_pass<true><<<blocks, 256, 0, st>>>(a, logN, logM, kp, T, T, P);
      else ntt_column_pass<false><<<blocks, 256, 0, st>>>(a, logN, logM, kp, T, T, P);
  }
#undef QFS_COLUMN_PASS
}

}  // namespace

cudaError_t polypow_launch(int d, int n, int nprimes, const uint32_t *coeffs_dev, uint32_t *out, uint32_t *scratch,
                           cudaStream_t st) {
  const int B = d * n + 1, D = d * n;
  uint32_t N = 1;
  int logN = 0;
  while ((uint64_t)N < (uint64_t)B * B * B) { N <<= 1; ++logN; }
  const int n_out = tet(D + 1);
  uint32_t *a = scratch;
  uint32_t *tw = a + N;                               // forward and inverse tables of every prime
  uint32_t *res = tw + 2 * kTwWords * (size_t)nprimes;
  const int grid = 152 * 8, block = 256;
  // passes: the innermost takes min(8, logN) stages on contiguous runs; the rest, outermost first, up to 8 each
  const int inner = logN < kPassMaxStages ? logN : kPassMaxStages;
  int outer[4], n_outer = 0;
  for (int rem = logN - inner; rem > 0;) {
    const int kp = rem > kPassMaxStages ? kPassMaxStages : rem;
    outer[n_outer++] = kp;
    rem -= kp;
  }
  CrtParams C;
  C.nprimes = nprimes;
  PrimeQ PQ[kPolyPowMaxPrimes];
  TwTab TF[kPolyPowMaxPrimes], TI[kPolyPowMaxPrimes];
  uint32_t ninv[kPolyPowMaxPrimes];
  TableJobs J;
  int njobs = 0;
  for (int j = 0; j < nprimes; ++j) {
    const uint32_t q = kQ[j];
    uint32_t qinv = 1;   // q^-1 mod 2^32 by Newton's iteration (each step doubles the correct low bits)
    for (int i = 0; i < 5; ++i) qinv *= 2u - q * qinv;
    const uint32_t rmod = (uint32_t)((((uint64_t)1) << 32) % q);
    PQ[j] = PrimeQ{q, barrett_mu(q), 0u - qinv, rmod, (uint32_t)host_mulmod(rmod, rmod, q)};
    C.q[j] = q;
    C.mu[j] = PQ[j].mu;
    for (int k = 0; k < kPolyPowMaxPrimes; ++k) C.inv[j][k] = k < j ? (uint32_t)host_powmod(kQ[k] % q, q - 2, q) : 0u;
    const uint32_t w = (uint32_t)host_powmod(kRoot[j], (q - 1) / N, q);   // primitive N-th root
    const uint32_t wi = (uint32_t)host_powmod(w, q - 2, q);
    ninv[j] = (uint32_t)host_powmod(N, q - 2, q);
    TF[j] = plan_tables(tw + 2 * kTwWords * (size_t)j, w, N, PQ[j], J, njobs);
    TI[j] = plan_tables(tw + 2 * kTwWords * (size_t)j + kTwWords, wi, N, PQ[j], J, njobs);
  }
  power_tables_kernel<<<dim3(16, njobs), block, 0, st>>>(J);
  // the packed input occupies indices < d B^2 + 1, so the first forward pass (columns of stride N >> outer[0]) finds
  // it in its leading rows only: those rows are cleared and read, the others are zero without a read
  const PassRows PR = first_pass_rows(d, B, logN, n_outer ? outer[0] : 0);
  for (int j = 0; j < nprimes; ++j) {
    const PrimeQ &P = PQ[j];
    zero_kernel<<<grid, block, 0, st>>>(a, PR.cleared);
    scatter_kernel<<<64, block, 0, st>>>(coeffs_dev, d, B, a, P);
    // forward: outer passes on blocks of M = N, N / 2^kp0, ...; the inner pass fuses the powers and the inverse
    int logM = logN;
    for (int i = 0; i < n_outer; ++i) {
      column_pass(false, outer[i], (N >> outer[i]) / kPassCols, a, logN, logM, TF[j], P, st,
                  i == 0 ? PR.rows : 1 << outer[i]);
      logM -= outer[i];
    }
    if (inner == kPassMaxStages && N >= (uint32_t)(kPassR * kPassCols)) {
      const uint32_t cn = (uint32_t)host_powmod(2, 32 * (uint64_t)n, P.q);
      ntt_inner_regs<<<N / (kPassR * kPassCols), kNttThreads, 0, st>>>(a, logN, (uint32_t)n, cn, TF[j], TI[j], P);
    } else {
      const uint32_t inner_words = N < (uint32_t)(kPassR * kPassCols) ? N : (uint32_t)(kPassR * kPassCols);
      ntt_inner_pow<<<N / inner_words, block, 0, st>>>(a, logN, inner, (uint32_t)n, TF[j], TI[j], P);
    }
    for (int i = n_outer - 1; i >= 0; --i) {
      logM += outer[i];
      column_pass(true, outer[i], (N >> outer[i]) / kPassCols, a, logN, logM, TI[j], P, st, 1 << outer[i]);
    }
    gather_kernel<<<(tri(D + 1) + 7) / 8, block, 0, st>>>(a, D, B, ninv[j], res + (size_t)j * n_out, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  crt_kernel<<<(tri(D + 1) + 7) / 8, block, 0, st>>>(res, n_out, D, C, out);
  return cudaGetLastError();
}

}  // namespace qfs
