// Coefficient layouts shared by every libqfs kernel.
//
// A homogeneous form of degree m in x1..x4 is addressed by (u, s, t) = (e2+e3+e4, e3+e4, e4) with
// 0 <= t <= s <= u <= m (the exponent of x1 is m - u).  Products of monomials add (u, s, t), so a product of
// forms is a 3-D convolution over this cone and the degree only bounds u.
//
// Packed layout ("descending lex"): index = tet(u) + tri(s) + t, with tet(u) = C(u+2,3), tri(s) = C(s+1,2).
// It enumerates the monomials with x1's exponent descending, then x2's, then x3's -- the order in which the paper
// prints quartics (Figures 4-7) and the order of every array that crosses the C ABI.  A form of degree m has
// C(m+3,3) = tet(m+1) entries (the paper's l_d, Sec. 4).
//
// Padded layout (device workspaces): the same order, but every column (u, s) -- the s+1 entries t = 0..s, one byte
// each -- starts on a 16-byte boundary and occupies chunks(s) = (s+4)/16 + 1 chunks of four 32-bit words; padding
// bytes are zero.  Sizing a column by s+4 rather than s gives two guarantees that the chain product relies on:
// the last word of every column is padding (so the word before any column start is zero), and column s - sI
// (sI <= 4) always has room for words 0 .. s/4 + 1 of column s.  Word offset of column (u, s) = SW[u] + 4 F(s),
// where F(s) = sum_{s' < s} chunks(s') = E(s+4) - 4 with E(n) = sum_{n' < n} (n'/16 + 1) = (q+1)(8q+r) for
// n = 16q + r, and SW[u] = sum_{v < u} 4 F(v+1).  SW does not depend on m; a degree-m form uses words
// [0, SW[m+1]).
#pragma once
#include <cstdint>

namespace qfs {

__host__ __device__ constexpr int tet(int u) { return u * (u + 1) * (u + 2) / 6; }
__host__ __device__ constexpr int tri(int s) { return s * (s + 1) / 2; }
__host__ __device__ constexpr int chunks_of(int s) { return ((s + 4) >> 4) + 1; }
// E(n) = sum_{n' < n} (n'/16 + 1); chunk_prefix(s) = F(s) = E(s + 4) - E(4)
__host__ __device__ constexpr int chunk_prefix16(int n) { return ((n >> 4) + 1) * (8 * (n >> 4) + (n & 15)); }
__host__ __device__ constexpr int chunk_prefix(int s) { return chunk_prefix16(s + 4) - 4; }
// word offset of column s inside its slice (16-byte aligned)
__host__ __device__ constexpr int colw(int s) { return 4 * chunk_prefix(s); }
__host__ __device__ constexpr int n_monomials(int m) { return tet(m + 1); }

// Largest prime the engine accepts and the derived sizes.
constexpr int kMaxP = 13;
constexpr int kMaxD = 4 * kMaxP * (kMaxP - 1);   // 624
constexpr int kSWLen = kMaxD + 6;                // SW[0 .. kMaxD+5]

template <int P>
struct Prime {
  static constexpr int p = P;
  static constexpr int p2 = P * P;
  static constexpr int d = 4 * (P - 1);          // degree of g = f^(p-1)
  static constexpr int D = 4 * P * (P - 1);      // degree of Delta_1(f^(p-1))
  static constexpr int ld = tet(d + 1);          // C(4p-1, 3)
  static constexpr int lD = tet(D + 1);
  // witness monomial (x1 x2 x3 x4)^(p-1) in degree d: (u, s, t) = (3(p-1), 2(p-1), p-1)
  static constexpr int wu = 3 * (P - 1), ws = 2 * (P - 1), wt = P - 1;
  static constexpr int witness = tet(wu) + tri(ws) + wt;
  // One chain output sums at most 35 products of a residue below p^2 and a coefficient below p.
  static constexpr uint32_t chain_max = 35u * (p2 - 1) * (P - 1);
  // a mod p^2 = a - p^2 floor(a M / 2^32) with M = ceil(2^32 / p^2): exact while a (M p^2 - 2^32) < 2^32, which
  // holds far beyond chain_max for every p <= 13 (a host test checks every a <= chain_max).
  static constexpr uint32_t mod_magic = (uint32_t)((0x100000000ull + p2 - 1) / p2);
  static_assert((uint64_t)chain_max * ((uint64_t)mod_magic * p2 - 0x100000000ull) < 0x100000000ull,
                "multiply-high reduction exact over the chain's range");
};

// a mod p^2 by one multiply-high (valid for a <= Prime<P>::chain_max).
template <int P>
__host__ __device__ __forceinline__ uint32_t mod_p2_mulhi(uint32_t a) {
#if defined(__CUDA_ARCH__)
  return a - (uint32_t)Prime<P>::p2 * __umulhi(a, Prime<P>::mod_magic);
#else
  return a - (uint32_t)Prime<P>::p2 * (uint32_t)(((uint64_t)a * Prime<P>::mod_magic) >> 32);
#endif
}

// Index of the highest set bit of x > 0.
__host__ __device__ inline int high_bit(unsigned x) {
#if defined(__CUDA_ARCH__)
  return 31 - __clz((int)x);
#else
  return 31 - __builtin_clz(x);
#endif
}

// floor(sqrt(x)) for 0 <= x < 2^30, digit by digit (integer arithmetic only).
__host__ __device__ inline int isqrt(int x) {
  if (x <= 0) return 0;
  int r = 0, bit = 1 << (high_bit((unsigned)x) & ~1);   // the highest power of four <= x
  while (bit != 0) {
    if (x >= r + bit) {
      x -= r + bit;
      r = (r >> 1) + bit;
    } else {
      r >>= 1;
    }
    bit >>= 2;
  }
  return r;
}

// floor(cbrt(x)) for 0 <= x < min(2^30, hi^3), by bisection.
__host__ __device__ inline int icbrt(int x, int hi = 1024) {
  int lo = 0;   // lo^3 <= x < hi^3
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)mid * mid * mid <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// SW table on the host (sizes, admission) -- same recurrence as the device copy.
inline int64_t host_sw(int u) {
  int64_t acc = 0;
  for (int v = 0; v < u; ++v) acc += colw(v + 1);
  return acc;
}
inline int64_t padded_words(int m) { return host_sw(m + 1); }

#if defined(__CUDACC__)
// Fill SW[0 .. n-1] in shared memory (n <= kSWLen); callers __syncthreads() afterwards.
__device__ __forceinline__ void build_sw(int *SW, int n) {
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int u = 0; u < n; ++u) {
      SW[u] = acc;
      acc += colw(u + 1);
    }
  }
}

// floor(x / m) for 0 <= x < 2^K m, m >= 1, by K compare-and-add steps (no division: a runtime divisor would be
// lowered through the floating-point reciprocal unit).
template <int K>
__host__ __device__ __forceinline__ int small_quotient(int x, int m) {
  int q = 0;
#pragma unroll
  for (int b = K - 1; b >= 0; --b)
    if (x >= (q + (1 << b)) * m) q += 1 << b;
  return q;
}

// Flat chunk index h of one slice (h = F(s) + c) -> column s and chunk c.  F(s) = E(s+4) - 4, so h + 4 is the
// flat index of chunk c of "column" s + 4 under E, which inverts in closed form.
__host__ __device__ inline void decode_chunk(int h, int &s, int &c) {
  h += 4;
  int q = (isqrt((h + 2) >> 1) - 1) >> 1;   // 8 q (q + 1) <= h, up to the corrections below
  if (q < 0) q = 0;
  while (8 * (q + 1) * (q + 2) <= h) ++q;
  while (q > 0 && 8 * q * (q + 1) > h) --q;
  const int rem = h - 8 * q * (q + 1);
  const int rr = small_quotient<4>(rem, q + 1);   // rem < 16 (q + 1)
  c = rem - rr * (q + 1);
  s = 16 * q + rr - 4;
}

// Flat chunk index k of a whole degree-m padded form -> (u, s, c); SW is the slice table (in words).
__device__ __forceinline__ void decode_form_chunk(int k, int m, const int *SW, int &u, int &s, int &c) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (SW[mid] <= 4 * k) lo = mid; else hi = mid - 1;
  }
  u = lo;
  decode_chunk(k - (SW[u] >> 2), s, c);
}

// Packed index i of a form (degree <= kMaxD) -> (u, s, t).
__host__ __device__ inline void decode_packed(int i, int &u, int &s, int &t, int max_deg = kMaxD) {
  // the slice u satisfies u^3 <= 6 tet(u) <= 6 i, and u <= max_deg for an index of a form of degree max_deg
  int uu = icbrt(6 * i, max_deg + 2);
  while (uu > 0 && tet(uu) > i) --uu;
  while (tet(uu + 1) <= i) ++uu;
  int rem = i - tet(uu);
  int ss = (isqrt(8 * rem + 1) - 1) >> 1;
  while (ss > 0 && tri(ss) > rem) --ss;
  while (tri(ss + 1) <= rem) ++ss;
  u = uu;
  s = ss;
  t = rem - tri(ss);
}
#endif

}  // namespace qfs
