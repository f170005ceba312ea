// Test helper (host code only): prints, as JSON, the index and sizing values that the CUDA kernels compute with
// their host-callable layout functions, so that tests/test_layout_host.py can check them on the CPU against
// sums and counts it forms itself.
#include <cstdio>

#include "qfs_kernels.cuh"

using namespace qfs;

template <int P>
void prime_line(bool last) {
  using Pr = Prime<P>;
  std::printf("\"%d\": {\"d\": %d, \"D\": %d, \"ld\": %d, \"lD\": %d, \"witness\": %d, \"stride\": %zu, "
              "\"smem_sweep\": %zu, \"smem_ring\": %zu, \"theta_ring_words\": %d}%s\n",
              P, Pr::d, Pr::D, Pr::ld, Pr::lD, Pr::witness, workspace_stride_words(P),
              smem_bytes_for(P, default_tile(P), false), smem_bytes_for(P, default_tile(P), true),
              theta_ring_words<P>(), last ? "" : ",");
}

// Mismatches of the integer index decoders against enumeration (all zero when they are right).
void decoder_lines() {
  long bad_sqrt = 0, bad_cbrt = 0, bad_half = 0, bad_chunk = 0, bad_packed = 0;
  for (long k = 0; k < 32768; ++k)
    for (long x = k * k - 1; x <= k * k + 1; ++x)
      if (x >= 0 && x < (1l << 30)) {
        const long r = isqrt((int)x);
        if (r * r > x || (r + 1) * (r + 1) <= x) ++bad_sqrt;
      }
  for (long k = 0; k < 1024; ++k)
    for (long x = k * k * k - 1; x <= k * k * k + 1; ++x)
      if (x >= 0 && x < (1l << 30)) {
        const long r = icbrt((int)x);
        if (r * r * r > x || (r + 1) * (r + 1) * (r + 1) <= x) ++bad_cbrt;
      }
  // half-chunk items of columns 0 .. kMaxD + 4, chunks of a slice of columns 0 .. kMaxD + 1, packed entries
  int i = 0;
  for (int s = 0; s <= kMaxD + 4; ++s)
    for (int h = 0; h < half_chunks_of(s); ++h, ++i) {
      int s2, h2;
      decode_half(i, s2, h2);
      if (s2 != s || h2 != h) ++bad_half;
    }
  i = 0;
  for (int s = 0; s <= kMaxD + 1; ++s)
    for (int c = 0; c < chunks_of(s); ++c, ++i) {
      int s2, c2;
      decode_chunk(i, s2, c2);
      if (s2 != s || c2 != c) ++bad_chunk;
    }
  i = 0;
  for (int u = 0; u <= kMaxD; ++u)
    for (int s = 0; s <= u; ++s)
      for (int t = 0; t <= s; ++t, ++i) {
        int u2, s2, t2;
        decode_packed(i, u2, s2, t2);
        if (u2 != u || s2 != s || t2 != t) ++bad_packed;
      }
  // the bounded form the kernels use for forms of degree 4 (reduced theta) and d = 4(p-1)
  const int degs[6] = {4, 8, 16, 24, 40, 48};
  for (int k = 0; k < 6; ++k) {
    int j = 0;
    for (int u = 0; u <= degs[k]; ++u)
      for (int s = 0; s <= u; ++s)
        for (int t = 0; t <= s; ++t, ++j) {
          int u2, s2, t2;
          decode_packed(j, u2, s2, t2, degs[k]);
          if (u2 != u || s2 != s || t2 != t) ++bad_packed;
        }
  }
  std::printf("\"decoder_mismatches\": {\"isqrt\": %ld, \"icbrt\": %ld, \"half\": %ld, \"chunk\": %ld, "
              "\"packed\": %ld, \"packed_entries\": %d},\n", bad_sqrt, bad_cbrt, bad_half, bad_chunk, bad_packed, i);
}

// Values a <= chain_max where the multiply-high reduction differs from a % p^2 (zero when it is exact).
template <int P>
long mod_mismatches() {
  long bad = 0;
  for (uint32_t a = 0; a <= Prime<P>::chain_max; ++a)
    if (mod_p2_mulhi<P>(a) != a % (uint32_t)Prime<P>::p2) ++bad;
  return bad;
}

int main() {
  std::printf("{\"max_d\": %d,\n", kMaxD);
  decoder_lines();
  std::printf("\"mod_mismatches\": [%ld, %ld, %ld, %ld, %ld],\n", mod_mismatches<3>(), mod_mismatches<5>(),
              mod_mismatches<7>(), mod_mismatches<11>(), mod_mismatches<13>());
  std::printf("\"chunks_of\": [");
  for (int s = 0; s <= kMaxD + 2; ++s) std::printf("%s%d", s ? "," : "", chunks_of(s));
  std::printf("],\n\"chunk_prefix\": [");
  for (int s = 0; s <= kMaxD + 2; ++s) std::printf("%s%d", s ? "," : "", chunk_prefix(s));
  std::printf("],\n\"half_prefix\": [");
  for (int s = 0; s <= kMaxD + 2; ++s) std::printf("%s%d", s ? "," : "", half_prefix(s));
  std::printf("],\n\"rcolw\": [");
  for (int s = 0; s <= 4 * (kMaxP - 1) + 2; ++s) std::printf("%s%d", s ? "," : "", rcolw(s));
  std::printf("],\n\"primes\": {\n");
  prime_line<3>(false);
  prime_line<5>(false);
  prime_line<7>(false);
  prime_line<11>(false);
  prime_line<13>(true);
  std::printf("}}\n");
  return 0;
}
