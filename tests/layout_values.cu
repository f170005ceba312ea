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

int main() {
  std::printf("{\"max_d\": %d,\n", kMaxD);
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
