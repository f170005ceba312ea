// Height-1 screen of a batch (Algorithm 3, first test; Fedder's criterion, Sec. 3): h = 1 iff the coefficient of
// (x1 x2 x3 x4)^(p-1) in f^(p-1) is nonzero mod p.  Most quartics stop there (about 84 % of dense quartics at
// p = 7), so the batch is screened before the persistent launch, one warp per quartic, and only the survivors reach
// the CTA-wide pipeline (which repeats the test on its own f^(p-1) mod p^2, with the same outcome).
//
// With k = (p-1)/2, f^(p-1) = F * F for F = f^k, so the coefficient is sum_a F[a] F[(p-1)1 - a] over the
// monomials a of degree 2(p-1) whose four exponents are all <= p-1 (exactly the a for which (p-1)1 - a is a
// monomial).  F is formed mod p by k-1 products with f in the warp's shared memory: in cone coordinates
// (u, s, t) = (e2+e3+e4, e3+e4, e4) a product of forms is a 3-D convolution over the cone t <= s <= u <= degree.
#include <cuda_runtime.h>

#include "qfs_layout.cuh"
#include "qfs_screen.cuh"

namespace qfs {
namespace {

constexpr int kScreenWarps = kScreenThreads / 32;

// Bytes of one warp's region for primes up to max_p: f (35, padded to 48) and two buffers of C(4k+3, 3).
__host__ __device__ constexpr int screen_buf_bytes(int max_p) {
  return (tet(4 * ((max_p - 1) / 2) + 1) + 15) & ~15;
}
__host__ __device__ constexpr int screen_warp_bytes(int max_p) { return 48 + 2 * screen_buf_bytes(max_p); }

// (s, t) of entry i of a slice (entries ordered by s, then t <= s).
__device__ __forceinline__ void decode_slice_entry(int i, int &s, int &t) {
  s = (isqrt(8 * i + 1) - 1) >> 1;
  while (tri(s + 1) <= i) ++s;
  while (s > 0 && tri(s) > i) --s;
  t = i - tri(s);
}

// out = in * f mod p, in of degree m (packed), out of degree m + 4; the warp's lanes split every slice.
template <int P>
__device__ void warp_times_f(const uint8_t *in, int m, uint8_t *out, const uint8_t *f, int lane) {
  const int M = m + 4;
  for (int u = 0; u <= M; ++u) {
    const int n = tri(u + 1);
    int s, t;
    decode_slice_entry(lane, s, t);
    for (int i = lane; i < n; i += 32, t += 32) {
      while (t > s) t -= ++s;   // entry i = tri(s) + t: advance (s, t) by the 32 entries since the last one
      int acc = 0;
#pragma unroll
      for (int uI = 0; uI <= 4; ++uI) {
        const int ui = u - uI;
        if (ui < 0 || ui > m) continue;
#pragma unroll
        for (int sI = 0; sI <= uI; ++sI) {
          const int si = s - sI;
          if (si < 0 || si > ui) continue;
#pragma unroll
          for (int tI = 0; tI <= sI; ++tI) {
            const int ti = t - tI;
            if (ti < 0 || ti > si) continue;
            acc += (int)f[tet(uI) + tri(sI) + tI] * (int)in[tet(ui) + tri(si) + ti];
          }
        }
      }
      out[tet(u) + tri(s) + t] = (uint8_t)(acc % P);
    }
  }
  __syncwarp();
}

// Screens one row with the calling warp; returns -1 (a coefficient >= p), 1 (height 1) or 0 (survivor), same in
// every lane.
template <int P>
__device__ int screen_row(const uint8_t *__restrict__ f35, uint8_t *wsm, int lane) {
  constexpr int k = (P - 1) / 2;
  uint8_t *f = wsm;
  uint8_t *A = wsm + 48;
  uint8_t *B = A + screen_buf_bytes(P);
  int bad = 0;
  for (int i = lane; i < 35; i += 32) {
    const int a = f35[i];
    bad |= a >= P;
    f[i] = (uint8_t)a;
  }
  if (__any_sync(0xffffffffu, bad)) return -1;
  __syncwarp();
  // F = f^k: f itself is the degree-4 form, then k - 1 products
  const uint8_t *F = f;
  for (int j = 1; j < k; ++j) {
    uint8_t *dst = (j & 1) ? A : B;
    warp_times_f<P>(F, 4 * j, dst, f, lane);
    F = dst;
  }
  // coefficient of (x1 x2 x3 x4)^(p-1) in F * F
  constexpr int m = 2 * (P - 1);
  int acc = 0;
  for (int i = lane; i < tet(m + 1); i += 32) {
    // (u, s, t) of packed entry i of degree m
    int u = 0;
    while (tet(u + 1) <= i) ++u;
    int s, t;
    decode_slice_entry(i - tet(u), s, t);
    const int e1 = m - u, e2 = u - s, e3 = s - t, e4 = t;
    if (e1 <= P - 1 && e2 <= P - 1 && e3 <= P - 1 && e4 <= P - 1) {
      const int ub = 3 * (P - 1) - u, sb = 2 * (P - 1) - s, tb = (P - 1) - t;
      acc += (int)F[i] * (int)F[tet(ub) + tri(sb) + tb];
    }
  }
  acc = __reduce_add_sync(0xffffffffu, acc);
  return (acc % P) != 0 ? 1 : 0;
}

__global__ void __launch_bounds__(kScreenThreads) screen_kernel(FusedParams prm, int warp_bytes, int64_t *list,
                                                                unsigned long long *n_list) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint8_t *wsm = smem_raw + (size_t)warp * warp_bytes;
  const int64_t stride = (int64_t)gridDim.x * kScreenWarps;
  for (int64_t item = (int64_t)blockIdx.x * kScreenWarps + warp; item < prm.n_items; item += stride) {
    int gi = 0;
    while (gi + 1 < prm.n_groups && item >= prm.g[gi + 1].item_begin) ++gi;
    const FusedGroup &G = prm.g[gi];
    const int64_t row = item - G.item_begin;
    const uint8_t *f = G.coeffs + 35 * row;
    int r;
    switch (G.p) {
      case 3: r = screen_row<3>(f, wsm, lane); break;
      case 5: r = screen_row<5>(f, wsm, lane); break;
      case 7: r = screen_row<7>(f, wsm, lane); break;
      case 11: r = screen_row<11>(f, wsm, lane); break;
      default: r = screen_row<13>(f, wsm, lane); break;
    }
    if (lane == 0) {
      if (r != 0) G.heights[row] = (int8_t)r;
      else list[atomicAdd(n_list, 1ull)] = item;
    }
    __syncwarp();
  }
}

}  // namespace

size_t screen_smem_bytes(int max_p) { return (size_t)kScreenWarps * screen_warp_bytes(max_p); }

cudaError_t screen_launch(const FusedParams &prm, int max_p, int64_t *list, unsigned long long *n_list,
                          int grid_ctas, cudaStream_t st) {
  const size_t smem = screen_smem_bytes(max_p);
  cudaError_t e = cudaFuncSetAttribute(screen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  screen_kernel<<<grid_ctas, kScreenThreads, smem, st>>>(prm, screen_warp_bytes(max_p), list, n_list);
  return cudaGetLastError();
}

}  // namespace qfs
