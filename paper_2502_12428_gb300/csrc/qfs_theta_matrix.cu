// The theta matrix of a quartic (Sec. 3.4, the matrix form of Algorithm 3's step): M[r][c] = Delta[p r + (p-1)1 - c]
// for r, c in B_d (both in descending-lex order), with Delta = Delta_1(f^(p-1)) mod p and the entry zero when the
// index p r + (p-1)1 - c falls outside the degree-D cone.  theta(g) = M g (mod p) for every form g of degree d.
// The height pipeline never forms M (it produces theta(g) directly); this file exports it.
//
// Two kernels per batch of quartics: one CTA per quartic runs A1, A2, A4 and A5 unconditionally (the Fedder test
// does not stop it) into the CTA's workspace buffers and records which buffer holds Delta; then a grid fills the
// rows of every M from Delta.
#include <cuda_runtime.h>

#include "../../include/qfs.h"
#include "qfs_kernels.cuh"
#include "qfs_theta_matrix.cuh"

namespace qfs {
namespace {

template <int P>
__global__ void __launch_bounds__(kThreads, 1) theta_delta_kernel(const uint8_t *__restrict__ coeffs, uint32_t *ws,
                                                                  size_t stride, int *which, uint32_t *status) {
  using Pr = Prime<P>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  uint8_t *gs = smem_raw + sizeof(Smem);
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem_raw + ring_offset_for(Pr::ld));
  build_sw(sm.SW, Pr::D + 2);
  init_task_queue(sm);
  if (threadIdx.x == 0) {
    sm.tile_round = default_tile(P).round_chunks;
    sm.tile_ring = default_tile(P).ring_words;
    sm.dense_min = kDefaultDenseMin;
  }
  uint32_t *bufA, *bufB;
  cta_buffers(ws, stride, bufA, bufB);
  __syncthreads();
  DebugPtrs dbg{nullptr, nullptr, nullptr, nullptr};
  if (!setup_quartic<P>(coeffs + 35 * (size_t)blockIdx.x, sm)) {
    if (threadIdx.x == 0) which[blockIdx.x] = -1;   // a coefficient >= p: M is left zero
    return;
  }
  uint32_t *cur = power_to_g<P, QFS_FORM_DP4A, false>(sm, gs, ring, bufA, bufB, status, dbg);
  uint32_t *other = cur == bufA ? bufB : bufA;
  constexpr int nsteps = P * (P - 1) - (P - 1);   // products from f~^(p-1) to f~^(p(p-1))
  uint32_t *delta = (nsteps % 2) ? other : cur;
  power_to_G<P, QFS_FORM_DP4A, true, false>(sm, gs, ring, cur, other, nullptr, status, dbg);
  if (threadIdx.x == 0) which[blockIdx.x] = delta == bufA ? 0 : 1;
}

// M rows [blockIdx.x * kRows, ...) of quartic blockIdx.y.  Dynamic shared memory: SW (D+2 ints) and the (u, s, t) of
// every column index c (ld words).
constexpr int kRows = 8;

template <int P>
__global__ void __launch_bounds__(kThreads) theta_matrix_fill(const uint32_t *ws, size_t stride, const int *which,
                                                              uint8_t *M) {
  using Pr = Prime<P>;
  constexpr int d = Pr::d, D = Pr::D, ld = Pr::ld;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int *SW = reinterpret_cast<int *>(smem_raw);
  uint32_t *cst = reinterpret_cast<uint32_t *>(SW + D + 2);
  build_sw(SW, D + 2);
  for (int c = threadIdx.x; c < ld; c += blockDim.x) {
    int u, s, t;
    decode_packed(c, u, s, t, d);
    cst[c] = (uint32_t)u | ((uint32_t)s << 10) | ((uint32_t)t << 20);
  }
  __syncthreads();
  const int q = blockIdx.y;
  const int w = which[q];
  const uint8_t *delta = reinterpret_cast<const uint8_t *>(ws + kGuardWords + (2 * (size_t)q + (w > 0)) * stride);
  uint8_t *Mq = M + (size_t)q * ld * ld;
  const int r_end = min(ld, (int)(blockIdx.x + 1) * kRows);
  for (int r = blockIdx.x * kRows; r < r_end; ++r) {
    const uint32_t xr = cst[r];
    const int Ue = P * (int)(xr & 1023u) + 3 * (P - 1), Se = P * (int)((xr >> 10) & 1023u) + 2 * (P - 1),
              Te = P * (int)(xr >> 20) + (P - 1);
    for (int c = threadIdx.x; c < ld; c += blockDim.x) {
      uint8_t v = 0;
      if (w >= 0) {
        const uint32_t xc = cst[c];
        const int eu = Ue - (int)(xc & 1023u), es = Se - (int)((xc >> 10) & 1023u), et = Te - (int)(xc >> 20);
        if (et >= 0 && et <= es && es <= eu && eu <= D) v = delta[4 * ((size_t)SW[eu] + colw(es)) + et];
      }
      Mq[(size_t)r * ld + c] = v;
    }
  }
}

template <int P>
cudaError_t launch(const uint8_t *coeffs, int n, uint8_t *M, uint32_t *ws, size_t stride, int *which,
                   uint32_t *status, cudaStream_t st) {
  using Pr = Prime<P>;
  const size_t smem = smem_bytes_for(P, uses_ring_chain(QFS_FORM_DP4A, P));
  cudaError_t e = cudaFuncSetAttribute(theta_delta_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  theta_delta_kernel<P><<<n, kThreads, smem, st>>>(coeffs, ws, stride, which, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t fsmem = sizeof(int) * (Pr::D + 2) + sizeof(uint32_t) * Pr::ld;
  e = cudaFuncSetAttribute(theta_matrix_fill<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
  if (e != cudaSuccess) return e;
  const dim3 grid((Pr::ld + kRows - 1) / kRows, n);
  theta_matrix_fill<P><<<grid, kThreads, fsmem, st>>>(ws, stride, which, M);
  return cudaGetLastError();
}

}  // namespace

cudaError_t theta_matrix_launch(int p, const uint8_t *coeffs, int n, uint8_t *M, uint32_t *ws, size_t stride,
                                int *which, uint32_t *status, cudaStream_t st) {
  switch (p) {
    case 3: return launch<3>(coeffs, n, M, ws, stride, which, status, st);
    case 5: return launch<5>(coeffs, n, M, ws, stride, which, status, st);
    case 7: return launch<7>(coeffs, n, M, ws, stride, which, status, st);
    case 11: return launch<11>(coeffs, n, M, ws, stride, which, status, st);
    default: return launch<13>(coeffs, n, M, ws, stride, which, status, st);
  }
}

}  // namespace qfs
