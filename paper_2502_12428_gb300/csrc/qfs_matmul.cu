// Matrix multiplication mod p on the int8 tensor cores (the paper's Sec. 5 workload: square matrices mod 11 of
// size 5,000 .. 20,000).  C = A B mod p for A (n x k), B (k x m), C (n x m), all uint8 row-major with values in
// [0, p).  Products of residues below 256 accumulate exactly in int32 (mma.sync m16n8k32, u8 x u8 -> s32), so the
// only reduction is the final one, plus one every few K tiles when k (p-1)^2 could reach 2^31.
//
// Layout: a pack kernel writes A and the transpose of B into scratch matrices with K padded to a multiple of 64 and
// 16-byte aligned rows; the GEMM then multiplies A_pad (n x kp) by Bt_pad (m x kp)^T.  CTA tile 128 x 128, K tile 64
// bytes, three cp.async stages in shared memory (16-byte chunks, XOR-swizzled so that ldmatrix reads without bank
// conflicts), 8 warps of 64 x 32 outputs each.
#include <cuda_runtime.h>

#include <cstdint>

#include "qfs_matmul.cuh"

namespace qfs {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64, kStages = 3, kMMThreads = 256;
constexpr int kTileBytes = kBM * kBK;   // one operand tile of one stage (same for A and B: kBM == kBN)

__device__ __forceinline__ void cp16(uint32_t smem, const void *g, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem), "l"(g), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}
__device__ __forceinline__ void mma_u8(int (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// byte offset of (row, 16-byte chunk) inside a 128 x 64-byte tile: rows of 4 chunks, chunk index XOR (row/2) % 4
__device__ __forceinline__ int swz(int row, int chunk) { return row * kBK + ((chunk ^ ((row >> 1) & 3)) << 4); }

// Pack: A_pad[i][kk] = A[i][kk] (kk < k, else 0); Bt_pad[j][kk] = B[kk][j] (kk < k, else 0).  32 x 32 byte tiles
// through shared memory so that both the reads of B and the writes of Bt_pad are coalesced.
__global__ void pack_kernel(const uint8_t *__restrict__ A, const uint8_t *__restrict__ B, int n, int m, int k,
                            int kp, uint8_t *__restrict__ Ap, uint8_t *__restrict__ Btp) {
  __shared__ uint8_t t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
  const int kk0 = blockIdx.x * 32;
  if (blockIdx.z == 0) {
    // A rows blockIdx.y * 32 .. +31, columns kk0 .. kk0+31
    for (int r = ty; r < 32; r += 8) {
      const int i = blockIdx.y * 32 + r, kk = kk0 + tx;
      if (i < n && kk < kp) Ap[(size_t)i * kp + kk] = kk < k ? A[(size_t)i * k + kk] : 0;
    }
  } else {
    // B rows kk0 .. kk0+31, columns j0 .. j0+31 -> Bt_pad rows j, columns kk
    const int j0 = blockIdx.y * 32;
    for (int r = ty; r < 32; r += 8) {
      const int kk = kk0 + r, j = j0 + tx;
      t[r][tx] = (kk < k && j < m) ? B[(size_t)kk * m + j] : 0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
      const int j = j0 + r, kk = kk0 + tx;
      if (j < m && kk < kp) Btp[(size_t)j * kp + kk] = t[tx][r];
    }
  }
}

__global__ void __launch_bounds__(kMMThreads, 2) matmul_kernel(const uint8_t *__restrict__ Ap,
                                                                const uint8_t *__restrict__ Btp, uint8_t *C, int n,
                                                                int m, int kp, int p, int reduce_every) {
  extern __shared__ __align__(128) uint8_t smem[];   // kStages x (A tile, B tile)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;            // warp tile: rows wm*64 .. +63, columns wn*32 .. +31
  const int i0 = blockIdx.y * kBM, j0 = blockIdx.x * kBN;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  const int ntiles = kp / kBK;

  // one stage: 128 rows x 4 chunks for A and for B = 1024 chunks, 4 per thread
  auto load_stage = [&](int kt, int stage) {
    const uint32_t sa = sbase + stage * 2 * kTileBytes, sb = sa + kTileBytes;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + q * kMMThreads;   // 0 .. 1023
      const int isB = idx >> 9, row = (idx >> 2) & 127, ch = idx & 3;
      const int grow = (isB ? j0 : i0) + row;
      const bool ok = grow < (isB ? m : n);
      const uint8_t *src = (isB ? Btp : Ap) + (size_t)(ok ? grow : 0) * kp + kt * kBK + ch * 16;
      cp16((isB ? sb : sa) + swz(row, ch), src, ok);
    }
  };

  int acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0;

#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    if (s < ntiles) load_stage(s, s);
    asm volatile("cp.async.commit_group;\n" ::);
  }
  for (int kt = 0; kt < ntiles; ++kt) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kStages - 2));
    __syncthreads();   // stage kt % kStages is complete; the stage refilled below was last read in tile kt - 1
    if (kt + kStages - 1 < ntiles) load_stage(kt + kStages - 1, (kt + kStages - 1) % kStages);
    asm volatile("cp.async.commit_group;\n" ::);
    const uint32_t sa = sbase + (kt % kStages) * 2 * kTileBytes, sb = sa + kTileBytes;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {   // two k32 steps per 64-byte tile
      uint32_t af[4][4], bf[4][2];
      // A fragments: 16 x 32-byte blocks; lane l reads row (l & 15), chunk 2 ks + (l >> 4)
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int row = wm * 64 + mt * 16 + (lane & 15);
        const int ch = 2 * ks + (lane >> 4);
        uint32_t r0, r1, r2, r3;
        ldsm_x4(sa + swz(row, ch), r0, r1, r2, r3);
        // matrices: 0 = rows 0-7 k 0-15, 1 = rows 8-15 k 0-15, 2 = rows 0-7 k 16-31, 3 = rows 8-15 k 16-31
        af[mt][0] = r0; af[mt][1] = r1; af[mt][2] = r2; af[mt][3] = r3;
      }
      // B fragments: two n8 tiles per ldmatrix.x4; lane l reads row (l & 7) + 8 ((l >> 4) & 1), chunk 2 ks + ((l >> 3) & 1)
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int row = wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
        const int ch = 2 * ks + ((lane >> 3) & 1);
        uint32_t r0, r1, r2, r3;
        ldsm_x4(sb + swz(row, ch), r0, r1, r2, r3);
        bf[2 * np][0] = r0; bf[2 * np][1] = r1; bf[2 * np + 1][0] = r2; bf[2 * np + 1][1] = r3;
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_u8(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
    }
    if (reduce_every > 0 && (kt + 1) % reduce_every == 0) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][b][c] = (int)((unsigned)acc[a][b][c] % (unsigned)p);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
  // C fragment of tile (mt, nt): c0, c1 at row g, columns 2 tig, 2 tig + 1; c2, c3 at row g + 8
  const int g = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = i0 + wm * 64 + mt * 16 + g + 8 * h;
        const int j = j0 + wn * 32 + nt * 8 + 2 * tig;
        if (i < n) {
          if (j < m) C[(size_t)i * m + j] = (uint8_t)((unsigned)acc[mt][nt][2 * h] % (unsigned)p);
          if (j + 1 < m) C[(size_t)i * m + j + 1] = (uint8_t)((unsigned)acc[mt][nt][2 * h + 1] % (unsigned)p);
        }
      }
}

}  // namespace

size_t matmul_scratch_bytes(int n, int m, int k) {
  const size_t kp = ((size_t)k + kBK - 1) / kBK * kBK;
  return kp * ((size_t)n + (size_t)m) + 256;
}

cudaError_t matmul_mod_launch(int p, int n, int m, int k, const uint8_t *A, const uint8_t *B, uint8_t *C,
                              uint8_t *scratch, cudaStream_t st) {
  const int kp = (k + kBK - 1) / kBK * kBK;
  uint8_t *Ap = scratch;
  uint8_t *Btp = scratch + (((size_t)kp * n + 255) & ~(size_t)255);
  const dim3 pgrid(kp / 32, (unsigned)((n > m ? n : m) + 31) / 32, 2);
  pack_kernel<<<pgrid, 256, 0, st>>>(A, B, n, m, k, kp, Ap, Btp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // K tiles between reductions: the int32 accumulator stays below 2^31 (a reduced residue plus the new products)
  const long long per_tile = (long long)kBK * (p - 1) * (p - 1);
  const long long tiles_ok = per_tile > 0 ? (0x7fffffffLL - p) / per_tile : (1LL << 30);
  const int reduce_every = (long long)(kp / kBK) <= tiles_ok ? 0 : (int)(tiles_ok > 0 ? tiles_ok : 1);
  const size_t smem = (size_t)kStages * 2 * kTileBytes;
  e = cudaFuncSetAttribute(matmul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((m + kBN - 1) / kBN, (n + kBM - 1) / kBM);
  matmul_kernel<<<grid, kMMThreads, smem, st>>>(Ap, Btp, C, n, m, kp, p, reduce_every);
  return cudaGetLastError();
}

}  // namespace qfs
