// Staged engine: one kernel per stage of the height computation, over chunks of quartics.
//
//   stage_fedder   A1-A3: f^(p-1) and the height-1 test for every quartic of the chunk; survivors are appended to a
//                  list (their height is written later), every other row gets 1 or -1 here
//   stage_power    A4: the chain to G = f~^(p(p-1)) mod p^2 for every survivor, written to its G slot, and
//                  g = f^(p-1) mod p to its g slot
//   stage_delta1   A5: Delta = (G - S) / p mod p, elementwise over all survivors' G slots (in place)
//   stage_theta    A6: one theta step g -> u(Delta g) for every survivor still undecided
//   stage_test     A7: witness test, zero test and the max_h bound; writes heights and retires survivors
//
// The stages compute exactly what the fused engine computes (same device functions), so heights agree bit for bit.
// This engine exists so that each stage can be profiled as its own kernel; the fused engine is faster.  Every
// kernel reads the survivor count from device memory, so the host enqueues a fixed sequence per chunk and never
// synchronises (the sequence can be captured in a CUDA graph once the workspace exists).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/qfs.h"
#include "qfs_kernels.cuh"
#include "qfs_staged.cuh"

namespace qfs {

namespace {

constexpr int kForm = 1;  // dp4a

struct StagedChunk {
  const uint8_t *coeffs;   // chunk rows
  int8_t *heights;
  int n;
  int max_h;
  unsigned *count;         // survivors in this chunk
  unsigned *queue;         // work-queue head of the current persistent kernel
  int *rows;               // survivor -> row in the chunk
  uint8_t *active;         // survivor still undecided
  uint32_t *G;             // survivor slots of padded words (degree D): G, then Delta
  uint8_t *gA, *gB;        // survivor slots of ld bytes: current iterate and the next one
  uint32_t *ws;            // per-CTA ping-pong buffers (fedder and power)
  size_t ws_words;
  unsigned long long *stats;
  uint32_t *status;
};

template <int P>
__device__ __forceinline__ void stage_smem(Smem *&sm, uint8_t *&gs, uint8_t *&gn, uint32_t *&ring) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sm = reinterpret_cast<Smem *>(smem_raw);
  if (threadIdx.x == 0) {
    sm->tile_round = default_tile(P).round_chunks;
    sm->tile_ring = default_tile(P).ring_words;
    sm->dense_min = kDefaultDenseMin;
  }
  gs = smem_raw + sizeof(Smem);
  gn = gs + Prime<P>::ld;
  ring = reinterpret_cast<uint32_t *>(smem_raw + ring_offset_for(Prime<P>::ld));
}

template <int P>
__global__ void __launch_bounds__(kThreads, 2) stage_fedder(StagedChunk c) {
  Smem *sm; uint8_t *gs, *gn; uint32_t *ring;
  stage_smem<P>(sm, gs, gn, ring);
  build_sw(sm->SW, Prime<P>::D + 2);
  init_task_queue(*sm);
  uint32_t *bufA, *bufB;
  cta_buffers(c.ws, c.ws_words, bufA, bufB);
  DebugPtrs dbg{nullptr, nullptr, nullptr, nullptr};
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sm->item = atomicAdd(c.queue, 1u);
    __syncthreads();
    const int row = (int)sm->item;
    if (row >= c.n) break;
    if (!setup_quartic<P>(c.coeffs + 35 * (size_t)row, *sm)) {
      if (threadIdx.x == 0) c.heights[row] = -1;
      continue;
    }
    power_to_g<P, kForm, false>(*sm, gs, ring, bufA, bufB, c.status, dbg);
    if (threadIdx.x == 0) {
      if (gs[Prime<P>::witness] != 0) {
        c.heights[row] = 1;
      } else if (c.max_h == 1) {
        c.heights[row] = 0;
      } else {
        const unsigned slot = atomicAdd(c.count, 1u);
        c.rows[slot] = row;
        c.active[slot] = 1;
        atomicAdd(c.stats, 1ull);
      }
    }
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads, 2) stage_power(StagedChunk c) {
  using Pr = Prime<P>;
  Smem *sm; uint8_t *gs, *gn; uint32_t *ring;
  stage_smem<P>(sm, gs, gn, ring);
  build_sw(sm->SW, Pr::D + 2);
  init_task_queue(*sm);
  uint32_t *bufA, *bufB;
  cta_buffers(c.ws, c.ws_words, bufA, bufB);
  DebugPtrs dbg{nullptr, nullptr, nullptr, nullptr};
  const unsigned total = *c.count;
  const size_t gwords = c.ws_words;  // slot stride (at least the padded words of degree D)
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sm->item = atomicAdd(c.queue, 1u);
    __syncthreads();
    const unsigned slot = (unsigned)sm->item;
    if (slot >= total) break;
    setup_quartic<P>(c.coeffs + 35 * (size_t)c.rows[slot], *sm);
    uint32_t *cur = power_to_g<P, kForm, false>(*sm, gs, ring, bufA, bufB, c.status, dbg);
    for (int i = threadIdx.x; i < Pr::ld; i += blockDim.x) c.gA[(size_t)slot * Pr::ld + i] = gs[i];
    power_to_G<P, kForm, false, false>(*sm, gs, ring, cur, cur == bufA ? bufB : bufA, c.G + slot * gwords,
                                       c.status, dbg);
  }
}

// Elementwise: one thread per 16-byte chunk of one survivor's G.
template <int P>
__global__ void __launch_bounds__(kThreads) stage_delta1(StagedChunk c) {
  using Pr = Prime<P>;
  __shared__ int SW[Pr::D + 2];
  __shared__ int powp[P];
  build_sw(SW, Pr::D + 2);
  if (threadIdx.x < P) {
    int v = 1;
    for (int e = 0; e < P; ++e) v = (v * (int)threadIdx.x) % Pr::p2;
    powp[threadIdx.x] = v;
  }
  __syncthreads();
  const unsigned total = *c.count;
  const size_t gwords = c.ws_words;            // stride of the G slots
  const size_t chunks = (size_t)SW[Pr::D + 1] / 4;  // 16-byte chunks of a degree-D form (the slot may be longer)
  bool bad = false;
  // slots by block, chunks by thread (no 64-bit division of a flat index)
  for (size_t slot = blockIdx.x; slot < total; slot += gridDim.x)
  for (size_t k = threadIdx.x; k < chunks; k += blockDim.x) {
    int u, s, ch;
    decode_form_chunk((int)k, Pr::D, SW, u, s, ch);
    uint4 *p4 = reinterpret_cast<uint4 *>(c.G + slot * gwords + 4 * k);
    const uint4 v = *p4;
    uint32_t words[4] = {v.x, v.y, v.z, v.w};
    const uint8_t *g = c.gA + slot * Pr::ld;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      uint32_t outw = 0;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int t = 16 * ch + 4 * w + b;
        int G = (int)((words[w] >> (8 * b)) & 0xFFu);
        if (t <= s && (u % P) == 0 && (s % P) == 0 && (t % P) == 0) {
          G -= powp[g[tet(u / P) + tri(s / P) + t / P]];
          if (G < 0) G += Pr::p2;
        }
        if (G % P) bad = true;
        outw |= (uint32_t)(G / P) << (8 * b);
      }
      words[w] = outw;
    }
    *p4 = make_uint4(words[0], words[1], words[2], words[3]);
  }
  if (bad) atomicOr(c.status, kStatusInexactDivision);
}

// One CTA per undecided survivor: g (gin slot) -> theta(g) (gout slot).
template <int P>
__global__ void __launch_bounds__(kThreads, 2) stage_theta(StagedChunk c, const uint8_t *gin, uint8_t *gout) {
  using Pr = Prime<P>;
  Smem *sm; uint8_t *gs, *gn; uint32_t *ring;
  stage_smem<P>(sm, gs, gn, ring);
  build_sw(sm->SW, Pr::D + 2);
  init_task_queue(*sm);
  uint32_t *dg, *unused;
  cta_buffers(c.ws, c.ws_words, dg, unused);  // the guarded copy of the survivor's Delta
  __syncthreads();
  const unsigned total = *c.count;
  const size_t gwords = c.ws_words;  // slot stride (at least the padded words of degree D)
  for (unsigned slot = blockIdx.x; slot < total; slot += gridDim.x) {
    if (!c.active[slot]) continue;
    for (int i = threadIdx.x; i < Pr::ld; i += blockDim.x) gs[i] = gin[(size_t)slot * Pr::ld + i];
    if constexpr (theta_streams<P>()) {
      __syncthreads();
      theta_stream<P>(c.G + slot * gwords, *sm, gs, gn, ring);
    } else if constexpr (theta_by_classes<P>()) {
      unsigned char *ringb = reinterpret_cast<unsigned char *>(ring);
      poly_tables<P>(ringb);
      delta_to_classes<P>(c.G + slot * gwords, dg, *sm, ringb);
      __syncthreads();
      theta_poly<P>(dg, gs, gn, ringb);
    } else {
      delta_to_guarded<P>(c.G + slot * gwords, dg, *sm);
      __syncthreads();
      theta_gather<P>(dg, *sm, gs, gn, ring);
    }
    for (int i = threadIdx.x; i < Pr::ld; i += blockDim.x) gout[(size_t)slot * Pr::ld + i] = gn[i];
    if (threadIdx.x == 0) atomicAdd(c.stats + 1, 1ull);
    __syncthreads();
  }
}

// One warp per undecided survivor: the iterate g_h in `g` decides height h, infinity, or another step.
template <int P>
__global__ void __launch_bounds__(kThreads) stage_test(StagedChunk c, const uint8_t *g, int h) {
  using Pr = Prime<P>;
  const unsigned total = *c.count;
  const int lane = threadIdx.x & 31;
  for (unsigned slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; slot < total;
       slot += (gridDim.x * blockDim.x) >> 5) {
    if (!c.active[slot]) continue;
    const uint8_t *gs = g + (size_t)slot * Pr::ld;
    bool nz = false;
    for (int i = lane; i < Pr::ld; i += 32) nz |= gs[i] != 0;
    nz = __any_sync(0xffffffffu, nz);
    if (lane == 0) {
      int8_t out = -2;
      if (gs[Pr::witness] != 0) out = (int8_t)h;
      else if (!nz || h == c.max_h) out = 0;
      if (out != -2) {
        c.heights[c.rows[slot]] = out;
        c.active[slot] = 0;
      }
    }
  }
}

template <int P>
cudaError_t run_chunks(const StagedPlan &pl, const uint8_t *coeffs, int8_t *heights, int64_t n, int max_h,
                       cudaStream_t st) {
  using Pr = Prime<P>;
  const size_t smem = smem_bytes_for(P, uses_ring_chain(QFS_FORM_DP4A, P));
  cudaError_t e;
  for (auto k : {(const void *)stage_fedder<P>, (const void *)stage_power<P>, (const void *)stage_theta<P>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  for (int64_t r0 = 0; r0 < n; r0 += pl.chunk) {
    StagedChunk c;
    c.coeffs = coeffs + 35 * r0;
    c.heights = heights + r0;
    c.n = (int)std::min<int64_t>(pl.chunk, n - r0);
    c.max_h = max_h;
    c.count = pl.counters;
    c.queue = pl.counters + 1;
    c.rows = pl.rows;
    c.active = pl.active;
    c.G = pl.G;
    c.gA = pl.gA;
    c.gB = pl.gB;
    c.ws = pl.ws;
    c.ws_words = pl.ws_words;
    c.stats = pl.stats;
    c.status = pl.status;
    if ((e = cudaMemsetAsync(pl.counters, 0, 2 * sizeof(unsigned), st)) != cudaSuccess) return e;
    stage_fedder<P><<<pl.grid, kThreads, smem, st>>>(c);
    if ((e = cudaMemsetAsync(pl.counters + 1, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    stage_power<P><<<pl.grid, kThreads, smem, st>>>(c);
    stage_delta1<P><<<pl.sms * 8, kThreads, 0, st>>>(c);
    uint8_t *gin = pl.gA, *gout = pl.gB;
    for (int h = 2; h <= max_h; ++h) {
      stage_theta<P><<<pl.grid, kThreads, smem, st>>>(c, gin, gout);
      stage_test<P><<<pl.sms * 4, kThreads, 0, st>>>(c, gout, h);
      std::swap(gin, gout);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

size_t staged_survivor_bytes(int p) {
  const int ld = tet(4 * (p - 1) + 1);
  return workspace_stride_words(p) * 4 + 2 * (size_t)ld + sizeof(int) + 1;
}

cudaError_t staged_run(const StagedPlan &pl, int p, const uint8_t *coeffs, int8_t *heights, int64_t n, int max_h,
                       cudaStream_t st) {
  switch (p) {
    case 3: return run_chunks<3>(pl, coeffs, heights, n, max_h, st);
    case 5: return run_chunks<5>(pl, coeffs, heights, n, max_h, st);
    case 7: return run_chunks<7>(pl, coeffs, heights, n, max_h, st);
    case 11: return run_chunks<11>(pl, coeffs, heights, n, max_h, st);
    default: return run_chunks<13>(pl, coeffs, heights, n, max_h, st);
  }
}

cudaError_t staged_occupancy(int p, int *blocks) {
  const size_t smem = smem_bytes_for(p, uses_ring_chain(QFS_FORM_DP4A, p));
  const void *k = p == 3 ? (const void *)stage_power<3> : p == 5 ? (const void *)stage_power<5>
                : p == 7 ? (const void *)stage_power<7> : p == 11 ? (const void *)stage_power<11>
                : (const void *)stage_power<13>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, kThreads, smem);
}

}  // namespace qfs
