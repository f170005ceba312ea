// Per-quartic device pipeline of the quasi-F-split height (paper Sec. 3; Algorithms 1-3 and the matrix form of
// Sec. 3.4), executed by one CTA per quartic.
//
//   A1  read the 35 coefficients, reject values >= p (height code -1)
//   A2  chain f~^(k+1) = f~^k * f~ mod p^2 up to k+1 = p-1                    (power kernel, "multiply by f")
//   A3  height 1 iff the coefficient of (x1..x4)^(p-1) in f^(p-1) is nonzero mod p   (Fedder's criterion)
//   A4  continue the chain to G = f~^(p(p-1)) mod p^2.  G = lift(g)^p mod p^2 for g = f^(p-1) mod p, because
//       (c + p b)^p = c^p mod p^2: Algorithm 1's "D <- lift^p" only depends on g mod p.
//   A5  Delta = (G - S) / p mod p with S[pJ] = (lift c_J)^p mod p^2 for the terms c_J x^J of g   (Algorithm 1)
//   A6  theta: out[r] = sum_c Delta[p r + (p-1,..,p-1) - c] g[c] mod p -- the part of Delta*g that the splitting
//       u keeps (Algorithm 2), produced directly; the matrix of Sec. 3.4 is never formed
//   A7  test out[witness]; zero iterate -> infinity (theta is linear); h = max_h -> infinity
//
// Residues mod p^2 are stored as one byte each (p <= 13: p^2 - 1 <= 168) in the padded layout of
// qfs_layout.cuh, and f's coefficients are lifted to [0, p).  One chain output sums at most 35 products of a
// residue (< p^2) and a coefficient (< p): 35 * 168 * 12 = 70,560 for p = 13, far inside int32 -- every form
// reduces once per output.  Theta sums at most C(4p-1,3) products below p^2: 20,825 * 144 < 2^31.
#pragma once
#include <algorithm>
#include <cstdint>
#include "qfs_layout.cuh"
#include "qfs_common.cuh"
#include "qfs_sweep.cuh"

namespace qfs {

// ------------------------------------------------------------------------------------------------ chain step
// out := in * f (mod p^2), in of degree m_in, out of degree m_in + 4 (one product of the chain).  When LAST, the
// Delta_1 epilogue turns G into Delta and writes residues mod p.
//
// Tiling.  Output columns are taken in blocks of 32 (s0 .. s0+31) and each block sweeps the slices u = s0 .. m_out,
// UPAR slices per round.  Output slice u reads input slices u-4 .. u (uI = 4 - i1) and columns s-4 .. s, so a ring
// of shared-memory slots holds input slices restricted to columns s0-4 .. s0+31, zero-filled outside the input
// cone: the inner loop has no bounds checks.  The next UPAR slices stream in with 16-byte cp.async while the
// current ones are computed.  Work items are flat: one lane = one (column, 16-byte chunk) pair of the round, so
// columns that do not exist yet in a slice (s > u) cost nothing.  A slot column holds chunk 0 = zeros (input words
// -4..-1) followed by the column's chunks, so output chunk c reads slot chunks c and c+1 (input words 4c-4..4c+3).
// Outputs past a column's end come out as zero by themselves (their inputs are all padding), so no output needs a
// bounds check outside the Delta_1 epilogue.
// Tile shape of the chain (per prime; the autotuner may change it at run time):
//   round_chunks  target (column, chunk) items per round: UPAR = ceil(round_chunks / chunks per slice), at most 8
//   ring_words    shared-memory words the slot ring may use (UPAR shrinks until 2 UPAR + 4 slots fit)
constexpr int kMaxUpar = 8;
constexpr int kDefaultRoundChunks = 512;
constexpr int kRingBudgetSmallP = 16384;   // default ring words for p <= 7 (64 KB)
constexpr int kRingBudgetLargeP = 26624;   // default ring words for p >= 11 (104 KB)

struct TileConfig {
  int round_chunks;
  int ring_words;
};

// Swept-chain launch shape of one prime and form (dp4a, int32): dense_min = nonzero tap pairs (of 15) from which
// a quartic takes the every-pair path (16: never), ctas_per_sm = CTAs per SM of the fused launch (0: as many as
// fit).  Results never depend on either.
constexpr int kDefaultDenseMin = 12;
struct SweepConfig {
  int dense_min;
  int ctas_per_sm;
};

__host__ __device__ inline TileConfig default_tile(int p) {
  return TileConfig{kDefaultRoundChunks, p <= 7 ? kRingBudgetSmallP : kRingBudgetLargeP};
}

struct ChainTile {
  int CR, stride, slot_words, upar, nslot;
};

__host__ __device__ inline ChainTile chain_tile(int s0, int m_out, TileConfig tc) {
  ChainTile T;
  const int s_hi = min(s0 + 31, m_out);
  T.CR = chunks_of(s_hi);
  T.stride = 4 * (T.CR + 1);
  T.slot_words = 36 * T.stride;
  const int per_slice = chunk_prefix(s_hi + 1) - chunk_prefix(s0);
  int up = 1;   // ceil(round_chunks / per_slice), at most kMaxUpar, counted up (no runtime division)
  while (up < kMaxUpar && up * per_slice < tc.round_chunks) ++up;
  while (up > 1 && (2 * up + 4) * T.slot_words > tc.ring_words) --up;
  T.upar = up;
  T.nslot = 2 * up + 4;
  return T;
}

// Shared-memory words the ring needs over every product of the chain for prime p under tile config tc.
__host__ __device__ inline int chain_slot_words(int p, TileConfig tc) {
  const int D = 4 * p * (p - 1);
  int best = 0;
  for (int m_out = 8; m_out <= D; m_out += 4)
    for (int s0 = 0; s0 <= m_out; s0 += 32) {
      const ChainTile T = chain_tile(s0, m_out, tc);
      best = max(best, T.nslot * T.slot_words);
    }
  return best;
}

__host__ __device__ inline int theta_ring_words_for(int p, int power = -1);

// Ring words the identity and reduced power modes need: three byte arrays (f^(p-2), Delta_1(f), E), and in the
// reduced mode a product to degree 4p whose own slot ring (int8 tensor form only) starts after f^(p-2),
// Delta_1(f) and q.
__host__ __device__ inline int aux_ring_words(int p, TileConfig tc, bool ring_chain) {
  const int l_fpm2 = tet(4 * (p - 2) + 1), l_d1f = tet(4 * p + 1), l_E = tet(4 * (p - 1) + 1);
  const int ring_off = (((l_fpm2 + l_d1f + 3) / 4 + 64) + 3) & ~3;
  int chain = 0;
  if (ring_chain)
    for (int s0 = 0; s0 <= 4 * p; s0 += 32) {
      const ChainTile T = chain_tile(s0, 4 * p, tc);
      chain = max(chain, T.nslot * T.slot_words);
    }
  return max(ring_off + chain, (l_fpm2 + l_d1f + l_E + 3) / 4);
}

// Which chain product a form runs at prime p: the shared-memory slice ring (the int8 tensor form, whose tiles read
// aligned words of a staged slice), or the lane sweep over global memory (dp4a and int32 forms).
__host__ __device__ constexpr bool uses_ring_chain(int form, int p) { return form == 2 && p > 0; }

// Shared-memory ring words for prime p: the chain's slice ring (when the chain stages slices in shared memory),
// theta's Delta slots, and the power modes' arrays.  ring_chain = true gives the size every form fits in;
// power (QFS_POWER_*, -1 for every mode) sizes theta for one power mode.
__host__ __device__ inline int ring_words_for(int p, TileConfig tc, bool ring_chain = true, int power = -1) {
  return max(max(ring_chain ? chain_slot_words(p, tc) : 0, theta_ring_words_for(p, power)),
             aux_ring_words(p, tc, ring_chain));
}

__host__ __device__ inline size_t smem_bytes_for(int p, TileConfig tc, bool ring_chain = true) {
  return ring_offset_for(tet(4 * (p - 1) + 1)) + 4 * (size_t)ring_words_for(p, tc, ring_chain);
}
__host__ __device__ inline size_t smem_bytes_for(int p, bool ring_chain = true) {
  return smem_bytes_for(p, default_tile(p), ring_chain);
}

__device__ __forceinline__ void cp_async16(uint32_t *smem, const uint32_t *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

namespace detail {

template <int UI, int SI>
struct Pair {
  static constexpr int index = UI * (UI + 1) / 2 + SI;
  static constexpr int tap0 = tet(UI) + tri(SI);  // tap index of tI = 0
};

// Contribution of pair (UI, SI) to the four output words (16 outputs) of one item.  `col` points at slot chunk c
// of input column s - SI; x[j] = input word 4c - 4 + j.
template <int UI, int SI, int FORM>
__device__ __forceinline__ void pair_item(const uint32_t *col, const Smem &sm, int (&acc)[4][4]) {
  uint32_t x[8];
  {
    const uint4 a = *reinterpret_cast<const uint4 *>(col);
    const uint4 b = *reinterpret_cast<const uint4 *>(col + 4);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
    x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  }
  if (FORM == 0) {
    int v[20];
#pragma unroll
    for (int j = 0; j < 20; ++j) v[j] = (int)((x[3 + (j >> 2)] >> (8 * (j & 3))) & 0xFFu);
#pragma unroll
    for (int tI = 0; tI <= SI; ++tI) {
      const int a = sm.taps[Pair<UI, SI>::tap0 + tI];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] += a * v[4 + 4 * q + r - tI];
    }
  } else {
    if (SI == 0) {
      const uint32_t a = (uint32_t)sm.taps[Pair<UI, SI>::tap0];
      const uint32_t a0 = a, a1 = a << 8, a2 = a << 16, a3 = a << 24;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q][0] = (int)__dp4a(x[4 + q], a0, (unsigned)acc[q][0]);
        acc[q][1] = (int)__dp4a(x[4 + q], a1, (unsigned)acc[q][1]);
        acc[q][2] = (int)__dp4a(x[4 + q], a2, (unsigned)acc[q][2]);
        acc[q][3] = (int)__dp4a(x[4 + q], a3, (unsigned)acc[q][3]);
      }
    } else {
      const uint32_t tw = sm.tapword[Pair<UI, SI>::index];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // window byte k = in(t - 3 + k), t = 4w + r: bytes r+1 .. r+4 of (lo = word w-1, hi = word w)
        acc[q][0] = (int)__dp4a(__byte_perm(x[3 + q], x[4 + q], 0x4321u), tw, (unsigned)acc[q][0]);
        acc[q][1] = (int)__dp4a(__byte_perm(x[3 + q], x[4 + q], 0x5432u), tw, (unsigned)acc[q][1]);
        acc[q][2] = (int)__dp4a(__byte_perm(x[3 + q], x[4 + q], 0x6543u), tw, (unsigned)acc[q][2]);
        acc[q][3] = (int)__dp4a(x[4 + q], tw, (unsigned)acc[q][3]);
      }
      if (SI == 4) {
        // the tap at tI = 4 reads in(t - 4) = byte r of word w - 1
        const uint32_t a = (uint32_t)sm.taps[Pair<UI, SI>::tap0 + 4];
        const uint32_t a0 = a, a1 = a << 8, a2 = a << 16, a3 = a << 24;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q][0] = (int)__dp4a(x[3 + q], a0, (unsigned)acc[q][0]);
          acc[q][1] = (int)__dp4a(x[3 + q], a1, (unsigned)acc[q][1]);
          acc[q][2] = (int)__dp4a(x[3 + q], a2, (unsigned)acc[q][2]);
          acc[q][3] = (int)__dp4a(x[3 + q], a3, (unsigned)acc[q][3]);
        }
      }
    }
  }
}

#define QFS_FOR_EACH_PAIR(X) \
  X(0, 0) X(1, 0) X(1, 1) X(2, 0) X(2, 1) X(2, 2) X(3, 0) X(3, 1) X(3, 2) X(3, 3) X(4, 0) X(4, 1) X(4, 2) X(4, 3) X(4, 4)

// All 15 pairs of one item; DENSE skips the per-pair test of the nonzero-pair mask.
template <int FORM, bool DENSE>
__device__ __forceinline__ void item_pairs(const uint32_t *sb0, const uint32_t *sb1, const uint32_t *sb2,
                                           const uint32_t *sb3, const uint32_t *sb4, int stride, uint32_t mask,
                                           const Smem &sm, int (&acc)[4][4]) {
#define QFS_PAIR(UI, SI)                                                                                      \
  if (DENSE || ((mask >> Pair<UI, SI>::index) & 1u)) pair_item<UI, SI, FORM>(sb##UI - SI * stride, sm, acc);
  QFS_FOR_EACH_PAIR(QFS_PAIR)
#undef QFS_PAIR
}

}  // namespace detail

// ------------------------------------------------------------------------------------------------ int8 tensor form
// One product of the chain as int8 tensor-core contractions: mma.sync m16n8k32 (u8 x u8 -> s32).  A tile is 16
// output columns (rows m) x 8 consecutive outputs t0 .. t0+7 (columns n) of one output slice.  The K dimension is
// 16 groups of four 32-bit words, group pi = tap pair (uI, sI) (the 16th group is empty): word j of group pi is
// input word t0/4 - 1 + j of column s - sI in slice u - uI (j = 3 carries no taps), so every A fragment register
// is one aligned shared-memory word -- no byte shuffling.  B is the Toeplitz of f's taps,
// B[k][n] = a(uI, sI, n + 4 - 4j - i) for byte i of word j (zero outside 0..sI), fixed per quartic.  A tile executes
// 16 x 8 x 256 MACs for 16 x 8 x 35 useful ones; accumulation is exact in int32 (at most 35 products per output).
__device__ __forceinline__ void mma_u8_16832(int (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                             uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// (uI, sI) of tap pair pi (pi = tri(uI) + sI), pi in [0, 15)
__host__ __device__ constexpr int pair_u(int pi) { return pi >= 10 ? 4 : pi >= 6 ? 3 : pi >= 3 ? 2 : pi >= 1 ? 1 : 0; }
__host__ __device__ constexpr int pair_s(int pi) { return pi - tri(pair_u(pi)); }

// B fragment registers of this thread (lane): b[2*kk] = rows 32kk + 4 tig .. +3, b[2*kk+1] = rows 32kk+16+4tig ..,
// column n = group.
__device__ __forceinline__ void tc_b_fragments(const Smem &sm, uint32_t (&b)[16]) {
  const int lane = threadIdx.x & 31, group = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int pi = 2 * kk + h;
      uint32_t w = 0;
      if (pi < 15 && tig < 3) {
        const int uI = pair_u(pi), sI = pair_s(pi);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int tI = group + 4 - 4 * tig - i;
          if (tI >= 0 && tI <= sI) w |= (uint32_t)sm.taps[tet(uI) + tri(sI) + tI] << (8 * i);
        }
      }
      b[2 * kk + h] = w;
    }
}

template <int P, int FORM, bool LAST, bool DEBUG>
__device__ __forceinline__ void ring_chain_step(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                int m_in, Smem &sm, uint32_t *ring, const uint8_t *gs,
                                                uint32_t *status, DebugPtrs dbg) {
  using Pr = Prime<P>;
  const int m_out = m_in + 4;
  const uint32_t mask = sm.pair_mask;
  // quartics with few zero (uI, sI) pairs run every pair: a zero tap costs less than a branch per pair
  const bool dense = __popc(mask) >= 12;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int nthreads = blockDim.x;
  bool bad = false;
  uint32_t tcb[16];
  if (FORM == 2) tc_b_fragments(sm, tcb);
  for (int s0 = 0; s0 <= m_out; s0 += 32) {
    const ChainTile T = chain_tile(s0, m_out, TileConfig{sm.tile_round, sm.tile_ring});
    const int s_last = min(s0 + 31, m_out);
    const int F0 = chunk_prefix(s0);
    const int ccols = T.CR + 1;  // slot chunks per column
    // fetch input slice u2 (columns s0-4 .. s0+31) into ring slot `slot`, zeros outside the input cone
    auto fetch = [&](int u2, int slot) {
      uint32_t *dst = ring + slot * T.slot_words;
      const bool slice_ok = u2 >= 0 && u2 <= m_in;
      const int base_u = slice_ok ? sm.SW[u2] : 0;
      for (int i = threadIdx.x; i < 36 * ccols; i += nthreads) {
        const int cs = small_quotient<6>(i, ccols), j = i - cs * ccols;   // i < 36 ccols
        const int s2 = s0 - 4 + cs;
        const bool ok = slice_ok && j >= 1 && s2 >= 0 && s2 <= u2 && j - 1 < chunks_of(s2);
        const uint32_t *src = ok ? in + base_u + colw(s2) + 4 * (j - 1) : in;
        cp_async16(dst + cs * T.stride + 4 * j, src, ok);
      }
    };
    // ring slot of slice u2: (u2 - s0 + 4) mod nslot (u2 - s0 + 4 <= D + 4 < 2^7 nslot)
    auto slot_of = [&](int u2) { const int x = u2 - s0 + 4; return x - small_quotient<7>(x, T.nslot) * T.nslot; };
    for (int u2 = s0 - 4; u2 < s0 + T.upar; ++u2) fetch(u2, slot_of(u2));
    cp_async_commit();
    if (threadIdx.x < kMaxUpar + 4) {
      const int u2 = s0 - 4 + (int)threadIdx.x;
      sm.slot_tab[0][threadIdx.x] = slot_of(u2) * T.slot_words;
    }
    for (int s = s0 + (int)threadIdx.x; s <= s_last; s += nthreads) {
      const int base = chunk_prefix(s) - F0;
      for (int c = 0; c < chunks_of(s); ++c) sm.chunk_tab[base + c] = (uint16_t)(((s - s0) << 8) | c);
    }
    cp_async_wait_all();
    __syncthreads();
    int tab = 0;
    for (int u = s0; u <= m_out; u += T.upar) {
      for (int u2 = u + T.upar; u2 < u + 2 * T.upar && u2 <= m_out; ++u2) fetch(u2, slot_of(u2));
      cp_async_commit();
      if (threadIdx.x < kMaxUpar + 4) {  // slot table of the next round (slices u + upar - 4 ..)
        const int u2 = u + T.upar - 4 + (int)threadIdx.x;
        sm.slot_tab[tab ^ 1][threadIdx.x] = slot_of(u2) * T.slot_words;
      }
      const int nU = min(T.upar, m_out - u + 1);
      // chunk prefix over the round's slices: slice u+du holds columns s0 .. min(s_last, u+du)
      int pre[kMaxUpar + 1];
      pre[0] = 0;
#pragma unroll
      for (int du = 0; du < kMaxUpar; ++du) {
        const int cols_hi = min(s_last, u + du);
        pre[du + 1] = pre[du] + (du < nU ? chunk_prefix(cols_hi + 1) - F0 : 0);
      }
      const int total = pre[kMaxUpar];
      const int *stab = sm.slot_tab[tab];
      if (FORM == 2) {
        // tiles: (slice du, column group of 16, word pair wp); word pairs of a group cover the data of its longest
        // column (s/8 + 1 pairs); the padding words after them are cleared below
        int tpre[2 * kMaxUpar + 1];
        tpre[0] = 0;
#pragma unroll
        for (int i = 0; i < 2 * kMaxUpar; ++i) {
          const int du = i >> 1, grp = i & 1;
          const int hi = min(s_last, u + du);
          const int sg = s0 + 16 * grp;
          tpre[i + 1] = tpre[i] + ((du < nU && sg <= hi) ? half_chunks_of(min(hi, sg + 15)) : 0);
        }
        const int ntiles = tpre[2 * kMaxUpar];
        const int group = lane >> 2, tig = lane & 3;
        const int joff = tig < 3 ? tig : 2;  // word j = 3 carries no taps: reload word 2
        for (int tile = warp; tile < ntiles; tile += nwarps) {
          int i = 0, tbase = 0;
#pragma unroll
          for (int k2 = 1; k2 < 2 * kMaxUpar; ++k2)
            if (tile >= tpre[k2]) { i = k2; tbase = tpre[k2]; }
          const int du = i >> 1, grp = i & 1, wp = tile - tbase;
          const int uo = u + du;
          const int hi = min(s_last, uo);
          const int sg = s0 + 16 * grp;
          int acc[4] = {0, 0, 0, 0};
          const int rbase_a = (sg - s0 + group + 4) * T.stride + 2 * wp + 3 + joff;
          const int rbase_b = rbase_a + 8 * T.stride;
          int sb[5];
#pragma unroll
          for (int uI = 0; uI < 5; ++uI) sb[uI] = stab[du + 4 - uI];
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const int p0 = 2 * kk, p1 = 2 * kk + 1;
            const int o0 = sb[pair_u(p0)] - pair_s(p0) * T.stride;
            const int o1 = p1 < 15 ? sb[pair_u(p1)] - pair_s(p1) * T.stride : sb[0];
            const uint32_t a0 = ring[o0 + rbase_a], a1 = ring[o0 + rbase_b];
            const uint32_t a2 = ring[o1 + rbase_a], a3 = ring[o1 + rbase_b];
            mma_u8_16832(acc, a0, a1, a2, a3, tcb[2 * kk], tcb[2 * kk + 1]);
          }
          // acc: rows group (c0, c1) and group + 8 (c2, c3), outputs t = 8 wp + 2 tig + {0, 1}
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int s = sg + group + 8 * h;
            uint32_t half = 0, ghalf = 0;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              int G = acc[2 * h + e] % Pr::p2;
              const int t = 8 * wp + 2 * tig + e;
              if (LAST) {
                if (DEBUG) ghalf |= (uint32_t)G << (8 * e);
                if (t <= s && (uo % P) == 0 && (s % P) == 0 && (t % P) == 0) {
                  const int J = tet(uo / P) + tri(s / P) + t / P;
                  G = G - sm.powp[gs[J]];
                  if (G < 0) G += Pr::p2;
                }
                if (s <= hi && G % P) bad = true;
                G /= P;
              }
              half |= (uint32_t)G << (8 * e);
            }
            const uint32_t other = __shfl_down_sync(0xffffffffu, half, 1);
            const uint32_t gother = __shfl_down_sync(0xffffffffu, ghalf, 1);
            const int w = 2 * wp + (tig >> 1);
            if ((tig & 1) == 0 && s <= hi && w < 4 * chunks_of(s)) {
              const int o = sm.SW[uo] + colw(s) + w;
              out[o] = half | (other << 16);
              if (DEBUG && LAST) dbg.G[o] = ghalf | (gother << 16);
            }
          }
        }
        // padding words of each column past the word pairs its group's tiles cover (columns hold s + 4 entries)
        for (int i = threadIdx.x; i < nU * 32; i += nthreads) {
          const int du = i >> 5, s = s0 + (i & 31), uo = u + du;
          const int hi = min(s_last, uo);
          if (s > hi) continue;
          const int sg = s0 + 16 * ((s - s0) >> 4);
          for (int w = 2 * half_chunks_of(min(hi, sg + 15)); w < 4 * chunks_of(s); ++w)
            out[sm.SW[uo] + colw(s) + w] = 0u;
        }
      } else
      for (int it = warp; it * 32 < total; it += nwarps) {
        const int g = it * 32 + lane;
        if (g >= total) continue;
        int du = 0, gbase = 0;
#pragma unroll
        for (int j = 1; j < kMaxUpar; ++j)
          if (g >= pre[j]) { du = j; gbase = pre[j]; }
        const int uo = u + du;
        const int sc_packed = sm.chunk_tab[g - gbase];
        const int s = s0 + (sc_packed >> 8), c = sc_packed & 0xFF;
        int acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = 0;
        const int colbase = (s - s0 + 4) * T.stride + 4 * c;
        const uint32_t *sb0 = ring + stab[du + 4] + colbase;
        const uint32_t *sb1 = ring + stab[du + 3] + colbase;
        const uint32_t *sb2 = ring + stab[du + 2] + colbase;
        const uint32_t *sb3 = ring + stab[du + 1] + colbase;
        const uint32_t *sb4 = ring + stab[du + 0] + colbase;
        if (dense)
          detail::item_pairs<FORM, true>(sb0, sb1, sb2, sb3, sb4, T.stride, mask, sm, acc);
        else
          detail::item_pairs<FORM, false>(sb0, sb1, sb2, sb3, sb4, T.stride, mask, sm, acc);
        uint32_t word[4], gword[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          word[q] = 0;
          gword[q] = 0;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            int G = acc[q][r] % Pr::p2;  // acc >= 0; zero past the column's end
            if (LAST) {
              const int t = 16 * c + 4 * q + r;
              if (DEBUG) gword[q] |= (uint32_t)G << (8 * r);
              if (t <= s && (uo % P) == 0 && (s % P) == 0 && (t % P) == 0) {
                const int J = tet(uo / P) + tri(s / P) + t / P;
                G = G - sm.powp[gs[J]];
                if (G < 0) G += Pr::p2;
              }
              if (G % P) bad = true;
              G /= P;
            }
            word[q] |= (uint32_t)G << (8 * r);
          }
        }
        const int o = sm.SW[uo] + colw(s) + 4 * c;
        *reinterpret_cast<uint4 *>(out + o) = make_uint4(word[0], word[1], word[2], word[3]);
        if (DEBUG && LAST) *reinterpret_cast<uint4 *>(dbg.G + o) = make_uint4(gword[0], gword[1], gword[2], gword[3]);
      }
      tab ^= 1;
      cp_async_wait_all();
      __syncthreads();
    }
  }
  if (bad) atomicOr(status, kStatusInexactDivision);
}

// One product of the chain: over the shared-memory slice ring above (int8 tensor form), or lane by lane over the
// input slices in global memory (qfs_sweep.cuh; dp4a and int32 forms).
template <int P, int FORM, bool LAST, bool DEBUG>
__device__ __forceinline__ void chain_step(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int m_in,
                                           Smem &sm, uint32_t *ring, const uint8_t *gs, uint32_t *status,
                                           DebugPtrs dbg) {
  if constexpr (uses_ring_chain(FORM, P))
    ring_chain_step<P, FORM, LAST, DEBUG>(in, out, m_in, sm, ring, gs, status, dbg);
  else
    sweep_chain_step<P, FORM, LAST, DEBUG>(in, out, m_in, sm, gs, status, dbg);
}

// ------------------------------------------------------------------------------------------------ theta
// g_next[r] = sum over c in B_d of Delta[p r + (p-1)1 - c] * g[c] mod p, for every r in B_d (Algorithm 2's u
// applied to Delta g, only at the outputs u keeps).  In (u,s,t) coordinates the Delta index is
// (p u_r + 3(p-1) - u_c, p s_r + 2(p-1) - s_c, p t_r + (p-1) - t_c) and a term is present iff that index lies in
// the degree-D cone.
//
// Layout for theta: a guarded copy of Delta in which every column keeps kThetaGuardWords zero words on each side
// (slice eu starts at word theta_gsw(eu) = SW[eu] + 6 eu (eu + 3); column es of it at + 12 (es + 1) + colw(es)).
// For output r and g column (u_c, s_c) the terms are then one run of bytes of one Delta column, read against g's
// column reversed: sum_j Delta[e_u, e_s, A + j] R[j] with A = p t_r + (p-1) - s_c and R[j] = g[u_c, s_c, s_c - j]
// (zero past s_c).  A is at least -3(p-1) and the run ends at most 3p + 7 bytes past the column's data, inside the
// guards, so the dot product needs no bounds checks: bytes outside the column are zero.
constexpr int kThetaGuardWords = 12;   // 48 bytes on each side of every column (p <= 13)

__host__ __device__ constexpr int theta_gsw_extra(int eu) { return 6 * eu * (eu + 3); }
// words of a degree-D guarded Delta
inline size_t theta_guarded_words(int p) {
  const int D = 4 * p * (p - 1);
  return (size_t)host_sw(D + 1) + (size_t)theta_gsw_extra(D + 1);
}

// Words of Delta in residue-class order (theta at p <= 7): every class of degree d - k starts on a 16-byte boundary.
inline size_t theta_class_words(int p);

// Workspace buffer stride (see qfs_common.cuh): a padded degree-D form, and room for theta's copy of Delta: the
// residue-class order at p <= 7, the guarded copy at p >= 11 (which is larger than the padded form).
inline size_t workspace_stride_words(int p) {
  const size_t padded = (size_t)padded_words(4 * p * (p - 1));
  return std::max(padded, p <= 7 ? theta_class_words(p) : theta_guarded_words(p)) + kGuardWords;
}

// Reversed g columns: column (u_c, s_c) holds g[u_c, s_c, s_c - j] at byte j (j <= s_c), zero-padded to whole words.
// rcolw(s) = words of the reversed columns 0 .. s-1 of one slice.
__host__ __device__ constexpr int rcolw(int s) { return ((s >> 2) + 1) * (2 * (s >> 2) + (s & 3)); }

template <int P>
__host__ __device__ constexpr int theta_r_words() {
  int r = 0;
  for (int u = 0; u <= 4 * (P - 1); ++u) r += rcolw(u + 1);
  return r;
}
// Theta at p = 7 in the chain power mode streams Delta slice by slice through shared memory (two guarded slice
// slots, theta_stream): the copy of Delta into class order that theta_poly reads would add a round trip of the whole
// 0.8 MB Delta through device memory per quartic.  At p <= 5, and for the identity power mode at p <= 7 (which forms
// Delta in class order directly), theta runs by residue classes; at p >= 11 it gathers from a guarded copy.
template <int P>
__host__ __device__ constexpr bool theta_streams() { return P == 7; }
// a slice slot: columns 0 .. D with the guards of the guarded layout
template <int P>
__host__ __device__ constexpr int theta_slot_words() { return kThetaGuardWords * (4 * P * (P - 1) + 2) + colw(4 * P * (P - 1) + 1); }
// slice slots of the streamed theta (prefetch distance slots - 1)
template <int P>
__host__ __device__ constexpr int theta_nslots() { return 2; }
// word offset of the slice slots in the ring (16-byte aligned for cp.async)
template <int P>
__host__ __device__ constexpr int theta_slots_off() { return (theta_r_words<P>() + 4 * (P - 1) + 2 + 3) & ~3; }
// ring words of the streamed theta: reversed g columns and their slice table, the slice slots, int32 accumulators,
// the chunk-to-slot table and the unpacked output coordinates
template <int P>
__host__ __device__ constexpr int theta_stream_ring_words() {
  constexpr int d = 4 * (P - 1), D = 4 * P * (P - 1), ld = tet(d + 1);
  return theta_slots_off<P>() + theta_nslots<P>() * theta_slot_words<P>() + ld + chunk_prefix(D + 1) + ld + D + 1;
}

// Theta by residue classes (theta_poly below) is built for p <= 7; at p >= 11 the padded cube of one class would not
// fit in shared memory.
template <int P>
__host__ __device__ constexpr bool theta_by_classes() { return P <= 7; }

// Residue classes of theta at p <= 7.  Writing c = p c' + rho with rho in [0,p)^4 (per exponent) turns
//   theta(g)[r] = sum_c Delta[p r + (p-1)1 - c] g[c]
// into a sum of products of forms: the exponent p (r - c') + (p-1)1 - rho is non-negative exactly when c' <= r, so
//   theta(g) = sum_rho Delta_sigma * g_rho,   Delta_sigma[e] = Delta[p e + sigma], g_rho[c'] = g[p c' + rho],
// with sigma = (p-1)1 - rho.  |rho| = d - p k with k = deg g_rho in {0, .., 3}, and deg Delta_sigma = d - k; the p^3
// classes hold every coefficient of g once and every coefficient of Delta once, and the MACs add up to the theta
// matrix's nonzeros.  Each class is a product with a kernel of at most 20 taps, computed on a zero-padded cube of
// Delta_sigma in shared memory, so no term needs a bounds check.
constexpr int kPolyStages = 4;   // class-data staging slots of theta_poly (prefetch distance 3 classes)

template <int P>
struct Poly {
  static constexpr int d = 4 * (P - 1), ld = tet(d + 1);
  static constexpr int pad = 4;                         // zero layers before coordinate 0 (kernels of degree <= 4)
  static constexpr int C = d + 1 + pad;                 // cube side: coordinates -pad .. d
  static constexpr int CB = (C * C * C + 15) & ~15;     // bytes of one cube
  static constexpr int NCLS = P * P * P;
  static constexpr int NOUT = (ld + kThreads - 1) / kThreads;   // outputs per thread
  // ring layout (bytes): two cubes, the taps of every class (ld bytes), the g index of every tap (ld x u16), the
  // cube address of every packed index of B_d (ld x u16), the class records (NCLS x 16 bytes), per-k counters
  static constexpr int taps_off = 2 * CB;
  static constexpr int tapsrc_off = taps_off + ((ld + 15) & ~15);
  static constexpr int cubeaddr_off = tapsrc_off + ((2 * ld + 15) & ~15);
  static constexpr int cls_off = cubeaddr_off + ((2 * ld + 15) & ~15);
  static constexpr int cnt_off = cls_off + 16 * NCLS;
  // identity power mode: the taps of Delta_1(f) split by class (C(4p+3, 3) bytes in all)
  static constexpr int idtaps_off = cnt_off + 16;
  // byte offset of each class in the class-ordered copy, indexed by sigma2 + p sigma3 + p^2 sigma4 (NCLS ints)
  static constexpr int sig_off = idtaps_off + ((tet(4 * P + 1) + 15) & ~15);
  // staging slots of theta_poly's class stream (kPolyStages slots of the largest class; 16-byte cp.async targets)
  static constexpr int stage_off = sig_off + ((4 * NCLS + 15) & ~15);
  static constexpr int bytes = stage_off + kPolyStages * ((ld + 15) & ~15);
  // every region starts on a 16-byte boundary (uint4 stores, int4 records, cp.async)
  static_assert(taps_off % 16 == 0 && tapsrc_off % 16 == 0 && cubeaddr_off % 16 == 0 && cls_off % 16 == 0 &&
                    cnt_off % 16 == 0 && idtaps_off % 16 == 0 && sig_off % 16 == 0 && stage_off % 16 == 0,
                "16-byte aligned ring regions");
};

// Classes of degree k (kernel degree) in residue-class order: rho in [0,p)^4 with |rho| = d - p k.
__host__ __device__ constexpr int poly_count(int p, int k) {
  int n = 0;
  for (int r1 = 0; r1 < p; ++r1)
    for (int r2 = 0; r2 < p; ++r2)
      for (int r3 = 0; r3 < p; ++r3)
        for (int r4 = 0; r4 < p; ++r4)
          if (r1 + r2 + r3 + r4 == 4 * (p - 1) - p * k) ++n;
  return n;
}
// bytes of one class of kernel degree k in global memory: C(d - k + 3, 3), rounded up to 16
__host__ __device__ constexpr int poly_class_bytes(int p, int k) { return (tet(4 * (p - 1) - k + 1) + 15) & ~15; }

inline size_t theta_class_words(int p) {
  size_t b = 0;
  for (int k = 0; k <= 3; ++k) b += (size_t)poly_count(p, k) * poly_class_bytes(p, k);
  return b / 4;
}

// Ring words of theta for one power mode (-1: every mode).  At p = 7 the chain mode streams (theta_stream) and
// the identity mode runs by classes; the reduced mode keeps its arrays in the power modes' part of the ring.
template <int P>
__host__ __device__ constexpr int theta_ring_words(int power = -1) {
  if constexpr (theta_by_classes<P>()) {
    constexpr int poly = (Poly<P>::bytes + 3) / 4;
    if constexpr (theta_streams<P>()) {
      constexpr int stream = theta_stream_ring_words<P>();
      return power == 0 ? stream : power == 1 ? poly : power == 2 ? 0 : (poly > stream ? poly : stream);
    } else {
      return power == 2 ? 0 : poly;
    }
  } else {
    return (theta_r_words<P>() + 4 * (P - 1) + 2 + 3) & ~3;   // reversed g columns and their slice table
  }
}

__host__ __device__ inline int theta_ring_words_for(int p, int power) {
  switch (p) {
    case 3: return theta_ring_words<3>(power);
    case 5: return theta_ring_words<5>(power);
    case 7: return theta_ring_words<7>(power);
    case 11: return theta_ring_words<11>(power);
    default: return theta_ring_words<13>(power);
  }
}

// Padded Delta (degree D) -> guarded copy.  One thread per 16-byte chunk; the thread of a column's first chunk
// writes the guard before the column, the thread of a slice's last chunk the guard after it.  The caller
// synchronises the CTA afterwards.
template <int P>
__device__ __forceinline__ void delta_to_guarded(const uint32_t *__restrict__ delta, uint32_t *__restrict__ dg,
                                                 const Smem &sm) {
  constexpr int D = Prime<P>::D;
  const int nchunks = sm.SW[D + 1] / 4;
  const uint4 z = make_uint4(0u, 0u, 0u, 0u);
  for (int k = threadIdx.x; k < nchunks; k += blockDim.x) {
    int u, s, c;
    decode_form_chunk(k, D, sm.SW, u, s, c);
    const int o = sm.SW[u] + theta_gsw_extra(u) + kThetaGuardWords * (s + 1) + colw(s) + 4 * c;
    *reinterpret_cast<uint4 *>(dg + o) = *reinterpret_cast<const uint4 *>(delta + 4 * k);
    if (c == 0)
#pragma unroll
      for (int w = 0; w < kThetaGuardWords; w += 4) *reinterpret_cast<uint4 *>(dg + o - kThetaGuardWords + w) = z;
    if (s == u && c == chunks_of(s) - 1)
#pragma unroll
      for (int w = 0; w < kThetaGuardWords; w += 4) *reinterpret_cast<uint4 *>(dg + o + 4 + w) = z;
  }
}

// One theta step: g (shared, packed) -> gn (shared, packed), Delta guarded in global memory.  One thread per
// output; returns whether some output is nonzero (same value in every thread).
template <int P>
__device__ __noinline__ bool theta_gather(const uint32_t *__restrict__ dg, const Smem &sm,
                                          const uint8_t *__restrict__ g, uint8_t *__restrict__ gn, uint32_t *ring) {
  using Pr = Prime<P>;
  constexpr int d = Pr::d, D = Pr::D;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  uint32_t *R = ring;
  int *RSW = reinterpret_cast<int *>(ring + theta_r_words<P>());   // d+2 slice offsets (words) of R
  if (tid == 0) {
    int a = 0;
    for (int u = 0; u <= d + 1; ++u) { RSW[u] = a; a += rcolw(u + 1); }
  }
  __syncthreads();
  for (int i = tid; i < theta_r_words<P>(); i += nthreads) {
    int u = 0;
    while (RSW[u + 1] <= i) ++u;
    const int rem = i - RSW[u];
    int sc = 0;
    while (rcolw(sc + 1) <= rem) ++sc;
    const int k = rem - rcolw(sc);
    const uint8_t *gcol = g + tet(u) + tri(sc);
    uint32_t w = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = 4 * k + b;
      if (j <= sc) w |= (uint32_t)gcol[sc - j] << (8 * b);
    }
    R[i] = w;
  }
  __syncthreads();
  bool any = false;
  for (int r = tid; r < Pr::ld; r += nthreads) {
    int ur, sr, tr;
    decode_packed(r, ur, sr, tr, d);
    const int Ue = P * ur + 3 * (P - 1), Se = P * sr + 2 * (P - 1), Te = P * tr + (P - 1);
    const int uc_lo = max(0, Ue - D), uc_hi = min(d, Ue);
    unsigned acc = 0;
    for (int uc = uc_lo; uc <= uc_hi; ++uc) {
      const int eu = Ue - uc;
      // g columns s_c with Delta column e_s = Se - s_c in [0, e_u]
      const int sc_lo = max(0, Se - eu), sc_hi = min(uc, Se);
      if (sc_lo > sc_hi) continue;
      int es = Se - sc_lo;
      // byte of Delta(e_u, e_s, Te - s_c) and word of R(u_c, s_c), both updated as s_c grows
      int byte = 4 * (sm.SW[eu] + theta_gsw_extra(eu) + kThetaGuardWords * (es + 1) + colw(es)) + Te - sc_lo;
      const uint32_t *Rc = R + RSW[uc] + rcolw(sc_lo);
      for (int sc = sc_lo; sc <= sc_hi; ++sc) {
        const uint32_t *dw = dg + (byte >> 2);
        const unsigned sh = 8u * (unsigned)(byte & 3);
        const int nw = (sc >> 2) + 1;   // at most p words
        // every word of the run is requested before the first is used, so a pair waits on memory once
        uint32_t dv[P + 1], rv[P];
#pragma unroll
        for (int k = 0; k <= P; ++k) dv[k] = k <= nw ? dw[k] : 0u;
#pragma unroll
        for (int k = 0; k < P; ++k) rv[k] = k < nw ? Rc[k] : 0u;
#pragma unroll
        for (int k = 0; k < P; ++k)
          if (k < nw) acc = __dp4a(__funnelshift_r(dv[k], dv[k + 1], sh), rv[k], acc);
        // next g column: e_s - 1, whose guarded column starts 12 + 4 chunks_of(e_s - 1) words earlier
        Rc += nw;
        --es;
        byte -= 4 * (kThetaGuardWords + 4 * chunks_of(es)) + 1;
      }
    }
    const int v = (int)(acc % P);
    gn[r] = (uint8_t)v;
    any |= v != 0;
  }
  return __syncthreads_or(any ? 1 : 0) != 0;
}

// Up to four g columns s_c = sc0 .. sc1 of a streamed theta round, all of NW words (sc0 / 4 == sc1 / 4), for the
// output r = (u_r, s_r, t_r) of this lane: each column s_c inside the lane's range [lo, hi] adds the lane's Delta
// window (NW + 1 words of the guarded slot, shifted to the window's first byte) against the NW words of g's
// reversed column s_c, which are the same for every lane.  ebase = p s_r + 2(p-1), so the Delta column is
// e_s = ebase - s_c; tbase = p t_r + (p-1), the window's last byte in that column.  A column without a term for
// this lane reads its window from the zero guard words at the start of the slot (kThetaGuardWords >= NW + 1), so
// no load is predicated: its g words are then multiplied by zeros whatever they hold (past sc1 they are words of
// the next reversed columns or of the table after them, inside the ring).  The g column offset advances by NW
// words per column (rcolw(s + 1) - rcolw(s) = s / 4 + 1).  All loads of the four columns are issued before the
// first product.
template <int P, int NW>
__device__ __forceinline__ unsigned theta_seg(const uint32_t *__restrict__ slot, const uint32_t *__restrict__ Rb,
                                              const int *__restrict__ gofs, int sc0, int sc1, int lo, int hi,
                                              int ebase, int tbase, unsigned a) {
  static_assert(kThetaGuardWords >= NW + 1, "a window read from the zero guard stays inside it");
  uint32_t dv[4][NW + 1], rv[4][NW];
  unsigned sh[4];
  const uint32_t *rw = Rb + rcolw(sc0);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int sc = sc0 + j;
    const bool on = sc <= sc1 && sc >= lo && sc <= hi;
    const int byte = on ? gofs[ebase - sc] + tbase - sc : 0;
    sh[j] = 8u * (unsigned)(byte & 3);
    const uint32_t *dw = slot + (byte >> 2);
#pragma unroll
    for (int k = 0; k <= NW; ++k) dv[j][k] = dw[k];
#pragma unroll
    for (int k = 0; k < NW; ++k) rv[j][k] = rw[NW * j + k];
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < NW; ++k) a = __dp4a(__funnelshift_r(dv[j][k], dv[j][k + 1], sh[j]), rv[j][k], a);
  return a;
}

// One theta step with Delta (padded, degree D, global memory) streamed through shared memory (p = 7).  Round e_u
// copies slice e_u into a guarded slot (16-byte cp.async, double buffered) and serves every output slice u_r whose
// g slice u_c = p u_r + 3(p-1) - e_u exists, in blocks of 32 consecutive outputs (one per lane) that sum over the
// g columns in registers; each round's sums go to shared int32 accumulators.  Every Delta byte is read from global
// memory once per step.  Returns whether some output is nonzero (same value in every thread).
template <int P>
__device__ __noinline__ bool theta_stream(const uint32_t *__restrict__ delta, const Smem &sm,
                                          const uint8_t *__restrict__ g, uint8_t *__restrict__ gn, uint32_t *ring) {
  static_assert(P <= 7, "g columns of at most 7 words");
  using Pr = Prime<P>;
  constexpr int d = Pr::d, D = Pr::D, ld = Pr::ld;
  constexpr int SLOT = theta_slot_words<P>();
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthreads >> 5;
  uint32_t *R = ring;
  int *RSW = reinterpret_cast<int *>(ring + theta_r_words<P>());
  constexpr int NS = theta_nslots<P>();
  uint32_t *slots = ring + theta_slots_off<P>();                        // NS x SLOT, 16-byte aligned
  int *acc = reinterpret_cast<int *>(slots + NS * SLOT);
  int *ctab = acc + ld;                                                 // flat chunk of a slice -> slot word
  uint32_t *rst = reinterpret_cast<uint32_t *>(ctab + chunk_prefix(D + 1));   // output r -> ur | sr << 8 | tr << 16
  int *gofs = reinterpret_cast<int *>(rst + ld);                        // column e_s -> byte offset in a slot
  for (int es = tid; es <= D; es += nthreads) gofs[es] = 4 * (kThetaGuardWords * (es + 1) + colw(es));
  if (tid == 0) {
    int a = 0;
    for (int u = 0; u <= d + 1; ++u) { RSW[u] = a; a += rcolw(u + 1); }
  }
  for (int i = tid; i < NS * SLOT; i += nthreads) slots[i] = 0u;
  for (int i = tid; i < ld; i += nthreads) {
    acc[i] = 0;
    int u, s, t;
    decode_packed(i, u, s, t, d);
    rst[i] = (uint32_t)u | ((uint32_t)s << 8) | ((uint32_t)t << 16);
  }
  for (int k = tid; k < chunk_prefix(D + 1); k += nthreads) {
    int es, c;
    decode_chunk(k, es, c);
    ctab[k] = kThetaGuardWords * (es + 1) + colw(es) + 4 * c;
  }
  __syncthreads();
  for (int i = tid; i < theta_r_words<P>(); i += nthreads) {
    int u = 0;
    while (RSW[u + 1] <= i) ++u;
    const int rem = i - RSW[u];
    int sc = 0;
    while (rcolw(sc + 1) <= rem) ++sc;
    const int k = rem - rcolw(sc);
    const uint8_t *gcol = g + tet(u) + tri(sc);
    uint32_t w = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = 4 * k + b;
      if (j <= sc) w |= (uint32_t)gcol[sc - j] << (8 * b);
    }
    R[i] = w;
  }
  auto fetch = [&](int eu, int buf) {
    uint32_t *dst = slots + buf * SLOT;
    const uint32_t *src = delta + sm.SW[eu];
    const int n = chunk_prefix(eu + 1);
    for (int k = tid; k < n; k += nthreads) cp_async16(dst + ctab[k], src + 4 * k, true);
  };
  // slices 0 .. NS-2 in flight; round e_u waits for its own slice, then refills the slot round e_u - 1 used
  for (int e = 0; e < NS - 1; ++e) {
    if (e <= D) fetch(e, e);
    cp_async_commit();
  }
  for (int eu = 0; eu <= D; ++eu) {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NS - 2));
    __syncthreads();   // slot eu % NS is complete for every thread; slot (eu - 1) % NS is no longer read
    if (eu + NS - 1 <= D) fetch(eu + NS - 1, (eu + NS - 1) % NS);
    cp_async_commit();
    const uint32_t *slot = slots + (eu % NS) * SLOT;
    // output slices with u_c = p u_r + 3(p-1) - e_u in [0, d]
    const int base = eu - 3 * (P - 1);
    const int ur_lo = max(0, (base + P - 1) / P);
    const int ur_hi = min(d, base + d >= 0 ? (base + d) / P : -1);
    if (ur_lo > ur_hi) continue;
    // blocks of 32 consecutive outputs of a slice u_r, one warp each (lane = output): a lane sums, over every g
    // column s_c whose Delta column e_s = p s_r + 2(p-1) - s_c lies in slice e_u, in registers, and adds the total
    // to its output once per round; the warp runs the union of its lanes' column ranges, four columns at a time
    int nblocks = 0;
    for (int ur = ur_lo; ur <= ur_hi; ++ur) nblocks += (tri(ur + 1) + 31) >> 5;
    for (int blk = warp; blk < nblocks; blk += nwarps) {
      int ur = ur_lo, b = blk;
      for (;;) {
        const int nb = (tri(ur + 1) + 31) >> 5;
        if (b < nb) break;
        b -= nb;
        ++ur;
      }
      const int uc = P * ur - base;   // in [0, d] for ur in [ur_lo, ur_hi]
      const int i = 32 * b + lane;
      const bool act = i < tri(ur + 1);
      const int r = tet(ur) + i;
      int lo = 1 << 30, hi = -1, ebase = 0, tbase = 0;
      if (act) {
        const uint32_t x = rst[r];
        ebase = P * (int)((x >> 8) & 255u) + 2 * (P - 1);
        tbase = P * (int)(x >> 16) + (P - 1);
        lo = max(0, ebase - eu);   // e_s <= e_u
        hi = min(uc, ebase);       // e_s >= 0
      }
      const int wlo = __reduce_min_sync(0xffffffffu, lo), whi = __reduce_max_sync(0xffffffffu, hi);
      if (wlo > whi) continue;
      const uint32_t *Rb = R + RSW[uc];
      unsigned a = 0;
      for (int q = wlo >> 2; q <= (whi >> 2); ++q) {
        const int sc0 = max(wlo, 4 * q), sc1 = min(whi, 4 * q + 3);
        switch (q) {   // words of g's reversed column: s_c / 4 + 1 <= p
          case 0: a = theta_seg<P, 1>(slot, Rb, gofs, sc0, sc1, lo, hi, ebase, tbase, a); break;
          case 1: a = theta_seg<P, 2>(slot, Rb, gofs, sc0, sc1, lo, hi, ebase, tbase, a); break;
          case 2: a = theta_seg<P, 3>(slot, Rb, gofs, sc0, sc1, lo, hi, ebase, tbase, a); break;
          case 3: a = theta_seg<P, 4>(slot, Rb, gofs, sc0, sc1, lo, hi, ebase, tbase, a); break;
          case 4: a = theta_seg<P, 5>(slot, Rb, gofs, sc0, sc1, lo, hi, ebase, tbase, a); break;
          case 5: a = theta_seg<P, 6>(slot, Rb, gofs, sc0, sc1, lo, hi, ebase, tbase, a); break;
          default: a = theta_seg<P, 7>(slot, Rb, gofs, sc0, sc1, lo, hi, ebase, tbase, a); break;
        }
      }
      if (act && a != 0u) atomicAdd(acc + r, (int)a);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  bool any = false;
  for (int r = tid; r < ld; r += nthreads) {
    const int v = acc[r] % P;
    gn[r] = (uint8_t)v;
    any |= v != 0;
  }
  return __syncthreads_or(any ? 1 : 0) != 0;
}

// Class records of theta_poly (ring, Poly<P>::cls_off): x = byte offset of Delta_sigma in the class-ordered copy,
// y = offset of g_rho's taps in the tap arrays, z = k | Su << 8 | Ss << 16 | St << 24 where (Su, Ss, St) is sigma in
// (u, s, t) coordinates (Delta_sigma[u', s', t'] = Delta[p u' + Su, p s' + Ss, p t' + St]), w = offset of the class's
// taps of Delta_1(f) (degree 4 - k; the identity power mode).  Classes are ordered by
// k, which theta_poly's cube clearing relies on; inside one k the order is whatever the atomic counters hand out.
// Also fills the tap sources (the packed index in B_d of g_rho's tap c', in the packed order of c' in B_k) and the
// cube address of every packed index of B_d.  Ends with a barrier.
template <int P>
__device__ __forceinline__ void poly_tables(unsigned char *ring) {
  using Q = Poly<P>;
  constexpr int d = Q::d, C = Q::C;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  uint16_t *tapsrc = reinterpret_cast<uint16_t *>(ring + Q::tapsrc_off);
  uint16_t *cubeaddr = reinterpret_cast<uint16_t *>(ring + Q::cubeaddr_off);
  int4 *cls = reinterpret_cast<int4 *>(ring + Q::cls_off);
  int *cnt = reinterpret_cast<int *>(ring + Q::cnt_off);
  if (tid < 4) cnt[tid] = 0;
  for (int i = tid; i < Q::ld; i += nthreads) {
    int u, s, t;
    decode_packed(i, u, s, t, d);
    cubeaddr[i] = (uint16_t)((u + Q::pad) * C * C + (s + Q::pad) * C + t + Q::pad);
  }
  __syncthreads();
  constexpr int NQ = (Q::NCLS + kThreads - 1) / kThreads;
  int slot[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int x = tid + kThreads * q;
    slot[q] = -1;
    if (x < Q::NCLS) {
      const int r2 = x % P, r3 = (x / P) % P, r4 = x / (P * P);
      const int r1 = ((d - r2 - r3 - r4) % P + P) % P;
      const int k = (d - (r1 + r2 + r3 + r4)) / P;
      slot[q] = atomicAdd(&cnt[k], 1);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int x = tid + kThreads * q;
    if (slot[q] < 0) continue;
    const int r2 = x % P, r3 = (x / P) % P, r4 = x / (P * P);
    const int r1 = ((d - r2 - r3 - r4) % P + P) % P;
    const int k = (d - (r1 + r2 + r3 + r4)) / P;
    int j = slot[q], goff = 0, toff = 0, ioff = 0;
    for (int kk = 0; kk < k; ++kk) {
      j += cnt[kk];
      goff += cnt[kk] * poly_class_bytes(P, kk);
      toff += cnt[kk] * tet(kk + 1);
      ioff += cnt[kk] * tet(4 - kk + 1);
    }
    goff += slot[q] * poly_class_bytes(P, k);
    toff += slot[q] * tet(k + 1);
    ioff += slot[q] * tet(4 - k + 1);
    const int s2 = P - 1 - r2, s3 = P - 1 - r3, s4 = P - 1 - r4;
    cls[j] = make_int4(goff, toff, k | ((s2 + s3 + s4) << 8) | ((s3 + s4) << 16) | (s4 << 24), ioff);
    reinterpret_cast<int *>(ring + Q::sig_off)[s2 + P * s3 + P * P * s4] = goff;
    // taps: g[p c' + rho] for c' = (uc, sc, tc) in B_k, rho = (r2 + r3 + r4, r3 + r4, r4) in (u, s, t)
    int i = 0;
    for (int uc = 0; uc <= k; ++uc)
      for (int sc = 0; sc <= uc; ++sc)
        for (int tc = 0; tc <= sc; ++tc, ++i)
          tapsrc[toff + i] = (uint16_t)(tet(P * uc + r2 + r3 + r4) + tri(P * sc + r3 + r4) + P * tc + r4);
  }
  __syncthreads();
}

// Padded Delta (degree D) -> class order: class sigma holds Delta_sigma in packed order of B_{d-k}, starting at byte
// sig_off[sigma] of `dc`.  One thread per 16-byte chunk of the padded Delta, read once and coalesced; each byte
// (U, S, T) goes to class sigma = (e2, e3, e4) mod p at the packed index of (e - sigma) / p, where
// (e2, e3, e4) = (U - S, S - T, T).  Within a chunk T advances by one, so e4 / p, e4 mod p, e3 / p and e3 mod p
// advance incrementally.  The caller synchronises the CTA afterwards.
template <int P>
__device__ __forceinline__ void delta_to_classes(const uint32_t *__restrict__ delta, uint32_t *__restrict__ dc,
                                                 const Smem &sm, const unsigned char *ring) {
  constexpr int D = Prime<P>::D;
  const int *sig = reinterpret_cast<const int *>(ring + Poly<P>::sig_off);
  uint8_t *db = reinterpret_cast<uint8_t *>(dc);
  const int nchunks = sm.SW[D + 1] / 4;
  for (int k = threadIdx.x; k < nchunks; k += blockDim.x) {
    int U, S, c;
    decode_form_chunk(k, D, sm.SW, U, S, c);
    const uint4 v = *reinterpret_cast<const uint4 *>(delta + 4 * k);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    const int e2 = U - S, q2 = e2 / P, r2 = e2 - P * q2;
    const int T0 = 16 * c;
    int q4 = T0 / P, r4 = T0 - P * q4;                 // e4 = T
    int q3 = (S - T0) / P, r3 = (S - T0) - P * q3;     // e3 = S - T (>= 0 while T <= S)
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      if (T0 + b <= S) {
        const int up = q2 + q3 + q4, sp = q3 + q4;
        db[sig[r2 + P * r3 + P * P * r4] + tet(up) + tri(sp) + q4] = (uint8_t)(w[b >> 2] >> (8 * (b & 3)));
      }
      if (++r4 == P) { r4 = 0; ++q4; }
      if (--r3 < 0) { r3 = P - 1; --q3; }
    }
  }
}

// Products of one class: acc[o] += sum over the taps c' in B_K of g_rho[c'] Delta_sigma[r_o - c'], reading
// Delta_sigma from the zero-padded cube at a[o] - offset(c').
template <int P, int K>
__device__ __forceinline__ void poly_macs(const uint8_t *cube, const uint8_t *tp, const int (&a)[Poly<P>::NOUT],
                                          int (&acc)[Poly<P>::NOUT]) {
  constexpr int C = Poly<P>::C;
#pragma unroll
  for (int uc = 0; uc <= K; ++uc)
#pragma unroll
    for (int sc = 0; sc <= uc; ++sc)
#pragma unroll
      for (int tc = 0; tc <= sc; ++tc) {
        const int tv = tp[tet(uc) + tri(sc) + tc];
        const int off = uc * C * C + sc * C + tc;
#pragma unroll
        for (int o = 0; o < Poly<P>::NOUT; ++o) acc[o] += tv * (int)cube[a[o] - off];
      }
}

// One theta step by residue classes (p <= 7): g (shared, packed) -> gn.  `dc` holds Delta in class order
// (delta_to_classes) and poly_tables has run.  Class data streams from `dc` into a ring of kPolyStages shared-memory
// slots by 16-byte cp.async, kPolyStages - 1 classes ahead.  Iteration j multiplies class j from one cube while
// every thread scatters four-byte words of class j + 1 (staged, and complete since the last barrier) into the other
// cube, then waits for its own copies of class j + 2; one barrier per class.  Cube positions outside B_d are zero
// from the start; when the degree d - k of the classes drops, the cube's slab of the old degree is cleared, so each
// cube always holds zeros outside its current class's cone.  Returns whether some output is nonzero (same value in
// every thread).
template <int P>
__device__ __noinline__ bool theta_poly(const uint32_t *__restrict__ dc, const uint8_t *__restrict__ g,
                                        uint8_t *__restrict__ gn, unsigned char *ring) {
  using Q = Poly<P>;
  constexpr int d = Q::d, ld = Q::ld, C = Q::C, NOUT = Q::NOUT, NS = kPolyStages;
  static_assert(NS >= 3, "the scatter of class j + 1 and the copies of classes j + 2 .. overlap");
  constexpr int SB = (ld + 15) & ~15;   // bytes of a staging slot (the largest class)
  const int tid = threadIdx.x, nthreads = blockDim.x;
  uint8_t *cube0 = ring;
  uint8_t *taps = ring + Q::taps_off;
  const uint16_t *tapsrc = reinterpret_cast<const uint16_t *>(ring + Q::tapsrc_off);
  const uint16_t *cubeaddr = reinterpret_cast<const uint16_t *>(ring + Q::cubeaddr_off);
  const int4 *cls = reinterpret_cast<const int4 *>(ring + Q::cls_off);
  uint8_t *stg = ring + Q::stage_off;
  // taps of every class in class order, and both cubes cleared
  for (int i = tid; i < ld; i += nthreads) taps[i] = g[tapsrc[i]];
  for (int i = tid; i < 2 * Q::CB / 16; i += nthreads) reinterpret_cast<uint4 *>(ring)[i] = make_uint4(0u, 0u, 0u, 0u);
  // class j -> slot j % NS by 16-byte chunks
  auto stage = [&](int j) {
    if (j < Q::NCLS) {
      const int4 c = cls[j];
      const int n16 = (tet(d - (c.z & 255) + 1) + 15) >> 4;
      uint32_t *dst = reinterpret_cast<uint32_t *>(stg + (j % NS) * SB);
      for (int i = tid; i < n16; i += nthreads) cp_async16(dst + 4 * i, dc + c.x / 4 + 4 * i, true);
    }
    cp_async_commit();
  };
  // scatter class j (staged and visible to every thread) into `cube`, four bytes per thread at a time
  auto scatter = [&](int j, uint8_t *cube) {
    const int len = tet(d - (cls[j].z & 255) + 1);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(stg + (j % NS) * SB);
    for (int w = tid; 4 * w < len; w += nthreads) {
      const uint32_t x = src[w];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * w + b < len) cube[cubeaddr[4 * w + b]] = (uint8_t)(x >> (8 * b));
    }
  };
  for (int j = 0; j < NS - 1; ++j) stage(j);
  asm volatile("cp.async.wait_group %0;\n" ::"n"(NS - 3));   // this thread's copies of classes 0 and 1
  __syncthreads();   // cubes cleared, taps written, classes 0 and 1 staged
  scatter(0, cube0);
  // output addresses: r_o = tid + kThreads o; threads past B_d read the cube around output (0, 0, 0), and drop it
  int a[NOUT], acc[NOUT];
#pragma unroll
  for (int o = 0; o < NOUT; ++o) {
    const int r = tid + kThreads * o;
    a[o] = r < ld ? (int)cubeaddr[r] : Q::pad * (C * C + C + 1);
    acc[o] = 0;
  }
  int degb[2] = {d, d};   // degree of the cone each cube was last filled with (uniform)
  __syncthreads();
  for (int j = 0; j < Q::NCLS; ++j) {
    const int4 c = cls[j];
    const int k = c.z & 255;
    stage(j + NS - 1);   // into the slot of class j - 1, scattered two iterations ago
    const uint8_t *tp = taps + c.y;
    const uint8_t *cube = cube0 + (j & 1) * Q::CB;
    switch (k) {
      case 0: poly_macs<P, 0>(cube, tp, a, acc); break;
      case 1: poly_macs<P, 1>(cube, tp, a, acc); break;
      case 2: poly_macs<P, 2>(cube, tp, a, acc); break;
      default: poly_macs<P, 3>(cube, tp, a, acc); break;
    }
    if (j + 1 < Q::NCLS) {
      // the other cube: clear the slab its previous class left beyond the new degree, then scatter class j + 1
      const int b = (j + 1) & 1;
      uint8_t *next = cube0 + b * Q::CB;
      const int nd = d - (cls[j + 1].z & 255);
      if (degb[b] > nd) {
        for (int i = tet(nd + 1) + tid; i < tet(degb[b] + 1); i += nthreads) next[cubeaddr[i]] = 0;
        degb[b] = nd;
      }
      scatter(j + 1, next);
    }
    asm volatile("cp.async.wait_group %0;\n" ::"n"(NS - 3));   // this thread's copies of class j + 2
    __syncthreads();
  }
  cp_async_wait_all();
  bool any = false;
#pragma unroll
  for (int o = 0; o < NOUT; ++o) {
    const int r = tid + kThreads * o;
    if (r < ld) {
      const int v = acc[o] % P;
      gn[r] = (uint8_t)v;
      any |= v != 0;
    }
  }
  return __syncthreads_or(any ? 1 : 0) != 0;
}

// ------------------------------------------------------------------------------------------------ one quartic
// Runs A1-A7 for one quartic with the CTA's two workspace buffers; returns the height code (thread 0 writes it).
// The same product behind a call boundary, for the cold call sites (the first p-2 products, the identity power
// mode): inlining the large tiled loop at every call site would multiply the build time without a speed gain.
template <int P, int FORM, bool DEBUG>
__device__ __noinline__ void chain_step_call(const uint32_t *in, uint32_t *out, int m_in, Smem &sm, uint32_t *ring,
                                             const uint8_t *gs, uint32_t *status, DebugPtrs dbg) {
  chain_step<P, FORM, false, DEBUG>(in, out, m_in, sm, ring, gs, status, dbg);
}

// A1: read the 35 coefficients into the tap tables; returns false (after a barrier) if one is >= p.
template <int P>
__device__ __forceinline__ bool setup_quartic(const uint8_t *__restrict__ f35, Smem &sm) {
  using Pr = Prime<P>;
  const int tid = threadIdx.x;
  int bad = 0;
  if (tid < 35) {
    const int a = f35[tid];
    bad = a >= P;
    sm.taps[tid] = a;
  }
  if (__syncthreads_or(bad)) return false;
  if (tid == 0) {
    uint32_t mask = 0;
    for (int uI = 0; uI <= 4; ++uI)
      for (int sI = 0; sI <= uI; ++sI) {
        uint32_t tw = 0;
        bool nz = false;
        for (int tI = 0; tI <= sI; ++tI) {
          const int a = sm.taps[tet(uI) + tri(sI) + tI];
          nz |= a != 0;
          if (tI <= 3) tw |= (uint32_t)a << (8 * (3 - tI));
        }
        sm.tapword[tri(uI) + sI] = tw;
        if (nz) mask |= 1u << (tri(uI) + sI);
      }
    sm.pair_mask = mask;
    for (int c = 0; c < P; ++c) {
      int v = 1;
      for (int e = 0; e < P; ++e) v = (v * c) % Pr::p2;
      sm.powp[c] = v;
    }
  }
  return true;
}

// A2 + A3: f into bufA, the chain to f~^(p-1) mod p^2, and g = f^(p-1) mod p (packed) into gs.  Returns the
// buffer holding f~^(p-1); gs[witness] != 0 means height 1 (read after the closing barrier).
template <int P, int FORM, bool DEBUG>
__device__ __forceinline__ uint32_t *power_to_g(Smem &sm, uint8_t *gs, uint32_t *ring, uint32_t *bufA,
                                                uint32_t *bufB, uint32_t *status, DebugPtrs dbg) {
  using Pr = Prime<P>;
  const int tid = threadIdx.x;
  // f into bufA (padded, degree 4: every column is one chunk)
  for (int k = tid; k < sm.SW[5] / 4; k += blockDim.x) {
    int u, s, c;
    decode_form_chunk(k, 4, sm.SW, u, s, c);
    uint32_t words[4] = {0, 0, 0, 0};
    for (int t = 0; t <= s; ++t) words[t >> 2] |= (uint32_t)sm.taps[tet(u) + tri(s) + t] << (8 * (t & 3));
    *reinterpret_cast<uint4 *>(bufA + 4 * k) = make_uint4(words[0], words[1], words[2], words[3]);
  }
  __syncthreads();
  uint32_t *cur = bufA, *nxt = bufB;
  int m = 4;
  for (int k = 1; k <= P - 2; ++k) {
    chain_step_call<P, FORM, DEBUG>(cur, nxt, m, sm, ring, gs, status, dbg);
    __syncthreads();
    uint32_t *t = cur; cur = nxt; nxt = t;
    m += 4;
  }
  for (int k = tid; k < sm.SW[Pr::d + 1] / 4; k += blockDim.x) {
    int u, s, c;
    decode_form_chunk(k, Pr::d, sm.SW, u, s, c);
    const uint4 v = *reinterpret_cast<const uint4 *>(cur + 4 * k);
    const uint32_t words[4] = {v.x, v.y, v.z, v.w};
    for (int b = 0; b < 16; ++b) {
      const int t = 16 * c + b;
      if (t <= s) gs[tet(u) + tri(s) + t] = (uint8_t)(((words[b >> 2] >> (8 * (b & 3))) & 0xFFu) % P);
    }
  }
  __syncthreads();
  return cur;
}

// A4 (+ A5 when LAST_DELTA): the chain from f~^(p-1) in `cur` to f~^(p(p-1)); the last product goes to `last_out`.
template <int P, int FORM, bool LAST_DELTA, bool DEBUG>
__device__ __forceinline__ void power_to_G(Smem &sm, const uint8_t *gs, uint32_t *ring, uint32_t *cur,
                                           uint32_t *other, uint32_t *last_out, uint32_t *status, DebugPtrs dbg) {
  using Pr = Prime<P>;
  uint32_t *nxt = other;
  int m = Pr::d;
  for (int k = P - 1; k <= P * (P - 1) - 2; ++k) {
    chain_step<P, FORM, false, DEBUG>(cur, nxt, m, sm, ring, gs, status, dbg);
    __syncthreads();
    uint32_t *t = cur; cur = nxt; nxt = t;
    m += 4;
  }
  chain_step<P, FORM, LAST_DELTA, DEBUG>(cur, last_out ? last_out : nxt, m, sm, ring, gs, status, dbg);
  __syncthreads();
}

// The identity power mode at p <= 7, by residue classes: Delta_1(f^(p-1)) = E(x^p) - f^(p-2)(x^p) Delta_1(f) (mod p)
// (see power_identity) is formed directly in theta_poly's class order.  Splitting Delta_1(f) = sum_sigma
// x^sigma D_sigma(x^p) by the residues sigma of its exponents gives, class by class,
//     Delta_sigma = [sigma = 0] E - f^(p-2) * D_sigma,   D_sigma[c'] = Delta_1(f)[p c' + sigma],  deg D_sigma = 4 - k,
// so every class is a product of the same f^(p-2) (one zero-padded cube in shared memory, loaded once) with a kernel of
// at most 35 taps: about 8e6 MACs per quartic at p = 7 for the whole Delta, and no barrier between classes.  Inputs:
// f^(p-2), Delta_1(f) and E packed (mod p) in global memory; output: the class-ordered copy `dc` that theta_poly
// reads.  poly_tables must have run.  In debug mode the padded Delta is also written to dbg.delta.
template <int P, bool DEBUG>
__device__ __noinline__ void identity_classes(const uint8_t *__restrict__ fpm2_g, const uint8_t *__restrict__ d1f_g,
                                              const uint8_t *__restrict__ E_g, uint32_t *__restrict__ dc,
                                              const Smem &sm, unsigned char *ring, DebugPtrs dbg) {
  using Q = Poly<P>;
  constexpr int d = Q::d, C = Q::C, NOUT = Q::NOUT, l_fpm2 = tet(4 * (P - 2) + 1), l_d1f = tet(4 * P + 1);
  const int tid = threadIdx.x, nthreads = blockDim.x;
  uint8_t *cube = ring;                       // f^(p-2), zero outside its cone
  uint8_t *d1f = ring + Q::CB;                // Delta_1(f) and E, packed, in the second cube's space
  uint8_t *E = d1f + l_d1f;
  uint8_t *dt = ring + Q::idtaps_off;
  const uint16_t *cubeaddr = reinterpret_cast<const uint16_t *>(ring + Q::cubeaddr_off);
  const int4 *cls = reinterpret_cast<const int4 *>(ring + Q::cls_off);
  for (int i = tid; i < Q::CB / 16; i += nthreads) reinterpret_cast<uint4 *>(cube)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < l_d1f; i += nthreads) d1f[i] = d1f_g[i];
  for (int i = tid; i < Q::ld; i += nthreads) E[i] = E_g[i];
  __syncthreads();
  for (int i = tid; i < l_fpm2; i += nthreads) cube[cubeaddr[i]] = fpm2_g[i];
  // taps of every class: D_sigma[c'] = Delta_1(f)[(p u_c + Su, p s_c + Ss, p t_c + St)], c' in B_{4-k}
  for (int j = tid; j < Q::NCLS; j += nthreads) {
    const int4 c = cls[j];
    const int k = c.z & 255, Su = (c.z >> 8) & 255, Ss = (c.z >> 16) & 255, St = (c.z >> 24) & 255;
    int i = 0;
    for (int uc = 0; uc <= 4 - k; ++uc)
      for (int sc = 0; sc <= uc; ++sc)
        for (int tc = 0; tc <= sc; ++tc, ++i)
          dt[c.w + i] = d1f[tet(P * uc + Su) + tri(P * sc + Ss) + P * tc + St];
  }
  __syncthreads();
  int a[NOUT];
#pragma unroll
  for (int o = 0; o < NOUT; ++o) {
    const int r = tid + kThreads * o;
    a[o] = r < Q::ld ? (int)cubeaddr[r] : Q::pad * (C * C + C + 1);
  }
  uint8_t *dcb = reinterpret_cast<uint8_t *>(dc);
  for (int j = 0; j < Q::NCLS; ++j) {
    const int4 c = cls[j];
    const int k = c.z & 255;
    int acc[NOUT];
#pragma unroll
    for (int o = 0; o < NOUT; ++o) acc[o] = 0;
    const uint8_t *tp = dt + c.w;
    switch (k) {
      case 0: poly_macs<P, 4>(cube, tp, a, acc); break;
      case 1: poly_macs<P, 3>(cube, tp, a, acc); break;
      case 2: poly_macs<P, 2>(cube, tp, a, acc); break;
      default: poly_macs<P, 1>(cube, tp, a, acc); break;
    }
    const int len = tet(d - k + 1);
    const bool lattice = ((c.z >> 8) & 0xFFFFFF) == 0;   // sigma = 0: the class that receives E(x^p)
#pragma unroll
    for (int o = 0; o < NOUT; ++o) {
      const int r = tid + kThreads * o;
      if (r < len) {
        int v = -(acc[o] % P);
        if (lattice) v += E[r];
        if (v < 0) v += P;
        dcb[c.x + r] = (uint8_t)v;
      }
    }
  }
  if (DEBUG) {
    // the padded Delta for the parity hook: every word cleared, then each class's bytes at (p u' + Su, ...)
    __syncthreads();
    for (int k2 = tid; k2 < sm.SW[Prime<P>::D + 1]; k2 += nthreads) dbg.delta[k2] = 0u;
    __syncthreads();
    uint8_t *pd = reinterpret_cast<uint8_t *>(dbg.delta);
    for (int j = 0; j < Q::NCLS; ++j) {
      const int4 c = cls[j];
      const int k = c.z & 255, Su = (c.z >> 8) & 255, Ss = (c.z >> 16) & 255, St = (c.z >> 24) & 255;
      for (int r = tid; r < tet(d - k + 1); r += nthreads) {
        const int ca = cubeaddr[r];
        const int u = ca / (C * C) - Q::pad, s = (ca / C) % C - Q::pad, t = ca % C - Q::pad;
        pd[4 * (sm.SW[P * u + Su] + colw(P * s + Ss)) + P * t + St] = dcb[c.x + r];
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------ identity power
// A4 + A5 by an exact algebraic shortcut (power mode QFS_POWER_IDENTITY).  It produces the same Delta_1(f^(p-1))
// array as the chain, and the chain stays the literal reading of Algorithm 1.
//   Write f~^p = A + p D~ with A = sum_I a~_I^p x^(pI) and D~ = Delta_1(f) mod p (Proposition of Sec. 3.1).  Then
//   lift(g)^p = f~^(p(p-1)) = (A + p D~)^(p-1) = A^(p-1) - p A^(p-2) D~ (mod p^2), and A = f(x^p) (mod p), so
//     Delta_1(f^(p-1)) = E(x^p) - f^(p-2)(x^p) Delta_1(f)   (mod p),
//   E_J = (A~^(p-1)[J] - c~_J^p) / p with A~(y) = sum_I (a~_I^p mod p^2) y^I and c_J the coefficients of g.
// Work per quartic at p = 7: one chain product to f~^p, p-2 small products for A~^(p-1), and about 8e6 MACs for
// f^(p-2)(x^p) Delta_1(f) -- against 2.9e8 for the chain.
template <int P, int FORM, bool DEBUG>
__device__ __noinline__ uint32_t *power_identity(Smem &sm, const uint8_t *gs, uint32_t *ring, uint32_t *cur,
                                                    uint32_t *other, uint32_t *status, DebugPtrs dbg) {
  using Pr = Prime<P>;
  constexpr int d = Pr::d, D = Pr::D, dm = 4 * (P - 2), d1 = 4 * P;
  constexpr int l_fpm2 = tet(dm + 1), l_d1f = tet(d1 + 1), l_E = Pr::ld;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  // byte scratch in global memory after f~^p in `other`
  uint8_t *fpm2_g = reinterpret_cast<uint8_t *>(other + sm.SW[d1 + 1]);
  uint8_t *d1f_g = fpm2_g + l_fpm2;
  uint8_t *E_g = d1f_g + l_d1f;
  // f^(p-2) mod p: `other` holds f~^(p-2) (degree dm) after power_to_g
  for (int k = tid; k < sm.SW[dm + 1] / 4; k += nthreads) {
    int u, s, c;
    decode_form_chunk(k, dm, sm.SW, u, s, c);
    const uint4 v = *reinterpret_cast<const uint4 *>(other + 4 * k);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    for (int b = 0; b < 16 && 16 * c + b <= s; ++b)
      fpm2_g[tet(u) + tri(s) + 16 * c + b] = (uint8_t)(((w[b >> 2] >> (8 * (b & 3))) & 0xFFu) % P);
  }
  __syncthreads();
  // f~^p = f~^(p-1) f~ (mod p^2) into `other`, then Delta_1(f) = (f~^p - sum a~_I^p x^(pI)) / p mod p
  chain_step_call<P, FORM, DEBUG>(cur, other, d, sm, ring, gs, status, dbg);
  __syncthreads();
  bool bad = false;
  for (int k = tid; k < sm.SW[d1 + 1] / 4; k += nthreads) {
    int u, s, c;
    decode_form_chunk(k, d1, sm.SW, u, s, c);
    const uint4 v = *reinterpret_cast<const uint4 *>(other + 4 * k);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    for (int b = 0; b < 16 && 16 * c + b <= s; ++b) {
      const int t = 16 * c + b;
      int G = (int)((w[b >> 2] >> (8 * (b & 3))) & 0xFFu);
      if ((u % P) == 0 && (s % P) == 0 && (t % P) == 0) {
        G -= sm.powp[sm.taps[tet(u / P) + tri(s / P) + t / P]];
        if (G < 0) G += Pr::p2;
      }
      if (G % P) bad = true;
      d1f_g[tet(u) + tri(s) + t] = (uint8_t)(G / P);
    }
  }
  __syncthreads();
  // A~ (coefficients a~_I^p mod p^2) into cur, then A~^(p-1) mod p^2 by p-2 chain products (ping-pong inside cur)
  if (tid < 35) sm.taps[tid] = sm.powp[sm.taps[tid]];
  __syncthreads();
  if (tid == 0) {
    uint32_t mask = 0;
    for (int uI = 0; uI <= 4; ++uI)
      for (int sI = 0; sI <= uI; ++sI) {
        uint32_t tw = 0;
        bool nz = false;
        for (int tI = 0; tI <= sI; ++tI) {
          const int a = sm.taps[tet(uI) + tri(sI) + tI];
          nz |= a != 0;
          if (tI <= 3) tw |= (uint32_t)a << (8 * (3 - tI));
        }
        sm.tapword[tri(uI) + sI] = tw;
        if (nz) mask |= 1u << (tri(uI) + sI);
      }
    sm.pair_mask = mask;
  }
  // pa = cur, pb after pa's largest form and a guard of zero words (chain products read from both)
  uint32_t *pa = cur, *pb = cur + sm.SW[d + 1] + kGuardWords;
  if (tid < kGuardWords) pb[tid - kGuardWords] = 0u;
  for (int k = tid; k < sm.SW[5] / 4; k += nthreads) {
    int u, s, c;
    decode_form_chunk(k, 4, sm.SW, u, s, c);
    uint32_t words[4] = {0, 0, 0, 0};
    for (int t = 0; t <= s; ++t) words[t >> 2] |= (uint32_t)sm.taps[tet(u) + tri(s) + t] << (8 * (t & 3));
    *reinterpret_cast<uint4 *>(pa + 4 * k) = make_uint4(words[0], words[1], words[2], words[3]);
  }
  __syncthreads();
  for (int m = 4; m < d; m += 4) {
    chain_step_call<P, FORM, DEBUG>(pa, pb, m, sm, ring, gs, status, dbg);
    __syncthreads();
    uint32_t *t = pa; pa = pb; pb = t;
  }
  // E_J = (A~^(p-1)[J] - c~_J^p) / p mod p
  for (int k = tid; k < sm.SW[d + 1] / 4; k += nthreads) {
    int u, s, c;
    decode_form_chunk(k, d, sm.SW, u, s, c);
    const uint4 v = *reinterpret_cast<const uint4 *>(pa + 4 * k);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    for (int b = 0; b < 16 && 16 * c + b <= s; ++b) {
      const int J = tet(u) + tri(s) + 16 * c + b;
      int G = (int)((w[b >> 2] >> (8 * (b & 3))) & 0xFFu) - sm.powp[gs[J]];
      if (G < 0) G += Pr::p2;
      if (G % P) bad = true;
      E_g[J] = (uint8_t)(G / P);
    }
  }
  __syncthreads();
  if constexpr (theta_by_classes<P>()) {
    // Delta straight into theta's class order, in `cur` (the products above are done with it)
    if (bad) atomicOr(status, kStatusInexactDivision);
    unsigned char *ringb = reinterpret_cast<unsigned char *>(ring);
    poly_tables<P>(ringb);
    identity_classes<P, DEBUG>(fpm2_g, d1f_g, E_g, cur, sm, ringb, dbg);
    __syncthreads();
    return cur;
  }
  // stage the three small arrays in shared memory
  uint8_t *fpm2 = reinterpret_cast<uint8_t *>(ring), *d1f = fpm2 + l_fpm2, *E = d1f + l_d1f;
  for (int i = tid; i < l_fpm2 + l_d1f + l_E; i += nthreads) fpm2[i] = fpm2_g[i];
  __syncthreads();
  // Delta[e] = E(x^p)[e] - sum_{pJ + K = e} f^(p-2)[J] Delta_1(f)[K] mod p, written to cur in the padded layout
  uint32_t *delta = cur;
  for (int k = tid; k < sm.SW[D + 1] / 4; k += nthreads) {
    int ue, se, c;
    decode_form_chunk(k, D, sm.SW, ue, se, c);
    int acc[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) acc[b] = 0;
    const int uj_lo = ue > d1 ? (ue - d1 + P - 1) / P : 0, uj_hi = min(dm, ue / P);
    for (int uj = uj_lo; uj <= uj_hi; ++uj) {
      const int uk = ue - P * uj;
      const int sj_lo = se > uk ? (se - uk + P - 1) / P : 0, sj_hi = min(uj, se / P);
      for (int sj = sj_lo; sj <= sj_hi; ++sj) {
        const int sk = se - P * sj;
        const uint8_t *fj = fpm2 + tet(uj) + tri(sj);
        const uint8_t *dk = d1f + tet(uk) + tri(sk);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          const int te = 16 * c + b;
          if (te <= se) {
            const int tj_lo = te > sk ? (te - sk + P - 1) / P : 0, tj_hi = min(sj, te / P);
            for (int tj = tj_lo; tj <= tj_hi; ++tj) acc[b] += (int)fj[tj] * (int)dk[te - P * tj];
          }
        }
      }
    }
    uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      const int te = 16 * c + b;
      if (te <= se) {
        int v = -(acc[b] % P);
        if ((ue % P) == 0 && (se % P) == 0 && (te % P) == 0) v += E[tet(ue / P) + tri(se / P) + te / P];
        if (v < 0) v += P;
        w[b >> 2] |= (uint32_t)v << (8 * (b & 3));
      }
    }
    *reinterpret_cast<uint4 *>(delta + 4 * k) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  if (bad) atomicOr(status, kStatusInexactDivision);
  __syncthreads();
  return delta;
}

// ------------------------------------------------------------------------------------------------ reduced theta
// Heights without Delta_1(f^(p-1)) (power mode QFS_POWER_REDUCED).  From f~^p = A + p Delta_1(f) and the
// semilinearity of u over p-th powers (Algorithm 2 moves x^(pJ) out as x^J), every iterate F that the loop applies
// theta to has F[witness] = 0, and for such F
//     theta(F) = u(F Delta_1(f^(p-1))) = - f^(p-2) u(F Delta_1(f))   (mod p),
// where u(F Delta_1(f)) is a quartic.  One step costs about 2e5 MACs at p = 7 instead of 6.8e6, and neither
// G nor the 819k-entry Delta is formed.  Same heights as the other modes (the oracle's route R is this identity).
template <int P>
__device__ __forceinline__ int cone_index(int u, int s, int t) { return tet(u) + tri(s) + t; }

template <int P, int FORM, bool DEBUG>
__device__ __noinline__ int reduced_height(Smem &sm, uint8_t *gs, uint8_t *gn, uint32_t *ring, uint32_t *cur,
                                           uint32_t *other, int max_h, uint32_t *status, DebugPtrs dbg,
                                           int &theta_steps) {
  using Pr = Prime<P>;
  constexpr int d = Pr::d, dm = 4 * (P - 2), d1 = 4 * P;
  constexpr int l_fpm2 = tet(dm + 1), l_d1f = tet(d1 + 1);
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nthreads >> 5;
  uint8_t *fpm2 = reinterpret_cast<uint8_t *>(ring);
  uint8_t *d1f = fpm2 + l_fpm2;
  int *q = reinterpret_cast<int *>(ring + (l_fpm2 + l_d1f + 3) / 4 + 1);
  // f^(p-2) mod p from `other` (degree dm)
  for (int k = tid; k < sm.SW[dm + 1] / 4; k += nthreads) {
    int u, s, c;
    decode_form_chunk(k, dm, sm.SW, u, s, c);
    const uint4 v = *reinterpret_cast<const uint4 *>(other + 4 * k);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    for (int b = 0; b < 16 && 16 * c + b <= s; ++b)
      fpm2[tet(u) + tri(s) + 16 * c + b] = (uint8_t)(((w[b >> 2] >> (8 * (b & 3))) & 0xFFu) % P);
  }
  __syncthreads();
  // f~^p = f~^(p-1) f~ (mod p^2), then Delta_1(f) = (f~^p - sum a~_I^p x^(pI)) / p mod p
  // the product's slot ring goes after fpm2, d1f and q, on a 16-byte boundary (16-byte cp.async and loads)
  constexpr int ring_off = (((l_fpm2 + l_d1f + 3) / 4 + 64) + 3) & ~3;   // same offset as aux_ring_words
  static_assert(ring_off % 4 == 0, "16-byte aligned ring");
  chain_step_call<P, FORM, DEBUG>(cur, other, d, sm, ring + ring_off, gs, status, dbg);
  __syncthreads();
  bool bad = false;
  for (int k = tid; k < sm.SW[d1 + 1] / 4; k += nthreads) {
    int u, s, c;
    decode_form_chunk(k, d1, sm.SW, u, s, c);
    const uint4 v = *reinterpret_cast<const uint4 *>(other + 4 * k);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    for (int b = 0; b < 16 && 16 * c + b <= s; ++b) {
      const int t = 16 * c + b;
      int G = (int)((w[b >> 2] >> (8 * (b & 3))) & 0xFFu);
      if ((u % P) == 0 && (s % P) == 0 && (t % P) == 0) {
        G -= sm.powp[sm.taps[tet(u / P) + tri(s / P) + t / P]];
        if (G < 0) G += Pr::p2;
      }
      if (G % P) bad = true;
      d1f[tet(u) + tri(s) + t] = (uint8_t)(G / P);
    }
  }
  if (bad) atomicOr(status, kStatusInexactDivision);
  __syncthreads();
  uint8_t *F = gs, *Fn = gn;
  for (int h = 2; h <= max_h; ++h) {
    // q[r] = u(F Delta_1(f))[r] = sum_c Delta_1(f)[p r + (p-1,..,p-1) - c] F[c], r in B_4: one warp per r
    for (int r = warp; r < 35; r += nwarps) {
      int ur, sr, tr;
      decode_packed(r, ur, sr, tr, 4);
      const int eu0 = P * ur + 3 * (P - 1), es0 = P * sr + 2 * (P - 1), et0 = P * tr + (P - 1);
      unsigned a = 0;
      // g column col = tri(uc) + sc of this lane, advanced 32 columns at a time
      int uc = (isqrt(8 * lane + 1) - 1) >> 1, sc = lane - tri(uc);
      for (int col = lane; col < tri(d + 1); col += 32, sc += 32) {
        while (sc > uc) sc -= ++uc;
        const int eu = eu0 - uc, es = es0 - sc;
        if (eu < 0 || eu > d1 || es < 0 || es > eu) continue;
        const int tlo = max(0, et0 - es), thi = min(sc, et0);
        const uint8_t *dcol = d1f + tet(eu) + tri(es) + et0;   // Delta_1(f)(eu, es, et0 - tc) = dcol[-tc]
        const uint8_t *fcol = F + tet(uc) + tri(sc);
        for (int tc = tlo; tc <= thi; ++tc) a += (unsigned)dcol[-tc] * fcol[tc];
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
      if (lane == 0) q[r] = (int)(a % P);
    }
    __syncthreads();
    // F_next = -f^(p-2) q  (mod p): a 35-tap product onto B_d
    bool any = false;
    for (int e = tid; e < Pr::ld; e += nthreads) {
      int ue, se, te;
      decode_packed(e, ue, se, te, d);
      int acc = 0;
      int I = 0;   // packed index tet(uI) + tri(sI) + tI of the tap
      for (int uI = 0; uI <= 4; ++uI)
        for (int sI = 0; sI <= uI; ++sI)
          for (int tI = 0; tI <= sI; ++tI, ++I) {
            const int qi = q[I];
            if (!qi) continue;
            const int u2 = ue - uI, s2 = se - sI, t2 = te - tI;
            if (t2 < 0 || s2 < t2 || u2 < s2 || u2 > dm) continue;
            acc += qi * (int)fpm2[tet(u2) + tri(s2) + t2];
          }
      int v = -(acc % P);
      if (v < 0) v += P;
      Fn[e] = (uint8_t)v;
      any |= v != 0;
    }
    const int nonzero = __syncthreads_or(any ? 1 : 0);
    theta_steps = h - 1;
    if (DEBUG)
      for (int i = tid; i < Pr::ld; i += nthreads) dbg.iters[(size_t)(h - 2) * Pr::ld + i] = Fn[i];
    if (Fn[Pr::witness] != 0) return h;
    if (!nonzero) return 0;
    uint8_t *t = F; F = Fn; Fn = t;
    __syncthreads();
  }
  return 0;
}

// Runs A1-A7 for one quartic with the CTA's two workspace buffers; returns the height code.
template <int P, int FORM, bool DEBUG>
__device__ int process_quartic(const uint8_t *__restrict__ f35, int max_h, Smem &sm, uint8_t *gs, uint8_t *gn,
                               uint32_t *ring, uint32_t *bufA, uint32_t *bufB, uint32_t *status, DebugPtrs dbg,
                               int &theta_steps, int power_mode = 0) {
  using Pr = Prime<P>;
  const int tid = threadIdx.x;
  theta_steps = 0;
  if (!setup_quartic<P>(f35, sm)) return -1;
  uint32_t *cur = power_to_g<P, FORM, DEBUG>(sm, gs, ring, bufA, bufB, status, dbg);
  uint32_t *other = cur == bufA ? bufB : bufA;
  if (DEBUG)
    for (int i = tid; i < Pr::ld; i += blockDim.x) dbg.g[i] = gs[i];
  if (gs[Pr::witness] != 0) return 1;
  if (power_mode == 2)
    return reduced_height<P, FORM, DEBUG>(sm, gs, gn, ring, cur, other, max_h, status, dbg, theta_steps);
  // A4 + A5 into `other` or `cur`, whichever the chain's parity leaves last
  constexpr int nsteps = P * (P - 1) - (P - 1);   // products from f~^(p-1) to f~^(p(p-1))
  uint32_t *delta;
  // the identity mode at p <= 7 leaves Delta already in theta's class order (and the debug copy written)
  const bool in_classes = power_mode == 1 && theta_by_classes<P>();
  if (power_mode == 1) {
    delta = power_identity<P, FORM, DEBUG>(sm, gs, ring, cur, other, status, dbg);
  } else {
    delta = (nsteps % 2) ? other : cur;
    power_to_G<P, FORM, true, DEBUG>(sm, gs, ring, cur, other, nullptr, status, dbg);
  }
  if (DEBUG && !in_classes)
    for (int k = tid; k < sm.SW[Pr::D + 1]; k += blockDim.x) dbg.delta[k] = delta[k];
  // A6 + A7.  Theta: by residue classes at p <= 5 and for the identity mode at p = 7 (Delta in class order, copied
  // into the buffer that does not hold Delta unless the identity mode wrote it so), streamed from the padded Delta
  // at p = 7 otherwise, and gathered from a guarded copy at p >= 11
  uint32_t *dg = delta == bufA ? bufB : bufA;
  unsigned char *ringb = reinterpret_cast<unsigned char *>(ring);
  const bool by_classes = theta_by_classes<P>() && (!theta_streams<P>() || in_classes);
  if constexpr (theta_by_classes<P>()) {
    if (in_classes) {
      dg = delta;
    } else if (by_classes) {
      poly_tables<P>(ringb);
      delta_to_classes<P>(delta, dg, sm, ringb);
    }
  } else {
    delta_to_guarded<P>(delta, dg, sm);
  }
  __syncthreads();
  uint8_t *g = gs, *g2 = gn;
  for (int h = 2; h <= max_h; ++h) {
    bool nonzero;
    if constexpr (theta_by_classes<P>()) {
      if (by_classes) nonzero = theta_poly<P>(dg, g, g2, ringb);
      else nonzero = theta_stream<P>(delta, sm, g, g2, ring);
    } else {
      nonzero = theta_gather<P>(dg, sm, g, g2, ring);
    }
    theta_steps = h - 1;
    if (DEBUG)
      for (int i = tid; i < Pr::ld; i += blockDim.x) dbg.iters[(size_t)(h - 2) * Pr::ld + i] = g2[i];
    if (g2[Pr::witness] != 0) return h;
    if (!nonzero) return 0;
    uint8_t *t = g; g = g2; g2 = t;
    __syncthreads();
  }
  return 0;
}

// ------------------------------------------------------------------------------------------------ fused launch
struct FusedGroup {
  int p;
  int64_t n;
  const uint8_t *coeffs;
  int8_t *heights;
  int64_t item_begin;
  int tile_round, tile_ring;
  int dense_min;
};

constexpr int kMaxGroups = 8;

struct FusedParams {
  FusedGroup g[kMaxGroups];
  int n_groups;
  int64_t n_items;
  int max_h;
  int sw_len;                         // SW entries to build (max D in this launch + 2)
  unsigned long long *counter;        // work queue head (zeroed before launch)
  uint32_t *status;
  unsigned long long *stats;          // [0] quartics past the height-1 test, [1] theta steps run
  uint32_t *ws;                       // workspace: a guard, then 2 buffers of ws_words (the stride) per CTA
  size_t ws_words;
  int power_mode;                     // 0: chain (Algorithm 1 literally), 1: identity shortcut, 2: reduced theta
  const int64_t *list;                // if set: the items to run (the survivors of the height-1 screen) ...
  const unsigned long long *n_list;   // ... and their count; if null, every item 0 .. n_items-1 runs
};

// SMALL: an int8 tensor form launch whose primes are all <= 5; the kernel then needs no code for larger primes and
// can keep three CTAs per SM.
template <int FORM, bool SMALL>
__device__ __forceinline__ void fused_body(const FusedParams &prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  uint8_t *gs = smem_raw + sizeof(Smem);
  // the second iterate buffer follows the largest ld in this launch
  int max_ld = 0;
  for (int i = 0; i < prm.n_groups; ++i) max_ld = max(max_ld, tet(4 * (prm.g[i].p - 1) + 1));
  uint8_t *gn = gs + max_ld;
  uint32_t *ring = reinterpret_cast<uint32_t *>(smem_raw + ring_offset_for(max_ld));
  build_sw(sm.SW, prm.sw_len);
  init_task_queue(sm);
  uint32_t *bufA, *bufB;
  cta_buffers(prm.ws, prm.ws_words, bufA, bufB);
  DebugPtrs dbg{nullptr, nullptr, nullptr, nullptr};
  const int64_t n_run = prm.list ? (int64_t)*prm.n_list : prm.n_items;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t k = (int64_t)atomicAdd(prm.counter, 1ull);
      sm.item = k < n_run ? (prm.list ? prm.list[k] : k) : -1;
    }
    __syncthreads();
    const int64_t item = sm.item;
    if (item < 0) break;
    int gi = 0;
    while (gi + 1 < prm.n_groups && item >= prm.g[gi + 1].item_begin) ++gi;
    const FusedGroup &G = prm.g[gi];
    const int64_t row = item - G.item_begin;
    if (threadIdx.x == 0) {
      sm.tile_round = G.tile_round;
      sm.tile_ring = G.tile_ring;
      sm.dense_min = G.dense_min;
    }
    const uint8_t *f = G.coeffs + 35 * row;
    int h, steps;
    switch (G.p) {
      case 3: h = process_quartic<3, FORM, false>(f, prm.max_h, sm, gs, gn, ring, bufA, bufB, prm.status, dbg, steps, prm.power_mode); break;
      case 5: h = process_quartic<5, FORM, false>(f, prm.max_h, sm, gs, gn, ring, bufA, bufB, prm.status, dbg, steps, prm.power_mode); break;
      default:
        if constexpr (SMALL) {
          h = -1;   // not reached: the host launches the small-prime kernel only when every group has p <= 5
        } else {
          switch (G.p) {
            case 7: h = process_quartic<7, FORM, false>(f, prm.max_h, sm, gs, gn, ring, bufA, bufB, prm.status, dbg, steps, prm.power_mode); break;
            case 11: h = process_quartic<11, FORM, false>(f, prm.max_h, sm, gs, gn, ring, bufA, bufB, prm.status, dbg, steps, prm.power_mode); break;
            default: h = process_quartic<13, FORM, false>(f, prm.max_h, sm, gs, gn, ring, bufA, bufB, prm.status, dbg, steps, prm.power_mode); break;
          }
        }
        break;
    }
    if (threadIdx.x == 0) {
      G.heights[row] = (int8_t)h;
      if (h != 1 && h != -1) {
        atomicAdd(prm.stats, 1ull);
        atomicAdd(prm.stats + 1, (unsigned long long)steps);
      }
    }
  }
}

}  // namespace qfs
