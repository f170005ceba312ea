// One product of the chain, out = in * f~ (mod p^2), by per-lane sweeps over the input slices (dp4a and int32
// forms).  Algorithm 1 needs lift(g)^p mod p^2; the chain forms it as f~^(p(p-1)) one multiplication by f~ at a time
// (see qfs_engine.cuh), and this file is that multiplication.
//
// Work item = one half-chunk of an output column: column s of the output slices, outputs t = 8h .. 8h+7 (h is
// the half-chunk; column s has s/8 + 1 of them).  A lane owns one item for every output slice u and walks the
// input slices v upwards.  Input slice v feeds output slices u = v .. v+4 (tap pairs uI = u - v): the lane loads
// the five input columns s - sI (sI = 0..4) of slice v once (eight bytes plus the word before them), builds the
// byte windows once, and adds every tap pair (uI, sI) with uI >= sI into the accumulator set of output u = v + uI.
// Six accumulator sets: five hold the output slices v .. v + 4 that slice v feeds, the sixth the output slice
// completed by the previous slice, which is reduced, packed and stored while this slice's loads are in flight.
// The dense dp4a path takes the slices two at a time, so the sets move down two places per pair.
//
// Compared with staging the slices through shared memory, every input word is loaded once per lane and slice
// rather than once per tap pair, windows are built once per input column rather than once per pair, and the
// warps of a CTA never wait for each other inside a product: a warp takes 32 consecutive items (a task) and
// sweeps them alone.  Neighbouring lanes and neighbouring warps read the same input columns at about the same
// slice, so the repeated reads are served by L1.
#pragma once
#include <cstdint>
#include "qfs_common.cuh"

namespace qfs {

// Half-chunk items of a degree-m form: column s has half_chunks_of(s) items; half_prefix(s) items precede
// column s.  For s = 8a + b: half_prefix(s) = sum_{s' < s} (s'/8 + 1) = (a + 1)(4a + b).
__host__ __device__ constexpr int half_chunks_of(int s) { return (s >> 3) + 1; }
__host__ __device__ constexpr int half_prefix(int s) { return ((s >> 3) + 1) * (4 * (s >> 3) + (s & 7)); }

// Item index i -> (column s, half-chunk h).  Columns 8a .. 8a+7 hold a+1 items each, starting at 4a(a+1).
__host__ __device__ inline void decode_half(int i, int &s, int &h) {
  int a = (isqrt(1 + i) - 1) >> 1;
  while (4 * (a + 1) * (a + 2) <= i) ++a;
  while (a > 0 && 4 * a * (a + 1) > i) --a;
  const int rem = i - 4 * a * (a + 1);
  const int b = small_quotient<3>(rem, a + 1);   // rem < 8 (a + 1)
  h = rem - b * (a + 1);
  s = 8 * a + b;
}

// Zeroes the task queue of the swept chain; every kernel that runs a chain product calls it once, before its
// first barrier.
__device__ __forceinline__ void init_task_queue(Smem &sm) {
  if (threadIdx.x == 0) {
    sm.task_next = 0;
    sm.task_done = 0;
  }
}

namespace sweep {

// Per-lane state of one task (fixed while the lane sweeps the slices).
struct Lane {
  int s, h;
  int off[5];      // word offset of input column s - sI, half-chunk h, inside a slice
  int first[5];    // first input slice holding column s - sI (s - sI; past every slice if the column or item does not exist)
  int out_off;     // word offset of the output half-chunk inside a slice
  int pad;         // half-chunks of zero padding after this item that this lane writes (0, 1 or 2)
  bool valid;      // the item exists
};

// Input words of slice v for one lane: X[sI] = {word 2h-1, word 2h, word 2h+1} of column s - sI.  The padded
// layout makes every such read safe and exact without predication: the column (sized for s - sI + 4 entries) holds
// words 2h .. 2h+1, the word before a column is padding, and a column that does not exist in slice v (s - sI > v,
// s - sI < 0, or no item) is read from the zero guard words in[-3 .. -1] in front of the buffer.
template <int P>
__device__ __forceinline__ void load_slice(const uint32_t *__restrict__ in, const Smem &sm, const Lane &L, int v,
                                           uint32_t (&X)[5][3]) {
  const int base = sm.SW[max(v, 0)];  // v = -1 (a leading slice with no columns) reads only guard words
#pragma unroll
  for (int sI = 0; sI < 5; ++sI) {
    const bool ex = v >= L.first[sI];
    const uint32_t *q = in + (ex ? base + L.off[sI] : -2);
    const uint2 w = *reinterpret_cast<const uint2 *>(q);
    X[sI][0] = q[-1];
    X[sI][1] = w.x;
    X[sI][2] = w.y;
  }
}

// Contributions of input column s - SI of slice v (words X) to the output sets J + uI, uI = SI .. 4.
template <int J, int SI, int FORM, bool DENSE>
__device__ __forceinline__ void column_macs(const uint32_t (&X)[3], const uint32_t (&tw)[15], uint32_t a44,
                                            const int (&taps)[35], uint32_t mask, uint32_t colmask,
                                            int (&acc)[6][8]) {
  if (!DENSE && !((colmask >> SI) & 1u)) return;  // every tap pair of this input column is zero
  if (FORM == 1) {
    // window of output t = 8h + 4q + r: bytes in(t-3 .. t) = bytes r+1 .. r+4 of (word q-1 of the half-chunk,
    // word q); word -1 is X[0]
    uint32_t W[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      W[q][0] = __byte_perm(X[q], X[q + 1], 0x4321u);
      W[q][1] = __byte_perm(X[q], X[q + 1], 0x5432u);
      W[q][2] = __byte_perm(X[q], X[q + 1], 0x6543u);
      W[q][3] = X[q + 1];
    }
#pragma unroll
    for (int uI = SI; uI < 5; ++uI) {
      const int pi = uI * (uI + 1) / 2 + SI;
      if (DENSE || ((mask >> pi) & 1u)) {
        const int set = J + uI;
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int r = 0; r < 4; ++r)
            acc[set][4 * q + r] = (int)__dp4a(W[q][r], tw[pi], (unsigned)acc[set][4 * q + r]);
      }
    }
    if (SI == 4 && (DENSE || ((mask >> 14) & 1u))) {
      // tap (4, 4, 4) reads in(t - 4) = byte r of word q-1
      const int set = J + 4;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          acc[set][4 * q + r] = (int)__dp4a(X[q], a44 << (8 * r), (unsigned)acc[set][4 * q + r]);
    }
  } else {
    // int32 form: b[k] = in(8h - 4 + k), k = 0 .. 11
    int b[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) b[k] = (int)((X[k >> 2] >> (8 * (k & 3))) & 0xFFu);
#pragma unroll
    for (int uI = SI; uI < 5; ++uI) {
      const int pi = uI * (uI + 1) / 2 + SI;
      if (DENSE || ((mask >> pi) & 1u)) {
        const int set = J + uI;
#pragma unroll
        for (int tI = 0; tI <= SI; ++tI) {
          const int a = taps[tet(uI) + tri(SI) + tI];
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[set][j] += a * b[j + 4 - tI];
        }
      }
    }
  }
}

// Byte windows of one input column: W[q][r] holds in(t - 3 .. t) (byte k = in(t - 3 + k)) for the output
// t = 8h + 4q + r, from the words X = {word 2h - 1, 2h, 2h + 1} of the column.
__device__ __forceinline__ void column_windows(const uint32_t (&X)[3], uint32_t (&W)[2][4]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    W[q][0] = __byte_perm(X[q], X[q + 1], 0x4321u);
    W[q][1] = __byte_perm(X[q], X[q + 1], 0x5432u);
    W[q][2] = __byte_perm(X[q], X[q + 1], 0x6543u);
    W[q][3] = X[q + 1];
  }
}

// dp4a form, every tap pair present: slice v into the sets J .. J + 4.  A pair (uI, sI) has sI + 1 taps, so the
// windows of the pairs (1, 1) and (uI, 2) leave their byte 0 unused; it carries the single tap of (uI, 0) instead
// (byte 0 of the window <- in_0(t), byte 0 of the tap word <- a(uI, 0, 0), merged into tw by the caller).  That is
// 12 dp4a per output in place of 16, for 16 byte permutes per slice.
template <int J>
__device__ __forceinline__ void slice_macs_merged(const uint32_t (&X)[5][3], const uint32_t (&tw)[15], uint32_t a44,
                                                  int (&acc)[6][8]) {
  // pair (0, 0) has the single tap a(0,0,0) (byte 3 of tw[0]) on in_0(t), which is byte r of word q + 1 of
  // column 0: no window, a dp4a against the tap shifted to byte r
  const uint32_t a00 = tw[0] >> 24;
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r)
      acc[J][4 * q + r] = (int)__dp4a(X[0][q + 1], a00 << (8 * r), (unsigned)acc[J][4 * q + r]);
  {
    uint32_t W1[2][4];
    column_windows(X[1], W1);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t m = __byte_perm(W1[q][r], X[0][q + 1], 0x3214u + r);   // byte 0 <- in_0(t)
        acc[J + 1][4 * q + r] = (int)__dp4a(m, tw[2], (unsigned)acc[J + 1][4 * q + r]);
      }
#pragma unroll
    for (int uI = 2; uI < 5; ++uI)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          acc[J + uI][4 * q + r] = (int)__dp4a(W1[q][r], tw[tri(uI) + 1], (unsigned)acc[J + uI][4 * q + r]);
  }
  {
    uint32_t W2[2][4];
    column_windows(X[2], W2);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t m = __byte_perm(W2[q][r], X[0][q + 1], 0x3214u + r);   // byte 0 <- in_0(t)
#pragma unroll
        for (int uI = 2; uI < 5; ++uI)
          acc[J + uI][4 * q + r] = (int)__dp4a(m, tw[tri(uI) + 2], (unsigned)acc[J + uI][4 * q + r]);
      }
  }
#pragma unroll
  for (int sI = 3; sI < 5; ++sI) {
    uint32_t W[2][4];
    column_windows(X[sI], W);
#pragma unroll
    for (int uI = sI; uI < 5; ++uI)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r)
          acc[J + uI][4 * q + r] = (int)__dp4a(W[q][r], tw[tri(uI) + sI], (unsigned)acc[J + uI][4 * q + r]);
  }
  // tap (4, 4, 4) reads in_4(t - 4) = byte r of word q - 1
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int r = 0; r < 4; ++r)
      acc[J + 4][4 * q + r] = (int)__dp4a(X[4][q], a44 << (8 * r), (unsigned)acc[J + 4][4 * q + r]);
}

// Slice v into the sets J .. J + 4.
template <int J, int FORM, bool DENSE>
__device__ __forceinline__ void slice_macs(const uint32_t (&X)[5][3], const uint32_t (&tw)[15], uint32_t a44,
                                           const int (&taps)[35], uint32_t mask, uint32_t colmask,
                                           int (&acc)[6][8]) {
  if (FORM == 1 && DENSE) {
    slice_macs_merged<J>(X, tw, a44, acc);
  } else {
    column_macs<J, 0, FORM, DENSE>(X[0], tw, a44, taps, mask, colmask, acc);
    column_macs<J, 1, FORM, DENSE>(X[1], tw, a44, taps, mask, colmask, acc);
    column_macs<J, 2, FORM, DENSE>(X[2], tw, a44, taps, mask, colmask, acc);
    column_macs<J, 3, FORM, DENSE>(X[3], tw, a44, taps, mask, colmask, acc);
    column_macs<J, 4, FORM, DENSE>(X[4], tw, a44, taps, mask, colmask, acc);
  }
}

// Output slice u of this lane is complete in set J: reduce mod p^2 (and, in the last product, apply the Delta_1
// epilogue), store, and clear the set.
template <int P, int J, bool LAST, bool DEBUG>
__device__ __forceinline__ void finalize(uint32_t *__restrict__ out, const Smem &sm, const Lane &L, int u,
                                         const uint8_t *gs, int (&acc)[6][8], bool &bad, DebugPtrs dbg) {
  using Pr = Prime<P>;
  if (L.valid && u >= L.s) {
    uint32_t w[2] = {0u, 0u}, gw[2] = {0u, 0u};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int G = (int)mod_p2_mulhi<P>((uint32_t)acc[J][j]);  // acc >= 0; outputs past the column's end are zero
      if (LAST) {
        const int t = 8 * L.h + j;
        if (DEBUG) gw[j >> 2] |= (uint32_t)G << (8 * (j & 3));
        if (t <= L.s && (u % P) == 0 && (L.s % P) == 0 && (t % P) == 0) {
          G -= sm.powp[gs[tet(u / P) + tri(L.s / P) + t / P]];
          if (G < 0) G += Pr::p2;
        }
        if (G % P) bad = true;
        G /= P;
      }
      // byte j & 3 of word j >> 2; a multiply-add (the bytes do not overlap), which keeps the packing off the
      // byte-permute pipe that the windows load
      w[j >> 2] += (uint32_t)G * (1u << (8 * (j & 3)));
    }
    const int o = sm.SW[u] + L.out_off;
    if (L.pad == 1) {
      *reinterpret_cast<uint4 *>(out + o) = make_uint4(w[0], w[1], 0u, 0u);
      if (DEBUG && LAST) *reinterpret_cast<uint4 *>(dbg.G + o) = make_uint4(gw[0], gw[1], 0u, 0u);
    } else {
      *reinterpret_cast<uint2 *>(out + o) = make_uint2(w[0], w[1]);
      if (DEBUG && LAST) *reinterpret_cast<uint2 *>(dbg.G + o) = make_uint2(gw[0], gw[1]);
      if (L.pad == 2) {
        *reinterpret_cast<uint4 *>(out + o + 2) = make_uint4(0u, 0u, 0u, 0u);
        if (DEBUG && LAST) *reinterpret_cast<uint4 *>(dbg.G + o + 2) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[J][j] = 0;
}

// Next task of the current product for this warp (warp-uniform), or -1 when the queue is empty.  Tasks are handed
// out in index order, which is longest first (a task of low columns sweeps more slices).  The last warp to find
// the queue empty resets it for the next product; the caller's barrier orders that reset before the next product.
__device__ __forceinline__ int next_task(Smem &sm, int n_tasks) {
  const int lane = threadIdx.x & 31;
  int t = 0;
  if (lane == 0) {
    t = atomicAdd(&sm.task_next, 1);
    if (t >= n_tasks && atomicAdd(&sm.task_done, 1) == (int)(blockDim.x >> 5) - 1) {
      sm.task_next = 0;
      sm.task_done = 0;
    }
  }
  t = __shfl_sync(0xffffffffu, t, 0);
  return t < n_tasks ? t : -1;
}

template <int P, int FORM, bool DENSE, bool LAST, bool DEBUG>
__device__ __noinline__ void run_tasks(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int m_in,
                                       Smem &sm, const uint8_t *gs, uint32_t *status, DebugPtrs dbg) {
  const int m_out = m_in + 4;
  const int n_items = half_prefix(m_out + 1);
  const int n_tasks = (n_items + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t mask = sm.pair_mask;
  uint32_t colmask = 0;  // bit sI: some pair (uI >= sI, sI) has a nonzero tap
#pragma unroll
  for (int sI = 0; sI < 5; ++sI)
#pragma unroll
    for (int uI = sI; uI < 5; ++uI)
      if ((mask >> (uI * (uI + 1) / 2 + sI)) & 1u) colmask |= 1u << sI;
  uint32_t tw[15];
  int taps[35];
  uint32_t a44 = 0;
  if (FORM == 1) {
#pragma unroll
    for (int k = 0; k < 15; ++k) tw[k] = sm.tapword[k];
    a44 = (uint32_t)sm.taps[34];
    if (DENSE) {
      // byte 0 of the pairs (1, 1) and (uI, 2) carries a(uI, 0, 0) (byte 3 of the pair (uI, 0)); see slice_macs_merged
      tw[2] |= tw[1] >> 24;
#pragma unroll
      for (int uI = 2; uI < 5; ++uI) tw[tri(uI) + 2] |= tw[tri(uI)] >> 24;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 35; ++k) taps[k] = sm.taps[k];
  }
  bool bad = false;
  for (int task = next_task(sm, n_tasks); task >= 0; task = next_task(sm, n_tasks)) {
    Lane L;
    const int i = task * 32 + lane;
    L.valid = i < n_items;
    decode_half(L.valid ? i : n_items - 1, L.s, L.h);
    const int s_first = __shfl_sync(0xffffffffu, L.s, 0);
#pragma unroll
    for (int sI = 0; sI < 5; ++sI) {
      const int sc = L.s - sI;
      L.first[sI] = L.valid && sc >= 0 ? sc : 1 << 30;
      L.off[sI] = colw(max(sc, 0)) + 2 * L.h;
    }
    L.out_off = colw(L.s) + 2 * L.h;
    // the last item of column s also clears the padding half-chunks after it (2 chunks_of(s) - (s/8 + 1) of them)
    L.pad = L.h == half_chunks_of(L.s) - 1 ? 2 * chunks_of(L.s) - half_chunks_of(L.s) : 0;
    int acc[6][8];
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[a][j] = 0;
    const int v0 = max(0, s_first - 4);
    if constexpr (FORM == 1 && DENSE) {
      // Slices are taken two at a time; an odd count starts one slice early, at a slice none of whose columns
      // exist for this warp (every lane has s >= s_first, so s - sI > v0 - 1), which reads only the zero guard
      // words.  Before the pair (v, v + 1), set k holds output slice v + k (k = 0 .. 4, set 4 zero) and set 5
      // holds output v - 1, complete: it is finalized while slice v's loads are in flight, and output v (set 0)
      // while slice v + 1's are.  Slice v adds into sets 0 .. 4 and slice v + 1 into sets 1 .. 5; the sets then
      // move down two places (set k <- set k + 2 mod 6), so one copy of the pair serves every slice.
      const int vb = v0 - ((m_in - v0 + 1) & 1);
      for (int v = vb; v <= m_in; v += 2) {
        uint32_t X[5][3];
        load_slice<P>(in, sm, L, v, X);
        if (v > vb) finalize<P, 5, LAST, DEBUG>(out, sm, L, v - 1, gs, acc, bad, dbg);
        slice_macs<0, FORM, DENSE>(X, tw, a44, taps, mask, colmask, acc);
        load_slice<P>(in, sm, L, v + 1, X);
        finalize<P, 0, LAST, DEBUG>(out, sm, L, v, gs, acc, bad, dbg);
        slice_macs<1, FORM, DENSE>(X, tw, a44, taps, mask, colmask, acc);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          // set 0 is zero (finalized): 0 <- 2 <- 4 <- 0 and 1 <- 3 <- 5 <- 1
          const int t1 = acc[1][j];
          acc[0][j] = acc[2][j];
          acc[2][j] = acc[4][j];
          acc[4][j] = 0;
          acc[1][j] = acc[3][j];
          acc[3][j] = acc[5][j];
          acc[5][j] = t1;
        }
      }
    } else {
      // One slice at a time (the int32 form and the sparse path hold more live registers): after slice v the
      // sets move down one place, and output v waits in set 5 to be finalized while slice v + 1's loads are in
      // flight.
      for (int v = v0; v <= m_in; ++v) {
        uint32_t X[5][3];
        load_slice<P>(in, sm, L, v, X);
        if (v > v0) finalize<P, 5, LAST, DEBUG>(out, sm, L, v - 1, gs, acc, bad, dbg);
        slice_macs<0, FORM, DENSE>(X, tw, a44, taps, mask, colmask, acc);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[5][j] = acc[0][j];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[a][j] = acc[a + 1][j];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[4][j] = 0;
      }
    }
    // output slice m_in (set 5), then m_in+1 .. m_out, which take no further input (sets 0 .. 3)
    finalize<P, 5, LAST, DEBUG>(out, sm, L, m_in, gs, acc, bad, dbg);
    finalize<P, 0, LAST, DEBUG>(out, sm, L, m_in + 1, gs, acc, bad, dbg);
    finalize<P, 1, LAST, DEBUG>(out, sm, L, m_in + 2, gs, acc, bad, dbg);
    finalize<P, 2, LAST, DEBUG>(out, sm, L, m_in + 3, gs, acc, bad, dbg);
    finalize<P, 3, LAST, DEBUG>(out, sm, L, m_in + 4, gs, acc, bad, dbg);
  }
  if (bad) atomicOr(status, kStatusInexactDivision);
}

}  // namespace sweep

// Entry point used by chain_step for the dp4a (FORM 1) and int32 (FORM 0) forms.  Quartics with at least
// sm.dense_min nonzero tap pairs (of 15) run every pair; the others skip zero pairs (and input columns none of whose
// pairs is nonzero).  The threshold is a per-prime tuning parameter (kDefaultDenseMin unless tuned).
// The caller runs it with every warp of the CTA, between two barriers, with sm.task_next and sm.task_done zero
// (init_task_queue at kernel start; run_tasks leaves them zero).
template <int P, int FORM, bool LAST, bool DEBUG>
__device__ __forceinline__ void sweep_chain_step(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                 int m_in, Smem &sm, const uint8_t *gs, uint32_t *status,
                                                 DebugPtrs dbg) {
  if (__popc(sm.pair_mask) >= sm.dense_min)
    sweep::run_tasks<P, FORM, true, LAST, DEBUG>(in, out, m_in, sm, gs, status, dbg);
  else
    sweep::run_tasks<P, FORM, false, LAST, DEBUG>(in, out, m_in, sm, gs, status, dbg);
}

}  // namespace qfs
