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
#include <cstdint>
#include "qfs_layout.cuh"

namespace qfs {

constexpr int kThreads = 256;

// Status bits (atomicOr into the device status word).
constexpr uint32_t kStatusInexactDivision = 1u;
constexpr uint32_t kStatusTheta = 2u;

struct DebugPtrs {
  uint32_t *G;        // padded, degree D: raw G (mod p^2) before the Delta_1 epilogue
  uint32_t *delta;    // padded, degree D: Delta (mod p)
  int32_t *g;         // packed, ld values
  int32_t *iters;     // packed, (max_h-1) x ld
};

struct Smem {
  int SW[kSWLen];
  int taps[35];           // coefficients of f, packed order (index tet(uI) + tri(sI) + tI)
  uint32_t tapword[15];   // dp4a tap words per (uI, sI) pair: byte k = a(uI, sI, 3-k)
  uint32_t pair_mask;     // bit tri(uI)+sI set iff that pair has a nonzero tap
  int powp[kMaxP];        // c^p mod p^2
  int64_t item;
  int flag;
  // followed in dynamic shared memory by two byte arrays of ld entries: g (current iterate) and g_next
};

__host__ __device__ constexpr size_t smem_bytes_for(int p) {
  return sizeof(Smem) + 2 * (size_t)tet(4 * (p - 1) + 1) + 16;
}

// ------------------------------------------------------------------------------------------------ chain step
// out := in * f (mod p^2), in of degree m_in, out of degree m_in + 4.  When LAST, the Delta_1 epilogue turns
// G into Delta and writes residues mod p.
template <int P, int FORM, bool LAST, bool DEBUG>
__device__ __forceinline__ void chain_step(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int m_in,
                                           const Smem &sm, const uint8_t *gs, uint32_t *status, DebugPtrs dbg);

namespace detail {

template <int UI, int SI>
struct Pair {
  static constexpr int index = UI * (UI + 1) / 2 + SI;
  static constexpr int tap0 = tet(UI) + tri(SI);  // tap index of tI = 0
};

// Loads the two input words that cover t' in [4w-4, 4w+3] of input column (u-UI, s-SI); false if the column is
// outside the degree-m_in cone.
template <int UI, int SI>
__device__ __forceinline__ bool load_pair(const uint32_t *__restrict__ in, const int *SW, int m_in, int u, int s,
                                          int w, uint32_t &lo, uint32_t &hi) {
  const int u2 = u - UI, s2 = s - SI;
  if (s2 < 0 || s2 > u2 || u2 > m_in) return false;
  const int base = SW[u2] + colw(s2);
  const int nw = (s2 >> 2) + 1;
  hi = (w < nw) ? __ldg(in + base + w) : 0u;
  lo = (w >= 1) ? __ldg(in + base + w - 1) : 0u;
  return true;
}

template <int UI, int SI>
__device__ __forceinline__ void pair_int32(const uint32_t *__restrict__ in, const int *SW, int m_in, int u, int s,
                                           int w, const int *taps, uint32_t mask, int (&acc)[4]) {
  constexpr int PI = Pair<UI, SI>::index;
  if (!((mask >> PI) & 1u)) return;
  uint32_t lo, hi;
  if (!load_pair<UI, SI>(in, SW, m_in, u, s, w, lo, hi)) return;
  int v[8];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = (int)((lo >> (8 * j)) & 0xFFu);
    v[4 + j] = (int)((hi >> (8 * j)) & 0xFFu);
  }
#pragma unroll
  for (int tI = 0; tI <= SI; ++tI) {
    const int a = taps[Pair<UI, SI>::tap0 + tI];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] += a * v[4 + r - tI];
  }
}

template <int UI, int SI>
__device__ __forceinline__ void pair_dp4a(const uint32_t *__restrict__ in, const int *SW, int m_in, int u, int s,
                                          int w, const Smem &sm, uint32_t mask, int (&acc)[4]) {
  constexpr int PI = Pair<UI, SI>::index;
  if (!((mask >> PI) & 1u)) return;
  uint32_t lo, hi;
  if (!load_pair<UI, SI>(in, SW, m_in, u, s, w, lo, hi)) return;
  if (SI == 0) {
    // single tap at t' = t: byte r of hi
    const uint32_t a = (uint32_t)sm.taps[Pair<UI, SI>::tap0];
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[r] = (int)__dp4a(hi, a << (8 * r), (unsigned)acc[r]);
  } else {
    const uint32_t tw = sm.tapword[PI];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      // window byte k = in(t - 3 + k) for t = 4w + r: bytes r+1 .. r+4 of the 8-byte (lo, hi) concatenation
      const uint32_t win = __byte_perm(lo, hi, (unsigned)((r + 1) | ((r + 2) << 4) | ((r + 3) << 8) | ((r + 4) << 12)));
      acc[r] = (int)__dp4a(win, tw, (unsigned)acc[r]);
    }
    if (SI == 4) {
      // the tap at tI = 4 reads in(t - 4) = byte r of lo
      const uint32_t a4 = (uint32_t)sm.taps[Pair<UI, SI>::tap0 + 4];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] = (int)__dp4a(lo, a4 << (8 * r), (unsigned)acc[r]);
    }
  }
}

#define QFS_FOR_EACH_PAIR(X) \
  X(0, 0) X(1, 0) X(1, 1) X(2, 0) X(2, 1) X(2, 2) X(3, 0) X(3, 1) X(3, 2) X(3, 3) X(4, 0) X(4, 1) X(4, 2) X(4, 3) X(4, 4)

}  // namespace detail

template <int P, int FORM, bool LAST, bool DEBUG>
__device__ __forceinline__ void chain_step(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, int m_in,
                                           const Smem &sm, const uint8_t *gs, uint32_t *status, DebugPtrs dbg) {
  using Pr = Prime<P>;
  const int m_out = m_in + 4;
  const int total = sm.SW[m_out + 1];
  const uint32_t mask = sm.pair_mask;
  int taps[35];
  if (FORM == 0) {
#pragma unroll
    for (int i = 0; i < 35; ++i) taps[i] = sm.taps[i];
  }
  bool bad = false;
  for (int k = threadIdx.x; k < total; k += blockDim.x) {
    int u, s, w;
    decode_word(k, m_out, sm.SW, u, s, w);
    int acc[4] = {0, 0, 0, 0};
    if (FORM == 0) {
#define QFS_PAIR_INT32(UI, SI) detail::pair_int32<UI, SI>(in, sm.SW, m_in, u, s, w, taps, mask, acc);
      QFS_FOR_EACH_PAIR(QFS_PAIR_INT32)
#undef QFS_PAIR_INT32
    } else {
#define QFS_PAIR_DP4A(UI, SI) detail::pair_dp4a<UI, SI>(in, sm.SW, m_in, u, s, w, sm, mask, acc);
      QFS_FOR_EACH_PAIR(QFS_PAIR_DP4A)
#undef QFS_PAIR_DP4A
    }
    uint32_t word = 0, gword = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int t = 4 * w + r;
      int G = acc[r] % Pr::p2;  // acc >= 0
      uint32_t byte = 0;
      if (t <= s) {
        if (LAST) {
          if (DEBUG) gword |= (uint32_t)G << (8 * r);
          if ((u % P) == 0 && (s % P) == 0 && (t % P) == 0) {
            const int J = tet(u / P) + tri(s / P) + t / P;
            G = G - sm.powp[gs[J]];
            if (G < 0) G += Pr::p2;
          }
          if (G % P) bad = true;
          byte = (uint32_t)(G / P);
        } else {
          byte = (uint32_t)G;
        }
      }
      word |= byte << (8 * r);
    }
    out[k] = word;
    if (DEBUG && LAST) dbg.G[k] = gword;
  }
  if (bad) atomicOr(status, kStatusInexactDivision);
}

// ------------------------------------------------------------------------------------------------ theta
// g_next[r] = sum over c in B_d of Delta[p r + (p-1)1 - c] * g[c] mod p, for every r in B_d.  In (u,s,t)
// coordinates the Delta index is (p u_r + 3(p-1) - u_c, p s_r + 2(p-1) - s_c, p t_r + (p-1) - t_c) and a term is
// present iff that index lies in the degree-D cone.  Returns true iff some output is nonzero.
template <int P>
__device__ __forceinline__ bool theta_step(const uint8_t *__restrict__ delta, const Smem &sm,
                                           const uint8_t *__restrict__ g, uint8_t *__restrict__ gn) {
  using Pr = Prime<P>;
  bool any = false;
  for (int r = threadIdx.x; r < Pr::ld; r += blockDim.x) {
    int ur, sr, tr;
    decode_packed(r, ur, sr, tr);
    const int eu0 = P * ur + 3 * (P - 1), es0 = P * sr + 2 * (P - 1), et0 = P * tr + (P - 1);
    int acc = 0;
    for (int uc = 0; uc <= Pr::d; ++uc) {
      const int eu = eu0 - uc;
      if (eu < 0) break;
      if (eu > Pr::D) continue;
      for (int sc = 0; sc <= uc; ++sc) {
        const int es = es0 - sc;
        if (es < 0) break;
        if (es > eu) continue;
        const int tlo = max(0, et0 - es), thi = min(sc, et0);
        if (tlo > thi) continue;
        const uint8_t *dcol = delta + 4 * (sm.SW[eu] + colw(es)) + et0;  // Delta(eu, es, et0 - tc) = dcol[-tc]
        const uint8_t *gcol = g + tet(uc) + tri(sc);
        for (int tc = tlo; tc <= thi; ++tc) acc += (int)__ldg(dcol - tc) * (int)gcol[tc];
      }
    }
    const int v = acc % P;
    gn[r] = (uint8_t)v;
    any |= (v != 0);
  }
  return any;
}

// ------------------------------------------------------------------------------------------------ one quartic
// Runs A1-A7 for one quartic with the CTA's two workspace buffers; returns the height code (thread 0 writes it).
template <int P, int FORM, bool DEBUG>
__device__ int process_quartic(const uint8_t *__restrict__ f35, int max_h, Smem &sm, uint8_t *gs, uint8_t *gn,
                               uint32_t *bufA, uint32_t *bufB, uint32_t *status, DebugPtrs dbg, int &theta_steps) {
  using Pr = Prime<P>;
  const int tid = threadIdx.x;
  theta_steps = 0;
  // A1: coefficients, validation, tap tables
  int bad = 0;
  if (tid < 35) {
    const int a = f35[tid];
    bad = a >= P;
    sm.taps[tid] = a;
  }
  if (__syncthreads_or(bad)) return -1;
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
  // f into bufA (padded, degree 4)
  for (int k = tid; k < sm.SW[5]; k += blockDim.x) {
    int u, s, w;
    decode_word(k, 4, sm.SW, u, s, w);
    uint32_t word = 0;
    for (int r = 0; r < 4; ++r) {
      const int t = 4 * w + r;
      if (t <= s) word |= (uint32_t)sm.taps[tet(u) + tri(s) + t] << (8 * r);
    }
    bufA[k] = word;
  }
  __syncthreads();
  // A2: f~^(k+1) = f~^k * f~ for k = 1 .. p-2
  uint32_t *cur = bufA, *nxt = bufB;
  int m = 4;
  for (int k = 1; k <= P - 2; ++k) {
    chain_step<P, FORM, false, DEBUG>(cur, nxt, m, sm, gs, status, dbg);
    __syncthreads();
    uint32_t *t = cur; cur = nxt; nxt = t;
    m += 4;
  }
  // A3: g = f^(p-1) mod p into shared memory (packed); witness test
  for (int k = tid; k < sm.SW[Pr::d + 1]; k += blockDim.x) {
    int u, s, w;
    decode_word(k, Pr::d, sm.SW, u, s, w);
    const uint32_t word = cur[k];
    for (int r = 0; r < 4; ++r) {
      const int t = 4 * w + r;
      if (t <= s) gs[tet(u) + tri(s) + t] = (uint8_t)(((word >> (8 * r)) & 0xFFu) % P);
    }
  }
  __syncthreads();
  if (DEBUG)
    for (int i = tid; i < Pr::ld; i += blockDim.x) dbg.g[i] = gs[i];
  if (gs[Pr::witness] != 0) return 1;
  // A4 + A5: chain to f~^(p(p-1)); the last product carries the Delta_1 epilogue
  for (int k = P - 1; k <= P * (P - 1) - 2; ++k) {
    chain_step<P, FORM, false, DEBUG>(cur, nxt, m, sm, gs, status, dbg);
    __syncthreads();
    uint32_t *t = cur; cur = nxt; nxt = t;
    m += 4;
  }
  chain_step<P, FORM, true, DEBUG>(cur, nxt, m, sm, gs, status, dbg);
  __syncthreads();
  if (DEBUG)
    for (int k = tid; k < sm.SW[Pr::D + 1]; k += blockDim.x) dbg.delta[k] = nxt[k];
  const uint8_t *delta = reinterpret_cast<const uint8_t *>(nxt);
  // A6 + A7
  uint8_t *g = gs, *g2 = gn;
  for (int h = 2; h <= max_h; ++h) {
    const bool any = theta_step<P>(delta, sm, g, g2);
    const int nonzero = __syncthreads_or(any ? 1 : 0);
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
  uint32_t *ws;                       // 2 buffers of ws_words per CTA
  size_t ws_words;
};

template <int FORM>
__device__ __forceinline__ void fused_body(const FusedParams &prm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  uint8_t *gs = smem_raw + sizeof(Smem);
  // the second iterate buffer follows the largest ld in this launch
  int max_ld = 0;
  for (int i = 0; i < prm.n_groups; ++i) max_ld = max(max_ld, tet(4 * (prm.g[i].p - 1) + 1));
  uint8_t *gn = gs + max_ld;
  build_sw(sm.SW, prm.sw_len);
  uint32_t *bufA = prm.ws + (size_t)blockIdx.x * 2 * prm.ws_words;
  uint32_t *bufB = bufA + prm.ws_words;
  DebugPtrs dbg{nullptr, nullptr, nullptr, nullptr};
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) sm.item = (int64_t)atomicAdd(prm.counter, 1ull);
    __syncthreads();
    const int64_t item = sm.item;
    if (item >= prm.n_items) break;
    int gi = 0;
    while (gi + 1 < prm.n_groups && item >= prm.g[gi + 1].item_begin) ++gi;
    const FusedGroup &G = prm.g[gi];
    const int64_t row = item - G.item_begin;
    const uint8_t *f = G.coeffs + 35 * row;
    int h, steps;
    switch (G.p) {
      case 3: h = process_quartic<3, FORM, false>(f, prm.max_h, sm, gs, gn, bufA, bufB, prm.status, dbg, steps); break;
      case 5: h = process_quartic<5, FORM, false>(f, prm.max_h, sm, gs, gn, bufA, bufB, prm.status, dbg, steps); break;
      case 7: h = process_quartic<7, FORM, false>(f, prm.max_h, sm, gs, gn, bufA, bufB, prm.status, dbg, steps); break;
      case 11: h = process_quartic<11, FORM, false>(f, prm.max_h, sm, gs, gn, bufA, bufB, prm.status, dbg, steps); break;
      default: h = process_quartic<13, FORM, false>(f, prm.max_h, sm, gs, gn, bufA, bufB, prm.status, dbg, steps); break;
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
