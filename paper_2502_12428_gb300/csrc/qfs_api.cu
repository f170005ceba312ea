// libqfs host runtime: argument checks, per-device workspaces, admission by device memory, launches.
// The C ABI is declared (and documented) in include/qfs.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/qfs.h"
#include "qfs_kernels.cuh"
#include "qfs_matmul.cuh"
#include "qfs_polypow.cuh"
#include "qfs_staged.cuh"
#include "qfs_screen.cuh"
#include "qfs_theta_matrix.cuh"

namespace qfs {

int noalloc_take_counters(uint32_t *status, unsigned long long *stats);   // qfs_noalloc.cu

namespace {

struct DeviceState {
  bool init = false;
  bool supported = false;
  int sms = 0;
  size_t total_mem = 0;
  void *ws = nullptr;          // persistent-CTA workspaces
  size_t ws_bytes = 0;
  void *ctrl = nullptr;        // [0]: work counter (u64), [8]: status (u32), [16]: stats (2 x u64), [32]: survivors (u64)
  void *staged = nullptr;      // staged-engine survivor buffers
  size_t staged_bytes = 0;
  int *which = nullptr;        // theta-matrix export: which workspace buffer holds each quartic's Delta
  int which_n = 0;
  void *mm = nullptr;          // mod-p matrix multiplication: padded A and transposed B
  size_t mm_bytes = 0;
  void *pp = nullptr;          // polynomial powering: transform, twiddles, residues, input
  size_t pp_bytes = 0;
  void *list = nullptr;        // survivors of the height-1 screen (int64 launch items)
  size_t list_bytes = 0;
};

constexpr int kMaxDevices = 64;
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;
int g_default_form = QFS_FORM_DP4A;
TileConfig g_tile[kMaxP + 1];   // per-prime chain tile shape (0 = not set: defaults)

TileConfig tile_for(int p) {
  const TileConfig t = g_tile[p];
  return t.round_chunks > 0 ? t : default_tile(p);
}
SweepConfig g_sweep[2][kMaxP + 1];   // per form (int32, dp4a) and prime: swept-chain launch shape (0: defaults)

bool sweep_form(int form) { return form == QFS_FORM_INT32 || form == QFS_FORM_DP4A; }
SweepConfig sweep_for(int form, int p) {
  SweepConfig c = sweep_form(form) ? g_sweep[form == QFS_FORM_DP4A][p] : SweepConfig{0, 0};
  if (c.dense_min == 0) c.dense_min = kDefaultDenseMin;
  return c;
}
int g_last_cuda = 0;

bool valid_p(int p) { return p == 3 || p == 5 || p == 7 || p == 11 || p == 13; }

int cuda_fail(cudaError_t e) {
  g_last_cuda = (int)e;
  return QFS_ERR_CUDA;
}

int device_state(DeviceState **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  if (dev < 0 || dev >= kMaxDevices) return QFS_ERR_DEVICE;
  DeviceState &S = g_dev[dev];
  if (!S.init) {
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    S.sms = prop.multiProcessorCount;
    S.total_mem = prop.totalGlobalMem;
    S.supported = (prop.major == 10 && prop.minor == 3);
    e = cudaMalloc(&S.ctrl, 64);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemset(S.ctrl, 0, 64);
    if (e != cudaSuccess) return cuda_fail(e);
    S.init = true;
  }
  if (!S.supported) return QFS_ERR_DEVICE;
  *out = &S;
  return QFS_OK;
}

int ensure_workspace(DeviceState &S, size_t bytes) {
  if (S.ws_bytes >= bytes) return QFS_OK;
  if (S.ws) {
    cudaError_t e = cudaFree(S.ws);
    S.ws = nullptr;
    S.ws_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  cudaError_t e = cudaMalloc(&S.ws, bytes);
  if (e != cudaSuccess) {
    S.ws = nullptr;
    (void)cudaGetLastError();
    return QFS_ERR_NO_MEMORY;
  }
  S.ws_bytes = bytes;
  return QFS_OK;
}

int ensure_list(DeviceState &S, size_t bytes) {
  if (S.list_bytes >= bytes) return QFS_OK;
  if (S.list) {
    cudaError_t e = cudaFree(S.list);
    S.list = nullptr;
    S.list_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (cudaMalloc(&S.list, bytes) != cudaSuccess) {
    S.list = nullptr;
    (void)cudaGetLastError();
    return QFS_ERR_NO_MEMORY;
  }
  S.list_bytes = bytes;
  return QFS_OK;
}

// Default workspace budget: a quarter of device memory.
size_t default_budget(const DeviceState &S) { return S.total_mem / 4; }

int ensure_staged(DeviceState &S, size_t bytes) {
  if (S.staged_bytes >= bytes) return QFS_OK;
  if (S.staged) {
    cudaError_t e = cudaFree(S.staged);
    S.staged = nullptr;
    S.staged_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (cudaMalloc(&S.staged, bytes) != cudaSuccess) {
    S.staged = nullptr;
    (void)cudaGetLastError();
    return QFS_ERR_NO_MEMORY;
  }
  S.staged_bytes = bytes;
  return QFS_OK;
}

// Staged engine: one group after another, each in chunks whose survivor buffers fit the budget.
int run_staged(DeviceState &S, const FusedParams &prm, const qfs_options_t *opts, cudaStream_t stream) {
  for (int gi = 0; gi < prm.n_groups; ++gi) {
    const FusedGroup &g = prm.g[gi];
    const int p = g.p;
    StagedPlan pl;
    pl.sms = S.sms;
    int blocks = 0;
    cudaError_t e = staged_occupancy(p, &blocks);
    if (e != cudaSuccess) return cuda_fail(e);
    int64_t grid = (int64_t)S.sms * std::max(1, opts && opts->ctas_per_sm > 0 ? opts->ctas_per_sm : blocks);
    if (opts && opts->max_ctas > 0) grid = std::min<int64_t>(grid, opts->max_ctas);
    pl.ws_words = workspace_stride_words(p);
    const size_t per_cta = 2 * pl.ws_words * sizeof(uint32_t);
    const size_t budget = opts && opts->workspace_budget ? opts->workspace_budget : default_budget(S);
    grid = std::min<int64_t>(grid, (int64_t)(budget / 2 / per_cta));
    if (grid < 1) return QFS_ERR_NO_MEMORY;
    pl.grid = (int)grid;
    int rc = ensure_workspace(S, workspace_words(grid, pl.ws_words) * sizeof(uint32_t));
    if (rc) return rc;
    const size_t per_surv = staged_survivor_bytes(p);
    int64_t chunk = std::min<int64_t>({g.n, (int64_t)8192, (int64_t)((budget / 2) / per_surv)});
    if (chunk < 1) return QFS_ERR_NO_MEMORY;
    const int ld = tet(4 * (p - 1) + 1);
    const size_t gbytes = (size_t)chunk * pl.ws_words * 4;
    const size_t need = 256 + gbytes + 2 * (size_t)chunk * ld + (size_t)chunk * 4 + (size_t)chunk + 64;
    rc = ensure_staged(S, need);
    if (rc) return rc;
    char *b = static_cast<char *>(S.staged);
    pl.counters = reinterpret_cast<unsigned *>(b);
    pl.G = reinterpret_cast<uint32_t *>(b + 256);
    pl.gA = reinterpret_cast<uint8_t *>(b + 256 + gbytes);
    pl.gB = pl.gA + (size_t)chunk * ld;
    pl.rows = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(pl.gB + (size_t)chunk * ld) + 15) & ~uintptr_t(15));
    pl.active = reinterpret_cast<uint8_t *>(pl.rows + chunk);
    pl.chunk = chunk;
    pl.ws = reinterpret_cast<uint32_t *>(S.ws);
    pl.stats = reinterpret_cast<unsigned long long *>(static_cast<char *>(S.ctrl) + 16);
    pl.status = reinterpret_cast<uint32_t *>(static_cast<char *>(S.ctrl) + 8);
    e = staged_run(pl, p, g.coeffs, g.heights, g.n, prm.max_h, stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return QFS_OK;
}

// small: an int8 tensor form launch whose groups all have p <= 5 (the small-prime kernel, three CTAs per SM)
cudaError_t form_occupancy(int form, int *blocks, size_t smem, bool small) {
  switch (form) {
    case QFS_FORM_INT32: return FormLauncher<0>::occupancy(blocks, smem, small);
    case QFS_FORM_INT8TC: return FormLauncher<2>::occupancy(blocks, smem, small);
    default: return FormLauncher<1>::occupancy(blocks, smem, small);
  }
}

cudaError_t form_fused(int form, const FusedParams &prm, int grid, size_t smem, cudaStream_t st, bool small) {
  switch (form) {
    case QFS_FORM_INT32: return FormLauncher<0>::fused(prm, grid, smem, st, small);
    case QFS_FORM_INT8TC: return FormLauncher<2>::fused(prm, grid, smem, st, small);
    default: return FormLauncher<1>::fused(prm, grid, smem, st, small);
  }
}

cudaError_t form_debug(int form, int p, const uint8_t *f, int max_h, int8_t *h_out, uint32_t *A, uint32_t *B,
                       uint32_t *status, DebugPtrs dbg, cudaStream_t st, int power_mode) {
  switch (form) {
    case QFS_FORM_INT32: return FormLauncher<0>::debug(p, f, max_h, h_out, A, B, status, dbg, st, power_mode);
    case QFS_FORM_INT8TC: return FormLauncher<2>::debug(p, f, max_h, h_out, A, B, status, dbg, st, power_mode);
    default: return FormLauncher<1>::debug(p, f, max_h, h_out, A, B, status, dbg, st, power_mode);
  }
}

bool form_supported(int form) { return form == QFS_FORM_INT32 || form == QFS_FORM_DP4A || form == QFS_FORM_INT8TC; }


struct Plan {
  int grid = 0;
  size_t smem = 0;
  size_t ws_words = 0;
};

int make_plan(DeviceState &S, int form, int max_p, int64_t n_items, const qfs_options_t *opts, Plan &plan,
              size_t smem) {
  plan.smem = smem;
  plan.ws_words = workspace_stride_words(max_p);
  int per_sm = opts && opts->ctas_per_sm > 0 ? opts->ctas_per_sm : 0;
  if (per_sm == 0) {
    int blocks = 0;
    cudaError_t e = form_occupancy(form, &blocks, plan.smem, form == QFS_FORM_INT8TC && max_p <= 5);
    if (e != cudaSuccess) return cuda_fail(e);
    per_sm = std::max(1, blocks);
    // a tuned swept-chain shape of the launch's largest prime caps the CTAs per SM
    const int tuned = sweep_for(form, max_p).ctas_per_sm;
    if (tuned > 0) per_sm = std::min(per_sm, tuned);
  }
  int64_t grid = (int64_t)S.sms * per_sm;
  if (opts && opts->max_ctas > 0) grid = std::min<int64_t>(grid, opts->max_ctas);
  const size_t per_cta = 2 * plan.ws_words * sizeof(uint32_t);
  const size_t budget = opts && opts->workspace_budget ? opts->workspace_budget : default_budget(S);
  grid = std::min<int64_t>(grid, (int64_t)(budget / per_cta));
  grid = std::min<int64_t>(grid, n_items);
  if (grid < 1) return QFS_ERR_NO_MEMORY;
  plan.grid = (int)grid;
  return ensure_workspace(S, workspace_words(grid, plan.ws_words) * sizeof(uint32_t));
}

}  // namespace

}  // namespace qfs

using namespace qfs;

extern "C" {

const char *qfs_strerror(int status) {
  switch (status) {
    case QFS_OK: return "ok";
    case QFS_ERR_INVALID_P: return "p must be one of 3, 5, 7, 11, 13";
    case QFS_ERR_INVALID_MAX_H: return "max_h must lie in [1, 10]";
    case QFS_ERR_INVALID_N: return "invalid quartic or group count";
    case QFS_ERR_NULL: return "a required pointer is NULL";
    case QFS_ERR_NO_MEMORY: return "not enough device memory for the workspace";
    case QFS_ERR_CUDA: return "a CUDA runtime call failed";
    case QFS_ERR_FORM: return "unknown or unsupported arithmetic form or engine";
    case QFS_ERR_DEVICE: return "the current device is not an sm_103 GPU";
    case QFS_ERR_CHECK: return "a device-side consistency check failed";
    default: return "unknown status";
  }
}

int qfs_last_cuda_error(void) { return g_last_cuda; }

int qfs_set_default_form(int form) {
  if (!form_supported(form)) return QFS_ERR_FORM;
  g_default_form = form;
  return QFS_OK;
}

int qfs_heights_multi_ex(int n_groups, const qfs_group_t *groups, int max_h, const qfs_options_t *opts,
                         cudaStream_t stream) {
  if (n_groups < 1 || n_groups > QFS_MAX_GROUPS) return QFS_ERR_INVALID_N;
  if (!groups) return QFS_ERR_NULL;
  if (max_h < 1 || max_h > 10) return QFS_ERR_INVALID_MAX_H;
  int64_t n_items = 0;
  int max_p = 0;
  for (int i = 0; i < n_groups; ++i) {
    const qfs_group_t &g = groups[i];
    if (!valid_p(g.p)) return QFS_ERR_INVALID_P;
    if (g.n < 0) return QFS_ERR_INVALID_N;
    if (g.n > 0 && (!g.coeffs || !g.heights_out)) return QFS_ERR_NULL;
    n_items += g.n;
    if (g.n > 0) max_p = std::max(max_p, g.p);
  }
  int form = opts && opts->form >= 0 ? opts->form : g_default_form;
  int engine = opts && opts->engine >= 0 ? opts->engine : QFS_ENGINE_FUSED;
  if (!form_supported(form) || (engine != QFS_ENGINE_FUSED && engine != QFS_ENGINE_STAGED)) return QFS_ERR_FORM;
  const int power = opts && opts->power >= 0 ? opts->power : QFS_POWER_CHAIN;
  if (power != QFS_POWER_CHAIN && power != QFS_POWER_IDENTITY && power != QFS_POWER_REDUCED) return QFS_ERR_FORM;
  if (engine == QFS_ENGINE_STAGED && (form != QFS_FORM_DP4A || power != QFS_POWER_CHAIN)) return QFS_ERR_FORM;
  if (n_items == 0) return QFS_OK;

  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;

  // Largest p first: the heaviest quartics start early, which shortens the tail of the persistent launch.
  std::vector<int> order(n_groups);
  for (int i = 0; i < n_groups; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return groups[a].p > groups[b].p; });
  FusedParams prm;
  std::memset(&prm, 0, sizeof(prm));
  int k = 0;
  int64_t begin = 0;
  for (int oi = 0; oi < n_groups; ++oi) {
    const qfs_group_t &g = groups[order[oi]];
    if (g.n == 0) continue;
    prm.g[k].p = g.p;
    prm.g[k].n = g.n;
    prm.g[k].coeffs = g.coeffs;
    prm.g[k].heights = g.heights_out;
    prm.g[k].item_begin = begin;
    prm.g[k].tile_round = tile_for(g.p).round_chunks;
    prm.g[k].tile_ring = tile_for(g.p).ring_words;
    prm.g[k].dense_min = sweep_for(form, g.p).dense_min;
    begin += g.n;
    ++k;
  }
  prm.n_groups = k;
  prm.n_items = n_items;
  prm.max_h = max_h;
  prm.sw_len = 4 * max_p * (max_p - 1) + 2;
  prm.power_mode = power;
  if (engine == QFS_ENGINE_STAGED) return run_staged(*S, prm, opts, stream);

  // shared memory: the largest iterate pair of the launch plus the largest ring any group's tile needs
  int ring_words = 0;
  for (int i = 0; i < prm.n_groups; ++i)
    ring_words = std::max(ring_words, ring_words_for(prm.g[i].p, tile_for(prm.g[i].p),
                                                     uses_ring_chain(form, prm.g[i].p), power));
  const size_t smem = ring_offset_for(tet(4 * (max_p - 1) + 1)) + 4 * (size_t)ring_words;
  Plan plan;
  rc = make_plan(*S, form, max_p, n_items, opts, plan, smem);
  if (rc) return rc;
  prm.counter = reinterpret_cast<unsigned long long *>(S->ctrl);
  prm.status = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(S->ctrl) + 8);
  prm.stats = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(S->ctrl) + 16);
  prm.ws = reinterpret_cast<uint32_t *>(S->ws);
  prm.ws_words = plan.ws_words;
  // height-1 screen first: the persistent launch then runs only the quartics that pass it
  rc = ensure_list(*S, (size_t)n_items * sizeof(int64_t));
  if (rc) return rc;
  auto *n_list = reinterpret_cast<unsigned long long *>(static_cast<char *>(S->ctrl) + 32);
  cudaError_t e = cudaMemsetAsync(n_list, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e);
  const int64_t screen_ctas = std::min<int64_t>((n_items + 7) / 8, (int64_t)S->sms * 8);
  e = screen_launch(prm, max_p, static_cast<int64_t *>(S->list), n_list, (int)screen_ctas, stream);
  if (e != cudaSuccess) return cuda_fail(e);
  prm.list = static_cast<const int64_t *>(S->list);
  prm.n_list = n_list;
  e = cudaMemsetAsync(prm.counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = form_fused(form, prm, plan.grid, plan.smem, stream, form == QFS_FORM_INT8TC && max_p <= 5);
  if (e != cudaSuccess) return cuda_fail(e);
  return QFS_OK;
}

int qfs_heights_multi(int n_groups, const qfs_group_t *groups, int max_h, cudaStream_t stream) {
  return qfs_heights_multi_ex(n_groups, groups, max_h, nullptr, stream);
}

int qfs_heights(int p, int64_t n, const uint8_t *coeffs, int max_h, int8_t *heights_out, cudaStream_t stream) {
  qfs_group_t g;
  g.p = p;
  g.n = n;
  g.coeffs = coeffs;
  g.heights_out = heights_out;
  return qfs_heights_multi_ex(1, &g, max_h, nullptr, stream);
}

int qfs_plan_prepare(int p, int64_t n_hint) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;
  Plan plan;
  int64_t n = n_hint > 0 ? n_hint : (int64_t)1 << 40;
  for (int form : {QFS_FORM_INT32, QFS_FORM_DP4A, QFS_FORM_INT8TC}) {
    rc = make_plan(*S, form, p, n, nullptr, plan, smem_bytes_for(p, tile_for(p), uses_ring_chain(form, p)));
    if (rc) return rc;
  }
  if (n_hint > 0) {
    rc = ensure_list(*S, (size_t)n_hint * sizeof(int64_t));
    if (rc) return rc;
  }
  cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? QFS_OK : cuda_fail(e);
}

int qfs_shutdown(void) {
  std::lock_guard<std::mutex> lock(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  int rc = QFS_OK;
  for (int d = 0; d < kMaxDevices; ++d) {
    DeviceState &S = g_dev[d];
    if (!S.init) continue;
    if (cudaSetDevice(d) != cudaSuccess) { rc = QFS_ERR_CUDA; continue; }
    if (S.ws && cudaFree(S.ws) != cudaSuccess) rc = QFS_ERR_CUDA;
    if (S.ctrl && cudaFree(S.ctrl) != cudaSuccess) rc = QFS_ERR_CUDA;
    if (S.staged && cudaFree(S.staged) != cudaSuccess) rc = QFS_ERR_CUDA;
    if (S.which && cudaFree(S.which) != cudaSuccess) rc = QFS_ERR_CUDA;
    if (S.mm && cudaFree(S.mm) != cudaSuccess) rc = QFS_ERR_CUDA;
    if (S.pp && cudaFree(S.pp) != cudaSuccess) rc = QFS_ERR_CUDA;
    if (S.list && cudaFree(S.list) != cudaSuccess) rc = QFS_ERR_CUDA;
    S = DeviceState();
  }
  cudaSetDevice(cur);
  return rc;
}

int qfs_tune_set(int p, int round_chunks, size_t ring_bytes) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  if (round_chunks == 0 && ring_bytes == 0) {
    g_tile[p] = TileConfig{0, 0};
    return QFS_OK;
  }
  const int ring_words = (int)(ring_bytes / 4);
  if (round_chunks < 32 || round_chunks > 4096 || ring_words < 1024) return QFS_ERR_FORM;
  const TileConfig t{round_chunks, ring_words};
  const size_t smem = smem_bytes_for(p, t);
  if (smem > 227 * 1024) return QFS_ERR_NO_MEMORY;
  g_tile[p] = t;
  return QFS_OK;
}

int qfs_tune_get(int p, int *round_chunks, size_t *ring_bytes, size_t *smem_bytes) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  const TileConfig t = tile_for(p);
  if (round_chunks) *round_chunks = t.round_chunks;
  if (ring_bytes) *ring_bytes = 4 * (size_t)t.ring_words;
  if (smem_bytes) *smem_bytes = smem_bytes_for(p, t);
  return QFS_OK;
}

int qfs_autotune(int p, int64_t n, const uint8_t *coeffs, int form, int *best_round, size_t *best_ring,
                 float *best_ms) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  if (n <= 0) return QFS_ERR_INVALID_N;
  if (!coeffs) return QFS_ERR_NULL;
  if (!form_supported(form)) return QFS_ERR_FORM;
  int8_t *out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)n);
  if (e != cudaSuccess) return cuda_fail(e);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int rounds[] = {256, 512, 768, 1024};
  const size_t rings_small[] = {48 << 10, 64 << 10, 80 << 10};
  const size_t rings_large[] = {104 << 10, 140 << 10};
  const size_t *rings = p <= 7 ? rings_small : rings_large;
  const int nrings = p <= 7 ? 3 : 2;
  const TileConfig saved = g_tile[p];
  float best = 1e30f;
  TileConfig best_t = tile_for(p);
  int rc = QFS_OK;
  qfs_options_t opt;
  memset(&opt, 0, sizeof(opt));
  opt.form = form;
  opt.engine = QFS_ENGINE_FUSED;
  opt.power = QFS_POWER_CHAIN;
  qfs_group_t g{p, n, coeffs, out};
  for (int r : rounds)
    for (int ri = 0; ri < nrings; ++ri) {
      if (qfs_tune_set(p, r, rings[ri]) != QFS_OK) continue;
      rc = qfs_heights_multi_ex(1, &g, 10, &opt, 0);  // warm-up (also grows the workspace)
      if (rc) break;
      cudaEventRecord(a, 0);
      rc = qfs_heights_multi_ex(1, &g, 10, &opt, 0);
      cudaEventRecord(b, 0);
      if (rc) break;
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) {
        best = ms;
        best_t = g_tile[p];
      }
    }
  g_tile[p] = rc ? saved : best_t;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (rc) return rc;
  if (best_round) *best_round = best_t.round_chunks;
  if (best_ring) *best_ring = 4 * (size_t)best_t.ring_words;
  if (best_ms) *best_ms = best;
  return QFS_OK;
}

int qfs_sweep_tune_set(int form, int p, int dense_min, int ctas_per_sm) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  if (!sweep_form(form) || dense_min < 0 || dense_min > 16 || ctas_per_sm < 0 || ctas_per_sm > 32)
    return QFS_ERR_FORM;
  g_sweep[form == QFS_FORM_DP4A][p] = SweepConfig{dense_min, ctas_per_sm};
  return QFS_OK;
}

int qfs_sweep_tune_get(int form, int p, int *dense_min, int *ctas_per_sm) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  if (!sweep_form(form)) return QFS_ERR_FORM;
  const SweepConfig c = sweep_for(form, p);
  if (dense_min) *dense_min = c.dense_min;
  if (ctas_per_sm) *ctas_per_sm = c.ctas_per_sm;
  return QFS_OK;
}

int qfs_sweep_autotune(int form, int p, int64_t n, const uint8_t *coeffs, int *best_dense_min, int *best_ctas,
                       float *best_ms) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  if (!sweep_form(form)) return QFS_ERR_FORM;
  if (n <= 0) return QFS_ERR_INVALID_N;
  if (!coeffs) return QFS_ERR_NULL;
  int8_t *out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)n);
  if (e != cudaSuccess) return cuda_fail(e);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int dense[] = {0, 6, 8, 10, 12, 14, 16};
  SweepConfig &slot = g_sweep[form == QFS_FORM_DP4A][p];
  const SweepConfig saved = slot;
  // the CTAs per SM that fit: the occupancy of the launch a default shape would make
  slot = SweepConfig{0, 0};
  int max_ctas = 1;
  {
    const size_t smem = ring_offset_for(tet(4 * (p - 1) + 1)) +
                        4 * (size_t)ring_words_for(p, tile_for(p), uses_ring_chain(form, p), QFS_POWER_CHAIN);
    int blocks = 0;
    if (form_occupancy(form, &blocks, smem, false) == cudaSuccess) max_ctas = std::max(1, blocks);
  }
  float best = 1e30f;
  SweepConfig best_c = saved;
  int rc = QFS_OK;
  qfs_options_t opt;
  memset(&opt, 0, sizeof(opt));
  opt.form = form;
  opt.engine = QFS_ENGINE_FUSED;
  opt.power = QFS_POWER_CHAIN;
  qfs_group_t g{p, n, coeffs, out};
  for (int dm : dense)
    for (int c = 1; c <= max_ctas && rc == QFS_OK; ++c) {
      slot = SweepConfig{dm, c};
      rc = qfs_heights_multi_ex(1, &g, 10, &opt, 0);  // warm-up
      if (rc) break;
      float ms = 1e30f;
      for (int rep = 0; rep < 2 && rc == QFS_OK; ++rep) {   // the faster of two timed launches
        cudaEventRecord(a, 0);
        rc = qfs_heights_multi_ex(1, &g, 10, &opt, 0);
        cudaEventRecord(b, 0);
        if (rc) break;
        cudaEventSynchronize(b);
        float t = 0;
        cudaEventElapsedTime(&t, a, b);
        ms = std::min(ms, t);
      }
      if (rc) break;
      if (ms < best) {
        best = ms;
        best_c = slot;
      }
    }
  // the largest count that fit is stored as 0 ("as many as fit"): a launch with other primes may fit more CTAs,
  // and a shape tuned on this prime alone must not cap it
  if (best_c.ctas_per_sm == max_ctas) best_c.ctas_per_sm = 0;
  slot = rc ? saved : best_c;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (rc) return rc;
  if (best_dense_min) *best_dense_min = best_c.dense_min;
  if (best_ctas) *best_ctas = best_c.ctas_per_sm;
  if (best_ms) *best_ms = best;
  return QFS_OK;
}

int qfs_read_stats(uint64_t *survivors, uint64_t *theta_steps) {
  if (!survivors || !theta_steps) return QFS_ERR_NULL;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned long long v[2] = {0, 0};
  e = cudaMemcpy(v, reinterpret_cast<char *>(S->ctrl) + 16, 16, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemset(reinterpret_cast<char *>(S->ctrl) + 16, 0, 16);
  if (e != cudaSuccess) return cuda_fail(e);
  unsigned long long na[2] = {0, 0};
  rc = noalloc_take_counters(nullptr, na);
  if (rc) return rc;
  *survivors = v[0] + na[0];
  *theta_steps = v[1] + na[1];
  return QFS_OK;
}

int qfs_read_status(uint32_t *status_out) {
  if (!status_out) return QFS_ERR_NULL;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e);
  uint32_t v = 0;
  e = cudaMemcpy(&v, reinterpret_cast<char *>(S->ctrl) + 8, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemset(reinterpret_cast<char *>(S->ctrl) + 8, 0, 4);
  if (e != cudaSuccess) return cuda_fail(e);
  uint32_t na = 0;
  rc = noalloc_take_counters(&na, nullptr);
  if (rc) return rc;
  *status_out = v | na;
  return QFS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------- parity hook
namespace qfs {
namespace {

__global__ void unpad_kernel(const uint32_t *__restrict__ padded, int m, const int *__restrict__ SWg,
                             int32_t *__restrict__ out) {
  const int n = tet(m + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int u, s, t;
    decode_packed(i, u, s, t);
    const uint8_t *bytes = reinterpret_cast<const uint8_t *>(padded);
    out[i] = bytes[4 * ((size_t)SWg[u] + colw(s)) + t];
  }
}

}  // namespace
}  // namespace qfs

extern "C" int qfs_debug_stages(int p, const uint8_t *coeffs, int max_h, int form, int32_t *g_out, int32_t *G_out,
                                int32_t *delta_out, int32_t *iters_out, int8_t *height_out) {
  const int power = form >> 8;
  form &= 0xFF;
  if (power != QFS_POWER_CHAIN && power != QFS_POWER_IDENTITY && power != QFS_POWER_REDUCED) return QFS_ERR_FORM;
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  if (max_h < 1 || max_h > 10) return QFS_ERR_INVALID_MAX_H;
  if (!coeffs || !height_out) return QFS_ERR_NULL;
  if (!form_supported(form)) return QFS_ERR_FORM;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;
  const int d = 4 * (p - 1), D = 4 * p * (p - 1);
  const size_t words = (size_t)padded_words(D);
  const size_t ld = (size_t)tet(d + 1);
  uint32_t *A = nullptr, *B = nullptr, *Gp = nullptr, *Dp = nullptr;
  int32_t *gtmp = nullptr, *itmp = nullptr;
  int *SWg = nullptr;
  cudaError_t e = cudaSuccess;
  auto fail = [&](cudaError_t err) {
    cudaFree(A); cudaFree(B); cudaFree(Gp); cudaFree(Dp); cudaFree(gtmp); cudaFree(itmp); cudaFree(SWg);
    return cuda_fail(err);
  };
  // the two workspace buffers, each behind a guard of zero words (one workspace stride each)
  const size_t stride = workspace_stride_words(p);
  if ((e = cudaMalloc(&A, stride * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&B, stride * 4)) != cudaSuccess) return fail(e);
  cudaMemset(A, 0, stride * 4);
  cudaMemset(B, 0, stride * 4);
  if ((e = cudaMalloc(&Gp, words * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&Dp, words * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&gtmp, ld * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&itmp, ld * 4 * 9)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&SWg, sizeof(int) * (D + 3))) != cudaSuccess) return fail(e);
  cudaMemset(Gp, 0, words * 4);
  cudaMemset(Dp, 0, words * 4);
  cudaMemset(gtmp, 0, ld * 4);
  cudaMemset(itmp, 0, ld * 4 * 9);
  std::vector<int> sw(D + 3);
  for (int u = 0; u < D + 3; ++u) sw[u] = (int)host_sw(u);
  cudaMemcpy(SWg, sw.data(), sizeof(int) * (D + 3), cudaMemcpyHostToDevice);
  DebugPtrs dbg{Gp, Dp, gtmp, itmp};
  uint32_t *status = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(S->ctrl) + 8);
  if ((e = form_debug(form, p, coeffs, max_h, height_out, A + kGuardWords, B + kGuardWords, status, dbg, 0, power)) != cudaSuccess) return fail(e);
  if (G_out) unpad_kernel<<<256, 256>>>(Gp, D, SWg, G_out);
  if (delta_out) unpad_kernel<<<256, 256>>>(Dp, D, SWg, delta_out);
  if (g_out) cudaMemcpy(g_out, gtmp, ld * 4, cudaMemcpyDeviceToDevice);
  if (iters_out && max_h > 1) cudaMemcpy(iters_out, itmp, ld * 4 * (max_h - 1), cudaMemcpyDeviceToDevice);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  cudaFree(A); cudaFree(B); cudaFree(Gp); cudaFree(Dp); cudaFree(gtmp); cudaFree(itmp); cudaFree(SWg);
  return QFS_OK;
}

extern "C" int qfs_theta_matrix(int p, int64_t n, const uint8_t *coeffs, uint8_t *M_out, cudaStream_t stream) {
  if (!valid_p(p)) return QFS_ERR_INVALID_P;
  if (n < 0) return QFS_ERR_INVALID_N;
  if (n > 0 && (!coeffs || !M_out)) return QFS_ERR_NULL;
  if (n == 0) return QFS_OK;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;
  const size_t stride = workspace_stride_words(p);
  const size_t ld = (size_t)tet(4 * (p - 1) + 1);
  // quartics per batch: one CTA each, bounded by the SM count and by the workspace budget
  int64_t batch = std::min<int64_t>(n, 2 * (int64_t)S->sms);
  batch = std::min<int64_t>(batch, (int64_t)(default_budget(*S) / (2 * stride * sizeof(uint32_t))));
  if (batch < 1) return QFS_ERR_NO_MEMORY;
  rc = ensure_workspace(*S, workspace_words(batch, stride) * sizeof(uint32_t));
  if (rc) return rc;
  if (S->which_n < batch) {
    if (S->which) cudaFree(S->which);
    S->which = nullptr;
    S->which_n = 0;
    if (cudaMalloc(&S->which, sizeof(int) * (size_t)batch) != cudaSuccess) {
      (void)cudaGetLastError();
      return QFS_ERR_NO_MEMORY;
    }
    S->which_n = (int)batch;
  }
  uint32_t *status = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(S->ctrl) + 8);
  for (int64_t i0 = 0; i0 < n; i0 += batch) {
    const int nb = (int)std::min<int64_t>(batch, n - i0);
    cudaError_t e = theta_matrix_launch(p, coeffs + 35 * i0, nb, M_out + (size_t)i0 * ld * ld,
                                        static_cast<uint32_t *>(S->ws), stride, S->which, status, stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return QFS_OK;
}

extern "C" int qfs_matmul_mod(int p, int n, int m, int k, const uint8_t *A, const uint8_t *B, uint8_t *C,
                              cudaStream_t stream) {
  if (p < 2 || p > 256) return QFS_ERR_INVALID_P;
  if (n < 0 || m < 0 || k < 0) return QFS_ERR_INVALID_N;
  if (n == 0 || m == 0) return QFS_OK;
  if (!C || (k > 0 && (!A || !B))) return QFS_ERR_NULL;
  if (k == 0) return cudaMemsetAsync(C, 0, (size_t)n * m, stream) == cudaSuccess ? QFS_OK : QFS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;
  const size_t need = matmul_scratch_bytes(n, m, k);
  if (S->mm_bytes < need) {
    if (S->mm && cudaFree(S->mm) != cudaSuccess) return cuda_fail(cudaGetLastError());
    S->mm = nullptr;
    S->mm_bytes = 0;
    if (cudaMalloc(&S->mm, need) != cudaSuccess) {
      (void)cudaGetLastError();
      return QFS_ERR_NO_MEMORY;
    }
    S->mm_bytes = need;
  }
  cudaError_t e = matmul_mod_launch(p, n, m, k, A, B, C, static_cast<uint8_t *>(S->mm), stream);
  return e == cudaSuccess ? QFS_OK : cuda_fail(e);
}

extern "C" int qfs_poly_power(int d, const uint32_t *coeffs, int n, uint32_t *out, cudaStream_t stream) {
  if (d < 1 || n < 1 || d * n > 255) return QFS_ERR_INVALID_N;
  if (!coeffs || !out) return QFS_ERR_NULL;
  const int n_in = tet(d + 1);
  uint64_t sum = 0;
  for (int i = 0; i < n_in; ++i) sum += coeffs[i];
  // every output coefficient is at most (sum of the coefficients)^n, checked exactly against the output width and
  // the primes' product
  const int nprimes = polypow_primes(sum, n);
  if (nprimes == 0) return QFS_ERR_INVALID_N;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceState *S = nullptr;
  int rc = device_state(&S);
  if (rc) return rc;
  const size_t need = polypow_scratch_words(d, n, nprimes) * sizeof(uint32_t);
  if (S->pp_bytes < need) {
    if (S->pp && cudaFree(S->pp) != cudaSuccess) return cuda_fail(cudaGetLastError());
    S->pp = nullptr;
    S->pp_bytes = 0;
    if (cudaMalloc(&S->pp, need) != cudaSuccess) {
      (void)cudaGetLastError();
      return QFS_ERR_NO_MEMORY;
    }
    S->pp_bytes = need;
  }
  uint32_t *scratch = static_cast<uint32_t *>(S->pp);
  uint32_t *cdev = scratch + (need / sizeof(uint32_t) - n_in - 16);   // the input sits at the end of the scratch
  cudaError_t e = cudaMemcpyAsync(cdev, coeffs, sizeof(uint32_t) * n_in, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = polypow_launch(d, n, nprimes, cdev, out, scratch, stream);
  return e == cudaSuccess ? QFS_OK : cuda_fail(e);
}

extern "C" int qfs_poly_power_info(int d, const uint32_t *coeffs, int n, int *nprimes, uint64_t *transform_len,
                                   uint64_t *hbm_bytes) {
  if (d < 1 || n < 1 || d * n > 255) return QFS_ERR_INVALID_N;
  if (!coeffs) return QFS_ERR_NULL;
  uint64_t sum = 0;
  for (int i = 0; i < tet(d + 1); ++i) sum += coeffs[i];
  const int np = polypow_primes(sum, n);
  if (np == 0) return QFS_ERR_INVALID_N;
  if (nprimes) *nprimes = np;
  polypow_plan(d, n, np, transform_len, hbm_bytes);
  return QFS_OK;
}
