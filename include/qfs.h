/*
 * libqfs -- quasi-F-split (Artin-Mazur) heights of quartic K3 surfaces over F_p on one NVIDIA GB300 (sm_103a).
 *
 * The operation (paper: "K3 surfaces of any Artin-Mazur height over F5 and F7 via quasi-F-split singularities
 * and GPU acceleration", arXiv 2502.12428):
 *   for each quartic f in F_p[x1,x2,x3,x4]
 *     g <- f^(p-1);  if the coefficient of (x1 x2 x3 x4)^(p-1) in g is nonzero, the height is 1
 *                                                   (Fedder's criterion, Sec. 2.2; matrix-based algorithm, Sec. 3.4)
 *     Delta <- Delta_1(f^(p-1)) = (lift(g)^p - sum over terms t of lift(g) of t^p) / p  mod p
 *                                                   (Proposition and Algorithm 1 of Sec. 3.1)
 *     for h = 2 .. max_h:  g <- u(Delta * g)  (Algorithm 2, the splitting u, Sec. 3.2);  test as above
 *                                                   (Algorithm 3 / matrix-based algorithm of Sec. 3.3-3.4)
 *   K3 heights are at most 10 or infinite (Sec. 3.3), so max_h = 10 decides every nonsingular quartic.
 *
 * Conventions shared by every entry point:
 *   - A quartic is 35 uint8 coefficients in descending lexicographic order of (e1, e2, e3, e4):
 *     x1^4, x1^3 x2, x1^3 x3, x1^3 x4, x1^2 x2^2, ..., x4^4 (the order the paper prints, Figures 4-7).
 *     `coeffs` is row-major n x 35.  Values must lie in [0, p).
 *   - Output codes (int8, one per quartic): 1..max_h = the height; 0 = infinity / no witness up to max_h;
 *     -1 = the row has a coefficient >= p (nothing else is computed for it).
 *   - Pointers named "device" are CUDA device memory owned by the caller; the library never frees them.
 *   - Work is stream-ordered on `stream` (a cudaStream_t; NULL = the legacy default stream).  Calls return after
 *     enqueue; results are valid once the stream reaches that point.  No call synchronises the host unless stated.
 *   - Errors that can be seen on the host are returned synchronously and nothing is enqueued.  n = 0 is a no-op.
 *   - The library owns its workspaces (one set per device, grown on demand, freed by qfs_shutdown).  Growing a
 *     workspace calls cudaMalloc; call qfs_plan_prepare for the largest p and batch first when capturing the
 *     calls into a CUDA graph.
 *   - Calls are not thread-safe with respect to each other on the same device.
 */
#ifndef QFS_H
#define QFS_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes returned by every entry point. */
enum {
  QFS_OK = 0,
  QFS_ERR_INVALID_P = 1,      /* p is not one of 3, 5, 7, 11, 13 */
  QFS_ERR_INVALID_MAX_H = 2,  /* max_h outside [1, 10] */
  QFS_ERR_INVALID_N = 3,      /* n < 0, or a group count outside [1, QFS_MAX_GROUPS] */
  QFS_ERR_NULL = 4,           /* a required pointer is NULL */
  QFS_ERR_NO_MEMORY = 5,      /* the workspace for even one quartic in flight does not fit */
  QFS_ERR_CUDA = 6,           /* a CUDA runtime call failed; qfs_last_cuda_error() has the code */
  QFS_ERR_FORM = 7,           /* unknown arithmetic form or engine */
  QFS_ERR_DEVICE = 8,         /* the current device is not sm_103 */
  QFS_ERR_CHECK = 9           /* a device-side consistency check failed (see qfs_read_status) */
};

/* Arithmetic forms of the contractions (all exact; they produce identical results). */
enum {
  QFS_FORM_INT32 = 0,   /* int32 multiply-add on CUDA cores (IMAD) */
  QFS_FORM_DP4A = 1,    /* 4-way int8 dot products with int32 accumulation on CUDA cores (IDP4A) */
  QFS_FORM_INT8TC = 2   /* int8 tensor cores (mma.sync m16n8k32 s8 -> s32), int32 accumulation */
};

/* Engines: how the per-quartic stages are scheduled. */
enum {
  QFS_ENGINE_FUSED = 0,   /* one persistent launch, work stealing over quartics, every stage fused per quartic */
  QFS_ENGINE_STAGED = 1   /* one kernel per stage (Fedder test, power, Delta_1, theta, test) over chunks of
                             quartics; dp4a form only; the groups of a multi call run one after another */
};

/* How A4 + A5 form Delta_1(f^(p-1)) (both produce the same array, bit for bit). */
enum {
  QFS_POWER_CHAIN = 0,     /* Algorithm 1 literally: lift(g)^p mod p^2 as the chain f~^(p(p-1)), then (G - S) / p */
  QFS_POWER_IDENTITY = 1,  /* the exact rewriting Delta_1(f^(p-1)) = E(x^p) - f^(p-2)(x^p) Delta_1(f) mod p, from
                              f~^p = A + p Delta_1(f) (Proposition of Sec. 3.1) and the binomial theorem mod p^2 */
  QFS_POWER_REDUCED = 2    /* never forms Delta_1(f^(p-1)): the loop applies theta only to iterates F with a zero
                              witness coefficient, and for those theta(F) = -f^(p-2) u(F Delta_1(f)) mod p (u moves
                              x^(pJ) out as x^J, Algorithm 2).  Same heights; about 30x less work per theta step */
};

#define QFS_MAX_GROUPS 8

/* One batch of quartics over one prime (all pointers device memory owned by the caller). */
typedef struct {
  int p;                   /* 3, 5, 7, 11 or 13 */
  int64_t n;               /* number of quartics, >= 0 */
  const uint8_t *coeffs;   /* device, n x 35 uint8, row-major, descending lex, values in [0, p) */
  int8_t *heights_out;     /* device, n int8 */
} qfs_group_t;

/* Per-call options.  Zero-initialised fields mean "library default". */
typedef struct {
  int form;                  /* QFS_FORM_*; -1 = process default (qfs_set_default_form) */
  int engine;                /* QFS_ENGINE_*; -1 = QFS_ENGINE_FUSED */
  int ctas_per_sm;           /* fused engine: resident CTAs per SM, 0 = auto */
  int max_ctas;              /* cap on persistent CTAs (admission), 0 = no cap beyond memory */
  size_t workspace_budget;   /* bytes of device workspace the call may use, 0 = library default */
  int power;                 /* QFS_POWER_*; -1 = QFS_POWER_CHAIN (fused engine only for the identity) */
} qfs_options_t;

/* Heights of n quartics over F_p.  coeffs: device, n x 35 uint8.  heights_out: device, n int8.
   Returns QFS_OK or an error status (nothing enqueued on error).
   The fused engine enqueues two kernels: a height-1 screen (Fedder's criterion, one warp per quartic), which writes
   1 or -1 for the rows it settles and lists the others, then the persistent launch over the listed rows. */
int qfs_heights(int p, int64_t n, const uint8_t *coeffs, int max_h, int8_t *heights_out, cudaStream_t stream);

/* Several batches, possibly over different primes, in one persistent launch (groups is a host array of
   n_groups <= QFS_MAX_GROUPS descriptors).  Work is ordered largest p first so the heaviest quartics start
   early.  Same return convention as qfs_heights. */
int qfs_heights_multi(int n_groups, const qfs_group_t *groups, int max_h, cudaStream_t stream);

/* qfs_heights_multi with explicit options (opts may be NULL). */
int qfs_heights_multi_ex(int n_groups, const qfs_group_t *groups, int max_h, const qfs_options_t *opts,
                         cudaStream_t stream);

/* Sets the process-wide default form used when opts->form is -1 (initially QFS_FORM_DP4A). */
int qfs_set_default_form(int form);

/* Prepares the current device for prime p: checks the device, tunes launch shapes and allocates the workspace
   a fused launch over up to n_hint quartics needs (n_hint <= 0: a full-device launch; the survivor list of the
   height-1 screen is sized only when n_hint > 0).  Synchronous; it may call cudaMalloc.  Optional: the first
   qfs_heights call does the same lazily. */
int qfs_plan_prepare(int p, int64_t n_hint);

/* Chain tile shape per prime (process-wide; the autotuner below picks it on the device at hand).
   round_chunks: target (column, 16-byte chunk) work items per round of the shared-memory sweep; ring_bytes: the
   shared memory the slice ring may use (it bounds how many slices a round covers, and with it the occupancy).
   qfs_tune_set(p, 0, 0) restores the built-in default.  Returns QFS_ERR_FORM for values outside
   [32, 4096] x [4 KB, ...) and QFS_ERR_NO_MEMORY if the CTA would need more than 227 KB of shared memory. */
int qfs_tune_set(int p, int round_chunks, size_t ring_bytes);
int qfs_tune_get(int p, int *round_chunks, size_t *ring_bytes, size_t *smem_bytes);

/* Times the fused engine on n quartics (device, n x 35) for every candidate tile shape of prime p, keeps the
   fastest with qfs_tune_set and reports it.  Synchronous; allocates a scratch output of n bytes. */
int qfs_autotune(int p, int64_t n, const uint8_t *coeffs, int form, int *best_round, size_t *best_ring,
                 float *best_ms);

/* Launch shape of the swept chain (the dp4a and int32 forms' chain products, Algorithm 1's powering) per prime and
   form, process-wide.  dense_min: the number of tap pairs (u_I, s_I) of f (15 in all) with a nonzero tap from which
   a quartic's products run every pair, two input slices per loop pass; quartics with fewer skip the zero pairs one
   slice at a time (16: every quartic skips).  ctas_per_sm: CTAs per SM of the fused launch whose largest prime is
   p (0: as many as fit; a launch's own qfs_options_t.ctas_per_sm overrides it).  Heights never depend on either.
   qfs_sweep_tune_set(form, p, 0, 0) restores the defaults (dense_min 12, as many CTAs as fit).  Returns QFS_OK,
   QFS_ERR_INVALID_P, or QFS_ERR_FORM (form not dp4a or int32, dense_min outside 0 .. 16 or ctas_per_sm outside
   0 .. 32).  No counterpart in the paper: it is the autotuned shape of the powering step's products. */
int qfs_sweep_tune_set(int form, int p, int dense_min, int ctas_per_sm);
int qfs_sweep_tune_get(int form, int p, int *dense_min, int *ctas_per_sm);

/* Times the fused engine (chain power mode, the given form) on n quartics (device, n x 35) for every candidate
   swept-chain shape of prime p: dense_min in {0, 6, 8, 10, 12, 14, 16} times ctas_per_sm in {1, .., as many as
   fit}; keeps the fastest (the faster of two timed launches each) with qfs_sweep_tune_set and reports it (best_ms:
   its launch time; best_ctas 0 when the fastest was the most CTAs that fit, so that the setting never caps a launch
   with other primes, which may fit more).  Synchronous;
   allocates a scratch output of n bytes.  Returns QFS_ERR_FORM for a form other than dp4a or int32. */
int qfs_sweep_autotune(int form, int p, int64_t n, const uint8_t *coeffs, int *best_dense_min, int *best_ctas,
                       float *best_ms);

/* Frees every workspace of every device this process used.  Synchronous. */
int qfs_shutdown(void);

/* Copies the device status word of the current device's last launches into *status_out (0 = no check failed;
   bit 0 = an exact division by p in Delta_1 found a remainder; bit 1 = the theta test saw an out-of-range value),
   then clears it.  The word covers every launch since the last call, qfs_heights_noalloc's included (that entry
   point keeps its own word in its fixed array; this call ORs it in and clears it too).  Synchronises the current
   device. */
int qfs_read_status(uint32_t *status_out);

/* Work counters of the current device's launches since the last call: quartics that passed the height-1 test
   (so ran the full power chain, Delta_1 and at least one theta step unless max_h = 1) and theta steps run in
   total, qfs_heights_noalloc's launches included.  Clears them.  Synchronises the current device.  Used to turn
   timings into algorithmic work rates. */
int qfs_read_stats(uint64_t *survivors, uint64_t *theta_steps);

/* Measured multiply-add rates of the current device's integer paths, the denominators of the height kernels'
   rooflines (the paper has no counterpart; this is a measurement aid).  macs_per_s: host, 3 doubles, filled with
   the multiply-accumulates per second of independent IMAD chains ([0]: the int32 form's instruction), IDP4A chains
   ([1]: 4 MACs each, the dp4a form's) and mma.sync m16n8k32 s8 tiles ([2]: the int8 tensor form's), each the best
   of three timed launches of 8 CTAs per SM.  sms / max_clock_khz (host, may be NULL): the device's SM count and
   its maximum SM clock, so that rates turn into per-SM-per-clock figures.  Allocates and frees a small device
   buffer; synchronous; takes about a tenth of a second.  Returns QFS_OK, QFS_ERR_NULL, QFS_ERR_NO_MEMORY or
   QFS_ERR_CUDA. */
int qfs_int_peaks(double *macs_per_s, int *sms, int *max_clock_khz);

/* Human-readable text for a status code (static storage). */
const char *qfs_strerror(int status);

/* The cudaError_t of the last failed CUDA call inside the library (0 if none). */
int qfs_last_cuda_error(void);

/* qfs_heights without any allocation, for callers that cannot allocate device memory when they call: code
   running inside a stream capture in global mode (cudaMalloc there invalidates the capture), code whose device
   memory is owned by another allocator, and code that must not stall the device (cudaFree synchronises it).
   The paper has no counterpart; this is a deployment aid.
   Same arguments, codes and stream semantics as qfs_heights (dp4a form).  All scratch lives in one fixed 64 MiB
   array of device memory that the library declares statically: every GPU that loads libqfs holds it until the
   process exits.  The first call on a device looks up that array's device address (cudaGetSymbolAddress), so
   make the first call on each device before any stream capture.  The array keeps the previous call's contents;
   each call clears the part that must start at zero (its work-queue counter).  The device check word and the
   work counters of these calls accumulate in the array until qfs_read_status and qfs_read_stats read and clear
   them, together with those of the other entry points.  Calls whose kernels overlap on the GPU (for example
   calls on two different streams of one device) share the array and race: keep them ordered on one stream.
   Returns QFS_ERR_NO_MEMORY when one persistent CTA's workspace does not fit in 64 MiB (p = 13); otherwise it
   runs as many CTAs as fit (p = 7: 39, p = 11: 2), so large p runs slower here than through qfs_heights.  It has
   no height-1 screen (the survivor list would need n x 8 bytes): every quartic enters the persistent launch,
   which takes the same decisions. */
int qfs_heights_noalloc(int p, int64_t n, const uint8_t *coeffs, int max_h, int8_t *heights_out,
                        cudaStream_t stream);

/* Kernel-level parity hook (tests only need it; it runs the same device code as qfs_heights on ONE quartic).
   coeffs: device, 35 uint8.  All outputs are device int32 arrays in descending-lex order; any may be NULL.
     g_out     C(4p-1,3) values: f^(p-1) mod p
     G_out     C(4p(p-1)+3,3) values: f~^(p(p-1)) mod p^2 (equal to lift(g)^p mod p^2), only if height != 1
     delta_out C(4p(p-1)+3,3) values: Delta_1(f^(p-1)) mod p, only if height != 1
     iters_out (max_h-1) x C(4p-1,3): row h-2 = the iterate g_h, for the rows computed
   height_out: device, 1 int8 (the same code qfs_heights writes).  form = QFS_FORM_* | (QFS_POWER_* << 8); with the
   identity power mode G_out is left untouched (that route never forms G); with the reduced mode G_out and
   delta_out are left untouched.  Synchronous. */
int qfs_debug_stages(int p, const uint8_t *coeffs, int max_h, int form, int32_t *g_out, int32_t *G_out,
                     int32_t *delta_out, int32_t *iters_out, int8_t *height_out);

/* The theta matrix of each of n quartics (the matrix form of the step of Algorithm 3, Sec. 3.4):
     M[r][c] = Delta_1(f^(p-1))[p r + (p-1,p-1,p-1,p-1) - c]  (mod p),  r, c in B_d (d = 4(p-1), descending lex),
   and 0 where that exponent falls outside the degree-4p(p-1) monomials, so that theta(g) = M g (mod p) for every
   form g of degree d.  The height pipeline never forms M; this exports it.  Unlike qfs_heights, the Fedder test
   does not stop the computation: M is produced for every quartic.
   coeffs: device, n x 35 uint8, row-major, descending lex, values in [0, p).  M_out: device, n x ld x ld uint8
   (ld = C(4p-1, 3): 2925 at p = 7, 12341 at p = 11), row-major; caller-owned.  A row of coeffs with a value >= p
   gives an all-zero M.  Stream-ordered; may grow the library workspace (cudaMalloc) on the first call for p.
   Returns QFS_OK or an error status (QFS_ERR_INVALID_P, QFS_ERR_INVALID_N, QFS_ERR_NULL, QFS_ERR_NO_MEMORY,
   QFS_ERR_CUDA). */
int qfs_theta_matrix(int p, int64_t n, const uint8_t *coeffs, uint8_t *M_out, cudaStream_t stream);

/* Matrix multiplication mod p (the paper's Sec. 5 workload, square matrices mod 11): C = A B mod p.
   A: device, n x k uint8, row-major; B: device, k x m uint8, row-major; C: device, n x m uint8, row-major; values
   in [0, p), 2 <= p <= 256 (p need not be prime); all caller-owned.  Exact: products accumulate in int32 on the
   int8 tensor cores and are reduced mod p.  Stream-ordered; may grow a library scratch buffer ((n + m) x k bytes
   rounded up) with cudaMalloc.  Returns QFS_OK or QFS_ERR_INVALID_P, QFS_ERR_INVALID_N, QFS_ERR_NULL,
   QFS_ERR_NO_MEMORY, QFS_ERR_CUDA (nothing enqueued on error).  n = 0 or m = 0 is a no-op; k = 0 zeroes C. */
int qfs_matmul_mod(int p, int n, int m, int k, const uint8_t *A, const uint8_t *B, uint8_t *C, cudaStream_t stream);

/* Exact n-th power over the integers of a homogeneous form of degree d in 4 variables (the paper's polynomial
   powering workload of Sec. 4: a degree-16 form with coefficients in {0..4} raised to the powers 5 .. 15).
   coeffs: HOST, C(d+3, 3) uint32 coefficients in descending lex order (read before the call returns).
   out: device, C(d n + 3, 3) x 8 uint32: the coefficients of f^n in descending lex order, each a 256-bit unsigned
   integer in 8 little-endian 32-bit limbs; caller-owned.  Requires d >= 1, n >= 1, d n <= 255 and
   (sum of coefficients)^n < 2^215 (QFS_ERR_INVALID_N otherwise).  Exact: the power is taken modulo up to seven
   word-size primes by number-theoretic transforms and recombined by the Chinese remainder theorem.
   Stream-ordered; may grow a library scratch buffer (cudaMalloc).  Returns QFS_OK or QFS_ERR_INVALID_N,
   QFS_ERR_NULL, QFS_ERR_NO_MEMORY, QFS_ERR_CUDA. */
int qfs_poly_power(int d, const uint32_t *coeffs, int n, uint32_t *out, cudaStream_t stream);

/* The plan of one qfs_poly_power call, without running it (host only, no GPU work): the number of NTT primes it
   takes, the transform length N (the power of two >= (d n + 1)^3), and the algorithmic device-memory bytes of the
   call, which are the reads plus writes of its kernels as launched:
   - the twiddle tables of every prime;
   - per prime: clearing and filling the packed input, and one read and one write of the N-word transform buffer
     per pass (2 k + 1 passes, k = the outer passes of 8 or fewer stages);
   - the gather of the output residues;
   - the Chinese remaindering.
   Any of nprimes, transform_len, hbm_bytes may be NULL.  coeffs: HOST, as for qfs_poly_power.  Returns QFS_OK,
   QFS_ERR_INVALID_N (the same conditions as qfs_poly_power) or QFS_ERR_NULL (coeffs NULL).  No counterpart in the
   paper: it states the traffic that the powering's roofline divides by. */
int qfs_poly_power_info(int d, const uint32_t *coeffs, int n, int *nprimes, uint64_t *transform_len,
                        uint64_t *hbm_bytes);

#ifdef __cplusplus
}
#endif
#endif /* QFS_H */
