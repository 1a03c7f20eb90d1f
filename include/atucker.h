/*
 * atucker.h: C ABI of the B300 (sm_103a) mode-wise flexible st-HOSVD library.
 *
 * Method: a-Tucker (Li, Xiao, Yang; arXiv 2010.10131).  Alg. 2 is the
 * mode-wise flexible st-HOSVD.  Per mode it runs either the EIG solver (Gram
 * S = Y_(n) Y_(n)^T, its leading R_n eigenvectors, then the truncating TTM) or
 * the ALS solver (Alg. 3, then QR of L, then TTM of the ALS factor by R^).
 * Every tensor operation is matricization-free (Sec. V).  The tensor stays in
 * its natural column-major layout, and mode n is viewed as a batch of
 * (I_<n, I_n, I_>n) slabs.
 *
 * Conventions (apply to every entry point):
 *   - Tensors are dense float32 and column-major, first index fastest (Sec. V).
 *     A C-contiguous torch tensor of shape (d_N, ..., d_1) is the column-major
 *     (d_1, ..., d_N) tensor.
 *   - Matrices are column-major.  Factor U^(n) is I_n x R_n (Sec. II-B).
 *   - Modes are 0-based; the paper counts from 1.
 *   - Unless a parameter says "host", every pointer is a device pointer that the
 *     caller owns.  The library never frees caller memory and never writes to
 *     input tensors.
 *   - `stream` is a cudaStream_t passed as void*.  NULL means the legacy default
 *     stream.  Work is stream-ordered.  Calls return when the work is enqueued,
 *     unless they are documented as synchronous.
 *   - Every call returns an atucker_status.  On failure, atucker_last_error()
 *     returns a thread-local message.  A status of ATK_ECUDA means the CUDA
 *     runtime reported an error.  The library does not reset the device.
 *   - Size limits: order <= 8, R_n <= 128, fewer than 2^31 elements.  EIG
 *     modes: I_n <= 1024 for the full Jacobi eigensolver, I_n <= 32768 for
 *     the subspace eigensolver (float32 rotations, R_n + p <= I_n / 2 with
 *     the guard p of atucker_eig_method; its n x n float64 Gram and float32
 *     copy take 12 n^2 bytes of device memory, 11 GB at 30648).
 */
#ifndef ATUCKER_H
#define ATUCKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ATK_OK = 0,
  ATK_EINVAL = -1,   /* bad argument (null pointer, bad order, bad permutation) */
  ATK_ERANK = -2,    /* infeasible ranks: need 1 <= R_n <= I_n and R_n <= prod_{k!=n} R_k,
                        or a Cholesky factorisation inside ALS met a non-positive pivot */
  ATK_ENOMEM = -3,   /* device allocation failed */
  ATK_ECUDA = -4,    /* CUDA runtime error */
  ATK_ENOCONV = -5,  /* the Jacobi eigensolver hit its sweep cap (results still written) */
  ATK_ETIMEOUT = -6, /* a bounded device-side wait gave up (grid barrier) */
  ATK_EUNSUPPORTED = -7 /* a size limit above was exceeded */
} atucker_status;

/* Per-mode solver, Alg. 2: 0 = EIG (Gram + eigen-decomposition), 1 = ALS (Alg. 3). */
typedef enum { ATK_AUTO = -1, ATK_EIG = 0, ATK_ALS = 1 } atucker_solver;

/* Per-mode configuration classes: the output space of the learned selector
 * (solver x tile class).  "Tile" is the row tile of the float32 Gram (a2):
 * AUTO picks 128 / 64 / 32 from I_n; SMALL takes the next smaller one.
 * The eigensolver methods are those of atucker_eig_method.
 *   ATK_CLASS_EIG             EIG, eigensolver ATK_EIG_AUTO (or the plan's
 *                             ATK_OPT_EIG_METHOD), Gram tile AUTO
 *   ATK_CLASS_EIG_SMALL       EIG, same eigensolver, Gram tile SMALL
 *   ATK_CLASS_EIG_JACOBI      EIG, full Jacobi eigensolver, Gram tile AUTO
 *   ATK_CLASS_EIG_JACOBI_SMALL EIG, full Jacobi, Gram tile SMALL
 *   ATK_CLASS_ALS             ALS (Alg. 3) with the plan's sweep count */
typedef enum {
  ATK_CLASS_EIG = 0,
  ATK_CLASS_EIG_SMALL = 1,
  ATK_CLASS_EIG_JACOBI = 2,
  ATK_CLASS_EIG_JACOBI_SMALL = 3,
  ATK_CLASS_ALS = 4,
  ATK_NUM_CLASSES = 5
} atucker_mode_class;

/* Arithmetic for the bulk Gram / TTM / ALS contractions.
 * ATK_FP32 is plain float32 on the CUDA cores, accumulated in float32 and
 * reduced in float64 across split-K partials.  The tensor-core forms
 * (tcgen05, float32 accumulation in tensor memory, the same float64 split-K
 * reduction) apply to the Gram of EIG modes:
 *   ATK_TF32     operands rounded to TF32 (round to nearest)
 *   ATK_BF16     operands rounded to BF16
 *   ATK_BF16X3   x = hi + lo (both BF16); hi hi^T + hi lo^T + lo hi^T
 *   ATK_FP8E4M3  each mode-n row i scaled by the power of two
 *                s_i = 2^floor(log2(448 / max |row i|)), rounded to e4m3; the
 *                product is divided by s_i s_j exactly afterwards
 * The tensor-core forms also run the truncating TTM of EIG modes with
 * R_n > 16 (tcgen05, operands converted from the float32 tensor in place;
 * below that the float32 TTM already reads Y at HBM speed); FP8 scales mode-n
 * index i of Y by s_i as above, folds 1 / s_i into U and scales each column
 * r of U by a power of two t_r, undone exactly after the product).
 *   ATK_FP32C    float32 on the CUDA cores with compensated sums: every
 *                product made exact (p + e with e = fma(a, b, -p)) and the
 *                running sum carried as a float-float pair (TwoSum), about
 *                48 bits per partial sum at about nine times the float32 cost
 * The eigensolver, the ALS solver and the orthonormalisation are the same
 * in every form; ATK_FP32C applies to the Gram (its TTM is ATK_FP32). */
typedef enum {
  ATK_FP32 = 0, ATK_TF32 = 1, ATK_BF16 = 2, ATK_BF16X3 = 3, ATK_FP8E4M3 = 4, ATK_FP32C = 5
} atucker_precision;

/* Arithmetic of the Jacobi rotations in the eigensolver.  Either way, the
 * Gram arrives in float64, and eigenvalue sums and the final
 * orthonormalisation of U run in float64. */
typedef enum { ATK_EIG_ROT_FP32 = 0, ATK_EIG_ROT_FP64 = 1 } atucker_eig_arith;

/* Eigensolver method for EIG modes (all give the R leading eigenvectors of S).
 * FULL_JACOBI diagonalises the whole I_n x I_n Gram.  SUBSPACE runs block
 * subspace iteration on m = R + p columns (p = min(max(8, R), 32)), projects
 * (Rayleigh-Ritz), and diagonalises the m x m projection with the same Jacobi.
 * It iterates until (theta_m / theta_R) * max_j<R ||S q_j - theta_j q_j|| /
 * (theta_R - theta_m) <= 1e-6.  That quantity is a Davis-Kahan bound times the
 * contraction of the refinement step below.  It falls back to FULL_JACOBI
 * when theta_m > theta_R / 2 (a clustered cut) or after 20 iterations.  AUTO uses SUBSPACE when
 * 2m <= I_n and float32 rotations are selected.  Every method ends with the
 * same float64 refinement of the leading block (the m Ritz vectors, or the R
 * Jacobi vectors): one subspace-iteration step, a Rayleigh-Ritz projection
 * and simultaneous Jacobi steps on it, all in float64. */
typedef enum { ATK_EIG_AUTO = 0, ATK_EIG_FULL_JACOBI = 1, ATK_EIG_SUBSPACE = 2 } atucker_eig_method;

/* Keys for atucker_plan_set_option. */
typedef enum {
  ATK_OPT_EIG_ARITH = 1,  /* atucker_eig_arith; default ATK_EIG_ROT_FP32 */
  ATK_OPT_SYNC = 2,       /* 1: atucker_sthosvd synchronises and returns the device status (default 0) */
  ATK_OPT_JACOBI_MAX_SWEEPS = 3, /* sweep cap of the Jacobi eigensolver (default 40) */
  ATK_OPT_TIMING = 4,     /* 1: record CUDA events around each phase (see atucker_plan_timings) */
  ATK_OPT_EIG_METHOD = 5, /* atucker_eig_method; default ATK_EIG_AUTO */
  /* Precise Gram for a cut that float32 does not resolve (float32 rotations).
   * A float32 Gram's rounding reaches eps_32 times its largest partial sum,
   * about eps_32 lambda_1 when the energy sits in few entries.  When the gap
   * between the R-th and the next Rayleigh quotient is below 64 eps_32
   * lambda_1 (the Gram cannot decide which vectors lie on either side of the
   * cut) or below 1e4 eps_32 sqrt(2 R) lambda_1 (the kept subspace could
   * turn by more than a 1e-4 projector distance), the mode's Gram is
   * recomputed in ATK_FP32C and solved again.  0: never; 1 (default): every
   * EIG mode but the first processed one (that mode reads the caller's
   * tensor, whose entries are of comparable size, so its float32 roundings
   * stay independent and small; later modes read the shrinking core, whose
   * energy sits in few entries); 2: every EIG mode. */
  ATK_OPT_GRAM_REFINE = 6,
  /* Poll limit of every grid-barrier wait of the cooperative block Jacobi
   * (full Jacobi with I_n > 160) in this plan's runs; 0 (default) keeps 2e7
   * polls of 64 ns, about a second.  A wait that reaches the limit records
   * ATK_ETIMEOUT in the plan's status and its CTA returns; the others give up
   * at their next wait, so the kernel ends on its own and the next
   * atucker_plan_sync reports ATK_ETIMEOUT.  The results of such a run are
   * not usable; the plan is.  Small values exist to test that path. */
  ATK_OPT_WAIT_LIMIT = 7,
  /* 1: explicit matricization, the baseline that Sec. V removes (the
   * ablation of Sec. VI-E).  Before each mode with I_<n > 1 the tensor's
   * mode-n unfolding is copied into a buffer (a batched transpose of the
   * view's slabs), the mode's Gram, eigensolver, TTM or ALS run on that
   * matrix as a mode-1 view, and the R_n x J_n result is transposed back into
   * the core's natural layout.  Same arithmetic, so the same results to
   * rounding; extra device memory (allocated at the first such run): the
   * largest unfolding plus the largest TTM result.  0 (default): the
   * matricization-free path. */
  ATK_OPT_EXPLICIT_UNFOLD = 8,
  /* 1: where the next mode in the processing order is an EIG mode with
   * 16 <= I_m <= 128, this mode's R_n <= 64 and the precision is ATK_FP32,
   * the TTM closing this mode also forms the next mode's Gram from its output
   * tiles (atucker_ttm_gram), and that mode skips its Gram pass over Y'.
   * 0 (default): every Gram reads its input from memory. */
  ATK_OPT_FUSE_TTM_GRAM = 9
} atucker_option;

typedef struct atucker_plan_s* atucker_plan_t;

/* Build a plan for one tensor shape (Alg. 2 inputs, Sec. III-A).
 *   order            N, 1 <= N <= 8
 *   dims, ranks      host arrays of N entries: I_n and R_n
 *   mode_order       host permutation of 0..N-1: the order modes are processed
 *                    in (the paper's loop runs n = 1..N); NULL = 0,1,..,N-1
 *   solver_per_mode  host array of N atucker_solver values indexed by mode;
 *                    NULL = EIG for every mode.  ATK_AUTO lets the learned
 *                    selector (atucker_selector_set or _set_tree) pick the
 *                    mode's class.  Where it cannot decide, the plan's first
 *                    atucker_sthosvd times the candidates on that input (an
 *                    exhaustive search, Sec. IV): with no selector loaded,
 *                    every class that can run the mode; with the network,
 *                    its best class and up to two more whose predicted log2
 *                    times are within 2 of it (4 x).  That call runs
 *                    each candidate twice (warm-up, then timed with CUDA
 *                    events), keeps each mode's fastest, and caches the choice
 *                    for the process, keyed by shape, ranks, order and the
 *                    plan's options; later plans of that key skip the search.
 *                    Until then atucker_plan_classes reports the starting
 *                    guess (the prediction, or ATK_CLASS_EIG).  The workspace
 *                    of such a plan covers every candidate.
 *   precision        atucker_precision
 *   als_sweeps       ALS iterations (num_iters of Eq. 5; the paper's default is
 *                    5); <= 0 selects 5
 *   seed             seed of the ALS initial guess L_0.  For mode n, entry
 *                    e = i + I_n r (column-major) is sqrt(-2 ln u1) cos(2 pi u2),
 *                    with u1 = (w(2e+1) + 1) 2^-53 and u2 = w(2e+2) 2^-53.  Here
 *                    w(c) is the top 53 bits of mix(s + c * 0x9E3779B97F4A7C15),
 *                    with s = seed ^ (0x9E3779B97F4A7C15 * (n + 1)) and mix the
 *                    splitmix64 output function.
 *   stream           cudaStream_t used by every call on this plan
 * The plan allocates its device workspace: two ping-pong buffers for the
 * shrinking core, the Gram split-K scratch, and the small matrices.
 * Returns ATK_ERANK for infeasible ranks, ATK_EUNSUPPORTED beyond the size
 * limits, ATK_ENOMEM if the workspace cannot be allocated. */
int atucker_plan_create(atucker_plan_t* plan, int order, const int64_t* dims, const int64_t* ranks,
                        const int* mode_order, const int* solver_per_mode, int precision, int als_sweeps,
                        uint64_t seed, void* stream);

/* Set a plan option (atucker_option).  Returns ATK_EINVAL for unknown keys/values. */
int atucker_plan_set_option(atucker_plan_t plan, int key, int64_t value);

/* Run Alg. 2 on the device tensor x (I_1 x ... x I_N, column-major, not modified).
 *   core_out      device, R_1 x ... x R_N column-major float32
 *   factors_out   device, U^(1) .. U^(N) in mode-index order (not processing
 *                 order), each I_n x R_n column-major float32, concatenated
 *   discarded_out device, N float64 (nullable): energy removed at mode n's
 *                 step.  EIG: the sum of the Gram eigenvalues beyond R_n.
 *                 ALS: ||Y||^2 - ||Y'||^2.  With EIG modes only,
 *                 ||X - X_hat||^2 = sum of these.
 * Eigenvectors are ordered by descending eigenvalue.  Each column is signed
 * so that its largest-magnitude entry is positive.  ALS factors come from a QR
 * with positive diag(R^).
 * Asynchronous on the plan's stream unless ATK_OPT_SYNC is set.  Device-side
 * conditions (Jacobi sweep cap, barrier timeout) are reported by the next
 * atucker_plan_sync. */
int atucker_sthosvd(atucker_plan_t plan, const float* x, float* core_out, float* factors_out,
                    double* discarded_out);

/* Same as atucker_sthosvd, with HOST buffers (preferably pinned).  Copies x to
 * the device, runs, copies core/factors/discarded back, and synchronises.
 * discarded_out is host, nullable.  The plan keeps a device copy buffer for x,
 * allocated on first use. */
int atucker_sthosvd_host(atucker_plan_t plan, const float* x_host, float* core_host, float* factors_host,
                         double* discarded_host);

/* Wait for the plan's stream and return the device status word of the last
 * run: ATK_OK, ATK_ENOCONV or ATK_ETIMEOUT. */
int atucker_plan_sync(atucker_plan_t plan);

/* Device time per phase of the runs since timing was enabled or last read,
 * from CUDA events recorded on the plan's stream (ATK_OPT_TIMING = 1).
 * Synchronises the stream.  out (host, count >= 10):
 *   [0] Gram partial-tile kernel ms   [1] Gram split-K reduction ms
 *   [2] eigensolver ms (Jacobi, selection, float64 polish)
 *   [3] TTM ms   [4] ALS mode ms   [5] norms ms   [6] total ms
 *   [7] Gram kernel launches   [8] kernel launches made by this plan's runs   [9] runs
 * Resets the accumulators. */
int atucker_plan_timings(atucker_plan_t plan, double* out, int count);

/* Free the plan and its workspace.  Safe on NULL. */
void atucker_plan_destroy(atucker_plan_t plan);

/* Several independent tensors at once (Alg. 2 per tensor).  Plan i runs
 * atucker_sthosvd(plans[i], xs[i], cores[i], factors[i], discarded[i]) on a
 * host thread of its own (a persistent pool), so one tensor's eigensolver,
 * which occupies a few CTAs, overlaps another tensor's Gram and TTM.  Give the
 * plans distinct streams for that overlap; on one shared stream the runs
 * serialise.  Stream priorities (cudaStreamCreateWithPriority) decide which
 * plan's kernels the GPU dispatches first when both have work; the plan on the
 * longest chain benefits from the highest priority.
 *   count            number of plans, >= 1
 *   plans            host array of count distinct plans
 *   xs, cores,       host arrays of count device pointers, as in
 *   factors          atucker_sthosvd
 *   discarded        host array of count device pointers (entries nullable),
 *                    or NULL for none
 * Returns when every run is enqueued (or finished, for plans with
 * ATK_OPT_SYNC).  On failure returns the first failing plan's status in plan
 * order; atucker_last_error() names the plan.  Per-plan timings and launch
 * counts (atucker_plan_timings) stay per plan. */
int atucker_sthosvd_many(int count, const atucker_plan_t* plans, const float* const* xs, float* const* cores,
                         float* const* factors, double* const* discarded);

/* As atucker_sthosvd_many with HOST buffers: plan i runs
 * atucker_sthosvd_host, so one plan's copies overlap another's kernels.
 * Synchronous: returns when every result is in host memory. */
int atucker_sthosvd_host_many(int count, const atucker_plan_t* plans, const float* const* xs_host,
                              float* const* cores_host, float* const* factors_host,
                              double* const* discarded_host);

/* One-shot form of the problem statement (Alg. 2): plan, run synchronously on
 * the default stream in FP32, free.  Device pointers as in atucker_sthosvd. */
int atucker_sthosvd_oneshot(const float* x, int order, const int64_t* dims, const int64_t* ranks,
                            const int* mode_order, const int* solver_per_mode, float* core_out,
                            float* factors_out);

/* Process-wide cap on the size of any single device allocation the library
 * makes: plan workspaces, host-buffer staging, step-level scratch, batch and
 * selector buffers.  A request above the cap fails with ATK_ENOMEM before
 * any CUDA call, exactly as an exhausted device would fail it, so a service
 * can bound what the library takes and tests can drive the out-of-memory
 * paths.  0 (default) removes the cap.  Always returns ATK_OK. */
int atucker_set_device_alloc_limit(uint64_t bytes);

/* Thread-local message of the last failing call ("" if none). */
const char* atucker_last_error(void);

/* Library version, e.g. "0.1.0". */
const char* atucker_version(void);

/* ------------------------------------------------------------------------
 * Step-level entry points: one row of the hot path each, on a mode-n slab view
 * (lo, n, hi) = (I_<n, I_n, I_>n) of a column-major tensor.  Element (a, i, b)
 * sits at a + lo * (i + n * b) (Sec. V: loops split outside/along/inside mode
 * n).  Each call allocates its own scratch from the stream-ordered allocator
 * and frees it before returning.
 * ------------------------------------------------------------------------ */

/* Gram matrix S = Y_(n) Y_(n)^T (Alg. 2, EIG branch; cost I_n^2 J_n, Eq. 4).
 * y: lo*n*hi float32.  S_out: n x n float64, full symmetric.  Single-pass
 * split-K: float32 partial tiles, reduced in float64 in a fixed order
 * (deterministic).  Synchronous.  The tensor-core forms read back the
 * kernels' status word and return ATK_ETIMEOUT if a bounded device-side wait
 * gave up. */
int atucker_gram(const float* y, int64_t lo, int64_t n, int64_t hi, int precision, double* S_out,
                 void* stream);

/* Gram matrix as atucker_gram, without allocating any device memory.  The
 * paper has no counterpart: this entry point serves callers that cannot
 * allocate GPU memory at call time.  Examples: a service that reserved its
 * whole memory budget up front, a process whose free device memory is already
 * held by a framework's caching allocator, or a hook that must not re-enter
 * the CUDA allocator.
 *   - The split-K partial tiles live in one fixed 16 MiB device array inside
 *     the library (float32).  Every GPU that loads the library holds it until
 *     the process exits.
 *   - Limit: n <= 2048 (one split's partial tiles must fit); larger n returns
 *     ATK_EUNSUPPORTED.  When a view needs more splits than the array holds,
 *     they run in rounds whose sums are added in float64, so every float32
 *     partial sum stays within 8192 terms, as in atucker_gram.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.  That lookup may load
 *     the library's module on the device and so reserve the 16 MiB then: make
 *     a first call before fixing a memory budget, and before any stream
 *     capture.  The address is cached for the process; after a device reset,
 *     start a new process.
 *   - All calls share the array: calls that overlap on the GPU (other streams,
 *     other threads) race and corrupt each other's results.  Nothing in the
 *     array needs to start at zero; each call writes every tile it reads.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
int atucker_gram_noalloc(const float* y, int64_t lo, int64_t n, int64_t hi, double* S_out, void* stream);

/* Truncating TTM Y' = Y x_n U^T (Eq. 2 with the matrix U^T; Alg. 2, EIG branch).
 * U: n x R float32 column-major.  out: lo x R x hi float32 column-major.
 * precision: ATK_FP32 (or ATK_FP32C, the same) on the CUDA cores, R <= 1024;
 * a tensor-core form (R <= 128) is synchronous and returns ATK_ETIMEOUT if a
 * bounded device-side wait gave up. */
int atucker_ttm(const float* y, int64_t lo, int64_t n, int64_t hi, const float* U, int64_t R, int precision,
                float* out, void* stream);

/* Fused truncating TTM and next-mode Gram (Alg. 2: the TTM that closes one
 * mode and the Gram that opens the next are adjacent steps).
 *   y, lo, n, hi, U, R  as atucker_ttm (ATK_FP32): out = Y x_n U^T, lo x R x hi
 *   s, m_size           the next mode m of out: its stride among the rows
 *                       c = a + lo b of the mode-n view, and its size I_m, so
 *                       that c = low + s (i + I_m high), i < I_m; s I_m must
 *                       divide lo hi.  For out's modes in storage order, s is
 *                       the product of the sizes of the modes below m other
 *                       than n.
 *   S_out               device, I_m x I_m float64: S = out_(m) out_(m)^T, the
 *                       Gram of out's mode m (summed in a fixed order, so
 *                       reproducible; not bit-identical to atucker_gram)
 * Needs 1 <= R <= 64 and 16 <= I_m <= 128 (ATK_EUNSUPPORTED otherwise).
 * Allocates its partial-Gram scratch (at most 8 x 148 x I_m^2 floats) on the
 * stream; synchronous. */
int atucker_ttm_gram(const float* y, int64_t lo, int64_t n, int64_t hi, const float* U, int64_t R, int64_t s,
                     int64_t m_size, float* out, double* S_out, void* stream);

/* Leading-R eigenpairs of the symmetric n x n float64 matrix S (Alg. 2, EIG
 * branch) by parallel-order cyclic Jacobi, on the whole matrix or on a
 * Rayleigh-Ritz projection (atucker_eig_method).  Rotations run in float32 or
 * float64 (atucker_eig_arith).  Full Jacobi on n > 128 uses block Jacobi with
 * 64 x 64 pair sub-problems.  The float64 refinement above follows, so the
 * kept vectors are orthonormal and the kept eigenvalues are float64 Rayleigh
 * quotients u^T S u.
 *   U_out       n x R float32: eigenvectors of the R largest eigenvalues,
 *               descending, sign rule as in atucker_sthosvd
 *   lambda_out  n float64 (nullable): [0, R) the kept eigenvalues; [R, n)
 *               the remaining eigenvalues, descending, from the full Jacobi
 *               (NaN when the subspace method ran)
 *   discarded_out 1 float64 (nullable): trace(S) minus the kept eigenvalues
 * Needs 1 <= R <= 128 and R <= n <= 1024, or n <= 32768 on the subspace path
 * (ATK_EUNSUPPORTED otherwise).  Returns ATK_ENOCONV if a sweep cap
 * was reached.  Synchronous. */
int atucker_eig(const double* S, int64_t n, int64_t R, int eig_arith, int eig_method, float* U_out,
                double* lambda_out, double* discarded_out, void* stream);

/* ALS solver for one mode (Alg. 2, ALS branch, with Alg. 3).
 *   L0       n x R float64, the initial guess (nullable: the plan's seeded
 *            L_0 for mode index `mode` with `seed`, see atucker_plan_create)
 *   sweeps   ALS iterations (exactly this many; <= 0 selects 5)
 *   U_out    n x R float32: Q^ of the QR of L_K (diag(R^) > 0)
 *   core_out lo x R x hi float32: the factor R_{K-1} tensorised, times R^ along mode n
 * Synchronous.  ATK_ERANK if a Cholesky pivot is not positive. */
int atucker_als_mode(const float* y, int64_t lo, int64_t n, int64_t hi, int64_t R, const double* L0,
                     uint64_t seed, int mode, int sweeps, int precision, float* U_out, float* core_out,
                     void* stream);

/* As atucker_plan_create, with one atucker_mode_class per mode (host array of
 * N values indexed by mode) instead of solver_per_mode. */
int atucker_plan_create_classes(atucker_plan_t* plan, int order, const int64_t* dims, const int64_t* ranks,
                                const int* mode_order, const int* class_per_mode, int precision, int als_sweeps,
                                uint64_t seed, void* stream);

/* The class each mode of the plan runs with (host array of N, by mode). */
int atucker_plan_classes(atucker_plan_t plan, int* class_out);

/* Per-mode device time (ms, CUDA events on the plan's stream, ATK_OPT_TIMING
 * = 1) summed over the runs since the last call; ms_out has N entries indexed
 * by mode.  Synchronises the plan's stream. */
int atucker_plan_mode_timings(atucker_plan_t plan, double* ms_out, int count);

/* ---------------------------------------------------------------------------
 * Learned per-mode selector (the paper's adaptive solver selection, Sec. IV,
 * with an MLP in place of the decision tree).
 *
 * Features of mode n when it is processed (Table I's ten, plus two):
 *   0 I_n  1 R_n  2 J_n  3 I_n^2  4 R_n^2  5 I_n R_n  6 R_n^2/I_n
 *   7 R_n^2/J_n  8 I_n/J_n  9 R_n/J_n  10 position  11 remaining size
 * J_n is the product of the other modes' current sizes (modes processed
 * earlier are already truncated to R), position = step / (N - 1) (0 for
 * N = 1) and remaining size = I_n J_n.  Every feature except the position
 * enters as log2.  The network is 12 -> 64 -> 64 -> ATK_NUM_CLASSES with
 * ReLU hidden layers; its outputs predict, for each class, log2 of the mode's
 * time relative to the fastest class, and the selector takes the smallest.
 * ------------------------------------------------------------------------ */
#define ATK_SELECTOR_FEATURES 12
#define ATK_SELECTOR_HIDDEN 64

/* Model inputs (log2 applied, not standardised) of every mode: out holds
 * order x 12 values, row n for mode n. */
int atucker_mode_features(int order, const int64_t* dims, const int64_t* ranks, const int* mode_order,
                          double* out);

/* Number of network parameters for (in, hidden, out): hidden*in + hidden +
 * hidden*hidden + hidden + out*hidden + out.  Layout, all row-major float32:
 * W1 [hidden x in], b1, W2 [hidden x hidden], b2, W3 [out x hidden], b3. */
int64_t atucker_mlp_param_count(int in, int hidden, int out);

/* Load the selector used by ATK_AUTO: 12 feature means, 12 feature scales
 * (standardised x = (f - mean) / scale), then the network parameters for
 * (12, 64, ATK_NUM_CLASSES).  count must be 24 + that parameter count.
 * Process-wide; the values are copied. */
int atucker_selector_set(const float* params, int64_t count);
void atucker_selector_clear(void);

/* The paper's own selector as an alternative (Sec. IV-B: a decision tree on
 * Table I's features, trained offline): a binary tree of `nodes` nodes, node
 * 0 the root.  Node i is a leaf when feature[i] < 0, choosing class
 * leaf_class[i]; otherwise it sends a row to left[i] when
 * features[feature[i]] <= threshold[i] (raw features, as from
 * atucker_mode_features), else to right[i], with both children numbered after
 * i.  Loading a tree makes it the active selector (AUTO and
 * atucker_selector_predict) until atucker_selector_set loads a network or
 * atucker_selector_clear removes both.  Process-wide; the arrays are copied. */
int atucker_selector_set_tree(int nodes, const int* feature, const double* threshold, const int* left,
                              const int* right, const int* leaf_class);

/* Host inference of the loaded selector on `rows` raw feature rows (rows x 12,
 * as from atucker_mode_features): class_out[rows] the chosen class,
 * scores_out (nullable) rows x ATK_NUM_CLASSES network outputs (for a tree:
 * 0 for the chosen class, 1 for the others).  A class is chosen only where
 * it can run: the full-Jacobi classes need I_n <= 1024, the other EIG
 * classes I_n <= 32768; beyond that the mode gets ATK_CLASS_ALS. */
int atucker_selector_predict(const double* features, int rows, int* class_out, float* scores_out);

/* GPU training of the network (the project's own CUDA kernels).  All pointers
 * are device float32:
 *   X       B x in standardised inputs (row-major)
 *   Y       B x out targets, M the B x out mask (1 = target present)
 *   params  parameter vector (layout above), updated in place
 *   grad    gradient of the loss, same layout
 * Loss = sum over masked entries of (output - Y)^2 / (number of masked entries).
 * atucker_mlp_forward: out (B x out) = network(X).
 * atucker_mlp_loss_grad: loss (1 value, device) and grad at params.
 * atucker_mlp_train: `steps` full-batch Adam steps (beta1 0.9, beta2 0.999,
 *   eps 1e-8, step size lr, bias-corrected; `state` holds 2 x param count
 *   floats of moments, zero at the first call, and step_base the number of
 *   steps already taken); loss_out (device, nullable) receives the loss of
 *   every step. */
int atucker_mlp_forward(const float* X, int B, int in, int hidden, int out, const float* params, float* Y_out,
                        void* stream);
int atucker_mlp_loss_grad(const float* X, const float* Y, const float* M, int B, int in, int hidden, int out,
                          const float* params, float* loss, float* grad, void* stream);
int atucker_mlp_train(const float* X, const float* Y, const float* M, int B, int in, int hidden, int out,
                      float* params, float* state, int steps, int step_base, float lr, float* loss_out,
                      void* stream);

/* ---------------------------------------------------------------------------
 * Batched form: many small order-3 tensors in one persistent launch.
 *
 * Alg. 2 runs on every tensor with the EIG solver in every mode and mode
 * order 1, 2, 3, exactly as atucker_sthosvd would, except that the Jacobi
 * eigenvectors are used as computed in float32 (no float64 refinement step)
 * and no discarded energies are returned.  Each CTA of one persistent kernel
 * takes whole tensors from a device work counter, largest first, so a whole
 * batch is one launch; it is captured once in a CUDA graph (pointer-table
 * upload, counter reset, kernel) and replayed by atucker_batch_run.
 *
 * Limits: every dimension in [1, 96], every rank in [1, min(dim, 32)], and
 * Tucker-feasible ranks (R_n <= product of the other two ranks), else
 * ATK_EUNSUPPORTED / ATK_ERANK at creation.
 * ------------------------------------------------------------------------ */
typedef struct atucker_batch_s* atucker_batch_t;

enum atucker_batch_option {
  ATK_BATCH_OPT_VARIANT = 1,            /* launch variant index (see atucker_batch_variants); set by tuning */
  ATK_BATCH_OPT_GRAPH = 2,              /* 1 (default): replay a CUDA graph; 0: plain launches */
  ATK_BATCH_OPT_SYNC = 3,               /* 1: atucker_batch_run waits and returns the device status */
  ATK_BATCH_OPT_JACOBI_MAX_SWEEPS = 4   /* sweep cap of the Jacobi eigensolver (default 40) */
};

/* Create a batch of `count` tensors.  dims3 and ranks3 are host arrays of
 * 3 * count values: tensor t has dims (dims3[3t], dims3[3t+1], dims3[3t+2])
 * and ranks likewise.  The batch owns its device workspace (one block of
 * R1 d2 d3 + R1 R2 d3 floats per resident CTA) and runs on `stream`. */
int atucker_batch_create(atucker_batch_t* batch, int count, const int64_t* dims3, const int64_t* ranks3,
                         void* stream);
int atucker_batch_set_option(atucker_batch_t batch, int option, int64_t value);

/* Decompose the batch.  xs, cores and factors are HOST arrays of `count`
 * device pointers: tensor t is read from xs[t] (d1 x d2 x d3 float32,
 * column-major, not modified), its core is written to cores[t] (R1 x R2 x R3)
 * and its factors to factors[t] (U1 | U2 | U3, each d_n x R_n column-major,
 * concatenated).  The pointer tables are copied at the call.  Asynchronous on
 * the batch's stream unless ATK_BATCH_OPT_SYNC is set; a later call waits for
 * the previous one to finish reading its tables. */
int atucker_batch_run(atucker_batch_t batch, const float* const* xs, float* const* cores, float* const* factors);

/* Wait for the last run; returns ATK_ENOCONV if any Jacobi reached its sweep
 * cap, ATK_ETIMEOUT for a timed-out wait, else ATK_OK. */
int atucker_batch_sync(atucker_batch_t batch);

/* Autotuner: run every launch variant on this batch (one warm-up and `reps`
 * timed runs each, CUDA events on the batch's stream), keep the fastest.
 * ms_out (nullable) receives the mean time of each variant. */
int atucker_batch_tune(atucker_batch_t batch, const float* const* xs, float* const* cores, float* const* factors,
                       int reps, float* ms_out);
int atucker_batch_get_variant(atucker_batch_t batch, int* variant_out);

/* The launch variants: count, and per variant threads per CTA and c values per
 * staged Gram chunk (each array sized by the count; nullable). */
int atucker_batch_variants(int* count_out, int* threads_out, int* chunk_out);
void atucker_batch_destroy(atucker_batch_t batch);

#ifdef __cplusplus
}
#endif
#endif /* ATUCKER_H */
