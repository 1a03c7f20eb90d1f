// Internal definitions shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>

#include "atucker.h"

namespace atk {

// ---------------------------------------------------------------- stride view
// Mode-n view of a column-major tensor (Sec. V): loops outside mode n merge into
// `hi`, loops inside it into `lo`.  Element (a, i, b) sits at a + lo*(i + n*b).
// The "other" index c in [0, lo*hi) enumerates (a, b) as c = a + lo*b; it is
// the column index of the mode-n matricization X_(n) (Sec. II-A), so every
// contraction over the non-n modes is a sum over c.
struct View {
  int64_t lo, n, hi;
  __host__ __device__ int64_t J() const { return lo * hi; }
  __host__ __device__ int64_t size() const { return lo * n * hi; }
  // Offset of (c, i) given the precomputed split of c.
  __host__ __device__ static int64_t off(int64_t a, int64_t b, int64_t i, int64_t lo, int64_t n) {
    return a + lo * (i + n * b);
  }
};

// View of mode `mode` for the current dims.
inline View make_view(int order, const int64_t* cur, int mode) {
  View v{1, cur[mode], 1};
  for (int k = 0; k < mode; ++k) v.lo *= cur[k];
  for (int k = mode + 1; k < order; ++k) v.hi *= cur[k];
  return v;
}

// ------------------------------------------------------------------- errors
void set_error(const std::string& msg);
int cuda_status(cudaError_t e, const char* what);

#define ATK_CUDA(call)                                    \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::atk::cuda_status(_e, #call); \
  } while (0)
// Every kernel launch site ends with ATK_LAUNCHED(): it checks the launch and
// counts it (the count is reported by atucker_plan_timings).
void count_launch();
long long launch_count();
void count_launches(long long k);
#define ATK_LAUNCHED()                                                   \
  do {                                                                   \
    cudaError_t _e = cudaGetLastError();                                 \
    if (_e != cudaSuccess) return ::atk::cuda_status(_e, "kernel launch"); \
    ::atk::count_launch();                                               \
  } while (0)
#define ATK_TRY(call)            \
  do {                           \
    int _s = (call);             \
    if (_s != ATK_OK) return _s; \
  } while (0)

// Device status word bits (written by kernels, read by atucker_plan_sync).
enum : int { DEV_NOCONV = 1, DEV_TIMEOUT = 2, DEV_CHOL = 4 };

// ------------------------------------------------------- compile-time loop
// f(std::integral_constant<int, P>{}) for P = B .. E-1: a loop whose index is
// a constant in the body, so register arrays indexed by it stay in registers.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ------------------------------------------------------------ float-float sum
// Fixed-order sum of float32 terms carried as an unevaluated pair hi + lo
// (Knuth's TwoSum makes each hi update exact; lo collects the errors).  The
// relative error is about (terms) * 2^-48, far below the float32 partials'
// own rounding, and it runs on the float32 pipe: B300's float64 pipe issues
// about two operations per clock per SM.  Converted to float64 once.
struct FFSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = hi + v;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (v - bp);
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ------------------------------------------------------------ grid barrier
// Sense-reversing barrier across the CTAs of a cooperative launch.  Every wait
// is bounded: after `limit` polls the CTA sets DEV_TIMEOUT in *status and
// leaves; callers check the return value and exit.  `bar` points at two
// zero-initialised words: [0] arrival count, [1] generation.
__device__ inline bool grid_barrier(unsigned* bar, unsigned nblocks, int* status, long long limit = 20000000LL) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    unsigned gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    ok = 1;
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long polls = 0;
      while (*vgen == gen) {
        if (++polls > limit) {
          atomicOr(status, DEV_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ok && (*(volatile int*)status & DEV_TIMEOUT)) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// ------------------------------------------------------------- host helpers
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
// Device allocations of the library (plan workspaces, host-buffer staging,
// step-level scratch, batch and selector buffers).  A request above the
// process-wide cap of atucker_set_device_alloc_limit fails with ATK_ENOMEM
// before any CUDA call; otherwise cudaMalloc / cudaMallocAsync.
int dev_alloc(void** ptr, size_t bytes, const char* what);
int dev_alloc_async(void** ptr, size_t bytes, cudaStream_t st, const char* what);
// Poll limit of the grid-barrier waits of the cooperative Jacobi for plan runs
// on the calling host thread (ATK_OPT_WAIT_LIMIT); 0 keeps the default.
void set_wait_limit(long long polls);
long long wait_limit();
int num_sms();

// Device scratch carved from one allocation; each take() is 256-byte aligned.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  void* take(size_t bytes) {
    size_t start = (used + 255) & ~size_t(255);
    if (start + bytes > cap) return nullptr;
    used = start + bytes;
    return base + start;
  }
};

// ------------------------------------------------------------ kernel entry points
// FP32 CUDA-core contractions (fp32_ops.cu).
// Gram row tile the float32 engine picks for a mode of size n (128, 64 or 32).
int gram_tile(int64_t n);
// True once atucker_selector_set has loaded a selector (selector.cu).
bool selector_loaded();
// Whether class k can run a mode with log2 I_n = lg (selector.cu).
bool selector_class_fits(int k, double lg);
// `bm` forces the Gram row tile (32, 64 or 128); 0 picks it from n.
size_t gram_scratch_bytes(const View& v, int bm = 0);
// `mid` (nullable) is recorded between the partial-tile kernel and the reduction.
// 128-row tiles of a view with rows contiguous in i (lo == 1, I_n % 4 == 0,
// 16-byte aligned) run in one cp.async-fed launch for every tile.
int gram_f32(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes, cudaStream_t st,
             cudaEvent_t mid = nullptr, int bm = 0);
// As gram_f32, with the number of split-K partials capped to fit scratch_bytes.
int gram_f32_fixed_scratch(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes,
                           cudaStream_t st);
int ttm_f32(const float* y, const View& v, const float* U, int64_t R, float* out, cudaStream_t st);
// Fused TTM and next-mode Gram (ttm_gram.cu): out = Y x_n U^T as ttm_f32, and
// S = the I_m x I_m Gram of the next mode m of out, whose stride among the
// TTM's rows c is s (c = low + s (i + I_m high)).  Needs 1 <= R <= 64,
// 16 <= I_m <= 128 and I_m s dividing J (ttm_gram_ok).
bool ttm_gram_ok(const View& v, int64_t R, int64_t s, int64_t Im);
size_t ttm_gram_scratch_bytes(const View& v, int64_t R, int64_t s, int64_t Im);
int ttm_gram(const float* y, const View& v, const float* U, int64_t R, int64_t s, int64_t Im, float* out,
             double* S, void* scratch, size_t scratch_bytes, cudaStream_t st);
// C (n x R, float64) = sum_c Y(c, i) P(c, r); P is a (lo, R, hi) tensor.
size_t cross_scratch_bytes(const View& v, int64_t R);
int cross_f32(const float* y, const View& v, const float* P, int64_t R, double* C, float* scratch,
              size_t scratch_bytes, cudaStream_t st);

// Compensated Gram (gram_cmp.cu): exact float32 products summed as
// float-float pairs (about 48 bits per partial sum); the split count adapts
// to scratch_bytes (at least one split must fit).
size_t gram_cmp_scratch_bytes(const View& v);
int gram_cmp(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes, cudaStream_t st);

// Tensor-core Gram (tc_ops.cu): precision is ATK_TF32, ATK_BF16, ATK_BF16X3 or
// ATK_FP8E4M3.  Bounded waits report DEV_TIMEOUT through *status.
size_t tc_gram_scratch_bytes(const View& v, int precision);
int tc_gram(const float* y, const View& v, int precision, double* S, float* scratch, size_t scratch_bytes,
            int* status, cudaStream_t st);
// max_c |Y(c, i)| for every mode-n index i (bits of the non-negative float,
// combined by atomicMax); rmax (n floats) must be zero on entry.
int tc_rowmax(const float* y, const View& v, float* rmax, cudaStream_t st);
// Fused ALS sweep (als_fused.cu): A = Y (Y^T Lt) (n x R float64) in one pass
// over Y for I_n <= 256 and R <= 32; Rk (nullable) receives Y^T Lt in the
// (lo, R, hi) layout.
bool als_fused_ok(const View& v, int64_t R);
size_t als_fused_scratch_bytes(const View& v, int64_t R);
int als_fused(const float* y, const View& v, const float* Lt, int64_t R, double* A, float* Rk, float* scratch,
              size_t scratch_bytes, cudaStream_t st);

// Explicit matricization (matricize.cu): dst slab b (B x A) = transpose of
// src slab b (A x B), both column-major, b < count.
int permute_slabs(const float* src, int64_t A, int64_t B, int64_t count, float* dst, cudaStream_t st);

// Tensor-core TTM (tc_ttm.cu): out = Y x_n U^T in the (lo, R, hi) layout for
// the precision forms of tc_gram, R <= 128.  Bounded waits report DEV_TIMEOUT
// through *status.
size_t tc_ttm_scratch_bytes(const View& v, int64_t R, int precision);
int tc_ttm(const float* y, const View& v, const float* U, int64_t R, int precision, float* out, char* scratch,
           size_t scratch_bytes, int* status, cudaStream_t st);

// Size limits of EIG modes: the full Jacobi eigensolver works on I_n <= 1024;
// the subspace eigensolver (R_n + p <= I_n / 2) on I_n <= EIG_MAX_N.
constexpr int64_t JACOBI_MAX_N = 1024;
constexpr int64_t EIG_MAX_N = 32768;

// Jacobi eigensolver (jacobi.cu).
size_t eig_scratch_bytes(int64_t n, int arith);
// method: ATK_EIG_AUTO (Rayleigh-Ritz when R + p <= n/2, else full Jacobi),
// ATK_EIG_FULL_JACOBI, ATK_EIG_SUBSPACE.
// With `unresolved` given, a level-0 cut that float32 arithmetic on S does
// not resolve sets *unresolved = 1 and returns at once (the caller recomputes
// S more precisely and calls again); otherwise the deflation levels run.
int eig_top(const double* S, int64_t n, int64_t R, int arith, int method, int max_sweeps, float* U_out,
            double* U64_out, double* lambda_out, double* discarded_out, int* dev_status, char* scratch,
            size_t scratch_bytes, cudaStream_t st, int* unresolved = nullptr);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (never
// lowers it; thread-safe).  Call outside stream capture.
int raise_smem_limit(const void* fn, size_t bytes);
// All eigenpairs of a small symmetric matrix on one CTA, float32
// (tridiag_eig.cu): S n x n float64, 1 <= n <= 160; diag_out (n) ascending,
// V_out n x n row-major with column j the eigenvector of diag_out[j].
// tridiag_eig_prepare() sets the kernel's shared-memory limit for every n
// (call it before capturing a launch into a graph).
int tridiag_eig_prepare();
int tridiag_eig_f32(const double* S, int n, float* diag_out, float* V_out, cudaStream_t st);
// Mout (m x m column-major, upper triangular) = L^{-T} for L L^T = G + shift
// max(diag G) I, G m x m float64, 1 <= m <= 160 (cholinv.cu).  A pivot at or
// below 1e-12 max(diag G) is raised to that floor and sets *breakdown
// (nullable).
int cholinv_f32(const double* G, int m, float shift, float* Mout, int* breakdown, cudaStream_t st);

// Float64 small dense linear algebra (smallla.cu).
size_t smallla_scratch_bytes(int64_t n, int64_t R);
// G (R x R) = A^T B, A and B n x R float64.
int gemm_tn_f64(const double* A, const double* B, int64_t n, int64_t R, double* G, cudaStream_t st);
// In place: X (m x R) <- X G^{-1}, G symmetric positive definite (R x R).
int solve_spd_right_f64(double* X, int64_t m, int64_t R, const double* G, double* chol_scratch,
                        int* dev_status, cudaStream_t st);
// One Newton-Schulz polar step in float64: U <- U (3I - U^T U) / 2.
int polar_step_f64(double* U, int64_t n, int64_t R, double* scratch, cudaStream_t st);
// One Gram-Schmidt-ordered orthonormalisation step in float64: U <- U T with
// U^T U = I + E and T = I - strict_upper(E) - diag(E) / 2; quadratic like the
// polar step, but column i only ever receives columns j < i.
int gs_step_f64(double* U, int64_t n, int64_t R, double* scratch, cudaStream_t st);
// CholeskyQR2 in float64: L (n x R) = Q R^, Q overwrites L, R^ (R x R) upper, diag > 0.
int cholqr2_f64(double* L, int64_t n, int64_t R, double* Rhat, double* scratch, int* dev_status,
                cudaStream_t st);
// C (m x p) = A (m x k) B (k x p), column-major float64 (C overlaps neither
// A nor B); split over k so that small outputs still cover the chip, the
// splits summed in a fixed order inside the launch.
int gemm_f64(const double* A, const double* B, int64_t m, int64_t k, int64_t p, double* C, cudaStream_t st);
int f64_to_f32(const double* src, float* dst, int64_t count, cudaStream_t st);
int f32_to_f64(const float* src, double* dst, int64_t count, cudaStream_t st);
// Square of the Frobenius norm of a float32 tensor, accumulated in float64.
// Needs NORM_SCRATCH_BYTES of scratch.
constexpr size_t NORM_SCRATCH_BYTES = 1184 * 8 + 256;
int norm2_f32(const float* x, int64_t count, double* out, double* scratch, cudaStream_t st);
// dst (R x R float32) = transpose of src (R x R float64).
int transpose_f64_to_f32(const double* src, int64_t R, float* dst, cudaStream_t st);

}  // namespace atk
