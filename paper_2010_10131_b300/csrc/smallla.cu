// Float64 small dense linear algebra for the factor matrices (I_n x R_n) and
// the R_n x R_n systems of Alg. 3: Gram products A^T B, Cholesky with the
// triangular inverse, right-multiplication, the Newton-Schulz polar step, and
// CholeskyQR2.
//
// On B300, float64 runs at about 1/60 of the float32 rate, and one SM manages
// only about 8 GFLOP/s.  So the products take float64 operands and results
// but compute in float-float on the float32 pipe, spread over many CTAs;
// only the O(R^3) factorisations run in float64 on a single CTA.
#include <cooperative_groups.h>

#include <algorithm>

#include "atk_internal.cuh"

namespace atk {

// ------------------------------------------------------------ tiled DGEMM
// C (m x p) = op(A) (m x k) op(B) (k x p), column-major float64 in and out;
// op(A) = A (lda >= m) or A^T (A stored k x m, lda >= k), likewise op(B).
//
// B300 issues about two float64 FMAs per clock per SM against 128 float32
// lanes, so the products run in float-float arithmetic on the float32 pipe:
// each operand is split into hi = fl32(x) and lo = fl32(x - hi) as it is
// staged (48 significant bits), each term a*b is formed as the float32 product
// of the high parts plus its exact rounding error (an FMA) and the two cross
// terms, and the running sum is a (hi, lo) pair updated by TwoSum (Knuth,
// TAOCP vol. 2, 4.2.2).  The omitted lo*lo term and the float32 rounding of
// the low-order sum leave a relative error near k * 2^-48 of the largest
// partial sum.  The intrinsics keep the compiler from contracting the
// TwoSum steps into FMAs, which would break them.
//
// A CTA of 256 threads computes a 32 x 32 tile, 2 x 2 values per thread,
// through 16-deep k tiles staged in shared memory (double-buffered).  With
// splits > 1 the splits of k for one tile form a thread-block cluster: each
// CTA leaves its float64 partial tile in its shared memory, and after a
// cluster barrier every CTA sums a share of the tile's elements over the
// splits in rank order (a fixed order) through distributed shared memory.
constexpr int DG_T = 32, DG_K = 16, DG_THREADS = 256, DG_MAXSPLIT = 8;

struct FF {
  float hi, lo;
};
// x = hi + lo: hi is x with its significand cut to the leading 24 bits and
// lo the remaining 29-bit integer of the significand, rounded to 24 bits and
// scaled by the exact power of two 2^(e - 1075) (e the biased exponent), so
// hi + lo = x to 2^-48 relative.  Both come from the bit pattern on the
// integer and float32 pipes: float64 conversions and arithmetic would run on
// B300's float64 pipe, about two per clock per SM, and every CTA splits its
// whole share of both operands.  Outside 949 <= e <= 1150 (|x| < 2^-74, where
// lo leaves float32's normal range, or |x| >= 2^128) the float64 conversions.
__device__ __forceinline__ FF ff_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7FF;
  if ((unsigned)(e - 949) <= 201u) {
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((unsigned)(b >> 29) & 0x7FFFFFu));
    const float scale = __uint_as_float(sign | ((unsigned)(e - 948) << 23));  // +-2^(e - 1075)
    return {hi, __uint2float_rn((unsigned)b & 0x1FFFFFFFu) * scale};
  }
  if ((b << 1) == 0) return {0.f, 0.f};  // +-0
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
// (sh, sl) += a * b for float-float a, b.
__device__ __forceinline__ void ff_fma(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// BX transforms op(B) = G (k x p, k = p) as it is staged, so the coefficient
// matrix of an orthonormalisation step never goes through memory:
//  - DG_POLAR: M = (3I - G) / 2, the Newton-Schulz polar coefficient.
//  - DG_GS: with G = U^T U = I + E, M = I - strict_upper(E) - diag(E) / 2
//    (upper triangular).  U M has column i built from columns j <= i only,
//    and (U M)^T (U M) = I + O(E^2): one step of an iteration that converges
//    quadratically like Newton-Schulz but, like Gram-Schmidt, never mixes a
//    later column into an earlier one.
enum { DG_PLAIN = 0, DG_POLAR = 1, DG_GS = 2 };
template <int BX>
__device__ __forceinline__ double dg_bx(double g, int64_t i, int64_t j) {
  if (BX == DG_POLAR) return (i == j ? 1.5 : 0.0) - 0.5 * g;
  if (BX == DG_GS) return i == j ? 1.0 - 0.5 * (g - 1.0) : (i < j ? -g : 0.0);
  return g;
}

template <bool TA, bool TB, int BX = DG_PLAIN>
__global__ void __launch_bounds__(DG_THREADS) dgemm_kernel(const double* __restrict__ A, int64_t lda,
                                                          const double* __restrict__ B, int64_t ldb, int64_t m,
                                                          int64_t k, int64_t p, int64_t kc, double* __restrict__ C,
                                                          int64_t ldc) {
  __shared__ float Ah[2][DG_K][DG_T + 1], Al[2][DG_K][DG_T + 1];
  __shared__ float Bh[2][DG_K][DG_T + 1], Bl[2][DG_K][DG_T + 1];
  __shared__ double ptile[DG_T * DG_T];  // this split's partial tile, column-major
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int64_t i0 = (int64_t)blockIdx.x * DG_T, c0 = (int64_t)blockIdx.y * DG_T;
  const int64_t kb = (int64_t)blockIdx.z * kc, ke = min(k, kb + kc);
  float sh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, sl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  double ra[2], rb[2];
  // Element e of this thread's share of a staged tile: (row ii, depth kk) of
  // op(A) and (depth kb2, column cc) of op(B); the fastest index follows the
  // operand's contiguous dimension so the global loads coalesce.
  auto a_at = [&](int e, int& ii, int& kk) {
    if (!TA) { ii = t % 32; kk = t / 32 + 8 * e; } else { kk = t % 16; ii = t / 16 + 16 * e; }
  };
  auto b_at = [&](int e, int& kb2, int& cc) {
    if (!TB) { kb2 = t % 16; cc = t / 16 + 16 * e; } else { cc = t % 32; kb2 = t / 32 + 8 * e; }
  };
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int ii, kk, kb2, cc;
      a_at(e, ii, kk);
      b_at(e, kb2, cc);
      const int64_t gi = i0 + ii, gk = k0 + kk, gc = c0 + cc, gk2 = k0 + kb2;
      ra[e] = (gi < m && gk < ke) ? (TA ? A[gk + lda * gi] : A[gi + lda * gk]) : 0.0;
      rb[e] = (gc < p && gk2 < ke) ? dg_bx<BX>(TB ? B[gc + ldb * gk2] : B[gk2 + ldb * gc], gk2, gc) : 0.0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int ii, kk, kb2, cc;
      a_at(e, ii, kk);
      b_at(e, kb2, cc);
      const FF a = ff_split(ra[e]), b = ff_split(rb[e]);
      Ah[buf][kk][ii] = a.hi;
      Al[buf][kk][ii] = a.lo;
      Bh[buf][kb2][cc] = b.hi;
      Bl[buf][kb2][cc] = b.lo;
    }
  };
  const int64_t ntile = kb < ke ? (ke - kb + DG_K - 1) / DG_K : 0;
  if (ntile > 0) {
    fetch(kb);
    store(0);
    __syncthreads();
    for (int64_t tt = 0; tt < ntile; ++tt) {
      const int buf = tt & 1;
      if (tt + 1 < ntile) fetch(kb + (tt + 1) * DG_K);
#pragma unroll 4
      for (int kk = 0; kk < DG_K; ++kk) {
        const float ah0 = Ah[buf][kk][ty], ah1 = Ah[buf][kk][ty + 16];
        const float al0 = Al[buf][kk][ty], al1 = Al[buf][kk][ty + 16];
        const float bh0 = Bh[buf][kk][tx], bh1 = Bh[buf][kk][tx + 16];
        const float bl0 = Bl[buf][kk][tx], bl1 = Bl[buf][kk][tx + 16];
        ff_fma(ah0, al0, bh0, bl0, sh[0][0], sl[0][0]);
        ff_fma(ah0, al0, bh1, bl1, sh[0][1], sl[0][1]);
        ff_fma(ah1, al1, bh0, bl0, sh[1][0], sl[1][0]);
        ff_fma(ah1, al1, bh1, bl1, sh[1][1], sl[1][1]);
      }
      if (tt + 1 < ntile) store(buf ^ 1);
      __syncthreads();
    }
  }
  const int splits = (int)gridDim.z;
  if (splits == 1) {
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        const int64_t gi = i0 + ty + 16 * u, gc = c0 + tx + 16 * v;
        if (gi < m && gc < p) C[gi + ldc * gc] = (double)sh[u][v] + (double)sl[u][v];
      }
    return;
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) ptile[(ty + 16 * u) + DG_T * (tx + 16 * v)] = (double)sh[u][v] + (double)sl[u][v];
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();  // every split's partial tile is written
  for (int e = (int)cl.block_rank() * DG_THREADS + t; e < DG_T * DG_T; e += splits * DG_THREADS) {
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += cl.map_shared_rank(ptile, sp)[e];
    const int64_t gi = i0 + e % DG_T, gc = c0 + e / DG_T;
    if (gi < m && gc < p) C[gi + ldc * gc] = s;
  }
  cl.sync();  // the partial tiles stay in place until every CTA has read them
}

// op(A) op(B) with a split count for about two CTAs per SM (the grid has to
// cover the chip: the tiles are small), limited by the k tiles and by the
// cluster size (at most DG_MAXSPLIT splits, one cluster per output tile).
template <bool TA, bool TB, int BX = DG_PLAIN>
static int dgemm(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t m, int64_t k, int64_t p,
                 double* C, int64_t ldc, cudaStream_t st) {
  if (m <= 0 || p <= 0) return ATK_OK;
  const int64_t tiles = ceil_div(m, DG_T) * ceil_div(p, DG_T);
  int64_t splits = std::max<int64_t>(1, ceil_div(2 * (int64_t)num_sms(), tiles));
  splits = std::min<int64_t>({splits, std::max<int64_t>(1, ceil_div(k, DG_K)), (int64_t)DG_MAXSPLIT});
  const int64_t kc = ceil_div(ceil_div(std::max<int64_t>(k, 1), splits), DG_K) * DG_K;
  splits = std::max<int64_t>(1, ceil_div(std::max<int64_t>(k, 1), kc));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ceil_div(m, DG_T), (unsigned)ceil_div(p, DG_T), (unsigned)splits);
  cfg.blockDim = dim3(DG_THREADS);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = (unsigned)splits;
  cfg.attrs = attr;
  cfg.numAttrs = splits > 1 ? 1 : 0;
  ATK_CUDA(cudaLaunchKernelEx(&cfg, dgemm_kernel<TA, TB, BX>, A, lda, B, ldb, m, k, p, kc, C, ldc));
  ATK_LAUNCHED();
  return ATK_OK;
}

size_t smallla_scratch_bytes(int64_t n, int64_t R) {
  // four R x R matrices + an n x R panel, plus alignment slack
  return sizeof(double) * (size_t)(4 * R * R + 2 * n * R) + 4096;
}

int gemm_tn_f64(const double* A, const double* B, int64_t n, int64_t R, double* G, cudaStream_t st) {
  if (n == 0) {
    ATK_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * R * R, st));
    return ATK_OK;
  }
  // G = A^T B, split over the n rows.
  return dgemm<true, false>(A, n, B, n, R, n, R, G, R, st);
}

// One CTA: Cholesky G = C C^T (C lower) and Cinv = C^{-1} (lower), R <= 128,
// float64 (Golub & Van Loan, Matrix Computations, Alg. 4.2.2 for the
// factor; forward substitution on the identity for the inverse, both
// right-looking and in the same loop).  Both live in one shared-memory
// R x (R + 1) array: C on and below the diagonal, the strictly lower part of
// Cinv transposed into the upper part, the diagonals in two vectors.  One
// barrier per column (the loop's comment gives the steps): the float64 pipe,
// not barriers, then bounds the kernel (about R^3 / 3 float64 FMAs).  A
// non-positive pivot sets DEV_CHOL and leaves identity factors, so later
// kernels stay finite.
constexpr int CI_THREADS = 512;
size_t chol_inv_smem(int R) { return sizeof(double) * ((size_t)R * (R + 1) + 2 * (size_t)R) + 16; }

__global__ void __launch_bounds__(CI_THREADS) chol_inv_kernel(const double* __restrict__ G, int R,
                                                              double* __restrict__ C, double* __restrict__ Cinv,
                                                              int* __restrict__ status) {
  extern __shared__ double cm[];
  const int ld = R + 1;
  double* M = cm;                 // R x ld, row-major: M[i * ld + j]
  double* dC = cm + (size_t)R * ld;  // diagonal of C
  double* dX = dC + R;               // diagonal of Cinv
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int idx = tid; idx < R * R; idx += CI_THREADS) {
    const int i = idx % R, j = idx / R;
    if (i >= j) M[i * ld + j] = G[i + (int64_t)R * j];
  }
  __shared__ double pinv[2];
  // One barrier per column j.  Pivot d_j = sqrt(M_jj) is known from the step
  // before; the step then, with L_ij = M_ij / d_j formed on the fly:
  //  - applies the rank-1 update of the Cholesky factorisation to the
  //    trailing lower triangle, M_ik -= L_ij L_kj (i >= k > j);
  //  - eliminates column j from the rows below of the inverse, by forward
  //    substitution run right-looking on the identity: with Xu the rows not
  //    yet divided by their pivot (Xu_jj = 1), X_j = Xu_j / d_j and
  //    Xu_ic -= L_ij X_jc for i > j, c <= j;
  //  - the thread that owns (j + 1, j + 1) finishes that entry first and takes
  //    the next pivot (square root and reciprocal on one thread: float64
  //    division and square root are long instruction sequences on B300's
  //    float64 pipe).
  // After the barrier, column j of L and row j of X are divided by d_j in
  // place (nothing in step j + 1 reads them).  X is stored transposed in the
  // strict upper triangle of M (X_ic at M[c][i]), its diagonal 1 / d_j in dX.
  auto take_pivot = [&](int j, double piv) {
    if (!(piv > 0.0)) {
      bad = 1;
      piv = 1.0;
    }
    const double d = sqrt(piv);
    dC[j] = d;
    dX[j] = 1.0 / d;
    pinv[j & 1] = dX[j];
  };
  if (tid == 0) take_pivot(0, M[0]);
  __syncthreads();
  for (int j = 0; j < R; ++j) {
    const double inv = pinv[j & 1];
    const int rem = R - j - 1;
    const int tri = rem * (rem + 1) / 2;     // trailing Cholesky entries
    const int total = tri + rem * (j + 1);   // and inverse entries
    // work item 0 is (j + 1, j + 1): thread 0 takes the next pivot
    for (int idx = tid; idx < total; idx += CI_THREADS) {
      if (idx < tri) {
        // idx -> (a, b), 0 <= b <= a < rem, row by row
        int a = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
        while (a * (a + 1) / 2 > idx) --a;
        while ((a + 1) * (a + 2) / 2 <= idx) ++a;
        const int b = idx - a * (a + 1) / 2;
        const int i = j + 1 + a, k = j + 1 + b;
        const double v = M[i * ld + k] - (M[i * ld + j] * inv) * (M[k * ld + j] * inv);
        M[i * ld + k] = v;
        if (idx == 0) take_pivot(j + 1, v);  // (j + 1, j + 1) is final now
      } else {
        const int q = idx - tri;
        const int i = j + 1 + q / (j + 1), c = q % (j + 1);
        const double xj = c == j ? inv : M[c * ld + j] * inv;  // X_jc = Xu_jc / d_j (Xu_jj = 1)
        const double lij = M[i * ld + j] * inv;
        M[c * ld + i] = (c == j ? 0.0 : M[c * ld + i]) - lij * xj;
      }
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < R; i += CI_THREADS) M[i * ld + j] *= inv;  // L column j
    for (int c = tid; c < j; c += CI_THREADS) M[c * ld + j] *= inv;          // X row j
  }
  __syncthreads();
  if (bad) {
    for (int idx = tid; idx < R * R; idx += CI_THREADS) {
      const double e = (idx % R == idx / R) ? 1.0 : 0.0;
      C[idx] = e;
      Cinv[idx] = e;
    }
    if (tid == 0) atomicOr(status, DEV_CHOL);
    return;
  }
  for (int idx = tid; idx < R * R; idx += CI_THREADS) {
    const int i = idx % R, j = idx / R;  // column-major outputs
    C[idx] = i > j ? M[i * ld + j] : (i == j ? dC[i] : 0.0);
    Cinv[idx] = i > j ? M[j * ld + i] : (i == j ? dX[i] : 0.0);
  }
}

static int launch_chol_inv(const double* G, int R, double* C, double* Cinv, int* status, cudaStream_t st) {
  if (R < 1 || R > 128) { set_error("chol_inv: need 1 <= R <= 128"); return ATK_EUNSUPPORTED; }
  static const bool attr = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)chol_inv_smem(128)) == cudaSuccess;
  if (!attr) { set_error("chol_inv: cannot set the kernel's shared-memory size"); return ATK_ECUDA; }
  chol_inv_kernel<<<1, CI_THREADS, chol_inv_smem(R), st>>>(G, R, C, Cinv, status);
  ATK_LAUNCHED();
  return ATK_OK;
}

int gemm_f64(const double* A, const double* B, int64_t m, int64_t k, int64_t p, double* C, cudaStream_t st) {
  return dgemm<false, false>(A, m, B, k, m, k, p, C, m, st);
}

// Rhat = C2^T C1^T (both factors lower), i.e. the product of the two upper factors.
__global__ void rhat_kernel(const double* __restrict__ C1, const double* __restrict__ C2, int64_t R,
                            double* __restrict__ Rhat) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= R * R) return;
  int64_t i = o % R, k = o / R;
  double s = 0.0;
  for (int64_t t = 0; t < R; ++t) s += C2[t + R * i] * C1[k + R * t];
  Rhat[o] = (i <= k) ? s : 0.0;
}

namespace {
struct SmallBufs {
  double *M1, *M2, *M3, *M4, *panel;
};
SmallBufs carve(double* scratch, int64_t n, int64_t R) {
  Arena ar{(char*)scratch, smallla_scratch_bytes(n, R), 0};
  SmallBufs b;
  b.M1 = (double*)ar.take(sizeof(double) * R * R);
  b.M2 = (double*)ar.take(sizeof(double) * R * R);
  b.M3 = (double*)ar.take(sizeof(double) * R * R);
  b.M4 = (double*)ar.take(sizeof(double) * R * R);
  b.panel = (double*)ar.take(sizeof(double) * n * R);
  return b;
}
}  // namespace

// X <- X G^{-1} = (X C^{-T}) C^{-1} with G = C C^T: two products with the
// triangular inverse, no explicit G^{-1}.
int solve_spd_right_f64(double* X, int64_t m, int64_t R, const double* G, double* scratch, int* dev_status,
                        cudaStream_t st) {
  SmallBufs b = carve(scratch, m, R);
  if (!b.panel) { set_error("solve_spd: scratch too small"); return ATK_EINVAL; }
  ATK_TRY(launch_chol_inv(G, (int)R, b.M1, b.M2, dev_status, st));
  ATK_TRY((dgemm<false, true>(X, m, b.M2, R, m, R, R, b.panel, m, st)));
  ATK_TRY((dgemm<false, false>(b.panel, m, b.M2, R, m, R, R, X, m, st)));
  return ATK_OK;
}

int polar_step_f64(double* U, int64_t n, int64_t R, double* scratch, cudaStream_t st) {
  SmallBufs b = carve(scratch, n, R);
  if (!b.panel) { set_error("polar: scratch too small"); return ATK_EINVAL; }
  ATK_TRY(gemm_tn_f64(U, U, n, R, b.M1, st));
  ATK_TRY((dgemm<false, false, DG_POLAR>(U, n, b.M1, R, n, R, R, b.panel, n, st)));
  ATK_CUDA(cudaMemcpyAsync(U, b.panel, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, st));
  return ATK_OK;
}

int gs_step_f64(double* U, int64_t n, int64_t R, double* scratch, cudaStream_t st) {
  SmallBufs b = carve(scratch, n, R);
  if (!b.panel) { set_error("gs_step: scratch too small"); return ATK_EINVAL; }
  ATK_TRY(gemm_tn_f64(U, U, n, R, b.M1, st));
  ATK_TRY((dgemm<false, false, DG_GS>(U, n, b.M1, R, n, R, R, b.panel, n, st)));
  ATK_CUDA(cudaMemcpyAsync(U, b.panel, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, st));
  return ATK_OK;
}

int cholqr2_f64(double* L, int64_t n, int64_t R, double* Rhat, double* scratch, int* dev_status, cudaStream_t st) {
  SmallBufs b = carve(scratch, n, R);
  if (!b.panel) { set_error("cholqr2: scratch too small"); return ATK_EINVAL; }
  // Pass 1: L^T L = C1 C1^T, Q1 = L C1^{-T}.
  ATK_TRY(gemm_tn_f64(L, L, n, R, b.M1, st));
  ATK_TRY(launch_chol_inv(b.M1, (int)R, b.M2, b.M3, dev_status, st));
  ATK_TRY((dgemm<false, true>(L, n, b.M3, R, n, R, R, b.panel, n, st)));
  // Pass 2 on Q1: Q1^T Q1 = C2 C2^T, Q = Q1 C2^{-T}.
  ATK_TRY(gemm_tn_f64(b.panel, b.panel, n, R, b.M1, st));
  ATK_TRY(launch_chol_inv(b.M1, (int)R, b.M4, b.M3, dev_status, st));
  ATK_TRY((dgemm<false, true>(b.panel, n, b.M3, R, n, R, R, L, n, st)));
  rhat_kernel<<<(unsigned)ceil_div(R * R, 256), 256, 0, st>>>(b.M2, b.M4, R, Rhat);
  ATK_LAUNCHED();
  return ATK_OK;
}

__global__ void f64_to_f32_kernel(const double* __restrict__ s, float* __restrict__ d, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) d[i] = (float)s[i];
}
__global__ void f32_to_f64_kernel(const float* __restrict__ s, double* __restrict__ d, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) d[i] = (double)s[i];
}
__global__ void transpose_kernel(const double* __restrict__ s, int64_t R, float* __restrict__ d) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= R * R) return;
  int64_t i = o % R, k = o / R;
  d[o] = (float)s[k + R * i];
}

int f64_to_f32(const double* src, float* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return ATK_OK;
  f64_to_f32_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(src, dst, count);
  ATK_LAUNCHED();
  return ATK_OK;
}
int f32_to_f64(const float* src, double* dst, int64_t count, cudaStream_t st) {
  if (count <= 0) return ATK_OK;
  f32_to_f64_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, st>>>(src, dst, count);
  ATK_LAUNCHED();
  return ATK_OK;
}
int transpose_f64_to_f32(const double* src, int64_t R, float* dst, cudaStream_t st) {
  transpose_kernel<<<(unsigned)ceil_div(R * R, 256), 256, 0, st>>>(src, R, dst);
  ATK_LAUNCHED();
  return ATK_OK;
}

// ||x||^2 in float64: per-CTA partial sums, then one CTA sums them in order.
constexpr int NORM_CTAS = 1184;
__global__ void norm2_part_kernel(const float* __restrict__ x, int64_t count, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    double v = x[i];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void norm2_final_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}
int norm2_f32(const float* x, int64_t count, double* out, double* scratch, cudaStream_t st) {
  int ctas = (int)std::min<int64_t>(NORM_CTAS, std::max<int64_t>(1, ceil_div(count, 256)));
  norm2_part_kernel<<<ctas, 256, 0, st>>>(x, count, scratch);
  ATK_LAUNCHED();
  norm2_final_kernel<<<1, 256, 0, st>>>(scratch, ctas, out);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
