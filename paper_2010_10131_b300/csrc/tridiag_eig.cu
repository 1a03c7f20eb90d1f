// Eigen-decomposition of a small dense symmetric matrix on one CTA, float32:
// the Rayleigh-Ritz projections of the subspace eigensolver (m = R + p <= 156)
// need all their eigenpairs, and a one-CTA Jacobi spends about 80 rounds x
// 10 sweeps of two barriers each on them.  Here the matrix is reduced to
// tridiagonal form and the tridiagonal problem is solved by methods whose
// steps are independent across eigenpairs:
//  1. Householder reduction A = Q T Q^T (Golub & Van Loan, Matrix
//     Computations, 4th ed., Alg. 8.3.1): step j reflects column j below the
//     diagonal with H_j = I - tau_j v_j v_j^T (v_j(0) = 1), p = tau A22 v,
//     w = p - (tau/2)(p^T v) v, A22 <- A22 - v w^T - w v^T.  Three barriers
//     per step; the reflectors stay in the columns they annihilate.
//  2. Eigenvalues of T by bisection on the Sturm count (ibid., Sec. 8.4.1):
//     thread t finds the t-th smallest eigenvalue.
//  3. Eigenvectors of T by inverse iteration (ibid., Sec. 8.2.2), thread t
//     for eigenvalue t: two solves of (T - lambda_t I) x = b by Gaussian
//     elimination without interchanges, pivots kept away from zero (the
//     classical guard of tridiagonal inverse iteration), from a
//     pseudo-random start; then, within each cluster of eigenvalues closer
//     than 1e-3 ||T||_1, modified Gram-Schmidt, so that near-equal
//     eigenvalues get an orthonormal basis of their eigenspace.
//  4. Back-transformation X <- H_0 H_1 ... H_{m-3} X, thread c for column c.
// The eigenvectors are as accurate as float32 allows (about eps ||T|| / gap);
// the float64 refinement that follows the subspace eigensolver polishes them.
#include "atk_internal.cuh"

namespace atk {

constexpr int TE_THREADS = 512;
constexpr int TE_NMAX = 160;  // largest matrix (the subspace eigensolver uses m <= 156)
constexpr int TE_BISECT = 40;  // bisection steps: float32 resolution from the Gershgorin interval

size_t tridiag_eig_smem(int n) {
  const int ld = n + 1;
  return sizeof(float) * ((size_t)2 * n * ld + 6 * (size_t)n + 8);
}

// Sturm count: the number of eigenvalues of T (diagonal d, squared
// off-diagonal e2) below x, from the signs of the pivots of T - x I.
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int n, float x, float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

__device__ __forceinline__ float te_rand(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return (float)(h & 0xFFFFFF) * (2.f / 16777216.f) - 1.f;
}

// S: n x n float64 (symmetric).  diag_out (n): eigenvalues, ascending.
// V_out (n x n, row-major, column j = eigenvector of diag_out[j]).
__global__ void __launch_bounds__(TE_THREADS) tridiag_eig_kernel(const double* __restrict__ S, int n,
                                                                  float* __restrict__ diag_out,
                                                                  float* __restrict__ V_out) {
  extern __shared__ __align__(16) float tsm[];
  const int ld = n + 1;
  float* A = tsm;             // n x ld, row-major; reflector j in column j below the diagonal
  float* X = A + n * ld;      // n x ld, row-major; column t = eigenvector t
  float* d = X + n * ld;      // diagonal of T
  float* e = d + n;           // off-diagonal of T: e[j] = T(j+1, j)
  float* e2 = e + n;          // e^2
  float* tau = e2 + n;        // reflector scalars
  float* p = tau + n;         // work vector (p of step j, indexed from j+1)
  float* lam = p + n;         // eigenvalues, ascending
  __shared__ float red[2];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  constexpr int NW = TE_THREADS / 32;
  for (int idx = tid; idx < n * n; idx += TE_THREADS) A[(idx / n) * ld + idx % n] = (float)S[idx];
  __syncthreads();

  // 1. Householder reduction to tridiagonal form.
  for (int j = 0; j + 2 < n; ++j) {
    const int nx = n - j - 1;
    if (warp == 0) {
      const float alpha = A[(j + 1) * ld + j];
      float sig = 0.f;
      for (int i = j + 2 + lane; i < n; i += 32) sig = fmaf(A[i * ld + j], A[i * ld + j], sig);
      for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
      float t = 0.f, beta = alpha, scale = 0.f;
      if (sig > 0.f) {
        const float mu = sqrtf(fmaf(alpha, alpha, sig));
        beta = alpha <= 0.f ? mu : -mu;
        t = (beta - alpha) / beta;
        scale = 1.f / (alpha - beta);
      }
      for (int i = j + 2 + lane; i < n; i += 32) A[i * ld + j] *= scale;
      if (lane == 0) {
        A[(j + 1) * ld + j] = 1.f;
        e[j] = beta;
        tau[j] = t;
      }
    }
    __syncthreads();
    const float t = tau[j];
    if (t == 0.f) continue;  // already reduced (uniform across the CTA)
    // p = tau A22 v: four lanes per row, shuffled together.
    {
      const int sub = tid % 4;
      const unsigned gmask = 0xFu << (lane & ~3);
      for (int i = j + 1 + tid / 4; i < n; i += TE_THREADS / 4) {
        float s0 = 0.f, s1 = 0.f;
        int k = j + 1 + sub;
        for (; k + 4 < n; k += 8) {
          s0 = fmaf(A[i * ld + k], A[k * ld + j], s0);
          s1 = fmaf(A[i * ld + k + 4], A[(k + 4) * ld + j], s1);
        }
        if (k < n) s0 = fmaf(A[i * ld + k], A[k * ld + j], s0);
        float s = s0 + s1;
        s += __shfl_xor_sync(gmask, s, 1);
        s += __shfl_xor_sync(gmask, s, 2);
        if (sub == 0) p[i] = t * s;
      }
    }
    __syncthreads();
    // K = (tau/2) p^T v, computed by every warp; then the rank-2 update.
    float kk = 0.f;
    for (int k = j + 1 + lane; k < n; k += 32) kk = fmaf(p[k], A[k * ld + j], kk);
    for (int o = 16; o > 0; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
    kk *= 0.5f * t;
    for (int i = j + 1 + warp; i < n; i += NW) {
      const float vi = A[i * ld + j], wi = fmaf(-kk, vi, p[i]);
      for (int k = j + 1 + lane; k < n; k += 32) {
        const float vk = A[k * ld + j], wk = fmaf(-kk, vk, p[k]);
        A[i * ld + k] = fmaf(-vi, wk, fmaf(-wi, vk, A[i * ld + k]));
      }
    }
    __syncthreads();
    (void)nx;
  }
  for (int i = tid; i < n; i += TE_THREADS) d[i] = A[i * ld + i];
  if (tid == 0 && n >= 2) e[n - 2] = A[(n - 1) * ld + (n - 2)];
  __syncthreads();
  for (int i = tid; i + 1 < n; i += TE_THREADS) e2[i] = e[i] * e[i];
  // Gershgorin interval and the one-norm of T (warp 0).
  if (warp == 0) {
    float lo = INFINITY, hi = -INFINITY, nrm = 0.f;
    for (int i = lane; i < n; i += 32) {
      const float r = (i > 0 ? fabsf(e[i - 1]) : 0.f) + (i + 1 < n ? fabsf(e[i]) : 0.f);
      lo = fminf(lo, d[i] - r);
      hi = fmaxf(hi, d[i] + r);
      nrm = fmaxf(nrm, fabsf(d[i]) + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      nrm = fmaxf(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
    }
    if (lane == 0) {
      const float pad = 2.f * 1.1920929e-7f * nrm + 1e-30f;
      red[0] = lo - pad;
      red[1] = hi + pad;
      p[0] = nrm;  // p is free again: keep ||T||_1 there
    }
  }
  __syncthreads();
  const float nrm = p[0];
  const float pivmin = 1e-30f * fmaxf(1.f, nrm * nrm);

  // 2. Bisection: thread t brackets the t-th smallest eigenvalue.
  for (int t = tid; t < n; t += TE_THREADS) {
    float a = red[0], b = red[1];
    for (int it = 0; it < TE_BISECT; ++it) {
      const float mid = 0.5f * (a + b);
      if (mid <= a || mid >= b) break;
      if (sturm_count(d, e2, n, mid, pivmin) > t) b = mid;
      else a = mid;
    }
    lam[t] = 0.5f * (a + b);
  }
  __syncthreads();

  // 3. Inverse iteration, thread t for eigenvalue t; the solution goes to
  // column t of X.  Elimination of T - lambda I: pivots q_i, multipliers
  // m_i = e_i / q_i; the right-hand side is eliminated alongside.
  const float guard = 1.1920929e-7f * nrm + 1e-30f;
  for (int t = tid; t < n; t += TE_THREADS) {
    const float lm = lam[t];
    float q[TE_NMAX];
    for (int i = 0; i < n; ++i) X[i * ld + t] = te_rand((uint32_t)t, (uint32_t)i);
    for (int iter = 0; iter < 2; ++iter) {
      float qi = d[0] - lm;
      if (fabsf(qi) < guard) qi = qi < 0.f ? -guard : guard;
      q[0] = qi;
      float y = X[t];
      for (int i = 1; i < n; ++i) {
        const float mlt = e[i - 1] / q[i - 1];
        qi = d[i] - lm - mlt * e[i - 1];
        if (fabsf(qi) < guard) qi = qi < 0.f ? -guard : guard;
        q[i] = qi;
        y = X[i * ld + t] - mlt * y;
        X[i * ld + t] = y;
      }
      float x = X[(n - 1) * ld + t] / q[n - 1];
      X[(n - 1) * ld + t] = x;
      float ss = x * x;
      for (int i = n - 2; i >= 0; --i) {
        x = (X[i * ld + t] - e[i] * x) / q[i];
        X[i * ld + t] = x;
        ss = fmaf(x, x, ss);
      }
      const float inv = ss > 0.f && ss < INFINITY ? rsqrtf(ss) : 0.f;
      for (int i = 0; i < n; ++i) X[i * ld + t] *= inv;
    }
  }
  __syncthreads();
  // Modified Gram-Schmidt inside clusters (warp 0, lanes over the rows).
  if (warp == 0) {
    const float ortol = 1e-3f * nrm;
    int c0 = 0;
    for (int t = 1; t < n; ++t) {
      if (lam[t] - lam[t - 1] > ortol) {
        c0 = t;
        continue;
      }
      for (int s = c0; s < t; ++s) {
        float dot = 0.f;
        for (int i = lane; i < n; i += 32) dot = fmaf(X[i * ld + s], X[i * ld + t], dot);
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        for (int i = lane; i < n; i += 32) X[i * ld + t] = fmaf(-dot, X[i * ld + s], X[i * ld + t]);
        __syncwarp();
      }
      float ss = 0.f;
      for (int i = lane; i < n; i += 32) ss = fmaf(X[i * ld + t], X[i * ld + t], ss);
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float inv = ss > 0.f ? rsqrtf(ss) : 0.f;
      for (int i = lane; i < n; i += 32) X[i * ld + t] *= inv;
      __syncwarp();
    }
  }
  __syncthreads();

  // 4. Back-transformation, thread c for column c: apply H_{n-3}, ..., H_0.
  for (int c = tid; c < n; c += TE_THREADS) {
    for (int j = n - 3; j >= 0; --j) {
      const float t = tau[j];
      if (t == 0.f) continue;
      float s0 = 0.f, s1 = 0.f;
      int i = j + 1;
      for (; i + 1 < n; i += 2) {
        s0 = fmaf(A[i * ld + j], X[i * ld + c], s0);
        s1 = fmaf(A[(i + 1) * ld + j], X[(i + 1) * ld + c], s1);
      }
      if (i < n) s0 = fmaf(A[i * ld + j], X[i * ld + c], s0);
      const float f = t * (s0 + s1);
      for (int r = j + 1; r < n; ++r) X[r * ld + c] = fmaf(-f, A[r * ld + j], X[r * ld + c]);
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += TE_THREADS) diag_out[i] = lam[i];
  for (int idx = tid; idx < n * n; idx += TE_THREADS) V_out[idx] = X[(idx / n) * ld + idx % n];
}

int tridiag_eig_prepare() {
  return raise_smem_limit((const void*)tridiag_eig_kernel, tridiag_eig_smem(TE_NMAX));
}

int tridiag_eig_f32(const double* S, int n, float* diag_out, float* V_out, cudaStream_t st) {
  if (n < 1 || n > TE_NMAX) {
    set_error("tridiag_eig: need 1 <= n <= 160");
    return ATK_EUNSUPPORTED;
  }
  tridiag_eig_kernel<<<1, TE_THREADS, tridiag_eig_smem(n), st>>>(S, n, diag_out, V_out);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
