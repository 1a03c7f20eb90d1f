// Eigen-decomposition of a small dense symmetric matrix on one CTA, float32:
// the Rayleigh-Ritz projections of the subspace eigensolver (m = R + p <= 156)
// need all their eigenpairs, and a one-CTA Jacobi spends about 80 rounds x
// 10 sweeps of two barriers each on them.  Here the matrix is reduced to
// tridiagonal form and the tridiagonal problem is solved by methods whose
// steps are independent across eigenpairs:
//  1. Householder reduction A = Q T Q^T (Golub & Van Loan, Matrix
//     Computations, 4th ed., Alg. 8.3.1): step j reflects column j below the
//     diagonal with H_j = I - tau_j v_j v_j^T (v_j(0) = 1), p = tau A22 v,
//     w = p - (tau/2)(p^T v) v, A22 <- A22 - v w^T - w v^T.  Two barriers per
//     step: every thread derives the reflector of step j from the column's
//     first entry and the sixteen per-warp partial sums of its squared norm,
//     which the warps accumulate while they update that column in step j-1
//     (summed in warp order, so the result is deterministic).  Column j keeps
//     the unscaled x; v = x * scale_j below its leading 1.
//  2. Eigenvalues of T by multisection on the Sturm count (ibid., Sec. 8.4.1):
//     G lanes per eigenvalue (G = 8, 4 or 2 as n allows) test G points of the
//     bracket at once, down to an absolute width of 4 eps ||T||_1.
//  3. Eigenvectors of T by inverse iteration (ibid., Sec. 8.2.2), thread t
//     for eigenvalue t: Gaussian elimination of T - lambda_t I without
//     interchanges, pivots kept away from zero (the classical guard of
//     tridiagonal inverse iteration), then two solves from a pseudo-random
//     start with the same factors; within each cluster of eigenvalues closer
//     than 1e-3 ||T||_1, modified Gram-Schmidt, so that near-equal
//     eigenvalues get an orthonormal basis of their eigenspace.
//  4. Back-transformation X <- H_0 H_1 ... H_{m-3} X, two barriers per
//     reflector (the projections v^T X, then the rank-1 update).
// The eigenvectors are as accurate as float32 allows (about eps ||T|| / gap);
// the float64 refinement that follows the subspace eigensolver polishes them.
#include "atk_internal.cuh"

namespace atk {

constexpr int TE_THREADS = 512;
constexpr int TE_WARPS = TE_THREADS / 32;
constexpr int TE_NMAX = 160;     // largest matrix (the subspace eigensolver uses m <= 156)
constexpr int TE_KREG = 5;       // columns per lane held in registers in the update (32 * 5 >= TE_NMAX)
constexpr int TE_MAXSECT = 40;   // multisection steps (a cap; the width test ends them sooner)

size_t tridiag_eig_smem(int n) {
  const int ld = n + 1;
  return sizeof(float) * ((size_t)2 * n * ld + 8 * (size_t)n + 3 * TE_WARPS + 8);
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
  float* A = tsm;             // n x ld, row-major; column j keeps x_j below the diagonal
  float* X = A + n * ld;      // n x ld, row-major; column t = eigenvector t
  float* d = X + n * ld;      // diagonal of T
  float* e = d + n;           // off-diagonal of T: e[j] = T(j+1, j)
  float* e2 = e + n;          // e^2
  float* tau = e2 + n;        // reflector scalars
  float* scl = tau + n;       // v_j(i) = x_j(i) * scl[j] for i >= j+2
  float* p = scl + n;         // work vector
  float* lam = p + n;         // eigenvalues, ascending
  float* part = lam + n;      // [2][TE_WARPS] partial squared norms of the next column
  float* kpart = part + 2 * TE_WARPS;  // [TE_WARPS] partial sums of p^T v
  __shared__ float red[4];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  for (int idx = tid; idx < n * n; idx += TE_THREADS) A[(idx / n) * ld + idx % n] = (float)S[idx];
  __syncthreads();
  // Partial norms of column 0 below its first subdiagonal entry.
  {
    float sg = 0.f;
    for (int i = 2 + tid; i < n; i += TE_THREADS) sg = fmaf(A[i * ld], A[i * ld], sg);
    for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
    if (lane == 0) part[warp] = sg;
  }
  __syncthreads();

  // 1. Householder reduction to tridiagonal form.
  for (int j = 0; j + 2 < n; ++j) {
    const float* pj = part + (j & 1) * TE_WARPS;
    float sig = 0.f;
#pragma unroll
    for (int w = 0; w < TE_WARPS; ++w) sig += pj[w];
    const float alpha = A[(j + 1) * ld + j];
    float t = 0.f, beta = alpha, scale = 0.f;
    if (sig > 0.f) {
      const float mu = sqrtf(fmaf(alpha, alpha, sig));
      beta = alpha <= 0.f ? mu : -mu;
      t = __fdividef(beta - alpha, beta);
      scale = __fdividef(1.f, alpha - beta);
    }
    if (tid == 0) {
      e[j] = beta;
      tau[j] = t;
      scl[j] = scale;
    }
    float* pn = part + ((j + 1) & 1) * TE_WARPS;
    if (t == 0.f) {
      // Column j is already reduced: carry the next column's norm forward.
      float sg = 0.f;
      for (int i = j + 3 + tid; i < n; i += TE_THREADS) sg = fmaf(A[i * ld + j + 1], A[i * ld + j + 1], sg);
      for (int o = 16; o > 0; o >>= 1) sg += __shfl_xor_sync(0xffffffffu, sg, o);
      if (lane == 0) pn[warp] = sg;
      __syncthreads();
      continue;
    }
    // p = tau A22 v, four lanes per row; each warp also sums its p_i v_i.
    {
      float pv = 0.f;
      const int sub = tid % 4;
      const unsigned gmask = 0xFu << (lane & ~3);
      for (int i = j + 1 + tid / 4; i < n; i += TE_THREADS / 4) {
        // v(j+1) = 1; the entries k >= j+2 hold the unscaled x, so their sum
        // is scaled once at the end.
        float s0 = 0.f, s1 = 0.f, lead = 0.f;
        int k = j + 1 + sub;
        if (sub == 0) {
          lead = A[i * ld + k];
          k += 4;
        }
#pragma unroll 4
        for (; k + 4 < n; k += 8) {
          s0 = fmaf(A[i * ld + k], A[k * ld + j], s0);
          s1 = fmaf(A[i * ld + k + 4], A[(k + 4) * ld + j], s1);
        }
        if (k < n) s1 = fmaf(A[i * ld + k], A[k * ld + j], s1);
        float s = fmaf(scale, s0 + s1, lead);
        s += __shfl_xor_sync(gmask, s, 1);
        s += __shfl_xor_sync(gmask, s, 2);
        if (sub == 0) {
          p[i] = t * s;
          pv = fmaf(t * s, i == j + 1 ? 1.f : A[i * ld + j] * scale, pv);
        }
      }
      for (int o = 16; o > 0; o >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, o);
      if (lane == 0) kpart[warp] = pv;
    }
    __syncthreads();
    // K = (tau/2) p^T v from the per-warp partials (warp order); then
    // A22 -= v w^T + w v^T with w = p - K v, lane-owned columns held in
    // registers; the warps add up the squared norm of the updated column j+1
    // below row j+2.
    float kk = 0.f;
#pragma unroll
    for (int w = 0; w < TE_WARPS; ++w) kk += kpart[w];
    kk *= 0.5f * t;
    float vk[TE_KREG], wk[TE_KREG];
#pragma unroll
    for (int q = 0; q < TE_KREG; ++q) {
      const int k = j + 1 + lane + 32 * q;
      const float v = k < n ? (k == j + 1 ? 1.f : A[k * ld + j] * scale) : 0.f;
      vk[q] = v;
      wk[q] = k < n ? fmaf(-kk, v, p[k]) : 0.f;
    }
    float sg = 0.f;
    // Two rows per pass: all ten loads are issued before any store.
    for (int i0 = j + 1 + warp; i0 < n; i0 += 2 * TE_WARPS) {
      const int i1 = i0 + TE_WARPS;
      const bool has1 = i1 < n;
      const float vi0 = i0 == j + 1 ? 1.f : A[i0 * ld + j] * scale;
      const float wi0 = fmaf(-kk, vi0, p[i0]);
      const float vi1 = has1 ? A[i1 * ld + j] * scale : 0.f;
      const float wi1 = has1 ? fmaf(-kk, vi1, p[i1]) : 0.f;
      float a0[TE_KREG], a1[TE_KREG];
#pragma unroll
      for (int q = 0; q < TE_KREG; ++q) {
        const int k = j + 1 + lane + 32 * q;
        a0[q] = k < n ? A[i0 * ld + k] : 0.f;
        a1[q] = (k < n && has1) ? A[i1 * ld + k] : 0.f;
      }
#pragma unroll
      for (int q = 0; q < TE_KREG; ++q) {
        const int k = j + 1 + lane + 32 * q;
        if (k < n) {
          const float v0 = fmaf(-vi0, wk[q], fmaf(-wi0, vk[q], a0[q]));
          A[i0 * ld + k] = v0;
          if (q == 0 && lane == 0 && i0 >= j + 3) sg = fmaf(v0, v0, sg);
          if (has1) {
            const float v1 = fmaf(-vi1, wk[q], fmaf(-wi1, vk[q], a1[q]));
            A[i1 * ld + k] = v1;
            if (q == 0 && lane == 0 && i1 >= j + 3) sg = fmaf(v1, v1, sg);
          }
        }
      }
    }
    if (lane == 0) pn[warp] = sg;
    __syncthreads();
  }
  for (int i = tid; i < n; i += TE_THREADS) d[i] = A[i * ld + i];
  if (tid == 0 && n >= 2) e[n - 2] = A[(n - 1) * ld + (n - 2)];
  if (tid == 0 && n >= 2) {
    tau[n - 2] = 0.f;
    scl[n - 2] = 0.f;
  }
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
      red[2] = nrm;
    }
  }
  __syncthreads();
  const float nrm = red[2];
  const float pivmin = 1e-30f * fmaxf(1.f, nrm * nrm);

  // 2. Multisection: G lanes per eigenvalue split its bracket into G + 1
  // parts per step (a group never straddles a warp).
  {
    const int G = n <= TE_THREADS / 8 ? 8 : (n <= TE_THREADS / 4 ? 4 : (n <= TE_THREADS / 2 ? 2 : 1));
    const float width = 4.f * 1.1920929e-7f * nrm + 1e-30f;
    const int g = tid % G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane / G * G));
    for (int t = tid / G; t < n; t += TE_THREADS / G) {  // the G lanes of a group share t
      float a = red[0], b = red[1];
      for (int it = 0; it < TE_MAXSECT; ++it) {
        const float h = (b - a) / (float)(G + 1);
        const float x = a + h * (float)(g + 1);
        const bool above = sturm_count(d, e2, n, x, pivmin) > t;
        const unsigned bal = __ballot_sync(gmask, above) >> (lane / G * G);
        // First test point past eigenvalue t: the new bracket ends there.
        const int f = bal ? __ffs(bal) - 1 : G;
        const float na = f == 0 ? a : a + h * (float)f;
        const float nb = f == G ? b : a + h * (float)(f + 1);
        a = na;
        b = nb;
        if (!(b - a > width)) break;
      }
      if (g == 0) lam[t] = 0.5f * (a + b);
    }
  }
  __syncthreads();

  // 3. Inverse iteration, thread t for eigenvalue t; the solution goes to
  // column t of X.  Factors of T - lambda I: reciprocal pivots r_i and
  // multipliers m_i = e_{i-1} r_{i-1}.
  const float guard = 1.1920929e-7f * nrm + 1e-30f;
  for (int t = tid; t < n; t += TE_THREADS) {
    const float lm = lam[t];
    float r[TE_NMAX], ml[TE_NMAX];
    float qi = d[0] - lm;
    if (fabsf(qi) < guard) qi = qi < 0.f ? -guard : guard;
    r[0] = 1.f / qi;
    ml[0] = 0.f;
    for (int i = 1; i < n; ++i) {
      const float mlt = e[i - 1] * r[i - 1];
      qi = d[i] - lm - mlt * e[i - 1];
      if (fabsf(qi) < guard) qi = qi < 0.f ? -guard : guard;
      r[i] = 1.f / qi;
      ml[i] = mlt;
    }
    for (int i = 0; i < n; ++i) X[i * ld + t] = te_rand((uint32_t)t, (uint32_t)i);
    for (int iter = 0; iter < 2; ++iter) {
      float y = X[t];
      for (int i = 1; i < n; ++i) {
        y = X[i * ld + t] - ml[i] * y;
        X[i * ld + t] = y;
      }
      float x = X[(n - 1) * ld + t] * r[n - 1];
      X[(n - 1) * ld + t] = x;
      float ss = x * x;
      for (int i = n - 2; i >= 0; --i) {
        x = (X[i * ld + t] - e[i] * x) * r[i];
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

  // 4. Back-transformation: for j = n-3 .. 0, X <- X - tau_j v_j (v_j^T X).
  for (int j = n - 3; j >= 0; --j) {
    const float t = tau[j];
    if (t == 0.f) continue;  // uniform
    const float sc = scl[j];
    {
      const int sub = tid % 4;
      const unsigned gmask = 0xFu << (lane & ~3);
      for (int c = tid / 4; c < n; c += TE_THREADS / 4) {
        float s0 = 0.f, s1 = 0.f;
#pragma unroll 4
        for (int i = j + 1 + sub; i < n; i += 8) {
          s0 = fmaf(i == j + 1 ? 1.f : A[i * ld + j] * sc, X[i * ld + c], s0);
          if (i + 4 < n) s1 = fmaf(A[(i + 4) * ld + j] * sc, X[(i + 4) * ld + c], s1);
        }
        float s = s0 + s1;
        s += __shfl_xor_sync(gmask, s, 1);
        s += __shfl_xor_sync(gmask, s, 2);
        if (sub == 0) p[c] = t * s;
      }
    }
    __syncthreads();
    float pc[TE_KREG];
#pragma unroll
    for (int q = 0; q < TE_KREG; ++q) pc[q] = lane + 32 * q < n ? p[lane + 32 * q] : 0.f;
    for (int i = j + 1 + warp; i < n; i += TE_WARPS) {
      const float vi = i == j + 1 ? 1.f : A[i * ld + j] * sc;
      float x[TE_KREG];  // the row's loads before its stores
#pragma unroll
      for (int q = 0; q < TE_KREG; ++q) x[q] = lane + 32 * q < n ? X[i * ld + lane + 32 * q] : 0.f;
#pragma unroll
      for (int q = 0; q < TE_KREG; ++q)
        if (lane + 32 * q < n) X[i * ld + lane + 32 * q] = fmaf(-vi, pc[q], x[q]);
    }
    __syncthreads();
  }
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
