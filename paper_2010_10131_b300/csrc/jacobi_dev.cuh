// Device-side cyclic Jacobi on a symmetric matrix held in shared memory, with
// the parallel (round-robin) ordering: the building block of the one-CTA
// eigensolvers (Alg. 2, EIG branch).
//
// Jacobi (Golub & Van Loan, Matrix Computations, Sec. 8.5): one rotation
// J(p, q) zeroes the off-diagonal entry (p, q) of A <- J^T A J, and V <- V J
// accumulates the eigenvectors.  The rotation is c = 1/sqrt(1+t^2), s = t c,
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / (2 a_pq).
// In the round-robin ("circle") ordering, each round holds m/2 disjoint pairs,
// and every pair meets once in m-1 rounds.  The rotations of one round commute,
// so J^T A J splits into independent 2x2 blocks: block (k, l) of rows {p_k, q_k}
// and columns {p_l, q_l} becomes R_k^T A_kl R_l.  One pass updates the whole
// matrix.  A rotation is skipped when |a_pq| <= max(tol_rel sqrt(|a_pp a_qq|),
// tol_abs ||A||_F).  A sweep with no rotation ends the iteration.
#pragma once

#include "atk_internal.cuh"

namespace atk {

template <typename T>
struct JTol;
// rel: the relative (Demmel-Veselic style) test that does the real work.
// abs: only stops rotations among entries that are negligible against ||A||_F.
// Near convergence, rounding noise on an off-diagonal entry scales with the
// off-diagonal entries themselves (diagonal 2x2 blocks are set to exact zeros),
// so the relative test terminates.
template <>
struct JTol<float> {
  static constexpr float rel = 1e-6f, abs = 1e-9f;
};
template <>
struct JTol<double> {
  static constexpr double rel = 1e-14, abs = 1e-15;
};

// Pair k of round r among m players (m even): the circle method keeps player
// m-1 fixed and rotates the others.
__device__ __forceinline__ void rr_pair(int r, int k, int m, int& p, int& q) {
  if (k == 0) {
    p = m - 1;
    q = r;
  } else {
    p = (r + k) % (m - 1);
    q = (r - k + (m - 1)) % (m - 1);
  }
}

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ void rot_params(T app, T aqq, T apq, T thr_abs, T& c, T& s, bool& rot) {
  T thr = JTol<T>::rel * sqrt(fabs(app * aqq));
  if (fabs(apq) > thr && fabs(apq) > thr_abs) {
    T tau = (aqq - app) / (T(2) * apq);
    T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
    c = rsq(T(1) + t * t);
    s = t * c;
    rot = true;
  } else {
    c = T(1);
    s = T(0);
    rot = false;
  }
}

// Shared-memory working set of one scalar Jacobi solve on an m x m matrix.
template <typename T>
struct JWork {
  T* A;   // m x m, row-major, leading dimension ld
  T* V;   // m x m, leading dimension ld
  T* cs;  // 2 * (m/2): c then s per pair
  int* pq;  // 2 * (m/2): p then q per pair
  int* flag;  // [0]: any rotation this sweep, [1]: any rotation at all
  unsigned short* blk;  // 2 * nblk: (k, l) of the k <= l pair blocks, filled once per solve
  int ld;               // leading dimension of A and V (m, or m + 1 to spread banks)
};
__host__ __device__ inline int nblocks_of(int m) { return (m / 2) * (m / 2 + 1) / 2; }

// Sweeps of the parallel-order Jacobi on shared-memory A (V accumulates).
// All threads of the CTA participate.  Returns the number of sweeps run;
// *converged is set when a sweep performed no rotation.
template <typename T>
__device__ int jacobi_smem(JWork<T> w, int m, T fro, int max_sweeps, bool* converged) {
  const int half = m / 2;
  const int ld = w.ld;
  const T thr_abs = JTol<T>::abs * fro;
  int sweep = 0;
  bool conv = false;
  const int nblk = nblocks_of(m);
  for (int k = threadIdx.x; k < half; k += blockDim.x) {
    int base = k * half - k * (k - 1) / 2;  // blocks before row k of the triangle
    for (int l = k; l < half; ++l) {
      w.blk[base + (l - k)] = (unsigned short)k;
      w.blk[nblk + base + (l - k)] = (unsigned short)l;
    }
  }
  if (threadIdx.x == 0) w.flag[1] = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) w.flag[0] = 0;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int k = threadIdx.x; k < half; k += blockDim.x) {
        int p, q;
        rr_pair(r, k, m, p, q);
        T c, s;
        bool rot;
        rot_params<T>(w.A[p * ld + p], w.A[q * ld + q], w.A[p * ld + q], thr_abs, c, s, rot);
        w.pq[k] = p;
        w.pq[half + k] = q;
        w.cs[k] = c;
        w.cs[half + k] = s;
        if (rot) w.flag[0] = 1;
      }
      __syncthreads();
      // A <- J^T A J on 2x2 blocks (k <= l), mirrored to keep A exactly symmetric.
      for (int idx = threadIdx.x; idx < nblk; idx += blockDim.x) {
        const int k = w.blk[idx], l = w.blk[nblk + idx];
        T ck = w.cs[k], sk = w.cs[half + k], cl = w.cs[l], sl = w.cs[half + l];
        if (sk == T(0) && sl == T(0)) continue;
        int pk = w.pq[k], qk = w.pq[half + k], pl = w.pq[l], ql = w.pq[half + l];
        T x11 = w.A[pk * ld + pl], x12 = w.A[pk * ld + ql];
        T x21 = w.A[qk * ld + pl], x22 = w.A[qk * ld + ql];
        T y11 = ck * x11 - sk * x21, y12 = ck * x12 - sk * x22;
        T y21 = sk * x11 + ck * x21, y22 = sk * x12 + ck * x22;
        T z11 = cl * y11 - sl * y12, z12 = sl * y11 + cl * y12;
        T z21 = cl * y21 - sl * y22, z22 = sl * y21 + cl * y22;
        if (k == l) {
          if (sk != T(0)) { z12 = T(0); z21 = T(0); }
          w.A[pk * ld + pk] = z11;
          w.A[qk * ld + qk] = z22;
          w.A[pk * ld + qk] = z12;
          w.A[qk * ld + pk] = z12;
        } else {
          w.A[pk * ld + pl] = z11; w.A[pl * ld + pk] = z11;
          w.A[pk * ld + ql] = z12; w.A[ql * ld + pk] = z12;
          w.A[qk * ld + pl] = z21; w.A[pl * ld + qk] = z21;
          w.A[qk * ld + ql] = z22; w.A[ql * ld + qk] = z22;
        }
      }
      // V <- V J.  Thread t owns pair l = t % half and the rows i = t / half,
      // t / half + groups, ...; the pair's rotation stays in registers and four
      // rows are loaded before any is written, so shared-memory latency overlaps.
      if ((int)blockDim.x < half) {
        for (int idx = threadIdx.x; idx < m * half; idx += blockDim.x) {
          int i = idx / half, l = idx % half;
          T sl = w.cs[half + l];
          if (sl == T(0)) continue;
          T cl = w.cs[l];
          int pl = w.pq[l], ql = w.pq[half + l];
          T vp = w.V[i * ld + pl], vq = w.V[i * ld + ql];
          w.V[i * ld + pl] = cl * vp - sl * vq;
          w.V[i * ld + ql] = sl * vp + cl * vq;
        }
      } else {
        const int groups = (int)blockDim.x / half;
        const int l = threadIdx.x % half, g = threadIdx.x / half;
        const T sl = w.cs[half + l];
        if (g < groups && sl != T(0)) {
          const T cl = w.cs[l];
          const int pl = w.pq[l], ql = w.pq[half + l];
          int i = g;
          for (; i + 3 * groups < m; i += 4 * groups) {
            T vp0 = w.V[i * ld + pl], vq0 = w.V[i * ld + ql];
            T vp1 = w.V[(i + groups) * ld + pl], vq1 = w.V[(i + groups) * ld + ql];
            T vp2 = w.V[(i + 2 * groups) * ld + pl], vq2 = w.V[(i + 2 * groups) * ld + ql];
            T vp3 = w.V[(i + 3 * groups) * ld + pl], vq3 = w.V[(i + 3 * groups) * ld + ql];
            w.V[i * ld + pl] = cl * vp0 - sl * vq0;
            w.V[i * ld + ql] = sl * vp0 + cl * vq0;
            w.V[(i + groups) * ld + pl] = cl * vp1 - sl * vq1;
            w.V[(i + groups) * ld + ql] = sl * vp1 + cl * vq1;
            w.V[(i + 2 * groups) * ld + pl] = cl * vp2 - sl * vq2;
            w.V[(i + 2 * groups) * ld + ql] = sl * vp2 + cl * vq2;
            w.V[(i + 3 * groups) * ld + pl] = cl * vp3 - sl * vq3;
            w.V[(i + 3 * groups) * ld + ql] = sl * vp3 + cl * vq3;
          }
          for (; i < m; i += groups) {
            T vp = w.V[i * ld + pl], vq = w.V[i * ld + ql];
            w.V[i * ld + pl] = cl * vp - sl * vq;
            w.V[i * ld + ql] = sl * vp + cl * vq;
          }
        }
        // threads beyond groups * half (blockDim not a multiple of half) idle here
      }
      __syncthreads();
    }
    int any = w.flag[0];
    __syncthreads();
    if (any) {
      if (threadIdx.x == 0) w.flag[1] = 1;
    } else {
      conv = true;
      break;
    }
  }
  __syncthreads();
  *converged = conv;
  return conv ? sweep + 1 : sweep;
}

// ------------------------------------------------------------ one-sided
// One-sided (Hestenes) Jacobi on the columns of a symmetric positive
// semidefinite H held column-major in shared memory (W[j * ldw + i] = h_ij; a
// symmetric matrix stored row-major is the same array).  The rotation of pair
// (p, q) makes columns w_p and w_q orthogonal: with alpha = |w_p|^2,
// beta = |w_q|^2, gamma = w_p . w_q, zeta = (beta - alpha) / (2 gamma),
// t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t:
// w_p <- c w_p - s w_q, w_q <- s w_p + c w_q.  This is the two-sided Jacobi
// of H^T H = H^2 carried on H's columns, so at convergence W = H V = U diag(s)
// with V orthogonal, and for PSD H the normalised columns u_i are
// eigenvectors of H with eigenvalue s_i = |w_i| (Golub & Van Loan, Matrix
// Computations, Sec. 8.6.3).  No separate eigenvector matrix is carried.
//
// Round-robin ordering as in jacobi_smem; groups of L lanes own one pair at a
// time (rows gl, gl + L, ... of the two columns in registers, the three dot
// products reduced with shuffles), one barrier per round.  A pair rotates when
// |gamma| > tol sqrt(alpha beta) with tol = 5e-7 sqrt(m) (the float32
// rounding level of an m-term dot product) and |gamma| > 1e-12 ||H||_F^2.
// m must be even (pad with a zero column) and at most L * MR.
// On return lam[i] = |w_i| and w_i is normalised (zero columns stay zero).
__device__ __forceinline__ float hj_rot_t(float x) {
  if (x > 1.1529215e18f) return __fdividef(0.5f, x);
  const float w = fmaf(x, x, 1.f);
  return __fdividef(1.f, fmaf(w, rsqrtf(w), x));
}

template <int L, int MR>
__device__ int hestenes_smem(float* W, int ldw, int m, float fro, int max_sweeps, float* lam, bool* converged) {
  static_assert(L == 8 || L == 16 || L == 32, "group width");
  const int t = threadIdx.x, gl = t % L, grp = t / L, ngrp = blockDim.x / L;
  const int lane = t % 32;
  const unsigned gmask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (lane / L * L));
  const int half = m / 2;
  const float tol = 5e-7f * sqrtf((float)m);
  const float tol2 = tol * tol;
  const float absg = 1e-12f * fro * fro;
  int sweep = 0;
  bool conv = false;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < m - 1; ++r) {
      for (int k = grp; k < half; k += ngrp) {
        int p, q;
        rr_pair(r, k, m, p, q);
        float a[MR], b[MR];
        float al = 0.f, be = 0.f, ga = 0.f;
#pragma unroll
        for (int j = 0; j < MR; ++j) {
          const int i = gl + L * j;
          a[j] = i < m ? W[p * ldw + i] : 0.f;
          b[j] = i < m ? W[q * ldw + i] : 0.f;
          al = fmaf(a[j], a[j], al);
          be = fmaf(b[j], b[j], be);
          ga = fmaf(a[j], b[j], ga);
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(gmask, al, o);
          be += __shfl_xor_sync(gmask, be, o);
          ga += __shfl_xor_sync(gmask, ga, o);
        }
        if (ga * ga > tol2 * (al * be) && fabsf(ga) > absg) {
          const float zeta = __fdividef(be - al, 2.f * ga);
          const float tt = zeta >= 0.f ? hj_rot_t(zeta) : -hj_rot_t(-zeta);
          const float c = rsqrtf(fmaf(tt, tt, 1.f)), s = c * tt;
#pragma unroll
          for (int j = 0; j < MR; ++j) {
            const int i = gl + L * j;
            if (i < m) {
              W[p * ldw + i] = c * a[j] - s * b[j];
              W[q * ldw + i] = s * a[j] + c * b[j];
            }
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) {
      conv = true;
      break;
    }
  }
  // Norms and normalisation, one group per column.
  for (int j = grp; j < m; j += ngrp) {
    float ss = 0.f;
    for (int i = gl; i < m; i += L) ss = fmaf(W[j * ldw + i], W[j * ldw + i], ss);
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) ss += __shfl_xor_sync(gmask, ss, o);
    const float nrm = sqrtf(ss);
    const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
    for (int i = gl; i < m; i += L) W[j * ldw + i] *= inv;
    if (gl == 0) lam[j] = nrm;
  }
  __syncthreads();
  *converged = conv;
  return conv ? sweep + 1 : sweep;
}

}  // namespace atk
