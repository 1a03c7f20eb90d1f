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

}  // namespace atk
