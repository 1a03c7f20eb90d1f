// Leading eigenvectors of the Gram matrix (Alg. 2, EIG branch:
// "U^(n) <- R_n leading eigenvectors of S") by the cyclic Jacobi method with
// parallel (round-robin) ordering.
//
// Jacobi (Golub & Van Loan, Matrix Computations, Sec. 8.5): one rotation
// J(p, q) zeroes the off-diagonal entry (p, q) of A <- J^T A J, and V <- V J
// accumulates the eigenvectors.  The rotation is c = 1/sqrt(1+t^2), s = t c,
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / (2 a_pq).
// In the round-robin ("circle") ordering, each round holds m/2 disjoint pairs,
// and every pair meets once in m-1 rounds.  The rotations of one round commute,
// so J^T A J splits into independent 2x2 blocks: block (k, l) of rows {p_k, q_k}
// and columns {p_l, q_l} becomes R_k^T A_kl R_l.  One pass updates the whole
// matrix.
//
// Two drivers:
//  * n <= 128 (float rotations) or n <= 112 (double): one CTA holds A and V in
//    shared memory and runs every round with __syncthreads between them.
//  * larger n: block Jacobi.  The index range is cut into blocks of b = 32.  A
//    round pairs blocks (P_k, Q_k).  Each 64 x 64 sub-problem is diagonalised
//    in shared memory by the same scalar routine, which yields W_k and the
//    rotated diagonal block.  Then the off-diagonal blocks A_kl <- W_k^T A_kl W_l
//    and V <- V W are applied as 64 x 64 block products across all SMs.  This is a persistent cooperative kernel with a bounded grid barrier
//    between phases.
// A rotation is skipped when |a_pq| <= max(tol_rel sqrt(|a_pp a_qq|),
// tol_abs ||A||_F).  A sweep with no rotation ends the iteration.
#include <algorithm>

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

template <typename T>
__device__ __forceinline__ void rot_params(T app, T aqq, T apq, T thr_abs, T& c, T& s, bool& rot) {
  T thr = JTol<T>::rel * sqrt(fabs(app * aqq));
  if (fabs(apq) > thr && fabs(apq) > thr_abs) {
    T tau = (aqq - app) / (T(2) * apq);
    T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
    c = T(1) / sqrt(T(1) + t * t);
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
  T* A;   // m x m, row-major, leading dimension m
  T* V;   // m x m
  T* cs;  // 2 * (m/2): c then s per pair
  int* pq;  // 2 * (m/2): p then q per pair
  int* flag;  // [0]: any rotation this sweep, [1]: any rotation at all
};

// Sweeps of the parallel-order Jacobi on shared-memory A (V accumulates).
// All threads of the CTA participate.  Returns the number of sweeps run;
// *converged is set when a sweep performed no rotation.
template <typename T>
__device__ int jacobi_smem(JWork<T> w, int m, T fro, int max_sweeps, bool* converged) {
  const int half = m / 2;
  const T thr_abs = JTol<T>::abs * fro;
  int sweep = 0;
  bool conv = false;
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
        rot_params<T>(w.A[p * m + p], w.A[q * m + q], w.A[p * m + q], thr_abs, c, s, rot);
        w.pq[k] = p;
        w.pq[half + k] = q;
        w.cs[k] = c;
        w.cs[half + k] = s;
        if (rot) w.flag[0] = 1;
      }
      __syncthreads();
      // A <- J^T A J on 2x2 blocks (k <= l), mirrored to keep A exactly symmetric.
      const int nblk = half * (half + 1) / 2;
      for (int idx = threadIdx.x; idx < nblk; idx += blockDim.x) {
        int k = 0, rem = idx;
        while (rem >= half - k) { rem -= half - k; ++k; }
        int l = k + rem;
        T ck = w.cs[k], sk = w.cs[half + k], cl = w.cs[l], sl = w.cs[half + l];
        if (sk == T(0) && sl == T(0)) continue;
        int pk = w.pq[k], qk = w.pq[half + k], pl = w.pq[l], ql = w.pq[half + l];
        T x11 = w.A[pk * m + pl], x12 = w.A[pk * m + ql];
        T x21 = w.A[qk * m + pl], x22 = w.A[qk * m + ql];
        T y11 = ck * x11 - sk * x21, y12 = ck * x12 - sk * x22;
        T y21 = sk * x11 + ck * x21, y22 = sk * x12 + ck * x22;
        T z11 = cl * y11 - sl * y12, z12 = sl * y11 + cl * y12;
        T z21 = cl * y21 - sl * y22, z22 = sl * y21 + cl * y22;
        if (k == l) {
          if (sk != T(0)) { z12 = T(0); z21 = T(0); }
          w.A[pk * m + pk] = z11;
          w.A[qk * m + qk] = z22;
          w.A[pk * m + qk] = z12;
          w.A[qk * m + pk] = z12;
        } else {
          w.A[pk * m + pl] = z11; w.A[pl * m + pk] = z11;
          w.A[pk * m + ql] = z12; w.A[ql * m + pk] = z12;
          w.A[qk * m + pl] = z21; w.A[pl * m + qk] = z21;
          w.A[qk * m + ql] = z22; w.A[ql * m + qk] = z22;
        }
      }
      // V <- V J
      for (int idx = threadIdx.x; idx < m * half; idx += blockDim.x) {
        int i = idx / half, l = idx % half;
        T sl = w.cs[half + l];
        if (sl == T(0)) continue;
        T cl = w.cs[l];
        int pl = w.pq[l], ql = w.pq[half + l];
        T vp = w.V[i * m + pl], vq = w.V[i * m + ql];
        w.V[i * m + pl] = cl * vp - sl * vq;
        w.V[i * m + ql] = sl * vp + cl * vq;
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

// ---------------------------------------------------------- one-CTA driver
// One matrix per CTA (blockIdx.x), padded to m = n rounded up to even.
// Writes diag (n) and V (n x n, row-major, column j = eigenvector j) to global.
template <typename T>
__global__ void __launch_bounds__(256) jacobi_small_kernel(const double* __restrict__ S, int n, int m, int max_sweeps,
                                                           T* __restrict__ diag_out, T* __restrict__ V_out,
                                                           int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* A = reinterpret_cast<T*>(smem_raw);
  T* V = A + m * m;
  T* cs = V + m * m;
  int* pq = reinterpret_cast<int*>(cs + m);
  int* flag = pq + m;
  __shared__ double red[256];
  const double* Sm = S + (size_t)blockIdx.x * n * n;
  double loc = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, j = idx % m;
    double v = (i < n && j < n) ? Sm[i + (size_t)n * j] : 0.0;
    A[idx] = (T)v;
    V[idx] = (i == j) ? T(1) : T(0);
    loc += v * v;
  }
  red[threadIdx.x] = loc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  T fro = (T)sqrt(red[0]);
  JWork<T> w{A, V, cs, pq, flag};
  bool conv = true;
  if (m >= 2) jacobi_smem<T>(w, m, fro, max_sweeps, &conv);
  if (!conv && threadIdx.x == 0) atomicOr(status, DEV_NOCONV);
  T* dg = diag_out + (size_t)blockIdx.x * n;
  T* vo = V_out + (size_t)blockIdx.x * n * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dg[i] = A[i * m + i];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int i = idx / n, j = idx % n;
    vo[idx] = V[i * m + j];
  }
}

// ------------------------------------------------------ block Jacobi driver
constexpr int JB = 32;       // block size b; sub-problems are 2b x 2b
constexpr int JS = 2 * JB;   // 64

struct BlockJacobiArgs {
  int n, m, mb;   // true size, padded size (multiple of 64), number of blocks
  int max_sweeps, inner_sweeps;
  unsigned* bar;  // grid barrier words (2)
  int* sweep_flags;  // per outer sweep: 1 if any rotation happened
  int* status;
};

// Global index of local index u (0..63) in the sub-problem of blocks (P, Q).
__device__ __forceinline__ int sub_index(int u, int P, int Q) { return u < JB ? P * JB + u : Q * JB + (u - JB); }

template <typename T>
__global__ void __launch_bounds__(256) jacobi_block_kernel(BlockJacobiArgs args, T* __restrict__ A,
                                                           T* __restrict__ V, T* __restrict__ W, T fro) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s0 = reinterpret_cast<T*>(smem_raw);  // 4 tiles of 64 x 64
  T* s1 = s0 + JS * JS;
  T* s2 = s1 + JS * JS;
  T* s3 = s2 + JS * JS;
  T* cs = s3 + JS * JS;
  int* pq = reinterpret_cast<int*>(cs + JS);
  int* flag = pq + JS;
  const int m = args.m, mb = args.mb, half = mb / 2;
  const unsigned G = gridDim.x;
  for (int sweep = 0; sweep < args.max_sweeps; ++sweep) {
    for (int r = 0; r < mb - 1; ++r) {
      // Phase 1: diagonalise the 64 x 64 sub-problem of each block pair.
      for (int k = blockIdx.x; k < half; k += G) {
        int P, Q;
        rr_pair(r, k, mb, P, Q);
        for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
          int u = idx / JS, v = idx % JS;
          s0[idx] = A[(size_t)sub_index(u, P, Q) * m + sub_index(v, P, Q)];
          s1[idx] = (u == v) ? T(1) : T(0);
        }
        __syncthreads();
        JWork<T> w{s0, s1, cs, pq, flag};
        bool conv;
        jacobi_smem<T>(w, JS, fro, args.inner_sweeps, &conv);
        if (threadIdx.x == 0 && flag[1]) atomicOr(args.sweep_flags + sweep, 1);
        // The rotated sub-problem is W_k^T A_kk W_k, computed by exact 2x2
        // rotations: write it back here.  Phase 2 skips the diagonal blocks, since
        // a 64-term product would put rounding noise of order eps * lambda_max
        // back into the entries just eliminated.
        T* Wk = W + (size_t)k * JS * JS;
        for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
          int u = idx / JS, v = idx % JS;
          Wk[idx] = s1[idx];
          A[(size_t)sub_index(u, P, Q) * m + sub_index(v, P, Q)] = s0[idx];
        }
        __syncthreads();
      }
      if (!grid_barrier(args.bar, G, args.status)) return;
      // Phase 2: A_kl <- W_k^T A_kl W_l (k < l, mirrored) and V_l <- V_l W_l.
      const int ntA = half * (half - 1) / 2;
      const int nrow = m / JS;
      const int ntV = half * nrow;
      for (int task = blockIdx.x; task < ntA + ntV; task += G) {
        if (task < ntA) {
          int k = 0, rem = task;
          while (rem >= half - 1 - k) { rem -= half - 1 - k; ++k; }
          int l = k + 1 + rem;
          int Pk, Qk, Pl, Ql;
          rr_pair(r, k, mb, Pk, Qk);
          rr_pair(r, l, mb, Pl, Ql);
          const T* Wk = W + (size_t)k * JS * JS;
          const T* Wl = W + (size_t)l * JS * JS;
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            s0[idx] = A[(size_t)sub_index(u, Pk, Qk) * m + sub_index(v, Pl, Ql)];
            s1[idx] = Wk[idx];
            s2[idx] = Wl[idx];
          }
          __syncthreads();
          // s3 = X W_l
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            T acc = 0;
#pragma unroll 8
            for (int t = 0; t < JS; ++t) acc += s0[u * JS + t] * s2[t * JS + v];
            s3[idx] = acc;
          }
          __syncthreads();
          // X' = W_k^T s3, written back (and mirrored for k < l)
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            T acc = 0;
#pragma unroll 8
            for (int t = 0; t < JS; ++t) acc += s1[t * JS + u] * s3[t * JS + v];
            int gu = sub_index(u, Pk, Qk), gv = sub_index(v, Pl, Ql);
            A[(size_t)gu * m + gv] = acc;
            A[(size_t)gv * m + gu] = acc;
          }
          __syncthreads();
        } else {
          int t2 = task - ntA;
          int l = t2 % half, rowc = t2 / half;
          int Pl, Ql;
          rr_pair(r, l, mb, Pl, Ql);
          const T* Wl = W + (size_t)l * JS * JS;
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            s0[idx] = V[(size_t)(rowc * JS + u) * m + sub_index(v, Pl, Ql)];
            s2[idx] = Wl[idx];
          }
          __syncthreads();
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            T acc = 0;
#pragma unroll 8
            for (int t = 0; t < JS; ++t) acc += s0[u * JS + t] * s2[t * JS + v];
            V[(size_t)(rowc * JS + u) * m + sub_index(v, Pl, Ql)] = acc;
          }
          __syncthreads();
        }
      }
      if (!grid_barrier(args.bar, G, args.status)) return;
    }
    if (*(volatile int*)(args.sweep_flags + sweep) == 0) return;  // converged
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(args.status, DEV_NOCONV);
}

// ------------------------------------------------------------- selection
// Sort eigenvalues descending (stable in index), keep the first R vectors,
// sign each so that its largest-magnitude entry is positive (ties: lowest
// row), write U (n x R column-major, float64), all eigenvalues (descending)
// and the discarded sum.  One CTA.  V is row-major with leading dimension ldv.
template <typename T>
__global__ void __launch_bounds__(1024) select_kernel(const T* __restrict__ diag, int64_t dstride,
                                                      const T* __restrict__ V, int ldv, int n, int R,
                                                      double* __restrict__ U, double* __restrict__ lam_out,
                                                      double* __restrict__ disc_out) {
  __shared__ int order[1024];
  __shared__ double lam[1024];
  __shared__ double red[1024];
  for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = (double)diag[(int64_t)i * dstride];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double li = lam[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double lj = lam[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  if (lam_out)
    for (int r = threadIdx.x; r < n; r += blockDim.x) lam_out[r] = lam[order[r]];
  // Discarded energy: fixed-order tree sum of the eigenvalues beyond R.
  double loc = 0.0;
  for (int r = R + threadIdx.x; r < n; r += blockDim.x) loc += lam[order[r]];
  red[threadIdx.x] = loc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && disc_out) *disc_out = red[0];
  // One warp per selected column.
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int r = warp; r < R; r += nw) {
    int col = order[r];
    double best = -1.0;
    int arg = 0;
    for (int i = lane; i < n; i += 32) {
      double a = fabs((double)V[(int64_t)i * ldv + col]);
      if (a > best) { best = a; arg = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_down_sync(0xffffffffu, best, o);
      int oa = __shfl_down_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    }
    arg = __shfl_sync(0xffffffffu, arg, 0);
    double sg = ((double)V[(int64_t)arg * ldv + col] < 0.0) ? -1.0 : 1.0;
    for (int i = lane; i < n; i += 32) U[i + (int64_t)n * r] = sg * (double)V[(int64_t)i * ldv + col];
  }
}

// --------------------------------------------------------------- host side
namespace {
template <typename T>
size_t small_smem(int m) {
  return (size_t)2 * m * m * sizeof(T) + (size_t)m * sizeof(T) + (size_t)(m + 2) * sizeof(int) + 16;
}
template <typename T>
bool use_small(int n) {
  int m = n + (n & 1);
  return small_smem<T>(m) <= 200 * 1024;
}
template <typename T>
size_t block_smem() {
  return (size_t)4 * JS * JS * sizeof(T) + JS * sizeof(T) + (JS + 2) * sizeof(int) + 16;
}
template <typename T>
size_t eig_bytes_t(int64_t n) {
  size_t b = 4096;
  if (use_small<T>((int)n)) {
    b += (size_t)(n * n + n) * sizeof(T) + 1024;
  } else {
    int64_t m = ceil_div(n, JS) * JS;
    int64_t mb = m / JB;
    b += (size_t)(2 * m * m + (mb / 2) * JS * JS) * sizeof(T) + 64 * sizeof(int) + 1024;
  }
  return b;
}

__global__ void init_block_kernel(const double* __restrict__ S, int n, int m, float* Af, float* Vf, double* Ad,
                                  double* Vd) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  int i = (int)(idx / m), j = (int)(idx % m);
  double v = (i < n && j < n) ? S[i + (int64_t)n * j] : 0.0;
  double e = (i == j) ? 1.0 : 0.0;
  if (Af) { Af[idx] = (float)v; Vf[idx] = (float)e; }
  if (Ad) { Ad[idx] = v; Vd[idx] = e; }
}

__global__ void fro_kernel(const double* __restrict__ S, int64_t count, double* out) {
  __shared__ double red[256];
  double loc = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) loc += S[i] * S[i];
  red[threadIdx.x] = loc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0]);
}

template <typename T>
int eig_top_t(const double* S, int64_t n, int64_t R, int max_sweeps, double* U64, double* lam_out,
              double* disc_out, int* dev_status, char* scratch, size_t scratch_bytes, cudaStream_t st) {
  Arena ar{scratch, scratch_bytes, 0};
  if (use_small<T>((int)n)) {
    int m = (int)(n + (n & 1));
    T* diag = (T*)ar.take(sizeof(T) * n);
    T* V = (T*)ar.take(sizeof(T) * n * n);
    if (!diag || !V) { set_error("eig: scratch too small"); return ATK_EINVAL; }
    size_t sm = small_smem<T>(m);
    ATK_CUDA(cudaFuncSetAttribute(jacobi_small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    jacobi_small_kernel<T><<<1, 256, sm, st>>>(S, (int)n, m, max_sweeps, diag, V, dev_status);
    ATK_LAUNCHED();
    select_kernel<T><<<1, 1024, 0, st>>>(diag, 1, V, (int)n, (int)n, (int)R, U64, lam_out, nullptr);
    ATK_LAUNCHED();
    return ATK_OK;
  }
  const int m = (int)(ceil_div(n, JS) * JS);
  const int mb = m / JB;
  T* A = (T*)ar.take(sizeof(T) * (size_t)m * m);
  T* V = (T*)ar.take(sizeof(T) * (size_t)m * m);
  T* W = (T*)ar.take(sizeof(T) * (size_t)(mb / 2) * JS * JS);
  int* words = (int*)ar.take(sizeof(int) * 64 + 64);
  double* fro_d = (double*)ar.take(sizeof(double));
  if (!A || !V || !W || !words || !fro_d) { set_error("eig: scratch too small"); return ATK_EINVAL; }
  ATK_CUDA(cudaMemsetAsync(words, 0, sizeof(int) * 64 + 64, st));
  const bool f = sizeof(T) == 4;
  init_block_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(
      S, (int)n, m, f ? (float*)A : nullptr, f ? (float*)V : nullptr, f ? nullptr : (double*)A,
      f ? nullptr : (double*)V);
  ATK_LAUNCHED();
  fro_kernel<<<1, 256, 0, st>>>(S, n * n, fro_d);
  ATK_LAUNCHED();
  double fro_h = 0.0;
  ATK_CUDA(cudaMemcpyAsync(&fro_h, fro_d, sizeof(double), cudaMemcpyDeviceToHost, st));
  ATK_CUDA(cudaStreamSynchronize(st));
  BlockJacobiArgs args;
  args.n = (int)n;
  args.m = m;
  args.mb = mb;
  args.max_sweeps = std::min(max_sweeps, 60);
  args.inner_sweeps = 3;
  args.bar = reinterpret_cast<unsigned*>(words);
  args.sweep_flags = words + 2;
  args.status = dev_status;
  size_t sm = block_smem<T>();
  ATK_CUDA(cudaFuncSetAttribute(jacobi_block_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  ATK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_block_kernel<T>, 256, sm));
  if (per_sm < 1) { set_error("eig: block Jacobi kernel does not fit on an SM"); return ATK_EUNSUPPORTED; }
  int ntasks = (mb / 2) * (mb / 2 - 1) / 2 + (mb / 2) * (m / JS);
  int grid = std::min(num_sms() * per_sm, std::max(ntasks, mb / 2));
  T fro = (T)fro_h;
  void* kargs[] = {(void*)&args, (void*)&A, (void*)&V, (void*)&W, (void*)&fro};
  ATK_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_block_kernel<T>, dim3(grid), dim3(256), kargs, sm, st));
  count_launch();
  select_kernel<T><<<1, 1024, 0, st>>>(A, (int64_t)m + 1, V, m, (int)n, (int)R, U64, lam_out, nullptr);
  ATK_LAUNCHED();
  return ATK_OK;
}
}  // namespace

size_t eig_scratch_bytes(int64_t n, int arith) {
  size_t jac = arith == ATK_EIG_ROT_FP64 ? eig_bytes_t<double>(n) : eig_bytes_t<float>(n);
  // refinement: Z (n x R) + the float64 small-LA scratch, for R up to n
  size_t ref = (size_t)n * std::min<int64_t>(n, 128) * 8 + smallla_scratch_bytes(n, std::min<int64_t>(n, 128)) + 1024;
  return std::max(jac, ref);
}

// W[:, r] = Z[:, r] / ||Z[:, r]|| when that norm is above thr, else U[:, r]
// (a kept eigenvalue at the level of rounding: keep the Jacobi vector).
// One warp per column.
__global__ void normalize_cols_kernel(const double* __restrict__ Z, const double* __restrict__ U, int64_t n,
                                      int64_t R, const double* __restrict__ scale, double rel,
                                      double* __restrict__ W) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= R) return;
  const double thr = rel * *scale;
  const double* z = Z + (int64_t)warp * n;
  double s = 0.0;
  for (int64_t i = lane; i < n; i += 32) s += z[i] * z[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  double nz = sqrt(s);
  double* w = W + (int64_t)warp * n;
  if (nz > thr) {
    for (int64_t i = lane; i < n; i += 32) w[i] = z[i] / nz;
  } else {
    const double* u = U + (int64_t)warp * n;
    for (int64_t i = lane; i < n; i += 32) w[i] = u[i];
  }
}

// Sign rule: flip each column so that its largest-magnitude entry is positive
// (ties: lowest row).  One warp per column.
__global__ void sign_fix_kernel(double* __restrict__ U, int64_t n, int64_t R) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (warp >= R) return;
  double* u = U + (int64_t)warp * n;
  double best = -1.0;
  int64_t arg = 0;
  for (int64_t i = lane; i < n; i += 32) {
    double a = fabs(u[i]);
    if (a > best) { best = a; arg = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_down_sync(0xffffffffu, best, o);
    int64_t oa = __shfl_down_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
  }
  arg = __shfl_sync(0xffffffffu, arg, 0);
  if (u[arg] < 0.0)
    for (int64_t i = lane; i < n; i += 32) u[i] = -u[i];
}

__global__ void max_abs_diag_kernel(const double* __restrict__ S, int64_t n, double* out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(S[i + n * i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Eigen-decomposition + selection + float64 polar orthonormalisation.
// U64_out (n x R float64) is the orthonormalised basis; U_out its float32 copy.
int eig_top(const double* S, int64_t n, int64_t R, int arith, int max_sweeps, float* U_out, double* U64_out,
            double* lambda_out, double* discarded_out, int* dev_status, char* scratch, size_t scratch_bytes,
            cudaStream_t st) {
  if (n <= 0 || R <= 0 || R > n || n > 1024) { set_error("eig: need 1 <= R <= n <= 1024"); return ATK_EUNSUPPORTED; }
  int s = arith == ATK_EIG_ROT_FP64
              ? eig_top_t<double>(S, n, R, max_sweeps, U64_out, lambda_out, discarded_out, dev_status, scratch,
                                  scratch_bytes, st)
              : eig_top_t<float>(S, n, R, max_sweeps, U64_out, lambda_out, discarded_out, dev_status, scratch,
                                 scratch_bytes, st);
  if (s != ATK_OK) return s;
  Arena ar{scratch, scratch_bytes, 0};
  double* Z = (double*)ar.take(sizeof(double) * n * R);
  double* pol = (double*)ar.take(smallla_scratch_bytes(n, R));
  if (!Z || !pol) { set_error("eig: scratch too small for the refinement"); return ATK_EINVAL; }
  if (arith != ATK_EIG_ROT_FP64) {
    // Float rotations have a backward error of a few hundred eps_32 ||S||, so
    // the selected vectors carry out-of-subspace components at that level.
    // One float64 subspace-iteration step, Z = S U with columns renormalised,
    // shrinks them by lambda_{R+1} / lambda_R.  The vectors stay in eigenvalue
    // order because S U ~ U diag(lambda) with lambda > 0.
    ATK_TRY(gemm_f64(S, U64_out, n, n, R, Z, st));
    double* dmax = pol;
    max_abs_diag_kernel<<<1, 256, 0, st>>>(S, n, dmax);
    ATK_LAUNCHED();
    normalize_cols_kernel<<<(unsigned)ceil_div(R * 32, 256), 256, 0, st>>>(Z, U64_out, n, R, dmax, 1e-7, U64_out);
    ATK_LAUNCHED();
  }
  // Accumulated rotations (and the refinement) leave U orthonormal only to
  // working precision; two float64 Newton-Schulz polar steps restore it
  // without reordering the columns.
  ATK_TRY(polar_step_f64(U64_out, n, R, pol, st));
  ATK_TRY(polar_step_f64(U64_out, n, R, pol, st));
  sign_fix_kernel<<<(unsigned)ceil_div(R * 32, 256), 256, 0, st>>>(U64_out, n, R);
  ATK_LAUNCHED();
  // The kept eigenvalues become float64 Rayleigh quotients of the polished
  // vectors (error ~ ||S|| * subspace error^2), and the discarded energy is
  // trace(S) minus their sum, so neither inherits the rounding of the
  // rotations.  The tail of lambda_out keeps the rotated diagonal.
  ATK_TRY(rayleigh_f64(S, U64_out, n, R, Z, lambda_out, discarded_out, st));
  if (U_out) ATK_TRY(f64_to_f32(U64_out, U_out, n * R, st));
  return ATK_OK;
}

}  // namespace atk
