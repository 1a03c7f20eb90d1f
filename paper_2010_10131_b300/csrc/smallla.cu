// Float64 small dense linear algebra for the factor matrices (I_n x R_n) and
// the R_n x R_n systems of Alg. 3: Gram products A^T B, Cholesky with the
// triangular inverse, right-multiplication, the Newton-Schulz polar step, and
// CholeskyQR2.
//
// On B300, float64 runs at about 1/60 of the float32 rate, and one SM manages
// only about 8 GFLOP/s.  So every O(n R^2) product here is spread over many
// CTAs.  Only the O(R^3) factorisations run on a single CTA.
#include <algorithm>

#include "atk_internal.cuh"

namespace atk {

constexpr int GT_CHUNK = 16;  // rows of A per CTA in A^T B

// part[chunk][R x R] = A[chunk rows]^T B[chunk rows]
__global__ void gemm_tn_part_kernel(const double* __restrict__ A, const double* __restrict__ B, int64_t n, int64_t R,
                                    double* __restrict__ part) {
  int64_t o = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (o >= R * R) return;
  int64_t r1 = o % R, r2 = o / R;
  int64_t i0 = (int64_t)blockIdx.x * GT_CHUNK, i1 = min(n, i0 + GT_CHUNK);
  double s = 0.0;
  for (int64_t i = i0; i < i1; ++i) s = fma(A[i + n * r1], B[i + n * r2], s);
  part[(int64_t)blockIdx.x * R * R + o] = s;
}

__global__ void sum_parts_kernel(const double* __restrict__ part, int nparts, int64_t len, double* __restrict__ out) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= len) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * len + o];
  out[o] = s;
}

size_t smallla_scratch_bytes(int64_t n, int64_t R) {
  int64_t chunks = ceil_div(std::max<int64_t>(n, 1), GT_CHUNK);
  // partials + three R x R matrices + an n x R panel, plus alignment slack
  return sizeof(double) * (size_t)(chunks * R * R + 4 * R * R + 2 * n * R) + 4096;
}

int gemm_tn_f64(const double* A, const double* B, int64_t n, int64_t R, double* G, double* scratch, cudaStream_t st) {
  int64_t chunks = ceil_div(std::max<int64_t>(n, 1), GT_CHUNK);
  if (n == 0) {
    ATK_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * R * R, st));
    return ATK_OK;
  }
  dim3 grid((unsigned)chunks, (unsigned)ceil_div(R * R, 256));
  gemm_tn_part_kernel<<<grid, 256, 0, st>>>(A, B, n, R, scratch);
  ATK_LAUNCHED();
  sum_parts_kernel<<<(unsigned)ceil_div(R * R, 256), 256, 0, st>>>(scratch, (int)chunks, R * R, G);
  ATK_LAUNCHED();
  return ATK_OK;
}

// One CTA: Cholesky G = C C^T (C lower), Cinv = C^{-1} (lower) and, if
// requested, Ginv = Cinv^T Cinv.  Everything lives in global memory (L2);
// R <= 128.  A non-positive pivot sets DEV_CHOL and leaves identity factors,
// so later kernels stay finite.
__global__ void __launch_bounds__(256) chol_inv_kernel(const double* __restrict__ G, int R, double* __restrict__ C,
                                                       double* __restrict__ Cinv, double* __restrict__ Ginv,
                                                       int* __restrict__ status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) C[idx] = G[idx];
  __syncthreads();
  // Right-looking Cholesky on the lower triangle (column-major, C[i + R*j]).
  for (int j = 0; j < R; ++j) {
    if (threadIdx.x == 0) {
      double d = C[j + R * j];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      C[j + R * j] = sqrt(d);
    }
    __syncthreads();
    double cjj = C[j + R * j];
    for (int i = j + 1 + threadIdx.x; i < R; i += blockDim.x) C[i + R * j] /= cjj;
    __syncthreads();
    int rem = R - j - 1;
    for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
      int i = j + 1 + idx % rem, k = j + 1 + idx / rem;
      if (i >= k) C[i + R * k] -= C[i + R * j] * C[k + R * j];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    int i = idx % R, k = idx / R;
    if (i < k) C[idx] = 0.0;
  }
  __syncthreads();
  if (bad) {
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
      double e = (idx % R == idx / R) ? 1.0 : 0.0;
      C[idx] = e;
      Cinv[idx] = e;
      if (Ginv) Ginv[idx] = e;
    }
    if (threadIdx.x == 0) atomicOr(status, DEV_CHOL);
    return;
  }
  // Cinv: column k solves C x = e_k by forward substitution (one thread per column).
  for (int k = threadIdx.x; k < R; k += blockDim.x) {
    for (int i = 0; i < R; ++i) {
      if (i < k) { Cinv[i + R * k] = 0.0; continue; }
      double s = (i == k) ? 1.0 : 0.0;
      for (int t = k; t < i; ++t) s -= C[i + R * t] * Cinv[t + R * k];
      Cinv[i + R * k] = s / C[i + R * i];
    }
  }
  __syncthreads();
  if (Ginv) {
    for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
      int i = idx % R, k = idx / R;
      double s = 0.0;
      for (int t = max(i, k); t < R; ++t) s += Cinv[t + R * i] * Cinv[t + R * k];
      Ginv[idx] = s;
    }
  }
}

// out (m x R) = X (m x R) * M (R x R), or X * M^T when transM.
__global__ void gemm_nn_kernel(const double* __restrict__ X, const double* __restrict__ M, int64_t m, int64_t R,
                               int transM, double* __restrict__ out) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= m * R) return;
  int64_t i = o % m, c = o / m;
  double s = 0.0;
  for (int64_t t = 0; t < R; ++t) s = fma(X[i + m * t], transM ? M[c + R * t] : M[t + R * c], s);
  out[o] = s;
}

// C (m x p) = A (m x k) B (k x p), all column-major float64; one thread per output.
__global__ void gemm_f64_kernel(const double* __restrict__ A, const double* __restrict__ B, int64_t m, int64_t k,
                                int64_t p, double* __restrict__ C) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= m * p) return;
  int64_t i = o % m, c = o / m;
  double s = 0.0;
  for (int64_t t = 0; t < k; ++t) s = fma(A[i + m * t], B[t + k * c], s);
  C[o] = s;
}

// lam[r] = u_r^T z_r (Rayleigh quotients, z = S u), disc = trace(S) - sum_r lam[r].
// One CTA; fixed-order reductions.
__global__ void __launch_bounds__(256) rayleigh_kernel(const double* __restrict__ S, const double* __restrict__ U,
                                                       const double* __restrict__ Z, int64_t n, int64_t R,
                                                       double* __restrict__ lam_out, double* __restrict__ disc_out) {
  __shared__ double red[256];
  __shared__ double lam_sum;
  if (threadIdx.x == 0) lam_sum = 0.0;
  __syncthreads();
  for (int64_t r = 0; r < R; ++r) {
    double part = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) part += U[i + n * r] * Z[i + n * r];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (lam_out) lam_out[r] = red[0];
      lam_sum += red[0];
    }
    __syncthreads();
  }
  double tr = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) tr += S[i + n * i];
  red[threadIdx.x] = tr;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && disc_out) *disc_out = red[0] - lam_sum;
}

int gemm_f64(const double* A, const double* B, int64_t m, int64_t k, int64_t p, double* C, cudaStream_t st) {
  gemm_f64_kernel<<<(unsigned)ceil_div(m * p, 256), 256, 0, st>>>(A, B, m, k, p, C);
  ATK_LAUNCHED();
  return ATK_OK;
}

int rayleigh_f64(const double* S, const double* U, int64_t n, int64_t R, double* Z, double* lam_out,
                 double* disc_out, cudaStream_t st) {
  gemm_f64_kernel<<<(unsigned)ceil_div(n * R, 256), 256, 0, st>>>(S, U, n, n, R, Z);
  ATK_LAUNCHED();
  rayleigh_kernel<<<1, 256, 0, st>>>(S, U, Z, n, R, lam_out, disc_out);
  ATK_LAUNCHED();
  return ATK_OK;
}

__global__ void polar_coef_kernel(const double* __restrict__ G, int64_t R, double* __restrict__ M) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= R * R) return;
  M[o] = ((o % R == o / R) ? 1.5 : 0.0) - 0.5 * G[o];
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
  double *part, *M1, *M2, *M3, *M4, *panel;
};
SmallBufs carve(double* scratch, int64_t n, int64_t R) {
  Arena ar{(char*)scratch, smallla_scratch_bytes(n, R), 0};
  int64_t chunks = ceil_div(std::max<int64_t>(n, 1), GT_CHUNK);
  SmallBufs b;
  b.part = (double*)ar.take(sizeof(double) * chunks * R * R);
  b.M1 = (double*)ar.take(sizeof(double) * R * R);
  b.M2 = (double*)ar.take(sizeof(double) * R * R);
  b.M3 = (double*)ar.take(sizeof(double) * R * R);
  b.M4 = (double*)ar.take(sizeof(double) * R * R);
  b.panel = (double*)ar.take(sizeof(double) * n * R);
  return b;
}
}  // namespace

int solve_spd_right_f64(double* X, int64_t m, int64_t R, const double* G, double* scratch, int* dev_status,
                        cudaStream_t st) {
  SmallBufs b = carve(scratch, m, R);
  if (!b.panel) { set_error("solve_spd: scratch too small"); return ATK_EINVAL; }
  chol_inv_kernel<<<1, 256, 0, st>>>(G, (int)R, b.M1, b.M2, b.M3, dev_status);
  ATK_LAUNCHED();
  gemm_nn_kernel<<<(unsigned)ceil_div(m * R, 256), 256, 0, st>>>(X, b.M3, m, R, 0, b.panel);
  ATK_LAUNCHED();
  ATK_CUDA(cudaMemcpyAsync(X, b.panel, sizeof(double) * m * R, cudaMemcpyDeviceToDevice, st));
  return ATK_OK;
}

int polar_step_f64(double* U, int64_t n, int64_t R, double* scratch, cudaStream_t st) {
  SmallBufs b = carve(scratch, n, R);
  if (!b.panel) { set_error("polar: scratch too small"); return ATK_EINVAL; }
  ATK_TRY(gemm_tn_f64(U, U, n, R, b.M1, b.part, st));
  polar_coef_kernel<<<(unsigned)ceil_div(R * R, 256), 256, 0, st>>>(b.M1, R, b.M2);
  ATK_LAUNCHED();
  gemm_nn_kernel<<<(unsigned)ceil_div(n * R, 256), 256, 0, st>>>(U, b.M2, n, R, 0, b.panel);
  ATK_LAUNCHED();
  ATK_CUDA(cudaMemcpyAsync(U, b.panel, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, st));
  return ATK_OK;
}

int cholqr2_f64(double* L, int64_t n, int64_t R, double* Rhat, double* scratch, int* dev_status, cudaStream_t st) {
  SmallBufs b = carve(scratch, n, R);
  if (!b.panel) { set_error("cholqr2: scratch too small"); return ATK_EINVAL; }
  // Pass 1: L^T L = C1 C1^T, Q1 = L C1^{-T}.
  ATK_TRY(gemm_tn_f64(L, L, n, R, b.M1, b.part, st));
  chol_inv_kernel<<<1, 256, 0, st>>>(b.M1, (int)R, b.M2, b.M3, nullptr, dev_status);
  ATK_LAUNCHED();
  gemm_nn_kernel<<<(unsigned)ceil_div(n * R, 256), 256, 0, st>>>(L, b.M3, n, R, 1, b.panel);
  ATK_LAUNCHED();
  // Pass 2 on Q1: Q1^T Q1 = C2 C2^T, Q = Q1 C2^{-T}.
  ATK_TRY(gemm_tn_f64(b.panel, b.panel, n, R, b.M1, b.part, st));
  chol_inv_kernel<<<1, 256, 0, st>>>(b.M1, (int)R, b.M4, b.M3, nullptr, dev_status);
  ATK_LAUNCHED();
  gemm_nn_kernel<<<(unsigned)ceil_div(n * R, 256), 256, 0, st>>>(b.panel, b.M3, n, R, 1, L);
  ATK_LAUNCHED();
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
