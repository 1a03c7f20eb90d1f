// Cholesky factor and its triangular inverse on one CTA, float32: the
// CholeskyQR passes of the subspace eigensolver and of the float64
// refinement need L^{-T} for L L^T = G + shift I, G m x m with m <= 160.
//
// Right-looking Cholesky (Golub & Van Loan, Matrix Computations, 4th ed.,
// Alg. 4.2.2, outer-product form) with the inverse X = L^{-1} carried along
// as the forward elimination of the identity: step j takes the pivot g_jj,
// l_i = g_ij / sqrt(g_jj) (i > j), G22 -= l l^T, and for the rows i > j
// W[i, :] -= l_i X[j, :] with X[j, :] = W[j, :] / sqrt(g_jj) (W = I at the
// start).  Both matrices stay in registers for all m steps: warp w holds the
// rows i = w + WH (rs + 2 s) and lane (rs = lane / 16, cg = lane % 16) the
// columns k = cg + 16 t.  Each step reads column j of G and row j of W from
// shared memory, where their owners published them at the end of the
// previous step (double-buffered, so one barrier per step suffices).
#include "atk_internal.cuh"

namespace atk {

constexpr int CI_THREADS = 512;
constexpr int CI_WARPS = CI_THREADS / 32;
constexpr int CI_NMAX = 160;
constexpr unsigned CI_FULL = 0xffffffffu;

// G: m x m float64 (symmetric positive semi-definite).  Mout (m x m,
// column-major) = L^{-T}, upper triangular, for L L^T = G + shift *
// max(diag G) I; a pivot at or below 1e-12 max(diag G) is raised to that
// floor (the factor stays finite) and *breakdown (nullable) is set.
template <int NT>
__global__ void __launch_bounds__(CI_THREADS, 1) cholinv_kernel(const double* __restrict__ G, int m, float shift,
                                                                 float* __restrict__ Mout,
                                                                 int* __restrict__ breakdown) {
  constexpr int WH = NT <= 6 ? 8 : 16;
  constexpr int NS = (8 * NT + WH - 1) / WH;
  __shared__ __align__(16) float cb[2][CI_NMAX];  // column j of the partly factored G
  __shared__ __align__(16) float wb[2][CI_NMAX];  // row j of W
  __shared__ float rinv[CI_NMAX];                 // 1 / l_jj
  __shared__ float pmax[CI_WARPS];
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int rs = lane / 16, cg = lane % 16;
  const bool hw = warp < WH;
  float a[NS][NT], w[NS][NT];
  float dl = 0.f;
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = warp + WH * (rs + 2 * s), k = cg + 16 * t;
      const bool in = hw && i < m && k < m;
      a[s][t] = in ? (float)G[(size_t)i * m + k] : 0.f;
      w[s][t] = (in && i == k) ? 1.f : 0.f;
      if (in && i == k) dl = fmaxf(dl, a[s][t]);
    }
  for (int o = 16; o > 0; o >>= 1) dl = fmaxf(dl, __shfl_xor_sync(CI_FULL, dl, o));
  if (lane == 0) pmax[warp] = dl;
  __syncthreads();
  float dmax = 0.f;
#pragma unroll
  for (int q = 0; q < CI_WARPS; ++q) dmax = fmaxf(dmax, pmax[q]);
  const float sh = shift * dmax, floor_v = 1e-12f * dmax + 1e-30f;
  if (hw) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int i = warp + WH * (rs + 2 * s), k = cg + 16 * t;
        if (i == k) a[s][t] += sh;
      }
    // Column 0 (slot 0 of the lanes with cg = 0) and row 0 of W (slot 0 of
    // lane group 0 in warp 0).
    if (cg == 0)
#pragma unroll
      for (int s = 0; s < NS; ++s) cb[0][warp + WH * (rs + 2 * s)] = a[s][0];
    if (warp == 0 && rs == 0)
#pragma unroll
      for (int t = 0; t < NT; ++t) wb[0][cg + 16 * t] = w[0][t];
  }
  __syncthreads();
  // Steps j = 16 P - 1 .. 16 P + 14 publish the columns c = j + 1 of slot P,
  // so P is a compile-time constant in their body: the publishing needs no
  // selects, and the slots that lie entirely above or left of j are skipped
  // without a branch (column slots t < P, row slots s < S0).
  static_for<0, NT + 1>([&](auto PC) {
    constexpr int P = decltype(PC)::value;
    constexpr int S0 = WH == 8 ? P : P / 2;
    constexpr int XT = P < NT ? P : NT - 1;  // last column slot of row j of X
    const int jhi = min(16 * P + 15, m);
    for (int j = P == 0 ? 0 : 16 * P - 1; j < jhi; ++j) {
      const int buf = j & 1;
      if (hw) {
        const float d = cb[buf][j];
        if (tid == 0 && !(d > floor_v) && breakdown) atomicOr(breakdown, 1);
        // 1/sqrt(d): the hardware estimate and one Newton step.
        const float dd = d > floor_v ? d : floor_v;
        float inv = rsqrtf(dd);
        inv = inv * fmaf(-0.5f * dd * inv, inv, 1.5f);
        if (tid == 0) rinv[j] = inv;
        float li[NS], lk[NT], xj[NT];
#pragma unroll
        for (int s = S0; s < NS; ++s) {
          const int i = warp + WH * (rs + 2 * s);
          li[s] = i > j && i < m ? cb[buf][i] * inv : 0.f;
        }
#pragma unroll
        for (int t = P; t < NT; ++t) {
          const int k = cg + 16 * t;
          lk[t] = k > j && k < m ? cb[buf][k] * inv : 0.f;
        }
#pragma unroll
        for (int t = 0; t <= XT; ++t) {
          const int k = cg + 16 * t;
          xj[t] = k <= j ? wb[buf][k] * inv : 0.f;  // row j of X (zero beyond j)
        }
#pragma unroll
        for (int s = S0; s < NS; ++s) {
#pragma unroll
          for (int t = P; t < NT; ++t) a[s][t] = fmaf(-li[s], lk[t], a[s][t]);
#pragma unroll
          for (int t = 0; t <= XT; ++t) w[s][t] = fmaf(-li[s], xj[t], w[s][t]);
        }
        if constexpr (P < NT) {
          const int c = j + 1;
          if (c < m) {
            if (cg == c % 16)
#pragma unroll
              for (int s = 0; s < NS; ++s) cb[buf ^ 1][warp + WH * (rs + 2 * s)] = a[s][P];
            constexpr int SC = WH == 8 ? P : P / 2;
            if (warp == c % WH && rs == (WH == 8 ? (c / 8) % 2 : P % 2))
#pragma unroll
              for (int t = 0; t < NT; ++t) wb[buf ^ 1][cg + 16 * t] = w[SC][t];
          }
        }
      }
      __syncthreads();
    }
  });
  // X[i, :] = W[i, :] / l_ii; Mout(c, i) = X(i, c) for c <= i, else 0.
  if (hw) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int i = warp + WH * (rs + 2 * s), c = cg + 16 * t;
        if (i < m && c < m) Mout[(size_t)i * m + c] = i >= c ? w[s][t] * rinv[i] : 0.f;
      }
  }
}

namespace {
using CiKernel = void (*)(const double*, int, float, float*, int*);
CiKernel ci_kernel(int m) {
  const int nt = (m + 15) / 16;
  switch (nt <= 2 ? 2 : nt <= 4 ? 4 : nt <= 6 ? nt : nt <= 8 ? 8 : 10) {
    case 2: return cholinv_kernel<2>;
    case 4: return cholinv_kernel<4>;
    case 5: return cholinv_kernel<5>;
    case 6: return cholinv_kernel<6>;
    case 8: return cholinv_kernel<8>;
    default: return cholinv_kernel<10>;
  }
}
}  // namespace

int cholinv_f32(const double* G, int m, float shift, float* Mout, int* breakdown, cudaStream_t st) {
  if (m < 1 || m > CI_NMAX) {
    set_error("cholinv: need 1 <= m <= 160");
    return ATK_EUNSUPPORTED;
  }
  ci_kernel(m)<<<1, CI_THREADS, 0, st>>>(G, m, shift, Mout, breakdown);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
