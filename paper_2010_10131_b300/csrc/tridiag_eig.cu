// Eigen-decomposition of a small dense symmetric matrix on one CTA, float32:
// the Rayleigh-Ritz projections of the subspace eigensolver (m = R + p <= 156)
// need all their eigenpairs.  The matrix is reduced to tridiagonal form and
// the tridiagonal problem is solved by methods whose steps are independent
// across eigenpairs:
//  1. Householder reduction A = Q T Q^T (Golub & Van Loan, Matrix
//     Computations, 4th ed., Alg. 8.3.1): step j reflects column j below the
//     diagonal with H_j = I - tau_j v_j v_j^T (v_j(j+1) = 1), p = tau A22 v,
//     w = p - (tau/2)(p^T v) v, A22 <- A22 - v w^T - w v^T.  A lives in
//     registers for the whole reduction: WH warps (8 for m <= 96, else 16),
//     lane (rs, cg) of warp w holding the rows w + WH (rs + 2 s) and the
//     columns cg + 16 t, so p is a register product plus a butterfly over 16
//     lanes, and the update touches no shared memory.  Two barriers per step:
//     one after p and the per-warp partials of p^T v, one after the owners of
//     column j+1 have published it (and the partial sums of its squared norm
//     below row j+2, from which every thread derives the next reflector).
//  2. Eigenvalues of T by multisection on the Sturm count (ibid., Sec. 8.4.1):
//     one Sturm count per thread on a grid of 512 points across the
//     Gershgorin interval brackets every eigenvalue to 1/513 of it; then G
//     lanes per eigenvalue test 2G points of its bracket per step (two
//     interleaved counts per lane), down to an absolute width of 4 eps ||T||_1.
//  3. Eigenvectors of T by inverse iteration (ibid., Sec. 8.2.2), thread t
//     for eigenvalue t: Gaussian elimination of T - lambda_t I without
//     interchanges, pivots kept away from zero (the classical guard of
//     tridiagonal inverse iteration), then two solves from a pseudo-random
//     start with the same factors.  Within each cluster of
//     eigenvalues closer than 1e-3 ||T||_1 the vectors are orthonormalised in
//     eigenvalue order by classical Gram-Schmidt applied twice (one warp per
//     cluster), so that near-equal eigenvalues get an orthonormal basis of
//     their eigenspace.
//  4. Back-transformation X <- H_0 H_1 ... H_{m-3} X: each warp holds eight
//     eigenvectors in registers and applies the reflectors four at a time
//     (their mutual inner products computed once), with register sums and
//     two shuffles per projection and no barrier.
// The eigenvectors are as accurate as float32 allows (about eps ||T|| / gap);
// the float64 refinement that follows the subspace eigensolver polishes them.
#include <algorithm>

#include "atk_internal.cuh"

namespace atk {

constexpr int TE_THREADS = 512;
constexpr int TE_WARPS = TE_THREADS / 32;
constexpr int TE_NMAX = 160;      // largest matrix (the subspace eigensolver uses m <= 156)
constexpr int TE_GRID = TE_THREADS;  // points of the first multisection step
constexpr int TE_VBUF = TE_NMAX + 4;  // length of the two column buffers (a multiple of 4)
constexpr int TE_MAXSECT = 40;    // multisection steps (a cap; the width test ends them sooner)
constexpr unsigned TE_FULL = 0xffffffffu;

// Shared memory: the per-warp partial sums and the grid counts, two vectors
// of length TE_VBUF, the reflectors (row j = v_j, n x ldv with ldv = n
// rounded up to 16), the eigenvector block X (n x (n+1)) and six vectors of
// length n.
size_t tridiag_eig_smem(int n) {
  const size_t ld = (size_t)n + 1, ldv = 16 * (((size_t)n + 15) / 16);
  return sizeof(float) * (2 * TE_WARPS + 8 + TE_GRID + 2 * TE_VBUF + (size_t)n * ldv + n * ld + 6 * (size_t)n);
}

// Sum of v over the 32 lanes of the warp by an xor butterfly: lanes l and
// l ^ o add the same two operands at every stage (addition commutes
// exactly), so every lane ends with the same bits.
template <int K>
__device__ __forceinline__ void te_warp_sum(float (&v)[K]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] += __shfl_xor_sync(TE_FULL, v[k], o);
}

// Reciprocal estimate (one hardware approximation; denormals flush to zero,
// so a denormal pivot acts as a zero one).
__device__ __forceinline__ float te_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Sturm count: the number of eigenvalues of T below x, from the signs of the
// pivots q_i = (d_i - x) - e_{i-1}^2 / q_{i-1} of T - x I; de[i] = (d_i,
// e_{i-1}^2).  No pivot guard: a zero pivot makes the next one -inf and the
// one after it finite again (IEEE arithmetic; the squared off-diagonal
// entries are kept >= a tiny positive floor, so 0 * inf never occurs).  The
// sign bit is counted, so q = -0 counts as negative and the +inf after it
// as positive, like q = +0 followed by -inf.  The next (d, e^2) pair is
// loaded one step ahead; de has n + 1 entries (the last one a pad).
__device__ __forceinline__ int sturm_count(const float2* __restrict__ de, int n, float x) {
  float q = de[0].x - x;
  unsigned c = __float_as_uint(q) >> 31;
  float2 v = de[1];
#pragma unroll 4
  for (int i = 1; i < n; ++i) {
    const float2 vn = de[i + 1];  // de[n] is a pad entry
    q = fmaf(-v.y, te_rcp(q), v.x - x);
    c += __float_as_uint(q) >> 31;
    v = vn;
  }
  return (int)c;
}

// The same recurrence at two points at once (two independent chains).
__device__ __forceinline__ void sturm_count2(const float2* __restrict__ de, int n, float x0, float x1, int& c0,
                                             int& c1) {
  float q0 = de[0].x - x0, q1 = de[0].x - x1;
  unsigned k0 = __float_as_uint(q0) >> 31, k1 = __float_as_uint(q1) >> 31;
  float2 v = de[1];
#pragma unroll 4
  for (int i = 1; i < n; ++i) {
    const float2 vn = de[i + 1];  // de[n] is a pad entry
    q0 = fmaf(-v.y, te_rcp(q0), v.x - x0);
    q1 = fmaf(-v.y, te_rcp(q1), v.x - x1);
    k0 += __float_as_uint(q0) >> 31;
    k1 += __float_as_uint(q1) >> 31;
    v = vn;
  }
  c0 = (int)k0;
  c1 = (int)k1;
}

__device__ __forceinline__ float te_rand(uint32_t a, uint32_t b) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u;
  h ^= h >> 15;
  h *= 0x2C1B3C6Du;
  h ^= h >> 12;
  return (float)(h & 0xFFFFFF) * (2.f / 16777216.f) - 1.f;
}

// Sum of the first K (a multiple of 4) per-warp partials, in a fixed order
// (the same bits in every thread).
template <int K>
__device__ __forceinline__ float te_sum(const float* p) {
  const float4* p4 = reinterpret_cast<const float4*>(p);
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < K / 4; ++q) {
    const float4 v = p4[q];
    s += v.x;
    s += v.y;
    s += v.z;
    s += v.w;
  }
  return s;
}

// S: n x n float64 (symmetric), n <= 16 NT.  diag_out (n): eigenvalues,
// ascending.  V_out (n x n, row-major, column j = eigenvector of diag_out[j]).
template <int NT>
__global__ void __launch_bounds__(TE_THREADS, 1) tridiag_eig_kernel(const double* __restrict__ S, int n,
                                                                     float* __restrict__ diag_out,
                                                                     float* __restrict__ V_out) {
  // Reduction layout: WH warps; in warp w, lane (rs = lane / 16, cg = lane %
  // 16) holds A(i, k) for the rows i = w + WH (rs + 2 s), s < NS, and the
  // columns k = cg + 16 t, t < NT.  The other phases work on NB = ceil(n/32)
  // chunks of 32 rows.
  constexpr int WH = NT <= 6 ? 8 : 16;
  constexpr int NS = (8 * NT + WH - 1) / WH;
  constexpr int NB = (NT + 1) / 2;
  extern __shared__ __align__(16) float tsm[];
  const int ld = n + 1;
  const int ldv = 16 * ((n + 15) / 16);
  float* part = tsm;                  // [TE_WARPS] partial squared norms of the next column
  float* kpart = part + TE_WARPS;     // [TE_WARPS] partial sums of p^T v
  float* red = kpart + TE_WARPS;      // [8] interval ends and norm
  int* cnt = reinterpret_cast<int*>(red + 8);  // [TE_GRID] Sturm counts of the grid
  float* xb = reinterpret_cast<float*>(cnt + TE_GRID);  // [TE_VBUF] column j+1, zero above row j+2
  float* pb = xb + TE_VBUF;           // [TE_VBUF] p, zero outside the trailing block
  float* Vr = pb + TE_VBUF;           // n x ldv: row j = v_j, zero beyond n
  float* X = Vr + n * ldv;            // n x ld, row-major; column t = eigenvector t
  float* d = X + n * ld;              // diagonal of T
  float* e = d + n;                   // off-diagonal of T: e[j] = T(j+1, j)
  float* e2 = e + n;                  // e^2
  float* tau = e2 + n;                // reflector scalars
  float* lam = tau + n;               // eigenvalues, ascending
  float* flag = lam + n;              // cluster starts
  const int tid = threadIdx.x, lane = tid % 32, warp = tid / 32;
  const int rs = lane / 16, cg = lane % 16;
  const bool hw = warp < WH;          // this warp takes part in the reduction

  // 1. Householder reduction.
  float a[NS][NT];
#pragma unroll
  for (int s = 0; s < NS; ++s)
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const int i = warp + WH * (rs + 2 * s), k = cg + 16 * t;
      a[s][t] = (hw && i < n && k < n) ? (float)S[(size_t)i * n + k] : 0.f;
    }
  // Column 0 below the diagonal (slot 0 of the lanes with cg = 0; xb is zero
  // at row 0 and beyond n) and the partial squared norms below row 1.
  if (hw) {
    float sg = 0.f;
    if (cg == 0)
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const int i = warp + WH * (rs + 2 * s);
        xb[i] = i > 0 ? a[s][0] : 0.f;
        if (i > 1) sg = fmaf(a[s][0], a[s][0], sg);
      }
    sg += __shfl_xor_sync(TE_FULL, sg, 16);
    if (lane == 0) part[warp] = sg;
  }
  __syncthreads();
  // Steps j = 16 P - 1 .. 16 P + 14 publish the columns c = j + 1 of slot P,
  // so P is a compile-time constant in their body: the publishing needs no
  // selects, and the slots that lie entirely above or left of the trailing
  // block are skipped without a branch (column slots t < P, row slots s < S0:
  // there v, p and w vanish, and xb and pb already hold the zeros read).
  static_for<0, NT + 1>([&](auto PC) {
    constexpr int P = decltype(PC)::value;
    if constexpr (P < NT) {
      constexpr int S0 = WH == 8 ? P : P / 2;
      const int jhi = min(16 * P + 15, n - 2);
      for (int j = P == 0 ? 0 : 16 * P - 1; j < jhi; ++j) {
        float t = 0.f, vk[NT], vi[NS], p[NS];
        if (hw) {
          const float sig = te_sum<WH>(part);
          const float alpha = xb[j + 1];
          float beta = alpha, scale = 0.f;
          if (sig > 0.f) {
            const float mu = sqrtf(fmaf(alpha, alpha, sig));
            beta = alpha <= 0.f ? mu : -mu;
            t = __fdividef(beta - alpha, beta);
            scale = __fdividef(1.f, alpha - beta);
          }
          if (tid == 0) {
            e[j] = beta;
            tau[j] = t;
          }
          // v_j(r) = 1 at r = j+1, x(r) * scale below, 0 elsewhere (xb is
          // zero at r <= j and beyond n).
          auto vval = [&](int r) -> float { return r == j + 1 ? 1.f : xb[r] * scale; };
          if (tid < ldv) Vr[j * ldv + tid] = t != 0.f ? vval(tid) : 0.f;
          if (t != 0.f) {  // uniform: every thread has the same sig
#pragma unroll
            for (int u = P; u < NT; ++u) vk[u] = vval(cg + 16 * u);
#pragma unroll
            for (int s = S0; s < NS; ++s) vi[s] = vval(warp + WH * (rs + 2 * s));
            // p = tau A v: register products, then a butterfly over the 16
            // lanes of the row group.
#pragma unroll
            for (int s = S0; s < NS; ++s) {
              float acc = 0.f;
#pragma unroll
              for (int u = P; u < NT; ++u) acc = fmaf(a[s][u], vk[u], acc);
              p[s] = acc;
            }
#pragma unroll
            for (int o = 1; o < 16; o <<= 1)
#pragma unroll
              for (int s = S0; s < NS; ++s) p[s] += __shfl_xor_sync(TE_FULL, p[s], o);
            // Rows <= j are outside the trailing block (their entries are stale).
            float pv = 0.f;
#pragma unroll
            for (int s = S0; s < NS; ++s) {
              const int i = warp + WH * (rs + 2 * s);
              p[s] = i > j ? t * p[s] : 0.f;
              pv = fmaf(p[s], vi[s], pv);
              if (cg == s) pb[i] = p[s];
            }
            pv += __shfl_xor_sync(TE_FULL, pv, 16);
            if (lane == 0) kpart[warp] = pv;
          }
        }
        __syncthreads();
        if (hw) {
          if (t != 0.f) {
            // w = p - K v, K = (tau/2) p^T v; A -= v w^T + w v^T.  Outside
            // the trailing block v, p and w vanish.
            const float kk = 0.5f * t * te_sum<WH>(kpart);
            float wk[NT];
#pragma unroll
            for (int u = P; u < NT; ++u) wk[u] = fmaf(-kk, vk[u], pb[cg + 16 * u]);
#pragma unroll
            for (int s = S0; s < NS; ++s) {
              const float wi = fmaf(-kk, vi[s], p[s]);
#pragma unroll
              for (int u = P; u < NT; ++u) a[s][u] = fmaf(-vi[s], wk[u], fmaf(-wi, vk[u], a[s][u]));
            }
          }
          // Column c = j+1 (slot P) below the diagonal, with the partial
          // squared norm below row c+1.
          const int c = j + 1;
          float sg = 0.f;
          if (cg == c % 16)
#pragma unroll
            for (int s = S0; s < NS; ++s) {
              const int i = warp + WH * (rs + 2 * s);
              xb[i] = i > c ? a[s][P] : 0.f;
              if (i > c + 1) sg = fmaf(a[s][P], a[s][P], sg);
            }
          sg += __shfl_xor_sync(TE_FULL, sg, 16);
          if (lane == c % 16) part[warp] = sg;
        }
        __syncthreads();
      }
    }
  });
  // T: the diagonal and the last off-diagonal entry from the registers.
  if (hw) {
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
      for (int u = 0; u < NT; ++u) {
        const int i = warp + WH * (rs + 2 * s), k = cg + 16 * u;
        if (i < n && k == i) d[i] = a[s][u];
        if (n >= 2 && i == n - 1 && k == n - 2) e[n - 2] = a[s][u];
      }
  }
  if (tid == 0 && n >= 2) tau[n - 2] = 0.f;
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
      lo = fminf(lo, __shfl_xor_sync(TE_FULL, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(TE_FULL, hi, o));
      nrm = fmaxf(nrm, __shfl_xor_sync(TE_FULL, nrm, o));
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
  // (d_i, e_{i-1}^2) interleaved for the Sturm counts, plus a zero pad entry
  // at n, in the space of xb and pb (free after the reduction; 2 TE_VBUF >=
  // 2 (n + 1) floats); e^2 is floored at 1e-30 max(1, ||T||^2).
  float2* de = reinterpret_cast<float2*>(xb);
  {
    const float e2min = 1e-30f * fmaxf(1.f, nrm * nrm);
    for (int i = tid; i <= n; i += TE_THREADS)
      de[i] = i < n ? make_float2(d[i], i > 0 ? fmaxf(e2[i - 1], e2min) : 0.f) : make_float2(0.f, 0.f);
  }
  __syncthreads();

  // 2. Multisection.  Grid point p (0 <= p <= TE_GRID + 1) is lo + hg p, with
  // count 0 at p = 0 and n at p = TE_GRID + 1 (the padded Gershgorin ends).
  const float glo = red[0], ghi = red[1];
  const float hg = (ghi - glo) / (float)(TE_GRID + 1);
  cnt[tid] = sturm_count(de, n, glo + hg * (float)(tid + 1));
  __syncthreads();
  {
    const int G = n <= TE_THREADS / 8 ? 8 : (n <= TE_THREADS / 4 ? 4 : (n <= TE_THREADS / 2 ? 2 : 1));
    const float width = 4.f * 1.1920929e-7f * nrm + 1e-30f;
    const int g = tid % G;
    const unsigned gmask = G == 32 ? TE_FULL : (((1u << G) - 1u) << (lane / G * G));
    for (int t = tid / G; t < n; t += TE_THREADS / G) {  // the G lanes of a group share t
      // Smallest grid point whose count exceeds t (counts taken as they are).
      int plo = 0, phi = TE_GRID + 1;
      while (phi - plo > 1) {
        const int mid = (plo + phi) / 2;
        if (cnt[mid - 1] > t) phi = mid; else plo = mid;
      }
      float a0 = plo == 0 ? glo : glo + hg * (float)plo;
      float b0 = phi == TE_GRID + 1 ? ghi : glo + hg * (float)phi;
      for (int it = 0; it < TE_MAXSECT && b0 - a0 > width; ++it) {
        // Points 1 .. 2G of the bracket; lane g tests 2g+1 and 2g+2.
        const float h = (b0 - a0) / (float)(2 * G + 1);
        int c0, c1;
        sturm_count2(de, n, a0 + h * (float)(2 * g + 1), a0 + h * (float)(2 * g + 2), c0, c1);
        const unsigned sh = lane / G * G;
        const unsigned any = (__ballot_sync(gmask, c0 > t || c1 > t) >> sh);
        const unsigned b0s = (__ballot_sync(gmask, c0 > t) >> sh);
        // First test point past eigenvalue t: the new bracket ends there.
        int f = 2 * G + 1;
        if (any) {
          const int gf = __ffs(any) - 1;
          f = 2 * gf + ((b0s >> gf) & 1u ? 1 : 2);
        }
        const float na = f == 1 ? a0 : a0 + h * (float)(f - 1);
        const float nb = f == 2 * G + 1 ? b0 : a0 + h * (float)f;
        a0 = na;
        b0 = nb;
      }
      if (g == 0) lam[t] = 0.5f * (a0 + b0);
    }
  }
  __syncthreads();

  // 3. Inverse iteration, thread t for eigenvalue t; the solution goes to
  // column t of X.  Factors of T - lambda I = L U: reciprocal pivots r_i and
  // multipliers m_i = e_{i-1} r_{i-1}.
  const float guard = 1.1920929e-7f * nrm + 1e-30f;
  for (int t = tid; t < n; t += TE_THREADS) {
    const float lm = lam[t];
    float r[TE_NMAX], ml[TE_NMAX];
    float qi = d[0] - lm;
    if (fabsf(qi) < guard) qi = qi < 0.f ? -guard : guard;
    r[0] = __fdividef(1.f, qi);
    ml[0] = 0.f;
    for (int i = 1; i < n; ++i) {
      const float mlt = e[i - 1] * r[i - 1];
      qi = d[i] - lm - mlt * e[i - 1];
      if (fabsf(qi) < guard) qi = qi < 0.f ? -guard : guard;
      r[i] = __fdividef(1.f, qi);
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
    flag[t] = (t == 0 || lam[t] - lam[t - 1] > 1e-3f * nrm) ? 1.f : 0.f;
  }
  __syncthreads();
  // Classical Gram-Schmidt twice inside each cluster, in eigenvalue order;
  // cluster number q goes to warp q mod 16.  Lane l holds rows l + 32 b.
  {
    int q = 0;
    for (int base = 0; base < n; base += 32) {
      const unsigned starts = __ballot_sync(TE_FULL, base + lane < n && flag[base + lane] != 0.f);
      unsigned rest = starts;
      while (rest) {
        const int c0 = base + __ffs(rest) - 1;
        rest &= rest - 1;
        // The cluster ends at the next start (possibly in a later chunk).
        int c1 = c0 + 1;
        if (rest) {
          c1 = base + __ffs(rest) - 1;
        } else {
          c1 = n;
          for (int nb = base + 32; nb < n; nb += 32) {
            const unsigned s2 = __ballot_sync(TE_FULL, nb + lane < n && flag[nb + lane] != 0.f);
            if (s2) {
              c1 = nb + __ffs(s2) - 1;
              break;
            }
          }
        }
        if (c1 - c0 > 1 && q % TE_WARPS == warp) {
          for (int t = c0 + 1; t < c1; ++t) {
            float xt[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) xt[b] = lane + 32 * b < n ? X[(lane + 32 * b) * ld + t] : 0.f;
            for (int pass = 0; pass < 2; ++pass) {
              float acc[NB];
#pragma unroll
              for (int b = 0; b < NB; ++b) acc[b] = 0.f;
              // Four projections per round (their sums share the butterfly).
              for (int s0 = c0; s0 < t; s0 += 4) {
                float xs[4][NB], dot[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  dot[u] = 0.f;
#pragma unroll
                  for (int b = 0; b < NB; ++b) {
                    xs[u][b] = (s0 + u < t && lane + 32 * b < n) ? X[(lane + 32 * b) * ld + s0 + u] : 0.f;
                    dot[u] = fmaf(xs[u][b], xt[b], dot[u]);
                  }
                }
                te_warp_sum<4>(dot);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                  for (int b = 0; b < NB; ++b) acc[b] = fmaf(dot[u], xs[u][b], acc[b]);
              }
#pragma unroll
              for (int b = 0; b < NB; ++b) xt[b] -= acc[b];
            }
            float ss[1] = {0.f};
#pragma unroll
            for (int b = 0; b < NB; ++b) ss[0] = fmaf(xt[b], xt[b], ss[0]);
            te_warp_sum<1>(ss);
            const float inv = ss[0] > 0.f ? rsqrtf(ss[0]) : 0.f;
#pragma unroll
            for (int b = 0; b < NB; ++b)
              if (lane + 32 * b < n) X[(lane + 32 * b) * ld + t] = xt[b] * inv;
            __syncwarp();
          }
        }
        ++q;
      }
    }
  }
  __syncthreads();

  // 4. Back-transformation, H_{n-3} first and H_0 last, four reflectors at
  // a time.  For a block k_q = n-3-4b-q (q = 0..3, applied in that order)
  // the projections of the partly transformed x follow from those of x:
  // d_q = v_q^T x - sum_{p<q} tau_p d_p (v_q^T v_p), and then
  // x <- x - sum_q tau_q d_q v_q.  The couplings v_q^T v_p come first (one
  // warp per dot; cpl reuses the grid counts).  A warp takes a tile of 8
  // eigenvectors (c = 8 tile + lane % 8); the four lane groups g = lane / 8
  // hold the rows r = rpl g + m, m < rpl = ldv / 4, of its vector, so each
  // projection is a register sum plus two butterfly steps.  Reflector rows
  // are zero beyond n (and entirely for tau = 0).
  float* cpl = reinterpret_cast<float*>(cnt);  // [6 * blocks]
  const int nblk = (n - 2 + 3) / 4;
  for (int qd = warp; qd < 6 * nblk; qd += TE_WARPS) {
    const int idx = qd % 6, q1 = idx < 1 ? 1 : (idx < 3 ? 2 : 3), q2 = idx - q1 * (q1 - 1) / 2;
    const int k1 = n - 3 - 4 * (qd / 6) - q1, k2 = n - 3 - 4 * (qd / 6) - q2;
    float acc[1] = {0.f};
    if (k1 >= 0)
      for (int r = lane; r < ldv; r += 32) acc[0] = fmaf(Vr[k1 * ldv + r], Vr[k2 * ldv + r], acc[0]);
    te_warp_sum<1>(acc);
    if (lane == 0) cpl[qd] = acc[0];
  }
  __syncthreads();
  {
    constexpr int RMAX = 8 * NB;  // rpl <= RMAX
    const int rpl = ldv / 4, g = lane / 8, r0 = rpl * g;
    for (int tile = warp; tile * 8 < n; tile += TE_WARPS) {
      const int c = 8 * tile + lane % 8;
      float xv[RMAX];
#pragma unroll
      for (int m = 0; m < RMAX; ++m) xv[m] = (m < rpl && c < n && r0 + m < n) ? X[(r0 + m) * ld + c] : 0.f;
      for (int b = 0; b < nblk; ++b) {
        const int kb = n - 3 - 4 * b;
        float tq[4], gq[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          tq[q] = kb - q >= 0 ? tau[kb - q] : 0.f;
          gq[q] = 0.f;
        }
#pragma unroll
        for (int m4 = 0; m4 < RMAX / 4; ++m4)
          if (4 * m4 < rpl)
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (kb - q >= 0) {
                const float4 v = reinterpret_cast<const float4*>(Vr + (kb - q) * ldv + r0)[m4];
                gq[q] = fmaf(v.x, xv[4 * m4], gq[q]);
                gq[q] = fmaf(v.y, xv[4 * m4 + 1], gq[q]);
                gq[q] = fmaf(v.z, xv[4 * m4 + 2], gq[q]);
                gq[q] = fmaf(v.w, xv[4 * m4 + 3], gq[q]);
              }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          gq[q] += __shfl_xor_sync(TE_FULL, gq[q], 8);
          gq[q] += __shfl_xor_sync(TE_FULL, gq[q], 16);
        }
        const float* cb = cpl + 6 * b;
        float dq[4];
        dq[0] = gq[0];
        dq[1] = fmaf(-tq[0] * dq[0], cb[0], gq[1]);
        dq[2] = fmaf(-tq[1] * dq[1], cb[2], fmaf(-tq[0] * dq[0], cb[1], gq[2]));
        dq[3] = fmaf(-tq[2] * dq[2], cb[5], fmaf(-tq[1] * dq[1], cb[4], fmaf(-tq[0] * dq[0], cb[3], gq[3])));
#pragma unroll
        for (int q = 0; q < 4; ++q) dq[q] *= -tq[q];
#pragma unroll
        for (int m4 = 0; m4 < RMAX / 4; ++m4)
          if (4 * m4 < rpl)
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (kb - q >= 0) {
                const float4 v = reinterpret_cast<const float4*>(Vr + (kb - q) * ldv + r0)[m4];
                xv[4 * m4] = fmaf(dq[q], v.x, xv[4 * m4]);
                xv[4 * m4 + 1] = fmaf(dq[q], v.y, xv[4 * m4 + 1]);
                xv[4 * m4 + 2] = fmaf(dq[q], v.z, xv[4 * m4 + 2]);
                xv[4 * m4 + 3] = fmaf(dq[q], v.w, xv[4 * m4 + 3]);
              }
      }
#pragma unroll
      for (int m = 0; m < RMAX; ++m)
        if (m < rpl && c < n && r0 + m < n) X[(r0 + m) * ld + c] = xv[m];
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += TE_THREADS) diag_out[i] = lam[i];
  for (int idx = tid; idx < n * n; idx += TE_THREADS) V_out[idx] = X[(idx / n) * ld + idx % n];
}

namespace {
using TeKernel = void (*)(const double*, int, float*, float*);
// Column slots per lane: n <= 16 NT.
int te_slots(int n) {
  const int nt = (n + 15) / 16;
  return nt <= 2 ? 2 : nt <= 4 ? 4 : nt <= 6 ? nt : nt <= 8 ? 8 : 10;
}
TeKernel te_kernel(int n) {
  switch (te_slots(n)) {
    case 2: return tridiag_eig_kernel<2>;
    case 4: return tridiag_eig_kernel<4>;
    case 5: return tridiag_eig_kernel<5>;
    case 6: return tridiag_eig_kernel<6>;
    case 8: return tridiag_eig_kernel<8>;
    default: return tridiag_eig_kernel<10>;
  }
}
}  // namespace

int tridiag_eig_prepare() {
  for (int n : {32, 64, 80, 96, 128, TE_NMAX}) ATK_TRY(raise_smem_limit((const void*)te_kernel(n), tridiag_eig_smem(n)));
  return ATK_OK;
}

int tridiag_eig_f32(const double* S, int n, float* diag_out, float* V_out, cudaStream_t st) {
  if (n < 1 || n > TE_NMAX) {
    set_error("tridiag_eig: need 1 <= n <= 160");
    return ATK_EUNSUPPORTED;
  }
  te_kernel(n)<<<1, TE_THREADS, tridiag_eig_smem(n), st>>>(S, n, diag_out, V_out);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
