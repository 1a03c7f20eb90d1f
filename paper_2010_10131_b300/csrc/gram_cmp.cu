// Compensated Gram S = Y_(n) Y_(n)^T (Alg. 2, EIG branch) over the stride
// view (Sec. V): float32 products made exact and summed as float-float pairs.
//
// Why: a float32 accumulator carries an absolute error of about eps_32 times
// the largest partial sum it holds.  For the first mode of a tensor whose
// entries are of comparable size those errors are many small, independent
// roundings and stay far below the eigenvalue gaps that matter.  A later mode
// works on the shrinking core of st-HOSVD, whose energy sits in a few large
// entries: one product can be ~lambda_1 / n^(1/2) and its float32 rounding
// alone is then ~eps_32 lambda_1, which swamps a cut whose gap is a tiny
// fraction of lambda_1 (a spectrum decaying like k^-3 at R = 128).  Here each
// term a b is split exactly into p + e (p = fl(a b), e = fma(a, b, -p)), p is
// added to the running pair by TwoSum (Knuth, TAOCP 4.2.2) and e joins the
// low word, so a partial sum holds about 48 bits whatever the term sizes.
// The partial tiles (pairs) of the split-K are summed in split order as
// float-float pairs and rounded once to float64: deterministic, like the
// float32 path.
//
// 256 threads as a 16 x 16 grid over a 64 x 64 output tile, 4 x 4 pairs per
// thread, 16-deep k tiles staged through double-buffered shared memory by the
// view loader of the float32 kernels (fp32_ops.cu).  Upper-triangle tiles
// only.  About nine float32 operations per term instead of one FMA: the plan
// runs it only when a later mode's cut is not resolved by the float32 Gram.
#include <algorithm>

#include "atk_internal.cuh"

namespace atk {

namespace {
constexpr int CB = 64;       // output tile rows = cols
constexpr int CT = 4;        // rows / cols per thread
constexpr int CNT = 256;     // threads
constexpr int CK = 16;       // k-tile depth
constexpr int CPAD = 4;
constexpr int CLD = CB + CPAD;

// (hi, lo) += a b: exact product, TwoSum into hi, the two error terms into lo.
// The _rn intrinsics keep the compiler from contracting p into the sum.
__device__ __forceinline__ void acc_prod(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// Stage a CK x CB tile of the view: k = c (the other index), m = i (mode
// index), into s[k * CLD + m]; zero outside the view.  Lanes run along
// whichever index is contiguous in memory.
struct CmpLoader {
  static constexpr int PER = CK * CB / CNT;  // 4
  const float* y;
  int lo, n, c_end, i0;
  int km, mm, step;
  bool lanes_on_m;
  float r[PER];
  __device__ void init(const float* y_, int64_t lo_, int64_t n_, int64_t c_end_, int64_t i0_) {
    y = y_; lo = (int)lo_; n = (int)n_; c_end = (int)c_end_; i0 = (int)i0_;
    lanes_on_m = lo == 1;
    const int t = threadIdx.x;
    if (lanes_on_m) { mm = t % CB; km = t / CB; step = CNT / CB; }
    else { km = t % CK; mm = t / CK; step = CNT / CK; }
  }
  __device__ void fetch(int c0) {
    if (lanes_on_m) {
      const int i = i0 + mm;
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const int c = c0 + km + e * step;
        r[e] = (c < c_end && i < n) ? __ldg(y + ((int64_t)i + (int64_t)n * c)) : 0.f;
      }
    } else {
      const int c = c0 + km;
      const bool cv = c < c_end;
      const int a = cv ? c % lo : 0, b = cv ? c / lo : 0;
      const float* base = y + ((int64_t)a + (int64_t)lo * n * b);
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const int i = i0 + mm + e * step;
        r[e] = (cv && i < n) ? __ldg(base + (int64_t)lo * i) : 0.f;
      }
    }
  }
  __device__ void store(float* s) const {
    if (lanes_on_m) {
#pragma unroll
      for (int e = 0; e < PER; ++e) s[(km + e * step) * CLD + mm] = r[e];
    } else {
#pragma unroll
      for (int e = 0; e < PER; ++e) s[km * CLD + mm + e * step] = r[e];
    }
  }
};

// One CTA per (upper-triangle tile, split); partial pairs to part_hi /
// part_lo at ((split * ntiles + tile) * CB + row) * CB + col.
__global__ void __launch_bounds__(CNT) gram_cmp_kernel(const float* __restrict__ y, int64_t lo, int64_t n, int64_t hi,
                                                       int T, int64_t kc, float* __restrict__ part_hi,
                                                       float* __restrict__ part_lo) {
  __shared__ __align__(16) float sA[2][CK * CLD];
  __shared__ __align__(16) float sB[2][CK * CLD];
  const int split = blockIdx.y;
  int ti = 0, id = blockIdx.x;
  while (id >= T - ti) { id -= T - ti; ++ti; }
  const int tj = ti + id;
  const bool diag = ti == tj;
  const int64_t J = lo * hi;
  const int64_t cb = (int64_t)split * kc, ce = min(J, cb + kc);
  CmpLoader la, lb;
  la.init(y, lo, n, ce, (int64_t)ti * CB);
  lb.init(y, lo, n, ce, (int64_t)tj * CB);
  float ah[CT][CT], al[CT][CT];
#pragma unroll
  for (int u = 0; u < CT; ++u)
#pragma unroll
    for (int v = 0; v < CT; ++v) ah[u][v] = al[u][v] = 0.f;
  const int tx = threadIdx.x % (CB / CT), ty = threadIdx.x / (CB / CT);
  const int ntile = cb < ce ? (int)((ce - cb + CK - 1) / CK) : 0;
  if (ntile > 0) {
    la.fetch((int)cb);
    la.store(sA[0]);
    if (!diag) {
      lb.fetch((int)cb);
      lb.store(sB[0]);
    }
    __syncthreads();
    for (int t = 0; t < ntile; ++t) {
      const int buf = t & 1;
      if (t + 1 < ntile) {
        la.fetch((int)cb + (t + 1) * CK);
        if (!diag) lb.fetch((int)cb + (t + 1) * CK);
      }
      const float* A = sA[buf];
      const float* B = diag ? sA[buf] : sB[buf];
#pragma unroll 4
      for (int k = 0; k < CK; ++k) {
        float a[CT], b[CT];
#pragma unroll
        for (int u = 0; u < CT; ++u) a[u] = A[k * CLD + ty * CT + u];
#pragma unroll
        for (int v = 0; v < CT; ++v) b[v] = B[k * CLD + tx * CT + v];
#pragma unroll
        for (int u = 0; u < CT; ++u)
#pragma unroll
          for (int v = 0; v < CT; ++v) acc_prod(a[u], b[v], ah[u][v], al[u][v]);
      }
      if (t + 1 < ntile) {
        la.store(sA[buf ^ 1]);
        if (!diag) lb.store(sB[buf ^ 1]);
      }
      __syncthreads();
    }
  }
  const int ntiles = T * (T + 1) / 2;
  const int64_t base = ((int64_t)split * ntiles + blockIdx.x) * (CB * CB);
#pragma unroll
  for (int u = 0; u < CT; ++u)
#pragma unroll
    for (int v = 0; v < CT; ++v) {
      const int64_t o = base + (int64_t)(ty * CT + u) * CB + tx * CT + v;
      part_hi[o] = ah[u][v];
      part_lo[o] = al[u][v];
    }
}

// S (n x n, float64, full symmetric) from the partial pairs, summed in split
// order as a float-float pair.
__global__ void reduce_cmp_kernel(const float* __restrict__ part_hi, const float* __restrict__ part_lo, int ns,
                                  int T, int64_t n, double* __restrict__ S) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  if (i > j) return;
  const int ti = (int)(i / CB), tj = (int)(j / CB);
  const int tile = ti * T - ti * (ti - 1) / 2 + (tj - ti);
  const int ntiles = T * (T + 1) / 2;
  const int64_t o = (int64_t)tile * CB * CB + (i - (int64_t)ti * CB) * CB + (j - (int64_t)tj * CB);
  const int64_t stride = (int64_t)ntiles * CB * CB;
  FFSum acc;
  for (int sp = 0; sp < ns; ++sp) {
    acc.add(part_hi[o + sp * stride]);
    acc.add(part_lo[o + sp * stride]);
  }
  const double s = acc.value();
  S[i + n * j] = s;
  S[j + n * i] = s;
}

struct CmpPlan {
  int T, nt, ns;
  int64_t kc;
};
// Enough splits for about four resident CTAs per SM, each split's k range a
// multiple of CK; the partials must fit in `budget` bytes (at least one split).
CmpPlan cmp_plan(const View& v, size_t budget) {
  CmpPlan g;
  g.T = (int)ceil_div(v.n, CB);
  g.nt = g.T * (g.T + 1) / 2;
  const size_t per_split = (size_t)g.nt * CB * CB * 2 * sizeof(float);
  const int64_t J = v.J();
  int64_t ns = std::max<int64_t>(1, (int64_t)4 * num_sms() / g.nt);
  ns = std::min<int64_t>(ns, std::max<int64_t>(1, ceil_div(J, CK)));
  if (budget) ns = std::min<int64_t>(ns, std::max<int64_t>(1, (int64_t)(budget / per_split)));
  g.kc = ceil_div(ceil_div(J, ns), CK) * CK;
  g.ns = (int)ceil_div(J, g.kc);
  return g;
}
}  // namespace

size_t gram_cmp_scratch_bytes(const View& v) {
  const CmpPlan g = cmp_plan(v, 0);
  return (size_t)g.ns * g.nt * CB * CB * 2 * sizeof(float);
}

int gram_cmp(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (v.n <= 0) return ATK_OK;
  if (v.J() == 0) {
    ATK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * v.n * v.n, st));
    return ATK_OK;
  }
  if (v.size() >= ((int64_t)1 << 31)) {
    set_error("gram_cmp: the view must have fewer than 2^31 elements");
    return ATK_EUNSUPPORTED;
  }
  const CmpPlan g = cmp_plan(v, scratch_bytes);
  const size_t half = (size_t)g.ns * g.nt * CB * CB;
  if (2 * half * sizeof(float) > scratch_bytes) {
    set_error("gram_cmp: scratch too small for one split");
    return ATK_EINVAL;
  }
  gram_cmp_kernel<<<dim3(g.nt, g.ns), CNT, 0, st>>>(y, v.lo, v.n, v.hi, g.T, g.kc, scratch, scratch + half);
  ATK_LAUNCHED();
  reduce_cmp_kernel<<<(unsigned)ceil_div(v.n * v.n, 256), 256, 0, st>>>(scratch, scratch + half, g.ns, g.T, v.n, S);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
