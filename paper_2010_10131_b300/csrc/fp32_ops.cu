// Matricization-free mode-n contractions on the CUDA cores, float32
// (Sec. V; Alg. 2 and Alg. 3).
//
// Every contraction on the hot path is one of two shapes over the mode-n view
// (lo, n, hi) of a column-major tensor, with c = a + lo*b the "other" index:
//   CI  C[i][j] = sum_c A(c, i) B(c, j)  -- contraction over c (TTT, Eq. 3):
//       the Gram S = Y_(n) Y_(n)^T, and the ALS products Y P and P^T P.
//   CO  O(c, r) = sum_i A(c, i) M[i][r]  -- contraction over i (TTM, Eq. 2):
//       the truncating TTM Y x_n U^T, the ALS product Y^T L~, and the ALS
//       core update.
// Both are one register-tiled kernel: 256 threads, a BM x BN output tile,
// 16-deep k tiles staged through double-buffered shared memory.  Each thread
// holds a TM x TN register block.  The loaders read the tensor in place through
// the stride view.  Lanes run along whichever index is contiguous in memory:
// i when lo == 1, c otherwise.  So no unfolding is ever materialised.
// CI outputs are split over c (split-K) into float32 partial tiles.  A second
// kernel sums them in a fixed order as float-float pairs (about 48 bits),
// rounded once to float64, so results are deterministic and no plain float32
// sum runs longer than one split (<= 8192 terms).
#include <algorithm>

#include "async_copy.cuh"
#include "atk_internal.cuh"
#include "fp32_block.cuh"

namespace atk {

constexpr int SPLIT_MAX_K = 8192;

// ------------------------------------------------------------------ loaders
// Each loader fetches a TK x W tile (k rows, W contiguous m columns in smem)
// into registers, then stores it to shared memory as s[k * (W + PAD) + m].

// A view operand with k = c (the other index) and m = i (mode index): CI role.
// Index state is 32-bit: every tensor the library accepts has fewer than 2^31
// elements, so every offset below fits.  When lo == 1, n % 4 == 0 and the
// tensor is 16-byte aligned (the first mode of any tensor with I_1 % 4 == 0),
// the VEC instantiation moves four consecutive i per thread per load and per
// store (128-bit accesses): a quarter of the load and store instructions,
// which compete with the FMAs for issue slots.  The caller checks those
// conditions (kc_vec_ok) before it picks VEC.
template <int W, bool VEC = false>
struct ViewLoaderKC {
  static constexpr int PER = TK * W / NT;
  static constexpr int PER4 = (TK * (W / 4) + NT - 1) / NT;  // float4 per thread (vector path)
  const float* y;
  int lo, n, c_end, i0;
  bool lanes_on_m;  // lo == 1: m (= i) is contiguous
  bool vec;
  int km, mm, step;
  float r[VEC ? 4 * PER4 : PER];
  __device__ void init(const float* y_, int64_t lo_, int64_t n_, int64_t c_end_, int64_t i0_) {
    y = y_; lo = (int)lo_; n = (int)n_; c_end = (int)c_end_; i0 = (int)i0_;
    lanes_on_m = (lo == 1);
    vec = VEC;
    int t = threadIdx.x;
    if (VEC) { mm = 4 * (t % (W / 4)); km = t / (W / 4); step = NT / (W / 4); }
    else if (lanes_on_m) { mm = t % W; km = t / W; step = NT / W; }
    else { km = t % TK; mm = t / TK; step = NT / TK; }
  }
  __device__ void fetch(int64_t c0_) {
    const int c0 = (int)c0_;
    if (VEC) {
      const int i = i0 + mm;
#pragma unroll
      for (int e = 0; e < PER4; ++e) {
        const int k = km + e * step;
        const int c = c0 + k;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < TK && c < c_end && i < n) v = __ldg(reinterpret_cast<const float4*>(y + (i + n * c)));
        r[4 * e] = v.x; r[4 * e + 1] = v.y; r[4 * e + 2] = v.z; r[4 * e + 3] = v.w;
      }
    } else if (lanes_on_m) {
      const int i = i0 + mm;
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        int c = c0 + km + e * step;
        r[e] = (c < c_end && i < n) ? __ldg(y + (i + n * c)) : 0.f;
      }
    } else {
      int c = c0 + km;
      bool cv = c < c_end;
      int a = cv ? c % lo : 0, b = cv ? c / lo : 0;
      const float* base = y + (a + lo * n * b);
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        int i = i0 + mm + e * step;
        r[e] = (cv && i < n) ? __ldg(base + lo * i) : 0.f;
      }
    }
  }
  __device__ void store(float* s) const {
    if (VEC) {
#pragma unroll
      for (int e = 0; e < PER4; ++e) {
        const int k = km + e * step;
        if (k < TK)
          *reinterpret_cast<float4*>(s + k * (W + PAD) + mm) =
              make_float4(r[4 * e], r[4 * e + 1], r[4 * e + 2], r[4 * e + 3]);
      }
    } else if (lanes_on_m) {
#pragma unroll
      for (int e = 0; e < PER; ++e) s[(km + e * step) * (W + PAD) + mm] = r[e];
    } else {
#pragma unroll
      for (int e = 0; e < PER; ++e) s[km * (W + PAD) + mm + e * step] = r[e];
    }
  }
};

// A view operand with k = i (mode index) and m = c (other index): CO role.
template <int W>
struct ViewLoaderKI {
  static constexpr int PER = TK * W / NT;
  const float* y;
  int lo, n, J, c0, cbase_off;
  bool lanes_on_k;  // lo == 1: k (= i) is contiguous
  bool cvalid;
  int km, mm, step;
  float r[PER];
  __device__ void init(const float* y_, int64_t lo_, int64_t n_, int64_t J_, int64_t c0_) {
    y = y_; lo = (int)lo_; n = (int)n_; J = (int)J_; c0 = (int)c0_;
    lanes_on_k = (lo == 1);
    int t = threadIdx.x;
    if (lanes_on_k) { km = t % TK; mm = t / TK; step = NT / TK; }
    else {
      mm = t % W; km = t / W; step = NT / W;
      int c = c0 + mm;
      cvalid = c < J;
      cbase_off = cvalid ? (c % lo) + lo * n * (c / lo) : 0;
    }
  }
  __device__ void fetch(int64_t i0_) {
    const int i0 = (int)i0_;
    if (lanes_on_k) {
      int i = i0 + km;
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        int c = c0 + mm + e * step;
        r[e] = (i < n && c < J) ? __ldg(y + (i + n * c)) : 0.f;
      }
    } else {
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        int i = i0 + km + e * step;
        r[e] = (cvalid && i < n) ? __ldg(y + (cbase_off + lo * i)) : 0.f;
      }
    }
  }
  __device__ void store(float* s) const {
    if (lanes_on_k) {
#pragma unroll
      for (int e = 0; e < PER; ++e) s[km * (W + PAD) + mm + e * step] = r[e];
    } else {
#pragma unroll
      for (int e = 0; e < PER; ++e) s[(km + e * step) * (W + PAD) + mm] = r[e];
    }
  }
};

// Dense column-major n x R matrix M, k = row i, m = column r (CO B operand).
template <int W>
struct MatLoader {
  static constexpr int PER = (TK * W + NT - 1) / NT;
  const float* M;
  int64_t n, R, r0;
  int km, mm;
  float r[PER];
  __device__ void init(const float* M_, int64_t n_, int64_t R_, int64_t r0_) {
    M = M_; n = n_; R = R_; r0 = r0_;
    km = threadIdx.x % TK; mm = threadIdx.x / TK;
  }
  __device__ void fetch(int64_t i0) {
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      int m = mm + e * (NT / TK);
      int64_t i = i0 + km, rr = r0 + m;
      r[e] = (m < W && i < n && rr < R) ? __ldg(M + i + n * rr) : 0.f;
    }
  }
  __device__ void store(float* s) const {
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      int m = mm + e * (NT / TK);
      if (m < W) s[km * (W + PAD) + m] = r[e];
    }
  }
};

// ------------------------------------------------------------- CI kernels
// Gram: C = sum_c Y(c, :)^T Y(c, :), upper-triangle tiles only; one partial
// tile (row-major BM x BM, float32) per (tile, split), indexed by the tile's
// row-major position in the upper triangle.  Diagonal and off-diagonal tiles
// are separate launches (DIAG): a diagonal tile loads one operand and uses it
// twice, and neither instantiation carries the other's registers.
template <int BM, int TM, bool DIAG, bool VEC>
__global__ void __launch_bounds__(NT, 2)
gram_ci_kernel(const float* __restrict__ y, int64_t lo, int64_t n, int64_t hi, int T, int64_t kc,
               float* __restrict__ part, int64_t c_base = 0) {
  constexpr int SA = TK * (BM + PAD);
  __shared__ __align__(16) float sA[2 * SA];
  __shared__ __align__(16) float sB[DIAG ? 1 : 2 * SA];
  const int split = blockIdx.y;
  int ti, tj;
  if (DIAG) {
    ti = tj = blockIdx.x;
  } else {
    // blockIdx.x enumerates the strict upper triangle row by row
    int id = blockIdx.x;
    ti = 0;
    while (id >= T - 1 - ti) { id -= T - 1 - ti; ++ti; }
    tj = ti + 1 + id;
  }
  const int tile = ti * T - ti * (ti - 1) / 2 + (tj - ti);
  const int64_t J = lo * hi;
  const int64_t cb = c_base + (int64_t)split * kc, ce = min(J, cb + kc);
  ViewLoaderKC<BM, VEC> la, lb;
  la.init(y, lo, n, ce, (int64_t)ti * BM);
  if (!DIAG) lb.init(y, lo, n, ce, (int64_t)tj * BM);
  Block<BM, BM, TM, TM> blk;
  blk.init();
  const int64_t ntile = cb < ce ? (ce - cb + TK - 1) / TK : 0;
  if (ntile > 0) {
    la.fetch(cb);
    la.store(sA);
    if (!DIAG) {
      lb.fetch(cb);
      lb.store(sB);
    }
    __syncthreads();
    for (int64_t t = 0; t < ntile; ++t) {
      const int buf = t & 1;
      if (t + 1 < ntile) {
        la.fetch(cb + (t + 1) * TK);
        if (!DIAG) lb.fetch(cb + (t + 1) * TK);
      }
      if (DIAG) blk.template mma<true>(sA + buf * SA, sA + buf * SA);
      else blk.mma(sA + buf * SA, sB + buf * SA);
      if (t + 1 < ntile) {
        la.store(sA + (buf ^ 1) * SA);
        if (!DIAG) lb.store(sB + (buf ^ 1) * SA);
      }
      __syncthreads();
    }
  }
  const int ntiles = T * (T + 1) / 2;
  float* out = part + ((int64_t)split * ntiles + tile) * (BM * BM);
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TM; ++v)
      out[Block<BM, BM, TM, TM>::row_of(blk.ty, u) * BM + Block<BM, BM, TM, TM>::col_of(blk.tx, v)] = blk.acc(u, v);
}

// The vector loader's conditions: the mode-n index is contiguous (lo == 1),
// rows of four floats stay inside one column (n % 4 == 0), and the base is
// 16-byte aligned.
static bool kc_vec_ok(const float* y, const View& v) {
  return v.lo == 1 && v.n % 4 == 0 && (reinterpret_cast<uintptr_t>(y) & 15) == 0;
}

// c_base: the first c of split 0 (a round of a split-K that runs in several
// rounds; 0 otherwise).
template <int BM, int TM, bool VEC>
static void launch_gram_tiles_v(const float* y, const View& v, int T, int ns_d, int64_t kc_d, int ns_o,
                                int64_t kc_o, float* part, cudaStream_t st, int64_t c_base) {
  gram_ci_kernel<BM, TM, true, VEC><<<dim3(T, ns_d), NT, 0, st>>>(y, v.lo, v.n, v.hi, T, kc_d, part, c_base);
  if (T > 1)
    gram_ci_kernel<BM, TM, false, VEC><<<dim3(T * (T - 1) / 2, ns_o), NT, 0, st>>>(y, v.lo, v.n, v.hi, T, kc_o,
                                                                                    part, c_base);
}
template <int BM, int TM>
static void launch_gram_tiles(const float* y, const View& v, int T, int ns_d, int64_t kc_d, int ns_o, int64_t kc_o,
                              float* part, cudaStream_t st, int64_t c_base = 0) {
  if (kc_vec_ok(y, v)) launch_gram_tiles_v<BM, TM, true>(y, v, T, ns_d, kc_d, ns_o, kc_o, part, st, c_base);
  else launch_gram_tiles_v<BM, TM, false>(y, v, T, ns_d, kc_d, ns_o, kc_o, part, st, c_base);
}

// Cross product C (n x R) = sum_c Y(c, i) P(c, r), P a (lo, R, hi) tensor.
template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(NT, 2)
cross_ci_kernel(const float* __restrict__ y, const float* __restrict__ p, int64_t lo, int64_t n, int64_t hi,
                int64_t R, int TR, int64_t kc, float* __restrict__ part) {
  __shared__ __align__(16) float sA[2][TK * (BM + PAD)];
  __shared__ __align__(16) float sB[2][TK * (BN + PAD)];
  int tile = blockIdx.x, split = blockIdx.y;
  int ti = tile / TR, tr = tile % TR;
  const int64_t J = lo * hi;
  const int64_t cb = (int64_t)split * kc, ce = min(J, cb + kc);
  ViewLoaderKC<BM> la;
  ViewLoaderKC<BN> lb;
  la.init(y, lo, n, ce, (int64_t)ti * BM);
  lb.init(p, lo, R, ce, (int64_t)tr * BN);
  Block<BM, BN, TM, TN> blk;
  blk.init();
  const int64_t ntile = cb < ce ? (ce - cb + TK - 1) / TK : 0;
  if (ntile > 0) {
    la.fetch(cb);
    lb.fetch(cb);
    la.store(sA[0]);
    lb.store(sB[0]);
    __syncthreads();
    for (int64_t t = 0; t < ntile; ++t) {
      const int buf = t & 1;
      if (t + 1 < ntile) {
        la.fetch(cb + (t + 1) * TK);
        lb.fetch(cb + (t + 1) * TK);
      }
      blk.mma(sA[buf], sB[buf]);
      if (t + 1 < ntile) {
        la.store(sA[buf ^ 1]);
        lb.store(sB[buf ^ 1]);
      }
      __syncthreads();
    }
  }
  float* out = part + ((int64_t)split * gridDim.x + tile) * (BM * BN);
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TN; ++v)
      out[Block<BM, BN, TM, TN>::row_of(blk.ty, u) * BN + Block<BM, BN, TM, TN>::col_of(blk.tx, v)] =
          blk.acc(u, v);
}

// p[0], p[stride], ..., p[(count-1) stride] summed in that order as a
// float-float pair.  The loads go out eight at a time ahead of the adds, so a
// long split count costs a few memory latencies rather than one per split.
__device__ __forceinline__ FFSum ff_sum_splits(const float* __restrict__ p, int64_t stride, int count) {
  FFSum acc;
  int sp = 0;
  for (; sp + 8 <= count; sp += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = p[(int64_t)(sp + u) * stride];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc.add(v[u]);
  }
  for (; sp < count; ++sp) acc.add(p[(int64_t)sp * stride]);
  return acc;
}

// ----------------------------------------- cp.async-fed Gram (mode-1 views)
// All upper-triangle 128 x 128 tiles of a view whose rows c are I_n
// contiguous floats (lo == 1, I_n % 4 == 0, 16-byte aligned base), diagonal
// ones included, in one launch.  A stage is GA_TK values of c: per operand,
// GA_TK rows of 128 floats moved by 16-byte cp.async copies straight into the
// k-major tile the register block reads (s[k * (128 + PAD) + i]), with no
// register staging and no staging stores; GA_NS - 1 stages are in flight
// while one is consumed, which covers the HBM latency.  The tile index runs
// fastest in the grid, so the T (T + 1) / 2 tiles of a split run side by side
// and each input row comes from HBM about once (its other uses hit L2).
// Diagonal tiles copy one operand and compute only the 4 x 4 blocks that meet
// the upper triangle (gram_async_diag); the reduction reads nothing else of
// them.  Out-of-range rows (c >= end of the split, i >= I_n) are zero-filled.
constexpr int GA_TK = TK;
constexpr int GA_NS = 4;
constexpr int GA_LD = 128 + PAD;
constexpr int GA_STAGE = 2 * GA_TK * GA_LD;  // floats per stage: A and B tiles
constexpr int GA_SMEM = GA_NS * GA_STAGE * (int)sizeof(float);

// A diagonal 128 x 128 tile as 4 x 4 blocks (bi, bj), bi, bj < 32: the
// blocks at or above the diagonal are the 256 of the top-right quadrant and
// the 136 + 136 upper ones of the two diagonal 64 x 64 quadrants.  Thread t
// takes top-right block (t / 16, t % 16) and one block of the diagonal
// quadrants: those 272 are 16 "pairs" of 17 (quadrant row p with row 15 - p,
// p < 8, which hold 16 - p and p + 1 blocks), thread t block t % 16 of pair
// t / 16, and the lanes l < 16 of one warp (it rotates with the CTA, to
// spread the extra work over the SM sub-partitions) the 17th block of pair l.
// Every warp's fragment loads touch at most 16 distinct 16-byte chunks of a
// stage row, as in the full-tile layout, and a thread holds 16 or 24 packed
// accumulators (8 per block): 7 of 8 warps issue 16 packed FMAs per k
// instead of 24.  Each block loads its own fragments, twice the loads per FMA
// of the full-tile layout, so a diagonal CTA is bound by shared memory rather
// than by the FMA pipe (measured: 4 % faster on a 128-row view, not 29 %).
struct DiagBlocks {
  int ra[3], cb[3];  // first row and column of each block in the tile
  bool extra;        // this warp takes the 17th blocks
  __device__ explicit DiagBlocks(int tid, unsigned cta) {
    const int warp = tid >> 5, lane = tid & 31;
    ra[0] = 4 * (tid >> 4);
    cb[0] = 64 + 4 * (tid & 15);
    {
      const int P = tid >> 4, q = tid & 15, p = P & 7, off = P < 8 ? 0 : 64;
      const bool first = q < 16 - p;
      ra[1] = off + 4 * (first ? p : 15 - p);
      cb[1] = off + 4 * (first ? p + q : q - 1);
    }
    {
      const int P = lane & 15, off = P < 8 ? 0 : 64;
      ra[2] = off + 4 * (15 - (P & 7));
      cb[2] = off + 60;
    }
    extra = warp == (int)(cta & 7u);
  }
};

// One 4 x 4 block's outer product for row k of a stage.
__device__ __forceinline__ void diag_block_step(const float* s, int ra, int cb, unsigned long long (&d)[4][2]) {
  const float4 a = *reinterpret_cast<const float4*>(s + ra);
  const float4 b = *reinterpret_cast<const float4*>(s + cb);
  const unsigned long long b0 = pack2(b.x, b.y), b1 = pack2(b.z, b.w);
  const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const unsigned long long a2 = pack2(av[u], av[u]);
    fma2(d[u][0], a2, b0);
    fma2(d[u][1], a2, b1);
  }
}

__global__ void __launch_bounds__(NT, 2)
gram_async_kernel(const float* __restrict__ y, int n, int64_t J, int T, int64_t kc, float* __restrict__ part) {
  extern __shared__ __align__(16) float gas[];
  const int split = blockIdx.y;
  int id = blockIdx.x, ti = 0;  // upper triangle, diagonal included, row by row
  while (id >= T - ti) { id -= T - ti; ++ti; }
  const int tj = ti + id;
  const bool diag = ti == tj;
  const int64_t cb = (int64_t)split * kc, ce = min(J, cb + kc);
  const int ntile = cb < ce ? (int)((ce - cb + GA_TK - 1) / GA_TK) : 0;
  const int tid = threadIdx.x;
  // A stage holds GA_TK x 32 chunks of 16 bytes per operand: thread t copies
  // chunks t and t + 256 (row q / 32, chunk q % 32).
  auto load_stage = [&](int t, int slot) {
    float* sa = gas + slot * GA_STAGE;
    float* sb = sa + GA_TK * GA_LD;
    const int64_t c0 = cb + (int64_t)t * GA_TK;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int q = tid + e * NT;
      const int k = q >> 5, ch = q & 31;
      const int64_t c = c0 + k;
      const bool cv = c < ce;
      const int ia = ti * 128 + ch * 4;
      const bool va = cv && ia < n;
      cp_async16(ac::smem_u32(sa + k * GA_LD + ch * 4), va ? y + (ia + (int64_t)n * c) : y, va ? 16u : 0u);
      if (!diag) {
        const int ib = tj * 128 + ch * 4;
        const bool vb = cv && ib < n;
        cp_async16(ac::smem_u32(sb + k * GA_LD + ch * 4), vb ? y + (ib + (int64_t)n * c) : y, vb ? 16u : 0u);
      }
    }
  };
  // The ring: GA_NS - 1 stages in flight, stage t consumed by `consume`.
  auto run = [&](auto&& consume) {
#pragma unroll
    for (int s = 0; s < GA_NS - 1; ++s) {
      if (s < ntile) load_stage(s, s);
      cp_async_commit();
    }
    for (int t = 0; t < ntile; ++t) {
      cp_async_wait<GA_NS - 2>();  // this thread's copies of stage t have landed
      __syncthreads();             // everyone's have, and stage t - 1's slot is free
      const int tn = t + GA_NS - 1;
      if (tn < ntile) load_stage(tn, tn % GA_NS);
      cp_async_commit();
      consume(gas + (t % GA_NS) * GA_STAGE);
    }
  };
  const int ntiles = T * (T + 1) / 2;
  float* out = part + ((int64_t)split * ntiles + blockIdx.x) * (128 * 128);
  if (diag) {
    const DiagBlocks db(tid, blockIdx.x + blockIdx.y);
    unsigned long long d[3][4][2];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int u = 0; u < 4; ++u) d[b][u][0] = d[b][u][1] = 0ull;
    run([&](const float* sa) {
      if (db.extra) {
#pragma unroll
        for (int k = 0; k < GA_TK; ++k)
#pragma unroll
          for (int b = 0; b < 3; ++b) diag_block_step(sa + k * GA_LD, db.ra[b], db.cb[b], d[b]);
      } else {
#pragma unroll
        for (int k = 0; k < GA_TK; ++k)
#pragma unroll
          for (int b = 0; b < 2; ++b) diag_block_step(sa + k * GA_LD, db.ra[b], db.cb[b], d[b]);
      }
    });
    // lanes >= 16 of the extra warp computed a copy of lane - 16's block
    const int nb = db.extra && (tid & 31) < 16 ? 3 : 2;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b < nb) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 f0 = unpack2(d[b][u][0]), f1 = unpack2(d[b][u][1]);
          *reinterpret_cast<float4*>(out + (db.ra[b] + u) * 128 + db.cb[b]) = make_float4(f0.x, f0.y, f1.x, f1.y);
        }
      }
    }
    return;
  }
  Block<128, 128, 8, 8> blk;
  blk.init();
  run([&](const float* sa) { blk.mma(sa, sa + GA_TK * GA_LD); });
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v)
      out[Block<128, 128, 8, 8>::row_of(blk.ty, u) * 128 + Block<128, 128, 8, 8>::col_of(blk.tx, v)] = blk.acc(u, v);
}

// ------------------------------------- small-I_n Gram (mode-1 views, I_n <= 64)
// For a view with lo == 1 and I_n <= 64 (I_n % 4 == 0, 16-byte aligned base)
// the whole I_n x I_n Gram fits one CTA's registers many times over, so the
// CTA's warps split its values of c instead of its tiles.  The Gram is cut
// into NB x NB blocks of 8 x 8 (NB = ceil(I_n / 8)); a group of GW warps
// owns the NB (NB + 1) / 2 upper-triangle blocks, one 8 x 8 block per lane
// (8 x 8 values, column pairs packed for fma.rn.f32x2), and the CTA's
// groups take disjoint rows of every stage.  A stage is 16 KB of rows of c
// (each I_n contiguous floats), moved by 16-byte cp.async copies into a
// GS_NS-deep ring (columns I_n .. 8 NB - 1 and rows past the split are
// zero-filled).  No tile is padded to 64 or 128 rows and no lower block is
// computed: at I_n = 48 the executed FMAs are 1.17 x the symmetric count,
// against 3.6 x for one 64 x 64 tile.  At the end the groups' blocks are
// added in group order through shared memory and the CTA writes one partial
// Gram (pitch 8 NB, upper blocks); small_reduce_kernel sums the partials in
// CTA order as float-float pairs.  A group's float32 chain covers the CTA's
// c range divided by the number of groups (kept <= 8192 terms).
constexpr int GS_NS = 4;
constexpr int GS_MAXN = 64;
constexpr int GS_STAGE_FLOATS = 4096;  // 16 KB per stage

// Rows of c per stage: a 16 KB stage, at most 256 rows.
__host__ __device__ inline int gs_rows(int LD) { return min(256, GS_STAGE_FLOATS / LD); }

// Groups: GW = 2 (I_n > 56, 36 blocks): two warps per group, 4 groups; GW = 1:
// groups of U lanes inside a warp (32 / U per warp), so small Grams keep the
// lanes busy.
template <int GW>
__global__ void __launch_bounds__(NT, 2)
gram_small_kernel(const float* __restrict__ y, int n, int64_t J, int64_t kc, float* __restrict__ part) {
  extern __shared__ __align__(16) float gss[];
  const int NB = (n + 7) / 8, LD = 8 * NB;  // stage row pitch (floats)
  const int U = NB * (NB + 1) / 2;
  const int TKR = gs_rows(LD);
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  int grp, gl, G;
  bool active;
  if (GW == 2) {
    G = 4;
    grp = warp / 2;
    gl = (warp % 2) * 32 + lane;
    active = gl < U;
  } else {
    const int gpw = 32 / U;  // groups per warp
    G = 8 * gpw;
    grp = warp * gpw + lane / U;
    gl = lane % U;
    active = lane / U < gpw;
  }
  // this lane's block (bi, bj), bi <= bj: the gl-th upper block, row by row
  int bi = 0, bj = 0;
  {
    int id = active ? gl : 0;
    while (id >= NB - bi) { id -= NB - bi; ++bi; }
    bj = bi + id;
  }
  const int64_t cb = (int64_t)blockIdx.x * kc, ce = min(J, cb + kc);
  const int nst = cb < ce ? (int)((ce - cb + TKR - 1) / TKR) : 0;
  const int chunks = TKR * (LD / 4);  // 16-byte chunks per stage
  auto load_stage = [&](int t, int slot) {
    float* sa = gss + slot * GS_STAGE_FLOATS;
    const int64_t c0 = cb + (int64_t)t * TKR;
    for (int q = tid; q < chunks; q += NT) {
      const int k = q / (LD / 4), ch = q % (LD / 4);
      const int64_t c = c0 + k;
      const bool v = c < ce && 4 * ch < n;
      cp_async16(ac::smem_u32(sa + k * LD + 4 * ch), v ? y + (4 * ch + (int64_t)n * c) : y, v ? 16u : 0u);
    }
  };
  unsigned long long acc[8][4];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[u][p] = 0ull;
#pragma unroll
  for (int s = 0; s < GS_NS - 1; ++s) {
    if (s < nst) load_stage(s, s);
    cp_async_commit();
  }
  for (int t = 0; t < nst; ++t) {
    cp_async_wait<GS_NS - 2>();
    __syncthreads();
    const int tn = t + GS_NS - 1;
    if (tn < nst) load_stage(tn, tn % GS_NS);
    cp_async_commit();
    if (active) {
      const float* sa = gss + (t % GS_NS) * GS_STAGE_FLOATS;
#pragma unroll 2
      for (int k = grp; k < TKR; k += G) {
        const float4 a0 = *reinterpret_cast<const float4*>(sa + k * LD + 8 * bi);
        const float4 a1 = *reinterpret_cast<const float4*>(sa + k * LD + 8 * bi + 4);
        const float4 b0 = *reinterpret_cast<const float4*>(sa + k * LD + 8 * bj);
        const float4 b1 = *reinterpret_cast<const float4*>(sa + k * LD + 8 * bj + 4);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const unsigned long long b2[4] = {pack2(b0.x, b0.y), pack2(b0.z, b0.w), pack2(b1.x, b1.y),
                                          pack2(b1.z, b1.w)};
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const unsigned long long a2 = pack2(av[u], av[u]);
#pragma unroll
          for (int p = 0; p < 4; ++p) fma2(acc[u][p], a2, b2[p]);
        }
      }
    }
  }
  // Groups' blocks added in group order through shared memory (the ring is
  // free: every thread has passed its last wait and barrier).
  cp_async_wait<0>();
  __syncthreads();
  float* red = gss;  // LD x LD <= 4096 floats
  for (int g = 0; g < G; ++g) {
    if (grp == g && active) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float2 f = unpack2(acc[u][p]);
          float* d = red + (8 * bi + u) * LD + 8 * bj + 2 * p;
          if (g == 0) { d[0] = f.x; d[1] = f.y; }
          else { d[0] += f.x; d[1] += f.y; }
        }
    }
    __syncthreads();
  }
  // this CTA's partial: red's upper blocks (rows 8 bi .., columns 8 bj .., bi <= bj)
  float* out = part + (int64_t)blockIdx.x * LD * LD;
  for (int e = tid; e < LD * LD; e += NT) {
    const int r = e / LD, c = e % LD;
    if (r / 8 <= c / 8) out[e] = red[e];
  }
}

// S(i, j) = sum over the CTAs' partials in CTA order (float-float, rounded to
// float64), read from the upper block holding (min(i, j), max(i, j)).
__global__ void small_reduce_kernel(const float* __restrict__ part, int nparts, int n, int LD, double* __restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e % n, j = e / n;
  const int lo = min(i, j), hi = max(i, j);
  const FFSum acc = ff_sum_splits(part + lo * LD + hi, (int64_t)LD * LD, nparts);
  S[e] = acc.value();
}

// Sum the split-K partial tiles in split order (deterministic), as a
// float-float pair rounded once to float64.
// sym: C is n x n from upper-triangle tiles (T x T grid of BM tiles); diagonal
// tiles have ns_d splits, off-diagonal tiles ns_o.
__global__ void reduce_sym_kernel(const float* __restrict__ part, int ns_d, int ns_o, int ntiles, int T, int BM,
                                  int64_t n, double* __restrict__ C, int accumulate = 0) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  int64_t i = idx / n, j = idx % n;  // lanes along j: contiguous within a tile row
  if (i > j) return;  // written together with (j, i)
  int ti = (int)(i / BM), tj = (int)(j / BM);
  int id = ti * T - ti * (ti - 1) / 2 + (tj - ti);
  int64_t o = (i - (int64_t)ti * BM) * BM + (j - (int64_t)tj * BM);
  const int nsplit = ti == tj ? ns_d : ns_o;
  const FFSum acc = ff_sum_splits(part + (int64_t)id * BM * BM + o, (int64_t)ntiles * BM * BM, nsplit);
  const double s = accumulate ? C[i + n * j] + acc.value() : acc.value();
  C[i + n * j] = s;
  C[j + n * i] = s;
}

__global__ void reduce_cross_kernel(const float* __restrict__ part, int nsplit, int ntiles, int TR, int BM, int BN,
                                    int64_t n, int64_t R, double* __restrict__ C) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * R) return;
  int64_t i = idx / R, r = idx % R;  // lanes along r: contiguous within a tile row
  int ti = (int)(i / BM), tr = (int)(r / BN);
  int id = ti * TR + tr;
  int64_t o = (i - (int64_t)ti * BM) * BN + (r - (int64_t)tr * BN);
  const FFSum acc = ff_sum_splits(part + (int64_t)id * BM * BN + o, (int64_t)ntiles * BM * BN, nsplit);
  C[i + n * r] = acc.value();
}

// ------------------------------------------------------------- CO kernel
// O(c, r) = sum_i Y(c, i) M[i][r]; O is a (lo, R, hi) tensor.
template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(NT, 2)
ttm_co_kernel(const float* __restrict__ y, int64_t lo, int64_t n, int64_t hi, const float* __restrict__ M,
              int64_t R, float* __restrict__ out) {
  __shared__ __align__(16) float sA[2][TK * (BM + PAD)];
  __shared__ __align__(16) float sB[2][TK * (BN + PAD)];
  const int64_t J = lo * hi;
  const int64_t c0 = (int64_t)blockIdx.x * BM;
  const int64_t r0 = (int64_t)blockIdx.y * BN;
  ViewLoaderKI<BM> la;
  MatLoader<BN> lb;
  la.init(y, lo, n, J, c0);
  lb.init(M, n, R, r0);
  // Packed FMAs except for the widest tile, where their extra registers spill
  // (measured 2 % slower there, 5 % faster at BN = 64).
  Block<BM, BN, TM, TN, (BN < 128)> blk;
  blk.init();
  const int64_t ntile = (n + TK - 1) / TK;
  la.fetch(0);
  lb.fetch(0);
  la.store(sA[0]);
  lb.store(sB[0]);
  __syncthreads();
  for (int64_t t = 0; t < ntile; ++t) {
    const int buf = t & 1;
    if (t + 1 < ntile) {
      la.fetch((t + 1) * TK);
      lb.fetch((t + 1) * TK);
    }
    blk.mma(sA[buf], sB[buf]);
    if (t + 1 < ntile) {
      la.store(sA[buf ^ 1]);
      lb.store(sB[buf ^ 1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < TM; ++u) {
    int64_t c = c0 + Block<BM, BN, TM, TN>::row_of(blk.ty, u);
    if (c >= J) continue;
    int64_t base = (c % lo) + lo * R * (c / lo);
#pragma unroll
    for (int v = 0; v < TN; ++v) {
      int64_t r = r0 + Block<BM, BN, TM, TN>::col_of(blk.tx, v);
      if (r < R) out[base + lo * r] = blk.acc(u, v);
    }
  }
}

// ------------------------------------------- cp.async-fed TTM (mode-1 views)
// O(c, r) = sum_i Y(c, i) U(i, r) for a view whose rows c are I_n contiguous
// floats (lo == 1, I_n % 4 == 0, Y and U 16-byte aligned).  Both operands
// are staged as they lie in memory: a row c of Y and a column r of U each
// hold the stage's TA_KS consecutive values of i, moved by 16-byte cp.async
// copies into shared rows of TA_LD floats.  That is one pass with no
// transpose and no register staging (the ttm_co_kernel loader transposes
// through registers into k-major tiles, and its stores conflict).  The ring
// holds TA_NS stages, TA_NS - 1 of them in flight.  A thread takes rows
// m = u TY + ty and columns r = v TX + tx (interleaved, so a warp's rows fall
// in different banks), reads each row's or column's fragment four values of i
// at a time (one 128-bit load), then takes the four outer products: the same
// two 128-bit loads per k for eight rows as a k-major tile.  Rows past J,
// columns past R and (n % 4 == 0) whole chunks past I_n are zero-filled.
// Used for R <= 32, where the TTM is bound by the movement of Y: against
// ttm_co_kernel, 128 x 2097152 R 16 0.45 -> 0.32 ms, 48 x 5308416 R 8
// 0.48 -> 0.32 ms, 640 x 409600 R 32 0.60 -> 0.48 ms.  At R = 64 the FMAs
// dominate, and there the k-major register block with packed FMAs is faster
// (0.81 against 1.10 ms): its column pairs come straight from one load, where
// here they would have to be assembled from two.
constexpr int TA_KS = 16;          // values of i per stage
constexpr int TA_LD = TA_KS + 4;   // row pitch in floats: 16-byte aligned rows, spread over the banks
constexpr int TA_NS = 4;
template <int BM, int BN>
constexpr int ttm_async_smem() { return TA_NS * (BM + BN) * TA_LD * (int)sizeof(float); }

template <int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(NT, 2)
ttm_async_kernel(const float* __restrict__ y, int n, int64_t J, const float* __restrict__ U, int R,
                 float* __restrict__ out) {
  constexpr int TX = BN / TN, TY = BM / TM;
  static_assert(TX * TY == NT, "thread grid must cover 256 threads");
  constexpr int STAGE = (BM + BN) * TA_LD;
  constexpr int CHUNKS = (BM + BN) * (TA_KS / 4);
  extern __shared__ __align__(16) float tas[];
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const int64_t c0 = (int64_t)blockIdx.x * BM;
  const int r0 = (int)blockIdx.y * BN;
  const int ntile = (n + TA_KS - 1) / TA_KS;
  auto load_stage = [&](int t, int slot) {
    float* s = tas + slot * STAGE;
    const int i0 = t * TA_KS;
#pragma unroll
    for (int q0 = 0; q0 < CHUNKS; q0 += NT) {
      const int q = q0 + tid;
      if (q < CHUNKS) {
        const int row = q / (TA_KS / 4), ch = q % (TA_KS / 4);
        const int i = i0 + 4 * ch;
        const float* src;
        bool ok;
        if (row < BM) {
          const int64_t c = c0 + row;
          ok = c < J && i < n;
          src = y + (i + (int64_t)n * c);
        } else {
          const int r = r0 + (row - BM);
          ok = r < R && i < n;
          src = U + (i + (int64_t)n * r);
        }
        cp_async16(ac::smem_u32(s + row * TA_LD + 4 * ch), ok ? src : y, ok ? 16u : 0u);
      }
    }
  };
  float acc[TM][TN];
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TN; ++v) acc[u][v] = 0.f;
#pragma unroll
  for (int s = 0; s < TA_NS - 1; ++s) {
    if (s < ntile) load_stage(s, s);
    cp_async_commit();
  }
  for (int t = 0; t < ntile; ++t) {
    cp_async_wait<TA_NS - 2>();  // this thread's copies of stage t have landed
    __syncthreads();             // everyone's have, and stage t - 1's slot is free
    const int tn = t + TA_NS - 1;
    if (tn < ntile) load_stage(tn, tn % TA_NS);
    cp_async_commit();
    const float* sa = tas + (t % TA_NS) * STAGE;
    const float* sb = sa + BM * TA_LD;
#pragma unroll
    for (int g = 0; g < TA_KS / 4; ++g) {
      float4 a[TM], b[TN];
#pragma unroll
      for (int u = 0; u < TM; ++u) a[u] = *reinterpret_cast<const float4*>(sa + (u * TY + ty) * TA_LD + 4 * g);
#pragma unroll
      for (int v = 0; v < TN; ++v) b[v] = *reinterpret_cast<const float4*>(sb + (v * TX + tx) * TA_LD + 4 * g);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        auto el = [kk](const float4& f) { return kk == 0 ? f.x : kk == 1 ? f.y : kk == 2 ? f.z : f.w; };
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
          for (int v = 0; v < TN; ++v) acc[u][v] = fmaf(el(a[u]), el(b[v]), acc[u][v]);
      }
    }
  }
  // O(c, r) at c R + r (lo == 1): lanes along r.
#pragma unroll
  for (int u = 0; u < TM; ++u) {
    const int64_t c = c0 + u * TY + ty;
    if (c >= J) continue;
#pragma unroll
    for (int v = 0; v < TN; ++v) {
      const int r = r0 + v * TX + tx;
      if (r < R) out[c * R + r] = acc[u][v];
    }
  }
}

// ------------------------------------------------------------ host side
int gram_tile(int64_t n) { return n > 64 ? 128 : (n > 32 ? 64 : 32); }

namespace {
struct SplitPlan {
  int nsplit;
  int64_t kc;
};
// Split count for a CI launch of `ntiles` output tiles: at least enough splits
// to keep every float32 partial sum within SPLIT_MAX_K terms, then as many as
// fill the needed waves of (2 CTAs per SM) slots without a partial tail wave.
SplitPlan choose_split(int64_t J, int ntiles) {
  const int slots = 2 * num_sms();
  const int64_t min_split = ceil_div(J, SPLIT_MAX_K);
  const int64_t waves = std::max<int64_t>(1, ceil_div(min_split * ntiles, slots));
  int64_t nsplit = std::max<int64_t>(min_split, (waves * slots) / ntiles);
  nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, ceil_div(J, TK)));
  int64_t kc = ceil_div(ceil_div(J, nsplit), TK) * TK;
  nsplit = ceil_div(J, kc);
  return {(int)std::max<int64_t>(1, nsplit), kc};
}
int gram_bm(int64_t n) { return gram_tile(n); }
int cross_bn(int64_t R) { return R > 64 ? 128 : (R > 32 ? 64 : (R > 16 ? 32 : 16)); }
}  // namespace

// Split plans of the two Gram launches (diagonal tiles, off-diagonal tiles).
struct GramPlan {
  int bm, T, nt;
  SplitPlan d, o;
};
static GramPlan gram_plan(const View& v, int bm_force = 0) {
  GramPlan g;
  g.bm = (bm_force == 32 || bm_force == 64 || bm_force == 128) ? bm_force : gram_bm(v.n);
  g.T = (int)ceil_div(v.n, g.bm);
  g.nt = g.T * (g.T + 1) / 2;
  g.d = choose_split(v.J(), g.T);
  g.o = g.T > 1 ? choose_split(v.J(), g.T * (g.T - 1) / 2) : g.d;
  return g;
}

// The small-I_n form (gram_small_kernel): contiguous mode-1 views with
// I_n <= 64, I_n % 4 == 0, 16-byte aligned; the plan's own tile choice only.
struct SmallPlan {
  int nparts, LD, gw;
  int64_t kc;
};
static bool small_shape(const View& v) { return v.lo == 1 && v.n >= 1 && v.n <= GS_MAXN && v.n % 4 == 0; }
static SmallPlan small_plan(const View& v) {
  SmallPlan sp;
  const int NB = (int)ceil_div(v.n, 8), U = NB * (NB + 1) / 2;
  sp.LD = 8 * NB;
  sp.gw = U > 32 ? 2 : 1;
  const int G = sp.gw == 2 ? 4 : 8 * (32 / U);
  const int rows = gs_rows(sp.LD);
  const int64_t J = v.J();
  // enough CTAs for two per SM, and few enough c per CTA that a group's
  // chain (its share of the CTA's rows) stays within SPLIT_MAX_K terms
  const int64_t need = ceil_div(J, (int64_t)SPLIT_MAX_K * std::min(G, rows));
  int64_t nparts = std::max<int64_t>(need, std::min<int64_t>(2 * num_sms(), ceil_div(J, rows)));
  sp.kc = ceil_div(ceil_div(J, nparts), rows) * rows;
  sp.nparts = (int)ceil_div(J, sp.kc);
  return sp;
}

size_t gram_scratch_bytes(const View& v, int bm) {
  GramPlan g = gram_plan(v, bm);
  // the single-launch form (gram_async_kernel) plans all tiles together
  const int ns = std::max({g.d.nsplit, g.o.nsplit, choose_split(v.J(), g.nt).nsplit});
  size_t bytes = (size_t)ns * g.nt * g.bm * g.bm * sizeof(float);
  if (bm == 0 && small_shape(v)) {
    const SmallPlan sp = small_plan(v);
    bytes = std::max(bytes, (size_t)sp.nparts * sp.LD * sp.LD * sizeof(float));
  }
  return bytes;
}

int gram_f32(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes, cudaStream_t st,
             cudaEvent_t mid, int bm) {
  if (v.n <= 0) return ATK_OK;
  if (v.J() == 0) {
    ATK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * v.n * v.n, st));
    return ATK_OK;
  }
  GramPlan g = gram_plan(v, bm);
  if (gram_scratch_bytes(v, bm) > scratch_bytes) {
    set_error("gram_f32: scratch too small");
    return ATK_EINVAL;
  }
  if (bm == 0 && small_shape(v) && kc_vec_ok(y, v)) {
    const SmallPlan sp = small_plan(v);
    constexpr int smem = GS_NS * GS_STAGE_FLOATS * (int)sizeof(float);
    static const bool attr_ok = [] {
      return cudaFuncSetAttribute(gram_small_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                 cudaSuccess &&
             cudaFuncSetAttribute(gram_small_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
                 cudaSuccess;
    }();
    if (!attr_ok) {
      set_error("gram: cannot set the shared-memory size of the small-I_n Gram kernel");
      return ATK_ECUDA;
    }
    if (sp.gw == 2) gram_small_kernel<2><<<sp.nparts, NT, smem, st>>>(y, (int)v.n, v.J(), sp.kc, scratch);
    else gram_small_kernel<1><<<sp.nparts, NT, smem, st>>>(y, (int)v.n, v.J(), sp.kc, scratch);
    ATK_LAUNCHED();
    if (mid) ATK_CUDA(cudaEventRecord(mid, st));
    small_reduce_kernel<<<(unsigned)ceil_div(v.n * v.n, 256), 256, 0, st>>>(scratch, sp.nparts, (int)v.n, sp.LD, S);
    ATK_LAUNCHED();
    return ATK_OK;
  }
  if (g.bm == 128 && kc_vec_ok(y, v)) {
    // one launch for every tile, one split plan for all of them
    static const bool attr_ok = [] {
      return cudaFuncSetAttribute(gram_async_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GA_SMEM) ==
             cudaSuccess;
    }();
    if (!attr_ok) {
      set_error("gram: cannot set the shared-memory size of the cp.async Gram kernel");
      return ATK_ECUDA;
    }
    g.d = g.o = choose_split(v.J(), g.nt);
    gram_async_kernel<<<dim3(g.nt, g.d.nsplit), NT, GA_SMEM, st>>>(y, (int)v.n, v.J(), g.T, g.d.kc, scratch);
    ATK_LAUNCHED();
  } else {
    if (g.bm == 128) launch_gram_tiles<128, 8>(y, v, g.T, g.d.nsplit, g.d.kc, g.o.nsplit, g.o.kc, scratch, st);
    else if (g.bm == 64) launch_gram_tiles<64, 4>(y, v, g.T, g.d.nsplit, g.d.kc, g.o.nsplit, g.o.kc, scratch, st);
    else launch_gram_tiles<32, 2>(y, v, g.T, g.d.nsplit, g.d.kc, g.o.nsplit, g.o.kc, scratch, st);
    ATK_LAUNCHED();
    if (g.T > 1) count_launch();
  }
  if (mid) ATK_CUDA(cudaEventRecord(mid, st));
  int64_t total = v.n * v.n;
  reduce_sym_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(scratch, g.d.nsplit, g.o.nsplit, g.nt, g.T, g.bm,
                                                                     v.n, S);
  ATK_LAUNCHED();
  return ATK_OK;
}

// Same kernels as gram_f32 for callers whose scratch is a fixed block.  The
// float32 chains keep the library's length (at most SPLIT_MAX_K terms); when
// the partial tiles of all splits do not fit in `scratch_bytes`, the splits
// run in rounds of as many as fit, and each round's sum (float-float, rounded
// to float64) is added to S in float64, in round order (deterministic).
int gram_f32_fixed_scratch(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes,
                           cudaStream_t st) {
  if (v.n <= 0) return ATK_OK;
  if (v.J() == 0) {
    ATK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * v.n * v.n, st));
    return ATK_OK;
  }
  GramPlan g = gram_plan(v);
  const size_t per_split = (size_t)g.nt * g.bm * g.bm * sizeof(float);
  const int64_t fit = (int64_t)(scratch_bytes / per_split);
  if (fit < 1) {
    set_error("gram: the partial tiles of one split do not fit in the fixed scratch");
    return ATK_EUNSUPPORTED;
  }
  // One split plan for both launches: chains of at most SPLIT_MAX_K terms.
  const int64_t J = v.J();
  const int64_t kc = std::min<int64_t>(std::min(g.d.kc, g.o.kc), SPLIT_MAX_K);
  const int64_t total = ceil_div(J, kc);
  for (int64_t first = 0; first < total; first += fit) {
    const int ns = (int)std::min<int64_t>(fit, total - first);
    const int64_t c_base = first * kc;
    if (g.bm == 128) launch_gram_tiles<128, 8>(y, v, g.T, ns, kc, ns, kc, scratch, st, c_base);
    else if (g.bm == 64) launch_gram_tiles<64, 4>(y, v, g.T, ns, kc, ns, kc, scratch, st, c_base);
    else launch_gram_tiles<32, 2>(y, v, g.T, ns, kc, ns, kc, scratch, st, c_base);
    ATK_LAUNCHED();
    if (g.T > 1) count_launch();
    reduce_sym_kernel<<<(unsigned)ceil_div(v.n * v.n, 256), 256, 0, st>>>(scratch, ns, ns, g.nt, g.T, g.bm, v.n, S,
                                                                           first > 0 ? 1 : 0);
    ATK_LAUNCHED();
  }
  return ATK_OK;
}

size_t cross_scratch_bytes(const View& v, int64_t R) {
  int bn = cross_bn(R);
  int TI = (int)ceil_div(v.n, 128), TR = (int)ceil_div(R, bn);
  int nt = TI * TR;
  SplitPlan sp = choose_split(v.J(), nt);
  return (size_t)sp.nsplit * nt * 128 * bn * sizeof(float);
}

int cross_f32(const float* y, const View& v, const float* P, int64_t R, double* C, float* scratch,
              size_t scratch_bytes, cudaStream_t st) {
  if (v.n <= 0 || R <= 0) return ATK_OK;
  if (v.J() == 0) {
    ATK_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * v.n * R, st));
    return ATK_OK;
  }
  int bn = cross_bn(R);
  int TI = (int)ceil_div(v.n, 128), TR = (int)ceil_div(R, bn);
  int nt = TI * TR;
  SplitPlan sp = choose_split(v.J(), nt);
  if ((size_t)sp.nsplit * nt * 128 * bn * sizeof(float) > scratch_bytes) {
    set_error("cross_f32: scratch too small");
    return ATK_EINVAL;
  }
  dim3 grid(nt, sp.nsplit);
  if (bn == 128) cross_ci_kernel<128, 128, 8, 8><<<grid, NT, 0, st>>>(y, P, v.lo, v.n, v.hi, R, TR, sp.kc, scratch);
  else if (bn == 64) cross_ci_kernel<128, 64, 8, 4><<<grid, NT, 0, st>>>(y, P, v.lo, v.n, v.hi, R, TR, sp.kc, scratch);
  else if (bn == 32) cross_ci_kernel<128, 32, 8, 2><<<grid, NT, 0, st>>>(y, P, v.lo, v.n, v.hi, R, TR, sp.kc, scratch);
  else cross_ci_kernel<128, 16, 8, 1><<<grid, NT, 0, st>>>(y, P, v.lo, v.n, v.hi, R, TR, sp.kc, scratch);
  ATK_LAUNCHED();
  int64_t total = v.n * R;
  reduce_cross_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(scratch, sp.nsplit, nt, TR, 128, bn, v.n, R, C);
  ATK_LAUNCHED();
  return ATK_OK;
}

namespace {
template <int BM, int BN, int TM, int TN>
int launch_ttm_async(const float* y, const View& v, const float* U, int64_t R, float* out, cudaStream_t st) {
  constexpr int smem = ttm_async_smem<BM, BN>();
  static const bool attr_ok =
      cudaFuncSetAttribute(ttm_async_kernel<BM, BN, TM, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
      cudaSuccess;
  if (!attr_ok) {
    set_error("ttm: cannot set the shared-memory size of the cp.async TTM kernel");
    return ATK_ECUDA;
  }
  const dim3 grid((unsigned)ceil_div(v.J(), BM), (unsigned)ceil_div(R, BN));
  ttm_async_kernel<BM, BN, TM, TN><<<grid, NT, smem, st>>>(y, (int)v.n, v.J(), U, (int)R, out);
  ATK_LAUNCHED();
  return ATK_OK;
}
}  // namespace

int ttm_f32(const float* y, const View& v, const float* U, int64_t R, float* out, cudaStream_t st) {
  const int64_t J = v.J();
  if (J == 0 || R <= 0) return ATK_OK;
  // Contiguous mode-1 views (16-byte aligned Y and U) with R <= 32 and at
  // least a CTA per SM: the cp.async-fed kernel.
  if (kc_vec_ok(y, v) && (reinterpret_cast<uintptr_t>(U) & 15) == 0 && R <= 32) {
    if (R <= 16 && ceil_div(J, 256) >= num_sms()) return launch_ttm_async<256, 16, 8, 2>(y, v, U, R, out, st);
    if (R > 16 && ceil_div(J, 128) >= num_sms()) return launch_ttm_async<128, 32, 8, 2>(y, v, U, R, out, st);
  }
  int bn = cross_bn(R);
  dim3 grid((unsigned)ceil_div(J, 128), (unsigned)ceil_div(R, bn));
  if ((int64_t)grid.x * grid.y < num_sms() / 2) {
    // A small product (the n x m panels of the eigensolver): 64 x 64 tiles
    // put four to eight times as many CTAs on the chip.
    dim3 g64((unsigned)ceil_div(J, 64), (unsigned)ceil_div(R, 64));
    ttm_co_kernel<64, 64, 2, 8><<<g64, NT, 0, st>>>(y, v.lo, v.n, v.hi, U, R, out);
  } else if (bn == 128) ttm_co_kernel<128, 128, 8, 8><<<grid, NT, 0, st>>>(y, v.lo, v.n, v.hi, U, R, out);
  else if (bn == 64) ttm_co_kernel<128, 64, 8, 4><<<grid, NT, 0, st>>>(y, v.lo, v.n, v.hi, U, R, out);
  else if (bn == 32) ttm_co_kernel<128, 32, 8, 2><<<grid, NT, 0, st>>>(y, v.lo, v.n, v.hi, U, R, out);
  else {
    // R <= 16: 256 rows of c by 16 columns, 8 x 2 per thread, so each shared
    // load feeds twice the FMAs of a 128 x 16 tile (which was load-bound).
    dim3 g256((unsigned)ceil_div(J, 256), (unsigned)ceil_div(R, 16));
    ttm_co_kernel<256, 16, 8, 2><<<g256, NT, 0, st>>>(y, v.lo, v.n, v.hi, U, R, out);
  }
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
