// Fused ALS sweep (Alg. 3; Eq. 5): one pass over Y per sweep.
//
// A sweep needs R_k = Y^T L~ (J x R, L~ = L_k (L_k^T L_k)^{-1}) and then
// A = Y R_k and B = R_k^T R_k.  Since B = L~^T Y Y^T L~ = L~^T A, only A has
// to come from the tensor, and A = Y (Y^T L~) needs R_k one slab of c at a
// time: each CTA stages BC = 32 values of c of the view (all I_n values of
// i) in shared memory, forms that slab of R_k on chip, P(c, r) =
// sum_i Y(c, i) L~(i, r), and accumulates A(i, r) += sum_c Y(c, i) P(c, r) in
// registers over its chunk of c.  R_k is written to memory only on the last
// sweep (the core update needs it).  So a sweep reads Y once and the
// (J x R) R_k never goes through memory in between, where the unfused form
// reads Y twice and writes and reads R_k.
//
// Shapes: I_n <= 256 and R <= 32 (RB = R rounded up to 8, 16 or 32); the
// other ALS modes are compute-bound and use the separate TTM and cross
// kernels.  256 threads.  The slab sits transposed, Ys[i][c] with a row pitch
// of 36 floats (16-byte aligned rows), so both phases read 4 values of c with
// one 128-bit load, and a quarter-warp's loads fall on distinct 16-byte
// pieces:
//  - P phase: warp w takes i = w, w + 8, ...; lane (c-quad q = lane % 8,
//    r-group g = lane / 8) holds 4 c x RB/4 r partial sums; the eight warps'
//    partials are summed through shared memory in a fixed order;
//  - A phase: item q = tid + 256 k is row i = q % I_n and columns
//    8 (q / I_n) .. + 7, so consecutive lanes read consecutive rows i.
// The next slab is loaded into registers while the current one is used.
// Each CTA writes its float32 partial A (I_n x RB); a second kernel sums the
// partials in CTA order as float-float pairs (deterministic), rounded once
// to float64.  A CTA's chunk holds at most 8192 values of c (the float32
// chain length of the other split-K sums).
#include <algorithm>

#include "atk_internal.cuh"

namespace atk {
namespace {

constexpr int AF_THREADS = 256;
constexpr int AF_BC = 32;           // c values per slab
constexpr int AF_PITCH = AF_BC + 4;  // Ys row pitch (floats): rows stay 16-byte aligned
constexpr int AF_NMAX = 256;
constexpr int AF_CHAIN = 8192;

template <int RB>
struct AfSmem {
  static constexpr int SG = RB / 4;  // r values per lane in the P phase
  float ys[AF_NMAX * AF_PITCH];      // Ys[i][c]
  float lt[AF_NMAX * RB];            // L~[i][r]
  float part[8 * AF_BC * RB];        // per-warp partial P
  float p[AF_BC * RB];               // P[c][r]
};

template <int RB>
__global__ void __launch_bounds__(AF_THREADS) als_fused_kernel(const float* __restrict__ y, int lo, int n, int64_t J,
                                                               const float* __restrict__ Lt, int R, int64_t chunk,
                                                               float* __restrict__ part_out, float* __restrict__ Rk,
                                                               int write_rk) {
  extern __shared__ __align__(16) unsigned char af_raw[];
  AfSmem<RB>& sm = *reinterpret_cast<AfSmem<RB>*>(af_raw);
  constexpr int SG = AfSmem<RB>::SG;
  constexpr int PER = AF_NMAX * AF_BC / AF_THREADS;  // slab values per thread (at most)
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int64_t cb = (int64_t)blockIdx.x * chunk, ce = min(J, cb + chunk);
  // L~ (n x R, column-major, float32) into lt[i][r], zero beyond R.
  for (int idx = tid; idx < n * RB; idx += AF_THREADS) {
    const int i = idx / RB, r = idx % RB;
    sm.lt[idx] = r < R ? Lt[i + (int64_t)n * r] : 0.f;
  }
  // A items of this thread: q = tid + 256 k -> row q % n, columns 8 (q / n) ..
  constexpr int MAXIT = AF_NMAX * RB / 8 / AF_THREADS > 0 ? AF_NMAX * RB / 8 / AF_THREADS : 1;
  const int items = n * (RB / 8);
  float acc[MAXIT][8];
#pragma unroll
  for (int k = 0; k < MAXIT; ++k)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[k][j] = 0.f;
  // Slab loader: this thread's values (c, i) of the slab starting at c0,
  // zero outside.  The (c, i) pattern is the same for every slab, so it is
  // stepped without divisions: lo == 1 (element (c, i) at i + n c):
  // consecutive threads along i, the pattern advancing by 256 values of the
  // slab; otherwise (element at a + lo (i + n b)): consecutive threads along
  // c, each thread's c fixed and i advancing by 8.
  const int cnt = (AF_BC * n + AF_THREADS - 1 - tid) / AF_THREADS;  // values of this thread per slab
  const int c_first = lo == 1 ? tid / n : tid % AF_BC, i_first = lo == 1 ? tid % n : tid / AF_BC;
  const int step_c = AF_THREADS / n, step_i = AF_THREADS % n;  // lo == 1 stepping
  float pre[PER];
  auto fetch = [&](int64_t c0) {
    if (lo == 1) {
      int c = c_first, i = i_first;
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        if (e < cnt) {
          const int64_t cg = c0 + c;
          pre[e] = cg < ce ? __ldg(y + (int64_t)i + (int64_t)n * cg) : 0.f;
          c += step_c;
          i += step_i;
          if (i >= n) { i -= n; ++c; }
        }
      }
    } else {
      const int64_t cg = c0 + c_first;
      const bool ok = cg < ce;
      const int64_t base = ok ? (cg % lo) + (int64_t)lo * n * (cg / lo) : 0;
#pragma unroll
      for (int e = 0; e < PER; ++e)
        if (e < cnt) pre[e] = ok ? __ldg(y + base + (int64_t)lo * (i_first + 8 * e)) : 0.f;
    }
  };
  auto stash = [&]() {
    int c = c_first, i = i_first;
#pragma unroll
    for (int e = 0; e < PER; ++e) {
      if (e < cnt) {
        sm.ys[i * AF_PITCH + c] = pre[e];
        if (lo == 1) {
          c += step_c;
          i += step_i;
          if (i >= n) { i -= n; ++c; }
        } else {
          i += 8;
        }
      }
    }
  };
  // A items of this thread (fixed for the whole kernel).
  int it_i[MAXIT], it_g[MAXIT];
#pragma unroll
  for (int k = 0; k < MAXIT; ++k) {
    const int q = tid + AF_THREADS * k;
    it_i[k] = q % n;
    it_g[k] = q / n;
  }
  const int64_t ntile = cb < ce ? (ce - cb + AF_BC - 1) / AF_BC : 0;
  if (ntile > 0) fetch(cb);
  const int cq = lane % 8, rg = lane / 8;
  for (int64_t t = 0; t < ntile; ++t) {
    const int64_t c0 = cb + t * AF_BC;
    __syncthreads();  // the previous slab's readers are done
    stash();
    __syncthreads();
    if (t + 1 < ntile) fetch(c0 + AF_BC);
    // P phase: partial sums over this warp's i.
    float ps[4][SG];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < SG; ++v) ps[u][v] = 0.f;
#pragma unroll 4
    for (int i = warp; i < n; i += 8) {
      // 4 values of c in one 128-bit load (a quarter-warp reads 8 distinct
      // 16-byte pieces of one row), RB/4 values of L~ broadcast
      const float4 y4 = *reinterpret_cast<const float4*>(&sm.ys[i * AF_PITCH + 4 * cq]);
      const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
      float lv[SG];
#pragma unroll
      for (int v = 0; v < SG; v += 2) {
        const float2 l2 = *reinterpret_cast<const float2*>(&sm.lt[i * RB + rg * SG + v]);
        lv[v] = l2.x;
        lv[v + 1] = l2.y;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < SG; ++v) ps[u][v] = fmaf(yv[u], lv[v], ps[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < SG; ++v) sm.part[(warp * AF_BC + 4 * cq + u) * RB + rg * SG + v] = ps[u][v];
    __syncthreads();
    for (int o = tid; o < AF_BC * RB; o += AF_THREADS) {
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) s += sm.part[w * AF_BC * RB + o];
      sm.p[o] = s;
      if (write_rk) {
        const int c = o / RB, r = o % RB;
        const int64_t cg = c0 + c;
        if (r < R && cg < ce) Rk[(cg % lo) + (int64_t)lo * (r + (int64_t)R * (cg / lo))] = s;
      }
    }
    __syncthreads();
    // A phase: A(i, r) += sum_c Y(c, i) P(c, r).
#pragma unroll
    for (int k = 0; k < MAXIT; ++k) {
      if (tid + AF_THREADS * k >= items) break;
      const int i = it_i[k], g = it_g[k];
#pragma unroll
      for (int c4 = 0; c4 < AF_BC; c4 += 4) {
        // row i's 4 values of c in one 128-bit load (lanes along i: 16-byte
        // pieces 144 bytes apart, distinct within each quarter-warp)
        const float4 y4 = *reinterpret_cast<const float4*>(&sm.ys[i * AF_PITCH + c4]);
        const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 p0 = *reinterpret_cast<const float4*>(&sm.p[(c4 + u) * RB + 8 * g]);
          const float4 p1 = *reinterpret_cast<const float4*>(&sm.p[(c4 + u) * RB + 8 * g + 4]);
          acc[k][0] = fmaf(yv[u], p0.x, acc[k][0]); acc[k][1] = fmaf(yv[u], p0.y, acc[k][1]);
          acc[k][2] = fmaf(yv[u], p0.z, acc[k][2]); acc[k][3] = fmaf(yv[u], p0.w, acc[k][3]);
          acc[k][4] = fmaf(yv[u], p1.x, acc[k][4]); acc[k][5] = fmaf(yv[u], p1.y, acc[k][5]);
          acc[k][6] = fmaf(yv[u], p1.z, acc[k][6]); acc[k][7] = fmaf(yv[u], p1.w, acc[k][7]);
        }
      }
    }
  }
  // Partial A of this CTA: part_out[(blockIdx.x * n + i) * RB + r].
  float* out = part_out + (int64_t)blockIdx.x * n * RB;
#pragma unroll
  for (int k = 0; k < MAXIT; ++k) {
    if (tid + AF_THREADS * k >= items) break;
#pragma unroll
    for (int j = 0; j < 8; ++j) out[(int64_t)it_i[k] * RB + 8 * it_g[k] + j] = acc[k][j];
  }
}

// A (n x R float64, column-major) from the partials: one warp per entry, lane
// l summing partials l, l + 32, ... as a float-float pair, then the 32 pairs
// combined by a fixed shuffle tree (deterministic), rounded once to float64.
__global__ void als_fused_reduce_kernel(const float* __restrict__ part, int nparts, int n, int RB, int R,
                                        double* __restrict__ A) {
  const int64_t o = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (o >= (int64_t)n * R) return;
  const int i = (int)(o % n), r = (int)(o / n);
  FFSum s;
  for (int b = lane; b < nparts; b += 32) s.add(part[((int64_t)b * n + i) * RB + r]);
  for (int off = 16; off > 0; off >>= 1) {
    const float hi = __shfl_xor_sync(0xffffffffu, s.hi, off), lo = __shfl_xor_sync(0xffffffffu, s.lo, off);
    s.add(hi);
    s.lo += lo;
  }
  if (lane == 0) A[o] = s.value();
}

int af_rb(int64_t R) { return R <= 8 ? 8 : (R <= 16 ? 16 : 32); }

template <int RB>
int launch_fused(const float* y, const View& v, const float* Lt, int64_t R, float* part, int nparts, int64_t chunk,
                 float* Rk, cudaStream_t st) {
  static const bool attr = cudaFuncSetAttribute(als_fused_kernel<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)sizeof(AfSmem<RB>)) == cudaSuccess;
  if (!attr) { set_error("als_fused: cannot set the kernel's shared-memory size"); return ATK_ECUDA; }
  als_fused_kernel<RB><<<nparts, AF_THREADS, sizeof(AfSmem<RB>), st>>>(y, (int)v.lo, (int)v.n, v.J(), Lt, (int)R,
                                                                       chunk, part, Rk, Rk ? 1 : 0);
  ATK_LAUNCHED();
  return ATK_OK;
}

void fused_plan(const View& v, int& nparts, int64_t& chunk) {
  const int64_t J = v.J();
  const int64_t slabs = ceil_div(J, AF_BC);
  const int64_t want = std::max<int64_t>(ceil_div(J, AF_CHAIN), 4 * (int64_t)num_sms());
  nparts = (int)std::max<int64_t>(1, std::min<int64_t>(slabs, want));
  chunk = ceil_div(slabs, nparts) * AF_BC;
  nparts = (int)ceil_div(J, chunk);
}

}  // namespace

bool als_fused_ok(const View& v, int64_t R) {
  return v.n >= 1 && v.n <= AF_NMAX && R >= 1 && R <= 32 && v.J() >= 1 && v.size() < ((int64_t)1 << 31);
}

size_t als_fused_scratch_bytes(const View& v, int64_t R) {
  if (!als_fused_ok(v, R)) return 0;
  int nparts;
  int64_t chunk;
  fused_plan(v, nparts, chunk);
  return (size_t)nparts * v.n * af_rb(R) * sizeof(float);
}

// A = Y (Y^T Lt) (n x R float64); with Rk given, also Rk = Y^T Lt in the
// (lo, R, hi) layout.  Lt: n x R float32, column-major.
int als_fused(const float* y, const View& v, const float* Lt, int64_t R, double* A, float* Rk, float* scratch,
              size_t scratch_bytes, cudaStream_t st) {
  if (!als_fused_ok(v, R)) { set_error("als_fused: needs I_n <= 256 and R <= 32"); return ATK_EUNSUPPORTED; }
  if (als_fused_scratch_bytes(v, R) > scratch_bytes) { set_error("als_fused: scratch too small"); return ATK_EINVAL; }
  int nparts;
  int64_t chunk;
  fused_plan(v, nparts, chunk);
  const int rb = af_rb(R);
  if (rb == 8) ATK_TRY(launch_fused<8>(y, v, Lt, R, scratch, nparts, chunk, Rk, st));
  else if (rb == 16) ATK_TRY(launch_fused<16>(y, v, Lt, R, scratch, nparts, chunk, Rk, st));
  else ATK_TRY(launch_fused<32>(y, v, Lt, R, scratch, nparts, chunk, Rk, st));
  als_fused_reduce_kernel<<<(unsigned)ceil_div(v.n * R * 32, 256), 256, 0, st>>>(scratch, nparts, (int)v.n, rb,
                                                                                  (int)R, A);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
