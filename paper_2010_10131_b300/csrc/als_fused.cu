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
//  - A phase: item q = tid + 256 k is rows i = q % nh and i + nh (nh =
//    ceil(I_n / 2)) and columns 4 (q / nh) .. + 3, so consecutive lanes read
//    consecutive rows and each 128-bit load of P feeds eight FMAs.
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
  static constexpr int SG = RB / 4;   // r values per lane in the P phase
  static constexpr int PP = RB + 4;   // row pitch of the per-warp partials
  float ys[AF_NMAX * AF_PITCH];       // Ys[i][c]
  float lt[AF_NMAX * RB];             // L~[i][r]
  float part[8 * AF_BC * PP];         // per-warp partial P, row 8 (c % 4) + c / 4
  float p[AF_BC * RB];                // P[c][r]
};

// CSN: the number of c ranges an A item is split over (a template
// parameter, so the common CSN = 1 kernel carries none of the split's code).
template <int RB, int CSN>
__global__ void __launch_bounds__(AF_THREADS, 2) als_fused_kernel(const float* __restrict__ y, int lo, int n, int64_t J,
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
  // A items: (row pair, column quad) = rows i and i + nh (nh = ceil(n / 2);
  // the second only when < n), columns 4 g .. + 3; when there are fewer than
  // the 256 threads, each item is split over cs_n ranges of the slab's c
  // (summed once, in range order, at the end).  Work unit q = tid + 256 k:
  // range q / items, item q % items -> i = item % nh, g = item / nh.
  constexpr int MAXIT = AF_NMAX / 2 * RB / 4 / AF_THREADS > 0 ? AF_NMAX / 2 * RB / 4 / AF_THREADS : 1;
  const int nh = (n + 1) / 2;
  const int items1 = nh * (RB / 4);
  constexpr int cs_n = CSN;
  const int items = items1 * cs_n;
  constexpr int c_len = AF_BC / cs_n;  // c values of one range (4 .. 32)
  float acc[MAXIT][2][4];
#pragma unroll
  for (int k = 0; k < MAXIT; ++k)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[k][0][j] = acc[k][1][j] = 0.f;
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
  int it_i[MAXIT], it_g[MAXIT], it_c[MAXIT];
#pragma unroll
  for (int k = 0; k < MAXIT; ++k) {
    const int q = tid + AF_THREADS * k;
    const int item = q % items1;
    it_i[k] = item % nh;
    it_g[k] = item / nh;
    it_c[k] = (q / items1) * c_len;
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
      if constexpr (SG % 4 == 0) {
#pragma unroll
        for (int v = 0; v < SG; v += 4) {
          const float4 l4 = *reinterpret_cast<const float4*>(&sm.lt[i * RB + rg * SG + v]);
          lv[v] = l4.x; lv[v + 1] = l4.y; lv[v + 2] = l4.z; lv[v + 3] = l4.w;
        }
      } else {
#pragma unroll
        for (int v = 0; v < SG; v += 2) {
          const float2 l2 = *reinterpret_cast<const float2*>(&sm.lt[i * RB + rg * SG + v]);
          lv[v] = l2.x;
          lv[v + 1] = l2.y;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < SG; ++v) ps[u][v] = fmaf(yv[u], lv[v], ps[u][v]);
    }
    // Row 8 u + cq for c = 4 cq + u, pitch RB + 4: the lanes of a quarter-warp
    // (or half-warp for 8-byte stores) hit distinct banks.
    constexpr int PP = AfSmem<RB>::PP;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      float* dst = &sm.part[(warp * AF_BC + 8 * u + cq) * PP + rg * SG];
      if constexpr (SG % 4 == 0) {
#pragma unroll
        for (int v = 0; v < SG; v += 4)
          *reinterpret_cast<float4*>(dst + v) = make_float4(ps[u][v], ps[u][v + 1], ps[u][v + 2], ps[u][v + 3]);
      } else {
#pragma unroll
        for (int v = 0; v < SG; v += 2) *reinterpret_cast<float2*>(dst + v) = make_float2(ps[u][v], ps[u][v + 1]);
      }
    }
    __syncthreads();
    for (int o = tid; o < AF_BC * RB; o += AF_THREADS) {
      const int c = o / RB, r = o % RB;
      const int prow = 8 * (c % 4) + c / 4;
      float s = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) s += sm.part[(w * AF_BC + prow) * PP + r];
      sm.p[o] = s;
      if (write_rk) {
        const int64_t cg = c0 + c;
        if (r < R && cg < ce) Rk[(cg % lo) + (int64_t)lo * (r + (int64_t)R * (cg / lo))] = s;
      }
    }
    __syncthreads();
    // A phase: A(i, r) += sum_c Y(c, i) P(c, r), two rows per item, over the
    // item's range of c (a compile-time length, so the loop unrolls).
#pragma unroll
    for (int k = 0; k < MAXIT; ++k) {
      if (tid + AF_THREADS * k >= items) break;
      const int i0 = it_i[k], i1 = it_i[k] + nh, g = it_g[k], cb0 = it_c[k];
      const bool two = i1 < n;
#pragma unroll
      for (int c4 = 0; c4 < c_len; c4 += 4) {
        // rows i0 and i1: 4 values of c each in one 128-bit load (lanes along
        // i: 16-byte pieces 144 bytes apart, distinct within a quarter-warp)
        const float4 ya = *reinterpret_cast<const float4*>(&sm.ys[i0 * AF_PITCH + cb0 + c4]);
        const float4 yb = two ? *reinterpret_cast<const float4*>(&sm.ys[i1 * AF_PITCH + cb0 + c4])
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        const float va[4] = {ya.x, ya.y, ya.z, ya.w}, vb[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 p4 = *reinterpret_cast<const float4*>(&sm.p[(cb0 + c4 + u) * RB + 4 * g]);
          acc[k][0][0] = fmaf(va[u], p4.x, acc[k][0][0]); acc[k][0][1] = fmaf(va[u], p4.y, acc[k][0][1]);
          acc[k][0][2] = fmaf(va[u], p4.z, acc[k][0][2]); acc[k][0][3] = fmaf(va[u], p4.w, acc[k][0][3]);
          acc[k][1][0] = fmaf(vb[u], p4.x, acc[k][1][0]); acc[k][1][1] = fmaf(vb[u], p4.y, acc[k][1][1]);
          acc[k][1][2] = fmaf(vb[u], p4.z, acc[k][1][2]); acc[k][1][3] = fmaf(vb[u], p4.w, acc[k][1][3]);
        }
      }
    }
  }
  // Partial A of this CTA: part_out[(blockIdx.x * n + i) * RB + r], the c
  // ranges of an item summed in range order through shared memory.
  float* out = part_out + (int64_t)blockIdx.x * n * RB;
  if constexpr (CSN == 1) {
#pragma unroll
    for (int k = 0; k < MAXIT; ++k) {
      if (tid + AF_THREADS * k >= items) break;
      const int i0 = it_i[k], i1 = it_i[k] + nh, g = it_g[k];
#pragma unroll
      for (int j = 0; j < 4; ++j) out[(int64_t)i0 * RB + 4 * g + j] = acc[k][0][j];
      if (i1 < n) {
#pragma unroll
        for (int j = 0; j < 4; ++j) out[(int64_t)i1 * RB + 4 * g + j] = acc[k][1][j];
      }
    }
  } else {
    // cs_n * n * RB <= AF_THREADS * 8 floats: fits in the slab buffer
    float* red = sm.ys;
    __syncthreads();  // the last slab's readers are done
#pragma unroll
    for (int k = 0; k < MAXIT; ++k) {
      if (tid + AF_THREADS * k >= items) break;
      const int i0 = it_i[k], i1 = it_i[k] + nh, g = it_g[k], cs = it_c[k] / c_len;
#pragma unroll
      for (int j = 0; j < 4; ++j) red[(cs * n + i0) * RB + 4 * g + j] = acc[k][0][j];
      if (i1 < n) {
#pragma unroll
        for (int j = 0; j < 4; ++j) red[(cs * n + i1) * RB + 4 * g + j] = acc[k][1][j];
      }
    }
    __syncthreads();
    for (int o = tid; o < n * RB; o += AF_THREADS) {
      float a = red[o];
      for (int cs = 1; cs < cs_n; ++cs) a += red[cs * n * RB + o];
      out[o] = a;
    }
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

template <int RB, int CSN>
int launch_fused_cs(const float* y, const View& v, const float* Lt, int64_t R, float* part, int nparts,
                    int64_t chunk, float* Rk, cudaStream_t st) {
  static const bool attr = cudaFuncSetAttribute(als_fused_kernel<RB, CSN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)sizeof(AfSmem<RB>)) == cudaSuccess;
  if (!attr) { set_error("als_fused: cannot set the kernel's shared-memory size"); return ATK_ECUDA; }
  als_fused_kernel<RB, CSN><<<nparts, AF_THREADS, sizeof(AfSmem<RB>), st>>>(y, (int)v.lo, (int)v.n, v.J(), Lt,
                                                                            (int)R, chunk, part, Rk, Rk ? 1 : 0);
  ATK_LAUNCHED();
  return ATK_OK;
}

// Items (row pair, column quad) of the A phase; while they fill at most half
// of the CTA's threads, each is split over twice as many ranges of c (<= 8).
template <int RB>
int launch_fused(const float* y, const View& v, const float* Lt, int64_t R, float* part, int nparts, int64_t chunk,
                 float* Rk, cudaStream_t st) {
  const int64_t items1 = (v.n + 1) / 2 * (RB / 4);
  int cs = 1;
  while (cs < 8 && items1 * cs * 2 <= AF_THREADS) cs *= 2;
  if (cs == 1) return launch_fused_cs<RB, 1>(y, v, Lt, R, part, nparts, chunk, Rk, st);
  if (cs == 2) return launch_fused_cs<RB, 2>(y, v, Lt, R, part, nparts, chunk, Rk, st);
  if (cs == 4) return launch_fused_cs<RB, 4>(y, v, Lt, R, part, nparts, chunk, Rk, st);
  return launch_fused_cs<RB, 8>(y, v, Lt, R, part, nparts, chunk, Rk, st);
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
