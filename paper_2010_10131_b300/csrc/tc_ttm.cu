// Tensor-core (tcgen05) forms of the truncating TTM O = Y x_n U^T (Eq. 2 with
// the matrix U^T; Alg. 2, EIG branch), matricization-free over the stride
// view (Sec. V): O(c, r) = sum_i Y(c, i) U(i, r), O written in the (lo, R, hi)
// layout.
//
// Precision forms, as for the Gram (tc_ops.cu): TF32 and BF16 round both
// operands; BF16X3 splits both into hi + lo and issues hi hi + hi lo + lo hi;
// FP8-e4m3 scales mode-n index i of Y by the power of two s_i that brings
// max_c |Y(c, i)| into [128, 256) (the Gram's row scale), folds 1 / s_i into
// U, scales column r of that U by the power of two t_r that brings it into
// the same range, and divides O(c, r) by t_r exactly after the product.
// Every form accumulates in float32 in tensor memory.
//
// One CTA per 128 values of c (the MMA's M), all R columns (N = R rounded up
// to 16), K = I_n in stages of 128 bytes per row:
//  - eight producer warps read Y in place (float32, natural layout), convert
//    16-byte pieces (8 BF16, 4 TF32 or 16 FP8 values along i) and store them
//    in the tcgen05 K-major no-swizzle layout (8-row x 16-byte core matrices,
//    LBO 128 B, SBO 1024 B), then fence the generic-proxy writes for the
//    tensor core and arrive on the stage's "full" mbarrier.  For lo == 1 a
//    warp reads 8 rows x 128 contiguous bytes (coalesced); otherwise lanes run
//    along c (contiguous a) and each thread gathers its piece along i.  Each
//    thread issues the loads of stage s + 1 before it converts stage s, so
//    two stages of loads are in flight per thread;
//  - producer thread 0 also streams the stage's block of U, packed once per
//    call in the same layout, with one cp.async.bulk counted on a separate
//    "bfull" mbarrier (so a drain waits only for its own bytes);
//  - one thread of a ninth warp issues the MMAs of a stage (four of 32 bytes
//    of K, three times that for BF16X3) and commits them to the stage's
//    "empty" mbarrier; after the last stage a commit releases the epilogue,
//    where the producer warps read the accumulator (tcgen05.ld 32x32b) and
//    write O.
// Three ring stages.  Every wait is bounded (2 s on %globaltimer); a wait
// that gives up raises the CTA's abort flag and DEV_TIMEOUT, thread 0 waits
// (bounded) for its bulk copies in flight, the MMA thread commits, and the
// CTA frees its tensor memory and writes nothing.
#include <algorithm>

#include "async_copy.cuh"
#include "atk_internal.cuh"
#include "tc_common.cuh"

namespace atk {
namespace tc {
namespace {

using ac::arrive_expect;
using ac::bulk_load;
using ac::mbar_arrive;
using ac::mbar_wait;
using ac::smem_u32;

constexpr int TT_M = 128;                    // c values per CTA (MMA M)
constexpr int TT_STAGES = 3;
constexpr int TT_PROD_WARPS = 8;
constexpr int TT_PROD = TT_PROD_WARPS * 32;  // producer threads
constexpr int TT_THREADS = TT_PROD + 32;     // + the MMA warp
constexpr int TT_ROWB = 128;                 // bytes of K per row per stage
constexpr int TT_ABYTES = TT_M * TT_ROWB;    // one A array of a stage: 16 KB

template <int P>
struct TT {
  static constexpr int ES = Form<P>::ES;
  static constexpr int KS = TT_ROWB / ES;  // i values per stage
  static constexpr int W = 16 / ES;        // i values per 16-byte piece
  static constexpr int ARR = Form<P>::ARR;
};

// Byte offset of the 16-byte piece (row, piece column cm) in a K-major
// no-swizzle array: 8-row groups 1024 B apart, pieces along K 128 B apart.
__device__ __forceinline__ uint32_t piece_off(int row, int cm) {
  return 1024u * (uint32_t)(row >> 3) + 128u * (uint32_t)cm + 16u * (uint32_t)(row & 7);
}

// Convert W consecutive values (i along K) into one 16-byte piece of each
// array (hi; lo for BF16X3).  FP8 values arrive already scaled.
template <int P>
__device__ __forceinline__ void to_piece(const float* x, uint4& hi, uint4& lo) {
  if constexpr (P == ATK_TF32) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w[k]) : "f"(x[k]));
    hi = make_uint4(w[0], w[1], w[2], w[3]);
  } else if constexpr (P == ATK_BF16 || P == ATK_BF16X3) {
    hi = make_uint4(pack_bf16x2(x[0], x[1]), pack_bf16x2(x[2], x[3]), pack_bf16x2(x[4], x[5]),
                    pack_bf16x2(x[6], x[7]));
    if constexpr (P == ATK_BF16X3) {
      const uint32_t hw[4] = {hi.x, hi.y, hi.z, hi.w};
      uint32_t lw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float h0 = __uint_as_float(hw[q] << 16), h1 = __uint_as_float(hw[q] & 0xFFFF0000u);
        lw[q] = pack_bf16x2(x[2 * q] - h0, x[2 * q + 1] - h1);
      }
      lo = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  } else {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_fp8x2_storage_t a = __nv_cvt_float2_to_fp8x2(make_float2(x[4 * q], x[4 * q + 1]), __NV_SATFINITE,
                                                             __NV_E4M3);
      const __nv_fp8x2_storage_t b = __nv_cvt_float2_to_fp8x2(make_float2(x[4 * q + 2], x[4 * q + 3]),
                                                             __NV_SATFINITE, __NV_E4M3);
      w[q] = (uint32_t)a | ((uint32_t)b << 16);
    }
    hi = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int P>
struct TtmArgs {
  const float* y;
  int lo, n;
  int64_t J;
  const unsigned char* upacked;  // nst stages x ARR arrays x Np rows x 128 B
  const float* rscale;           // FP8: s_i per mode-n index i (else null)
  const float* cinv;             // FP8: 1 / t_r per column (else null)
  int Np, nst, R;
  uint32_t tmem_cols;
  float* out;
  int* status;
};

template <int P>
__global__ void __launch_bounds__(TT_THREADS, 1) tc_ttm_kernel(TtmArgs<P> a) {
  using C = TT<P>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[TT_STAGES], bfull[TT_STAGES], empty[TT_STAGES], done;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int64_t c0 = (int64_t)blockIdx.x * TT_M;
  const uint32_t bbytes = (uint32_t)a.Np * TT_ROWB;           // one B array of a stage
  const uint32_t slot_bytes = C::ARR * (TT_ABYTES + bbytes);  // A arrays, then B arrays

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < TT_STAGES; ++s) {
      ac::mbar_init(smem_u32(&full[s]), TT_PROD);
      ac::mbar_init(smem_u32(&bfull[s]), 1);
      ac::mbar_init(smem_u32(&empty[s]), 1);
    }
    ac::mbar_init(smem_u32(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;

  if (warp < TT_PROD_WARPS) {
    // ------------------------------------------------------------ producers
    // lo > 1: thread t owns row t % 128 and piece columns 4 (t / 128) .. + 3;
    // its row's base offset a + lo n b is fixed for the whole K loop.
    const int prow = tid % TT_M;
    const int64_t pc = c0 + prow;
    const bool prow_ok = pc < a.J;
    const int64_t pbase = prow_ok ? (pc % a.lo) + (int64_t)a.lo * a.n * (pc / a.lo) : 0;
    const bool vec = a.lo == 1 && (a.n % 4) == 0 && ((reinterpret_cast<uintptr_t>(a.y) & 15) == 0);
    int issued = 0;
    // Four pieces per thread per stage.  lo == 1: piece q = tid + 256 e is
    // row 8 g + r8, piece column cm (a warp reads 8 rows x 128 contiguous
    // bytes); lo > 1: row prow, piece column 4 (tid / 128) + e.
    auto piece_at = [&](int e, int& row, int& cm) {
      if (a.lo == 1) {
        const int q = tid + TT_PROD * e;
        row = 8 * (q >> 6) + (q & 7);
        cm = (q >> 3) & 7;
      } else {
        row = prow;
        cm = 4 * (tid / TT_M) + e;
      }
    };
    // Global loads of stage s into registers (issued one stage ahead of the
    // conversion, so two stages of loads are in flight per thread).
    auto load_stage = [&](int s, float (&x)[4][C::W]) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int row, cm;
        piece_at(e, row, cm);
        const int i0 = s * C::KS + cm * C::W;
        if (a.lo == 1) {
          const int64_t c = c0 + row;
          if (c < a.J && vec && i0 + C::W <= a.n) {
            const float4* src = reinterpret_cast<const float4*>(a.y + (int64_t)i0 + (int64_t)a.n * c);
#pragma unroll
            for (int k = 0; k < C::W / 4; ++k) {
              const float4 v = __ldg(src + k);
              x[e][4 * k] = v.x; x[e][4 * k + 1] = v.y; x[e][4 * k + 2] = v.z; x[e][4 * k + 3] = v.w;
            }
          } else {
#pragma unroll
            for (int k = 0; k < C::W; ++k)
              x[e][k] = (c < a.J && i0 + k < a.n) ? __ldg(a.y + (int64_t)(i0 + k) + (int64_t)a.n * c) : 0.f;
          }
        } else {
#pragma unroll
          for (int k = 0; k < C::W; ++k)
            x[e][k] = (prow_ok && i0 + k < a.n) ? __ldg(a.y + pbase + (int64_t)a.lo * (i0 + k)) : 0.f;
        }
      }
    };
    // Convert stage s (in x) and store it into its slot, then fence and arrive.
    auto stage = [&](int s, float (&x)[4][C::W], float (&nx)[4][C::W]) -> bool {
      if (s >= a.nst) return true;
      if (s + 1 < a.nst) load_stage(s + 1, nx);
      const int slot = s % TT_STAGES;
      if (s >= TT_STAGES &&
          !mbar_wait(smem_u32(&empty[slot]), (uint32_t)(((s / TT_STAGES) - 1) & 1), &abort_flag))
        return false;
      const uint32_t sA = sbase + slot * slot_bytes;
      const uint32_t sB = sA + C::ARR * TT_ABYTES;
      if (tid == 0) {
        const uint32_t bar = smem_u32(&bfull[slot]);
        arrive_expect(bar, C::ARR * bbytes);
        bulk_load(sB, a.upacked + (int64_t)s * C::ARR * bbytes, C::ARR * bbytes, bar);
        issued = s + 1;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        int row, cm;
        piece_at(e, row, cm);
        if constexpr (P == ATK_FP8E4M3) {
          const int i0 = s * C::KS + cm * C::W;
#pragma unroll
          for (int k = 0; k < C::W; ++k) x[e][k] *= (i0 + k < a.n) ? a.rscale[i0 + k] : 0.f;
        }
        uint4 h, l;
        to_piece<P>(x[e], h, l);
        const uint32_t off = piece_off(row, cm);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sA + off), "r"(h.x), "r"(h.y), "r"(h.z),
                     "r"(h.w));
        if constexpr (P == ATK_BF16X3)
          asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sA + TT_ABYTES + off), "r"(l.x), "r"(l.y),
                       "r"(l.z), "r"(l.w));
      }
      // Make the generic-proxy stores visible to the tensor core, then arrive.
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full[slot]));
      return true;
    };
    float xa[4][C::W], xb[4][C::W];
    if (a.nst > 0) load_stage(0, xa);
    for (int s = 0; s < a.nst && ok; s += 2) {
      if (!stage(s, xa, xb) || !stage(s + 1, xb, xa)) ok = false;
    }
    if (tid == 0) {
      // Drain: every bulk copy this thread issued has landed before the CTA
      // can leave (bounded, never cut short by the abort flag).
      for (int s = issued > TT_STAGES ? issued - TT_STAGES : 0; s < issued; ++s)
        if (!mbar_wait(smem_u32(&bfull[s % TT_STAGES]), (uint32_t)((s / TT_STAGES) & 1), nullptr)) ok = false;
    }
    if (!ok) abort_flag = 1;
  } else if (lane == 0) {
    // ------------------------------------------------------------ MMA issue
    const uint32_t idesc = (1u << 4) | ((uint32_t)Form<P>::FMT << 7) | ((uint32_t)Form<P>::FMT << 10) |
                           ((uint32_t)(a.Np >> 3) << 17) | ((uint32_t)(TT_M >> 4) << 24);
    for (int s = 0; s < a.nst; ++s) {
      const int slot = s % TT_STAGES;
      const uint32_t ph = (uint32_t)((s / TT_STAGES) & 1);
      if (!mbar_wait(smem_u32(&full[slot]), ph, &abort_flag) || !mbar_wait(smem_u32(&bfull[slot]), ph, &abort_flag)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = sbase + slot * slot_bytes;
      const uint32_t b0 = a0 + C::ARR * TT_ABYTES;
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // four MMAs of 32 bytes of K per 128-byte row
        const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
        const uint32_t off = j * 256;
        mma(tmem, sdesc(a0 + off, 128, 1024), sdesc(b0 + off, 128, 1024), idesc, acc, Form<P>::KIND);
        if constexpr (P == ATK_BF16X3) {
          mma(tmem, sdesc(a0 + off, 128, 1024), sdesc(b0 + bbytes + off, 128, 1024), idesc, 1u, 0);
          mma(tmem, sdesc(a0 + TT_ABYTES + off, 128, 1024), sdesc(b0 + off, 128, 1024), idesc, 1u, 0);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&empty[slot])));
    }
    if (!ok) abort_flag = 1;
    // A commit tracks every MMA this thread issued before it.
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(&done)));
  }
  __syncwarp();
  // Epilogue: wait for the final commit (never cut short), then read TMEM.
  if (!mbar_wait(smem_u32(&done), 0u, nullptr)) ok = false;
  if (!ok) abort_flag = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  const bool good = abort_flag == 0;
  if (!good && tid == 0) atomicOr(a.status, DEV_TIMEOUT);
  if (good && warp < TT_PROD_WARPS) {
    const int quarter = warp & 3;  // TMEM lanes 32 quarter .. + 31
    const int row = 32 * quarter + lane;
    const int64_t c = c0 + row;
    const bool crow = c < a.J;
    const int64_t obase = crow ? (c % a.lo) + (int64_t)a.lo * a.R * (c / a.lo) : 0;
    const bool ovec = a.lo == 1 && (a.R % 4) == 0 && ((reinterpret_cast<uintptr_t>(a.out) & 15) == 0);
#pragma unroll 1
    for (int cc = 16 * (warp >> 2); cc < a.Np; cc += 32) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (!crow) continue;
      float val[16];
#pragma unroll
      for (int v = 0; v < 16; ++v) {
        val[v] = __uint_as_float(r[v]);
        if constexpr (P == ATK_FP8E4M3) val[v] *= (cc + v < a.R) ? a.cinv[cc + v] : 0.f;
      }
      if (ovec && cc + 16 <= a.R) {
        // lo == 1: the row's R values are contiguous (16-byte aligned for R % 4 == 0)
        float4* o4 = reinterpret_cast<float4*>(a.out + obase + cc);
#pragma unroll
        for (int v = 0; v < 4; ++v) o4[v] = make_float4(val[4 * v], val[4 * v + 1], val[4 * v + 2], val[4 * v + 3]);
      } else {
#pragma unroll
        for (int v = 0; v < 16; ++v)
          if (cc + v < a.R) a.out[obase + (int64_t)a.lo * (cc + v)] = val[v];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
}

// Pack U (n x R float32, column-major) into the stage blocks of the B
// operand: stage s, array (hi, lo), row r, piece column cm holds
// U(s KS + cm W .. + W - 1, r), zero outside U.  FP8: U(i, r) / s_i * t_r.
template <int P>
__global__ void tc_ttm_pack_u_kernel(const float* __restrict__ U, int n, int R, int Np, int nst,
                                     const float* __restrict__ rscale, const float* __restrict__ cinv,
                                     unsigned char* __restrict__ out) {
  using C = TT<P>;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // piece index
  const int64_t per_stage = (int64_t)Np * 8;
  if (q >= per_stage * nst) return;
  const int s = (int)(q / per_stage), rem = (int)(q % per_stage);
  const int r = rem / 8, cm = rem % 8;
  const int i0 = s * C::KS + cm * C::W;
  float x[C::W];
#pragma unroll
  for (int k = 0; k < C::W; ++k) {
    const int i = i0 + k;
    float v = (r < R && i < n) ? U[(int64_t)i + (int64_t)n * r] : 0.f;
    if constexpr (P == ATK_FP8E4M3) v = (r < R && i < n) ? v / rscale[i] / cinv[r] : 0.f;
    x[k] = v;
  }
  uint4 h, l;
  to_piece<P>(x, h, l);
  const uint32_t bbytes = (uint32_t)Np * TT_ROWB;
  unsigned char* dst = out + (int64_t)s * C::ARR * bbytes + piece_off(r, cm);
  *reinterpret_cast<uint4*>(dst) = h;
  if constexpr (P == ATK_BF16X3) *reinterpret_cast<uint4*>(dst + bbytes) = l;
}

// FP8: s_i = 2^(8 - e_i) from the row maxima (bits of non-negative floats),
// and 1 / t_r for column r of U / s: t_r = 2^(8 - e_r) with max_i |U(i, r) /
// s_i| in [2^(e_r - 1), 2^e_r).  One warp per column.
__global__ void tc_ttm_fp8_scales_kernel(const float* __restrict__ U, int n, int R, const float* __restrict__ rmax,
                                         float* __restrict__ rscale, float* __restrict__ cinv) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) rscale[i] = fp8_row_scale(rmax[i]);
  if (warp >= R) return;
  float m = 0.f;
  for (int i = lane; i < n; i += 32) m = fmaxf(m, fabsf(U[(int64_t)i + (int64_t)n * warp]) / fp8_row_scale(rmax[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) cinv[warp] = 1.f / fp8_row_scale(m);
}

struct TtmPlan {
  int Np, nst;
  uint32_t cols;
  size_t packed_bytes;
};
template <int P>
TtmPlan ttm_plan(const View& v, int64_t R) {
  TtmPlan g;
  g.Np = (int)std::max<int64_t>(16, ceil_div(R, 16) * 16);
  g.nst = (int)ceil_div(v.n, TT<P>::KS);
  g.cols = 32;
  while ((int)g.cols < g.Np) g.cols *= 2;
  g.packed_bytes = (size_t)g.nst * TT<P>::ARR * g.Np * TT_ROWB;
  return g;
}

template <int P>
size_t ttm_scratch_t(const View& v, int64_t R) {
  return ttm_plan<P>(v, R).packed_bytes + 2 * 256 + 4 * (size_t)(v.n + R) + (P == ATK_FP8E4M3 ? 4 * (size_t)v.n : 0) +
         4 * 256;
}

template <int P>
int tc_ttm_t(const float* y, const View& v, const float* U, int64_t R, float* out, char* scratch, size_t bytes,
             int* status, cudaStream_t st) {
  const TtmPlan g = ttm_plan<P>(v, R);
  if (ttm_scratch_t<P>(v, R) > bytes) { set_error("tc_ttm: scratch too small"); return ATK_EINVAL; }
  Arena ar{scratch, bytes, 0};
  unsigned char* packed = (unsigned char*)ar.take(g.packed_bytes);
  float* rscale = nullptr;
  float* cinv = nullptr;
  if (P == ATK_FP8E4M3) {
    float* rmax = (float*)ar.take(sizeof(float) * v.n);
    rscale = (float*)ar.take(sizeof(float) * v.n);
    cinv = (float*)ar.take(sizeof(float) * R);
    ATK_CUDA(cudaMemsetAsync(rmax, 0, sizeof(float) * v.n, st));
    ATK_TRY(tc_rowmax(y, v, rmax, st));
    tc_ttm_fp8_scales_kernel<<<(unsigned)ceil_div(R * 32, 256), 256, 0, st>>>(U, (int)v.n, (int)R, rmax, rscale,
                                                                              cinv);
    ATK_LAUNCHED();
  }
  const int64_t pieces = (int64_t)g.Np * 8 * g.nst;
  tc_ttm_pack_u_kernel<P><<<(unsigned)ceil_div(pieces, 256), 256, 0, st>>>(U, (int)v.n, (int)R, g.Np, g.nst, rscale,
                                                                           cinv, packed);
  ATK_LAUNCHED();
  const size_t smem = (size_t)TT_STAGES * TT<P>::ARR * (TT_ABYTES + (size_t)g.Np * TT_ROWB);
  static const bool attr = [] {
    const size_t most = (size_t)TT_STAGES * TT<P>::ARR * (TT_ABYTES + 128 * TT_ROWB);
    return cudaFuncSetAttribute(tc_ttm_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most) ==
           cudaSuccess;
  }();
  if (!attr) { set_error("tc_ttm: cannot set the kernel's shared-memory size"); return ATK_ECUDA; }
  TtmArgs<P> a;
  a.y = y;
  a.lo = (int)v.lo;
  a.n = (int)v.n;
  a.J = v.J();
  a.upacked = packed;
  a.rscale = rscale;
  a.cinv = cinv;
  a.Np = g.Np;
  a.nst = g.nst;
  a.R = (int)R;
  a.tmem_cols = g.cols;
  a.out = out;
  a.status = status;
  tc_ttm_kernel<P><<<(unsigned)ceil_div(v.J(), TT_M), TT_THREADS, smem, st>>>(a);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace
}  // namespace tc

size_t tc_ttm_scratch_bytes(const View& v, int64_t R, int precision) {
  switch (precision) {
    case ATK_TF32: return tc::ttm_scratch_t<ATK_TF32>(v, R);
    case ATK_BF16: return tc::ttm_scratch_t<ATK_BF16>(v, R);
    case ATK_BF16X3: return tc::ttm_scratch_t<ATK_BF16X3>(v, R);
    case ATK_FP8E4M3: return tc::ttm_scratch_t<ATK_FP8E4M3>(v, R);
    default: return 0;
  }
}

int tc_ttm(const float* y, const View& v, const float* U, int64_t R, int precision, float* out, char* scratch,
           size_t scratch_bytes, int* status, cudaStream_t st) {
  if (v.J() == 0 || R <= 0) return ATK_OK;
  if (R > 128) { set_error("tc_ttm: R <= 128"); return ATK_EUNSUPPORTED; }
  if (v.size() >= ((int64_t)1 << 31)) { set_error("tc_ttm: fewer than 2^31 elements"); return ATK_EUNSUPPORTED; }
  switch (precision) {
    case ATK_TF32: return tc::tc_ttm_t<ATK_TF32>(y, v, U, R, out, scratch, scratch_bytes, status, st);
    case ATK_BF16: return tc::tc_ttm_t<ATK_BF16>(y, v, U, R, out, scratch, scratch_bytes, status, st);
    case ATK_BF16X3: return tc::tc_ttm_t<ATK_BF16X3>(y, v, U, R, out, scratch, scratch_bytes, status, st);
    case ATK_FP8E4M3: return tc::tc_ttm_t<ATK_FP8E4M3>(y, v, U, R, out, scratch, scratch_bytes, status, st);
    default: set_error("tc_ttm: unknown precision"); return ATK_EINVAL;
  }
}

}  // namespace atk
