// Tensor-core (tcgen05) forms of the Gram product S = Y_(n) Y_(n)^T
// (Alg. 2, EIG branch; matricization-free over the stride view, Sec. V).
//
// Precision forms (the paper computes in float64 throughout; these are the
// bulk-arithmetic variants of this library):
//   TF32    operands rounded to TF32 (cvt.rna), kind::tf32
//   BF16    operands rounded to BF16, kind::f16
//   BF16X3  x = hi + lo with hi = bf16(x), lo = bf16(x - hi);
//           hi hi^T + hi lo^T + lo hi^T, three kind::f16 MMAs per step
//   FP8E4M3 each mode-n row i is scaled by s_i = 2^(8 - e_i), where
//           max_c |y_ic| lies in [2^(e_i - 1), 2^e_i) (a row-max pre-pass),
//           so every scaled value is below 256 < 448; rounded to e4m3,
//           kind::f8f6f4; the reduction multiplies S_ij by 1 / (s_i s_j) exactly.
// Every form accumulates in float32 in tensor memory (TMEM).  Split-K partial
// tiles are summed in a fixed order as float-float pairs, as in the float32 path.
//
// Two kernels per Gram:
//  1. pack: one pass over the view converts it into the MMA operand format and
//     writes it in "blocks" of 128 rows x 128 bytes of K (16 KB per array),
//     already in the tcgen05 K-major no-swizzle canonical layout: 8-row x
//     16-byte core matrices, adjacent along K (LBO = 128 B), 8-row groups
//     1024 B apart (SBO).  Rows beyond n and c beyond J are zero.  The
//     transpose needed when the rows are the contiguous index (lo == 1) goes
//     through shared memory, so both the reads and the writes are coalesced.
//  2. gram: one CTA per (upper-triangle 128 x 128 tile, range of blocks).  One
//     thread streams the A and B blocks with cp.async.bulk into a 3-slot ring
//     (completion counted on the slot's "full" mbarrier); one thread issues the
//     MMAs of a slot and commits them to its "empty" mbarrier; after the last
//     slot a final commit releases the four epilogue warps, which move the
//     accumulator from TMEM to the split's partial tile.  The tiles of one
//     range run side by side (tile index fastest in the grid), so each block
//     is read from HBM about once and re-read by its other tiles from L2.
// Every mbarrier wait is bounded (a time limit on %globaltimer).  A loop that
// gives up raises the CTA's abort flag and the device status DEV_TIMEOUT; the
// producer then waits (bounded) for its copies in flight, the MMA thread
// commits and waits (bounded) for its MMAs, and the CTA frees its TMEM and
// returns with a zero partial.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "async_copy.cuh"
#include "atk_internal.cuh"
#include "tc_common.cuh"

namespace atk {

namespace tc {

constexpr int BM = 128;              // tile rows = cols = MMA M = N
constexpr int KP = 64;               // c values per pack tile
constexpr int CPAD = 128;            // the packed c extent is a multiple of this (one FP8 block)
constexpr int ARRAY_BYTES = 16384;   // one block array: 128 rows x 128 bytes
constexpr int STAGES = 3;            // ring slots of the gram kernel
constexpr int GRAM_THREADS = 128;    // warp 0: producer + epilogue, warp 1: MMA + epilogue, 2-3: epilogue
constexpr int PACK_THREADS = 256;
constexpr int PACK_LD = BM + 1;      // shared-memory pitch (floats) between the tile's c values
constexpr int SPLIT_MAX_TERMS = 8192;  // c values per float32 partial sum
using ac::WAIT_NS;

using ac::smem_u32;
using ac::gtime;
using ac::mbar_try;
using ac::mbar_wait;
using ac::bulk_load;
using ac::arrive_expect;

template <int P>
struct Blk {
  static constexpr int KB = 128 / Form<P>::ES;          // c values per block
  static constexpr int BYTES = ARRAY_BYTES * Form<P>::ARR;
  static constexpr int W = 16 / Form<P>::ES;            // values per 16-byte piece
};


// ---------------------------------------------------------------------------
// Pack

// Load the 128 (rows i0..) x KP (c from c0) float32 tile of the view into
// shared memory as sm[k * PACK_LD + r], zero outside the view.  Rows are the
// contiguous index when lo == 1 (threads run along i), c is otherwise (threads
// run along c, which is a within one b).
__device__ __forceinline__ void load_tile(const float* __restrict__ y, int lo, int n, int64_t J, int i0, int64_t c0,
                                          float* sm) {
  const int t = threadIdx.x;
  if (lo == 1) {
    const int r = t % BM, kk = t / BM;
    const int i = i0 + r;
#pragma unroll
    for (int e = 0; e < KP * BM / PACK_THREADS; ++e) {
      const int k = kk + (PACK_THREADS / BM) * e;
      const int64_t c = c0 + k;
      sm[k * PACK_LD + r] = (i < n && c < J) ? __ldg(y + ((int64_t)i + (int64_t)n * c)) : 0.f;
    }
  } else {
    const int k = t % KP, r0 = t / KP;
    const int64_t c = c0 + k;
    const bool cv = c < J;
    const int64_t a = cv ? c % lo : 0, b = cv ? c / lo : 0;
    const float* base = y + (a + (int64_t)lo * n * b);
#pragma unroll
    for (int e = 0; e < KP * BM / PACK_THREADS; ++e) {
      const int r = r0 + (PACK_THREADS / KP) * e;
      const int i = i0 + r;
      sm[k * PACK_LD + r] = (cv && i < n) ? __ldg(base + (int64_t)lo * i) : 0.f;
    }
  }
}

template <int P>
__global__ void __launch_bounds__(PACK_THREADS) tc_pack_kernel(const float* __restrict__ y, int lo, int n, int64_t J,
                                                               int64_t nkb, const float* __restrict__ rmax,
                                                               unsigned char* __restrict__ out) {
  using B = Blk<P>;
  extern __shared__ float sm[];
  const int ti = blockIdx.y;
  const int64_t c0 = (int64_t)blockIdx.x * KP;
  load_tile(y, lo, n, J, ti * BM, c0, sm);
  __syncthreads();
  // Pieces: 16 bytes = W consecutive c of one row.  In a block array, the
  // piece of row 8 g + r8 and core-matrix column cm (c values W cm .. W cm +
  // W - 1 of the block) sits at byte 1024 g + 128 cm + 16 r8.  Consecutive
  // threads take consecutive r8, then piece columns, then g, so each warp
  // writes whole 128-byte runs.
  constexpr int PCOLS = KP / B::W;  // piece columns per tile row
  const int64_t pcol0 = c0 / B::W;  // first piece column of the tile along c
#pragma unroll
  for (int it = 0; it < BM * PCOLS / PACK_THREADS; ++it) {
    const int q = threadIdx.x + it * PACK_THREADS;
    const int r8 = q % 8, lp = (q / 8) % PCOLS, g = q / (8 * PCOLS);
    const int row = 8 * g + r8;
    const int64_t pc = pcol0 + lp;
    const float* src = sm + (lp * B::W) * PACK_LD + row;
    unsigned char* dst =
        out + ((int64_t)ti * nkb + pc / 8) * B::BYTES + 1024 * g + 128 * (int)(pc % 8) + 16 * r8;
    if (P == ATK_TF32) {
      uint4 v;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(v.x) : "f"(src[0]));
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(v.y) : "f"(src[PACK_LD]));
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(v.z) : "f"(src[2 * PACK_LD]));
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(v.w) : "f"(src[3 * PACK_LD]));
      *reinterpret_cast<uint4*>(dst) = v;
    } else if (P == ATK_BF16 || P == ATK_BF16X3) {
      float x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = src[j * PACK_LD];
      uint4 h;
      h.x = pack_bf16x2(x[0], x[1]);
      h.y = pack_bf16x2(x[2], x[3]);
      h.z = pack_bf16x2(x[4], x[5]);
      h.w = pack_bf16x2(x[6], x[7]);
      *reinterpret_cast<uint4*>(dst) = h;
      if (P == ATK_BF16X3) {
        const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
        uint32_t lw[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float h0 = __uint_as_float(hw[q] << 16), h1 = __uint_as_float(hw[q] & 0xFFFF0000u);
          lw[q] = pack_bf16x2(x[2 * q] - h0, x[2 * q + 1] - h1);
        }
        *reinterpret_cast<uint4*>(dst + ARRAY_BYTES) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
    } else {
      const float s = fp8_row_scale(ti * BM + row < n ? rmax[ti * BM + row] : 0.f);
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_fp8x2_storage_t lo2 = __nv_cvt_float2_to_fp8x2(
            make_float2(src[(4 * q) * PACK_LD] * s, src[(4 * q + 1) * PACK_LD] * s), __NV_SATFINITE, __NV_E4M3);
        const __nv_fp8x2_storage_t hi2 = __nv_cvt_float2_to_fp8x2(
            make_float2(src[(4 * q + 2) * PACK_LD] * s, src[(4 * q + 3) * PACK_LD] * s), __NV_SATFINITE, __NV_E4M3);
        w[q] = (uint32_t)lo2 | ((uint32_t)hi2 << 16);
      }
      *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Row maxima of |y| for the FP8 scales: the same tiles as the pack, one
// atomicMax per row and tile (non-negative floats order like their bits).
__global__ void __launch_bounds__(PACK_THREADS) tc_rowmax_kernel(const float* __restrict__ y, int lo, int n,
                                                                 int64_t J, int* __restrict__ rmax_bits) {
  extern __shared__ float sm[];
  const int i0 = blockIdx.y * BM;
  load_tile(y, lo, n, J, i0, (int64_t)blockIdx.x * KP, sm);
  __syncthreads();
  const int r = threadIdx.x;
  if (r < BM && i0 + r < n) {
    float m = 0.f;
    for (int k = 0; k < KP; ++k) m = fmaxf(m, fabsf(sm[k * PACK_LD + r]));
    atomicMax(rmax_bits + i0 + r, __float_as_int(m));
  }
}

// ---------------------------------------------------------------------------
// Gram

template <int P>
struct Ring {
  static constexpr int SLOT = 2 * Blk<P>::BYTES;  // A and B blocks
  static constexpr int BYTES = STAGES * SLOT;
};

// Tile blockIdx.x (row-major upper triangle of the T x T tile grid) over
// blocks [split * kbps, min(nkb, (split + 1) * kbps)).
template <int P>
__global__ void __launch_bounds__(GRAM_THREADS) tc_gram_kernel(const unsigned char* __restrict__ packed, int T,
                                                               int64_t nkb, int kbps, float* __restrict__ part,
                                                               int* __restrict__ status) {
  using B = Blk<P>;
  using RG = Ring<P>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int tile = blockIdx.x, split = blockIdx.y;
  int ti = 0, id = tile;
  while (id >= T - ti) { id -= T - ti; ++ti; }
  const int tj = ti + id;
  const bool diag = ti == tj;
  const int64_t kb0 = (int64_t)split * kbps;
  const int64_t kend = kb0 + kbps < nkb ? kb0 + kbps : nkb;
  const int nst = kend > kb0 ? (int)(kend - kb0) : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(BM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&done)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // Producer.
    const unsigned char* pa = packed + ((int64_t)ti * nkb + kb0) * B::BYTES;
    const unsigned char* pb = packed + ((int64_t)tj * nkb + kb0) * B::BYTES;
    const uint32_t bytes = diag ? B::BYTES : 2 * B::BYTES;
    int issued = 0;
    for (int s = 0; s < nst; ++s) {
      const int slot = s % STAGES;
      if (s >= STAGES && !mbar_wait(smem_u32(&empty[slot]), (uint32_t)(((s / STAGES) - 1) & 1), &abort_flag)) {
        ok = false;
        break;
      }
      const uint32_t dst = sbase + slot * RG::SLOT, bar = smem_u32(&full[slot]);
      arrive_expect(bar, bytes);
      bulk_load(dst, pa + (int64_t)s * B::BYTES, B::BYTES, bar);
      if (!diag) bulk_load(dst + B::BYTES, pb + (int64_t)s * B::BYTES, B::BYTES, bar);
      issued = s + 1;
    }
    // Drain: the last copy issued into each slot has landed.
    for (int s = issued > STAGES ? issued - STAGES : 0; s < issued; ++s)
      if (!mbar_wait(smem_u32(&full[s % STAGES]), (uint32_t)((s / STAGES) & 1), nullptr)) ok = false;
    if (!ok) abort_flag = 1;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer.
    constexpr uint32_t idesc = (1u << 4) | ((uint32_t)Form<P>::FMT << 7) | ((uint32_t)Form<P>::FMT << 10) |
                               ((uint32_t)(BM >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    for (int s = 0; s < nst; ++s) {
      const int slot = s % STAGES;
      if (!mbar_wait(smem_u32(&full[slot]), (uint32_t)((s / STAGES) & 1), &abort_flag)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = sbase + slot * RG::SLOT, b0 = diag ? a0 : a0 + B::BYTES;
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // 4 MMAs of 32 bytes of K each per 128-byte array row
        const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
        const uint32_t off = j * 256;
        mma(tmem, sdesc(a0 + off, 128, 1024), sdesc(b0 + off, 128, 1024), idesc, acc, Form<P>::KIND);
        if (P == ATK_BF16X3) {
          const uint32_t al = a0 + ARRAY_BYTES, bl = b0 + ARRAY_BYTES;
          mma(tmem, sdesc(a0 + off, 128, 1024), sdesc(bl + off, 128, 1024), idesc, 1u, 0);
          mma(tmem, sdesc(al + off, 128, 1024), sdesc(b0 + off, 128, 1024), idesc, 1u, 0);
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
  // Epilogue: every thread waits for the final commit (never cut short).
  if (!mbar_wait(smem_u32(&done), 0u, nullptr)) ok = false;
  if (!ok) abort_flag = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();
  const bool failed = abort_flag != 0;
  const bool good = !failed && nst > 0;
  if (failed && tid == 0) atomicOr(status, DEV_TIMEOUT);
  const int ntiles = T * (T + 1) / 2;
  float* out = part + ((int64_t)split * ntiles + tile) * (BM * BM);
  const int row = 32 * warp + lane;
#pragma unroll 1
  for (int c0 = 0; c0 < BM; c0 += 16) {
    uint32_t r[16];
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    float4* o4 = reinterpret_cast<float4*>(out + (int64_t)row * BM + c0);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float4 f;
      f.x = good ? __uint_as_float(r[4 * v + 0]) : 0.f;
      f.y = good ? __uint_as_float(r[4 * v + 1]) : 0.f;
      f.z = good ? __uint_as_float(r[4 * v + 2]) : 0.f;
      f.w = good ? __uint_as_float(r[4 * v + 3]) : 0.f;
      o4[v] = f;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BM));
}

// Fixed-order float-float reduction of the split partials, with the optional FP8 row scales
// (from the row maxima) undone exactly.  Block (tile, chunk): one thread per
// entry of the upper-triangle tile, reading the partials coalesced.
constexpr int RED_THREADS = 256;
__global__ void __launch_bounds__(RED_THREADS) tc_reduce_sym_kernel(const float* __restrict__ part, int ns, int T,
                                                                    int n, const float* __restrict__ rmax,
                                                                    double* __restrict__ C) {
  const int tile = blockIdx.x, ntiles = T * (T + 1) / 2;
  int ti = 0, id = tile;
  while (id >= T - ti) { id -= T - ti; ++ti; }
  const int tj = ti + id;
  const int o = blockIdx.y * RED_THREADS + threadIdx.x;
  const int i = ti * BM + o / BM, j = tj * BM + o % BM;
  if (i >= n || j >= n || i > j) return;
  const float* p = part + (int64_t)tile * BM * BM + o;
  const int64_t stride = (int64_t)ntiles * BM * BM;
  FFSum acc;
  int sp = 0;
  for (; sp + 4 <= ns; sp += 4) {
    const float v0 = p[sp * stride], v1 = p[(sp + 1) * stride], v2 = p[(sp + 2) * stride],
                v3 = p[(sp + 3) * stride];
    acc.add(v0);
    acc.add(v1);
    acc.add(v2);
    acc.add(v3);
  }
  for (; sp < ns; ++sp) acc.add(p[sp * stride]);
  double s = acc.value();
  if (rmax) s /= (double)fp8_row_scale(rmax[i]) * (double)fp8_row_scale(rmax[j]);
  C[i + (int64_t)n * j] = s;
  C[j + (int64_t)n * i] = s;
}

template <int P>
int gram_ctas_per_sm() {
  // Depends only on the kernel and the device; thread-safe one-time initialisation.
  static const int per = [] {
    cudaFuncSetAttribute(tc_gram_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, Ring<P>::BYTES);
    cudaFuncSetAttribute(tc_pack_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(KP * PACK_LD * sizeof(float)));
    int v = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, tc_gram_kernel<P>, GRAM_THREADS, Ring<P>::BYTES);
    return std::max(1, std::min(v, 4));  // TMEM: 4 x 128 columns
  }();
  return per;
}

struct TcPlan {
  int T, nt;
  int64_t nkp, nkb;  // pack tiles and blocks along c
  int ns, kbps;      // splits and blocks per split
  size_t part_bytes, packed_bytes;
};

template <int P>
TcPlan tc_plan(const View& v) {
  using B = Blk<P>;
  TcPlan g;
  g.T = (int)ceil_div(v.n, BM);
  g.nt = g.T * (g.T + 1) / 2;
  const int64_t jp = ceil_div(v.J(), CPAD) * CPAD;
  g.nkp = jp / KP;
  g.nkb = jp / B::KB;
  // Each partial sum stays within SPLIT_MAX_TERMS values of c, and the launch
  // fills whole waves of resident CTAs.
  const int64_t slots = (int64_t)gram_ctas_per_sm<P>() * num_sms();
  const int64_t max_kb = SPLIT_MAX_TERMS / B::KB;
  const int64_t min_split = ceil_div(g.nkb, max_kb);
  const int64_t waves = std::max<int64_t>(1, ceil_div(min_split * g.nt, slots));
  int64_t ns = std::max<int64_t>(min_split, (waves * slots) / g.nt);
  ns = std::min<int64_t>(ns, g.nkb);
  const int64_t kbps = ceil_div(g.nkb, ns);
  g.kbps = (int)kbps;
  g.ns = (int)ceil_div(g.nkb, kbps);
  g.part_bytes = (size_t)g.ns * g.nt * BM * BM * sizeof(float);
  g.packed_bytes = (size_t)g.T * g.nkb * B::BYTES;
  return g;
}

template <int P>
size_t tc_scratch_t(const View& v) {
  TcPlan g = tc_plan<P>(v);
  return g.part_bytes + g.packed_bytes + (size_t)v.n * sizeof(float) + 3 * 256;
}

template <int P>
int tc_gram_t(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes, int* status,
              cudaStream_t st) {
  TcPlan g = tc_plan<P>(v);
  if (tc_scratch_t<P>(v) > scratch_bytes) {
    set_error("tc_gram: scratch too small");
    return ATK_EINVAL;
  }
  Arena ar{reinterpret_cast<char*>(scratch), scratch_bytes, 0};
  float* part = reinterpret_cast<float*>(ar.take(g.part_bytes));
  unsigned char* packed = reinterpret_cast<unsigned char*>(ar.take(g.packed_bytes));
  float* rmax = nullptr;
  const size_t pack_smem = (size_t)KP * PACK_LD * sizeof(float);
  const dim3 pgrid((unsigned)g.nkp, (unsigned)g.T);
  if (P == ATK_FP8E4M3) {
    rmax = reinterpret_cast<float*>(ar.take((size_t)v.n * sizeof(float)));
    ATK_CUDA(cudaMemsetAsync(rmax, 0, (size_t)v.n * sizeof(float), st));
    cudaFuncSetAttribute(tc_rowmax_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pack_smem);
    tc_rowmax_kernel<<<pgrid, PACK_THREADS, pack_smem, st>>>(y, (int)v.lo, (int)v.n, v.J(),
                                                            reinterpret_cast<int*>(rmax));
    ATK_LAUNCHED();
  }
  tc_pack_kernel<P><<<pgrid, PACK_THREADS, pack_smem, st>>>(y, (int)v.lo, (int)v.n, v.J(), g.nkb, rmax, packed);
  ATK_LAUNCHED();
  tc_gram_kernel<P><<<dim3(g.nt, g.ns), GRAM_THREADS, Ring<P>::BYTES, st>>>(packed, g.T, g.nkb, g.kbps, part,
                                                                            status);
  ATK_LAUNCHED();
  tc_reduce_sym_kernel<<<dim3(g.nt, BM * BM / RED_THREADS), RED_THREADS, 0, st>>>(part, g.ns, g.T, (int)v.n, rmax,
                                                                                  S);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace tc

int tc_rowmax(const float* y, const View& v, float* rmax, cudaStream_t st) {
  const size_t pack_smem = (size_t)tc::KP * tc::PACK_LD * sizeof(float);
  static const bool attr = cudaFuncSetAttribute(tc::tc_rowmax_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)pack_smem) == cudaSuccess;
  if (!attr) { set_error("tc_rowmax: cannot set the kernel's shared-memory size"); return ATK_ECUDA; }
  const dim3 grid((unsigned)ceil_div(v.J(), tc::KP), (unsigned)ceil_div(v.n, tc::BM));
  tc::tc_rowmax_kernel<<<grid, tc::PACK_THREADS, pack_smem, st>>>(y, (int)v.lo, (int)v.n, v.J(),
                                                                  reinterpret_cast<int*>(rmax));
  ATK_LAUNCHED();
  return ATK_OK;
}

size_t tc_gram_scratch_bytes(const View& v, int precision) {
  switch (precision) {
    case ATK_TF32: return tc::tc_scratch_t<ATK_TF32>(v);
    case ATK_BF16: return tc::tc_scratch_t<ATK_BF16>(v);
    case ATK_BF16X3: return tc::tc_scratch_t<ATK_BF16X3>(v);
    case ATK_FP8E4M3: return tc::tc_scratch_t<ATK_FP8E4M3>(v);
    default: return 0;
  }
}

int tc_gram(const float* y, const View& v, int precision, double* S, float* scratch, size_t scratch_bytes,
            int* status, cudaStream_t st) {
  if (v.n <= 0) return ATK_OK;
  if (v.J() == 0) {
    ATK_CUDA(cudaMemsetAsync(S, 0, sizeof(double) * v.n * v.n, st));
    return ATK_OK;
  }
  switch (precision) {
    case ATK_TF32: return tc::tc_gram_t<ATK_TF32>(y, v, S, scratch, scratch_bytes, status, st);
    case ATK_BF16: return tc::tc_gram_t<ATK_BF16>(y, v, S, scratch, scratch_bytes, status, st);
    case ATK_BF16X3: return tc::tc_gram_t<ATK_BF16X3>(y, v, S, scratch, scratch_bytes, status, st);
    case ATK_FP8E4M3: return tc::tc_gram_t<ATK_FP8E4M3>(y, v, S, scratch, scratch_bytes, status, st);
    default: set_error("tc_gram: unknown precision"); return ATK_EINVAL;
  }
}

}  // namespace atk
