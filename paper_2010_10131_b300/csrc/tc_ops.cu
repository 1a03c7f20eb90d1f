// Tensor-core (tcgen05) forms of the Gram product S = Y_(n) Y_(n)^T
// (Alg. 2, EIG branch; matricization-free over the stride view, Sec. V).
//
// Precision forms (the paper computes in float64 throughout; these are the
// bulk-arithmetic variants of this library):
//   TF32    operands rounded to TF32 (cvt.rna), kind::tf32
//   BF16    operands rounded to BF16, kind::f16
//   BF16X3  x = hi + lo with hi = bf16(x), lo = bf16(x - hi);
//           hi hi^T + hi lo^T + lo hi^T, three kind::f16 MMAs per step
//   FP8E4M3 each mode-n row i is scaled by s_i = 2^floor(log2(448 / max_c |y_ic|))
//           (a power of two, from a row-max pre-pass), rounded to e4m3,
//           kind::f8f6f4; the reduction multiplies S_ij by 1 / (s_i s_j) exactly.
// Every form accumulates in float32 in tensor memory (TMEM).  Split-K partial
// tiles are summed in float64 in a fixed order, as in the float32 path.
//
// One CTA computes one 128 x 128 tile (rows ti, columns tj of the upper
// triangle) over a range of the other index c.  Stage t of a 4-slot
// shared-memory ring holds KC = 32 values of c for the tile's 128 + 128 rows,
// converted and stored K-major in the no-swizzle canonical layout: 8-row x
// 16-byte core matrices, adjacent along K (LBO = 128 B), 8-row groups SBO
// apart.  All 256 threads stage operands, with the next stage prefetched into
// registers.  Thread 0 issues the MMAs of a stage and commits them to that
// slot's mbarrier.  Before a slot is refilled, its previous MMAs must have
// completed.  Every mbarrier wait is bounded: on timeout the CTA records
// DEV_TIMEOUT, waits once more (bounded) for its MMAs, frees its TMEM and
// returns.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "atk_internal.cuh"

namespace atk {

namespace tc {

constexpr int BM = 128;       // tile rows = cols = MMA M = N
constexpr int KC = 32;        // c values per stage
constexpr int STAGES = 4;
constexpr int THREADS = 256;
constexpr long long WAIT_LIMIT = 50000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Byte offset of (row, kbyte) in the K-major no-swizzle canonical layout.
__device__ __forceinline__ uint32_t koff(int row, int kbyte, uint32_t sbo) {
  return (uint32_t)((row >> 3) * sbo + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15));
}

template <int P>
struct Form;
// Element bytes, bytes of one stage row, arrays per operand (hi[/lo]), MMA format code.
template <>
struct Form<ATK_TF32> {
  static constexpr int ES = 4, ARR = 1, FMT = 2, KIND = 1;
};
template <>
struct Form<ATK_BF16> {
  static constexpr int ES = 2, ARR = 1, FMT = 1, KIND = 0;
};
template <>
struct Form<ATK_BF16X3> {
  static constexpr int ES = 2, ARR = 2, FMT = 1, KIND = 0;
};
template <>
struct Form<ATK_FP8E4M3> {
  static constexpr int ES = 1, ARR = 1, FMT = 0, KIND = 2;
};

template <int P>
struct Stage {
  static constexpr int ROWB = KC * Form<P>::ES;           // bytes of one row of one array
  static constexpr uint32_t SBO = (ROWB / 16) * 128;      // bytes per 8-row group
  static constexpr int ARRB = BM * ROWB;                  // bytes of one array (128 rows)
  static constexpr int OPB = ARRB * Form<P>::ARR;         // one operand (hi [+ lo])
  static constexpr int BYTES = 2 * OPB;                   // A and B
  static constexpr int KSTEPS = ROWB / 32;                // MMAs (32 B of K each) per array pair
};

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc, int kind) {
  if (kind == 0)
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
  else if (kind == 1)
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
  else
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(bar), "r"(parity));
    if (done) return true;
  }
  return false;
}

// Convert one float32 value into the stage arrays at byte offset `o`.
template <int P>
__device__ __forceinline__ void put(unsigned char* hi, unsigned char* lo, uint32_t o, float x) {
  if (P == ATK_TF32) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    *reinterpret_cast<uint32_t*>(hi + o) = t;
  } else if (P == ATK_BF16) {
    *reinterpret_cast<__nv_bfloat16*>(hi + o) = __float2bfloat16_rn(x);
  } else if (P == ATK_BF16X3) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    *reinterpret_cast<__nv_bfloat16*>(hi + o) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + o) = __float2bfloat16_rn(x - __bfloat162float(h));
  } else {
    *reinterpret_cast<__nv_fp8_e4m3*>(hi + o) = __nv_fp8_e4m3(x);
  }
}

// Registers of one stage: 2 operands x 128 rows x KC values over 256 threads.
// lo == 1 (rows contiguous): thread t owns row t % 128 and 16 consecutive c.
// lo > 1  (c contiguous):    thread t owns c = t % 32 and 16 rows.
struct StageRegs {
  float a[16], b[16];
};

template <bool TWO>
__device__ __forceinline__ void fetch_stage(const float* __restrict__ y, int lo, int n, int c_end, int i0a, int i0b,
                                            int c0, const float* __restrict__ rscale, StageRegs& r) {
  const int t = threadIdx.x;
  if (lo == 1) {
    const int row = t % BM, kg = (t / BM) * 16;
    const int ia = i0a + row, ib = i0b + row;
    const float sa = (rscale && ia < n) ? rscale[ia] : 1.f;
    const float sb = (rscale && ib < n) ? rscale[ib] : 1.f;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int c = c0 + kg + e;
      const bool cv = c < c_end;
      r.a[e] = (cv && ia < n) ? __ldg(y + (ia + n * c)) * sa : 0.f;
      if (TWO) r.b[e] = (cv && ib < n) ? __ldg(y + (ib + n * c)) * sb : 0.f;
    }
  } else {
    const int kk = t % KC, rg = t / KC;  // rg in [0, 8)
    const int c = c0 + kk;
    const bool cv = c < c_end;
    const int ca = cv ? c % lo : 0, cb = cv ? c / lo : 0;
    const float* base = y + (ca + lo * n * cb);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int row = rg + 8 * e;
      const int ia = i0a + row, ib = i0b + row;
      r.a[e] = (cv && ia < n) ? __ldg(base + lo * ia) * (rscale ? rscale[ia] : 1.f) : 0.f;
      if (TWO) r.b[e] = (cv && ib < n) ? __ldg(base + lo * ib) * (rscale ? rscale[ib] : 1.f) : 0.f;
    }
  }
}

template <int P, bool TWO>
__device__ __forceinline__ void store_stage(unsigned char* st, int lo, const StageRegs& r) {
  using SG = Stage<P>;
  constexpr int ES = Form<P>::ES;
  unsigned char* ahi = st;
  unsigned char* alo = st + SG::ARRB;
  unsigned char* bhi = st + SG::OPB;
  unsigned char* blo = st + SG::OPB + SG::ARRB;
  const int t = threadIdx.x;
  if (lo == 1) {
    const int row = t % BM, kg = (t / BM) * 16;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const uint32_t o = koff(row, (kg + e) * ES, SG::SBO);
      put<P>(ahi, alo, o, r.a[e]);
      if (TWO) put<P>(bhi, blo, o, r.b[e]);
    }
  } else {
    const int kk = t % KC, rg = t / KC;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const uint32_t o = koff(rg + 8 * e, kk * ES, SG::SBO);
      put<P>(ahi, alo, o, r.a[e]);
      if (TWO) put<P>(bhi, blo, o, r.b[e]);
    }
  }
}

// One Gram tile (ti, tj) over c in [split * kc, min(J, (split + 1) * kc)).
template <int P, bool DIAG>
__global__ void __launch_bounds__(THREADS) tc_gram_kernel(const float* __restrict__ y, int lo, int n, int hi, int T,
                                                          int kc, const float* __restrict__ rscale,
                                                          float* __restrict__ part, int* __restrict__ status) {
  using SG = Stage<P>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bars[STAGES];
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid / 32;
  const int split = blockIdx.y;
  int ti, tj;
  if (DIAG) {
    ti = tj = blockIdx.x;
  } else {
    int id = blockIdx.x;
    ti = 0;
    while (id >= T - 1 - ti) { id -= T - 1 - ti; ++ti; }
    tj = ti + 1 + id;
  }
  const int tile = ti * T - ti * (ti - 1) / 2 + (tj - ti);
  const int J = lo * hi;
  const int cb = split * kc, ce = min(J, cb + kc);
  const int nst = cb < ce ? (ce - cb + KC - 1) / KC : 0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(BM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    failed = 0;
    for (int s = 0; s < STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[s])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = (1u << 4) | ((uint32_t)Form<P>::FMT << 7) | ((uint32_t)Form<P>::FMT << 10) |
                             ((uint32_t)(BM >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  const int i0a = ti * BM, i0b = tj * BM;

  StageRegs regs;
  int last = -1;  // last stage whose MMAs were committed
  if (nst > 0) fetch_stage<!DIAG>(y, lo, n, ce, i0a, i0b, cb, rscale, regs);
  for (int s = 0; s < nst; ++s) {
    const int slot = s % STAGES;
    unsigned char* st = smem + slot * SG::BYTES;
    if (s >= STAGES) {
      // the MMAs that last read this slot (stage s - STAGES) must be done
      if (!mbar_wait(smem_u32(&bars[slot]), (uint32_t)(((s / STAGES) - 1) & 1))) failed = 1;
      __syncthreads();
      if (failed) break;
    }
    store_stage<P, !DIAG>(st, lo, regs);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (s + 1 < nst) fetch_stage<!DIAG>(y, lo, n, ce, i0a, i0b, cb + (s + 1) * KC, rscale, regs);
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(st), b0 = DIAG ? a0 : smem_u32(st + SG::OPB);
#pragma unroll
      for (int j = 0; j < SG::KSTEPS; ++j) {
        const uint32_t acc = (s > 0 || j > 0) ? 1u : 0u;
        const uint32_t off = j * 256;
        mma(tmem, sdesc(a0 + off, 128, SG::SBO), sdesc(b0 + off, 128, SG::SBO), idesc, acc, Form<P>::KIND);
        if (P == ATK_BF16X3) {
          const uint32_t al = a0 + SG::ARRB, bl = b0 + SG::ARRB;
          mma(tmem, sdesc(a0 + off, 128, SG::SBO), sdesc(bl + off, 128, SG::SBO), idesc, 1u, 0);
          mma(tmem, sdesc(al + off, 128, SG::SBO), sdesc(b0 + off, 128, SG::SBO), idesc, 1u, 0);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bars[slot])));
    }
    last = s;
  }
  // Wait for the last committed stage; a commit covers every MMA the thread
  // issued before it, so this drains all of them.
  bool ok = !failed;
  if (last >= 0) {
    bool done = mbar_wait(smem_u32(&bars[last % STAGES]), (uint32_t)((last / STAGES) & 1));
    if (!done) done = mbar_wait(smem_u32(&bars[last % STAGES]), (uint32_t)((last / STAGES) & 1));
    ok = ok && done;
  }
  if (!ok && tid == 0) atomicOr(status, DEV_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  const int ntiles = T * (T + 1) / 2;
  float* out = part + ((size_t)split * ntiles + tile) * (BM * BM);
  // Epilogue: warp w reads lanes 32 (w % 4) .. +31, columns 64 (w / 4) .. +63.
  const int q = warp % 4, h = warp / 4;
  const int row = 32 * q + (tid % 32);
#pragma unroll
  for (int c0 = 0; c0 < 64; c0 += 16) {
    uint32_t r[16];
    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(64 * h + c0);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
    float4* o4 = reinterpret_cast<float4*>(out + (size_t)row * BM + 64 * h + c0);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float4 f;
      f.x = (ok && last >= 0) ? __uint_as_float(r[4 * v + 0]) : 0.f;
      f.y = (ok && last >= 0) ? __uint_as_float(r[4 * v + 1]) : 0.f;
      f.z = (ok && last >= 0) ? __uint_as_float(r[4 * v + 2]) : 0.f;
      f.w = (ok && last >= 0) ? __uint_as_float(r[4 * v + 3]) : 0.f;
      o4[v] = f;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BM));
}

// Row scales for FP8: s_i = 2^floor(log2(448 / max_c |y_ic|)) (1 for an all-zero row).
// One CTA per row i; the view's c runs over (a, b) pairs.
__global__ void rowscale_kernel(const float* __restrict__ y, int lo, int n, int hi, float* __restrict__ scale) {
  __shared__ float red[256];
  const int i = blockIdx.x;
  float m = 0.f;
  const int J = lo * hi;
  for (int c = threadIdx.x; c < J; c += blockDim.x) {
    const int a = c % lo, b = c / lo;
    m = fmaxf(m, fabsf(y[a + lo * (i + n * b)]));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    float mx = red[0];
    scale[i] = mx > 0.f ? exp2f(floorf(log2f(448.f / mx))) : 1.f;
  }
}

// Float64 reduction of the split partials (diagonal tiles ns_d splits,
// off-diagonal ns_o), with the optional FP8 row scales undone exactly.
__global__ void tc_reduce_sym_kernel(const float* __restrict__ part, int ns_d, int ns_o, int ntiles, int T, int n,
                                     const float* __restrict__ rscale, double* __restrict__ C) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (i > j) return;
  const int ti = i / BM, tj = j / BM;
  const int id = ti * T - ti * (ti - 1) / 2 + (tj - ti);
  const int64_t o = (int64_t)(i - ti * BM) * BM + (j - tj * BM);
  const int ns = ti == tj ? ns_d : ns_o;
  double s = 0.0;
  for (int sp = 0; sp < ns; ++sp) s += (double)part[((int64_t)sp * ntiles + id) * BM * BM + o];
  if (rscale) s /= (double)rscale[i] * (double)rscale[j];
  C[i + (int64_t)n * j] = s;
  C[j + (int64_t)n * i] = s;
}

struct TcSplit {
  int nsplit, kc;
};
TcSplit tc_split(int64_t J, int ntiles, int slots) {
  // Each partial sum stays within 8192 terms of float32 accumulation, and the
  // launch fills whole waves.
  const int64_t min_split = ceil_div(J, 8192);
  const int64_t waves = std::max<int64_t>(1, ceil_div(min_split * ntiles, slots));
  int64_t ns = std::max<int64_t>(min_split, (waves * slots) / ntiles);
  ns = std::min<int64_t>(ns, std::max<int64_t>(1, ceil_div(J, KC)));
  int64_t kc = ceil_div(ceil_div(J, ns), KC) * KC;
  ns = ceil_div(J, kc);
  return {(int)std::max<int64_t>(1, ns), (int)kc};
}

template <int P>
int stage_bytes() {
  return STAGES * Stage<P>::BYTES;
}

template <int P>
int slots_per_sm() {
  int per = 0;
  // Requested shared memory also caps residency at 4 CTAs (TMEM: 4 x 128 columns).
  size_t sm = std::max<size_t>((size_t)stage_bytes<P>(), 57 * 1024);
  cudaFuncSetAttribute(tc_gram_kernel<P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(tc_gram_kernel<P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tc_gram_kernel<P, false>, THREADS, sm);
  return std::max(1, std::min(per, 4));
}

struct TcPlan {
  int T, nt;
  TcSplit d, o;
  size_t smem;
};

template <int P>
TcPlan tc_plan(const View& v) {
  TcPlan g;
  g.T = (int)ceil_div(v.n, BM);
  g.nt = g.T * (g.T + 1) / 2;
  const int slots = slots_per_sm<P>() * num_sms();
  g.d = tc_split(v.J(), g.T, slots);
  g.o = g.T > 1 ? tc_split(v.J(), g.T * (g.T - 1) / 2, slots) : g.d;
  g.smem = std::max<size_t>((size_t)stage_bytes<P>(), 57 * 1024);
  return g;
}

template <int P>
size_t tc_scratch_t(const View& v) {
  TcPlan g = tc_plan<P>(v);
  return (size_t)std::max(g.d.nsplit, g.o.nsplit) * g.nt * BM * BM * sizeof(float) + (size_t)v.n * sizeof(float) +
         256;
}

template <int P>
int tc_gram_t(const float* y, const View& v, double* S, float* scratch, size_t scratch_bytes, int* status,
              cudaStream_t st) {
  TcPlan g = tc_plan<P>(v);
  if (tc_scratch_t<P>(v) > scratch_bytes) {
    set_error("tc_gram: scratch too small");
    return ATK_EINVAL;
  }
  float* part = scratch;
  float* rscale = nullptr;
  if (P == ATK_FP8E4M3) {
    rscale = scratch + (size_t)std::max(g.d.nsplit, g.o.nsplit) * g.nt * BM * BM;
    rowscale_kernel<<<(unsigned)v.n, 256, 0, st>>>(y, (int)v.lo, (int)v.n, (int)v.hi, rscale);
    ATK_LAUNCHED();
  }
  tc_gram_kernel<P, true><<<dim3(g.T, g.d.nsplit), THREADS, g.smem, st>>>(y, (int)v.lo, (int)v.n, (int)v.hi, g.T,
                                                                            g.d.kc, rscale, part, status);
  ATK_LAUNCHED();
  if (g.T > 1) {
    tc_gram_kernel<P, false><<<dim3(g.T * (g.T - 1) / 2, g.o.nsplit), THREADS, g.smem, st>>>(
        y, (int)v.lo, (int)v.n, (int)v.hi, g.T, g.o.kc, rscale, part, status);
    ATK_LAUNCHED();
  }
  tc_reduce_sym_kernel<<<(unsigned)ceil_div(v.n * v.n, 256), 256, 0, st>>>(part, g.d.nsplit, g.o.nsplit, g.nt, g.T,
                                                                            (int)v.n, rscale, S);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace tc

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
