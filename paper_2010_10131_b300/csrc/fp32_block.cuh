// Register-tiled float32 outer-product block shared by the CUDA-core
// contraction kernels (fp32_ops.cu: Gram, cross product, TTM; ttm_gram.cu:
// the fused TTM and next-mode Gram).  A CTA of NT = 256 threads owns a
// BM x BN tile; each thread accumulates TM x TN of it from operand tiles
// staged in shared memory as s[k * (W + PAD) + m].
#pragma once

#include "atk_internal.cuh"

namespace atk {

constexpr int NT = 256;   // threads per CTA
constexpr int TK = 16;    // k-tile depth
constexpr int PAD = 4;    // smem row padding (floats); keeps 16-byte row alignment

// ----------------------------------------------------------- register block
// Packed float32 pairs (PTX fma.rn.f32x2, sm_100 and later): one instruction
// does two FMAs, so the outer product takes half the issue slots it would with
// scalar FMAs.  These kernels are issue-bound: every shared-memory load and
// address computation competes with the FMAs for the scheduler.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(r));
  return f;
}
__device__ __forceinline__ void fma2(unsigned long long& c, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(a), "l"(b));
}

template <int BM, int BN, int TM, int TN, bool X2 = true>
struct Block {
  static constexpr int TX = BN / TN, TY = BM / TM;
  static_assert(TX * TY == NT, "thread grid must cover 256 threads");
  static constexpr bool PAIRS = X2 && TN % 2 == 0;
  // Accumulators: column pairs (v, v+1) packed in one 64-bit register when
  // TN is even, scalars otherwise.
  unsigned long long acc2[TM][PAIRS ? TN / 2 : 1];
  float acc1[TM][PAIRS ? 1 : TN];
  int tx, ty;
  __device__ void init() {
    tx = threadIdx.x % TX; ty = threadIdx.x / TX;
#pragma unroll
    for (int u = 0; u < TM; ++u) {
      if constexpr (PAIRS) {
#pragma unroll
        for (int p = 0; p < TN / 2; ++p) acc2[u][p] = 0ull;
      } else {
#pragma unroll
        for (int v = 0; v < TN; ++v) acc1[u][v] = 0.f;
      }
    }
  }
  __device__ float acc(int u, int v) const {
    if constexpr (PAIRS) {
      const float2 f = unpack2(acc2[u][v / 2]);
      return (v & 1) ? f.y : f.x;
    } else {
      return acc1[u][v];
    }
  }
  __device__ static int row_of(int ty, int u) {
    return (u < TM / 2) ? ty * (TM / 2) + u : BM / 2 + ty * (TM / 2) + (u - TM / 2);
  }
  __device__ static int col_of(int tx, int v) {
    if (TN == 1) return tx;
    return (v < TN / 2) ? tx * (TN / 2) + v : BN / 2 + tx * (TN / 2) + (v - TN / 2);
  }
  // Load H = TM/2 (or TN/2) consecutive floats starting at a 4*H-byte aligned address.
  template <int H>
  __device__ static void ld(float* dst, const float* src) {
    if (H == 4) {
      float4 t = *reinterpret_cast<const float4*>(src);
      dst[0] = t.x; dst[1] = t.y; dst[2] = t.z; dst[3] = t.w;
    } else if (H == 2) {
      float2 t = *reinterpret_cast<const float2*>(src);
      dst[0] = t.x; dst[1] = t.y;
    } else {
#pragma unroll
      for (int h = 0; h < H; ++h) dst[h] = src[h];
    }
  }
  // SKIP_LOWER (diagonal Gram tiles, BM == BN): leave out the accumulators of
  // the lower-left quadrant (rows >= BM/2, columns < BN/2), which lie wholly
  // below the diagonal and are never read; a quarter of the tile's FMAs.
  // One k step: the outer product of row k of the staged A and B tiles
  // (row strides LDA, LDB floats).
  template <bool SKIP_LOWER, int LDA, int LDB>
  __device__ __forceinline__ void step(const float* sa, const float* sb, int k) {
    float a[TM], b[TN];
    ld<TM / 2>(a, sa + k * LDA + ty * (TM / 2));
    ld<TM / 2>(a + TM / 2, sa + k * LDA + BM / 2 + ty * (TM / 2));
    if constexpr (PAIRS) {
      ld<TN / 2>(b, sb + k * LDB + tx * (TN / 2));
      ld<TN / 2>(b + TN / 2, sb + k * LDB + BN / 2 + tx * (TN / 2));
      unsigned long long b2[TN / 2];
#pragma unroll
      for (int p = 0; p < TN / 2; ++p) b2[p] = pack2(b[2 * p], b[2 * p + 1]);
#pragma unroll
      for (int u = 0; u < TM; ++u) {
        const unsigned long long a2 = pack2(a[u], a[u]);
#pragma unroll
        for (int p = 0; p < TN / 2; ++p)
          if (!(SKIP_LOWER && u >= TM / 2 && p < TN / 4)) fma2(acc2[u][p], a2, b2[p]);
      }
    } else {
      if (TN == 1) {
        b[0] = sb[k * LDB + tx];
      } else {
        ld<TN / 2>(b, sb + k * LDB + tx * (TN / 2));
        ld<TN / 2>(b + TN / 2, sb + k * LDB + BN / 2 + tx * (TN / 2));
      }
#pragma unroll
      for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v)
          if (!(SKIP_LOWER && TN > 1 && u >= TM / 2 && v < TN / 2)) acc1[u][v] = fmaf(a[u], b[v], acc1[u][v]);
    }
  }
  template <bool SKIP_LOWER = false, int KT = TK, int LDA = BM + PAD, int LDB = BN + PAD>
  __device__ void mma(const float* sa, const float* sb) {
#pragma unroll
    for (int k = 0; k < KT; ++k) step<SKIP_LOWER, LDA, LDB>(sa, sb, k);
  }
};

}  // namespace atk
