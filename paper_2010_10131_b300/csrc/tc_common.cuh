// tcgen05 building blocks shared by the tensor-core Gram (tc_ops.cu) and the
// tensor-core TTM (tc_ttm.cu): the shared-memory matrix descriptor, the
// operand formats of the precision forms and the MMA issue (PTX ISA,
// tcgen05.mma with a kind::f16 / kind::tf32 / kind::f8f6f4 operand pair).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "atucker.h"

namespace atk {
namespace tc {

// tcgen05 shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

template <int P>
struct Form;
// ES: element bytes; ARR: arrays per block (hi [, lo]); FMT: MMA operand format
// code; KIND: 0 kind::f16, 1 kind::tf32, 2 kind::f8f6f4.
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

// FP8 row scale from the row max: 2^(8 - e) with max in [2^(e-1), 2^e).
__device__ __forceinline__ float fp8_row_scale(float m) {
  if (!(m > 0.f)) return 1.f;
  int e;
  frexpf(m, &e);
  e = min(max(8 - e, -126), 127);
  return ldexpf(1.f, e);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

}  // namespace tc
}  // namespace atk
