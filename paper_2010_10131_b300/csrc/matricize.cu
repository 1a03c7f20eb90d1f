// Explicit matricization: the baseline that Sec. V removes (the ablation of
// Sec. VI-E, Fig. 7).  With ATK_OPT_EXPLICIT_UNFOLD a plan copies the
// mode-n unfolding of the current tensor into a buffer before the mode's
// contractions (Alg. 2 writes "Mode-n matricization" as a step) and folds
// the TTM result back afterwards.  Both copies are batched transposes of the
// view's slabs: the tensor's mode-n view (lo, n, hi) is hi column-major
// lo x n slabs; the unfolding stores the n x J matrix column-major, i.e. the
// same slabs transposed (element (i, a + lo b) at i + n (a + lo b)).  The
// contractions then see a mode-1 view (1, n, J), and the TTM writes an
// R x J matrix whose hi slabs R x lo are transposed back into the
// (lo, R, hi) layout.
#include <algorithm>

#include "atk_internal.cuh"

namespace atk {

namespace {
constexpr int PT = 32;  // tile edge

// dst slab b (B x A, column-major) = transpose of src slab b (A x B,
// column-major), for b in [0, count).  32 x 32 tiles through shared memory
// (padded row, so both the reads and the writes are coalesced and the
// transposed shared-memory reads are conflict-free); grid x enumerates the
// tiles of a slab (gx along A), grid y strides over the slabs.
__global__ void __launch_bounds__(PT * 8) permute_slabs_kernel(const float* __restrict__ src, int64_t A, int64_t B,
                                                               int64_t count, int64_t gx, float* __restrict__ dst) {
  __shared__ float tile[PT][PT + 1];
  const int64_t p0 = ((int64_t)blockIdx.x % gx) * PT, q0 = ((int64_t)blockIdx.x / gx) * PT;
  const int tx = threadIdx.x % PT, ty = threadIdx.x / PT;  // 32 x 8 threads
  for (int64_t b = blockIdx.y; b < count; b += gridDim.y) {
    const float* s = src + b * A * B;
    float* d = dst + b * A * B;
    for (int k = ty; k < PT; k += 8) {
      const int64_t p = p0 + tx, q = q0 + k;
      if (p < A && q < B) tile[k][tx] = s[p + A * q];
    }
    __syncthreads();
    for (int k = ty; k < PT; k += 8) {
      const int64_t q = q0 + tx, p = p0 + k;
      if (p < A && q < B) d[q + B * p] = tile[tx][k];
    }
    __syncthreads();
  }
}
}  // namespace

int permute_slabs(const float* src, int64_t A, int64_t B, int64_t count, float* dst, cudaStream_t st) {
  if (A <= 0 || B <= 0 || count <= 0) return ATK_OK;
  const int64_t gx = ceil_div(A, PT), tiles = gx * ceil_div(B, PT);
  if (tiles > 0x7fffffff) { set_error("permute_slabs: slab too large"); return ATK_EUNSUPPORTED; }
  const unsigned gy = (unsigned)std::min<int64_t>(count, 65535);
  permute_slabs_kernel<<<dim3((unsigned)tiles, gy), PT * 8, 0, st>>>(src, A, B, count, gx, dst);
  ATK_LAUNCHED();
  return ATK_OK;
}

}  // namespace atk
