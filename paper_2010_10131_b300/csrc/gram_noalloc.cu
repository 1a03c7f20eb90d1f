// Gram entry point that allocates no device memory.
//
// Some callers cannot allocate GPU memory at call time.  Examples: a service
// that reserves its whole memory budget up front, code running under a
// framework whose caching allocator already owns the free device memory, or
// a hook that must not re-enter the CUDA allocator.  For them, the split-K
// partial tiles of the Gram product live in the fixed device array below.
// The library's module carries the array, so every GPU that loads the library
// holds it until the process exits.
#include <mutex>

#include "atk_internal.cuh"

namespace atk {

// 16 MiB of float32 partial tiles: enough for one split of any n <= 2048
// (136 tiles of 128 x 128).  When a view needs more splits than fit, they run
// in rounds (gram_f32_fixed_scratch), so every float32 chain stays as short
// as in atucker_gram.
constexpr size_t NOALLOC_GRAM_FLOATS = size_t(4) << 20;
static __device__ __align__(256) float g_gram_partials[NOALLOC_GRAM_FLOATS];

// Device address of g_gram_partials for each device, looked up once with that
// device current.  In host code the array's name is only a host-side stand-in,
// so kernels must be handed this address instead.  The lookup can load the
// library's module on that device (which reserves the array), and the cached
// address belongs to that context: after a device reset, use a new process.
static std::mutex g_partials_mutex;
static float* g_partials_ptr[64] = {nullptr};

static int partials_for_current_device(float** out) {
  int dev = 0;
  ATK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("gram_noalloc: device index out of range");
    return ATK_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_partials_mutex);
  if (!g_partials_ptr[dev]) {
    float* p = nullptr;
    ATK_CUDA(cudaGetSymbolAddress((void**)&p, g_gram_partials));
    g_partials_ptr[dev] = p;
  }
  *out = g_partials_ptr[dev];
  return ATK_OK;
}

}  // namespace atk

using namespace atk;

extern "C" int atucker_gram_noalloc(const float* y, int64_t lo, int64_t n, int64_t hi, double* S_out, void* stream) {
  if (!y || !S_out) { set_error("null argument"); return ATK_EINVAL; }
  if (lo < 1 || n < 1 || hi < 1) { set_error("view extents must be >= 1"); return ATK_EINVAL; }
  if ((double)lo * (double)n * (double)hi >= 2147483648.0) {
    set_error("tensor must have fewer than 2^31 elements");
    return ATK_EUNSUPPORTED;
  }
  if (n > 2048) {
    set_error("gram_noalloc: n > 2048 does not fit the fixed 16 MiB scratch; use atucker_gram");
    return ATK_EUNSUPPORTED;
  }
  float* partials = nullptr;
  ATK_TRY(partials_for_current_device(&partials));
  // Every partial tile the reduction reads is written by this call's Gram
  // kernel first, so nothing in the array needs clearing.
  View v{lo, n, hi};
  return gram_f32_fixed_scratch(y, v, S_out, partials, NOALLOC_GRAM_FLOATS * sizeof(float), (cudaStream_t)stream);
}
