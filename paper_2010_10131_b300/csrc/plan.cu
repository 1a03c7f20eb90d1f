// Plan, mode loop (Alg. 2) and the C ABI of the library.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "atk_internal.cuh"

namespace atk {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
int cuda_status(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return ATK_ENOMEM;
  return ATK_ECUDA;
}
// Kernel launches are counted per host thread: a plan's run happens on one
// thread, so its launches are the thread's count before and after, even when
// other plans run on other threads (atucker_sthosvd_many).
static thread_local long long t_launches = 0;
void count_launch() { ++t_launches; }
long long launch_count() { return t_launches; }
void count_launches(long long k) { t_launches += k; }

static std::atomic<unsigned long long> g_alloc_limit{0};
static int alloc_over_limit(size_t bytes, const char* what) {
  const unsigned long long lim = g_alloc_limit.load();
  if (lim && bytes > lim) {
    g_err = std::string("device allocation above the library's limit: ") + what;
    return ATK_ENOMEM;
  }
  return ATK_OK;
}
int dev_alloc(void** ptr, size_t bytes, const char* what) {
  *ptr = nullptr;
  ATK_TRY(alloc_over_limit(bytes, what));
  const cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) { *ptr = nullptr; return cuda_status(e, what); }
  return ATK_OK;
}
int dev_alloc_async(void** ptr, size_t bytes, cudaStream_t st, const char* what) {
  *ptr = nullptr;
  ATK_TRY(alloc_over_limit(bytes, what));
  const cudaError_t e = cudaMallocAsync(ptr, bytes, st);
  if (e != cudaSuccess) { *ptr = nullptr; return cuda_status(e, what); }
  return ATK_OK;
}
static thread_local long long t_wait_limit = 0;
void set_wait_limit(long long polls) { t_wait_limit = polls; }
long long wait_limit() { return t_wait_limit; }

int num_sms() {
  static const int sms = [] {  // thread-safe one-time initialisation
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return sms;
}

// ALS initial guess L_0 (Alg. 3 input; the paper leaves it open).  N(0,1)
// entries: Box-Muller on a counter-based splitmix64 stream (Steele, Lea and
// Flood, OOPSLA 2014).  The c-th output of the stream with state s is
// mix(s + c * 0x9E3779B97F4A7C15).
static uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static void als_initial_guess(uint64_t seed, int mode, int64_t I, int64_t R, double* out) {
  const uint64_t gamma = 0x9E3779B97F4A7C15ULL;
  const uint64_t state = seed ^ (gamma * (uint64_t)(mode + 1));
  const double inv53 = 1.0 / 9007199254740992.0;
  for (int64_t e = 0; e < I * R; ++e) {
    uint64_t w1 = splitmix_mix(state + (2 * (uint64_t)e + 1) * gamma) >> 11;
    uint64_t w2 = splitmix_mix(state + (2 * (uint64_t)e + 2) * gamma) >> 11;
    double u1 = ((double)w1 + 1.0) * inv53, u2 = (double)w2 * inv53;
    out[e] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
}

__global__ void sub_kernel(const double* a, const double* b, double* out) { *out = *a - *b; }

// Classes predicted within this of the best (log2 of the time ratio: 4 x), at
// most SELECTOR_SEARCH_MAX of them, are settled by timing them at the plan's
// first run.  On the 64 held-out shapes of the selector workload the regret
// is 4.5 % for the network alone, 3.3 % with a margin of 0.3 (193 of 258
// modes searched) and 0.12 % with this one (257 searched): the timing labels
// age as the kernels change, and the network's three best fitting classes
// nearly always hold the fastest.
constexpr float SELECTOR_MARGIN = 2.0f;
constexpr int SELECTOR_SEARCH_MAX = 3;

// Below this rank the float32 TTM reads Y at HBM speed, and the tensor-core
// TTM of the precision forms is no faster (measured at I_n = 128, R = 16).
constexpr int64_t TC_TTM_MIN_R = 16;

// Phase slots of atucker_plan_timings.
enum { PH_GRAM = 0, PH_GRAM_REDUCE, PH_EIG, PH_TTM, PH_ALS, PH_OTHER, PH_TOTAL, PH_SLOTS = PH_TOTAL + 4 };

// ------------------------------------------------------------ ALS mode update
struct AlsBufs {
  double *L, *Lt, *G, *A, *B, *Rhat;
  float *Lt32, *M32, *P;
  char* scratch;
  size_t scratch_bytes;
  int* dev_status;
};

static size_t als_scratch_need(const View& v, int64_t R) {
  size_t s = std::max(cross_scratch_bytes(v, R), als_fused_scratch_bytes(v, R));
  s = std::max(s, smallla_scratch_bytes(std::max(v.n, R), R));
  return s;
}

// One ALS solve (Alg. 3 with `sweeps` iterations), QR of L (CholeskyQR2 in
// float64, the unique QR with diag(R^) > 0), and the core update
// Y' = R_{K-1} x_n R^ written to `out` (a (lo, R, hi) tensor).
// A sweep needs A = Y R_k with R_k = Y^T L~, and B = R_k^T R_k, which equals
// L~^T A: only A is taken from the tensor.  Small modes (I_n <= 256, R <= 32)
// form A in one fused pass over Y that keeps R_k on chip (als_fused.cu) and
// write R_k only on the last sweep; the others run the TTM kernel for R_k and
// the cross kernel for A.
static int als_mode_run(const float* y, const View& v, int64_t R, const double* L0, int sweeps, float* U_out,
                        float* out, AlsBufs& b, cudaStream_t st) {
  const int64_t n = v.n;
  View vp{v.lo, R, v.hi};
  double* ss = (double*)b.scratch;
  const bool fused = als_fused_ok(v, R);
  ATK_CUDA(cudaMemcpyAsync(b.L, L0, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, st));
  for (int k = 0; k < sweeps; ++k) {
    const bool last = k == sweeps - 1;
    // L~ = L_k (L_k^T L_k)^{-1}.
    ATK_TRY(gemm_tn_f64(b.L, b.L, n, R, b.G, st));
    ATK_CUDA(cudaMemcpyAsync(b.Lt, b.L, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, st));
    ATK_TRY(solve_spd_right_f64(b.Lt, n, R, b.G, ss, b.dev_status, st));
    ATK_TRY(f64_to_f32(b.Lt, b.Lt32, n * R, st));
    // A = Y R_k with R_k = Y^T L~ (R_k kept, as a (lo, R, hi) tensor, on the last sweep).
    if (fused) {
      ATK_TRY(als_fused(y, v, b.Lt32, R, b.A, last ? b.P : nullptr, (float*)b.scratch, b.scratch_bytes, st));
    } else {
      ATK_TRY(ttm_f32(y, v, b.Lt32, R, b.P, st));
      ATK_TRY(cross_f32(y, v, b.P, R, b.A, (float*)b.scratch, b.scratch_bytes, st));
    }
    // B = R_k^T R_k = L~^T A; L_{k+1} = A B^{-1}.
    ATK_TRY(gemm_tn_f64(b.Lt, b.A, n, R, b.B, st));
    ATK_TRY(solve_spd_right_f64(b.A, n, R, b.B, ss, b.dev_status, st));
    ATK_CUDA(cudaMemcpyAsync(b.L, b.A, sizeof(double) * n * R, cudaMemcpyDeviceToDevice, st));
  }
  // L_K = Q^ R^; U = Q^; Y' = TTM(R_{K-1}, R^).
  ATK_TRY(cholqr2_f64(b.L, n, R, b.Rhat, ss, b.dev_status, st));
  ATK_TRY(f64_to_f32(b.L, U_out, n * R, st));
  ATK_TRY(transpose_f64_to_f32(b.Rhat, R, b.M32, st));
  ATK_TRY(ttm_f32(b.P, vp, b.M32, R, out, st));
  return ATK_OK;
}

}  // namespace atk

using namespace atk;

// ====================================================================== plan
struct atucker_plan_s {
  int order = 0;
  int64_t dims[8], ranks[8], foff[8];
  int mode_order[8], solver[8];
  int cls[8], eigm[8], gbm[8];  // per-mode class, eigensolver method (-1 = plan's), Gram row tile (0 = auto)
  int precision = ATK_FP32, als_sweeps = 5;
  uint64_t seed = 0;
  cudaStream_t st = nullptr;
  int eig_arith = ATK_EIG_ROT_FP32, eig_method = ATK_EIG_AUTO, sync = 0, max_sweeps = 40, gram_refine = 1;
  long long wait_polls = 0;  // ATK_OPT_WAIT_LIMIT (0: default)
  int explicit_unfold = 0;  // ATK_OPT_EXPLICIT_UNFOLD
  int fuse_tg = 0;          // ATK_OPT_FUSE_TTM_GRAM
  // Exhaustive timed search (AUTO modes without a confident prediction):
  // candidate classes per mode, timed at the first run.
  int ncand[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int cand[8][ATK_NUM_CLASSES];
  bool tune_pending = false;
  bool both[8] = {false, false, false, false, false, false, false, false};  // workspace for EIG and ALS
  float* xunf = nullptr;     // unfolding buffer and TTM result of the explicit form (one allocation)
  float* xttm = nullptr;
  // device workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  float* buf[2] = {nullptr, nullptr};
  float* bufP = nullptr;
  double *S = nullptr, *U64 = nullptr, *norms = nullptr, *L0 = nullptr;
  int64_t l0off[8];
  AlsBufs als{};
  char* scratch = nullptr;
  size_t scratch_bytes = 0;
  int* dev_status = nullptr;
  // phase timing (ATK_OPT_TIMING): events recorded on the plan's stream
  int timing = 0;
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  struct Rec { int phase; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  std::vector<Rec> mrecs;  // per-mode records: phase = mode index
  long long gram_launches = 0, runs = 0, launches = 0;
  cudaEvent_t ev() {
    if (evnext == evpool.size()) {
      cudaEvent_t e = nullptr;
      cudaEventCreate(&e);
      evpool.push_back(e);
    }
    return evpool[evnext++];
  }
  // host-buffer entry point
  float *x_dev = nullptr, *core_dev = nullptr, *fac_dev = nullptr;
  double* disc_dev = nullptr;
  int64_t total = 0, core_total = 0, fac_total = 0;
};

static int validate(int order, const int64_t* dims, const int64_t* ranks, const int* mode_order,
                    const int* solver) {
  if (order < 1 || order > 8 || !dims || !ranks) { set_error("order must be in [1, 8]; dims/ranks non-null"); return ATK_EINVAL; }
  double total = 1.0;
  for (int k = 0; k < order; ++k) {
    if (dims[k] < 1) { set_error("dims must be >= 1"); return ATK_EINVAL; }
    total *= (double)dims[k];
  }
  if (total >= 2147483648.0) { set_error("tensor must have fewer than 2^31 elements"); return ATK_EUNSUPPORTED; }
  for (int k = 0; k < order; ++k) {
    if (ranks[k] < 1 || ranks[k] > dims[k]) { set_error("need 1 <= R_n <= I_n"); return ATK_ERANK; }
    double others = 1.0;
    for (int j = 0; j < order; ++j)
      if (j != k) others *= (double)ranks[j];
    if (order > 1 && (double)ranks[k] > others) { set_error("need R_n <= prod_{k!=n} R_k"); return ATK_ERANK; }
    if (ranks[k] > 128) { set_error("R_n > 128 is not supported"); return ATK_EUNSUPPORTED; }
  }
  if (mode_order) {
    int seen[8] = {0};
    for (int k = 0; k < order; ++k) {
      if (mode_order[k] < 0 || mode_order[k] >= order || seen[mode_order[k]]) { set_error("mode_order must be a permutation"); return ATK_EINVAL; }
      seen[mode_order[k]] = 1;
    }
  }
  for (int k = 0; k < order; ++k) {
    int s = solver ? solver[k] : ATK_EIG;
    if (s != ATK_EIG && s != ATK_ALS && s != ATK_AUTO) {
      set_error("solver_per_mode entries must be 0 (EIG), 1 (ALS) or -1 (AUTO)");
      return ATK_EINVAL;
    }
    if (s == ATK_EIG && dims[k] > EIG_MAX_N) { set_error("EIG modes need I_n <= 32768"); return ATK_EUNSUPPORTED; }
  }
  return ATK_OK;
}

// The next mode's stride among the TTM rows of mode n and its size, when the
// fused TTM + next-mode Gram can run the step (float32 form only).  cur is the
// shape before mode n is truncated.
static bool fuse_geometry(const atucker_plan_s* p, int step, const int64_t* cur, const View& v, int64_t R,
                          int64_t* s, int64_t* Im) {
  // Only from a TTM whose rows are contiguous in k (lo == 1, the first mode
  // in storage order): for lo > 1 a group's fibres lie s apart in memory and
  // its loads do not coalesce, which costs more than the Gram pass saves.
  if (p->precision != ATK_FP32 || step + 1 >= p->order || v.lo != 1) return false;
  const int n = p->mode_order[step], m = p->mode_order[step + 1];
  int64_t st = 1;
  for (int k = 0; k < m; ++k)
    if (k != n) st *= cur[k];
  *s = st;
  *Im = cur[m];
  return ttm_gram_ok(v, R, st, cur[m]);
}

static int plan_alloc(atucker_plan_s* p) {
  int64_t cur[8];
  for (int k = 0; k < p->order; ++k) cur[k] = p->dims[k];
  size_t bufsz[2] = {0, 0}, pbuf = 0, scratch = 4096, s_elems = 1, u_elems = 1, l0_elems = 0;
  int64_t maxn = 1, maxr = 1;
  bool any_als = false;
  for (int step = 0; step < p->order; ++step) {
    int n = p->mode_order[step];
    View v = make_view(p->order, cur, n);
    int64_t R = p->ranks[n];
    size_t out_elems = (size_t)(v.J() * R);
    if (step < p->order - 1) bufsz[step & 1] = std::max(bufsz[step & 1], out_elems);
    u_elems = std::max(u_elems, (size_t)(v.n * R));
    maxn = std::max(maxn, v.n);
    maxr = std::max(maxr, R);
    if (p->solver[n] == ATK_EIG || p->both[n]) {
      s_elems = std::max(s_elems, (size_t)(v.n * v.n));
      scratch = std::max(scratch, gram_scratch_bytes(v, p->gbm[n]));
      if (p->ncand[n] > 0)  // a timed search may try the smaller Gram tile
        scratch = std::max(scratch, gram_scratch_bytes(v, std::max(32, gram_tile(v.n) / 2)));
      if (p->precision != ATK_FP32 && p->precision != ATK_FP32C) {
        scratch = std::max(scratch, tc_gram_scratch_bytes(v, p->precision));
        scratch = std::max(scratch, tc_ttm_scratch_bytes(v, R, p->precision));
      }
      scratch = std::max(scratch, gram_cmp_scratch_bytes(v));
      scratch = std::max(scratch, eig_scratch_bytes(v.n, ATK_EIG_ROT_FP64));
      scratch = std::max(scratch, eig_scratch_bytes(v.n, ATK_EIG_ROT_FP32));
      scratch = std::max(scratch, smallla_scratch_bytes(v.n, R));
      int64_t fs = 0, fim = 0;
      const int m = step + 1 < p->order ? p->mode_order[step + 1] : -1;
      if (m >= 0 && (p->solver[m] == ATK_EIG || p->both[m]) && fuse_geometry(p, step, cur, v, R, &fs, &fim))
        scratch = std::max(scratch, ttm_gram_scratch_bytes(v, R, fs, fim));
    }
    if (p->solver[n] == ATK_ALS || p->both[n]) {
      any_als = true;
      pbuf = std::max(pbuf, out_elems);
      scratch = std::max(scratch, als_scratch_need(v, R));
      p->l0off[n] = (int64_t)l0_elems;
      l0_elems += (size_t)(v.n * R);
    }
    cur[n] = R;
  }
  scratch = std::max(scratch, (size_t)NORM_SCRATCH_BYTES);
  size_t need = 0;
  auto add = [&](size_t b) { need += (b + 255) & ~size_t(255); };
  add(bufsz[0] * 4); add(bufsz[1] * 4); add(pbuf * 4);
  add(s_elems * 8); add(u_elems * 8); add(64 * 8); add(l0_elems * 8);
  if (any_als) {
    size_t nr = (size_t)(maxn * maxr), rr = (size_t)(maxr * maxr);
    add(nr * 8); add(nr * 8); add(rr * 8); add(nr * 8); add(rr * 8); add(rr * 8);
    add(nr * 4); add(rr * 4);
  }
  add(scratch); add(256);
  ATK_TRY(dev_alloc((void**)&p->ws, need, "cudaMalloc(plan workspace)"));
  p->ws_bytes = need;
  Arena ar{p->ws, need, 0};
  p->buf[0] = (float*)ar.take(bufsz[0] * 4);
  p->buf[1] = (float*)ar.take(bufsz[1] * 4);
  p->bufP = (float*)ar.take(pbuf * 4);
  p->S = (double*)ar.take(s_elems * 8);
  p->U64 = (double*)ar.take(u_elems * 8);
  p->norms = (double*)ar.take(64 * 8);
  p->L0 = (double*)ar.take(l0_elems * 8);
  if (any_als) {
    size_t nr = (size_t)(maxn * maxr), rr = (size_t)(maxr * maxr);
    p->als.L = (double*)ar.take(nr * 8);
    p->als.Lt = (double*)ar.take(nr * 8);
    p->als.G = (double*)ar.take(rr * 8);
    p->als.A = (double*)ar.take(nr * 8);
    p->als.B = (double*)ar.take(rr * 8);
    p->als.Rhat = (double*)ar.take(rr * 8);
    p->als.Lt32 = (float*)ar.take(nr * 4);
    p->als.M32 = (float*)ar.take(rr * 4);
  }
  p->scratch = (char*)ar.take(scratch);
  p->scratch_bytes = scratch;
  p->dev_status = (int*)ar.take(256);
  p->als.P = p->bufP;
  p->als.scratch = p->scratch;
  p->als.scratch_bytes = scratch;
  p->als.dev_status = p->dev_status;
  ATK_CUDA(cudaMemsetAsync(p->dev_status, 0, sizeof(int), p->st));
  if (l0_elems) {
    std::vector<double> h(l0_elems);
    for (int n = 0; n < p->order; ++n)
      if (p->solver[n] == ATK_ALS || p->both[n])
        als_initial_guess(p->seed, n, p->dims[n], p->ranks[n], h.data() + p->l0off[n]);
    ATK_CUDA(cudaMemcpyAsync(p->L0, h.data(), l0_elems * 8, cudaMemcpyHostToDevice, p->st));
    ATK_CUDA(cudaStreamSynchronize(p->st));
  }
  return ATK_OK;
}

extern "C" {

static int plan_create_impl(atucker_plan_t* plan, int order, const int64_t* dims, const int64_t* ranks,
                            const int* mode_order, const int* class_per_mode, int precision, int als_sweeps,
                            uint64_t seed, void* stream, const int* ncand, const int (*cand)[ATK_NUM_CLASSES]);

int atucker_plan_create(atucker_plan_t* plan, int order, const int64_t* dims, const int64_t* ranks,
                        const int* mode_order, const int* solver_per_mode, int precision, int als_sweeps,
                        uint64_t seed, void* stream) {
  if (!plan) { set_error("plan is null"); return ATK_EINVAL; }
  *plan = nullptr;
  ATK_TRY(validate(order, dims, ranks, mode_order, solver_per_mode));
  int cls[8];
  bool any_auto = false;
  for (int k = 0; k < order; ++k) {
    const int s = solver_per_mode ? solver_per_mode[k] : ATK_EIG;
    cls[k] = s == ATK_ALS ? ATK_CLASS_ALS : ATK_CLASS_EIG;
    any_auto = any_auto || s == ATK_AUTO;
  }
  int ncand[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int cand[8][ATK_NUM_CLASSES];
  if (any_auto) {
    double feat[8 * ATK_SELECTOR_FEATURES];
    int pick[8];
    float scores[8 * ATK_NUM_CLASSES];
    ATK_TRY(atucker_mode_features(order, dims, ranks, mode_order, feat));
    const bool have = selector_loaded() && atucker_selector_predict(feat, order, pick, scores) == ATK_OK;
    for (int k = 0; k < order; ++k) {
      if (solver_per_mode[k] != ATK_AUTO) continue;
      const double lg = feat[k * ATK_SELECTOR_FEATURES];  // log2 I_n
      if (have) {
        // The prediction, and up to two runners-up whose predicted times are
        // too close to it to call.
        cls[k] = pick[k];
        cand[k][0] = pick[k];
        ncand[k] = 1;
        const float* sk = scores + k * ATK_NUM_CLASSES;
        for (int extra = 0; extra < SELECTOR_SEARCH_MAX - 1; ++extra) {
          int next = -1;
          for (int c = 0; c < ATK_NUM_CLASSES; ++c) {
            bool taken = false;
            for (int j = 0; j < ncand[k]; ++j) taken = taken || cand[k][j] == c;
            if (!taken && selector_class_fits(c, lg) && (next < 0 || sk[c] < sk[next])) next = c;
          }
          if (next < 0 || sk[next] - sk[pick[k]] >= SELECTOR_MARGIN) break;
          cand[k][ncand[k]++] = next;
        }
        if (ncand[k] == 1) ncand[k] = 0;  // a clear call: no search
      } else {
        // No selector: every class that can run the mode is timed.
        for (int c = 0; c < ATK_NUM_CLASSES; ++c)
          if (selector_class_fits(c, lg)) cand[k][ncand[k]++] = c;
        cls[k] = selector_class_fits(ATK_CLASS_EIG, lg) ? ATK_CLASS_EIG : ATK_CLASS_ALS;
      }
    }
  }
  return plan_create_impl(plan, order, dims, ranks, mode_order, cls, precision, als_sweeps, seed, stream, ncand,
                          cand);
}

// Plan creation; ncand / cand (nullable): candidate classes of the modes that
// the first run settles by timing them (exhaustive search).
static int plan_create_impl(atucker_plan_t* plan, int order, const int64_t* dims, const int64_t* ranks,
                            const int* mode_order, const int* class_per_mode, int precision, int als_sweeps,
                            uint64_t seed, void* stream, const int* ncand, const int (*cand)[ATK_NUM_CLASSES]) {
  if (!plan) { set_error("plan is null"); return ATK_EINVAL; }
  *plan = nullptr;
  if (!class_per_mode) { set_error("class_per_mode is null"); return ATK_EINVAL; }
  int solver[8];
  if (order < 1 || order > 8) { set_error("order must be in [1, 8]; dims/ranks non-null"); return ATK_EINVAL; }
  for (int k = 0; k < order; ++k) {
    if (class_per_mode[k] < 0 || class_per_mode[k] >= ATK_NUM_CLASSES) { set_error("unknown mode class"); return ATK_EINVAL; }
    solver[k] = class_per_mode[k] == ATK_CLASS_ALS ? ATK_ALS : ATK_EIG;
  }
  ATK_TRY(validate(order, dims, ranks, mode_order, solver));
  for (int k = 0; k < order; ++k)
    if ((class_per_mode[k] == ATK_CLASS_EIG_JACOBI || class_per_mode[k] == ATK_CLASS_EIG_JACOBI_SMALL) &&
        dims[k] > JACOBI_MAX_N) {
      set_error("the full-Jacobi classes need I_n <= 1024");
      return ATK_EUNSUPPORTED;
    }
  if (precision < ATK_FP32 || precision > ATK_FP32C) { set_error("unsupported precision"); return ATK_EUNSUPPORTED; }
  atucker_plan_s* p = new atucker_plan_s();
  p->order = order;
  int64_t off = 0;
  for (int k = 0; k < order; ++k) {
    p->dims[k] = dims[k];
    p->ranks[k] = ranks[k];
    p->mode_order[k] = mode_order ? mode_order[k] : k;
    p->solver[k] = solver[k];
    p->cls[k] = class_per_mode[k];
    p->foff[k] = off;
    off += dims[k] * ranks[k];
  }
  // Per-mode eigensolver method and Gram row tile.  The tile depends on the
  // mode's size, which is fixed by the shape whatever the mode order.
  for (int k = 0; k < order; ++k) {
    const int c = p->cls[k];
    const bool jac = c == ATK_CLASS_EIG_JACOBI || c == ATK_CLASS_EIG_JACOBI_SMALL;
    const bool small = c == ATK_CLASS_EIG_SMALL || c == ATK_CLASS_EIG_JACOBI_SMALL;
    p->eigm[k] = jac ? ATK_EIG_FULL_JACOBI : -1;
    const int t = gram_tile(dims[k]);
    p->gbm[k] = small ? std::max(32, t / 2) : 0;
  }
  p->fac_total = off;
  p->total = 1;
  p->core_total = 1;
  for (int k = 0; k < order; ++k) { p->total *= dims[k]; p->core_total *= ranks[k]; }
  p->precision = precision;
  p->als_sweeps = als_sweeps > 0 ? als_sweeps : 5;
  p->seed = seed;
  p->st = (cudaStream_t)stream;
  if (ncand && cand) {
    for (int k = 0; k < order; ++k) {
      p->ncand[k] = ncand[k];
      bool eig = false, als = false;
      for (int j = 0; j < ncand[k]; ++j) {
        p->cand[k][j] = cand[k][j];
        (cand[k][j] == ATK_CLASS_ALS ? als : eig) = true;
      }
      p->both[k] = eig && als;
      if (ncand[k] > 0) p->tune_pending = true;
    }
  }
  int s = plan_alloc(p);
  if (s != ATK_OK) { atucker_plan_destroy(p); return s; }
  *plan = p;
  return ATK_OK;
}

int atucker_plan_create_classes(atucker_plan_t* plan, int order, const int64_t* dims, const int64_t* ranks,
                                const int* mode_order, const int* class_per_mode, int precision, int als_sweeps,
                                uint64_t seed, void* stream) {
  return plan_create_impl(plan, order, dims, ranks, mode_order, class_per_mode, precision, als_sweeps, seed, stream,
                          nullptr, nullptr);
}

int atucker_plan_classes(atucker_plan_t p, int* class_out) {
  if (!p || !class_out) { set_error("plan_classes: null argument"); return ATK_EINVAL; }
  for (int k = 0; k < p->order; ++k) class_out[k] = p->cls[k];
  return ATK_OK;
}

int atucker_plan_mode_timings(atucker_plan_t p, double* out, int count) {
  if (!p || !out || count < p->order) { set_error("mode_timings: need a plan and one slot per mode"); return ATK_EINVAL; }
  ATK_CUDA(cudaStreamSynchronize(p->st));
  for (int i = 0; i < count; ++i) out[i] = 0.0;
  for (const auto& r : p->mrecs) {
    float ms = 0.f;
    ATK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    out[r.phase] += ms;
  }
  p->mrecs.clear();
  if (p->recs.empty()) p->evnext = 0;
  return ATK_OK;
}

int atucker_plan_set_option(atucker_plan_t p, int key, int64_t value) {
  if (!p) { set_error("plan is null"); return ATK_EINVAL; }
  switch (key) {
    case ATK_OPT_EIG_ARITH:
      if (value != ATK_EIG_ROT_FP32 && value != ATK_EIG_ROT_FP64) break;
      p->eig_arith = (int)value;
      return ATK_OK;
    case ATK_OPT_SYNC:
      p->sync = value ? 1 : 0;
      return ATK_OK;
    case ATK_OPT_EIG_METHOD:
      if (value < ATK_EIG_AUTO || value > ATK_EIG_SUBSPACE) break;
      p->eig_method = (int)value;
      return ATK_OK;
    case ATK_OPT_TIMING:
      p->timing = value ? 1 : 0;
      p->recs.clear();
      p->evnext = 0;
      p->gram_launches = p->runs = p->launches = 0;
      return ATK_OK;
    case ATK_OPT_JACOBI_MAX_SWEEPS:
      if (value < 1 || value > 200) break;
      p->max_sweeps = (int)value;
      return ATK_OK;
    case ATK_OPT_GRAM_REFINE:
      if (value < 0 || value > 2) break;
      p->gram_refine = (int)value;
      return ATK_OK;
    case ATK_OPT_WAIT_LIMIT:
      if (value < 0) break;
      p->wait_polls = value;
      return ATK_OK;
    case ATK_OPT_EXPLICIT_UNFOLD:
      if (value != 0 && value != 1) break;
      p->explicit_unfold = (int)value;
      return ATK_OK;
    case ATK_OPT_FUSE_TTM_GRAM:
      if (value != 0 && value != 1) break;
      p->fuse_tg = (int)value;
      return ATK_OK;
    default:
      break;
  }
  set_error("unknown option key or value");
  return ATK_EINVAL;
}

int atucker_plan_sync(atucker_plan_t p) {
  if (!p) { set_error("plan is null"); return ATK_EINVAL; }
  int h = 0;
  ATK_CUDA(cudaMemcpyAsync(&h, p->dev_status, sizeof(int), cudaMemcpyDeviceToHost, p->st));
  ATK_CUDA(cudaStreamSynchronize(p->st));
  ATK_CUDA(cudaMemsetAsync(p->dev_status, 0, sizeof(int), p->st));
  if (h & DEV_TIMEOUT) { set_error("device-side bounded wait timed out"); return ATK_ETIMEOUT; }
  if (h & DEV_CHOL) { set_error("ALS: Cholesky pivot not positive (rank-deficient L or R)"); return ATK_ERANK; }
  if (h & DEV_NOCONV) { set_error("Jacobi eigensolver reached its sweep cap"); return ATK_ENOCONV; }
  return ATK_OK;
}

// Buffers of the explicit-matricization form, at its first run: the largest
// unfolding of a mode with lo > 1 and the largest R x J TTM result.
static int explicit_buffers(atucker_plan_t p) {
  if (p->xunf) return ATK_OK;
  int64_t cur[8];
  for (int k = 0; k < p->order; ++k) cur[k] = p->dims[k];
  size_t unf = 1, ttm = 1;
  for (int step = 0; step < p->order; ++step) {
    const int n = p->mode_order[step];
    const View v = make_view(p->order, cur, n);
    if (v.lo > 1) {
      unf = std::max(unf, (size_t)v.size());
      ttm = std::max(ttm, (size_t)(v.J() * p->ranks[n]));
    }
    cur[n] = p->ranks[n];
  }
  char* base = nullptr;
  const size_t need = 4 * (unf + ttm) + 512;
  ATK_TRY(dev_alloc((void**)&base, need, "cudaMalloc(explicit unfolding)"));
  Arena ar{base, need, 0};
  p->xunf = (float*)ar.take(4 * unf);
  p->xttm = (float*)ar.take(4 * ttm);
  return ATK_OK;
}

static int sthosvd_run(atucker_plan_t p, const float* x, float* core_out, float* factors_out, double* discarded_out) {
  cudaStream_t st = p->st;
  if (p->explicit_unfold) ATK_TRY(explicit_buffers(p));
  int64_t cur[8];
  for (int k = 0; k < p->order; ++k) cur[k] = p->dims[k];
  const float* Y = x;
  const bool need_norms = discarded_out != nullptr;
  const bool tm = p->timing != 0;
  cudaEvent_t e_first = nullptr, e_prev = nullptr;
  // mark(phase): close the running phase at a new event (timing mode only).
  auto mark = [&](int phase) -> int {
    if (!tm) return ATK_OK;
    cudaEvent_t e = p->ev();
    ATK_CUDA(cudaEventRecord(e, st));
    if (phase >= 0) p->recs.push_back({phase, e_prev, e});
    e_prev = e;
    return ATK_OK;
  };
  if (tm) {
    ATK_TRY(mark(-1));
    e_first = e_prev;
    p->runs++;
  }
  bool s_ready = false;  // p->S already holds this mode's Gram (fused into the last TTM)
  for (int step = 0; step < p->order; ++step) {
    const int n = p->mode_order[step];
    const View vn = make_view(p->order, cur, n);
    cudaEvent_t e_mode = e_prev;
    const int64_t R = p->ranks[n];
    float* const out_final = (step == p->order - 1) ? core_out : p->buf[step & 1];
    // Explicit form: the mode-n unfolding is materialised and the mode's
    // contractions run on its mode-1 view; their (R, J) result is folded
    // into out_final after the mode.
    const bool unfold = p->explicit_unfold && vn.lo > 1;
    if (unfold) ATK_TRY(permute_slabs(Y, vn.lo, vn.n, vn.hi, p->xunf, st));
    const View v = unfold ? View{1, vn.n, vn.J()} : vn;
    if (unfold) Y = p->xunf;
    float* out = unfold ? p->xttm : out_final;
    float* U32 = factors_out + p->foff[n];
    double* disc = discarded_out ? discarded_out + n : nullptr;
    if (p->solver[n] == ATK_EIG) {
      // S = Y_(n) Y_(n)^T; U = leading eigenvectors; Y' = Y x_n U^T.
      cudaEvent_t mid = tm ? p->ev() : nullptr;
      if (s_ready) {
        // formed by the previous mode's TTM
      } else if (p->precision == ATK_FP32) {
        ATK_TRY(gram_f32(Y, v, p->S, (float*)p->scratch, p->scratch_bytes, st, mid, p->gbm[n]));
      } else if (p->precision == ATK_FP32C) {
        ATK_TRY(gram_cmp(Y, v, p->S, (float*)p->scratch, p->scratch_bytes, st));
        if (mid) ATK_CUDA(cudaEventRecord(mid, st));
      } else {
        ATK_TRY(tc_gram(Y, v, p->precision, p->S, (float*)p->scratch, p->scratch_bytes, p->dev_status, st));
        if (mid) ATK_CUDA(cudaEventRecord(mid, st));
      }
      if (tm && !s_ready) {
        p->recs.push_back({PH_GRAM, e_prev, mid});
        e_prev = mid;
        p->gram_launches++;
        ATK_TRY(mark(PH_GRAM_REDUCE));
      }
      s_ready = false;
      const int em = p->eigm[n] >= 0 ? p->eigm[n] : p->eig_method;
      // A cut that the float32 Gram cannot resolve (ATK_OPT_GRAM_REFINE):
      // recompute this mode's Gram with compensated sums and solve again.
      const bool refine = p->precision != ATK_FP32C && p->eig_arith == ATK_EIG_ROT_FP32 &&
                          (p->gram_refine == 2 || (p->gram_refine == 1 && step > 0));
      int unresolved = 0;
      ATK_TRY(eig_top(p->S, v.n, R, p->eig_arith, em, p->max_sweeps, U32, p->U64, nullptr, disc,
                      p->dev_status, p->scratch, p->scratch_bytes, st, refine ? &unresolved : nullptr));
      if (unresolved) {
        ATK_TRY(gram_cmp(Y, v, p->S, (float*)p->scratch, p->scratch_bytes, st));
        ATK_TRY(eig_top(p->S, v.n, R, p->eig_arith, em, p->max_sweeps, U32, p->U64, nullptr, disc,
                        p->dev_status, p->scratch, p->scratch_bytes, st));
      }
      ATK_TRY(mark(PH_EIG));
      // Tensor cores where the TTM is a dense contraction: with R <= 16 the
      // float32 kernel is already bound by HBM (and exact in float32).
      // Fused with the next mode's Gram where that mode is an EIG mode the
      // fused kernel covers (ATK_OPT_FUSE_TTM_GRAM).
      int64_t fs = 0, fim = 0;
      const int m = step + 1 < p->order ? p->mode_order[step + 1] : -1;
      if (p->fuse_tg && !unfold && !p->explicit_unfold && m >= 0 && p->solver[m] == ATK_EIG &&
          fuse_geometry(p, step, cur, v, R, &fs, &fim)) {
        ATK_TRY(ttm_gram(Y, v, U32, R, fs, fim, out, p->S, p->scratch, p->scratch_bytes, st));
        s_ready = true;
      } else if (p->precision == ATK_FP32 || p->precision == ATK_FP32C || R <= TC_TTM_MIN_R)
        ATK_TRY(ttm_f32(Y, v, U32, R, out, st));
      else
        ATK_TRY(tc_ttm(Y, v, U32, R, p->precision, out, p->scratch, p->scratch_bytes, p->dev_status, st));
      ATK_TRY(mark(PH_TTM));
    } else {
      ATK_TRY(als_mode_run(Y, v, R, p->L0 + p->l0off[n], p->als_sweeps, U32, out, p->als, st));
      ATK_TRY(mark(PH_ALS));
      if (need_norms) {
        ATK_TRY(norm2_f32(Y, v.size(), p->norms, (double*)p->scratch, st));
        ATK_TRY(norm2_f32(out, v.J() * R, p->norms + 1, (double*)p->scratch, st));
        sub_kernel<<<1, 1, 0, st>>>(p->norms, p->norms + 1, disc);
        ATK_LAUNCHED();
        ATK_TRY(mark(PH_OTHER));
      }
    }
    if (unfold) ATK_TRY(permute_slabs(p->xttm, R, vn.lo, vn.hi, out_final, st));
    if (tm) p->mrecs.push_back({n, e_mode, e_prev});
    cur[n] = R;
    Y = out_final;
  }
  if (tm) p->recs.push_back({PH_TOTAL, e_first, e_prev});
  if (p->order == 0) return ATK_OK;
  if (p->sync) return atucker_plan_sync(p);
  return ATK_OK;
}

// ------------------------------------------- exhaustive timed search (AUTO)
// The classes chosen by timing, per shape and settings, for the process.
static std::mutex g_tuned_mu;
static std::map<std::vector<int64_t>, std::vector<int>> g_tuned;

static std::vector<int64_t> tune_key(const atucker_plan_s* p) {
  std::vector<int64_t> k{p->order, p->precision, p->eig_arith, p->eig_method, p->als_sweeps, p->gram_refine};
  for (int i = 0; i < p->order; ++i) {
    k.push_back(p->dims[i]);
    k.push_back(p->ranks[i]);
    k.push_back(p->mode_order[i]);
    k.push_back(p->ncand[i]);
  }
  return k;
}

static void set_mode_class(atucker_plan_s* p, int k, int c) {
  p->cls[k] = c;
  p->solver[k] = c == ATK_CLASS_ALS ? ATK_ALS : ATK_EIG;
  const bool jac = c == ATK_CLASS_EIG_JACOBI || c == ATK_CLASS_EIG_JACOBI_SMALL;
  const bool small = c == ATK_CLASS_EIG_SMALL || c == ATK_CLASS_EIG_JACOBI_SMALL;
  p->eigm[k] = jac ? ATK_EIG_FULL_JACOBI : -1;
  p->gbm[k] = small ? std::max(32, gram_tile(p->dims[k]) / 2) : 0;
}

// Time every candidate class of the AUTO modes on this input (round t runs
// every such mode with its t-th candidate; one warm-up and one timed run, the
// per-mode CUDA-event times), keep each mode's fastest, and cache the choice.
static int tune_plan(atucker_plan_s* p, const float* x, float* core_out, float* factors_out) {
  const std::vector<int64_t> key = tune_key(p);
  {
    std::lock_guard<std::mutex> g(g_tuned_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      for (int k = 0; k < p->order; ++k)
        if (p->ncand[k] > 0) set_mode_class(p, k, it->second[k]);
      p->tune_pending = false;
      return ATK_OK;
    }
  }
  int rounds = 0;
  for (int k = 0; k < p->order; ++k) rounds = std::max(rounds, p->ncand[k]);
  double best_ms[8];
  int best[8];
  for (int k = 0; k < p->order; ++k) {
    best_ms[k] = 1e300;
    best[k] = p->cls[k];
  }
  const int timing = p->timing, sync = p->sync;
  p->timing = 1;
  p->sync = 0;
  for (int t = 0; t < rounds; ++t) {
    for (int k = 0; k < p->order; ++k)
      if (p->ncand[k] > 0) set_mode_class(p, k, p->cand[k][std::min(t, p->ncand[k] - 1)]);
    double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      p->recs.clear();
      p->mrecs.clear();
      p->evnext = 0;
      ok = sthosvd_run(p, x, core_out, factors_out, nullptr) == ATK_OK && atucker_plan_sync(p) == ATK_OK;
      if (ok && rep == 1) ok = atucker_plan_mode_timings(p, ms, p->order) == ATK_OK;
    }
    if (!ok) continue;  // a class that fails on this input is not chosen
    for (int k = 0; k < p->order; ++k)
      if (p->ncand[k] > t && ms[k] < best_ms[k]) {
        best_ms[k] = ms[k];
        best[k] = p->cand[k][t];
      }
  }
  for (int k = 0; k < p->order; ++k) set_mode_class(p, k, best[k]);
  p->timing = timing;
  p->sync = sync;
  p->recs.clear();
  p->mrecs.clear();
  p->evnext = 0;
  p->tune_pending = false;
  std::lock_guard<std::mutex> g(g_tuned_mu);
  g_tuned[key] = std::vector<int>(best, best + p->order);
  return ATK_OK;
}

int atucker_sthosvd(atucker_plan_t p, const float* x, float* core_out, float* factors_out, double* discarded_out) {
  if (!p || !x || !core_out || !factors_out) { set_error("null argument"); return ATK_EINVAL; }
  const long long l0 = launch_count();
  set_wait_limit(p->wait_polls);
  if (p->tune_pending) {
    const int s = tune_plan(p, x, core_out, factors_out);
    if (s != ATK_OK) {
      set_wait_limit(0);
      return s;
    }
  }
  const int s = sthosvd_run(p, x, core_out, factors_out, discarded_out);
  set_wait_limit(0);
  p->launches += launch_count() - l0;
  return s;
}

int atucker_sthosvd_host(atucker_plan_t p, const float* x_host, float* core_host, float* factors_host,
                         double* discarded_host) {
  if (!p || !x_host || !core_host || !factors_host) { set_error("null argument"); return ATK_EINVAL; }
  if (!p->x_dev) {
    size_t need = (size_t)p->total * 4 + (size_t)p->core_total * 4 + (size_t)p->fac_total * 4 + 8 * 8 + 1024;
    char* base = nullptr;
    ATK_TRY(dev_alloc((void**)&base, need, "cudaMalloc(host-buffer staging)"));
    Arena ar{base, need, 0};
    p->x_dev = (float*)ar.take((size_t)p->total * 4);
    p->core_dev = (float*)ar.take((size_t)p->core_total * 4);
    p->fac_dev = (float*)ar.take((size_t)p->fac_total * 4);
    p->disc_dev = (double*)ar.take(8 * 8);
  }
  ATK_CUDA(cudaMemcpyAsync(p->x_dev, x_host, (size_t)p->total * 4, cudaMemcpyHostToDevice, p->st));
  int s = atucker_sthosvd(p, p->x_dev, p->core_dev, p->fac_dev, discarded_host ? p->disc_dev : nullptr);
  if (s != ATK_OK) return s;
  ATK_CUDA(cudaMemcpyAsync(core_host, p->core_dev, (size_t)p->core_total * 4, cudaMemcpyDeviceToHost, p->st));
  ATK_CUDA(cudaMemcpyAsync(factors_host, p->fac_dev, (size_t)p->fac_total * 4, cudaMemcpyDeviceToHost, p->st));
  if (discarded_host)
    ATK_CUDA(cudaMemcpyAsync(discarded_host, p->disc_dev, (size_t)p->order * 8, cudaMemcpyDeviceToHost, p->st));
  return atucker_plan_sync(p);
}

int atucker_plan_timings(atucker_plan_t p, double* out, int count) {
  if (!p || !out || count < PH_SLOTS) { set_error("timings: need a plan and >= 10 output slots"); return ATK_EINVAL; }
  ATK_CUDA(cudaStreamSynchronize(p->st));
  for (int i = 0; i < count; ++i) out[i] = 0.0;
  for (const auto& r : p->recs) {
    float ms = 0.f;
    ATK_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    out[r.phase] += ms;
  }
  out[PH_TOTAL + 1] = (double)p->gram_launches;
  out[PH_TOTAL + 2] = (double)p->launches;
  out[PH_TOTAL + 3] = (double)p->runs;
  p->recs.clear();
  p->mrecs.clear();  // per-mode records are read first (atucker_plan_mode_timings) or dropped here
  p->evnext = 0;
  p->gram_launches = p->runs = p->launches = 0;
  return ATK_OK;
}

void atucker_plan_destroy(atucker_plan_t p) {
  if (!p) return;
  if (p->st) cudaStreamSynchronize(p->st);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : p->evpool) cudaEventDestroy(e);
  if (p->ws) cudaFree(p->ws);
  if (p->x_dev) cudaFree(p->x_dev);
  if (p->xunf) cudaFree(p->xunf);
  delete p;
}

int atucker_sthosvd_oneshot(const float* x, int order, const int64_t* dims, const int64_t* ranks, const int* mode_order,
                            const int* solver_per_mode, float* core_out, float* factors_out) {
  atucker_plan_t p = nullptr;
  ATK_TRY(atucker_plan_create(&p, order, dims, ranks, mode_order, solver_per_mode, ATK_FP32, 5, 0, nullptr));
  p->sync = 1;
  int s = atucker_sthosvd(p, x, core_out, factors_out, nullptr);
  atucker_plan_destroy(p);
  return s;
}

int atucker_set_device_alloc_limit(uint64_t bytes) {
  g_alloc_limit.store(bytes);
  return ATK_OK;
}

const char* atucker_last_error(void) { return g_err.c_str(); }
const char* atucker_version(void) { return "0.1.0"; }

// ------------------------------------------------------ step-level entry points
struct StreamScratch {
  void* ptr = nullptr;
  cudaStream_t st;
  explicit StreamScratch(cudaStream_t s) : st(s) {}
  int alloc(size_t bytes) { return dev_alloc_async(&ptr, bytes, st, "cudaMallocAsync(scratch)"); }
  ~StreamScratch() {
    if (ptr) cudaFreeAsync(ptr, st);
  }
};

static int check_view(int64_t lo, int64_t n, int64_t hi) {
  if (lo < 1 || n < 1 || hi < 1) { set_error("view extents must be >= 1"); return ATK_EINVAL; }
  if ((double)lo * (double)n * (double)hi >= 2147483648.0) { set_error("tensor must have fewer than 2^31 elements"); return ATK_EUNSUPPORTED; }
  return ATK_OK;
}

static int read_status(int* dev, cudaStream_t st) {
  int h = 0;
  ATK_CUDA(cudaMemcpyAsync(&h, dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  ATK_CUDA(cudaStreamSynchronize(st));
  if (h & DEV_TIMEOUT) { set_error("device-side bounded wait timed out"); return ATK_ETIMEOUT; }
  if (h & DEV_CHOL) { set_error("Cholesky pivot not positive"); return ATK_ERANK; }
  if (h & DEV_NOCONV) { set_error("Jacobi eigensolver reached its sweep cap"); return ATK_ENOCONV; }
  return ATK_OK;
}

int atucker_gram(const float* y, int64_t lo, int64_t n, int64_t hi, int precision, double* S_out, void* stream) {
  if (!y || !S_out) { set_error("null argument"); return ATK_EINVAL; }
  ATK_TRY(check_view(lo, n, hi));
  if (precision < ATK_FP32 || precision > ATK_FP32C) { set_error("unsupported precision"); return ATK_EUNSUPPORTED; }
  if (n > 4096) { set_error("Gram needs n <= 4096"); return ATK_EUNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  View v{lo, n, hi};
  StreamScratch sc(st);
  if (precision == ATK_FP32C) {
    const size_t bytes = gram_cmp_scratch_bytes(v);
    ATK_TRY(sc.alloc(bytes));
    ATK_TRY(gram_cmp(y, v, S_out, (float*)sc.ptr, bytes, st));
    ATK_CUDA(cudaStreamSynchronize(st));
    return ATK_OK;
  }
  if (precision == ATK_FP32) {
    size_t bytes = gram_scratch_bytes(v);
    ATK_TRY(sc.alloc(bytes));
    ATK_TRY(gram_f32(y, v, S_out, (float*)sc.ptr, bytes, st));
    ATK_CUDA(cudaStreamSynchronize(st));
    return ATK_OK;
  }
  size_t bytes = tc_gram_scratch_bytes(v, precision) + 256;
  ATK_TRY(sc.alloc(bytes));
  int* status = (int*)((char*)sc.ptr + bytes - 256);
  ATK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  ATK_TRY(tc_gram(y, v, precision, S_out, (float*)sc.ptr, bytes - 256, status, st));
  return read_status(status, st);
}

int atucker_ttm(const float* y, int64_t lo, int64_t n, int64_t hi, const float* U, int64_t R, int precision,
                float* out, void* stream) {
  if (!y || !U || !out) { set_error("null argument"); return ATK_EINVAL; }
  ATK_TRY(check_view(lo, n, hi));
  if (R < 1 || R > 1024) { set_error("TTM needs 1 <= R <= 1024"); return ATK_EUNSUPPORTED; }
  if (precision < ATK_FP32 || precision > ATK_FP32C) { set_error("unsupported precision"); return ATK_EUNSUPPORTED; }
  View v{lo, n, hi};
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == ATK_FP32 || precision == ATK_FP32C) return ttm_f32(y, v, U, R, out, st);
  if (R > 128) { set_error("tensor-core TTM needs R <= 128"); return ATK_EUNSUPPORTED; }
  StreamScratch sc(st);
  const size_t bytes = tc_ttm_scratch_bytes(v, R, precision) + 256;
  ATK_TRY(sc.alloc(bytes));
  int* status = (int*)((char*)sc.ptr + bytes - 256);
  ATK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  ATK_TRY(tc_ttm(y, v, U, R, precision, out, (char*)sc.ptr, bytes - 256, status, st));
  return read_status(status, st);
}

int atucker_ttm_gram(const float* y, int64_t lo, int64_t n, int64_t hi, const float* U, int64_t R, int64_t s,
                     int64_t m_size, float* out, double* S_out, void* stream) {
  if (!y || !U || !out || !S_out) { set_error("null argument"); return ATK_EINVAL; }
  ATK_TRY(check_view(lo, n, hi));
  View v{lo, n, hi};
  if (!ttm_gram_ok(v, R, s, m_size)) {
    set_error("ttm_gram needs 1 <= R <= 64, 16 <= I_m <= 128 and s I_m dividing lo hi");
    return ATK_EUNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  StreamScratch sc(st);
  const size_t bytes = ttm_gram_scratch_bytes(v, R, s, m_size);
  ATK_TRY(sc.alloc(bytes));
  ATK_TRY(ttm_gram(y, v, U, R, s, m_size, out, S_out, sc.ptr, bytes, st));
  ATK_CUDA(cudaStreamSynchronize(st));
  return ATK_OK;
}

int atucker_eig(const double* S, int64_t n, int64_t R, int eig_arith, int eig_method, float* U_out,
                double* lambda_out, double* discarded_out, void* stream) {
  if (!S || !U_out) { set_error("null argument"); return ATK_EINVAL; }
  if (n < 1 || R < 1 || R > n || n > EIG_MAX_N || R > 128) {
    set_error("need 1 <= R <= n <= 32768 and R <= 128");
    return ATK_EUNSUPPORTED;
  }
  if (eig_arith != ATK_EIG_ROT_FP32 && eig_arith != ATK_EIG_ROT_FP64) { set_error("bad eig_arith"); return ATK_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  StreamScratch sc(st);
  size_t sb = std::max(eig_scratch_bytes(n, eig_arith), (size_t)n * R * 8 + smallla_scratch_bytes(n, R) + 1024);
  size_t bytes = sb + (size_t)n * R * 8 + 1024;
  ATK_TRY(sc.alloc(bytes));
  Arena ar{(char*)sc.ptr, bytes, 0};
  int* status = (int*)ar.take(256);
  double* U64 = (double*)ar.take((size_t)n * R * 8);
  char* scratch = (char*)ar.take(sb);
  ATK_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  if (eig_method < ATK_EIG_AUTO || eig_method > ATK_EIG_SUBSPACE) { set_error("bad eig_method"); return ATK_EINVAL; }
  ATK_TRY(eig_top(S, n, R, eig_arith, eig_method, 40, U_out, U64, lambda_out, discarded_out, status, scratch, sb,
                  st));
  return read_status(status, st);
}

int atucker_als_mode(const float* y, int64_t lo, int64_t n, int64_t hi, int64_t R, const double* L0, uint64_t seed,
                     int mode, int sweeps, int precision, float* U_out, float* core_out, void* stream) {
  if (!y || !U_out || !core_out) { set_error("null argument"); return ATK_EINVAL; }
  ATK_TRY(check_view(lo, n, hi));
  if (R < 1 || R > n || R > 128 || R > lo * hi) { set_error("ALS needs 1 <= R <= min(n, J, 128)"); return ATK_ERANK; }
  if (precision != ATK_FP32) { set_error("unsupported precision"); return ATK_EUNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  View v{lo, n, hi};
  size_t sb = als_scratch_need(v, R);
  size_t nr = (size_t)(n * R), rr = (size_t)(R * R);
  size_t bytes = sb + (nr * 8) * 4 + rr * 8 * 3 + nr * 4 + rr * 4 + (size_t)v.J() * R * 4 + 16 * 256;
  StreamScratch sc(st);
  ATK_TRY(sc.alloc(bytes));
  Arena ar{(char*)sc.ptr, bytes, 0};
  AlsBufs b{};
  b.dev_status = (int*)ar.take(256);
  b.L = (double*)ar.take(nr * 8);
  b.Lt = (double*)ar.take(nr * 8);
  b.A = (double*)ar.take(nr * 8);
  double* l0d = (double*)ar.take(nr * 8);
  b.G = (double*)ar.take(rr * 8);
  b.B = (double*)ar.take(rr * 8);
  b.Rhat = (double*)ar.take(rr * 8);
  b.Lt32 = (float*)ar.take(nr * 4);
  b.M32 = (float*)ar.take(rr * 4);
  b.P = (float*)ar.take((size_t)v.J() * R * 4);
  b.scratch = (char*)ar.take(sb);
  b.scratch_bytes = sb;
  if (!b.scratch) { set_error("als: scratch carve failed"); return ATK_EINVAL; }
  ATK_CUDA(cudaMemsetAsync(b.dev_status, 0, sizeof(int), st));
  if (L0) {
    ATK_CUDA(cudaMemcpyAsync(l0d, L0, nr * 8, cudaMemcpyDeviceToDevice, st));
  } else {
    std::vector<double> h(nr);
    als_initial_guess(seed, mode, n, R, h.data());
    ATK_CUDA(cudaMemcpyAsync(l0d, h.data(), nr * 8, cudaMemcpyHostToDevice, st));
    ATK_CUDA(cudaStreamSynchronize(st));
  }
  ATK_TRY(als_mode_run(y, v, R, l0d, sweeps > 0 ? sweeps : 5, U_out, core_out, b, st));
  return read_status(b.dev_status, st);
}

}  // extern "C"
