// Batched st-HOSVD of many small order-3 tensors in one persistent launch
// (Alg. 2 applied to each tensor, EIG every mode, mode order 1, 2, 3).
//
// Each CTA takes whole tensors from an atomic work counter, largest first
// (tensors are queued by decreasing work, so the tail of the launch holds the
// small ones).  A tensor never leaves its CTA:
//   for each mode n:  S = Y_(n) Y_(n)^T over the stride view (a2), staged
//                     through shared memory, split over c among thread groups;
//                     one-sided (Hestenes) Jacobi on S in shared memory
//                     (a3, float32 rotations): S's columns rotate into
//                     lambda_i u_i, so no eigenvector matrix is carried;
//                     U = the R_n leading eigenvectors, one polar step,
//                     sign rule, written out;
//                     Y <- Y x_n U^T (a4) into this CTA's workspace (L2), or
//                     into the core after the last mode.
// Sizes: every mode <= 96, every rank <= 32.  Shared memory (54 KB, so up to
// four tensors per SM) holds the Gram matrix A (96 x 97 floats), a 16 KB
// staging area for the Gram and TTM tiles, and the eigenvalues; the kept
// factor reuses A's space.
//
// The launch shape (threads per CTA, CTAs per SM, c values per staged chunk)
// is a template/launch choice picked by an autotuner that times every
// variant on the batch itself.  The launch (pointer-table upload, counter
// reset, kernel) is captured once in a CUDA graph and replayed.
#include <algorithm>
#include <mutex>
#include <vector>

#include "jacobi_dev.cuh"

namespace atk {
namespace batch {

constexpr int DMAX = 96;
constexpr int RMAX = 32;
constexpr int LDA = DMAX + 1;                 // pitch of A
constexpr int MAT = DMAX * LDA;               // floats of A
constexpr int STG = 4096;                     // floats of the staging area

struct Desc {
  int d[3], r[3];
};
struct Ptrs {
  const float* x;
  float* core;
  float* factors;
};

// Shared-memory layout (floats): A | stage | lam | ord (int).
constexpr size_t SMEM_FLOATS = (size_t)MAT + STG + 2 * DMAX;
constexpr size_t SMEM_BYTES = SMEM_FLOATS * sizeof(float);

// ------------------------------------------------------------------ Gram
// S (shared, pitch lds, n x n) = sum over c of Y[:, c] Y[:, c]^T for the view
// (lo, n, hi).  Threads form G groups of np positions; position (bi, bj),
// bi <= bj, owns rows bi + p u and columns bj + p v (u, v < TM), which covers
// every unordered pair {i, j} once.  Group g takes the c values g KC .. g KC +
// KC - 1 of each staged chunk of KC G values; the groups' partial tiles are
// then added into S in group order.
template <int NT, int KC, int TM>
__device__ void gram_tm(const float* y, int lo, int n, int64_t J, float* S, int lds, float* stage, int G) {
  const int p = (n + TM - 1) / TM, np = p * (p + 1) / 2;
  const int lt = (p * TM) | 1;  // stage pitch (odd), covers rows up to p TM
  const int t = threadIdx.x;
  const int g = t / np;
  int pos = t % np, bi = 0;
  while (pos >= p - bi) { pos -= p - bi; ++bi; }
  const int bj = bi + pos;
  const bool active = g < G;
  float acc[TM][TM];
#pragma unroll
  for (int u = 0; u < TM; ++u)
#pragma unroll
    for (int v = 0; v < TM; ++v) acc[u][v] = 0.f;
  const int ck = KC * G;
  for (int64_t c0 = 0; c0 < J; c0 += ck) {
    __syncthreads();
    const int cnt = ck * n;
    if (lo == 1) {
      for (int idx = t; idx < cnt; idx += NT) {
        const int cl = idx / n, i = idx % n;
        const int64_t c = c0 + cl;
        stage[cl * lt + i] = c < J ? y[i + (int64_t)n * c] : 0.f;
      }
    } else {
      for (int idx = t; idx < cnt; idx += NT) {
        const int cl = idx % ck, i = idx / ck;
        const int64_t c = c0 + cl;
        float v = 0.f;
        if (c < J) v = y[(c % lo) + (int64_t)lo * (i + (int64_t)n * (c / lo))];
        stage[cl * lt + i] = v;
      }
    }
    __syncthreads();
    if (active) {
      const float* tk = stage + (g * KC) * lt;
#pragma unroll 4
      for (int k = 0; k < KC; ++k, tk += lt) {
        float a[TM], b[TM];
#pragma unroll
        for (int u = 0; u < TM; ++u) a[u] = tk[bi + p * u];
#pragma unroll
        for (int v = 0; v < TM; ++v) b[v] = tk[bj + p * v];
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
          for (int v = 0; v < TM; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
      }
    }
  }
  // Reduce the groups in order: group 0 writes, the others add.
  for (int gg = 0; gg < G; ++gg) {
    __syncthreads();
    if (active && g == gg) {
#pragma unroll
      for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int v = 0; v < TM; ++v) {
          const int i = bi + p * u, j = bj + p * v;
          // a diagonal block holds both (i, j) and (j, i): take i <= j only
          if (i < n && j < n && (bi != bj || i <= j)) {
            const float s = gg == 0 ? acc[u][v] : S[i * lds + j] + acc[u][v];
            S[i * lds + j] = s;
            if (i != j) S[j * lds + i] = s;
          }
        }
    }
  }
  __syncthreads();
}

// Register tile TM for n: the largest count of active threads (ties: larger
// TM), with the groups capped so that a staged chunk fits in `cap` floats.
template <int NT, int KC>
__device__ __host__ inline void gram_shape(int n, int cap, int& tm_out, int& g_out) {
  const int tms[4] = {8, 6, 4, 2};
  int best = -1;
  tm_out = 2;
  g_out = 1;
  for (int q = 0; q < 4; ++q) {
    const int tm = tms[q];
    const int p = (n + tm - 1) / tm, np = p * (p + 1) / 2;
    if (np > NT) continue;
    const int lt = (p * tm) | 1;
    int G = NT / np;
    G = std::min(G, std::max(1, cap / (KC * lt)));
    const int act = G * np;
    if (act > best) {
      best = act;
      tm_out = tm;
      g_out = G;
    }
  }
}

template <int NT, int KC>
__device__ void cta_gram(const float* y, int lo, int n, int64_t J, float* S, int lds, float* stage) {
  int tm, G;
  gram_shape<NT, KC>(n, STG, tm, G);
  switch (tm) {
    case 8: gram_tm<NT, KC, 8>(y, lo, n, J, S, lds, stage, G); break;
    case 6: gram_tm<NT, KC, 6>(y, lo, n, J, S, lds, stage, G); break;
    case 4: gram_tm<NT, KC, 4>(y, lo, n, J, S, lds, stage, G); break;
    default: gram_tm<NT, KC, 2>(y, lo, n, J, S, lds, stage, G); break;
  }
}

// ------------------------------------------------------------------- TTM
// out[a + lo (r + R b)] = sum_i U[i][r] Y[a + lo (i + n b)] (Alg. 2, TTM with
// U^T).  Us is row-major n x r4 (r4 = R rounded up to 4, zero padded).  A
// chunk of c values is staged; each work item is one c and four r.
template <int NT>
__device__ void cta_ttm(const float* y, int lo, int n, int64_t hi, const float* Us, int R, int r4, float* out,
                        float* stage) {
  const int64_t J = (int64_t)lo * hi;
  const int lt = n | 1;
  const int ct = std::min(256, STG / lt);
  const int rg = r4 / 4;
  const int t = threadIdx.x;
  for (int64_t c0 = 0; c0 < J; c0 += ct) {
    __syncthreads();
    const int cn = (int)std::min<int64_t>(ct, J - c0);
    if (lo == 1) {
      for (int idx = t; idx < cn * n; idx += NT) {
        const int cl = idx / n, i = idx % n;
        stage[cl * lt + i] = y[i + (int64_t)n * (c0 + cl)];
      }
    } else {
      for (int idx = t; idx < cn * n; idx += NT) {
        const int cl = idx % cn, i = idx / cn;
        const int64_t c = c0 + cl;
        stage[cl * lt + i] = y[(c % lo) + (int64_t)lo * (i + (int64_t)n * (c / lo))];
      }
    }
    __syncthreads();
    for (int w = t; w < cn * rg; w += NT) {
      int cl, q;
      if (lo == 1) {  // r fastest: a thread's outputs are contiguous
        q = w % rg;
        cl = w / rg;
      } else {  // c fastest: consecutive a are contiguous
        cl = w % cn;
        q = w / cn;
      }
      const float* tc = stage + cl * lt;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      for (int i = 0; i < n; ++i) {
        const float yv = tc[i];
        const float4 u = *reinterpret_cast<const float4*>(Us + i * r4 + 4 * q);
        s0 = fmaf(u.x, yv, s0);
        s1 = fmaf(u.y, yv, s1);
        s2 = fmaf(u.z, yv, s2);
        s3 = fmaf(u.w, yv, s3);
      }
      const int64_t c = c0 + cl;
      const int64_t a = c % lo, b = c / lo;
      float* o = out + a + (int64_t)lo * ((int64_t)R * b);
      const int r0 = 4 * q;
      if (r0 < R) o[(int64_t)lo * r0] = s0;
      if (r0 + 1 < R) o[(int64_t)lo * (r0 + 1)] = s1;
      if (r0 + 2 < R) o[(int64_t)lo * (r0 + 2)] = s2;
      if (r0 + 3 < R) o[(int64_t)lo * (r0 + 3)] = s3;
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------- kernel
template <int NT, int KC, int MINB>
__global__ void __launch_bounds__(NT, MINB) batched_kernel(const Desc* __restrict__ desc, const int* __restrict__ queue,
                                                           const Ptrs* __restrict__ ptrs, int count,
                                                           int* __restrict__ counter, float* __restrict__ ws,
                                                           int64_t ws_per_cta, int max_sweeps,
                                                           int* __restrict__ status) {
  extern __shared__ __align__(16) float smem[];
  float* A = smem;
  float* stage = A + MAT;
  float* lam = stage + STG;
  int* ord = reinterpret_cast<int*>(lam + DMAX);
  __shared__ int cur;
  __shared__ double red[32];
  const int t = threadIdx.x, lane = t % 32, warp = t / 32;
  float* myws = ws + (int64_t)blockIdx.x * ws_per_cta;
  for (;;) {
    if (t == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int slot = cur;
    __syncthreads();
    if (slot >= count) break;
    const int ti = queue[slot];
    const Desc dsc = desc[ti];
    const Ptrs pt = ptrs[ti];
    const float* src = pt.x;
    float* fac = pt.factors;
    int64_t lo = 1, hi = (int64_t)dsc.d[1] * dsc.d[2];
    float* bufs[2] = {myws, myws + (int64_t)dsc.r[0] * dsc.d[1] * dsc.d[2]};
    for (int k = 0; k < 3; ++k) {
      const int n = dsc.d[k], R = dsc.r[k];
      const int m = n + (n & 1), ld = m + 1;
      const int r4 = (R + 3) & ~3;
      // 1. Gram into A (pitch ld); padding row/column of an odd n is zero.
      cta_gram<NT, KC>(src, (int)lo, n, lo * hi, A, ld, stage);
      if (m != n) {
        for (int i = t; i < m; i += NT) {
          A[(m - 1) * ld + i] = 0.f;
          A[i * ld + (m - 1)] = 0.f;
        }
        __syncthreads();
      }
      // 2. One-sided Jacobi on S (PSD): its normalised columns become the
      //    eigenvectors, lam the eigenvalues.  ||S||_F for the absolute floor.
      double fl = 0.0;
      for (int idx = t; idx < m * m; idx += NT) {
        const double a = A[(idx / m) * ld + idx % m];
        fl += a * a;
      }
      for (int o = 16; o > 0; o >>= 1) fl += __shfl_xor_sync(0xffffffffu, fl, o);
      if (lane == 0) red[warp] = fl;
      __syncthreads();
      if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += red[w];
        red[0] = s;
      }
      __syncthreads();
      const float fro = (float)sqrt(red[0]);
      bool conv = true;
      if (m >= 2) hestenes_smem<8, DMAX / 8>(A, ld, m, fro, max_sweeps, lam, &conv);
      if (!conv && t == 0) atomicOr(status, DEV_NOCONV);
      // 3. Order by eigenvalue (descending; NaN lowest; ties by index).
      for (int i = t; i < n; i += NT) {
        const float di = lam[i];
        const float ki = isnan(di) ? -INFINITY : di;
        int rank = 0;
        for (int j = 0; j < n; ++j) {
          const float dj = lam[j];
          const float kj = isnan(dj) ? -INFINITY : dj;
          rank += (kj > ki) || (kj == ki && j < i);
        }
        ord[rank] = i;
      }
      __syncthreads();
      // 4. U = the kept eigenvectors (row-major n x r4, zero padded), one
      //    Newton-Schulz polar step U <- U (3 I - U^T U) / 2 to undo the
      //    rounding the float32 rotations left in its orthonormality, then
      //    the sign rule: each column's largest-magnitude entry positive
      //    (ties: lowest row).  Gathered copy and U^T U in the staging area,
      //    the result in A's space.
      float* Ug = stage;                   // n x r4
      float* M = stage + DMAX * RMAX;      // U^T U, r4 x r4
      float* Us = A;                       // polished factor, n x r4
      for (int idx = t; idx < n * r4; idx += NT) {
        const int i = idx / r4, r = idx % r4;
        Ug[idx] = r < R ? A[ord[r] * ld + i] : 0.f;  // column ord[r] of the rotated S
      }
      __syncthreads();
      for (int idx = t; idx < r4 * r4; idx += NT) {
        const int r = idx / r4, q = idx % r4;
        float g = 0.f;
        for (int i = 0; i < n; ++i) g = fmaf(Ug[i * r4 + r], Ug[i * r4 + q], g);
        M[idx] = g;
      }
      __syncthreads();
      for (int idx = t; idx < n * r4; idx += NT) {
        const int i = idx / r4, r = idx % r4;
        float v = 0.f;
        for (int q = 0; q < r4; ++q) v = fmaf(Ug[i * r4 + q], M[q * r4 + r], v);
        Us[idx] = 1.5f * Ug[idx] - 0.5f * v;
      }
      __syncthreads();
      for (int r = warp; r < R; r += NT / 32) {
        float best = -1.f;
        int arg = 0;
        for (int i = lane; i < n; i += 32) {
          const float a = fabsf(Us[i * r4 + r]);
          if (a > best) { best = a; arg = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const float ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oa = __shfl_down_sync(0xffffffffu, arg, o);
          if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
        }
        arg = __shfl_sync(0xffffffffu, arg, 0);
        const float sg = Us[arg * r4 + r] < 0.f ? -1.f : 1.f;
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
          const float u = sg * Us[i * r4 + r];
          Us[i * r4 + r] = u;
          fac[i + (int64_t)n * r] = u;
        }
      }
      __syncthreads();
      // 5. TTM into the workspace, or the core after the last mode.
      float* dst = k == 2 ? pt.core : bufs[k & 1];
      cta_ttm<NT>(src, (int)lo, n, hi, Us, R, r4, dst, stage);
      src = dst;
      fac += (int64_t)n * R;
      lo *= R;
      if (k < 2) hi /= dsc.d[k + 1];
    }
  }
}

// ------------------------------------------------------------- variants
struct Variant {
  int nt, kc, minb;
  const void* fn;
  void (*launch)(int grid, cudaStream_t st, const Desc*, const int*, const Ptrs*, int, int*, float*, int64_t, int,
                 int*);
};

template <int NT, int KC, int MINB>
void launch_t(int grid, cudaStream_t st, const Desc* d, const int* q, const Ptrs* p, int count, int* counter,
              float* ws, int64_t wpc, int sweeps, int* status) {
  batched_kernel<NT, KC, MINB><<<grid, NT, SMEM_BYTES, st>>>(d, q, p, count, counter, ws, wpc, sweeps, status);
}

template <int NT, int KC, int MINB>
Variant make_variant() {
  return Variant{NT, KC, MINB, reinterpret_cast<const void*>(&batched_kernel<NT, KC, MINB>), &launch_t<NT, KC, MINB>};
}

const std::vector<Variant>& variants() {
  static const std::vector<Variant> v = {
      make_variant<128, 16, 4>(), make_variant<128, 32, 4>(), make_variant<256, 16, 2>(),
      make_variant<256, 32, 2>(), make_variant<512, 16, 1>(), make_variant<512, 32, 1>(),
  };
  return v;
}

// CTAs per SM a variant reaches (shared memory and registers), at most 4.
int resident(const Variant& v) {
  cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, v.fn, v.nt, SMEM_BYTES);
  return std::max(1, std::min(per, 4));
}

}  // namespace batch
}  // namespace atk

// ----------------------------------------------------------------- C ABI
using namespace atk;
using namespace atk::batch;

struct atucker_batch_s {
  int count = 0;
  cudaStream_t user = nullptr;   // stream the caller runs on
  cudaStream_t cap = nullptr;    // private stream used for graph capture
  Desc* d_desc = nullptr;
  int* d_queue = nullptr;
  Ptrs* d_ptrs = nullptr;
  Ptrs* h_ptrs = nullptr;        // pinned; uploaded by each run
  int* d_counter = nullptr;
  int* d_status = nullptr;
  float* ws = nullptr;
  int64_t ws_per_cta = 0;
  int max_grid = 0;
  std::vector<int> grid;         // per variant: resident CTAs per SM x SMs
  int variant = 2;
  int max_sweeps = 40;
  int use_graph = 1;
  int sync = 0;
  cudaEvent_t done = nullptr;
  bool pending = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_variant = -1;
};

namespace {

void free_graph(atucker_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_variant = -1;
}

// Enqueue one whole batch (upload, reset, kernel) on stream st.
int enqueue(atucker_batch_s* b, int vi, cudaStream_t st) {
  const Variant& v = variants()[vi];
  ATK_CUDA(cudaMemcpyAsync(b->d_ptrs, b->h_ptrs, sizeof(Ptrs) * b->count, cudaMemcpyHostToDevice, st));
  ATK_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st));
  v.launch(b->grid[vi], st, b->d_desc, b->d_queue, b->d_ptrs, b->count, b->d_counter, b->ws, b->ws_per_cta,
           b->max_sweeps, b->d_status);
  ATK_LAUNCHED();
  return ATK_OK;
}

int build_graph(atucker_batch_s* b) {
  free_graph(b);
  ATK_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  int s = enqueue(b, b->variant, b->cap);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (s != ATK_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  ATK_CUDA(e);
  b->graph = g;
  ATK_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
  b->graph_variant = b->variant;
  return ATK_OK;
}

int wait_pending(atucker_batch_s* b) {
  if (b->pending) {
    ATK_CUDA(cudaEventSynchronize(b->done));
    b->pending = false;
  }
  return ATK_OK;
}

int read_status(atucker_batch_s* b) {
  int h = 0;
  ATK_CUDA(cudaMemcpy(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  ATK_CUDA(cudaMemset(b->d_status, 0, sizeof(int)));
  if (h & DEV_TIMEOUT) { set_error("batch: a bounded wait timed out"); return ATK_ETIMEOUT; }
  if (h & DEV_NOCONV) { set_error("batch: Jacobi reached the sweep cap"); return ATK_ENOCONV; }
  return ATK_OK;
}

int set_pointers(atucker_batch_s* b, const float* const* xs, float* const* cores, float* const* factors) {
  if (!xs || !cores || !factors) { set_error("batch: null pointer table"); return ATK_EINVAL; }
  ATK_TRY(wait_pending(b));
  for (int i = 0; i < b->count; ++i) {
    if (!xs[i] || !cores[i] || !factors[i]) { set_error("batch: null tensor pointer"); return ATK_EINVAL; }
    b->h_ptrs[i] = Ptrs{xs[i], cores[i], factors[i]};
  }
  return ATK_OK;
}

}  // namespace

extern "C" {

int atucker_batch_create(atucker_batch_t* out, int count, const int64_t* dims3, const int64_t* ranks3,
                         void* cuda_stream) {
  if (!out || count <= 0 || !dims3 || !ranks3) { set_error("batch_create: bad arguments"); return ATK_EINVAL; }
  *out = nullptr;
  std::vector<Desc> desc(count);
  std::vector<double> cost(count);
  int64_t wpc = 0;
  for (int i = 0; i < count; ++i) {
    Desc d;
    for (int k = 0; k < 3; ++k) {
      const int64_t dk = dims3[3 * i + k], rk = ranks3[3 * i + k];
      if (dk < 1 || dk > DMAX) { set_error("batch_create: every dimension must be in [1, 96]"); return ATK_EUNSUPPORTED; }
      if (rk < 1 || rk > dk || rk > RMAX) { set_error("batch_create: need 1 <= rank <= min(dim, 32)"); return ATK_ERANK; }
      d.d[k] = (int)dk;
      d.r[k] = (int)rk;
    }
    // Tucker feasibility: R_n <= prod_{k != n} R_k.
    for (int k = 0; k < 3; ++k)
      if ((int64_t)d.r[k] > (int64_t)d.r[(k + 1) % 3] * d.r[(k + 2) % 3]) {
        set_error("batch_create: infeasible ranks (R_n > product of the other ranks)");
        return ATK_ERANK;
      }
    desc[i] = d;
    const double d0 = d.d[0], d1 = d.d[1], d2 = d.d[2];
    cost[i] = d0 * d0 * d1 * d2 + d1 * d1 * d.r[0] * d2 + 20.0 * (d0 * d0 * d0 + d1 * d1 * d1 + d2 * d2 * d2);
    wpc = std::max<int64_t>(wpc, (int64_t)d.r[0] * d.d[1] * d.d[2] + (int64_t)d.r[0] * d.r[1] * d.d[2]);
  }
  std::vector<int> queue(count);
  for (int i = 0; i < count; ++i) queue[i] = i;
  std::stable_sort(queue.begin(), queue.end(), [&](int a, int b) { return cost[a] > cost[b]; });

  auto* b = new atucker_batch_s();
  b->count = count;
  b->user = (cudaStream_t)cuda_stream;
  b->ws_per_cta = ((wpc + 63) / 64) * 64;
  // Resident CTAs per variant, fixed before any graph capture.
  for (const Variant& v : variants()) b->grid.push_back(resident(v) * num_sms());
  b->max_grid = *std::max_element(b->grid.begin(), b->grid.end());
  auto fail = [&](const char* what) {
    atucker_batch_destroy(b);
    set_error(what);
    return ATK_ENOMEM;
  };
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return fail("batch: stream");
  if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) return fail("batch: event");
  if (cudaMalloc(&b->d_desc, sizeof(Desc) * count) != cudaSuccess) return fail("batch: out of device memory");
  if (cudaMalloc(&b->d_queue, sizeof(int) * count) != cudaSuccess) return fail("batch: out of device memory");
  if (cudaMalloc(&b->d_ptrs, sizeof(Ptrs) * count) != cudaSuccess) return fail("batch: out of device memory");
  if (cudaMalloc(&b->d_counter, sizeof(int) * 2) != cudaSuccess) return fail("batch: out of device memory");
  if (cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess) return fail("batch: out of device memory");
  if (dev_alloc((void**)&b->ws, sizeof(float) * b->ws_per_cta * b->max_grid, "cudaMalloc(batch workspace)") != ATK_OK)
    return fail("batch: out of device memory (workspace)");
  if (cudaMallocHost(&b->h_ptrs, sizeof(Ptrs) * count) != cudaSuccess) return fail("batch: pinned memory");
  if (cudaMemcpy(b->d_desc, desc.data(), sizeof(Desc) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_queue, queue.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess)
    return fail("batch: upload failed");
  *out = b;
  return ATK_OK;
}

int atucker_batch_set_option(atucker_batch_t b, int option, int64_t value) {
  if (!b) { set_error("batch_set_option: null batch"); return ATK_EINVAL; }
  switch (option) {
    case ATK_BATCH_OPT_VARIANT:
      if (value < 0 || value >= (int64_t)variants().size()) { set_error("batch: no such variant"); return ATK_EINVAL; }
      b->variant = (int)value;
      return ATK_OK;
    case ATK_BATCH_OPT_GRAPH: b->use_graph = value != 0; return ATK_OK;
    case ATK_BATCH_OPT_SYNC: b->sync = value != 0; return ATK_OK;
    case ATK_BATCH_OPT_JACOBI_MAX_SWEEPS:
      if (value < 1 || value > 1000) { set_error("batch: sweeps in [1, 1000]"); return ATK_EINVAL; }
      b->max_sweeps = (int)value;
      free_graph(b);
      return ATK_OK;
    default: set_error("batch_set_option: unknown option"); return ATK_EINVAL;
  }
}

int atucker_batch_variants(int* count_out, int* threads_out, int* chunk_out) {
  const auto& v = variants();
  if (count_out) *count_out = (int)v.size();
  for (size_t i = 0; i < v.size(); ++i) {
    if (threads_out) threads_out[i] = v[i].nt;
    if (chunk_out) chunk_out[i] = v[i].kc;
  }
  return ATK_OK;
}

int atucker_batch_run(atucker_batch_t b, const float* const* xs, float* const* cores, float* const* factors) {
  if (!b) { set_error("batch_run: null batch"); return ATK_EINVAL; }
  ATK_TRY(set_pointers(b, xs, cores, factors));
  if (b->use_graph) {
    if (b->graph_variant != b->variant) ATK_TRY(build_graph(b));
    ATK_CUDA(cudaGraphLaunch(b->exec, b->user));
  } else {
    ATK_TRY(enqueue(b, b->variant, b->user));
  }
  ATK_CUDA(cudaEventRecord(b->done, b->user));
  b->pending = true;
  if (b->sync) return atucker_batch_sync(b);
  return ATK_OK;
}

int atucker_batch_sync(atucker_batch_t b) {
  if (!b) { set_error("batch_sync: null batch"); return ATK_EINVAL; }
  ATK_TRY(wait_pending(b));
  return read_status(b);
}

int atucker_batch_tune(atucker_batch_t b, const float* const* xs, float* const* cores, float* const* factors,
                       int reps, float* ms_out) {
  if (!b) { set_error("batch_tune: null batch"); return ATK_EINVAL; }
  if (reps < 1) reps = 1;
  ATK_TRY(set_pointers(b, xs, cores, factors));
  cudaEvent_t e0, e1;
  ATK_CUDA(cudaEventCreate(&e0));
  ATK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  int bestv = b->variant;
  int st = ATK_OK;
  for (size_t vi = 0; vi < variants().size() && st == ATK_OK; ++vi) {
    st = enqueue(b, (int)vi, b->user);  // warm-up
    float tot = 0.f;
    for (int r = 0; r < reps && st == ATK_OK; ++r) {
      if (cudaEventRecord(e0, b->user) != cudaSuccess) st = ATK_ECUDA;
      if (st == ATK_OK) st = enqueue(b, (int)vi, b->user);
      if (st == ATK_OK && cudaEventRecord(e1, b->user) != cudaSuccess) st = ATK_ECUDA;
      if (st == ATK_OK && cudaEventSynchronize(e1) != cudaSuccess) st = ATK_ECUDA;
      float ms = 0.f;
      if (st == ATK_OK) cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    if (st != ATK_OK) break;
    const float ms = tot / reps;
    if (ms_out) ms_out[vi] = ms;
    if (vi == 0 || ms < best) {
      best = ms;
      bestv = (int)vi;
    }
    st = read_status(b);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ATK_OK) return st;
  b->variant = bestv;
  return ATK_OK;
}

int atucker_batch_get_variant(atucker_batch_t b, int* variant_out) {
  if (!b || !variant_out) { set_error("batch_get_variant: bad arguments"); return ATK_EINVAL; }
  *variant_out = b->variant;
  return ATK_OK;
}

void atucker_batch_destroy(atucker_batch_t b) {
  if (!b) return;
  if (b->pending && b->done) cudaEventSynchronize(b->done);
  free_graph(b);
  cudaFree(b->d_desc);
  cudaFree(b->d_queue);
  cudaFree(b->d_ptrs);
  cudaFree(b->d_counter);
  cudaFree(b->d_status);
  cudaFree(b->ws);
  if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
  if (b->done) cudaEventDestroy(b->done);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

}  // extern "C"
