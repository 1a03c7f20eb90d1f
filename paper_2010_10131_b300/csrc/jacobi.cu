// Leading eigenvectors of the Gram matrix (Alg. 2, EIG branch:
// "U^(n) <- R_n leading eigenvectors of S") by the cyclic Jacobi method with
// parallel (round-robin) ordering; the rotation rules and the shared-memory
// sweep routine are in jacobi_dev.cuh.
//
// Two drivers:
//  * n <= 128 (float rotations) or n <= 112 (double): one CTA holds A and V in
//    shared memory and runs every round with __syncthreads between them.
//  * larger n: block Jacobi.  The index range is cut into blocks of b = 32.  A
//    round pairs blocks (P_k, Q_k).  Each 64 x 64 sub-problem is diagonalised
//    in shared memory by the same scalar routine, which yields W_k and the
//    rotated diagonal block.  Then the off-diagonal blocks A_kl <- W_k^T A_kl W_l
//    and V <- V W are applied as 64 x 64 block products across all SMs.  This
//    is a persistent cooperative kernel with a bounded grid barrier between
//    phases.
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>
#include <vector>

#include "jacobi_dev.cuh"

namespace atk {

// Raise a kernel's dynamic shared-memory limit to at least `bytes`, never
// lower it: launches captured in cached graphs keep their sizes, so a later
// call with a smaller block must not shrink the limit under them.
int raise_smem_limit(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, size_t>> seen;
  std::lock_guard<std::mutex> g(mu);
  for (auto& e : seen)
    if (e.first == fn) {
      if (e.second >= bytes) return ATK_OK;
      ATK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      e.second = bytes;
      return ATK_OK;
    }
  ATK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  seen.push_back({fn, bytes});
  return ATK_OK;
}

// ---------------------------------------------------------- one-CTA driver
// One matrix per CTA (blockIdx.x), padded to m = n rounded up to even.
// Writes diag (n) and V (n x n, row-major, column j = eigenvector j) to global.
template <typename T>
__global__ void __launch_bounds__(1024) jacobi_small_kernel(const double* __restrict__ S, int n, int m, int max_sweeps,
                                                           T* __restrict__ diag_out, T* __restrict__ V_out,
                                                           int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = m + 1;
  T* A = reinterpret_cast<T*>(smem_raw);
  T* V = A + m * ld;
  T* cs = V + m * ld;
  int* pq = reinterpret_cast<int*>(cs + m);
  int* flag = pq + m;
  unsigned short* blk = reinterpret_cast<unsigned short*>(flag + 2);
  __shared__ double red[1024];
  const double* Sm = S + (size_t)blockIdx.x * n * n;
  double loc = 0.0;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, j = idx % m;
    double v = (i < n && j < n) ? Sm[i + (size_t)n * j] : 0.0;
    A[i * ld + j] = (T)v;
    V[i * ld + j] = (i == j) ? T(1) : T(0);
    loc += v * v;
  }
  red[threadIdx.x] = loc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  T fro = (T)sqrt(red[0]);
  JWork<T> w{A, V, cs, pq, flag, blk, ld};
  bool conv = true;
  if (m >= 2) jacobi_smem<T>(w, m, fro, max_sweeps, &conv);
  if (!conv && threadIdx.x == 0) atomicOr(status, DEV_NOCONV);
  T* dg = diag_out + (size_t)blockIdx.x * n;
  T* vo = V_out + (size_t)blockIdx.x * n * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dg[i] = A[i * ld + i];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int i = idx / n, j = idx % n;
    vo[idx] = V[i * ld + j];
  }
}

// ------------------------------------------------------ block Jacobi driver
constexpr int JB = 32;       // block size b; sub-problems are 2b x 2b
constexpr int JS = 2 * JB;   // 64

struct BlockJacobiArgs {
  int n, m, mb;   // true size, padded size (multiple of 64), number of blocks
  int max_sweeps, inner_sweeps;
  unsigned* bar;  // grid barrier words (2)
  int* sweep_flags;  // per outer sweep: 1 if any rotation happened
  int* status;
  long long wait_polls;  // poll limit of each grid-barrier wait
};

// Global index of local index u (0..63) in the sub-problem of blocks (P, Q).
__device__ __forceinline__ int sub_index(int u, int P, int Q) { return u < JB ? P * JB + u : Q * JB + (u - JB); }

template <typename T>
__global__ void __launch_bounds__(256) jacobi_block_kernel(BlockJacobiArgs args, T* __restrict__ A,
                                                           T* __restrict__ V, T* __restrict__ W, T fro) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s0 = reinterpret_cast<T*>(smem_raw);  // 4 tiles of 64 x 64
  T* s1 = s0 + JS * JS;
  T* s2 = s1 + JS * JS;
  T* s3 = s2 + JS * JS;
  T* cs = s3 + JS * JS;
  int* pq = reinterpret_cast<int*>(cs + JS);
  int* flag = pq + JS;
  unsigned short* blk = reinterpret_cast<unsigned short*>(flag + 2);
  const int m = args.m, mb = args.mb, half = mb / 2;
  const unsigned G = gridDim.x;
  for (int sweep = 0; sweep < args.max_sweeps; ++sweep) {
    for (int r = 0; r < mb - 1; ++r) {
      // Phase 1: diagonalise the 64 x 64 sub-problem of each block pair.
      for (int k = blockIdx.x; k < half; k += G) {
        int P, Q;
        rr_pair(r, k, mb, P, Q);
        for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
          int u = idx / JS, v = idx % JS;
          s0[idx] = A[(size_t)sub_index(u, P, Q) * m + sub_index(v, P, Q)];
          s1[idx] = (u == v) ? T(1) : T(0);
        }
        __syncthreads();
        JWork<T> w{s0, s1, cs, pq, flag, blk, JS};
        bool conv;
        jacobi_smem<T>(w, JS, fro, args.inner_sweeps, &conv);
        if (threadIdx.x == 0 && flag[1]) atomicOr(args.sweep_flags + sweep, 1);
        // The rotated sub-problem is W_k^T A_kk W_k, computed by exact 2x2
        // rotations: write it back here.  Phase 2 skips the diagonal blocks, since
        // a 64-term product would put rounding noise of order eps * lambda_max
        // back into the entries just eliminated.
        T* Wk = W + (size_t)k * JS * JS;
        for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
          int u = idx / JS, v = idx % JS;
          Wk[idx] = s1[idx];
          A[(size_t)sub_index(u, P, Q) * m + sub_index(v, P, Q)] = s0[idx];
        }
        __syncthreads();
      }
      if (!grid_barrier(args.bar, G, args.status, args.wait_polls)) return;
      // Phase 2: A_kl <- W_k^T A_kl W_l (k < l, mirrored) and V_l <- V_l W_l.
      const int ntA = half * (half - 1) / 2;
      const int nrow = m / JS;
      const int ntV = half * nrow;
      for (int task = blockIdx.x; task < ntA + ntV; task += G) {
        if (task < ntA) {
          int k = 0, rem = task;
          while (rem >= half - 1 - k) { rem -= half - 1 - k; ++k; }
          int l = k + 1 + rem;
          int Pk, Qk, Pl, Ql;
          rr_pair(r, k, mb, Pk, Qk);
          rr_pair(r, l, mb, Pl, Ql);
          const T* Wk = W + (size_t)k * JS * JS;
          const T* Wl = W + (size_t)l * JS * JS;
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            s0[idx] = A[(size_t)sub_index(u, Pk, Qk) * m + sub_index(v, Pl, Ql)];
            s1[idx] = Wk[idx];
            s2[idx] = Wl[idx];
          }
          __syncthreads();
          // s3 = X W_l
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            T acc = 0;
#pragma unroll 8
            for (int t = 0; t < JS; ++t) acc += s0[u * JS + t] * s2[t * JS + v];
            s3[idx] = acc;
          }
          __syncthreads();
          // X' = W_k^T s3, written back (and mirrored for k < l)
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            T acc = 0;
#pragma unroll 8
            for (int t = 0; t < JS; ++t) acc += s1[t * JS + u] * s3[t * JS + v];
            int gu = sub_index(u, Pk, Qk), gv = sub_index(v, Pl, Ql);
            A[(size_t)gu * m + gv] = acc;
            A[(size_t)gv * m + gu] = acc;
          }
          __syncthreads();
        } else {
          int t2 = task - ntA;
          int l = t2 % half, rowc = t2 / half;
          int Pl, Ql;
          rr_pair(r, l, mb, Pl, Ql);
          const T* Wl = W + (size_t)l * JS * JS;
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            s0[idx] = V[(size_t)(rowc * JS + u) * m + sub_index(v, Pl, Ql)];
            s2[idx] = Wl[idx];
          }
          __syncthreads();
          for (int idx = threadIdx.x; idx < JS * JS; idx += blockDim.x) {
            int u = idx / JS, v = idx % JS;
            T acc = 0;
#pragma unroll 8
            for (int t = 0; t < JS; ++t) acc += s0[u * JS + t] * s2[t * JS + v];
            V[(size_t)(rowc * JS + u) * m + sub_index(v, Pl, Ql)] = acc;
          }
          __syncthreads();
        }
      }
      if (!grid_barrier(args.bar, G, args.status, args.wait_polls)) return;
    }
    if (*(volatile int*)(args.sweep_flags + sweep) == 0) return;  // converged
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(args.status, DEV_NOCONV);
}

// ------------------------------------------------------------- selection
// Sort eigenvalues descending (stable in index), keep the first R vectors,
// sign each so that its largest-magnitude entry is positive (ties: lowest
// row), write U (n x R column-major, float64), all eigenvalues (descending)
// and the discarded sum.  One CTA, a warp per selected column.  V is row-major
// with leading dimension ldv.
constexpr int SEL_THREADS = 1024;
template <typename T>
__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const T* __restrict__ diag, int64_t dstride,
                                                     const T* __restrict__ V, int ldv, int n, int R,
                                                     double* __restrict__ U, double* __restrict__ lam_out,
                                                     double* __restrict__ disc_out) {
  __shared__ int order[1024];
  __shared__ T lam[1024];
  __shared__ double wsum[SEL_THREADS / 32];
  // Sort key: the eigenvalue, with NaN ordered below everything, ties broken by
  // index.  That is a total order, so the ranks below are a permutation of
  // 0..n-1 whatever the input holds, and every gathered column stays in range.
  // The comparisons run in T (float32 keys need no float64 pipe).
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T v = diag[(int64_t)i * dstride];
    lam[i] = isnan(v) ? -(T)INFINITY : v;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T li = lam[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T lj = lam[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
  if (lam_out)
    for (int r = threadIdx.x; r < n; r += blockDim.x) lam_out[r] = (double)lam[order[r]];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  if (disc_out) {
    // Discarded energy: per-thread strided sums, then a fixed-order tree.
    double loc = 0.0;
    for (int r = R + threadIdx.x; r < n; r += blockDim.x) loc += (double)lam[order[r]];
    for (int o = 16; o > 0; o >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, o);
    if (lane == 0) wsum[warp] = loc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += wsum[w];
      *disc_out = s;
    }
  }
  // One warp per selected column; the sign rule compares in T.
  for (int r = warp; r < R; r += nw) {
    const int col = order[r];
    T best = (T)-1;
    int arg = 0;
    for (int i = lane; i < n; i += 32) {
      const T a = fabs(V[(int64_t)i * ldv + col]);
      if (a > best) { best = a; arg = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oa = __shfl_down_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
    }
    arg = __shfl_sync(0xffffffffu, arg, 0);
    const double sg = (V[(int64_t)arg * ldv + col] < (T)0) ? -1.0 : 1.0;
    for (int i = lane; i < n; i += 32) U[i + (int64_t)n * r] = sg * (double)V[(int64_t)i * ldv + col];
  }
}

// --------------------------------------------------------------- host side
namespace {
template <typename T>
size_t small_smem(int m) {
  return (size_t)2 * m * (m + 1) * sizeof(T) + (size_t)m * sizeof(T) + (size_t)(m + 2) * sizeof(int) +
         (size_t)2 * nblocks_of(m) * sizeof(unsigned short) + 16;
}
template <typename T>
bool use_small(int n) {
  int m = n + (n & 1);
  return small_smem<T>(m) <= 220 * 1024;
}
template <typename T>
size_t block_smem() {
  return (size_t)4 * JS * JS * sizeof(T) + JS * sizeof(T) + (JS + 2) * sizeof(int) +
         (size_t)2 * nblocks_of(JS) * sizeof(unsigned short) + 16;
}
template <typename T>
size_t eig_bytes_t(int64_t n) {
  size_t b = 4096;
  if (use_small<T>((int)n)) {
    b += (size_t)(n * n + n) * sizeof(T) + 1024;
  } else {
    int64_t m = ceil_div(n, JS) * JS;
    int64_t mb = m / JB;
    b += (size_t)(2 * m * m + (mb / 2) * JS * JS) * sizeof(T) + 64 * sizeof(int) + 1024;
  }
  return b;
}

__global__ void init_block_kernel(const double* __restrict__ S, int n, int m, float* Af, float* Vf, double* Ad,
                                  double* Vd) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  int i = (int)(idx / m), j = (int)(idx % m);
  double v = (i < n && j < n) ? S[i + (int64_t)n * j] : 0.0;
  double e = (i == j) ? 1.0 : 0.0;
  if (Af) { Af[idx] = (float)v; Vf[idx] = (float)e; }
  if (Ad) { Ad[idx] = v; Vd[idx] = e; }
}

__global__ void fro_kernel(const double* __restrict__ S, int64_t count, double* out) {
  __shared__ double red[256];
  double loc = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) loc += S[i] * S[i];
  red[threadIdx.x] = loc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sqrt(red[0]);
}

template <typename T>
int eig_top_t(const double* S, int64_t n, int64_t R, int max_sweeps, double* U64, double* lam_out,
              double* disc_out, int* dev_status, char* scratch, size_t scratch_bytes, cudaStream_t st) {
  Arena ar{scratch, scratch_bytes, 0};
  if (use_small<T>((int)n)) {
    int m = (int)(n + (n & 1));
    T* diag = (T*)ar.take(sizeof(T) * n);
    T* V = (T*)ar.take(sizeof(T) * n * n);
    if (!diag || !V) { set_error("eig: scratch too small"); return ATK_EINVAL; }
    size_t sm = small_smem<T>(m);
    ATK_TRY(raise_smem_limit((const void*)jacobi_small_kernel<T>, sm));
    jacobi_small_kernel<T><<<1, 256, sm, st>>>(S, (int)n, m, max_sweeps, diag, V, dev_status);
    ATK_LAUNCHED();
    select_kernel<T><<<1, SEL_THREADS, 0, st>>>(diag, 1, V, (int)n, (int)n, (int)R, U64, lam_out, nullptr);
    ATK_LAUNCHED();
    return ATK_OK;
  }
  const int m = (int)(ceil_div(n, JS) * JS);
  const int mb = m / JB;
  T* A = (T*)ar.take(sizeof(T) * (size_t)m * m);
  T* V = (T*)ar.take(sizeof(T) * (size_t)m * m);
  T* W = (T*)ar.take(sizeof(T) * (size_t)(mb / 2) * JS * JS);
  int* words = (int*)ar.take(sizeof(int) * 64 + 64);
  double* fro_d = (double*)ar.take(sizeof(double));
  if (!A || !V || !W || !words || !fro_d) { set_error("eig: scratch too small"); return ATK_EINVAL; }
  ATK_CUDA(cudaMemsetAsync(words, 0, sizeof(int) * 64 + 64, st));
  const bool f = sizeof(T) == 4;
  init_block_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(
      S, (int)n, m, f ? (float*)A : nullptr, f ? (float*)V : nullptr, f ? nullptr : (double*)A,
      f ? nullptr : (double*)V);
  ATK_LAUNCHED();
  fro_kernel<<<1, 256, 0, st>>>(S, n * n, fro_d);
  ATK_LAUNCHED();
  double fro_h = 0.0;
  ATK_CUDA(cudaMemcpyAsync(&fro_h, fro_d, sizeof(double), cudaMemcpyDeviceToHost, st));
  ATK_CUDA(cudaStreamSynchronize(st));
  BlockJacobiArgs args;
  args.n = (int)n;
  args.m = m;
  args.mb = mb;
  args.max_sweeps = std::min(max_sweeps, 60);
  args.inner_sweeps = 3;
  args.bar = reinterpret_cast<unsigned*>(words);
  args.sweep_flags = words + 2;
  args.status = dev_status;
  args.wait_polls = wait_limit() > 0 ? wait_limit() : 20000000LL;
  size_t sm = block_smem<T>();
  ATK_TRY(raise_smem_limit((const void*)jacobi_block_kernel<T>, sm));
  int per_sm = 0;
  ATK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_block_kernel<T>, 256, sm));
  if (per_sm < 1) { set_error("eig: block Jacobi kernel does not fit on an SM"); return ATK_EUNSUPPORTED; }
  int ntasks = (mb / 2) * (mb / 2 - 1) / 2 + (mb / 2) * (m / JS);
  int grid = std::min(num_sms() * per_sm, std::max(ntasks, mb / 2));
  T fro = (T)fro_h;
  void* kargs[] = {(void*)&args, (void*)&A, (void*)&V, (void*)&W, (void*)&fro};
  ATK_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_block_kernel<T>, dim3(grid), dim3(256), kargs, sm, st));
  count_launch();
  select_kernel<T><<<1, SEL_THREADS, 0, st>>>(A, (int64_t)m + 1, V, m, (int)n, (int)R, U64, lam_out, nullptr);
  ATK_LAUNCHED();
  return ATK_OK;
}
}  // namespace

// ------------------------------------------------------------ graph cache
// A launch sequence with no host synchronisation inside (the refinement tail
// of the eigensolver: about 60 small kernels) is captured once into a CUDA
// graph per key (every pointer and size it uses) and replayed afterwards, so
// the host enqueues one graph instead of every kernel.  A key fixes every
// kernel argument, so a replay does exactly what the direct launches would.
namespace {
struct GraphKey {
  const void* p[8];
  int64_t v[4];
  bool operator==(const GraphKey& o) const {
    for (int i = 0; i < 8; ++i)
      if (p[i] != o.p[i]) return false;
    for (int i = 0; i < 4; ++i)
      if (v[i] != o.v[i]) return false;
    return true;
  }
};
struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
  long long kernels;  // launches recorded at capture, counted again per replay
};
constexpr size_t GRAPH_CACHE_MAX = 64;
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;

template <class F>
int run_graph(const GraphKey& key, cudaStream_t st, F&& body) {
  {
    std::lock_guard<std::mutex> g(g_graph_mu);
    for (const GraphEntry& e : g_graphs)
      if (e.key == key) {
        ATK_CUDA(cudaGraphLaunch(e.exec, st));
        count_launches(e.kernels);
        return ATK_OK;
      }
  }
  thread_local cudaStream_t cap = nullptr;
  if (!cap && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    cap = nullptr;
    return body(st);
  }
  const long long before = launch_count();
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return body(st);
  const int s = body(cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cap, &graph);
  cudaGraphExec_t exec = nullptr;
  if (s != ATK_OK || e != cudaSuccess || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (s != ATK_OK) return s;
    return body(st);  // capture refused: run the launches directly
  }
  cudaGraphDestroy(graph);
  const long long kernels = launch_count() - before;
  ATK_CUDA(cudaGraphLaunch(exec, st));
  std::lock_guard<std::mutex> g(g_graph_mu);
  if (g_graphs.size() >= GRAPH_CACHE_MAX) {
    cudaGraphExecDestroy(g_graphs.front().exec);
    g_graphs.erase(g_graphs.begin());
  }
  g_graphs.push_back({key, exec, kernels});
  return ATK_OK;
}
}  // namespace

// ------------------------------------------------- Rayleigh-Ritz subspace path
// Only the R leading eigenvectors are needed (Alg. 2: "R_n leading
// eigenvectors of S").  For m = R + p well below n, this path works on an
// n x m block:
//  1. one power step from a random block, Q <- orth(S Q), orthonormalised by
//     shifted CholeskyQR3;
//  2. a Rayleigh-Ritz projection B = Q^T S Q diagonalised by the one-CTA
//     tridiagonal eigensolver (tridiag_eig.cu), giving Ritz vectors Q W;
//  3. power steps from the Ritz vectors (S Q W = Z W is already at hand, two
//     CholeskyQR passes suffice) and further Rayleigh-Ritz projections until
//     the predicted error after the float64 refinement,
//       (theta_m / theta_K) * max_{j<K} ||S q_j - theta_j q_j|| / (theta_K - theta_m),
//     drops below RR_TARGET, or stops falling while below RR_FLOOR_OK (the
//     float32 floor of the residuals).  That is a Davis-Kahan bound on the angle
//     between q_K and the leading space, times the contraction of the
//     refinement's subspace step.  K is R, or fewer: Ritz values below
//     RR_RESOLVE eps_32 theta_1 are not resolved by float32 products at all,
//     so they take no part in the test (eig_top resolves them on a deflated
//     matrix).  Between two projections the path takes as many power steps
//     as the observed rate theta_m / theta_K predicts (at most RR_POWER_CHUNK).
// When theta_m / theta_K > RR_MAX_RATE (the cut sits inside a cluster that
// the block does not cover) or RR_MAX_POWER power steps pass, the full
// Jacobi runs instead.  On the deflated levels of eig_top (floor_ok) a stall
// or the step cap ends the iteration as converged to the float32 floor.  Every product runs on the contraction engine of
// fp32_ops.cu: the n x m block is the mode-2 view (lo = n, I = m, hi = 1) of
// an n x m column-major matrix.
constexpr int RR_MAX_POWER = 160;
constexpr int RR_POWER_CHUNK = 8;
constexpr double RR_TARGET = 1e-6;
constexpr double RR_MAX_RATE = 0.92;
// Stall test: a projection after power steps that leaves the predicted error
// above RR_STALL times the previous one has met the float32 floor; below
// RR_FLOOR_OK that is accepted, above it three such projections in a row
// mean no convergence.
constexpr double RR_STALL = 0.5;
constexpr double RR_FLOOR_OK = 1e-4;
constexpr float RR_RESOLVE = 32.f * 1.1920929e-7f;
constexpr double RR_CUT_RESOLVE = 64.0 * 1.1920928955078125e-7;
// Relative gap at the cut above which a converged Ritz block takes the light
// float64 finish.
constexpr double RR_LIGHT_GAP = 1e-3;
// ... and whose largest kept residual is below this fraction of the gap to the
// guard block (a Davis-Kahan bound on the float32 vectors themselves).
constexpr double RR_LIGHT_RES = 1e-4;

// Block width m = R + p.  The default guard p = clamp(R / 2, 8, 16) suits a
// spectrum with a gap at the cut; `wide` (the deflated levels of eig_top,
// where the cut lies in a slowly decaying tail) takes p = max(32, R).
int rr_width(int64_t n, int64_t R, bool wide) {
  int64_t p = wide ? std::max<int64_t>(32, R) : std::max<int64_t>(8, std::min<int64_t>(16, R / 2));
  return (int)std::min<int64_t>(std::min<int64_t>(n, R + p), 156);
}

__global__ void rand_fill_kernel(float* __restrict__ Q, int64_t count, uint64_t seed) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z ^= z >> 31;
  Q[i] = (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// Y += sigma X with sigma = rel * max_i S_ii (S n x n float32, every CTA
// finds the maximum itself): the power steps use S + sigma I, which has the
// same eigenvectors as S.  For an S of rank below the block width m (a mode
// whose rank equals the product of the other ranks, or an exactly low-rank
// tensor) S Q spans only rank(S) directions and the unshifted CholeskyQR
// passes would break down; the shift keeps the block at full rank, the
// surplus columns becoming null-space directions.  The Rayleigh-Ritz
// projection and the residuals use S itself.
constexpr float RR_POWER_SHIFT = 1e-5f;
__global__ void shift_axpy_kernel(float* __restrict__ Y, const float* __restrict__ X, const float* __restrict__ S,
                                  int64_t n, int64_t count, float rel) {
  __shared__ float red[32];
  float mx = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, S[i * (n + 1)]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const float sigma = rel * red[0];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) Y[i] = fmaf(sigma, X[i], Y[i]);
}

// Column kernels of the eigensolver: one CTA of COL_THREADS threads per
// column (a warp per column left each of them 20 dependent trips to L2 at
// I_n = 640).  Per-thread strided partial sums, then warp shuffles and the
// warps' sums in warp order: a fixed order, so results do not depend on
// scheduling.
constexpr int COL_THREADS = 128;
constexpr int COL_WARPS = COL_THREADS / 32;
__device__ __forceinline__ double col_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x % 32 == 0) sh[threadIdx.x / 32] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < COL_WARPS; ++w) t += sh[w];
  __syncthreads();  // sh is free for the next reduction
  return t;
}

// Normalise each column of Y (n x m) to unit length; one CTA per column.
__global__ void __launch_bounds__(COL_THREADS) colnorm_f32_kernel(float* __restrict__ Y, int64_t n) {
  __shared__ double sh[COL_WARPS];
  float* y = Y + n * blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) s += (double)y[i] * y[i];
  s = col_sum(s, sh);
  const float inv = s > 0.0 ? (float)(1.0 / sqrt(s)) : 0.f;
  for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) y[i] *= inv;
}


// res[j] = ||Z[:, j] - theta_j Q[:, j]|| for j < R; one CTA per column.
__global__ void __launch_bounds__(COL_THREADS) ritz_residual_kernel(const float* __restrict__ Z,
                                                                     const float* __restrict__ Q,
                                                                     const double* __restrict__ theta, int64_t n,
                                                                     double* __restrict__ res) {
  __shared__ double sh[COL_WARPS];
  const int64_t j = blockIdx.x;
  const double th = theta[j];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) {
    const double d = (double)Z[i + n * j] - th * Q[i + n * j];
    s += d * d;
  }
  s = col_sum(s, sh);
  if (threadIdx.x == 0) res[j] = sqrt(s);
}

// K = the number of leading Ritz values (theta descending) at or above
// RR_RESOLVE theta_0, at most R.  out[0] = max_{j<K} res[j] (NaN if any is
// NaN), out[1] = theta[0], out[2] = theta[K-1], out[3] = theta[m-1], out[4] =
// 1 if a CholeskyQR pass broke down since the last summary (the flag is
// cleared), out[5] = K.
__global__ void ritz_summary_kernel(const double* __restrict__ res, const double* __restrict__ theta, int R, int m,
                                    int* __restrict__ breakdown, double* __restrict__ out) {
  // One warp: K by a warp count (theta is sorted), then strided residuals
  // (independent loads) and a max over the warp; NaN wins (a NaN residual
  // must reach the host).
  const int lane = threadIdx.x;
  const double floor_ = (double)RR_RESOLVE * theta[0];
  int cnt = 0;
  for (int j = lane; j < R; j += 32) cnt += theta[j] >= floor_ ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  const int K = cnt > 0 ? cnt : 1;
  double w = 0.0;
  for (int j = lane; j < K; j += 32) w = (res[j] > w || res[j] != res[j]) ? res[j] : w;
  for (int o = 16; o > 0; o >>= 1) {
    const double ow = __shfl_xor_sync(0xffffffffu, w, o);
    w = (ow > w || ow != ow) ? ow : w;
  }
  if (lane != 0) return;
  out[0] = w;
  out[1] = theta[0];
  out[2] = theta[K - 1];
  out[3] = theta[m - 1];
  out[4] = *breakdown ? 1.0 : 0.0;
  out[5] = (double)K;
  out[6] = theta[R < m ? R : m - 1];  // the first Ritz value past the cut
  *breakdown = 0;
}

__global__ void f32_to_f64_kernel2(const float* __restrict__ s, double* __restrict__ d, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) d[i] = (double)s[i];
}

namespace {
struct RRBufs {
  float *Sf, *Q, *Y, *Z, *T, *LinvT, *Vb, *diag, *Wf;  // LinvT = L^{-T} of the last CholeskyQR pass
  double *G, *W64, *theta, *res, *summary, *Cd;  // Cd: n x m float64 product S Q
  int* breakdown;  // set by cholinv_f32 when a pivot hits its floor
  float* part;  // split-K partials of the m x m products
  size_t part_bytes;
};
size_t rr_part_bytes(int64_t n, int m) {
  View v{n, m, 1};
  const View sv{n, n, 1};  // S's rows as the contracted index (S = S^T): S Q by split-K
  return std::max(std::max(gram_scratch_bytes(v), cross_scratch_bytes(v, m)), cross_scratch_bytes(sv, m));
}
size_t rr_bytes(int64_t n, int m) {
  size_t nm = (size_t)n * m, mm = (size_t)m * m;
  return sizeof(float) * ((size_t)n * n + 4 * nm + 3 * mm + m) + sizeof(double) * (2 * mm + 2 * m + 8 + nm) +
         rr_part_bytes(n, m) + 18 * 256 + 16;
}
// out = S Q (n x m, float32) for the symmetric float32 S.  With the view
// (lo = n, n, hi = 1) the contracted index c is S's row index and the right
// operand P(c, r) = Q[c + n r] is column-major, as the CI kernel reads it;
// split-K keeps many CTAs busy even for small n x m outputs, the partials are
// summed in a fixed order, then rounded to float32.
int sq_product(const float* Sf, int64_t n, const float* Q, int m, float* out, RRBufs& b, cudaStream_t st) {
  const View sv{n, n, 1};
  ATK_TRY(cross_f32(Sf, sv, Q, m, b.Cd, b.part, b.part_bytes, st));
  return f64_to_f32(b.Cd, out, n * (int64_t)m, st);
}
// One CholeskyQR pass: Q = Y L^{-T} with L L^T = Y^T Y + shift I, after
// normalising the columns of Y (in place).
int cholqr_pass_f32(float* Y, float* Q, int64_t n, int m, float shift, RRBufs& b, cudaStream_t st) {
  const View v{n, m, 1};
  colnorm_f32_kernel<<<(unsigned)m, COL_THREADS, 0, st>>>(Y, n);
  ATK_LAUNCHED();
  ATK_TRY(gram_f32(Y, v, b.G, b.part, b.part_bytes, st));
  ATK_TRY(cholinv_f32(b.G, m, shift, b.LinvT, b.breakdown, st));
  return ttm_f32(Y, v, b.LinvT, m, Q, st);  // Q = Y L^{-T}
}
// Shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Zhang, Yamamoto, SISC 2020):
// the shifted first pass cannot break down, and it leaves a basis with modest
// condition number.  The two plain passes then make it orthonormal to
// float32 accuracy.  Y and T are overwritten; the result is in Q.
int cholqr3_f32(float* Y, float* T, float* Q, int64_t n, int m, RRBufs& b, cudaStream_t st) {
  ATK_TRY(cholqr_pass_f32(Y, T, n, m, 1e-5f, b, st));
  ATK_TRY(cholqr_pass_f32(T, Y, n, m, 0.f, b, st));
  ATK_TRY(cholqr_pass_f32(Y, Q, n, m, 0.f, b, st));
  return ATK_OK;
}
}  // namespace

// Leading Ritz block of S by subspace iteration + Rayleigh-Ritz.  On
// success writes Qblk (n x m float64, Ritz vectors in descending Ritz-value
// order, orthonormal to float32 accuracy) and returns ATK_OK; returns
// ATK_ENOCONV to request the full Jacobi.
int rr_top(const double* S, int64_t n, int64_t R, int m, int max_sweeps, double* Qblk, int* dev_status,
           char* scratch, size_t scratch_bytes, cudaStream_t st, bool floor_ok, bool* at_floor, bool* tight,
           double* theta_cut) {
  *at_floor = false;
  *tight = false;
  *theta_cut = 0.0;
  Arena ar{scratch, scratch_bytes, 0};
  RRBufs b;
  size_t nm = (size_t)n * m, mm = (size_t)m * m;
  b.Sf = (float*)ar.take(sizeof(float) * n * n);
  b.Q = (float*)ar.take(sizeof(float) * nm);
  b.Y = (float*)ar.take(sizeof(float) * nm);
  b.Z = (float*)ar.take(sizeof(float) * nm);
  b.T = (float*)ar.take(sizeof(float) * nm);
  b.LinvT = (float*)ar.take(sizeof(float) * mm);
  b.Vb = (float*)ar.take(sizeof(float) * mm);
  b.Wf = (float*)ar.take(sizeof(float) * mm);
  b.diag = (float*)ar.take(sizeof(float) * m);
  b.G = (double*)ar.take(sizeof(double) * mm);
  b.W64 = (double*)ar.take(sizeof(double) * mm);
  b.theta = (double*)ar.take(sizeof(double) * m);
  b.res = (double*)ar.take(sizeof(double) * m);
  b.summary = (double*)ar.take(sizeof(double) * 8);
  b.Cd = (double*)ar.take(sizeof(double) * nm);
  b.breakdown = (int*)ar.take(sizeof(int) * 4);
  b.part_bytes = rr_part_bytes(n, m);
  b.part = (float*)ar.take(b.part_bytes);
  if (!b.part) { set_error("rr: scratch too small"); return ATK_EINVAL; }
  const View qv{n, m, 1};
  // Shared-memory limit of the one-CTA eigensolver, set outside the captured
  // launch sequences.
  ATK_TRY(tridiag_eig_prepare());
  // The launch sequences between host reads, each a cached graph: setup (the
  // float32 copy of S, a random block, one power step, shifted CholeskyQR3),
  // one Rayleigh-Ritz step up to its summary, the power step from the Ritz
  // vectors, and a plain power step.
  const GraphKey kpre{{S, scratch, nullptr, nullptr, nullptr, nullptr, nullptr, (const void*)1},
                      {n, R, m, (int64_t)scratch_bytes}};
  ATK_TRY(run_graph(kpre, st, [&](cudaStream_t s2) -> int {
    ATK_CUDA(cudaMemsetAsync(b.breakdown, 0, sizeof(int), s2));
    ATK_TRY(f64_to_f32(S, b.Sf, n * n, s2));
    rand_fill_kernel<<<(unsigned)ceil_div((int64_t)nm, 256), 256, 0, s2>>>(b.Q, (int64_t)nm,
                                                                          0x5EEDULL + (uint64_t)n);
    ATK_LAUNCHED();
    ATK_TRY(sq_product(b.Sf, n, b.Q, m, b.Y, b, s2));  // Y = S Q
    shift_axpy_kernel<<<(unsigned)ceil_div((int64_t)nm, 256), 256, 0, s2>>>(b.Y, b.Q, b.Sf, n, (int64_t)nm,
                                                                          RR_POWER_SHIFT);  // Y = (S + sigma I) Q
    ATK_LAUNCHED();
    return cholqr3_f32(b.Y, b.T, b.Q, n, m, b, s2);
  }));
  const GraphKey kit{{scratch, dev_status, nullptr, nullptr, nullptr, nullptr, nullptr, (const void*)2},
                     {n, R, m, (int64_t)max_sweeps}};
  const GraphKey knext{{scratch, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, (const void*)3},
                       {n, R, m, (int64_t)scratch_bytes}};
  const GraphKey kpow{{scratch, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, (const void*)4},
                      {n, R, m, (int64_t)scratch_bytes}};
  int power = 0;
  double prev_pred = 0.0;
  int stalls = 0;
  for (;;) {
    // Rayleigh-Ritz: Z = S Q, B = Q^T Z = W diag(theta) W^T; Ritz vectors
    // Y = Q W (descending theta) and S Q W = Z W; residuals and summary.
    ATK_TRY(run_graph(kit, st, [&](cudaStream_t s2) -> int {
      ATK_TRY(sq_product(b.Sf, n, b.Q, m, b.Z, b, s2));
      ATK_TRY(cross_f32(b.Q, qv, b.Z, m, b.G, b.part, b.part_bytes, s2));
      ATK_TRY(tridiag_eig_f32(b.G, m, b.diag, b.Vb, s2));
      select_kernel<float><<<1, SEL_THREADS, 0, s2>>>(b.diag, 1, b.Vb, m, m, m, b.W64, b.theta, nullptr);
      ATK_LAUNCHED();
      ATK_TRY(f64_to_f32(b.W64, b.Wf, (int64_t)mm, s2));
      ATK_TRY(ttm_f32(b.Q, qv, b.Wf, m, b.Y, s2));
      ATK_TRY(ttm_f32(b.Z, qv, b.Wf, m, b.T, s2));
      ritz_residual_kernel<<<(unsigned)R, COL_THREADS, 0, s2>>>(b.T, b.Y, b.theta, n, b.res);
      ATK_LAUNCHED();
      ritz_summary_kernel<<<1, 32, 0, s2>>>(b.res, b.theta, (int)R, m, b.breakdown, b.summary);
      ATK_LAUNCHED();
      return ATK_OK;
    }));
    double h[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    ATK_CUDA(cudaMemcpyAsync(h, b.summary, sizeof(h), cudaMemcpyDeviceToHost, st));
    ATK_CUDA(cudaStreamSynchronize(st));
    const double res = h[0], thK = h[2], thm = fmax(h[3], 0.0);
    if (h[4] != 0.0) return ATK_ENOCONV;  // rank-deficient basis in float32: full Jacobi
    if (!(res == res) || !(thK == thK) || !(h[1] == h[1]) || res > 1e300) return ATK_ENOCONV;  // non-finite
    if (!(thK > 0.0)) return ATK_ENOCONV;
    const double rate = thm / thK;
    if (rate > RR_MAX_RATE) return ATK_ENOCONV;  // the cut sits in a cluster wider than the guard
    const double predicted = rate * res / (thK - thm);
    // Converged, or at the float32 floor: the residuals of float32 products
    // stop falling (a deflated level reaches eps_32 ||S|| long before 1e-6 of
    // its gap).  Below RR_FLOOR_OK the float64 refinement that follows removes
    // what is left; a stall above it is no convergence.
    const bool stalled = prev_pred > 0.0 && predicted > RR_STALL * prev_pred;
    // A deflation level accepts its float32 floor wherever it lies: its
    // vectors near the cut sit below that floor by construction, and
    // eig_top resolves them on the next level.  So does a level whose cut
    // float32 cannot resolve (a kept Ritz value below RR_RESOLVE eps_32
    // theta_1, or the guard block spread over less than RR_CUT_RESOLVE
    // theta_1): eig_top then continues on deflated levels.
    const bool floor_here = floor_ok || (int)h[5] < R || thK - thm < RR_CUT_RESOLVE * h[1];
    // (A block that lost its accuracy on the way shows as non-finite values
    // after the float64 refinement; eig_top then runs the full Jacobi.)
    const bool accept = stalled && (floor_here || predicted <= RR_FLOOR_OK);
    stalls = stalled && !accept ? stalls + 1 : 0;
    if (accept && predicted > RR_FLOOR_OK) *at_floor = true;
    if (stalls >= 3) return ATK_ENOCONV;  // three projections in a row without progress
    if (floor_here && power >= RR_MAX_POWER) *at_floor = true;
    // Converged outright, every kept Ritz value resolvable and a clear gap at
    // the cut: the light float64 finish suffices (refine_light).
    // (A guard Ritz value at or below zero makes `predicted` vanish whatever
    // the residual, so the residual itself must be small too.)
    *tight = !floor_ok && predicted <= RR_TARGET && (int)h[5] == R && h[2] - h[6] >= RR_LIGHT_GAP * h[1] &&
             res <= RR_LIGHT_RES * (thK - thm);
    *theta_cut = h[6];
    if (predicted <= RR_TARGET || accept || (floor_here && power >= RR_MAX_POWER)) {
      f32_to_f64_kernel2<<<(unsigned)ceil_div(n * m, 256), 256, 0, st>>>(b.Y, Qblk, n * (int64_t)m);
      ATK_LAUNCHED();
      return ATK_OK;
    }
    // Power steps to the predicted convergence (each multiplies the error by
    // about `rate`), at most RR_POWER_CHUNK before the next projection.
    int steps = 1;
    if (rate > 0.0 && predicted > 0.0)
      steps = (int)std::ceil(std::log(RR_TARGET / predicted) / std::log(rate));
    steps = std::max(1, std::min(steps, RR_POWER_CHUNK));
    if (floor_here) steps = std::min(steps, RR_MAX_POWER - power);  // ends at the cap, accepted above
    else if (power + steps > RR_MAX_POWER) return ATK_ENOCONV;
    power += steps;
    prev_pred = predicted;
    // First step from the Ritz vectors: S (Q W) = Z W is in T; its columns are
    // nearly orthogonal, so two plain CholeskyQR passes orthonormalise it.
    ATK_TRY(run_graph(knext, st, [&](cudaStream_t s2) -> int {
      // T = S Q W is in T and Q W in Y: T <- (S + sigma I) Q W.
      shift_axpy_kernel<<<(unsigned)ceil_div((int64_t)nm, 256), 256, 0, s2>>>(b.T, b.Y, b.Sf, n, (int64_t)nm,
                                                                            RR_POWER_SHIFT);
      ATK_LAUNCHED();
      ATK_TRY(cholqr_pass_f32(b.T, b.Y, n, m, 0.f, b, s2));
      return cholqr_pass_f32(b.Y, b.Q, n, m, 0.f, b, s2);
    }));
    // Further steps from Q: the block stays close to the Ritz vectors, so
    // S Q keeps nearly orthogonal columns and two passes still suffice.
    for (int k = 1; k < steps; ++k)
      ATK_TRY(run_graph(kpow, st, [&](cudaStream_t s2) -> int {
        ATK_TRY(sq_product(b.Sf, n, b.Q, m, b.T, b, s2));
        shift_axpy_kernel<<<(unsigned)ceil_div((int64_t)nm, 256), 256, 0, s2>>>(b.T, b.Q, b.Sf, n, (int64_t)nm,
                                                                              RR_POWER_SHIFT);
        ATK_LAUNCHED();
        ATK_TRY(cholqr_pass_f32(b.T, b.Y, n, m, 0.f, b, s2));
        return cholqr_pass_f32(b.Y, b.Q, n, m, 0.f, b, s2);
      }));
  }
}

// ----------------------------------------------------- float64 refinement
__global__ void normalize_cols_kernel(const double* __restrict__ Z, const double* U, int64_t n, int64_t R,
                                      const double* __restrict__ norms, const double* __restrict__ dots, double rel,
                                      double min_ratio, double* W);
__global__ void colnorms_f64_kernel(const double* __restrict__ Z, const double* __restrict__ U, int64_t n, int64_t R,
                                    double* __restrict__ norms, double* __restrict__ dots);
__global__ void sign_fix_kernel(double* __restrict__ U, int64_t n, int64_t R);

// W = I + X for the k x k symmetric float64 matrix B: for every pair p < q,
// the Jacobi rotation that zeroes b_pq in its own 2 x 2 problem, to first order
// (W_pq = s, W_qp = -s).  Pairs whose angle would be large (a nearly
// degenerate pair, |b_pq| > |b_pp - b_qq| / 10) are left alone, and so are
// pairs whose diagonal entries agree to 1e-7 relative (a degenerate cluster:
// there b_pq and b_pp - b_qq are both at the level of the input's float32
// errors squared, and the many rotations of up to 0.1 rad inside a large
// cluster would add up to a W that two polar steps cannot orthonormalise).
// Rotations inside a cluster do not change the subspaces this refinement
// serves; the Rayleigh quotients of its vectors stay within the cluster's
// width.
__global__ void simrot_kernel(const double* __restrict__ B, int64_t k, double* __restrict__ W) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= k * k) return;
  int64_t i = o % k, j = o / k;
  if (i == j) { W[o] = 1.0; return; }
  int64_t p = i < j ? i : j, q = i < j ? j : i;
  double bpp = B[p + k * p], bqq = B[q + k * q], bpq = B[p + k * q];
  double s = 0.0;
  const double gap = fabs(bqq - bpp);
  if (bpq != 0.0 && fabs(bpq) * 10.0 <= gap && gap >= 1e-7 * fmax(fabs(bpp), fabs(bqq))) {
    double tau = (bqq - bpp) / (2.0 * bpq);
    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    s = t / sqrt(1.0 + t * t);
  }
  // column p of the rotated basis gains -s * (old column q); column q gains +s * (old column p)
  W[o] = (i == p) ? s : -s;  // (row p, col q) = +s ; (row q, col p) = -s
}

// order[0..k) = indices of diag(B) sorted descending (NaN lowest, ties by
// index), lam[r] = B[order[r], order[r]] for r < R, disc = trace(S) - sum lam,
// and (nullable) lam_sorted[r] = B[order[r], order[r]] for every r < k.
// One CTA, k <= 1024.
__global__ void __launch_bounds__(256) order_diag_kernel(const double* __restrict__ B, int k, int R,
                                                         const double* __restrict__ S, int64_t n,
                                                         int* __restrict__ order, double* __restrict__ lam_out,
                                                         double* __restrict__ disc_out,
                                                         double* __restrict__ lam_sorted) {
  // Ranks by an integer key that orders like the float64 value (sign-folded
  // bit pattern; NaN lowest), so the k^2 comparisons stay off the float64
  // pipe; ties by index.
  __shared__ long long key[1024];
  __shared__ int ord[1024];
  __shared__ double wsum[8], lam_s[128];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double v = B[i + (int64_t)k * i];
    const long long b = __double_as_longlong(v);
    key[i] = isnan(v) ? LLONG_MIN : (b >= 0 ? b : (long long)((unsigned long long)b ^ 0x7fffffffffffffffULL));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const long long li = key[i];
    int rank = 0;
    for (int j = 0; j < k; ++j) rank += (key[j] > li) || (key[j] == li && j < i);
    ord[rank] = i;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    order[r] = ord[r];
    if (lam_sorted) lam_sorted[r] = B[ord[r] + (int64_t)k * ord[r]];
  }
  // trace(S): per-thread strided sums, then a fixed-order tree.
  double part = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) part += S[i + n * i];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) wsum[warp] = part;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double l = B[ord[r] + (int64_t)k * ord[r]];
    lam_s[r] = l;
    if (lam_out) lam_out[r] = l;
  }
  __syncthreads();
  if (warp == 0 && disc_out) {
    double kept = 0.0;
    for (int r = lane; r < R; r += 32) kept += lam_s[r];
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if (lane == 0) {
      double tr = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) tr += wsum[w];
      *disc_out = tr - kept;
    }
  }
}

// U[:, r] = QW[:, order[r]] for r < R (n x R float64).
__global__ void gather_cols_kernel(const double* __restrict__ QW, const int* __restrict__ order, int64_t n, int64_t R,
                                   double* __restrict__ U) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n * R) return;
  int64_t i = o % n, r = o / n;
  U[o] = QW[i + n * order[r]];
}

__global__ void identity_kernel(double* __restrict__ W, int64_t k) {
  int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o < k * k) W[o] = (o % k == o / k) ? 1.0 : 0.0;
}

constexpr int REFINE_ROTATION_STEPS = 2;

size_t refine_bytes(int64_t n, int64_t k) {
  return sizeof(double) * (size_t)(2 * n * k + 6 * k * k + 2 * k + 8) +
         sizeof(int) * (size_t)k + smallla_scratch_bytes(std::max(n, k), k) + 4096;
}

// Float64 refinement of an approximate leading block Qb (n x k, columns
// roughly the leading eigenvectors of S in descending order), then the kept
// R vectors.  Steps:
//  1. subspace_steps subspace-iteration steps, Qb <- orth(S Qb): normalise
//     the columns, then orthonormalise in Gram-Schmidt order.  Components
//     outside the leading k-space shrink by lambda_{k+1}/lambda_j per step.
//     The Ritz block of the float32 subspace iteration needs one step: its
//     float32 products leave about 1e-6 of each direction outside the
//     subspace, which adds up over R = 128 columns to a projector error above
//     1e-4.  A column whose image is below keep_rel times the largest image
//     (the numerical null space of S) or mostly leakage keeps its vector.
//     With no step, Qb is only orthonormalised (two polar steps).
//  2. Rayleigh-Ritz in float64: B = Qb^T S Qb.  The Ritz block is nearly
//     diagonal; REFINE_ROTATION_STEPS (2) simultaneous Jacobi steps (W from
//     simrot_kernel, orthonormalised by two polar steps, B <- W^T B W) take
//     the off-diagonal entries to float64 level.
//  3. U = (Qb W)[:, top R of diag(B)], one more polar step and the sign rule.
//     The kept eigenvalues are diag(B), the float64 Rayleigh quotients, and the
//     discarded energy is trace(S) minus their sum.
int refine_f64(const double* S, int64_t n, double* Qb, int64_t k, int64_t R, double* U64, double* lambda_out,
               double* discarded_out, double* lam_sorted, char* scratch, size_t scratch_bytes, cudaStream_t st,
               int subspace_steps, double keep_rel) {
  Arena ar{scratch, scratch_bytes, 0};
  double* Z = (double*)ar.take(sizeof(double) * n * k);
  double* QW = (double*)ar.take(sizeof(double) * n * k);
  double* B = (double*)ar.take(sizeof(double) * k * k);
  double* W = (double*)ar.take(sizeof(double) * k * k);
  double* Wt = (double*)ar.take(sizeof(double) * k * k);
  double* T = (double*)ar.take(sizeof(double) * k * k);
  double* T2 = (double*)ar.take(sizeof(double) * k * k);
  float* Tf = (float*)ar.take(sizeof(float) * k * k);
  double* norms = (double*)ar.take(sizeof(double) * (2 * k + 8));
  int* order = (int*)ar.take(sizeof(int) * k);
  double* pol = (double*)ar.take(smallla_scratch_bytes(std::max(n, k), k));
  if (!pol) { set_error("eig: scratch too small for the refinement"); return ATK_EINVAL; }
  const unsigned gk = (unsigned)ceil_div(k * k, 256);
  // 1. subspace steps (none: only orthonormalise Qb)
  for (int step = 0; step < subspace_steps; ++step) {
    ATK_TRY(gemm_f64(S, Qb, n, n, k, Z, st));
    colnorms_f64_kernel<<<(unsigned)k, COL_THREADS, 0, st>>>(Z, Qb, n, k, norms, norms + k);
    ATK_LAUNCHED();
    normalize_cols_kernel<<<(unsigned)k, COL_THREADS, 0, st>>>(Z, Qb, n, k, norms, norms + k, keep_rel,
                                                                          0.9, Qb);
    ATK_LAUNCHED();
    // Orthonormalise in Gram-Schmidt order (column j against the columns
    // before it; Qb is sorted by descending Ritz value).  The subspace step
    // multiplies the float32 leakage of a trailing, small-eigenvalue column
    // into the leading subspace by lambda_1 / lambda_j (overlaps up to about
    // 0.1); a symmetric orthonormalisation (the polar factor) would rotate
    // that leakage back into the leading columns, Gram-Schmidt order leaves
    // their span alone.  One CholeskyQR pass with a float32 factor (robust for
    // any such overlap) takes the columns to float32 orthogonality, then two
    // Gram-Schmidt-ordered quadratic steps to float64 level.
    // k <= 156 here (k = m <= 156 on the subspace path, k = R <= 128 after
    // the full Jacobi), within the one-CTA factor's limit of 160.
    ATK_TRY(gemm_tn_f64(Qb, Qb, n, k, B, st));
    ATK_TRY(cholinv_f32(B, (int)k, 0.f, Tf, nullptr, st));
    ATK_TRY(f32_to_f64(Tf, T, k * k, st));
    ATK_TRY(gemm_f64(Qb, T, n, k, k, Z, st));
    ATK_CUDA(cudaMemcpyAsync(Qb, Z, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, st));
    for (int it = 0; it < 2; ++it) ATK_TRY(gs_step_f64(Qb, n, k, pol, st));
  }
  if (subspace_steps == 0) {
    ATK_TRY(polar_step_f64(Qb, n, k, pol, st));
    ATK_TRY(polar_step_f64(Qb, n, k, pol, st));
  }
  // 2. Rayleigh-Ritz and simultaneous rotations
  ATK_TRY(gemm_f64(S, Qb, n, n, k, Z, st));
  ATK_TRY(gemm_tn_f64(Qb, Z, n, k, B, st));
  identity_kernel<<<gk, 256, 0, st>>>(Wt, k);
  ATK_LAUNCHED();
  for (int step = 0; step < REFINE_ROTATION_STEPS && k > 1; ++step) {
    simrot_kernel<<<gk, 256, 0, st>>>(B, k, W);
    ATK_LAUNCHED();
    ATK_TRY(polar_step_f64(W, k, k, pol, st));
    ATK_TRY(polar_step_f64(W, k, k, pol, st));
    ATK_TRY(gemm_f64(B, W, k, k, k, T, st));
    ATK_TRY(gemm_tn_f64(W, T, k, k, B, st));
    ATK_TRY(gemm_f64(Wt, W, k, k, k, T2, st));
    std::swap(Wt, T2);
  }
  // 3. kept vectors
  order_diag_kernel<<<1, 256, 0, st>>>(B, (int)k, (int)R, S, n, order, lambda_out, discarded_out, lam_sorted);
  ATK_LAUNCHED();
  ATK_TRY(gemm_f64(Qb, Wt, n, k, k, QW, st));
  gather_cols_kernel<<<(unsigned)ceil_div(n * R, 256), 256, 0, st>>>(QW, order, n, R, U64);
  ATK_LAUNCHED();
  ATK_TRY(polar_step_f64(U64, n, R, pol, st));
  sign_fix_kernel<<<(unsigned)R, COL_THREADS, 0, st>>>(U64, n, R);
  ATK_LAUNCHED();
  return ATK_OK;
}

// B = diag(d_j / q_j^2): the Rayleigh quotients u^T S u / u^T u from
// d_j = u_j^T S u_j and q_j = ||u_j||.
__global__ void rq_diag_kernel(const double* __restrict__ d, const double* __restrict__ q, int64_t k,
                               double* __restrict__ B) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= k * k) return;
  const int64_t i = o % k;
  B[o] = (i == o / k) ? d[i] / (q[i] * q[i]) : 0.0;
}

// Light float64 finish of a Ritz block that the float32 iteration has
// converged outright with a clear gap at the cut (rr_top's `tight`: its
// predicted error after one float64 subspace step is below RR_TARGET and its
// kept residuals are below RR_LIGHT_RES of the gap to the guard block, so
// each float32 vector is within about 1e-4 of the leading space).
//  1. Z = S Qb in float64.  q_j^T z_j / q_j^T q_j are the columns' Rayleigh
//     quotients, exact to second order in the vectors' error (below 1e-8
//     relative): they rank the columns and give the kept eigenvalues and the
//     discarded energy.
//  2. The subspace step Qb <- normalise(Z), then the orthonormalisation in
//     Gram-Schmidt order: a CholeskyQR pass with a float32 factor (the float32
//     block is not orthonormal beyond float32 level, and may be far from it
//     when S spans many decades), then one quadratic step, which takes the
//     float32-level error of that pass to float64 level.
//  3. The top R columns, the sign rule.
// Without the Rayleigh-Ritz rotations a column inside a cluster of kept
// eigenvalues is accurate to the float32 level of the iteration, the level
// the float32 Gram already sets; the kept subspace is accurate to float64
// level.
int refine_light(const double* S, int64_t n, double* Qb, int64_t k, int64_t R, double* U64, double* lambda_out,
                 double* discarded_out, double* lam_sorted, char* scratch, size_t scratch_bytes, cudaStream_t st) {
  Arena ar{scratch, scratch_bytes, 0};
  double* Z = (double*)ar.take(sizeof(double) * n * k);
  double* B = (double*)ar.take(sizeof(double) * k * k);
  double* T = (double*)ar.take(sizeof(double) * k * k);
  float* Tf = (float*)ar.take(sizeof(float) * k * k);
  double* norms = (double*)ar.take(sizeof(double) * (2 * k + 8));
  double* qn = (double*)ar.take(sizeof(double) * (k + 8));
  int* order = (int*)ar.take(sizeof(int) * k);
  double* pol = (double*)ar.take(smallla_scratch_bytes(std::max(n, k), k));
  if (!pol) { set_error("eig: scratch too small for the refinement"); return ATK_EINVAL; }
  // 1. Z = S Qb and the Rayleigh quotients of the float32 columns
  ATK_TRY(gemm_f64(S, Qb, n, n, k, Z, st));
  colnorms_f64_kernel<<<(unsigned)k, COL_THREADS, 0, st>>>(Z, Qb, n, k, norms, norms + k);
  ATK_LAUNCHED();
  colnorms_f64_kernel<<<(unsigned)k, COL_THREADS, 0, st>>>(Qb, nullptr, n, k, qn, nullptr);
  ATK_LAUNCHED();
  rq_diag_kernel<<<(unsigned)ceil_div(k * k, 256), 256, 0, st>>>(norms + k, qn, k, B);
  ATK_LAUNCHED();
  // 2. subspace step and orthonormalisation in Gram-Schmidt order
  normalize_cols_kernel<<<(unsigned)k, COL_THREADS, 0, st>>>(Z, Qb, n, k, norms, norms + k, 1e-5, 0.9,
                                                                        Qb);
  ATK_LAUNCHED();
  ATK_TRY(gemm_tn_f64(Qb, Qb, n, k, T, st));
  ATK_TRY(cholinv_f32(T, (int)k, 0.f, Tf, nullptr, st));
  ATK_TRY(f32_to_f64(Tf, T, k * k, st));
  ATK_TRY(gemm_f64(Qb, T, n, k, k, Z, st));
  ATK_CUDA(cudaMemcpyAsync(Qb, Z, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, st));
  ATK_TRY(gs_step_f64(Qb, n, k, pol, st));
  // 3. kept vectors
  order_diag_kernel<<<1, 256, 0, st>>>(B, (int)k, (int)R, S, n, order, lambda_out, discarded_out, lam_sorted);
  ATK_LAUNCHED();
  gather_cols_kernel<<<(unsigned)ceil_div(n * R, 256), 256, 0, st>>>(Qb, order, n, R, U64);
  ATK_LAUNCHED();
  sign_fix_kernel<<<(unsigned)R, COL_THREADS, 0, st>>>(U64, n, R);
  ATK_LAUNCHED();
  return ATK_OK;
}

// Scratch of one level (eig_level): the Ritz block, then the largest of the
// solvers' and the refinement's needs.
static size_t level_scratch_bytes(int64_t n, int arith) {
  size_t jac = n > JACOBI_MAX_N ? 0 : arith == ATK_EIG_ROT_FP64 ? eig_bytes_t<double>(n) : eig_bytes_t<float>(n);
  size_t rr = rr_bytes(n, 156);
  const int64_t kmax = std::min<int64_t>(n, 156);
  // the Ritz block is carved first and outlives the solver that fills it
  return (size_t)n * kmax * 8 + 512 + std::max(std::max(jac, rr), refine_bytes(n, kmax));
}

size_t eig_scratch_bytes(int64_t n, int arith) {
  // sorted Rayleigh quotients, the combined and the per-level vector blocks
  // and the two deflation products (n x 128 each), U^T S U (128 x 128) and
  // the deflated matrix (n x n), then one level's scratch
  return 8 * (size_t)(160 + 4 * n * std::min<int64_t>(n, 128) + 128 * 128 + n * n) + 8 * 256 +
         level_scratch_bytes(n, arith);
}

// norms[r] = ||Z[:, r]||; one warp per column.
// norms[r] = ||Z[:, r]|| and, when U is given, dots[r] = U[:, r]^T Z[:, r].
// One warp per column.
__global__ void colnorms_f64_kernel(const double* __restrict__ Z, const double* __restrict__ U, int64_t n, int64_t R,
                                    double* __restrict__ norms, double* __restrict__ dots) {
  __shared__ double sh[COL_WARPS];
  const int64_t j = blockIdx.x;
  const double* z = Z + j * n;
  const double* u = U ? U + j * n : nullptr;
  double s = 0.0, d = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) {
    s += z[i] * z[i];
    if (u) d += u[i] * z[i];
  }
  s = col_sum(s, sh);
  if (u) d = col_sum(d, sh);
  if (threadIdx.x == 0) {
    norms[j] = sqrt(s);
    if (dots) dots[j] = d;
  }
}

// W[:, r] = Z[:, r] / ||Z[:, r]|| when that norm is above rel * max_r ||Z[:, r]||
// and (dots given) the Rayleigh quotient U[:, r]^T Z[:, r] is at least
// min_ratio ||Z[:, r]||, else U[:, r].  Z = S U.  A column whose image is at
// rounding level lies in the numerical null space, and a column whose image is
// mostly leakage into other eigendirections (||S u|| well above u^T S u: a
// null-space or small-eigenvalue Ritz vector with float32 errors along the
// leading directions) is not improved by S u; normalising would turn that
// leakage into a near copy of a leading direction.  Such columns keep their
// vectors.  One CTA per column; W may be U (each element is read and then
// written by the same thread).
__global__ void normalize_cols_kernel(const double* __restrict__ Z, const double* U, int64_t n, int64_t R,
                                      const double* __restrict__ norms, const double* __restrict__ dots, double rel,
                                      double min_ratio, double* W) {
  __shared__ double sh[COL_WARPS];
  const int64_t j = blockIdx.x;
  double mx = 0.0;
  for (int64_t r = threadIdx.x; r < R; r += COL_THREADS) mx = fmax(mx, norms[r]);
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x % 32 == 0) sh[threadIdx.x / 32] = mx;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < COL_WARPS; ++w) mx = fmax(mx, sh[w]);
  const double thr = rel * mx;
  const double* z = Z + j * n;
  const double nz = norms[j];
  double* w = W + j * n;
  if (nz > thr && (!dots || dots[j] >= min_ratio * nz)) {
    const double inv = 1.0 / nz;
    for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) w[i] = z[i] * inv;
  } else {
    const double* u = U + j * n;
    for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) w[i] = u[i];
  }
}

// Sign rule: flip each column so that its largest-magnitude entry is positive
// (ties: lowest row).  One CTA per column.
__global__ void sign_fix_kernel(double* __restrict__ U, int64_t n, int64_t R) {
  __shared__ double sbest[COL_WARPS];
  __shared__ int64_t sarg[COL_WARPS];
  double* u = U + (int64_t)blockIdx.x * n;
  double best = -1.0;
  int64_t arg = 0;
  for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) {
    const double a = fabs(u[i]);
    if (a > best) { best = a; arg = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
    if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
  }
  if (threadIdx.x % 32 == 0) { sbest[threadIdx.x / 32] = best; sarg[threadIdx.x / 32] = arg; }
  __syncthreads();
#pragma unroll
  for (int w = 0; w < COL_WARPS; ++w)
    if (sbest[w] > best || (sbest[w] == best && sarg[w] < arg)) { best = sbest[w]; arg = sarg[w]; }
  const bool neg = u[arg] < 0.0;
  __syncthreads();  // every thread has read u[arg] before any flips it
  if (neg)
    for (int64_t i = threadIdx.x; i < n; i += COL_THREADS) u[i] = -u[i];
}

// One level of the eigensolver: the R leading eigenvectors of the symmetric
// S by the subspace path or the full Jacobi, then the float64 refinement of
// the leading block of k = rr_width(n, R, wide) vectors (R of them plus the
// guard vectors, which make the gap at the cut visible).  Writes U64 (n x R,
// descending Rayleigh quotients), lambda_out / discarded_out as
// atucker_eig documents (nullable), lam_sorted[0..k) the sorted float64
// Rayleigh quotients of the whole block.  The refined block stays in the
// level's scratch for further steps: lv->Qb (n x k) and the scratch after it.
struct Level {
  double* Qb;
  int64_t k;
  char* rest;
  size_t rest_bytes;
  bool at_floor;  // the subspace iteration stopped at its float32 floor
  bool tight;     // converged with a clear gap at the cut: the light finish ran
};
static int eig_level(const double* S, int64_t n, int64_t R, int arith, int method, int max_sweeps, bool wide,
                     double* U64, double* lambda_out, double* discarded_out, double* lam_sorted, int* dev_status,
                     char* scratch, size_t scratch_bytes, cudaStream_t st, Level* lv) {
  const int m = rr_width(n, R, wide);
  const bool rr = arith == ATK_EIG_ROT_FP32 && m >= R + 8 &&
                  ((method == ATK_EIG_AUTO && 2 * m <= n) || (method == ATK_EIG_SUBSPACE && m < n));
  Arena ar{scratch, scratch_bytes, 0};
  const int64_t k = m;  // both paths refine the leading m vectors
  double* Qb = (double*)ar.take(sizeof(double) * n * k);
  if (!Qb) { set_error("eig: scratch too small"); return ATK_EINVAL; }
  char* rest = scratch + ar.used;
  const size_t rest_bytes = scratch_bytes - ar.used;
  *lv = Level{Qb, k, rest, rest_bytes, false, false};
  double theta_cut = 0.0;  // float32 Ritz value R + 1 (rr_top)
  int s = ATK_ENOCONV;
  if (rr) {
    s = rr_top(S, n, R, m, max_sweeps, Qb, dev_status, rest, rest_bytes, st, wide, &lv->at_floor, &lv->tight,
               &theta_cut);
    if (s != ATK_OK && s != ATK_ENOCONV) return s;
    if (s == ATK_OK && lambda_out && n > R) {
      // Only the kept eigenvalues exist on this path; the tail is marked NaN.
      ATK_CUDA(cudaMemsetAsync(lambda_out + R, 0xFF, sizeof(double) * (n - R), st));
    }
  }
  if (s != ATK_OK && n > JACOBI_MAX_N) {
    set_error(rr ? "eig: the subspace eigensolver did not converge and I_n > 1024 has no full-Jacobi fallback"
                 : "eig: I_n > 1024 needs the subspace eigensolver (float32 rotations, R + p <= I_n / 2)");
    return rr ? ATK_ENOCONV : ATK_EUNSUPPORTED;
  }
  if (s != ATK_OK) {
    // Full Jacobi: the k leading vectors (and all eigenvalues) of the whole matrix.
    s = arith == ATK_EIG_ROT_FP64
            ? eig_top_t<double>(S, n, k, max_sweeps, Qb, lambda_out, nullptr, dev_status, rest, rest_bytes, st)
            : eig_top_t<float>(S, n, k, max_sweeps, Qb, lambda_out, nullptr, dev_status, rest, rest_bytes, st);
    if (s != ATK_OK) return s;
  }
  // The refinement: no host synchronisation inside, so one cached graph per
  // (buffers, sizes, form).
  // The light finish refines the R kept columns only: both of its
  // orthonormalisations build column j from columns <= j, so the guard
  // columns do not enter the kept ones, and with the gap its gate demands no
  // guard can overtake a kept column in the ordering.  The value past the cut
  // that eig_top's gap test reads is the float32 Ritz value theta_R (the gate
  // puts the gap at >= RR_LIGHT_GAP theta_1, far above that value's error).
  if (s == ATK_OK && rr && lv->tight) {
    if (lam_sorted) ATK_CUDA(cudaMemcpyAsync(lam_sorted + R, &theta_cut, sizeof(double), cudaMemcpyHostToDevice, st));
    const GraphKey lkey{{S, Qb, U64, lambda_out, discarded_out, lam_sorted, rest, (const void*)5},
                        {n, R, R, (int64_t)rest_bytes}};
    return run_graph(lkey, st, [&](cudaStream_t s2) -> int {
      return refine_light(S, n, Qb, R, R, U64, lambda_out, discarded_out, lam_sorted, rest, rest_bytes, s2);
    });
  }
  lv->tight = false;
  const GraphKey key{{S, Qb, U64, lambda_out, discarded_out, lam_sorted, rest, nullptr},
                     {n, k, R, (int64_t)rest_bytes}};
  return run_graph(key, st, [&](cudaStream_t s2) -> int {
    return refine_f64(S, n, Qb, k, R, U64, lambda_out, discarded_out, lam_sorted, rest, rest_bytes, s2, 1, 1e-5);
  });
}

// Projected deflation S_out = P S_in P with P = I - U U^T (U n x h, orthonormal):
// S_in - U W^T - W U^T + (V U^T + U V^T) / 2 with W = S_in U and V = U (U^T W),
// over the upper triangle, mirrored.  Its error from an inexact U is second
// order in the error of U (a direct S - U diag(lambda) U^T is first order).
// Thread (i, j), i <= j, reads S_in(i, j) only and writes (i, j) and (j, i),
// so S_out may be S_in.
__global__ void deflate_kernel(const double* S_in, const double* __restrict__ U, const double* __restrict__ W,
                               const double* __restrict__ V, int64_t n, int64_t h, double* S_out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx % n, j = idx / n;
  if (i > j) return;
  double v = S_in[i + n * j];
  for (int64_t t = 0; t < h; ++t) {
    const int64_t ci = i + n * t, cj = j + n * t;
    v -= U[ci] * W[cj] + W[ci] * U[cj] - 0.5 * (V[ci] * U[cj] + U[ci] * V[cj]);
  }
  S_out[i + n * j] = v;
  S_out[j + n * i] = v;
}

// Floating-point resolution of a level, in units of eps_32 times the level's
// largest eigenvalue: the float32 products and rotations of a level resolve
// eigenvalue differences down to about eps_32 lambda_1 of the matrix they
// work on, and the float64 refinement's first-order rotations need a margin
// above that.
constexpr double LEVEL_RESOLVE = 64.0 * 1.1920928955078125e-7;
// A Gram computed with float32 sums errs by up to about eps_32 lambda_1 where
// its energy sits in few entries, which turns the kept subspace by about
// eps_32 lambda_1 / gap per direction; the projector distance stays within
// 1e-4 only while gap >= GRAM_PROJ_RESOLVE sqrt(2 R) lambda_1.
constexpr double GRAM_PROJ_RESOLVE = 1e4 * 1.1920928955078125e-7;
constexpr int MAX_LEVELS = 4;
// Float64 subspace steps on a level's block before its leading vectors are
// deflated (each shrinks their components outside the block by
// lambda_{k+1} / lambda_j), and the image floor of those steps: the float64
// rounding level of the products rather than the float32 level of the Gram.
constexpr int DEFLATE_STEPS = 3;
constexpr double DEFLATE_KEEP_REL = 1e-10;

// Leading-R eigenvectors (Alg. 2, EIG branch).  U64_out (n x R float64) is the
// orthonormalised basis; U_out its float32 copy.
//
// Deflation levels (float32 rotations).  Level 0 solves S.  When the gap at
// the cut, lambda_R - lambda_{R+1} (float64 Rayleigh quotients of the refined
// block), is below LEVEL_RESOLVE lambda_1, float32 arithmetic on S cannot
// resolve the cut: the split between the vectors on either side of it is
// decided by rounding (a spectrum that decays like k^-3 reaches that at
// R = 64 for a 256^3 tensor).  The level's block then takes DEFLATE_STEPS
// more float64 subspace steps; its leading vectors whose eigenvalues lie
// LEVEL_RESOLVE lambda_1 or more above the cut are resolved and final.  They
// are deflated in float64, S_1 = P S P with P = I - U_h U_h^T, and the
// remaining R - h vectors are the leading ones of S_1, whose largest
// eigenvalue is about lambda_{h+1}, so the same float32 arithmetic resolves
// the cut some lambda_1 / lambda_{h+1} times finer.  Each level repeats this
// test.  The kept vectors of all levels are then refined together on S
// (orthonormalisation, Rayleigh-Ritz, simultaneous rotations), which also
// gives the kept eigenvalues and the discarded energy.  With float64
// rotations the cut is resolved at level 0.
int eig_top(const double* S, int64_t n, int64_t R, int arith, int method, int max_sweeps, float* U_out,
            double* U64_out, double* lambda_out, double* discarded_out, int* dev_status, char* scratch,
            size_t scratch_bytes, cudaStream_t st, int* unresolved) {
  if (n <= 0 || R <= 0 || R > n || n > EIG_MAX_N) {
    set_error("eig: need 1 <= R <= n <= 32768");
    return ATK_EUNSUPPORTED;
  }
  if (unresolved) *unresolved = 0;
  Arena ar{scratch, scratch_bytes, 0};
  double* lam_s = (double*)ar.take(sizeof(double) * 160);
  double* Ufin = (double*)ar.take(sizeof(double) * n * R);
  double* Ulev = (double*)ar.take(sizeof(double) * n * R);
  double* W = (double*)ar.take(sizeof(double) * n * R);
  double* V = (double*)ar.take(sizeof(double) * n * R);
  double* M = (double*)ar.take(sizeof(double) * R * R);
  double* SL = (double*)ar.take(sizeof(double) * n * n);
  if (!SL) { set_error("eig: scratch too small"); return ATK_EINVAL; }
  char* rest = scratch + ar.used;
  const size_t rest_bytes = scratch_bytes - ar.used;
  Level lv{};
  ATK_TRY(eig_level(S, n, R, arith, method, max_sweeps, false, U64_out, lambda_out, discarded_out, lam_s, dev_status,
                    rest, rest_bytes, st, &lv));
  if (arith == ATK_EIG_ROT_FP32 && lv.k > R) {
    double h[161];
    auto read_lam = [&](int64_t count) -> int {
      ATK_CUDA(cudaMemcpyAsync(h, lam_s, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
      ATK_CUDA(cudaStreamSynchronize(st));
      return ATK_OK;
    };
    ATK_TRY(read_lam(R + 1));
    if (!std::isfinite(h[0]) || !std::isfinite(h[R - 1]) || !std::isfinite(h[R])) {
      // A level-0 block that lost its accuracy: the full Jacobi instead.
      if (n > JACOBI_MAX_N) { set_error("eig: non-finite Ritz values"); return ATK_ENOCONV; }
      ATK_TRY(eig_level(S, n, R, arith, ATK_EIG_FULL_JACOBI, max_sweeps, false, U64_out, lambda_out, discarded_out,
                        lam_s, dev_status, rest, rest_bytes, st, &lv));
      ATK_TRY(read_lam(R + 1));
    }
    const double gap0 = h[R - 1] - h[R];
    if (unresolved && gap0 < std::max(LEVEL_RESOLVE, GRAM_PROJ_RESOLVE * sqrt(2.0 * R)) * fabs(h[0])) {
      *unresolved = 1;
      return ATK_OK;
    }
    if (gap0 < LEVEL_RESOLVE * fabs(h[0]) || lv.at_floor) {
      // The cut is not resolved at level 0 (or level 0 stopped at its
      // float32 floor): deflation levels, which start with float64 steps.
      const double* src = S;
      int64_t done = 0, RL = R;
      for (int level = 1;; ++level) {
        // More float64 steps on this level's block, so that the vectors to be
        // deflated are accurate to float64 level.
        ATK_TRY(refine_f64(src, n, lv.Qb, lv.k, RL, Ulev, nullptr, nullptr, lam_s, lv.rest, lv.rest_bytes, st,
                           DEFLATE_STEPS, DEFLATE_KEEP_REL));
        ATK_TRY(read_lam(RL + 1));
        const double delta = LEVEL_RESOLVE * fabs(h[0]);
        if (level >= MAX_LEVELS || h[RL - 1] - h[RL] >= delta) break;  // resolved at this level
        int64_t hd = 0;
        while (hd < RL && h[hd] >= h[RL - 1] + delta) ++hd;
        if (hd == 0) break;  // nothing to deflate: the kept vectors all sit at the cut
        ATK_CUDA(cudaMemcpyAsync(Ufin + n * done, Ulev, sizeof(double) * n * hd, cudaMemcpyDeviceToDevice, st));
        ATK_TRY(gemm_f64(src, Ulev, n, n, hd, W, st));          // W = S_L U_h
        ATK_TRY(gemm_tn_f64(Ulev, W, n, hd, M, st));            // M = U_h^T W
        ATK_TRY(gemm_f64(Ulev, M, n, hd, hd, V, st));           // V = U_h M
        deflate_kernel<<<(unsigned)ceil_div(n * n, 256), 256, 0, st>>>(src, Ulev, W, V, n, hd, SL);
        ATK_LAUNCHED();
        src = SL;
        done += hd;
        RL -= hd;
        ATK_TRY(eig_level(SL, n, RL, arith, method, max_sweeps, true, Ulev, nullptr, nullptr, lam_s, dev_status,
                          rest, rest_bytes, st, &lv));
        if (lv.k <= RL) break;
        ATK_TRY(read_lam(RL + 1));
        if (h[RL - 1] - h[RL] >= LEVEL_RESOLVE * fabs(h[0])) break;  // resolved without more steps
      }
      ATK_CUDA(cudaMemcpyAsync(Ufin + n * done, Ulev, sizeof(double) * n * RL, cudaMemcpyDeviceToDevice, st));
      // The kept vectors of every level, refined together on S.
      ATK_TRY(refine_f64(S, n, Ufin, R, R, U64_out, lambda_out, discarded_out, nullptr, rest, rest_bytes, st, 0,
                         0.0));
      if (lambda_out && n > R) ATK_CUDA(cudaMemsetAsync(lambda_out + R, 0xFF, sizeof(double) * (n - R), st));
    }
  }
  if (U_out) ATK_TRY(f64_to_f32(U64_out, U_out, n * R, st));
  return ATK_OK;
}

}  // namespace atk
