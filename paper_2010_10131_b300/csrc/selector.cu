// Learned per-mode selector (the paper's adaptive solver selection, Sec. IV):
// features of each mode (Table I plus the mode's position and the remaining
// tensor size), host inference of a 12 -> 64 -> 64 -> K ReLU network, and the
// CUDA kernels that train it on the GPU (forward, masked squared loss,
// backward, Adam).  The network replaces the paper's decision tree; its
// outputs predict log2 of each class's time relative to the fastest class.
//
// Training kernels are plain one-thread-per-output loops: the network has
// about 5,300 parameters and the data set a few thousand rows, so every
// launch is latency-bound; sums over the batch run in a fixed order, so a
// training run is deterministic.
#include <cmath>
#include <mutex>
#include <vector>

#include "atk_internal.cuh"

namespace atk {
namespace sel {

// The active selector is the MLP (kind 0) or the decision tree (kind 1),
// whichever was loaded last.
struct Tree {
  std::vector<int> feature, left, right, cls;
  std::vector<double> threshold;
};
struct State {
  std::mutex mu;
  bool loaded = false;
  int kind = 0;
  float fmean[ATK_SELECTOR_FEATURES], fscale[ATK_SELECTOR_FEATURES];
  std::vector<float> params;
  Tree tree;
};
}  // namespace sel
bool selector_class_fits(int k, double lg);
namespace sel {
// Whether a class can run a mode of log2 size lg: the full-Jacobi classes
// need I_n <= 1024, the other EIG classes I_n <= 32768 (feature 0 is log2 I_n).
bool class_fits(int k, double lg) {
  if (k == ATK_CLASS_ALS) return true;
  const bool jac = k == ATK_CLASS_EIG_JACOBI || k == ATK_CLASS_EIG_JACOBI_SMALL;
  return lg <= (jac ? 10.0 : 15.0) + 1e-9;
}

}  // namespace sel
bool selector_class_fits(int k, double lg) { return sel::class_fits(k, lg); }
namespace sel {

State& state() {
  static State s;
  return s;
}

int64_t param_count(int in, int hidden, int out) {
  return (int64_t)hidden * in + hidden + (int64_t)hidden * hidden + hidden + (int64_t)out * hidden + out;
}

// ---------------------------------------------------------------- kernels
// out[b][j] = sum_i W[j][i] x[b][i] + bias[j]; z (nullable) keeps the
// pre-activation, a = relu(z) when relu, else z.
__global__ void dense_fwd_kernel(const float* __restrict__ X, int B, int in, const float* __restrict__ W,
                                 const float* __restrict__ bias, int out, int relu, float* __restrict__ Z,
                                 float* __restrict__ A) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * out) return;
  const int b = (int)(idx / out), j = (int)(idx % out);
  float s = bias[j];
  for (int i = 0; i < in; ++i) s = fmaf(W[(int64_t)j * in + i], X[(int64_t)b * in + i], s);
  if (Z) Z[idx] = s;
  A[idx] = relu ? fmaxf(s, 0.f) : s;
}

// Masked squared loss: G = 2 (P - Y) M / cnt, loss = sum M (P - Y)^2 / cnt,
// cnt = sum M (1 if zero).  One CTA, fixed-order tree reduction.
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ P, const float* __restrict__ Y,
                                                   const float* __restrict__ M, int64_t count,
                                                   float* __restrict__ G, float* __restrict__ loss) {
  __shared__ float red[256], cred[256];
  float s = 0.f, c = 0.f;
  for (int64_t i = threadIdx.x; i < count; i += 256) {
    const float d = P[i] - Y[i];
    s = fmaf(M[i] * d, d, s);
    c += M[i];
  }
  red[threadIdx.x] = s;
  cred[threadIdx.x] = c;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      red[threadIdx.x] += red[threadIdx.x + k];
      cred[threadIdx.x] += cred[threadIdx.x + k];
    }
    __syncthreads();
  }
  const float cnt = cred[0] > 0.f ? cred[0] : 1.f;
  for (int64_t i = threadIdx.x; i < count; i += 256) G[i] = 2.f * (P[i] - Y[i]) * M[i] / cnt;
  if (threadIdx.x == 0 && loss) *loss = red[0] / cnt;
}

// Gin[b][i] = (sum_o G[b][o] W[o][i]) * (Zin[b][i] > 0): the gradient through a
// dense layer and the ReLU of its input.
__global__ void dense_bwd_input_kernel(const float* __restrict__ G, int B, int out, const float* __restrict__ W,
                                       int in, const float* __restrict__ Zin, float* __restrict__ Gin) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)B * in) return;
  const int b = (int)(idx / in), i = (int)(idx % in);
  float s = 0.f;
  for (int o = 0; o < out; ++o) s = fmaf(G[(int64_t)b * out + o], W[(int64_t)o * in + i], s);
  Gin[idx] = Zin[idx] > 0.f ? s : 0.f;
}

// dW[o][i] = sum_b G[b][o] A[b][i] (i < in), db[o] = sum_b G[b][o] (i == in).
__global__ void dense_bwd_weight_kernel(const float* __restrict__ G, const float* __restrict__ A, int B, int in,
                                        int out, float* __restrict__ dW, float* __restrict__ db) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)out * (in + 1)) return;
  const int o = (int)(idx / (in + 1)), i = (int)(idx % (in + 1));
  float s = 0.f;
  if (i < in) {
    for (int b = 0; b < B; ++b) s = fmaf(G[(int64_t)b * out + o], A[(int64_t)b * in + i], s);
    dW[(int64_t)o * in + i] = s;
  } else {
    for (int b = 0; b < B; ++b) s += G[(int64_t)b * out + o];
    db[o] = s;
  }
}

// Adam (Kingma & Ba 2015), bias-corrected, step t (1-based).
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

unsigned blocks(int64_t n) { return (unsigned)ceil_div(std::max<int64_t>(n, 1), 256); }

struct Layers {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};
Layers layers(const float* p, int in, int h, int out) {
  Layers L;
  L.W1 = p;
  L.b1 = L.W1 + (int64_t)h * in;
  L.W2 = L.b1 + h;
  L.b2 = L.W2 + (int64_t)h * h;
  L.W3 = L.b2 + h;
  L.b3 = L.W3 + (int64_t)out * h;
  return L;
}

struct Acts {
  float *z1, *a1, *z2, *a2, *o, *g3, *g2, *g1;
};

int forward(const float* X, int B, int in, int h, int out, const float* params, Acts& a, cudaStream_t st) {
  Layers L = layers(params, in, h, out);
  dense_fwd_kernel<<<blocks((int64_t)B * h), 256, 0, st>>>(X, B, in, L.W1, L.b1, h, 1, a.z1, a.a1);
  ATK_LAUNCHED();
  dense_fwd_kernel<<<blocks((int64_t)B * h), 256, 0, st>>>(a.a1, B, h, L.W2, L.b2, h, 1, a.z2, a.a2);
  ATK_LAUNCHED();
  dense_fwd_kernel<<<blocks((int64_t)B * out), 256, 0, st>>>(a.a2, B, h, L.W3, L.b3, out, 0, nullptr, a.o);
  ATK_LAUNCHED();
  return ATK_OK;
}

int loss_grad(const float* X, const float* Y, const float* M, int B, int in, int h, int out, const float* params,
              float* loss, float* grad, Acts& a, cudaStream_t st) {
  ATK_TRY(forward(X, B, in, h, out, params, a, st));
  loss_kernel<<<1, 256, 0, st>>>(a.o, Y, M, (int64_t)B * out, a.g3, loss);
  ATK_LAUNCHED();
  Layers L = layers(params, in, h, out);
  Layers D = layers(grad, in, h, out);
  float* dW1 = const_cast<float*>(D.W1);
  float* db1 = const_cast<float*>(D.b1);
  float* dW2 = const_cast<float*>(D.W2);
  float* db2 = const_cast<float*>(D.b2);
  float* dW3 = const_cast<float*>(D.W3);
  float* db3 = const_cast<float*>(D.b3);
  dense_bwd_weight_kernel<<<blocks((int64_t)out * (h + 1)), 256, 0, st>>>(a.g3, a.a2, B, h, out, dW3, db3);
  ATK_LAUNCHED();
  dense_bwd_input_kernel<<<blocks((int64_t)B * h), 256, 0, st>>>(a.g3, B, out, L.W3, h, a.z2, a.g2);
  ATK_LAUNCHED();
  dense_bwd_weight_kernel<<<blocks((int64_t)h * (h + 1)), 256, 0, st>>>(a.g2, a.a1, B, h, h, dW2, db2);
  ATK_LAUNCHED();
  dense_bwd_input_kernel<<<blocks((int64_t)B * h), 256, 0, st>>>(a.g2, B, h, L.W2, h, a.z1, a.g1);
  ATK_LAUNCHED();
  dense_bwd_weight_kernel<<<blocks((int64_t)h * (in + 1)), 256, 0, st>>>(a.g1, X, B, in, h, dW1, db1);
  ATK_LAUNCHED();
  return ATK_OK;
}

// Scratch for the activations of a batch of B rows.
struct ActBuf {
  float* base = nullptr;
  Acts a{};
  int alloc(int B, int h, int out, cudaStream_t st) {
    const size_t bh = (size_t)B * h, bo = (size_t)B * out;
    ATK_TRY(dev_alloc_async((void**)&base, sizeof(float) * (6 * bh + 2 * bo), st, "cudaMallocAsync(mlp buffers)"));
    a.z1 = base;
    a.a1 = a.z1 + bh;
    a.z2 = a.a1 + bh;
    a.a2 = a.z2 + bh;
    a.g2 = a.a2 + bh;
    a.g1 = a.g2 + bh;
    a.o = a.g1 + bh;
    a.g3 = a.o + bo;
    return ATK_OK;
  }
  void release(cudaStream_t st) {
    if (base) cudaFreeAsync(base, st);
    base = nullptr;
  }
};

int check_shape(int B, int in, int h, int out) {
  if (B < 1 || in < 1 || h < 1 || out < 1 || in > 4096 || h > 4096 || out > 4096) {
    set_error("mlp: sizes must be positive (and <= 4096 per layer)");
    return ATK_EINVAL;
  }
  return ATK_OK;
}

}  // namespace sel

bool selector_loaded() {
  std::lock_guard<std::mutex> g(sel::state().mu);
  return sel::state().loaded;
}

}  // namespace atk

using namespace atk;

extern "C" {

int atucker_mode_features(int order, const int64_t* dims, const int64_t* ranks, const int* mode_order,
                          double* out) {
  if (order < 1 || order > 8 || !dims || !ranks || !out) { set_error("mode_features: bad arguments"); return ATK_EINVAL; }
  double cur[8];
  for (int k = 0; k < order; ++k) {
    if (dims[k] < 1 || ranks[k] < 1) { set_error("mode_features: sizes must be >= 1"); return ATK_EINVAL; }
    cur[k] = (double)dims[k];
  }
  int seen[8] = {0};
  for (int step = 0; step < order; ++step) {
    const int n = mode_order ? mode_order[step] : step;
    if (n < 0 || n >= order || seen[n]) { set_error("mode_features: mode_order must be a permutation"); return ATK_EINVAL; }
    seen[n] = 1;
    const double I = cur[n], R = (double)ranks[n];
    double J = 1.0;
    for (int k = 0; k < order; ++k)
      if (k != n) J *= cur[k];
    double* f = out + (int64_t)n * ATK_SELECTOR_FEATURES;
    const double raw[10] = {I, R, J, I * I, R * R, I * R, R * R / I, R * R / J, I / J, R / J};
    for (int q = 0; q < 10; ++q) f[q] = std::log2(raw[q]);
    f[10] = order > 1 ? (double)step / (double)(order - 1) : 0.0;
    f[11] = std::log2(I * J);
    cur[n] = R;
  }
  return ATK_OK;
}

int64_t atucker_mlp_param_count(int in, int hidden, int out) { return sel::param_count(in, hidden, out); }

int atucker_selector_set(const float* params, int64_t count) {
  const int64_t np = sel::param_count(ATK_SELECTOR_FEATURES, ATK_SELECTOR_HIDDEN, ATK_NUM_CLASSES);
  if (!params || count != 2 * ATK_SELECTOR_FEATURES + np) { set_error("selector_set: wrong parameter count"); return ATK_EINVAL; }
  for (int q = 0; q < ATK_SELECTOR_FEATURES; ++q)
    if (!(params[ATK_SELECTOR_FEATURES + q] > 0.f)) { set_error("selector_set: feature scales must be > 0"); return ATK_EINVAL; }
  auto& s = sel::state();
  std::lock_guard<std::mutex> g(s.mu);
  for (int q = 0; q < ATK_SELECTOR_FEATURES; ++q) {
    s.fmean[q] = params[q];
    s.fscale[q] = params[ATK_SELECTOR_FEATURES + q];
  }
  s.params.assign(params + 2 * ATK_SELECTOR_FEATURES, params + count);
  s.loaded = true;
  s.kind = 0;
  return ATK_OK;
}

int atucker_selector_set_tree(int nodes, const int* feature, const double* threshold, const int* left,
                              const int* right, const int* leaf_class) {
  if (nodes < 1 || nodes > (1 << 20) || !feature || !threshold || !left || !right || !leaf_class) {
    set_error("selector_set_tree: bad arguments");
    return ATK_EINVAL;
  }
  for (int i = 0; i < nodes; ++i) {
    if (feature[i] < 0) {
      if (leaf_class[i] < 0 || leaf_class[i] >= ATK_NUM_CLASSES) {
        set_error("selector_set_tree: leaf class out of range");
        return ATK_EINVAL;
      }
    } else if (feature[i] >= ATK_SELECTOR_FEATURES || left[i] <= i || right[i] <= i || left[i] >= nodes ||
               right[i] >= nodes || !(threshold[i] == threshold[i])) {
      // children after their parent: every path ends, no cycle
      set_error("selector_set_tree: bad split node");
      return ATK_EINVAL;
    }
  }
  auto& s = sel::state();
  std::lock_guard<std::mutex> g(s.mu);
  s.tree.feature.assign(feature, feature + nodes);
  s.tree.threshold.assign(threshold, threshold + nodes);
  s.tree.left.assign(left, left + nodes);
  s.tree.right.assign(right, right + nodes);
  s.tree.cls.assign(leaf_class, leaf_class + nodes);
  s.loaded = true;
  s.kind = 1;
  return ATK_OK;
}

void atucker_selector_clear(void) {
  auto& s = sel::state();
  std::lock_guard<std::mutex> g(s.mu);
  s.loaded = false;
  s.params.clear();
  s.tree = sel::Tree{};
}

int atucker_selector_predict(const double* features, int rows, int* class_out, float* scores_out) {
  if (!features || rows < 0 || !class_out) { set_error("selector_predict: bad arguments"); return ATK_EINVAL; }
  auto& s = sel::state();
  std::lock_guard<std::mutex> g(s.mu);
  if (!s.loaded) { set_error("selector_predict: no selector loaded"); return ATK_EINVAL; }
  constexpr int IN = ATK_SELECTOR_FEATURES, H = ATK_SELECTOR_HIDDEN, K = ATK_NUM_CLASSES;
  if (s.kind == 1) {
    const sel::Tree& t = s.tree;
    for (int r = 0; r < rows; ++r) {
      const double* f = features + (int64_t)r * IN;
      int node = 0;
      while (t.feature[node] >= 0) node = f[t.feature[node]] <= t.threshold[node] ? t.left[node] : t.right[node];
      int c = t.cls[node];
      if (!sel::class_fits(c, f[0])) c = ATK_CLASS_ALS;
      class_out[r] = c;
      if (scores_out)
        for (int k = 0; k < K; ++k) scores_out[(int64_t)r * K + k] = k == c ? 0.f : 1.f;
    }
    return ATK_OK;
  }
  const float* W1 = s.params.data();
  const float* b1 = W1 + H * IN;
  const float* W2 = b1 + H;
  const float* b2 = W2 + H * H;
  const float* W3 = b2 + H;
  const float* b3 = W3 + K * H;
  for (int r = 0; r < rows; ++r) {
    const double* f = features + (int64_t)r * IN;
    float x[IN], h1[H], h2[H], o[K];
    for (int q = 0; q < IN; ++q) x[q] = (float)((f[q] - s.fmean[q]) / s.fscale[q]);
    for (int j = 0; j < H; ++j) {
      float a = b1[j];
      for (int q = 0; q < IN; ++q) a = std::fma(W1[j * IN + q], x[q], a);
      h1[j] = a > 0.f ? a : 0.f;
    }
    for (int j = 0; j < H; ++j) {
      float a = b2[j];
      for (int q = 0; q < H; ++q) a = std::fma(W2[j * H + q], h1[q], a);
      h2[j] = a > 0.f ? a : 0.f;
    }
    for (int k = 0; k < K; ++k) {
      float a = b3[k];
      for (int q = 0; q < H; ++q) a = std::fma(W3[k * H + q], h2[q], a);
      o[k] = a;
    }
    int best = ATK_CLASS_ALS;
    for (int k = 0; k < K; ++k) {
      if (!sel::class_fits(k, f[0])) continue;
      if (o[k] < o[best] || (o[k] == o[best] && k < best)) best = k;
    }
    class_out[r] = best;
    if (scores_out)
      for (int k = 0; k < K; ++k) scores_out[(int64_t)r * K + k] = o[k];
  }
  return ATK_OK;
}

int atucker_mlp_forward(const float* X, int B, int in, int hidden, int out, const float* params, float* Y_out,
                        void* stream) {
  if (!X || !params || !Y_out) { set_error("mlp_forward: null pointer"); return ATK_EINVAL; }
  ATK_TRY(sel::check_shape(B, in, hidden, out));
  cudaStream_t st = (cudaStream_t)stream;
  sel::ActBuf buf;
  ATK_TRY(buf.alloc(B, hidden, out, st));
  sel::Acts a = buf.a;
  a.o = Y_out;
  int s = sel::forward(X, B, in, hidden, out, params, a, st);
  buf.release(st);
  if (s != ATK_OK) return s;
  ATK_CUDA(cudaStreamSynchronize(st));
  return ATK_OK;
}

int atucker_mlp_loss_grad(const float* X, const float* Y, const float* M, int B, int in, int hidden, int out,
                          const float* params, float* loss, float* grad, void* stream) {
  if (!X || !Y || !M || !params || !loss || !grad) { set_error("mlp_loss_grad: null pointer"); return ATK_EINVAL; }
  ATK_TRY(sel::check_shape(B, in, hidden, out));
  cudaStream_t st = (cudaStream_t)stream;
  sel::ActBuf buf;
  ATK_TRY(buf.alloc(B, hidden, out, st));
  int s = sel::loss_grad(X, Y, M, B, in, hidden, out, params, loss, grad, buf.a, st);
  buf.release(st);
  if (s != ATK_OK) return s;
  ATK_CUDA(cudaStreamSynchronize(st));
  return ATK_OK;
}

int atucker_mlp_train(const float* X, const float* Y, const float* M, int B, int in, int hidden, int out,
                      float* params, float* state, int steps, int step_base, float lr, float* loss_out,
                      void* stream) {
  if (!X || !Y || !M || !params || !state) { set_error("mlp_train: null pointer"); return ATK_EINVAL; }
  ATK_TRY(sel::check_shape(B, in, hidden, out));
  if (steps < 0 || step_base < 0 || !(lr > 0.f)) { set_error("mlp_train: need steps >= 0, step_base >= 0, lr > 0"); return ATK_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t np = sel::param_count(in, hidden, out);
  sel::ActBuf buf;
  ATK_TRY(buf.alloc(B, hidden, out, st));
  float* grad = nullptr;
  if (dev_alloc_async((void**)&grad, sizeof(float) * (np + 1), st, "cudaMallocAsync(mlp gradient)") != ATK_OK) {
    buf.release(st);
    set_error("mlp_train: out of device memory");
    return ATK_ENOMEM;
  }
  float* scratch_loss = grad + np;
  int s = ATK_OK;
  for (int k = 0; k < steps && s == ATK_OK; ++k) {
    s = sel::loss_grad(X, Y, M, B, in, hidden, out, params, loss_out ? loss_out + k : scratch_loss, grad, buf.a, st);
    if (s != ATK_OK) break;
    const int t = step_base + k + 1;
    const float c1 = 1.f - std::pow(0.9f, (float)t), c2 = 1.f - std::pow(0.999f, (float)t);
    sel::adam_kernel<<<sel::blocks(np), 256, 0, st>>>(params, grad, state, state + np, np, lr, c1, c2);
    if (cudaGetLastError() != cudaSuccess) { set_error("mlp_train: adam launch failed"); s = ATK_ECUDA; }
    count_launch();
  }
  cudaFreeAsync(grad, st);
  buf.release(st);
  if (s != ATK_OK) return s;
  ATK_CUDA(cudaStreamSynchronize(st));
  return ATK_OK;
}

}  // extern "C"
