// Fused truncating TTM and next-mode Gram.  In Alg. 2 the TTM that closes
// mode n (Y' = Y x_n U^T) and the Gram that opens the next mode m
// (S_m = Y'_(m) Y'_(m)^T) are adjacent steps, so the second re-reads the
// whole of Y' that the first has just written.  This kernel computes Y' in
// tiles that hold complete mode-m fibres of Y' and, while the tile is still
// on chip, adds those fibres' outer products into the CTA's own partial
// S_m.  Y' is still written (the mode-m TTM reads it), but nothing reads it
// for the Gram, and the Gram's FMAs overlap the TTM's HBM stream.
//
// Geometry.  The TTM's rows are c = a + lo b over the mode-n view (lo, n, hi)
// of Y, and its columns are r < R.  In that row index mode m has a stride s
// (the product of the current sizes of the modes below m other than n) and
// extent I_m, so c = low + s (i + I_m high).  A mode-m fibre of Y' is a fixed
// (low, high, r) with i running over [0, I_m).  A group is L lows x H highs
// ("fibre slots", L H I_m <= 128 rows) with all their i and all r: its TTM
// tile is 128 x R, and its Gram contribution is T T^T with T the I_m x (L H R)
// matrix of its fibres.
//
// Determinism: every CTA owns a fixed set of groups (g = blockIdx.x + k
// gridDim.x) and sums them in a fixed order into float32 registers; the
// partial Grams are summed in CTA order as float-float pairs rounded to
// float64.  The grid is large enough that no float32 chain has more than 8192
// terms, the split bound the plain Gram keeps.
#include <algorithm>

#include "atk_internal.cuh"

namespace atk {

namespace {
constexpr int FG_NT = 256;      // threads: a 16 x 16 grid
constexpr int FG_TK = 16;       // k-tile depth of the TTM
constexpr int FG_BM = 128;      // TTM rows per group
constexpr int FG_PAD = 4;       // smem row padding (floats)
constexpr int FG_TG_FLOATS = 12288;  // staged fibres per group: at most 48 KB
constexpr int FG_MAX_CHAIN = 8192;

struct FibreGeom {
  int lo, n, J;      // mode-n view of Y; J = lo * hi TTM rows
  int R;             // TTM columns (R_n)
  int s, Im, nhigh;  // c = low + s (i + Im high)
  int L, H;          // fibre slots per group: L lows x H highs
  int nlowc;         // groups along low
  int ngroups;
};

// Row rho of group g -> its TTM row c, or -1 for a padding row.  Rows are
// ordered rho = l + L (i + Im h), so consecutive rows are consecutive lows
// (consecutive addresses when lo > 1).
__device__ __forceinline__ int fibre_row(const FibreGeom& G, int g, int rho) {
  const int l = rho % G.L, t = rho / G.L;
  const int i = t % G.Im, h = t / G.Im;
  if (h >= G.H) return -1;
  const int low = (g % G.nlowc) * G.L + l;
  const int high = (g / G.nlowc) * G.H + h;
  if (low >= G.s || high >= G.nhigh) return -1;
  return low + G.s * (i + G.Im * high);
}

// RB: R rounded up to 16 / 32 / 64 (TN = RB / 16 columns per thread, 8 rows).
// GI: I_m rounded up to 32 / 64 / 128 (GT = GI / 16 Gram rows and columns per
// thread).  The Gram accumulators live in registers across the CTA's groups.
template <int RB, int GI, int MINB>
__global__ void __launch_bounds__(FG_NT, MINB)
ttm_gram_kernel(const float* __restrict__ y, const float* __restrict__ U, float* __restrict__ out,
                const FibreGeom G, float* __restrict__ part) {
  constexpr int TN = RB / 16;
  constexpr int GT = GI / 16;
  constexpr int SA = FG_TK * (FG_BM + FG_PAD), SB = FG_TK * (RB + FG_PAD), TGP = GI + FG_PAD;
  extern __shared__ __align__(16) float smem[];
  float* const sA = smem;           // [2][TK][BM + PAD]: Y rows, k-major
  float* const sB = smem + 2 * SA;  // [2][TK][RB + PAD]: U
  float* const Tg = sB + 2 * SB;    // [L H R][GI + PAD]: the group's fibres
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int KG = G.L * G.H * G.R;
  // Columns i >= Im of the staged fibres are never written: zero them once.
  for (int e = tid; e < KG * TGP; e += FG_NT) Tg[e] = 0.f;
  float gacc[GT][GT];
#pragma unroll
  for (int u = 0; u < GT; ++u)
#pragma unroll
    for (int v = 0; v < GT; ++v) gacc[u][v] = 0.f;

  const bool lanes_k = G.lo == 1;  // Y(c, k) contiguous in k
  const int ntile = (G.n + FG_TK - 1) / FG_TK;
  // A loader: lanes_k: k = km, rows mm + 16 e; else: row mm, k = km + 2 e.
  const int a_km = lanes_k ? tid % 16 : tid / FG_BM;
  const int a_mm = lanes_k ? tid / 16 : tid % FG_BM;
  // B loader: k = tid % 16, columns tid / 16 + 16 e.
  const int b_km = tid % 16, b_mm = tid / 16;

  for (int g = blockIdx.x; g < G.ngroups; g += gridDim.x) {
    int aoff[8];
    if (lanes_k) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = fibre_row(G, g, a_mm + 16 * e);
        aoff[e] = c >= 0 ? G.n * c : -1;
      }
    } else {
      const int c = fibre_row(G, g, a_mm);
      aoff[0] = c >= 0 ? (c % G.lo) + G.lo * G.n * (c / G.lo) : -1;
    }
    float ra[8], rb[TN];
    auto fetch = [&](int k0) {
      if (lanes_k) {
        const int k = k0 + a_km;
#pragma unroll
        for (int e = 0; e < 8; ++e) ra[e] = (aoff[e] >= 0 && k < G.n) ? __ldg(y + aoff[e] + k) : 0.f;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = k0 + a_km + 2 * e;
          ra[e] = (aoff[0] >= 0 && k < G.n) ? __ldg(y + aoff[0] + G.lo * k) : 0.f;
        }
      }
      const int k = k0 + b_km;
#pragma unroll
      for (int e = 0; e < TN; ++e) {
        const int r = b_mm + 16 * e;
        rb[e] = (k < G.n && r < G.R) ? __ldg(U + k + G.n * r) : 0.f;
      }
    };
    auto store = [&](int buf) {
      float* a = sA + buf * SA;
      float* b = sB + buf * SB;
      if (lanes_k) {
#pragma unroll
        for (int e = 0; e < 8; ++e) a[a_km * (FG_BM + FG_PAD) + a_mm + 16 * e] = ra[e];
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) a[(a_km + 2 * e) * (FG_BM + FG_PAD) + a_mm] = ra[e];
      }
#pragma unroll
      for (int e = 0; e < TN; ++e) b[b_km * (RB + FG_PAD) + b_mm + 16 * e] = rb[e];
    };

    // ---- TTM: acc(rho, r) = sum_k Y(c(rho), k) U(k, r), rows ty*8.., columns tx*TN..
    float acc[8][TN];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < TN; ++v) acc[u][v] = 0.f;
    fetch(0);
    store(0);
    __syncthreads();
    for (int t = 0; t < ntile; ++t) {
      const int buf = t & 1;
      if (t + 1 < ntile) fetch((t + 1) * FG_TK);
      const float* a = sA + buf * SA;
      const float* b = sB + buf * SB;
#pragma unroll
      for (int kk = 0; kk < FG_TK; ++kk) {
        const float4 a0 = *reinterpret_cast<const float4*>(a + kk * (FG_BM + FG_PAD) + ty * 8);
        const float4 a1 = *reinterpret_cast<const float4*>(a + kk * (FG_BM + FG_PAD) + ty * 8 + 4);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float bv[TN];
#pragma unroll
        for (int v = 0; v < TN; ++v) bv[v] = b[kk * (RB + FG_PAD) + tx * TN + v];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < TN; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
      }
      if (t + 1 < ntile) store(buf ^ 1);
      __syncthreads();
    }

    // ---- epilogue: write Y' and stage the fibres (zeros for padding slots)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int rho = ty * 8 + u;
      const int c = fibre_row(G, g, rho);
      const int l = rho % G.L, t = rho / G.L;
      const int i = t % G.Im, h = t / G.Im;
      const bool slot = h < G.H;  // rho < L Im H
      const int base = c >= 0 ? (c % G.lo) + G.lo * G.R * (c / G.lo) : 0;
#pragma unroll
      for (int v = 0; v < TN; ++v) {
        const int r = tx * TN + v;
        if (r >= G.R) continue;
        if (c >= 0) out[base + G.lo * r] = acc[u][v];
        if (slot) Tg[(r + G.R * (l + G.L * h)) * TGP + i] = c >= 0 ? acc[u][v] : 0.f;
      }
    }
    __syncthreads();

    // ---- Gram: gacc(i, j) += sum over the group's fibres T(i, kg) T(j, kg)
    for (int kg = 0; kg < KG; ++kg) {
      const float* row = Tg + kg * TGP;
      float ai[GT], aj[GT];
#pragma unroll
      for (int u = 0; u < GT; u += 2) {
        const float2 p = *reinterpret_cast<const float2*>(row + ty * GT + u);
        const float2 q = *reinterpret_cast<const float2*>(row + tx * GT + u);
        ai[u] = p.x; ai[u + 1] = p.y;
        aj[u] = q.x; aj[u + 1] = q.y;
      }
#pragma unroll
      for (int u = 0; u < GT; ++u)
#pragma unroll
        for (int v = 0; v < GT; ++v) gacc[u][v] = fmaf(ai[u], aj[v], gacc[u][v]);
    }
    // The next group's first shared-memory writes go to sA / sB; Tg is
    // rewritten only after that group's main loop, whose barriers order it
    // after every thread's Gram reads here.
  }
  // ---- this CTA's partial Gram (I_m x I_m, column-major)
  float* p = part + (int64_t)blockIdx.x * G.Im * G.Im;
#pragma unroll
  for (int u = 0; u < GT; ++u)
#pragma unroll
    for (int v = 0; v < GT; ++v) {
      const int i = ty * GT + u, j = tx * GT + v;
      if (i < G.Im && j < G.Im) p[i + G.Im * j] = gacc[u][v];
    }
}

// S(i, j) = sum over the CTAs' partials in CTA order, float-float, rounded to
// float64.  The partials are exactly symmetric (fmaf(a, b) == fmaf(b, a)), so
// S is too.
__global__ void ttm_gram_reduce_kernel(const float* __restrict__ part, int nparts, int Im, double* __restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Im * Im) return;
  FFSum acc;
  for (int p = 0; p < nparts; ++p) acc.add(part[(int64_t)p * Im * Im + e]);
  S[e] = acc.value();
}

int rb_of(int64_t R) { return R <= 16 ? 16 : (R <= 32 ? 32 : 64); }
int gi_of(int64_t Im) { return Im <= 32 ? 32 : (Im <= 64 ? 64 : 128); }

size_t smem_of(int rb, int gi, int KG) {
  return sizeof(float) * ((size_t)2 * FG_TK * (FG_BM + FG_PAD) + (size_t)2 * FG_TK * (rb + FG_PAD) +
                          (size_t)KG * (gi + FG_PAD));
}

// Fibre slots and group counts for the geometry; false if it does not fit.
bool make_geom(const View& v, int64_t R, int64_t s, int64_t Im, FibreGeom& G) {
  const int64_t J = v.J();
  if (R < 1 || R > 64 || Im < 16 || Im > FG_BM || s < 1 || J % (s * Im) != 0) return false;
  const int gi = gi_of(Im);
  int64_t P = std::min<int64_t>(FG_BM / Im, FG_TG_FLOATS / (R * (gi + FG_PAD)));
  if (P < 1) return false;
  G.lo = (int)v.lo;
  G.n = (int)v.n;
  G.J = (int)J;
  G.R = (int)R;
  G.s = (int)s;
  G.Im = (int)Im;
  G.nhigh = (int)(J / (s * Im));
  if (s >= P) {
    G.L = (int)P;
    G.H = 1;
  } else {
    G.L = (int)s;
    G.H = (int)std::max<int64_t>(1, P / s);
  }
  G.nlowc = (int)ceil_div(G.s, G.L);
  const int64_t groups = (int64_t)G.nlowc * ceil_div(G.nhigh, G.H);
  if (groups > 0x7fffffff) return false;
  G.ngroups = (int)groups;
  return true;
}

template <int RB, int GI>
struct FgVariant {
  static constexpr int MINB = (RB == 64 && GI == 128) ? 1 : 2;
  static int occupancy(size_t smem) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(ttm_gram_kernel<RB, GI, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_of(RB, GI, FG_TG_FLOATS / (GI + FG_PAD)));
      attr = true;
    }
    int o = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, ttm_gram_kernel<RB, GI, MINB>, FG_NT, smem);
    return std::max(1, o);
  }
  static void launch(int grid, size_t smem, const float* y, const float* U, float* out, const FibreGeom& G,
                     float* part, cudaStream_t st) {
    ttm_gram_kernel<RB, GI, MINB><<<grid, FG_NT, smem, st>>>(y, U, out, G, part);
  }
};

// One wave of resident CTAs, or more where the 8192-term chain bound needs it.
template <int RB, int GI>
int grid_for(const FibreGeom& G, size_t smem) {
  const int occ = FgVariant<RB, GI>::occupancy(smem);
  const int64_t KG = (int64_t)G.L * G.H * G.R;
  const int64_t need = ceil_div((int64_t)G.ngroups * KG, FG_MAX_CHAIN);
  return (int)std::min<int64_t>(G.ngroups, std::max<int64_t>((int64_t)occ * num_sms(), need));
}

template <int RB, int GI>
int run_variant(const float* y, const float* U, float* out, const FibreGeom& G, float* part, size_t part_floats,
                double* S, cudaStream_t st, int* grid_out) {
  const size_t smem = smem_of(RB, GI, G.L * G.H * G.R);
  const int grid = grid_for<RB, GI>(G, smem);
  if (grid_out) {  // sizing query only
    *grid_out = grid;
    return ATK_OK;
  }
  if ((size_t)grid * G.Im * G.Im > part_floats) { set_error("ttm_gram: scratch too small"); return ATK_ENOMEM; }
  FgVariant<RB, GI>::launch(grid, smem, y, U, out, G, part, st);
  ATK_LAUNCHED();
  ttm_gram_reduce_kernel<<<(unsigned)ceil_div((int64_t)G.Im * G.Im, 256), 256, 0, st>>>(part, grid, G.Im, S);
  ATK_LAUNCHED();
  return ATK_OK;
}

int dispatch(const float* y, const FibreGeom& G, const float* U, float* out, double* S, float* part, size_t pf,
             cudaStream_t st, int* grid_out) {
  const int rb = rb_of(G.R), gi = gi_of(G.Im);
#define ATK_FG(RB_, GI_) \
  if (rb == RB_ && gi == GI_) return run_variant<RB_, GI_>(y, U, out, G, part, pf, S, st, grid_out);
  ATK_FG(16, 32) ATK_FG(16, 64) ATK_FG(16, 128)
  ATK_FG(32, 32) ATK_FG(32, 64) ATK_FG(32, 128)
  ATK_FG(64, 32) ATK_FG(64, 64) ATK_FG(64, 128)
#undef ATK_FG
  set_error("ttm_gram: no variant");
  return ATK_EUNSUPPORTED;
}
}  // namespace

bool ttm_gram_ok(const View& v, int64_t R, int64_t s, int64_t Im) {
  FibreGeom G;
  return make_geom(v, R, s, Im, G);
}

size_t ttm_gram_scratch_bytes(const View& v, int64_t R, int64_t s, int64_t Im) {
  FibreGeom G;
  int grid = 0;
  if (!make_geom(v, R, s, Im, G) || dispatch(nullptr, G, nullptr, nullptr, nullptr, nullptr, 0, nullptr, &grid) != ATK_OK)
    return 0;
  return sizeof(float) * (size_t)grid * (size_t)(Im * Im);
}

int ttm_gram(const float* y, const View& v, const float* U, int64_t R, int64_t s, int64_t Im, float* out,
             double* S, void* scratch, size_t scratch_bytes, cudaStream_t st) {
  FibreGeom G;
  if (!make_geom(v, R, s, Im, G)) { set_error("ttm_gram: unsupported geometry"); return ATK_EUNSUPPORTED; }
  return dispatch(y, G, U, out, S, (float*)scratch, scratch_bytes / sizeof(float), st, nullptr);
}

}  // namespace atk
