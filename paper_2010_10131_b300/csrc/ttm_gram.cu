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
#include "fp32_block.cuh"

namespace atk {

namespace {
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

// Rows are ordered rho = l + L (i + Im h), so consecutive rows are
// consecutive lows (consecutive addresses when lo > 1).  RowInfo caches the
// group-independent part of each row's index arithmetic in shared memory
// (the divisions would otherwise outnumber the FMAs):
//   x  = l + s (i + Im h), the row's offset from the group's first row c, or
//        -1 when rho is beyond the group's L Im H rows;
//   y  = l | h << 16, checked against the group's remaining lows and highs;
//   z  = R (l + L h) (GI + PAD) + i, the row's place in the staged fibres.
struct GroupBase {
  int c0, lowrem, highrem;
};

__device__ __forceinline__ GroupBase group_base(const FibreGeom& G, int g) {
  const int lc = g % G.nlowc, hb = g / G.nlowc;
  return {lc * G.L + G.s * G.Im * (hb * G.H), G.s - lc * G.L, G.nhigh - hb * G.H};
}

// Row c of a cached row in group gb, or -1 for a padding row.
__device__ __forceinline__ int row_c(const int4& q, const GroupBase& gb) {
  if (q.x < 0) return -1;
  return ((q.y & 0xffff) < gb.lowrem && (q.y >> 16) < gb.highrem) ? gb.c0 + q.x : -1;
}

// TTM tile BM x RB (the plain TTM kernel's shapes: 256 x 16, 128 x 32,
// 128 x 64); Gram tile GI x GI with GI = I_m rounded up to 32 / 64 / 128,
// accumulated in registers across the CTA's groups.  Both are the shared
// register block (packed FMA pairs); the Gram's diagonal tile skips its
// lower-left quadrant, which the reduction reads from the mirror entries.
template <int BM, int RB, int TM, int TN, int GI, int MINB>
__global__ void __launch_bounds__(NT, MINB)
ttm_gram_kernel(const float* __restrict__ y, const float* __restrict__ U, float* __restrict__ out,
                const FibreGeom G, float* __restrict__ part) {
  using TB = Block<BM, RB, TM, TN, true>;
  constexpr int GT = GI / 16;
  using GB = Block<GI, GI, GT, GT, true>;
  constexpr int LDA = BM + PAD, LDB = RB + PAD, TGP = GI + PAD;
  constexpr int SA = TK * LDA, SB = TK * LDB;
  constexpr int PER = TK * BM / NT;  // A values per thread per k-tile
  constexpr int BPER = TK * RB / NT > 0 ? TK * RB / NT : 1;
  extern __shared__ __align__(16) float smem[];
  __shared__ int4 rinfo[BM];
  float* const sA = smem;           // [2][TK][BM + PAD]: Y rows, k-major
  float* const sB = smem + 2 * SA;  // [2][TK][RB + PAD]: U
  float* const Tg = sB + 2 * SB;    // [L H R][GI + PAD]: the group's fibres
  const int tid = threadIdx.x;
  const int KG = G.L * G.H * G.R;
  // Columns i >= Im of the staged fibres are never written: zero them once.
  for (int e = tid; e < KG * TGP; e += NT) Tg[e] = 0.f;
  for (int rho = tid; rho < BM; rho += NT) {
    const int l = rho % G.L, t = rho / G.L;
    const int i = t % G.Im, h = t / G.Im;
    rinfo[rho] = h < G.H ? make_int4(l + G.s * (i + G.Im * h), l | (h << 16), G.R * (l + G.L * h) * TGP + i, 0)
                         : make_int4(-1, 0, 0, 0);
  }
  __syncthreads();
  GB gb;
  gb.init();

  const bool lanes_k = G.lo == 1;  // Y(c, k) contiguous in k
  const int ntile = (G.n + TK - 1) / TK;
  // A loader: lanes_k: k = a_km, rows a_mm + 16 e; else: row a_mm, k = a_km + (NT / BM) e.
  const int a_km = lanes_k ? tid % 16 : tid / BM;
  const int a_mm = lanes_k ? tid / 16 : tid % BM;
  // B loader: k = tid % 16, columns tid / 16 + 16 e.
  const int b_km = tid % 16, b_mm = tid / 16;

  for (int g = blockIdx.x; g < G.ngroups; g += gridDim.x) {
    const GroupBase gbase = group_base(G, g);
    int aoff[PER];
    if (lanes_k) {
#pragma unroll
      for (int e = 0; e < PER; ++e) {
        const int c = row_c(rinfo[a_mm + 16 * e], gbase);
        aoff[e] = c >= 0 ? G.n * c : -1;
      }
    } else {
      const int c = row_c(rinfo[a_mm], gbase);
      aoff[0] = c >= 0 ? (c % G.lo) + G.lo * G.n * (c / G.lo) : -1;
    }
    float ra[PER], rb[BPER];
    auto fetch = [&](int k0) {
      if (lanes_k) {
        const int k = k0 + a_km;
#pragma unroll
        for (int e = 0; e < PER; ++e) ra[e] = (aoff[e] >= 0 && k < G.n) ? __ldg(y + aoff[e] + k) : 0.f;
      } else {
#pragma unroll
        for (int e = 0; e < PER; ++e) {
          const int k = k0 + a_km + (NT / BM) * e;
          ra[e] = (aoff[0] >= 0 && k < G.n) ? __ldg(y + aoff[0] + G.lo * k) : 0.f;
        }
      }
      const int k = k0 + b_km;
#pragma unroll
      for (int e = 0; e < BPER; ++e) {
        const int r = b_mm + 16 * e;
        rb[e] = (k < G.n && r < G.R) ? __ldg(U + k + G.n * r) : 0.f;
      }
    };
    auto store = [&](int buf) {
      float* a = sA + buf * SA;
      float* b = sB + buf * SB;
      if (lanes_k) {
#pragma unroll
        for (int e = 0; e < PER; ++e) a[a_km * LDA + a_mm + 16 * e] = ra[e];
      } else {
#pragma unroll
        for (int e = 0; e < PER; ++e) a[(a_km + (NT / BM) * e) * LDA + a_mm] = ra[e];
      }
#pragma unroll
      for (int e = 0; e < BPER; ++e) b[b_km * LDB + b_mm + 16 * e] = rb[e];
    };

    // ---- TTM: T(rho, r) = sum_k Y(c(rho), k) U(k, r)
    TB tb;
    tb.init();
    fetch(0);
    store(0);
    __syncthreads();
    for (int t = 0; t < ntile; ++t) {
      const int buf = t & 1;
      if (t + 1 < ntile) fetch((t + 1) * TK);
      tb.mma(sA + buf * SA, sB + buf * SB);
      if (t + 1 < ntile) store(buf ^ 1);
      __syncthreads();
    }

    // ---- epilogue: write Y' and stage the fibres (zeros for padding slots)
#pragma unroll
    for (int u = 0; u < TM; ++u) {
      const int4 q = rinfo[TB::row_of(tb.ty, u)];
      const int c = row_c(q, gbase);
      const int base = c < 0 ? 0 : (lanes_k ? G.R * c : (c % G.lo) + G.lo * G.R * (c / G.lo));
#pragma unroll
      for (int v = 0; v < TN; ++v) {
        const int r = TB::col_of(tb.tx, v);
        if (r >= G.R) continue;
        const float val = tb.acc(u, v);
        if (c >= 0) out[base + G.lo * r] = val;
        if (q.x >= 0) Tg[q.z + r * TGP] = c >= 0 ? val : 0.f;
      }
    }
    __syncthreads();

    // ---- Gram: S_part(i, j) += sum over the group's fibres T(i, kg) T(j, kg)
#pragma unroll 4
    for (int kg = 0; kg < KG; ++kg) gb.template step<true, TGP, TGP>(Tg, Tg, kg);
    // The next group's first shared-memory writes go to sA / sB; Tg is
    // rewritten only after that group's main loop, whose barriers order it
    // after every thread's Gram reads here.
  }
  // ---- this CTA's partial Gram (I_m x I_m, column-major; lower-left
  // quadrant entries of the tile are not computed and never read)
  float* p = part + (int64_t)blockIdx.x * G.Im * G.Im;
#pragma unroll
  for (int u = 0; u < GT; ++u)
#pragma unroll
    for (int v = 0; v < GT; ++v) {
      const int i = GB::row_of(gb.ty, u), j = GB::col_of(gb.tx, v);
      if (i <= j && j < G.Im) p[i + G.Im * j] = gb.acc(u, v);
    }
}

// S(i, j) = sum over the CTAs' partials in CTA order, float-float, rounded to
// float64, read from the upper triangle for both (i, j) and (j, i), so S is
// exactly symmetric.
__global__ void ttm_gram_reduce_kernel(const float* __restrict__ part, int nparts, int Im, double* __restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Im * Im) return;
  const int i = e % Im, j = e / Im;
  const int up = min(i, j) + Im * max(i, j);  // the partials hold the upper triangle
  FFSum acc;
  for (int p = 0; p < nparts; ++p) acc.add(part[(int64_t)p * Im * Im + up]);
  S[e] = acc.value();
}

int rb_of(int64_t R) { return R <= 16 ? 16 : (R <= 32 ? 32 : 64); }
int bm_of(int rb) { return rb == 16 ? 256 : 128; }
int gi_of(int64_t Im) { return Im <= 32 ? 32 : (Im <= 64 ? 64 : 128); }

size_t smem_of(int rb, int gi, int KG) {
  return sizeof(float) * ((size_t)2 * TK * (bm_of(rb) + PAD) + (size_t)2 * TK * (rb + PAD) + (size_t)KG * (gi + PAD));
}

// Fibre slots and group counts for the geometry; false if it does not fit.
bool make_geom(const View& v, int64_t R, int64_t s, int64_t Im, FibreGeom& G) {
  const int64_t J = v.J();
  if (R < 1 || R > 64 || Im < 16 || Im > 128 || s < 1 || J % (s * Im) != 0) return false;
  const int gi = gi_of(Im);
  int64_t P = std::min<int64_t>(bm_of(rb_of(R)) / Im, FG_TG_FLOATS / (R * (gi + PAD)));
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
  static constexpr int BM = RB == 16 ? 256 : 128;
  static constexpr int TM = 8, TN = RB == 64 ? 4 : 2;
  static constexpr int MINB = 2;
  static constexpr auto kernel = ttm_gram_kernel<BM, RB, TM, TN, GI, MINB>;
  static int occupancy(size_t smem) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem_of(RB, GI, FG_TG_FLOATS / (GI + PAD)));
      attr = true;
    }
    int o = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, NT, smem);
    return std::max(1, o);
  }
  static void launch(int grid, size_t smem, const float* y, const float* U, float* out, const FibreGeom& G,
                     float* part, cudaStream_t st) {
    kernel<<<grid, NT, smem, st>>>(y, U, out, G, part);
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
