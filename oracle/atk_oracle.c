/*
 * CPU oracle for the mode-wise flexible st-HOSVD (a-Tucker, arXiv 2010.10131).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library.  It shares no code, header or table
 * with the CUDA path.
 *
 * Plain, slow and explicit: every routine works in float64.  Tensor ops first
 * build the mode-n matricization as a separate matrix (Sec. II-A), then call
 * plain triple-loop matrix products.  Nothing is blocked, fused or reordered
 * beyond the definitions.
 *
 * Conventions
 *   - A tensor with dims (I_1..I_N) is column-major, first index fastest (Sec. V).
 *   - X_(n) is I_n x J_n, column-major (Sec. II-A).  Its column index j enumerates
 *     the remaining indices, with the lowest remaining mode fastest.
 *   - Factor U^(n) is I_n x R_n, column-major (Sec. II-B).
 *   - Modes are 0-based here; the paper counts from 1.
 *
 * Readings of the paper, where it is silent or ambiguous:
 *   - Alg. 3 runs exactly `sweeps` iterations (default 5, Sec. III-B after Eq. 5).
 *     It returns L = L_K and R = R_{K-1}, the R that produced L_K.
 *   - ALS initial guess L_0: N(0,1) entries from a counter-based splitmix64
 *     stream and the Box-Muller transform (see ora_als_init).
 *   - "Matrix inversion" (Eq. 5) is applied as a Cholesky solve.
 *   - Eigenvalues are sorted descending.  Equal values keep their original
 *     index order.  Each eigenvector column is flipped so that its
 *     largest-magnitude entry is positive (ties: lowest row).
 *   - QR: Householder, with diag(R) > 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_EINVAL (-1)
#define ORA_ERANK (-2)
#define ORA_ENOMEM (-3)
#define ORA_ENOCONV (-5)

/* ---------------------------------------------------------------- helpers */

static int64_t prod_dims(int order, const int64_t* dims) {
  int64_t p = 1;
  for (int k = 0; k < order; ++k) p *= dims[k];
  return p;
}

/* Mode-n matricization, Sec. II-A: entry (i_1..i_N) goes to row i_n and to
 * column j = sum_{k != n} i_k * prod_{m < k, m != n} I_m. */
void ora_unfold(const double* x, int order, const int64_t* dims, int n, double* xn) {
  int64_t total = prod_dims(order, dims);
  int64_t In = dims[n];
  int64_t idx[16];
  for (int k = 0; k < order; ++k) idx[k] = 0;
  for (int64_t lin = 0; lin < total; ++lin) {
    int64_t j = 0, stride = 1;
    for (int k = 0; k < order; ++k) {
      if (k == n) continue;
      j += idx[k] * stride;
      stride *= dims[k];
    }
    xn[idx[n] + In * j] = x[lin];
    for (int k = 0; k < order; ++k) { /* advance the column-major multi-index */
      if (++idx[k] < dims[k]) break;
      idx[k] = 0;
    }
  }
}

/* Tensorization, the inverse of ora_unfold. */
void ora_fold(const double* xn, int order, const int64_t* dims, int n, double* x) {
  int64_t total = prod_dims(order, dims);
  int64_t In = dims[n];
  int64_t idx[16];
  for (int k = 0; k < order; ++k) idx[k] = 0;
  for (int64_t lin = 0; lin < total; ++lin) {
    int64_t j = 0, stride = 1;
    for (int k = 0; k < order; ++k) {
      if (k == n) continue;
      j += idx[k] * stride;
      stride *= dims[k];
    }
    x[lin] = xn[idx[n] + In * j];
    for (int k = 0; k < order; ++k) {
      if (++idx[k] < dims[k]) break;
      idx[k] = 0;
    }
  }
}

/* C (m x p) = op(A) op(B), column-major.  op(A) is m x k; ta/tb select the
 * transpose.  A plain triple loop; OpenMP over the columns of C. */
void ora_matmul(int ta, int tb, int64_t m, int64_t p, int64_t k, const double* A, int64_t lda,
                const double* B, int64_t ldb, double* C, int64_t ldc) {
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < p; ++c) {
    for (int64_t r = 0; r < m; ++r) {
      double s = 0.0;
      for (int64_t t = 0; t < k; ++t) {
        double a = ta ? A[t + lda * r] : A[r + lda * t];
        double b = tb ? B[c + ldb * t] : B[t + ldb * c];
        s += a * b;
      }
      C[r + ldc * c] = s;
    }
  }
}

/* Squared Frobenius norm, Eq. (1). */
double ora_norm2(const double* x, int64_t len) {
  double s = 0.0;
  for (int64_t i = 0; i < len; ++i) s += x[i] * x[i];
  return s;
}

/* Gram matrix S = Y_(n) Y_(n)^T (Alg. 2, EIG branch).  S is I_n x I_n. */
int ora_gram(const double* x, int order, const int64_t* dims, int n, double* S) {
  int64_t In = dims[n], total = prod_dims(order, dims), Jn = total / In;
  double* xn = (double*)malloc(sizeof(double) * (size_t)total);
  if (!xn) return ORA_ENOMEM;
  ora_unfold(x, order, dims, n, xn);
  ora_matmul(0, 1, In, In, Jn, xn, In, xn, In, S, In);
  free(xn);
  return ORA_OK;
}

/* TTM, Eq. (2), with the matrix W = U^T (U is I_n x R): Y = X x_n U^T, i.e.
 * Y_(n) = U^T X_(n).  The output has mode n of size R. */
int ora_ttm(const double* x, int order, const int64_t* dims, int n, const double* U, int64_t R, double* y) {
  int64_t In = dims[n], total = prod_dims(order, dims), Jn = total / In;
  double* xn = (double*)malloc(sizeof(double) * (size_t)total);
  double* yn = (double*)malloc(sizeof(double) * (size_t)(R * Jn));
  if (!xn || !yn) { free(xn); free(yn); return ORA_ENOMEM; }
  ora_unfold(x, order, dims, n, xn);
  ora_matmul(1, 0, R, Jn, In, U, In, xn, In, yn, R);
  int64_t odims[16];
  for (int k = 0; k < order; ++k) odims[k] = dims[k];
  odims[n] = R;
  ora_fold(yn, order, odims, n, y);
  free(xn);
  free(yn);
  return ORA_OK;
}

/* -------------------------------------------------- symmetric eigensolver */

/* Eigen-decomposition of a symmetric n x n matrix by the cyclic Jacobi method
 * (row-cyclic order, Golub & Van Loan, Matrix Computations, Sec. 8.5).  It
 * stops when off(A) <= 1e-14 * ||A||_F (far below float32 resolution) or
 * after 60 sweeps.
 * Output: lambda sorted descending, V with the matching orthonormal columns
 * under the sign rule above.  Returns ORA_ENOCONV if the sweep cap is hit. */
int ora_jacobi_eig(int64_t n, const double* S, double* lambda, double* V, int* sweeps_out) {
  double* A = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* W = (double*)malloc(sizeof(double) * (size_t)(n * n));
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!A || !W || !ord) { free(A); free(W); free(ord); return ORA_ENOMEM; }
  memcpy(A, S, sizeof(double) * (size_t)(n * n));
  for (int64_t i = 0; i < n * n; ++i) W[i] = 0.0;
  for (int64_t i = 0; i < n; ++i) W[i + n * i] = 1.0;
  double fro = sqrt(ora_norm2(A, n * n));
  int status = ORA_ENOCONV, sweep = 0;
  for (sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int64_t q = 0; q < n; ++q)
      for (int64_t p = 0; p < n; ++p)
        if (p != q) off += A[p + n * q] * A[p + n * q];
    if (sqrt(off) <= 1e-14 * fro || fro == 0.0) { status = ORA_OK; break; }
    for (int64_t p = 0; p < n - 1; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        double apq = A[p + n * q];
        if (apq == 0.0) continue;
        /* Choose (c, s) so that the (p, q) entry of J^T A J vanishes. */
        double tau = (A[q + n * q] - A[p + n * p]) / (2.0 * apq);
        double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                : -1.0 / (-tau + sqrt(1.0 + tau * tau));
        double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
        /* A <- J^T A J: first the columns p, q ... */
        for (int64_t k = 0; k < n; ++k) {
          double akp = A[k + n * p], akq = A[k + n * q];
          A[k + n * p] = c * akp - s * akq;
          A[k + n * q] = s * akp + c * akq;
        }
        /* ... then the rows p, q. */
        for (int64_t k = 0; k < n; ++k) {
          double apk = A[p + n * k], aqk = A[q + n * k];
          A[p + n * k] = c * apk - s * aqk;
          A[q + n * k] = s * apk + c * aqk;
        }
        /* V <- V J */
        for (int64_t k = 0; k < n; ++k) {
          double vkp = W[k + n * p], vkq = W[k + n * q];
          W[k + n * p] = c * vkp - s * vkq;
          W[k + n * q] = s * vkp + c * vkq;
        }
      }
    }
  }
  if (sweeps_out) *sweeps_out = sweep;
  /* Sort descending by eigenvalue; stable, so ties keep index order. */
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  for (int64_t i = 1; i < n; ++i) { /* insertion sort: plain and stable */
    int64_t key = ord[i];
    int64_t j = i - 1;
    while (j >= 0 && A[ord[j] + n * ord[j]] < A[key + n * key]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = key;
  }
  for (int64_t c = 0; c < n; ++c) {
    int64_t src = ord[c];
    lambda[c] = A[src + n * src];
    int64_t arg = 0;
    double best = -1.0;
    for (int64_t r = 0; r < n; ++r) {
      double a = fabs(W[r + n * src]);
      if (a > best) { best = a; arg = r; }
    }
    double sg = (W[arg + n * src] < 0.0) ? -1.0 : 1.0;
    for (int64_t r = 0; r < n; ++r) V[r + n * c] = sg * W[r + n * src];
  }
  free(A);
  free(W);
  free(ord);
  return status;
}

/* ------------------------------------------------- small dense linear algebra */

/* Cholesky G = C C^T (C lower triangular), r x r.  Returns ORA_ERANK if G is
 * not numerically positive definite. */
int ora_cholesky(int64_t r, const double* G, double* C) {
  for (int64_t i = 0; i < r * r; ++i) C[i] = 0.0;
  for (int64_t j = 0; j < r; ++j) {
    double d = G[j + r * j];
    for (int64_t k = 0; k < j; ++k) d -= C[j + r * k] * C[j + r * k];
    if (!(d > 0.0)) return ORA_ERANK;
    double cjj = sqrt(d);
    C[j + r * j] = cjj;
    for (int64_t i = j + 1; i < r; ++i) {
      double s = G[i + r * j];
      for (int64_t k = 0; k < j; ++k) s -= C[i + r * k] * C[j + r * k];
      C[i + r * j] = s / cjj;
    }
  }
  return ORA_OK;
}

/* X (m x r) <- X G^{-1} with G = C C^T symmetric positive definite:
 * each row x^T is replaced by the solution z^T of G z = x. */
static void chol_solve_rows(int64_t m, int64_t r, const double* C, double* X) {
#pragma omp parallel for schedule(static)
  for (int64_t row = 0; row < m; ++row) {
    double z[1024];
    double* zz = z;
    double* heap = NULL;
    if (r > 1024) { heap = (double*)malloc(sizeof(double) * (size_t)r); zz = heap; }
    for (int64_t i = 0; i < r; ++i) { /* forward: C y = x */
      double s = X[row + m * i];
      for (int64_t k = 0; k < i; ++k) s -= C[i + r * k] * zz[k];
      zz[i] = s / C[i + r * i];
    }
    for (int64_t i = r - 1; i >= 0; --i) { /* backward: C^T z = y */
      double s = zz[i];
      for (int64_t k = i + 1; k < r; ++k) s -= C[k + r * i] * zz[k];
      zz[i] = s / C[i + r * i];
    }
    for (int64_t i = 0; i < r; ++i) X[row + m * i] = zz[i];
    free(heap);
  }
}

/* Householder QR of the m x r matrix M (m >= r): M = Q R with Q m x r having
 * orthonormal columns and R r x r upper triangular with diag(R) > 0
 * (Golub & Van Loan, Sec. 5.2). */
int ora_householder_qr(int64_t m, int64_t r, const double* M, double* Q, double* R) {
  if (m < r) return ORA_EINVAL;
  double* A = (double*)malloc(sizeof(double) * (size_t)(m * r));
  double* vs = (double*)malloc(sizeof(double) * (size_t)(m * r));
  double* beta = (double*)malloc(sizeof(double) * (size_t)r);
  if (!A || !vs || !beta) { free(A); free(vs); free(beta); return ORA_ENOMEM; }
  memcpy(A, M, sizeof(double) * (size_t)(m * r));
  for (int64_t j = 0; j < r; ++j) {
    /* Reflector H = I - beta v v^T mapping A[j:, j] onto a multiple of e_1. */
    double* v = vs + m * j;
    double norm = 0.0;
    for (int64_t i = j; i < m; ++i) norm += A[i + m * j] * A[i + m * j];
    norm = sqrt(norm);
    for (int64_t i = 0; i < m; ++i) v[i] = 0.0;
    double alpha = A[j + m * j];
    double v0 = alpha + ((alpha >= 0.0) ? norm : -norm);
    v[j] = v0;
    for (int64_t i = j + 1; i < m; ++i) v[i] = A[i + m * j];
    double vtv = 0.0;
    for (int64_t i = j; i < m; ++i) vtv += v[i] * v[i];
    beta[j] = (vtv > 0.0) ? 2.0 / vtv : 0.0;
    for (int64_t c = j; c < r; ++c) {
      double s = 0.0;
      for (int64_t i = j; i < m; ++i) s += v[i] * A[i + m * c];
      s *= beta[j];
      for (int64_t i = j; i < m; ++i) A[i + m * c] -= s * v[i];
    }
  }
  /* R is the upper triangle of A; Q = H_0 ... H_{r-1} applied to [I_r; 0]. */
  for (int64_t c = 0; c < r; ++c)
    for (int64_t i = 0; i < r; ++i) R[i + r * c] = (i <= c) ? A[i + m * c] : 0.0;
  for (int64_t c = 0; c < r; ++c)
    for (int64_t i = 0; i < m; ++i) Q[i + m * c] = (i == c) ? 1.0 : 0.0;
  for (int64_t j = r - 1; j >= 0; --j) {
    double* v = vs + m * j;
    for (int64_t c = 0; c < r; ++c) {
      double s = 0.0;
      for (int64_t i = j; i < m; ++i) s += v[i] * Q[i + m * c];
      s *= beta[j];
      for (int64_t i = j; i < m; ++i) Q[i + m * c] -= s * v[i];
    }
  }
  /* Make diag(R) positive: flip row i of R and column i of Q together. */
  for (int64_t i = 0; i < r; ++i) {
    if (R[i + r * i] < 0.0) {
      for (int64_t c = 0; c < r; ++c) R[i + r * c] = -R[i + r * c];
      for (int64_t k = 0; k < m; ++k) Q[k + m * i] = -Q[k + m * i];
    }
  }
  free(A);
  free(vs);
  free(beta);
  return ORA_OK;
}

/* ----------------------------------------------------------- ALS (Alg. 3) */

/* splitmix64 (Steele, Lea and Flood, OOPSLA 2014): the c-th output of the
 * stream whose state starts at `state` is mix(state + c * gamma), c >= 1. */
static uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static uint64_t sm64_at(uint64_t state, uint64_t c) { return sm64_mix(state + c * 0x9E3779B97F4A7C15ULL); }
uint64_t ora_splitmix64_at(uint64_t state, uint64_t c) { return sm64_at(state, c); }

/* ALS initial guess L_0 for mode `mode` (0-based): entry e = i + I*r (column-major)
 * is sqrt(-2 ln u1) cos(2 pi u2), the Box-Muller transform of u1 = (w(2e+1) + 1) 2^-53
 * and u2 = w(2e+2) 2^-53, where w(c) = top 53 bits of the c-th splitmix64 output for
 * the state seed ^ (0x9E3779B97F4A7C15 * (mode + 1)). */
void ora_als_init(uint64_t seed, int mode, int64_t I, int64_t R, double* L0) {
  uint64_t state = seed ^ (0x9E3779B97F4A7C15ULL * (uint64_t)(mode + 1));
  const double two53 = 1.0 / 9007199254740992.0;
  for (int64_t e = 0; e < I * R; ++e) {
    double u1 = ((double)(sm64_at(state, 2 * (uint64_t)e + 1) >> 11) + 1.0) * two53;
    double u2 = (double)(sm64_at(state, 2 * (uint64_t)e + 2) >> 11) * two53;
    L0[e] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  }
}

/* Alg. 3 with exactly `sweeps` iterations on the explicit I x J matrix Y:
 *   R_k     = (Y^T L_k)(L_k^T L_k)^{-1}
 *   L_{k+1} = (Y R_k)(R_k^T R_k)^{-1}
 * Returns L = L_K (I x R) and Rk = R_{K-1} (J x R). */
int ora_als(int64_t I, int64_t J, int64_t R, const double* Y, const double* L0, int sweeps, double* L, double* Rk) {
  double* G = (double*)malloc(sizeof(double) * (size_t)(R * R));
  double* C = (double*)malloc(sizeof(double) * (size_t)(R * R));
  if (!G || !C) { free(G); free(C); return ORA_ENOMEM; }
  memcpy(L, L0, sizeof(double) * (size_t)(I * R));
  int st = ORA_OK;
  for (int k = 0; k < sweeps && st == ORA_OK; ++k) {
    ora_matmul(1, 0, J, R, I, Y, I, L, I, Rk, J);      /* Y^T L_k          */
    ora_matmul(1, 0, R, R, I, L, I, L, I, G, R);       /* L_k^T L_k        */
    st = ora_cholesky(R, G, C);
    if (st != ORA_OK) break;
    chol_solve_rows(J, R, C, Rk);                      /* R_k              */
    ora_matmul(0, 0, I, R, J, Y, I, Rk, J, L, I);      /* Y R_k            */
    ora_matmul(1, 0, R, R, J, Rk, J, Rk, J, G, R);     /* R_k^T R_k        */
    st = ora_cholesky(R, G, C);
    if (st != ORA_OK) break;
    chol_solve_rows(I, R, C, L);                       /* L_{k+1}          */
  }
  free(G);
  free(C);
  return st;
}

/* ----------------------------------------------------- st-HOSVD (Alg. 2) */

/* Mode-wise flexible st-HOSVD.
 *   x          column-major input, dims[0..order)
 *   mode_order permutation of 0..order-1 (the order modes are processed in)
 *   solver     per mode index: 0 = EIG (Gram + eigenvectors + TTM), 1 = ALS
 *   core       R_1 x ... x R_N column-major
 *   factors    U^(1) .. U^(N) in mode-index order, each I_n x R_n, concatenated
 *   discarded  per mode index: energy removed at that step
 *              (EIG: sum of the discarded Gram eigenvalues; ALS: ||Y||^2 - ||Y'||^2) */
int ora_sthosvd(const double* x, int order, const int64_t* dims, const int64_t* ranks, const int* mode_order,
                const int* solver, int als_sweeps, uint64_t seed, double* core, double* factors, double* discarded) {
  if (order < 1 || order > 16) return ORA_EINVAL;
  int64_t cur[16];
  int64_t foff[16];
  int64_t off = 0;
  for (int k = 0; k < order; ++k) {
    cur[k] = dims[k];
    foff[k] = off;
    off += dims[k] * ranks[k];
    if (ranks[k] < 1 || ranks[k] > dims[k]) return ORA_ERANK;
  }
  int64_t total = prod_dims(order, dims);
  double* Y = (double*)malloc(sizeof(double) * (size_t)total);
  if (!Y) return ORA_ENOMEM;
  memcpy(Y, x, sizeof(double) * (size_t)total);
  int st = ORA_OK;
  for (int step = 0; step < order && st == ORA_OK; ++step) {
    int n = mode_order[step];
    int64_t In = cur[n], Rn = ranks[n], len = prod_dims(order, cur), Jn = len / In;
    double* U = factors + foff[n];
    int64_t ndims[16];
    for (int k = 0; k < order; ++k) ndims[k] = cur[k];
    ndims[n] = Rn;
    double* Ynew = (double*)malloc(sizeof(double) * (size_t)(Rn * Jn));
    if (!Ynew) { st = ORA_ENOMEM; break; }
    if (solver[n] == 0) {
      /* EIG branch: S = Y_(n) Y_(n)^T, U = leading eigenvectors, Y <- Y x_n U^T. */
      double* S = (double*)malloc(sizeof(double) * (size_t)(In * In));
      double* lam = (double*)malloc(sizeof(double) * (size_t)In);
      double* V = (double*)malloc(sizeof(double) * (size_t)(In * In));
      if (!S || !lam || !V) { free(S); free(lam); free(V); free(Ynew); st = ORA_ENOMEM; break; }
      st = ora_gram(Y, order, cur, n, S);
      if (st == ORA_OK) st = ora_jacobi_eig(In, S, lam, V, NULL);
      if (st == ORA_OK) {
        memcpy(U, V, sizeof(double) * (size_t)(In * Rn));
        double d = 0.0;
        for (int64_t r = Rn; r < In; ++r) d += lam[r];
        if (discarded) discarded[n] = d;
        st = ora_ttm(Y, order, cur, n, U, Rn, Ynew);
      }
      free(S);
      free(lam);
      free(V);
    } else {
      /* ALS branch: L, R = ALS(Y_(n)); L = Q R^; U = Q; Y_(n) <- R^ R^T. */
      double* Yn = (double*)malloc(sizeof(double) * (size_t)len);
      double* L0 = (double*)malloc(sizeof(double) * (size_t)(In * Rn));
      double* L = (double*)malloc(sizeof(double) * (size_t)(In * Rn));
      double* Rk = (double*)malloc(sizeof(double) * (size_t)(Jn * Rn));
      double* Rh = (double*)malloc(sizeof(double) * (size_t)(Rn * Rn));
      double* Yn2 = (double*)malloc(sizeof(double) * (size_t)(Rn * Jn));
      if (!Yn || !L0 || !L || !Rk || !Rh || !Yn2) st = ORA_ENOMEM;
      if (st == ORA_OK) {
        ora_unfold(Y, order, cur, n, Yn);
        ora_als_init(seed, n, In, Rn, L0);
        st = ora_als(In, Jn, Rn, Yn, L0, als_sweeps, L, Rk);
      }
      if (st == ORA_OK) st = ora_householder_qr(In, Rn, L, U, Rh);
      if (st == ORA_OK) {
        ora_matmul(0, 1, Rn, Jn, Rn, Rh, Rn, Rk, Jn, Yn2, Rn);
        ora_fold(Yn2, order, ndims, n, Ynew);
        if (discarded) discarded[n] = ora_norm2(Y, len) - ora_norm2(Ynew, Rn * Jn);
      }
      free(Yn); free(L0); free(L); free(Rk); free(Rh); free(Yn2);
    }
    free(Y);
    Y = Ynew;
    cur[n] = Rn;
  }
  if (st == ORA_OK) memcpy(core, Y, sizeof(double) * (size_t)prod_dims(order, ranks));
  free(Y);
  return st;
}

/* X_hat = G x_1 U^(1) ... x_N U^(N) (Sec. II-B), applied one mode at a time by
 * explicit matricization: Z_(n) <- U^(n) Z_(n). */
int ora_reconstruct(const double* core, int order, const int64_t* ranks, const double* factors, const int64_t* dims,
                    double* xhat) {
  int64_t cur[16];
  int64_t foff[16], off = 0;
  for (int k = 0; k < order; ++k) { cur[k] = ranks[k]; foff[k] = off; off += dims[k] * ranks[k]; }
  int64_t len = prod_dims(order, ranks);
  double* Z = (double*)malloc(sizeof(double) * (size_t)len);
  if (!Z) return ORA_ENOMEM;
  memcpy(Z, core, sizeof(double) * (size_t)len);
  for (int n = 0; n < order; ++n) {
    int64_t Rn = cur[n], Jn = len / Rn, In = dims[n];
    double* zn = (double*)malloc(sizeof(double) * (size_t)len);
    double* yn = (double*)malloc(sizeof(double) * (size_t)(In * Jn));
    double* Znew = (double*)malloc(sizeof(double) * (size_t)(In * Jn));
    if (!zn || !yn || !Znew) { free(zn); free(yn); free(Znew); free(Z); return ORA_ENOMEM; }
    ora_unfold(Z, order, cur, n, zn);
    ora_matmul(0, 0, In, Jn, Rn, factors + foff[n], In, zn, Rn, yn, In);
    cur[n] = In;
    ora_fold(yn, order, cur, n, Znew);
    free(zn);
    free(yn);
    free(Z);
    Z = Znew;
    len = In * Jn;
  }
  memcpy(xhat, Z, sizeof(double) * (size_t)len);
  free(Z);
  return ORA_OK;
}

/* -------------------------------------------- st-HOSVD-SVD (Alg. 1), tiny */

/* Left singular vectors of the m x p matrix M by one-sided (Hestenes) Jacobi.
 * The method rotates the m columns of B = M^T (B <- B J) until they are
 * mutually orthogonal, accumulating the rotations in the orthogonal m x m
 * matrix W, so that M^T W = B.  Then B = Q diag(sigma) and M = W diag(sigma) Q^T:
 * the columns of W are the left singular vectors.  Used only as an independent
 * cross-check on tiny inputs.  Returns sigma (descending, min(m,p) values) and
 * Uout (m x min(m,p)) under the eigenvector sign rule. */
int ora_jacobi_svd_left(int64_t m, int64_t p, const double* M, double* sigma, double* Uout) {
  double* B = (double*)malloc(sizeof(double) * (size_t)(p * m));
  double* W = (double*)malloc(sizeof(double) * (size_t)(m * m));
  double* sv = (double*)malloc(sizeof(double) * (size_t)m);
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
  if (!B || !W || !sv || !ord) { free(B); free(W); free(sv); free(ord); return ORA_ENOMEM; }
  for (int64_t i = 0; i < m; ++i)
    for (int64_t j = 0; j < p; ++j) B[j + p * i] = M[i + m * j];
  for (int64_t i = 0; i < m * m; ++i) W[i] = 0.0;
  for (int64_t i = 0; i < m; ++i) W[i + m * i] = 1.0;
  double fro2 = 0.0;
  for (int64_t i = 0; i < p * m; ++i) fro2 += B[i] * B[i];
  int status = ORA_ENOCONV;
  for (int sweep = 0; sweep < 80; ++sweep) {
    int rotated = 0;
    for (int64_t a = 0; a < m - 1; ++a) {
      for (int64_t b = a + 1; b < m; ++b) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t k = 0; k < p; ++k) {
          alpha += B[k + p * a] * B[k + p * a];
          beta += B[k + p * b] * B[k + p * b];
          gamma += B[k + p * a] * B[k + p * b];
        }
        /* Columns already orthogonal to working precision, or one of them
         * negligible against the whole matrix (rank-deficient M): no rotation. */
        if (fabs(gamma) <= 1e-15 * sqrt(alpha * beta) || gamma == 0.0) continue;
        if (alpha <= 1e-28 * fro2 || beta <= 1e-28 * fro2) continue;
        rotated = 1;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = ((zeta >= 0.0) ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int64_t k = 0; k < p; ++k) {
          double x = B[k + p * a], y = B[k + p * b];
          B[k + p * a] = c * x - s * y;
          B[k + p * b] = s * x + c * y;
        }
        for (int64_t k = 0; k < m; ++k) {
          double x = W[k + m * a], y = W[k + m * b];
          W[k + m * a] = c * x - s * y;
          W[k + m * b] = s * x + c * y;
        }
      }
    }
    if (!rotated) { status = ORA_OK; break; }
  }
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t k = 0; k < p; ++k) s += B[k + p * i] * B[k + p * i];
    sv[i] = sqrt(s);
    ord[i] = i;
  }
  for (int64_t i = 1; i < m; ++i) {
    int64_t key = ord[i];
    int64_t j = i - 1;
    while (j >= 0 && sv[ord[j]] < sv[key]) { ord[j + 1] = ord[j]; --j; }
    ord[j + 1] = key;
  }
  int64_t q = (m < p) ? m : p;
  for (int64_t c = 0; c < q; ++c) {
    int64_t src = ord[c];
    sigma[c] = sv[src];
    int64_t arg = 0;
    double best = -1.0;
    for (int64_t r = 0; r < m; ++r) {
      double v = fabs(W[r + m * src]);
      if (v > best) { best = v; arg = r; }
    }
    double sg = (W[arg + m * src] < 0.0) ? -1.0 : 1.0;
    for (int64_t r = 0; r < m; ++r) Uout[r + m * c] = sg * W[r + m * src];
  }
  free(B); free(W); free(sv); free(ord);
  return status;
}

/* Alg. 1 (st-HOSVD-SVD) with the factor taken from the SVD of Y_(n) and the core
 * update Y_(n) <- Sigma V^T, written as U^T Y_(n) (equal for the leading R
 * singular triplets).  Tiny inputs only. */
int ora_sthosvd_svd(const double* x, int order, const int64_t* dims, const int64_t* ranks, const int* mode_order,
                    double* core, double* factors) {
  int64_t cur[16], foff[16], off = 0;
  for (int k = 0; k < order; ++k) { cur[k] = dims[k]; foff[k] = off; off += dims[k] * ranks[k]; }
  int64_t total = prod_dims(order, dims);
  double* Y = (double*)malloc(sizeof(double) * (size_t)total);
  if (!Y) return ORA_ENOMEM;
  memcpy(Y, x, sizeof(double) * (size_t)total);
  int st = ORA_OK;
  for (int step = 0; step < order && st == ORA_OK; ++step) {
    int n = mode_order[step];
    int64_t In = cur[n], Rn = ranks[n], len = prod_dims(order, cur), Jn = len / In;
    int64_t q = (In < Jn) ? In : Jn;
    double* Yn = (double*)malloc(sizeof(double) * (size_t)len);
    double* sig = (double*)malloc(sizeof(double) * (size_t)In);
    double* Ul = (double*)malloc(sizeof(double) * (size_t)(In * In));
    double* Ynew = (double*)malloc(sizeof(double) * (size_t)(Rn * Jn));
    if (!Yn || !sig || !Ul || !Ynew) { free(Yn); free(sig); free(Ul); free(Ynew); st = ORA_ENOMEM; break; }
    ora_unfold(Y, order, cur, n, Yn);
    st = ora_jacobi_svd_left(In, Jn, Yn, sig, Ul);
    if (st == ORA_OK && Rn > q) st = ORA_ERANK;
    if (st == ORA_OK) {
      memcpy(factors + foff[n], Ul, sizeof(double) * (size_t)(In * Rn));
      st = ora_ttm(Y, order, cur, n, factors + foff[n], Rn, Ynew);
    }
    free(Yn); free(sig); free(Ul);
    free(Y);
    Y = Ynew;
    cur[n] = Rn;
  }
  if (st == ORA_OK) memcpy(core, Y, sizeof(double) * (size_t)prod_dims(order, ranks));
  free(Y);
  return st;
}
