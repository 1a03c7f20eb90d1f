"""Seeded synthetic inputs for the st-HOSVD path.

This module only *makes* input tensors and shape lists; it holds none of the
decomposition's arithmetic and is imported by both the tests/bench (which feed
the CUDA library) and the CPU oracle checks, so that both sides see identical
bytes.

Conventions
-----------
* A tensor of dims (d_1, ..., d_N) is stored column-major (first index fastest,
  Sec. V of the paper).  The flat float32 buffer returned here is exactly that
  layout; a C-contiguous array of shape (d_N, ..., d_1) views the same bytes.
* All randomness comes from ``numpy.random.Generator(PCG64(seed))`` drawn in
  float64 and rounded to float32 once.

Workload recipes (the paper's tensors, Table II, are not available; these
synthetic stand-ins carry the shapes and structure of its workloads):

* ``random_tucker``: core G ~ N(0,1) of size R_1 x ... x R_N, factors U_n = Q of
  the QR of an N(0,1) I_n x R_n matrix, X = G x_1 U_1 ... x_N U_N + noise * N(0,1).
* ``decaying_tucker``: same, but the core is Z x_1 D ... x_N D with
  Z ~ N(0,1) of size (2 R_max)^N and D = diag(k^-1.5), so each mode's singular
  values decay about like k^-1.5; the signal is scaled to RMS 1 per element.
* ``selector_shapes``: the learned-selector shape set (order 3..5, dims
  log-uniform on [16, 1024], at most 2 GB of float32, rank ratios on
  [0.02, 0.5]).
* ``batched_shapes``: 4096 order-3 tensors, dims uniform in [16, 96], ranks
  uniform in [4, 16]; ``batched_tensor`` draws member t as a random Tucker
  tensor (noise 1e-3) from the stream (seed, t).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng", "random_tucker", "decaying_tucker", "feasible_ranks",
    "selector_shapes", "batched_shapes", "batched_tensor", "to_colmajor_f32", "from_colmajor",
]


def rng(seed) -> np.random.Generator:
    """PCG64 stream for an int seed or a tuple of ints (e.g. (batch seed, tensor index))."""
    if isinstance(seed, (tuple, list)):
        seed = np.random.SeedSequence([int(v) for v in seed])
    return np.random.Generator(np.random.PCG64(seed))


def to_colmajor_f32(x: np.ndarray) -> np.ndarray:
    """Flatten an array indexed (i_1, ..., i_N) into the column-major float32 buffer."""
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel(order="F").astype(np.float32))


def from_colmajor(flat: np.ndarray, dims) -> np.ndarray:
    """View a column-major flat buffer as an array indexed (i_1, ..., i_N)."""
    return np.asarray(flat).reshape(tuple(int(d) for d in dims), order="F")


def _orthonormal(g: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    q, r = np.linalg.qr(g.standard_normal((rows, cols)))
    # Fix the sign so the factor is a deterministic function of the draw.
    return q * np.sign(np.where(np.diag(r) == 0, 1.0, np.diag(r)))[None, :]


def _expand(core: np.ndarray, factors) -> np.ndarray:
    x = core
    for n, u in enumerate(factors):
        x = np.moveaxis(np.tensordot(u, x, axes=(1, n)), 0, n)
    return x


def random_tucker(dims, ranks, noise: float = 1e-3, seed: int = 0):
    """Random Tucker tensor plus Gaussian noise.

    Returns (x_flat_f32, core_true, factors_true): the column-major float32
    input buffer and the float64 ground truth used to build it.
    """
    dims = [int(d) for d in dims]
    ranks = [int(r) for r in ranks]
    g = rng(seed)
    core = g.standard_normal(ranks)
    factors = [_orthonormal(g, d, r) for d, r in zip(dims, ranks)]
    x = _expand(core, factors)
    if noise:
        x = x + noise * g.standard_normal(dims)
    return to_colmajor_f32(x), core, factors


def decaying_tucker(dims, r_max: int, noise: float = 1e-3, seed: int = 0):
    """Tucker tensor whose mode-n singular values decay about like k^-1.5."""
    dims = [int(d) for d in dims]
    g = rng(seed)
    k = 2 * int(r_max)
    kk = [min(k, d) for d in dims]
    z = g.standard_normal(kk)
    for n, kn in enumerate(kk):
        d = np.arange(1, kn + 1, dtype=np.float64) ** -1.5
        shape = [1] * len(kk)
        shape[n] = kn
        z = z * d.reshape(shape)
    factors = [_orthonormal(g, d, kn) for d, kn in zip(dims, kk)]
    x = _expand(z, factors)
    x *= 1.0 / math.sqrt(np.mean(x * x))
    if noise:
        x = x + noise * g.standard_normal(dims)
    return to_colmajor_f32(x), z, factors


def feasible_ranks(dims, ranks):
    """Clamp ranks to 1 <= R_n <= I_n and R_n <= prod_{k != n} R_k.

    The paper is silent on feasibility; a Tucker core with R_n larger than the
    product of the other ranks would have a rank-deficient unfolding.
    """
    r = [max(1, min(int(x), int(d))) for x, d in zip(ranks, dims)]
    changed = True
    while changed:
        changed = False
        for n in range(len(r)):
            others = 1
            for k, v in enumerate(r):
                if k != n:
                    others *= v
            if r[n] > others:
                r[n] = others
                changed = True
    return r


def selector_shapes(count: int = 256, seed: int = 0, max_bytes: float = 2e9):
    """Shapes for the learned selector: [(dims, ranks)], order 3..5."""
    g = rng(seed)
    out = []
    while len(out) < count:
        order = int(g.integers(3, 6))
        while True:
            dims = [int(round(math.exp(g.uniform(math.log(16), math.log(1024))))) for _ in range(order)]
            if float(np.prod(dims, dtype=np.float64)) * 4.0 <= max_bytes:
                break
        rho = g.uniform(0.02, 0.5, size=order)
        ranks = [int(round(p * d)) for p, d in zip(rho, dims)]
        out.append((dims, feasible_ranks(dims, ranks)))
    return out


def batched_shapes(count: int = 4096, seed: int = 0, lo: int = 16, hi: int = 96, rlo: int = 4, rhi: int = 16):
    """Order-3 shapes for the batched workload: [(dims, ranks)]."""
    g = rng(seed)
    out = []
    for _ in range(count):
        dims = [int(v) for v in g.integers(lo, hi + 1, size=3)]
        ranks = [int(v) for v in g.integers(rlo, rhi + 1, size=3)]
        out.append((dims, feasible_ranks(dims, ranks)))
    return out


def batched_tensor(shapes, t: int, seed: int = 0, noise: float = 1e-3):
    """Tensor t of a batch: random Tucker of shapes[t] from the stream (seed, t).

    Any subset of a batch regenerates bit-identically, so the oracle can check
    sampled members of a large batch.
    """
    dims, ranks = shapes[t]
    return random_tucker(dims, ranks, noise=noise, seed=(seed, t))[0]

