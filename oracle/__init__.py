"""CPU oracle for the mode-wise flexible st-HOSVD (a-Tucker, arXiv 2010.10131).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never links, loads or calls it, and it imports nothing from the CUDA package.

The heavy parts are plain C in ``atk_oracle.c`` (float64, explicit
matricization, textbook cyclic Jacobi, Householder QR, Cholesky, a literal
Alg. 3), loaded through ctypes.  This module only marshals numpy arrays.  The
learned-selector MLP reference lives in ``oracle.mlp``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, library routines it does not itself call, brute force on
tiny inputs, or invariants of the method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "atk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_atk_oracle.so")
_lib = None

OK, EINVAL, ERANK, ENOMEM, ENOCONV = 0, -1, -2, -3, -5


def build(force: bool = False) -> str:
    """Compile the C oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        sig = {
            "ora_unfold": (None, [d, i32, d, i32, d]),
            "ora_fold": (None, [d, i32, d, i32, d]),
            "ora_matmul": (None, [i32, i32, i64, i64, i64, d, i64, d, i64, d, i64]),
            "ora_norm2": (ctypes.c_double, [d, i64]),
            "ora_gram": (i32, [d, i32, d, i32, d]),
            "ora_ttm": (i32, [d, i32, d, i32, d, i64, d]),
            "ora_jacobi_eig": (i32, [i64, d, d, d, d]),
            "ora_cholesky": (i32, [i64, d, d]),
            "ora_householder_qr": (i32, [i64, i64, d, d, d]),
            "ora_als_init": (None, [u64, i32, i64, i64, d]),
            "ora_als": (i32, [i64, i64, i64, d, d, i32, d, d]),
            "ora_sthosvd": (i32, [d, i32, d, d, d, d, i32, u64, d, d, d]),
            "ora_reconstruct": (i32, [d, i32, d, d, d, d]),
            "ora_jacobi_svd_left": (i32, [i64, i64, d, d, d]),
            "ora_sthosvd_svd": (i32, [d, i32, d, d, d, d, d]),
            "ora_splitmix64_at": (u64, [u64, u64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64).ravel())


def _check(st: int, what: str):
    if st != OK:
        raise RuntimeError(f"oracle {what} failed with status {st}")


# ----------------------------------------------------------------- tensor ops

def unfold(x_flat, dims, n: int) -> np.ndarray:
    """Mode-n matricization X_(n) (I_n x J_n), returned as a (I_n, J_n) array."""
    dims = _i64(dims)
    x = _f64(x_flat)
    out = np.empty(x.size, dtype=np.float64)
    lib().ora_unfold(_p(x), len(dims), _p(dims), int(n), _p(out))
    return out.reshape((int(dims[n]), -1), order="F")


def fold(xn: np.ndarray, dims, n: int) -> np.ndarray:
    dims = _i64(dims)
    a = _f64(np.asarray(xn, dtype=np.float64).ravel(order="F"))
    out = np.empty(a.size, dtype=np.float64)
    lib().ora_fold(_p(a), len(dims), _p(dims), int(n), _p(out))
    return out


def matmul(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Plain loop product of two 2-D arrays (column-major inside the oracle)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, k = a.shape
    k2, p = b.shape
    assert k == k2
    af = _f64(a.ravel(order="F"))
    bf = _f64(b.ravel(order="F"))
    c = np.empty(m * p, dtype=np.float64)
    lib().ora_matmul(0, 0, m, p, k, _p(af), m, _p(bf), k, _p(c), m)
    return c.reshape((m, p), order="F")


def norm2(x) -> float:
    x = _f64(x)
    return float(lib().ora_norm2(_p(x), x.size))


def gram(x_flat, dims, n: int) -> np.ndarray:
    """S = Y_(n) Y_(n)^T (I_n x I_n)."""
    dims = _i64(dims)
    x = _f64(x_flat)
    s = np.empty(int(dims[n]) ** 2, dtype=np.float64)
    _check(lib().ora_gram(_p(x), len(dims), _p(dims), int(n), _p(s)), "gram")
    return s.reshape((int(dims[n]),) * 2, order="F")


def ttm(x_flat, dims, n: int, U: np.ndarray) -> np.ndarray:
    """Y = X x_n U^T with U of shape (I_n, R): flat column-major output."""
    dims = _i64(dims)
    x = _f64(x_flat)
    U = np.asarray(U, dtype=np.float64)
    R = U.shape[1]
    uf = _f64(U.ravel(order="F"))
    out = np.empty(x.size // int(dims[n]) * R, dtype=np.float64)
    _check(lib().ora_ttm(_p(x), len(dims), _p(dims), int(n), _p(uf), R, _p(out)), "ttm")
    return out


def jacobi_eig(S: np.ndarray):
    """(lambda descending, V, sweeps) of a symmetric matrix by cyclic Jacobi."""
    S = np.asarray(S, dtype=np.float64)
    n = S.shape[0]
    sf = _f64(S.ravel(order="F"))
    lam = np.empty(n)
    V = np.empty(n * n)
    sw = ctypes.c_int(0)
    _check(lib().ora_jacobi_eig(n, _p(sf), _p(lam), _p(V), ctypes.cast(ctypes.byref(sw), ctypes.c_void_p)), "jacobi")
    return lam, V.reshape((n, n), order="F"), sw.value


def cholesky(G: np.ndarray) -> np.ndarray:
    G = np.asarray(G, dtype=np.float64)
    r = G.shape[0]
    gf = _f64(G.ravel(order="F"))
    c = np.empty(r * r)
    _check(lib().ora_cholesky(r, _p(gf), _p(c)), "cholesky")
    return c.reshape((r, r), order="F")


def householder_qr(M: np.ndarray):
    M = np.asarray(M, dtype=np.float64)
    m, r = M.shape
    mf = _f64(M.ravel(order="F"))
    q = np.empty(m * r)
    rr = np.empty(r * r)
    _check(lib().ora_householder_qr(m, r, _p(mf), _p(q), _p(rr)), "qr")
    return q.reshape((m, r), order="F"), rr.reshape((r, r), order="F")


def splitmix64_at(state: int, c: int) -> int:
    return int(lib().ora_splitmix64_at(ctypes.c_uint64(state & 0xFFFFFFFFFFFFFFFF), ctypes.c_uint64(c)))


def als_init(seed: int, mode: int, I: int, R: int) -> np.ndarray:
    out = np.empty(I * R)
    lib().ora_als_init(ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(mode), I, R, _p(out))
    return out.reshape((I, R), order="F")


def als(Y: np.ndarray, L0: np.ndarray, sweeps: int = 5):
    """Alg. 3 on an explicit I x J matrix: returns (L_K, R_{K-1})."""
    Y = np.asarray(Y, dtype=np.float64)
    I, J = Y.shape
    R = L0.shape[1]
    yf = _f64(Y.ravel(order="F"))
    lf = _f64(np.asarray(L0).ravel(order="F"))
    L = np.empty(I * R)
    Rk = np.empty(J * R)
    _check(lib().ora_als(I, J, R, _p(yf), _p(lf), int(sweeps), _p(L), _p(Rk)), "als")
    return L.reshape((I, R), order="F"), Rk.reshape((J, R), order="F")


def sthosvd(x_flat, dims, ranks, mode_order=None, solver=None, als_sweeps: int = 5, seed: int = 0):
    """Alg. 2.  Returns dict(core=flat, factors=[I_n x R_n], discarded=[...])."""
    dims = _i64(dims)
    ranks = _i64(ranks)
    N = len(dims)
    mo = np.ascontiguousarray(np.arange(N) if mode_order is None else mode_order, dtype=np.int32)
    sv = np.ascontiguousarray(np.zeros(N) if solver is None else solver, dtype=np.int32)
    x = _f64(x_flat)
    core = np.empty(int(np.prod(ranks)))
    fac = np.empty(int(np.sum(dims * ranks)))
    disc = np.empty(N)
    st = lib().ora_sthosvd(_p(x), N, _p(dims), _p(ranks), _p(mo), _p(sv), int(als_sweeps),
                           ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _p(core), _p(fac), _p(disc))
    _check(st, "sthosvd")
    factors, off = [], 0
    for d, r in zip(dims, ranks):
        factors.append(fac[off:off + d * r].reshape((int(d), int(r)), order="F").copy())
        off += int(d * r)
    return {"core": core, "factors": factors, "discarded": disc}


def reconstruct(core, ranks, factors, dims) -> np.ndarray:
    dims = _i64(dims)
    ranks = _i64(ranks)
    c = _f64(core)
    fac = _f64(np.concatenate([np.asarray(u, dtype=np.float64).ravel(order="F") for u in factors]))
    out = np.empty(int(np.prod(dims)))
    _check(lib().ora_reconstruct(_p(c), len(dims), _p(ranks), _p(fac), _p(dims), _p(out)), "reconstruct")
    return out


def relerr(x_flat, core, ranks, factors, dims) -> float:
    """||X - X_hat||_F / ||X||_F (Sec. VI-B) by explicit reconstruction."""
    x = _f64(x_flat)
    xh = reconstruct(core, ranks, factors, dims)
    return float(np.sqrt(norm2(x - xh) / norm2(x)))


def jacobi_svd_left(M: np.ndarray):
    M = np.asarray(M, dtype=np.float64)
    m, p = M.shape
    q = min(m, p)
    mf = _f64(M.ravel(order="F"))
    s = np.empty(m)
    U = np.empty(m * m)
    _check(lib().ora_jacobi_svd_left(m, p, _p(mf), _p(s), _p(U)), "jacobi_svd")
    return s[:q], U[: m * q].reshape((m, q), order="F")


def sthosvd_svd(x_flat, dims, ranks, mode_order=None):
    """Alg. 1 (SVD solver), tiny inputs only."""
    dims = _i64(dims)
    ranks = _i64(ranks)
    N = len(dims)
    mo = np.ascontiguousarray(np.arange(N) if mode_order is None else mode_order, dtype=np.int32)
    x = _f64(x_flat)
    core = np.empty(int(np.prod(ranks)))
    fac = np.empty(int(np.sum(dims * ranks)))
    _check(lib().ora_sthosvd_svd(_p(x), N, _p(dims), _p(ranks), _p(mo), _p(core), _p(fac)), "sthosvd_svd")
    factors, off = [], 0
    for d, r in zip(dims, ranks):
        factors.append(fac[off:off + d * r].reshape((int(d), int(r)), order="F").copy())
        off += int(d * r)
    return {"core": core, "factors": factors}


def projector_distance(U: np.ndarray, V: np.ndarray) -> float:
    """||U U^T - V V^T||_F (sign- and rotation-free subspace distance)."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    return float(np.linalg.norm(U @ U.T - V @ V.T))
