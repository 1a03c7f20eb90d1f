"""Python binding of the B300 mode-wise flexible st-HOSVD library (a-Tucker).

Argument marshalling only: every step of the decomposition runs in the CUDA
library ``_atucker.so`` (built from ``csrc/`` for sm_103a).  The functions
named ``atucker_*`` mirror the C ABI in ``include/atucker.h`` one to one.  The
lower-case helpers take torch CUDA tensors.  PyTorch supplies device memory and
streams only.  If the shared library is missing or cannot be loaded, every call
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

__all__ = [
    "lib", "abi_symbols", "AtuckerError", "Plan", "Batch", "sthosvd", "gram", "ttm", "ttm_gram", "eig", "als_mode",
    "EIG", "ALS", "FP32", "TF32", "BF16", "BF16X3", "FP8E4M3", "FP32C", "EIG_ROT_FP32", "EIG_ROT_FP64",
]

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
LIB_PATH = os.path.join(_PKG, "_atucker.so")
HEADER = os.path.join(_ROOT, "include", "atucker.h")

OK, EINVAL, ERANK, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
EIG, ALS = 0, 1
FP32, TF32, BF16, BF16X3, FP8E4M3, FP32C = 0, 1, 2, 3, 4, 5
EIG_ROT_FP32, EIG_ROT_FP64 = 0, 1
OPT_EIG_ARITH, OPT_SYNC, OPT_JACOBI_MAX_SWEEPS, OPT_TIMING, OPT_EIG_METHOD, OPT_GRAM_REFINE = 1, 2, 3, 4, 5, 6
OPT_WAIT_LIMIT, OPT_EXPLICIT_UNFOLD, OPT_FUSE_TTM_GRAM = 7, 8, 9
EIG_AUTO, EIG_FULL_JACOBI, EIG_SUBSPACE = 0, 1, 2
BATCH_OPT_VARIANT, BATCH_OPT_GRAPH, BATCH_OPT_SYNC, BATCH_OPT_JACOBI_MAX_SWEEPS = 1, 2, 3, 4
AUTO = -1
CLASS_EIG, CLASS_EIG_SMALL, CLASS_EIG_JACOBI, CLASS_EIG_JACOBI_SMALL, CLASS_ALS, NUM_CLASSES = 0, 1, 2, 3, 4, 5
CLASS_NAMES = ("EIG", "EIG-small-tile", "EIG-Jacobi", "EIG-Jacobi-small-tile", "ALS")
SELECTOR_FEATURES, SELECTOR_HIDDEN = 12, 64
PHASES = ("gram", "gram_reduce", "eig", "ttm", "als", "norms", "total", "gram_launches", "launches", "runs")
_STATUS = {EINVAL: "EINVAL", ERANK: "ERANK", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ENOCONV: "ENOCONV",
           ETIMEOUT: "ETIMEOUT", EUNSUPPORTED: "EUNSUPPORTED"}


class AtuckerError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp, _i64, _i32, _u64, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
_SIGS = {
    "atucker_plan_create": (_i32, [ctypes.POINTER(_vp), _i32, _vp, _vp, _vp, _vp, _i32, _i32, _u64, _vp]),
    "atucker_plan_set_option": (_i32, [_vp, _i32, _i64]),
    "atucker_sthosvd": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "atucker_sthosvd_host": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "atucker_sthosvd_many": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "atucker_sthosvd_host_many": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "atucker_plan_sync": (_i32, [_vp]),
    "atucker_plan_timings": (_i32, [_vp, _vp, _i32]),
    "atucker_plan_destroy": (None, [_vp]),
    "atucker_sthosvd_oneshot": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "atucker_last_error": (ctypes.c_char_p, []),
    "atucker_set_device_alloc_limit": (_i32, [_u64]),
    "atucker_version": (ctypes.c_char_p, []),
    "atucker_gram": (_i32, [_vp, _i64, _i64, _i64, _i32, _vp, _vp]),
    "atucker_gram_noalloc": (_i32, [_vp, _i64, _i64, _i64, _vp, _vp]),
    "atucker_ttm": (_i32, [_vp, _i64, _i64, _i64, _vp, _i64, _i32, _vp, _vp]),
    "atucker_ttm_gram": (_i32, [_vp, _i64, _i64, _i64, _vp, _i64, _i64, _i64, _vp, _vp, _vp]),
    "atucker_eig": (_i32, [_vp, _i64, _i64, _i32, _i32, _vp, _vp, _vp, _vp]),
    "atucker_als_mode": (_i32, [_vp, _i64, _i64, _i64, _i64, _vp, _u64, _i32, _i32, _i32, _vp, _vp, _vp]),
    "atucker_batch_create": (_i32, [ctypes.POINTER(_vp), _i32, _vp, _vp, _vp]),
    "atucker_batch_set_option": (_i32, [_vp, _i32, _i64]),
    "atucker_batch_run": (_i32, [_vp, _vp, _vp, _vp]),
    "atucker_batch_sync": (_i32, [_vp]),
    "atucker_batch_tune": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "atucker_batch_get_variant": (_i32, [_vp, _vp]),
    "atucker_batch_variants": (_i32, [_vp, _vp, _vp]),
    "atucker_batch_destroy": (None, [_vp]),
    "atucker_plan_create_classes": (_i32, [ctypes.POINTER(_vp), _i32, _vp, _vp, _vp, _vp, _i32, _i32, _u64, _vp]),
    "atucker_plan_classes": (_i32, [_vp, _vp]),
    "atucker_plan_mode_timings": (_i32, [_vp, _vp, _i32]),
    "atucker_mode_features": (_i32, [_i32, _vp, _vp, _vp, _vp]),
    "atucker_mlp_param_count": (_i64, [_i32, _i32, _i32]),
    "atucker_selector_set": (_i32, [_vp, _i64]),
    "atucker_selector_clear": (None, []),
    "atucker_selector_set_tree": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "atucker_selector_predict": (_i32, [_vp, _i32, _vp, _vp]),
    "atucker_mlp_forward": (_i32, [_vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp]),
    "atucker_mlp_loss_grad": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "atucker_mlp_train": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _vp, _vp, _i32, _i32, ctypes.c_float, _vp,
                                 _vp]),
}


def abi_symbols() -> list[str]:
    """Every function name declared in include/atucker.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(atucker_[a-z0-9_]+)\s*\(", text)))


def lib(build_if_missing: bool = True):
    """Load the CUDA library (raises if it cannot be built or loaded)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            if not build_if_missing:
                raise ImportError(f"CUDA library not built: {LIB_PATH}")
            from . import build as _build
            _build.build()
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(handle, name)
            f.restype = res
            f.argtypes = args
        _lib = handle
    return _lib


def _check(status: int, what: str):
    if status != OK:
        msg = lib().atucker_last_error()
        raise AtuckerError(status, what, msg.decode() if msg else "")


# ------------------------------------------------------------ same-name wrappers
def __getattr__(name):
    if name.startswith("atucker_") and name in _SIGS:
        return getattr(lib(), name)
    raise AttributeError(name)


# ------------------------------------------------------------- torch helpers
def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _i64arr(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


def _i32arr(vals):
    return (ctypes.c_int * len(vals))(*[int(v) for v in vals])


def _dev(t, dtype):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"expected a contiguous CUDA tensor of dtype {dtype}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A reusable st-HOSVD plan (atucker_plan_create) bound to one shape."""

    def __init__(self, dims, ranks, mode_order=None, solver=None, precision: int = FP32, als_sweeps: int = 5,
                 seed: int = 0, stream=None, eig_arith: int | None = None, sync: bool = False,
                 eig_method: int | None = None, classes=None, gram_refine: int | None = None):
        """solver: per-mode EIG / ALS / AUTO (learned selector); classes: per-mode
        atucker_mode_class values instead (atucker_plan_create_classes)."""
        self.dims = [int(d) for d in dims]
        self.ranks = [int(r) for r in ranks]
        self.order = len(self.dims)
        self._h = ctypes.c_void_p(None)
        self.stream = stream
        mo = _i32arr(mode_order) if mode_order is not None else None
        if classes is not None:
            _check(lib().atucker_plan_create_classes(ctypes.byref(self._h), self.order, _i64arr(self.dims),
                                                     _i64arr(self.ranks), mo, _i32arr(classes), int(precision),
                                                     int(als_sweeps), int(seed) & (2**64 - 1), _stream_ptr(stream)),
                   "atucker_plan_create_classes")
        else:
            sv = _i32arr(solver) if solver is not None else None
            _check(lib().atucker_plan_create(ctypes.byref(self._h), self.order, _i64arr(self.dims),
                                             _i64arr(self.ranks), mo, sv, int(precision), int(als_sweeps),
                                             int(seed) & (2**64 - 1), _stream_ptr(stream)), "atucker_plan_create")
        if eig_arith is not None:
            _check(lib().atucker_plan_set_option(self._h, OPT_EIG_ARITH, int(eig_arith)), "set_option")
        if sync:
            _check(lib().atucker_plan_set_option(self._h, OPT_SYNC, 1), "set_option")
        if eig_method is not None:
            _check(lib().atucker_plan_set_option(self._h, OPT_EIG_METHOD, int(eig_method)), "set_option")
        if gram_refine is not None:
            _check(lib().atucker_plan_set_option(self._h, OPT_GRAM_REFINE, int(gram_refine)), "set_option")

    @property
    def core_numel(self):
        n = 1
        for r in self.ranks:
            n *= r
        return n

    @property
    def factors_numel(self):
        return sum(d * r for d, r in zip(self.dims, self.ranks))

    def run(self, x, core=None, factors=None, discarded=None):
        torch = _torch()
        if core is None:
            core = torch.empty(self.core_numel, device=x.device, dtype=torch.float32)
        if factors is None:
            factors = torch.empty(self.factors_numel, device=x.device, dtype=torch.float32)
        dptr = _dev(discarded, torch.float64) if discarded is not None else None
        _check(lib().atucker_sthosvd(self._h, _dev(x, torch.float32), _dev(core, torch.float32),
                                     _dev(factors, torch.float32), dptr), "atucker_sthosvd")
        return core, factors

    def run_host(self, x_host, core_host, factors_host, discarded_host=None):
        """Host-buffer form (atucker_sthosvd_host); tensors must be contiguous CPU tensors."""
        torch = _torch()
        for t in (x_host, core_host, factors_host):
            assert t.device.type == "cpu" and t.is_contiguous() and t.dtype == torch.float32
        d = ctypes.c_void_p(discarded_host.data_ptr()) if discarded_host is not None else None
        _check(lib().atucker_sthosvd_host(self._h, ctypes.c_void_p(x_host.data_ptr()),
                                          ctypes.c_void_p(core_host.data_ptr()),
                                          ctypes.c_void_p(factors_host.data_ptr()), d), "atucker_sthosvd_host")

    def set_option(self, key: int, value: int):
        _check(lib().atucker_plan_set_option(self._h, int(key), int(value)), "set_option")

    def set_timing(self, on: bool = True):
        _check(lib().atucker_plan_set_option(self._h, OPT_TIMING, 1 if on else 0), "set_option")

    def timings(self) -> dict:
        """Per-phase device ms since timing was enabled / last read (atucker_plan_timings)."""
        buf = (ctypes.c_double * 10)()
        _check(lib().atucker_plan_timings(self._h, buf, 10), "atucker_plan_timings")
        return dict(zip(PHASES, list(buf)))

    def mode_timings(self):
        """Per-mode device ms (by mode index) since the last read (atucker_plan_mode_timings)."""
        buf = (ctypes.c_double * self.order)()
        _check(lib().atucker_plan_mode_timings(self._h, buf, self.order), "atucker_plan_mode_timings")
        return list(buf)

    @property
    def classes(self):
        buf = _i32arr([0] * self.order)
        _check(lib().atucker_plan_classes(self._h, buf), "atucker_plan_classes")
        return list(buf)

    def sync(self):
        _check(lib().atucker_plan_sync(self._h), "atucker_plan_sync")

    def split_factors(self, factors):
        """View the concatenated factor buffer as [U^(n)] (I_n x R_n, column-major -> (I_n, R_n) tensors)."""
        out, off = [], 0
        for d, r in zip(self.dims, self.ranks):
            out.append(factors[off:off + d * r].view(r, d).t())
            off += d * r
        return out

    def close(self):
        if self._h and self._h.value:
            lib().atucker_plan_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptrs(vals):
    return (_vp * len(vals))(*vals)


def run_many(plans, xs, cores, factors, discarded=None):
    """Independent tensors at once (atucker_sthosvd_many): plan i on its own host
    thread and stream.  Every argument is a list with one entry per plan."""
    torch = _torch()
    k = len(plans)
    if not (len(xs) == len(cores) == len(factors) == k) or (discarded is not None and len(discarded) != k):
        raise ValueError("run_many: one x, core and factor buffer per plan")
    d = None
    if discarded is not None:
        d = _ptrs([_dev(t, torch.float64).value if t is not None else None for t in discarded])
    _check(lib().atucker_sthosvd_many(k, _ptrs([p._h.value for p in plans]),
                                      _ptrs([_dev(x, torch.float32).value for x in xs]),
                                      _ptrs([_dev(c, torch.float32).value for c in cores]),
                                      _ptrs([_dev(f, torch.float32).value for f in factors]), d),
           "atucker_sthosvd_many")


def run_many_host(plans, xs_host, cores_host, factors_host, discarded_host=None):
    """Host-buffer form of run_many (atucker_sthosvd_host_many); synchronous."""
    torch = _torch()
    k = len(plans)
    if not (len(xs_host) == len(cores_host) == len(factors_host) == k):
        raise ValueError("run_many_host: one x, core and factor buffer per plan")
    for group in (xs_host, cores_host, factors_host):
        for t in group:
            assert t.device.type == "cpu" and t.is_contiguous() and t.dtype == torch.float32
    d = _ptrs([t.data_ptr() for t in discarded_host]) if discarded_host is not None else None
    _check(lib().atucker_sthosvd_host_many(k, _ptrs([p._h.value for p in plans]),
                                           _ptrs([t.data_ptr() for t in xs_host]),
                                           _ptrs([t.data_ptr() for t in cores_host]),
                                           _ptrs([t.data_ptr() for t in factors_host]), d),
           "atucker_sthosvd_host_many")


def sthosvd(x, dims, ranks, mode_order=None, solver=None, als_sweeps: int = 5, seed: int = 0,
            eig_arith: int | None = None, with_discarded: bool = False, eig_method: int | None = None,
            precision: int = FP32, gram_refine: int | None = None):
    """Decompose the column-major tensor x (flat CUDA float32).

    Returns (core_flat, [U^(n)], discarded or None)."""
    torch = _torch()
    p = Plan(dims, ranks, mode_order, solver, precision, als_sweeps, seed, eig_arith=eig_arith, eig_method=eig_method,
             gram_refine=gram_refine)
    disc = torch.zeros(len(dims), device=x.device, dtype=torch.float64) if with_discarded else None
    core, fac = p.run(x, discarded=disc)
    p.sync()
    facs = p.split_factors(fac)
    p.close()
    return core, facs, disc


def gram(y, lo: int, n: int, hi: int, precision: int = FP32):
    torch = _torch()
    S = torch.empty(n * n, device=y.device, dtype=torch.float64)
    _check(lib().atucker_gram(_dev(y, torch.float32), lo, n, hi, precision, _dev(S, torch.float64), _stream_ptr()),
           "atucker_gram")
    return S.view(n, n).t()


def ttm(y, lo: int, n: int, hi: int, U, precision: int = FP32):
    """U: (n, R) tensor (any layout); returns the flat (lo, R, hi) column-major output."""
    torch = _torch()
    R = U.shape[1]
    Ucm = U.t().contiguous().to(torch.float32)
    out = torch.empty(lo * R * hi, device=y.device, dtype=torch.float32)
    _check(lib().atucker_ttm(_dev(y, torch.float32), lo, n, hi, _dev(Ucm, torch.float32), R, precision,
                             _dev(out, torch.float32), _stream_ptr()), "atucker_ttm")
    return out


def ttm_gram(y, lo: int, n: int, hi: int, U, s: int, m_size: int):
    """Fused TTM and next-mode Gram (atucker_ttm_gram): returns (out, S) with out
    the flat (lo, R, hi) TTM result and S the (I_m, I_m) Gram of out's mode of
    size m_size and row stride s."""
    torch = _torch()
    R = U.shape[1]
    Ucm = U.t().contiguous().to(torch.float32)
    out = torch.empty(lo * R * hi, device=y.device, dtype=torch.float32)
    S = torch.empty(m_size * m_size, device=y.device, dtype=torch.float64)
    _check(lib().atucker_ttm_gram(_dev(y, torch.float32), lo, n, hi, _dev(Ucm, torch.float32), R, s, m_size,
                                  _dev(out, torch.float32), _dev(S, torch.float64), _stream_ptr()),
           "atucker_ttm_gram")
    return out, S.view(m_size, m_size).t()


def eig(S, R: int, eig_arith: int = EIG_ROT_FP32, method: int = EIG_AUTO):
    """S: (n, n) float64 CUDA tensor (symmetric).  Returns (U (n,R) float32, lambda (n,), discarded)."""
    torch = _torch()
    n = S.shape[0]
    Scm = S.t().contiguous().to(torch.float64)
    U = torch.empty(n * R, device=S.device, dtype=torch.float32)
    lam = torch.empty(n, device=S.device, dtype=torch.float64)
    disc = torch.empty(1, device=S.device, dtype=torch.float64)
    _check(lib().atucker_eig(_dev(Scm, torch.float64), n, R, eig_arith, method, _dev(U, torch.float32),
                             _dev(lam, torch.float64), _dev(disc, torch.float64), _stream_ptr()), "atucker_eig")
    return U.view(R, n).t(), lam, disc


def als_mode(y, lo: int, n: int, hi: int, R: int, L0=None, seed: int = 0, mode: int = 0, sweeps: int = 5,
             precision: int = FP32):
    """ALS solver for one mode.  Returns (U (n,R) float32, core flat (lo, R, hi))."""
    torch = _torch()
    U = torch.empty(n * R, device=y.device, dtype=torch.float32)
    core = torch.empty(lo * R * hi, device=y.device, dtype=torch.float32)
    l0 = None
    if L0 is not None:
        L0cm = L0.t().contiguous().to(torch.float64)
        l0 = _dev(L0cm, torch.float64)
    _check(lib().atucker_als_mode(_dev(y, torch.float32), lo, n, hi, R, l0, int(seed) & (2**64 - 1), mode, sweeps,
                                  precision, _dev(U, torch.float32), _dev(core, torch.float32), _stream_ptr()),
           "atucker_als_mode")
    return U.view(R, n).t(), core


class Batch:
    """Many small order-3 tensors decomposed by one persistent launch (atucker_batch_*).

    dims, ranks: sequences of (d1, d2, d3) and (R1, R2, R3), one per tensor.
    run() takes lists of CUDA float32 tensors (each contiguous, column-major
    d1 x d2 x d3 data) and returns lists of cores and concatenated factors.
    """

    def __init__(self, dims, ranks, stream=None, max_sweeps: int | None = None):
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.ranks = [tuple(int(v) for v in r) for r in ranks]
        if len(self.dims) != len(self.ranks) or not self.dims:
            raise ValueError("dims and ranks need the same, non-zero length")
        self.count = len(self.dims)
        flat_d = [v for d in self.dims for v in d]
        flat_r = [v for r in self.ranks for v in r]
        self._h = ctypes.c_void_p(None)
        self.stream = stream
        _check(lib().atucker_batch_create(ctypes.byref(self._h), self.count, _i64arr(flat_d), _i64arr(flat_r),
                                          _stream_ptr(stream)), "atucker_batch_create")
        if max_sweeps is not None:
            self.set_option(BATCH_OPT_JACOBI_MAX_SWEEPS, max_sweeps)

    def set_option(self, option: int, value: int):
        _check(lib().atucker_batch_set_option(self._h, option, int(value)), "atucker_batch_set_option")

    @property
    def variant(self) -> int:
        v = ctypes.c_int(0)
        _check(lib().atucker_batch_get_variant(self._h, ctypes.byref(v)), "atucker_batch_get_variant")
        return v.value

    @staticmethod
    def variants():
        """[(threads per CTA, c values per Gram chunk)] for every launch variant."""
        n = ctypes.c_int(0)
        _check(lib().atucker_batch_variants(ctypes.byref(n), None, None), "atucker_batch_variants")
        th, kc = _i32arr([0] * n.value), _i32arr([0] * n.value)
        _check(lib().atucker_batch_variants(None, th, kc), "atucker_batch_variants")
        return list(zip(list(th), list(kc)))

    def outputs(self):
        """Freshly allocated (cores, factors) lists on the current device."""
        torch = _torch()
        cores = [torch.empty(r[0] * r[1] * r[2], device="cuda", dtype=torch.float32) for r in self.ranks]
        facs = [torch.empty(sum(d * r for d, r in zip(dd, rr)), device="cuda", dtype=torch.float32)
                for dd, rr in zip(self.dims, self.ranks)]
        return cores, facs

    def _tables(self, xs, cores, factors):
        torch = _torch()
        if not (len(xs) == len(cores) == len(factors) == self.count):
            raise ValueError("need one input, core and factor buffer per tensor")
        for t, d in zip(xs, self.dims):
            _dev(t, torch.float32)
            if t.numel() != d[0] * d[1] * d[2]:
                raise ValueError("input size does not match its dims")
        for c, r in zip(cores, self.ranks):
            _dev(c, torch.float32)
            if c.numel() < r[0] * r[1] * r[2]:
                raise ValueError("core buffer too small")
        for f, d, r in zip(factors, self.dims, self.ranks):
            _dev(f, torch.float32)
            if f.numel() < sum(a * b for a, b in zip(d, r)):
                raise ValueError("factor buffer too small")
        mk = lambda ts: (ctypes.c_void_p * self.count)(*[t.data_ptr() for t in ts])  # noqa: E731
        return mk(xs), mk(cores), mk(factors)

    def run(self, xs, cores=None, factors=None, sync: bool = True):
        if cores is None or factors is None:
            cores, factors = self.outputs()
        px, pc, pf = self._tables(xs, cores, factors)
        _check(lib().atucker_batch_run(self._h, px, pc, pf), "atucker_batch_run")
        if sync:
            self.sync()
        return cores, factors

    def sync(self):
        _check(lib().atucker_batch_sync(self._h), "atucker_batch_sync")

    def tune(self, xs, cores=None, factors=None, reps: int = 2):
        """Time every launch variant on this batch and keep the fastest; returns ms per variant."""
        if cores is None or factors is None:
            cores, factors = self.outputs()
        px, pc, pf = self._tables(xs, cores, factors)
        nv = len(self.variants())
        ms = (ctypes.c_float * nv)()
        _check(lib().atucker_batch_tune(self._h, px, pc, pf, int(reps), ms), "atucker_batch_tune")
        return list(ms)

    def close(self):
        if self._h:
            lib().atucker_batch_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def split_factors(flat, dims, ranks):
        out, off = [], 0
        for d, r in zip(dims, ranks):
            out.append(flat[off:off + d * r].view(r, d).t())
            off += d * r
        return out

