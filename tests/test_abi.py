"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os

import pytest

import paper_2010_10131_b300 as atk


def test_header_declares_the_bound_entry_points():
    declared = set(atk.abi_symbols())
    assert "atucker_sthosvd" in declared and "atucker_plan_create" in declared
    bound = set(atk._SIGS)
    assert declared == bound, (declared - bound, bound - declared)


def test_library_exports_every_declared_symbol():
    path = atk.LIB_PATH
    if not os.path.exists(path):
        from paper_2010_10131_b300 import build
        build.build()
    handle = ctypes.CDLL(path)
    missing = [s for s in atk.abi_symbols() if not hasattr(handle, s)]
    assert not missing, missing


def test_version_and_error_string_without_gpu():
    lib = atk.lib()
    assert lib.atucker_version().decode().count(".") == 2
    assert isinstance(lib.atucker_last_error(), bytes)


def test_argument_validation_runs_on_host():
    """Bad arguments are rejected before any device call."""
    lib = atk.lib()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(4, 4, 4)
    bad_ranks = (ctypes.c_int64 * 3)(5, 2, 2)
    assert lib.atucker_plan_create(ctypes.byref(h), 3, dims, bad_ranks, None, None, 0, 5, 0, None) == atk.ERANK
    infeasible = (ctypes.c_int64 * 3)(4, 1, 1)
    assert lib.atucker_plan_create(ctypes.byref(h), 3, dims, infeasible, None, None, 0, 5, 0, None) == atk.ERANK
    ranks = (ctypes.c_int64 * 3)(2, 2, 2)
    perm = (ctypes.c_int * 3)(0, 0, 1)
    assert lib.atucker_plan_create(ctypes.byref(h), 3, dims, ranks, perm, None, 0, 5, 0, None) == atk.EINVAL
    solver = (ctypes.c_int * 3)(0, 2, 0)
    assert lib.atucker_plan_create(ctypes.byref(h), 3, dims, ranks, None, solver, 0, 5, 0, None) == atk.EINVAL
    assert lib.atucker_plan_create(ctypes.byref(h), 9, dims, ranks, None, None, 0, 5, 0, None) == atk.EINVAL
    assert b"order" in lib.atucker_last_error()
    assert lib.atucker_gram(None, 1, 1, 1, 0, None, None) == atk.EINVAL


def test_run_many_validation_runs_on_host():
    """The concurrent entry points check their plan list before any device call."""
    lib = atk.lib()
    fake = ctypes.c_void_p(0x1000)
    plans = (ctypes.c_void_p * 2)(fake, fake)
    arr = (ctypes.c_void_p * 2)(None, None)
    assert lib.atucker_sthosvd_many(2, plans, arr, arr, arr, None) == atk.EINVAL
    assert b"twice" in lib.atucker_last_error()
    none = (ctypes.c_void_p * 2)(fake, None)
    assert lib.atucker_sthosvd_many(2, none, arr, arr, arr, None) == atk.EINVAL
    assert lib.atucker_sthosvd_many(0, plans, arr, arr, arr, None) == atk.EINVAL
    assert lib.atucker_sthosvd_host_many(2, plans, None, arr, arr, None) == atk.EINVAL


def test_batch_validation_runs_on_host():
    """The batched form rejects shapes outside its limits before touching the device."""
    lib = atk.lib()
    h = ctypes.c_void_p()
    too_big = (ctypes.c_int64 * 6)(16, 16, 16, 97, 20, 20)
    ranks = (ctypes.c_int64 * 6)(4, 4, 4, 4, 4, 4)
    assert lib.atucker_batch_create(ctypes.byref(h), 2, too_big, ranks, None) == atk.EUNSUPPORTED
    dims = (ctypes.c_int64 * 3)(16, 16, 16)
    infeasible = (ctypes.c_int64 * 3)(9, 2, 4)
    assert lib.atucker_batch_create(ctypes.byref(h), 1, dims, infeasible, None) == atk.ERANK
    rank_over_dim = (ctypes.c_int64 * 3)(17, 4, 4)
    assert lib.atucker_batch_create(ctypes.byref(h), 1, dims, rank_over_dim, None) == atk.ERANK
    assert lib.atucker_batch_create(ctypes.byref(h), 0, dims, ranks, None) == atk.EINVAL
    assert lib.atucker_batch_run(None, None, None, None) == atk.EINVAL
    n = ctypes.c_int(0)
    assert lib.atucker_batch_variants(ctypes.byref(n), None, None) == atk.OK and n.value >= 2


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(atk, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(atk, "_lib", None)
    with pytest.raises(ImportError):
        atk.lib(build_if_missing=False)
