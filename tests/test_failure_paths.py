"""Failure paths of the C ABI, driven without faulting a GPU.

* ATK_ENOMEM: the library's allocation cap (atucker_set_device_alloc_limit)
  refuses a plan's workspace before any CUDA call, as an exhausted device
  would; this runs on the host alone.
* ATK_ENOCONV: a sweep cap of one on the full Jacobi eigensolver.
* ATK_ETIMEOUT: a poll limit of one on the grid-barrier waits of the
  cooperative block Jacobi (I_n > 160): the waits give up, every CTA returns,
  the status word carries the timeout, and the same plan runs correctly once
  the limit is lifted.
"""
import ctypes

import numpy as np
import pytest

import paper_2010_10131_b300 as atk


def _plan_create(dims, ranks):
    lib = atk.lib()
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * len(dims))(*dims)
    r = (ctypes.c_int64 * len(ranks))(*ranks)
    s = lib.atucker_plan_create(ctypes.byref(h), len(dims), d, r, None, None, atk.FP32, 5, 0, None)
    return s, h


def test_allocation_cap_returns_enomem_on_host():
    lib = atk.lib()
    try:
        assert lib.atucker_set_device_alloc_limit(4096) == atk.OK
        s, h = _plan_create([64, 64, 64], [8, 8, 8])
        assert s == atk.ENOMEM
        assert b"limit" in lib.atucker_last_error()
        assert not h.value  # no plan handed out
        assert lib.atucker_gram(ctypes.c_void_p(16), 1, 64, 64, atk.FP32C, ctypes.c_void_p(16), None) == atk.ENOMEM
    finally:
        lib.atucker_set_device_alloc_limit(0)


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    atk.lib()
    return atk


@pytest.mark.gpu
def test_allocation_cap_on_device_then_recovery(gpu):
    import synth
    dims, ranks = [48, 40, 36], [4, 4, 4]
    lib = atk.lib()
    try:
        lib.atucker_set_device_alloc_limit(4096)
        with pytest.raises(atk.AtuckerError) as e:
            atk.Plan(dims, ranks)
        assert e.value.status == atk.ENOMEM
    finally:
        lib.atucker_set_device_alloc_limit(0)
    x, _, _ = synth.random_tucker(dims, ranks, seed=1)
    core, facs, _ = atk.sthosvd(torch.from_numpy(x).cuda(), dims, ranks)
    assert np.isfinite(core.cpu().numpy()).all()


def _x(dims, ranks, seed=3):
    import synth
    x, _, _ = synth.random_tucker(dims, ranks, noise=1e-2, seed=seed)
    return torch.from_numpy(x).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("n", [96, 200])
def test_jacobi_sweep_cap_returns_enoconv(gpu, n):
    dims, ranks = [n, 20, 18], [6, 5, 4]
    x = _x(dims, ranks)
    p = atk.Plan(dims, ranks, eig_method=atk.EIG_FULL_JACOBI)
    p.set_option(atk.OPT_JACOBI_MAX_SWEEPS, 1)
    p.run(x)
    assert atk.lib().atucker_plan_sync(p._h) == atk.ENOCONV
    p.set_option(atk.OPT_JACOBI_MAX_SWEEPS, 40)
    p.run(x)
    assert atk.lib().atucker_plan_sync(p._h) == atk.OK
    p.close()


@pytest.mark.gpu
def test_grid_barrier_poll_limit_returns_etimeout(gpu):
    import oracle
    dims, ranks = [220, 16, 12], [6, 5, 4]
    x = _x(dims, ranks)
    p = atk.Plan(dims, ranks, eig_method=atk.EIG_FULL_JACOBI)
    p.set_option(atk.OPT_WAIT_LIMIT, 1)
    p.run(x)
    assert atk.lib().atucker_plan_sync(p._h) == atk.ETIMEOUT
    p.set_option(atk.OPT_WAIT_LIMIT, 0)
    core, fac = p.run(x)
    assert atk.lib().atucker_plan_sync(p._h) == atk.OK
    ref = oracle.sthosvd(x.cpu().double().numpy(), dims, ranks)
    for U, Uo in zip(p.split_factors(fac), ref["factors"]):
        assert oracle.projector_distance(U.cpu().double().numpy(), Uo) <= 1e-4
    p.close()
