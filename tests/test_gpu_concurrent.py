"""Concurrent plans (atucker_sthosvd_many): independent tensors on their own
streams and host threads give exactly the results of running them one by one.

Every reduction in the library has a fixed order, so a run's output does not
depend on what else shares the GPU; the concurrent results are compared bit
for bit with serial runs of the same plans, and with the float64 oracle.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # (dims, ranks, solver): the subspace eigensolver (host reads between its
    # launch groups), the one-CTA Jacobi, and ALS modes, in one batch.
    ([300, 40, 64], [24, 6, 8], [0, 0, 0]),
    ([96, 96, 96], [8, 8, 8], [0, 1, 0]),
    ([20, 30, 40, 24], [4, 5, 6, 3], [1, 1, 0, 1]),
]


@pytest.fixture(scope="module")
def atk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2010_10131_b300 as m
    m.lib()
    return m


def _setup(atk, seed=0):
    streams = [torch.cuda.Stream(priority=-5 if i == 0 else 0) for i in range(len(CASES))]
    plans, xs, xnps, cores, facs = [], [], [], [], []
    for i, ((dims, ranks, solver), st) in enumerate(zip(CASES, streams)):
        x, _, _ = synth.random_tucker(dims, ranks, noise=1e-3, seed=seed + i)
        xnps.append(x)
        xs.append(torch.from_numpy(x).cuda())
        p = atk.Plan(dims, ranks, solver=solver, stream=st)
        plans.append(p)
        cores.append(torch.empty(p.core_numel, device="cuda"))
        facs.append(torch.empty(p.factors_numel, device="cuda"))
    torch.cuda.synchronize()
    return plans, xs, xnps, cores, facs


def test_run_many_matches_serial_runs_bitwise(atk):
    plans, xs, xnps, cores, facs = _setup(atk)
    serial_c, serial_f = [], []
    for p, x in zip(plans, xs):
        p.set_timing(True)
        c, f = p.run(x)
        p.sync()
        serial_c.append(c.clone())
        serial_f.append(f.clone())
    serial_launches = [p.timings()["launches"] for p in plans]
    for p in plans:
        p.set_timing(True)
    for _ in range(3):  # repeated: graph replays and concurrent host syncs
        atk.run_many(plans, xs, cores, facs)
    for p in plans:
        p.sync()
    conc_launches = [p.timings()["launches"] / 3 for p in plans]
    for i in range(len(plans)):
        assert torch.equal(cores[i], serial_c[i]), f"plan {i}: core differs"
        assert torch.equal(facs[i], serial_f[i]), f"plan {i}: factors differ"
    assert conc_launches == serial_launches
    for (dims, ranks, solver), p, x, f in zip(CASES, plans, xnps, facs):
        ref = oracle.sthosvd(x.astype(np.float64), dims, ranks, solver=solver)
        for U, Uo in zip(p.split_factors(f), ref["factors"]):
            assert oracle.projector_distance(U.double().cpu().numpy(), Uo) <= 1e-4
    for p in plans:
        p.close()


def test_run_many_host_matches_device_runs(atk):
    plans, xs, xnps, cores, facs = _setup(atk, seed=10)
    atk.run_many(plans, xs, cores, facs)
    for p in plans:
        p.sync()
    hx = [torch.from_numpy(x).pin_memory() for x in xnps]
    hc = [torch.empty(p.core_numel).pin_memory() for p in plans]
    hf = [torch.empty(p.factors_numel).pin_memory() for p in plans]
    atk.run_many_host(plans, hx, hc, hf)
    for i in range(len(plans)):
        assert torch.equal(hc[i], cores[i].cpu())
        assert torch.equal(hf[i], facs[i].cpu())
    for p in plans:
        p.close()


def test_run_many_reports_the_failing_plan(atk):
    """A plan whose run is rejected (a null input pointer) is named in the
    error; the other plans' runs still complete correctly."""
    import ctypes
    plans, xs, _, cores, facs = _setup(atk, seed=20)
    atk.run_many(plans, xs, cores, facs)
    for p in plans:
        p.sync()
    want = [c.clone() for c in cores]
    for c in cores:
        c.zero_()
    vp = ctypes.c_void_p
    arr = lambda vals: (vp * len(vals))(*vals)
    st = atk.lib().atucker_sthosvd_many(3, arr([p._h.value for p in plans]),
                                        arr([xs[0].data_ptr(), xs[1].data_ptr(), None]),
                                        arr([c.data_ptr() for c in cores]), arr([f.data_ptr() for f in facs]), None)
    assert st == atk.EINVAL
    assert atk.lib().atucker_last_error().startswith(b"plan 2:")
    for p in plans:
        p.sync()
    assert torch.equal(cores[0], want[0]) and torch.equal(cores[1], want[1])
    for p in plans:
        p.close()
