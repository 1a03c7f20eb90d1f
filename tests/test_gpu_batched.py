"""Batched persistent st-HOSVD (many small order-3 tensors, one launch) vs the oracle.

Each tensor of the batch is Alg. 2 with EIG in every mode; the batched kernel
keeps the float32 Jacobi vectors (no float64 refinement), so it is held to the
float32 bar of the single-tensor path: |relerr - relerr_oracle| <= 1e-5 and
||U U^T - U_o U_o^T||_F <= 1e-4 per factor, orthonormal factors to 1e-6, and
the core equal to the oracle's (same sign rule) within 1e-3 of its largest
entry.  The tensors are random Tucker plus 1e-3 noise, so every cut sits at a
signal/noise gap.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def atk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2010_10131_b300 as m
    m.lib()
    return m


def _check_member(x, dims, ranks, core, flat_fac):
    x64 = x.astype(np.float64)
    ref = oracle.sthosvd(x64, dims, ranks, solver=[0, 0, 0])
    facs, off = [], 0
    for d, r in zip(dims, ranks):
        facs.append(flat_fac[off:off + d * r].reshape((d, r), order="F"))
        off += d * r
    rel_g = oracle.relerr(x64, core, ranks, facs, dims)
    rel_o = oracle.relerr(x64, ref["core"], ranks, ref["factors"], dims)
    assert abs(rel_g - rel_o) <= 1e-5, (dims, ranks, rel_g, rel_o)
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4, (dims, ranks)
        assert np.linalg.norm(U.T @ U - np.eye(U.shape[1])) <= 1e-6
    core = _align_signs(core, facs, ref["factors"], ranks)
    np.testing.assert_allclose(core, ref["core"], atol=1e-3 * np.abs(ref["core"]).max())


def _align_signs(core, facs, facs_o, ranks):
    """The sign rule (largest-magnitude entry positive) is only determined when
    a column's two largest magnitudes differ by more than the float32
    eigenvector error.  A column whose sign differs from the oracle's is
    accepted only at such a near-tie (within 1e-3 relative), and is then
    flipped, with its core slice, before the cores are compared."""
    g = core.reshape(ranks, order="F").copy()
    for n, (U, Uo) in enumerate(zip(facs, facs_o)):
        for r in range(U.shape[1]):
            if U[:, r] @ Uo[:, r] < 0:
                top = np.sort(np.abs(Uo[:, r]))[::-1]
                assert top[0] - top[1] <= 1e-3 * top[0], ("sign rule violated", n, r)
                U[:, r] *= -1.0
                idx = [slice(None)] * len(ranks)
                idx[n] = r
                g[tuple(idx)] *= -1.0
    return g.ravel(order="F")


def _run(atk, shapes, xs_np, variant=None, graph=True):
    b = atk.Batch([s[0] for s in shapes], [s[1] for s in shapes])
    if variant is not None:
        b.set_option(atk.BATCH_OPT_VARIANT, variant)
    b.set_option(atk.BATCH_OPT_GRAPH, 1 if graph else 0)
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    cores, facs = b.run(xs)
    out = [(c.cpu().double().numpy(), f.cpu().double().numpy()) for c, f in zip(cores, facs)]
    b.close()
    return out


EDGE = [([16, 16, 16], [4, 4, 4]), ([17, 5, 96], [5, 5, 16]), ([96, 96, 96], [16, 16, 16]),
        ([33, 61, 47], [9, 7, 13]), ([95, 18, 40], [16, 4, 12]), ([8, 8, 8], [8, 8, 8]),
        ([20, 90, 21], [4, 16, 5]), ([64, 64, 2], [4, 4, 2])]


def test_batched_matches_oracle(atk):
    shapes = synth.batched_shapes(count=24, seed=11) + [(d, synth.feasible_ranks(d, r)) for d, r in EDGE]
    xs = [synth.batched_tensor(shapes, t, seed=11) for t in range(len(shapes))]
    out = _run(atk, shapes, xs)
    for (dims, ranks), x, (core, fac) in zip(shapes, xs, out):
        _check_member(x, dims, ranks, core, fac)


def test_batched_every_variant(atk):
    shapes = synth.batched_shapes(count=12, seed=5)
    xs = [synth.batched_tensor(shapes, t, seed=5) for t in range(len(shapes))]
    for v in range(len(atk.Batch.variants())):
        out = _run(atk, shapes, xs, variant=v)
        for (dims, ranks), x, (core, fac) in zip(shapes, xs, out):
            _check_member(x, dims, ranks, core, fac)


def test_batched_graph_replay_matches_plain_launch(atk):
    """The captured graph reads the pointer table of each run, not of the first."""
    shapes = synth.batched_shapes(count=16, seed=7)
    b = atk.Batch([s[0] for s in shapes], [s[1] for s in shapes])
    runs = []
    for seed in (7, 8):
        xs = [torch.from_numpy(synth.batched_tensor(shapes, t, seed=seed)).cuda() for t in range(len(shapes))]
        cores, facs = b.run(xs)
        runs.append((xs, [c.clone() for c in cores], [f.clone() for f in facs]))
    b.set_option(atk.BATCH_OPT_GRAPH, 0)
    for xs, cores, facs in runs:
        c2, f2 = b.run(xs)
        for a, c in zip(cores, c2):
            assert torch.equal(a, c)
        for a, c in zip(facs, f2):
            assert torch.equal(a, c)
    assert not all(torch.equal(a, c) for a, c in zip(runs[0][1], runs[1][1]))
    b.close()


def test_batched_tuner_keeps_fastest(atk):
    shapes = synth.batched_shapes(count=64, seed=3)
    b = atk.Batch([s[0] for s in shapes], [s[1] for s in shapes])
    xs = [torch.from_numpy(synth.batched_tensor(shapes, t, seed=3)).cuda() for t in range(len(shapes))]
    ms = b.tune(xs, reps=1)
    assert len(ms) == len(atk.Batch.variants()) and all(m > 0 for m in ms)
    assert b.variant == int(np.argmin(ms))
    cores, facs = b.run(xs)
    for t in (0, 31, 63):
        dims, ranks = shapes[t]
        _check_member(xs[t].cpu().numpy(), dims, ranks, cores[t].cpu().double().numpy(),
                      facs[t].cpu().double().numpy())
    b.close()


def test_batched_full_size_sampled(atk):
    """The 4096-tensor workload in the bench's launch configuration; members
    spread over the size-ordered queue are checked against the oracle."""
    shapes = synth.batched_shapes(count=4096, seed=0)
    b = atk.Batch([s[0] for s in shapes], [s[1] for s in shapes])
    xs = [torch.from_numpy(synth.batched_tensor(shapes, t, seed=0)).cuda() for t in range(len(shapes))]
    b.tune(xs, reps=1)
    cores, facs = b.run(xs)
    for t in (0, 1, 777, 2048, 3000, 4095):
        dims, ranks = shapes[t]
        _check_member(xs[t].cpu().numpy(), dims, ranks, cores[t].cpu().double().numpy(),
                      facs[t].cpu().double().numpy())
    b.close()
