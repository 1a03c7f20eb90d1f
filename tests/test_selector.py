"""Learned selector: features, host inference and the GPU training kernels.

CPU: the library's features follow their definition (Table I plus position and
remaining size) and its host inference equals the float64 oracle network.
GPU: the training kernels' forward pass and gradient equal the oracle's
(float32 vs float64, relative 1e-5), and Adam steps follow the oracle's.
"""
import ctypes

import numpy as np
import pytest

import paper_2010_10131_b300 as atk
from oracle import mlp as omlp

IN, H, K = atk.SELECTOR_FEATURES, atk.SELECTOR_HIDDEN, atk.NUM_CLASSES


def _features(dims, ranks, mode_order=None):
    from paper_2010_10131_b300 import selector
    return selector.mode_features(dims, ranks, mode_order)


def test_mode_features_follow_the_definition():
    dims, ranks, order = [40, 300, 7, 90], [5, 30, 7, 9], [2, 0, 3, 1]
    F = _features(dims, ranks, order)
    cur = [float(d) for d in dims]
    for step, n in enumerate(order):
        I, R = cur[n], float(ranks[n])
        J = float(np.prod([cur[k] for k in range(4) if k != n]))
        want = np.log2([I, R, J, I * I, R * R, I * R, R * R / I, R * R / J, I / J, R / J])
        np.testing.assert_allclose(F[n, :10], want, rtol=0, atol=1e-12)
        assert F[n, 10] == step / 3.0
        np.testing.assert_allclose(F[n, 11], np.log2(I * J), atol=1e-12)
        cur[n] = R


def _packed(seed):
    g = np.random.default_rng(seed)
    mean = g.standard_normal(IN)
    scale = 0.5 + g.random(IN)
    p = (g.standard_normal(omlp.param_count(IN, H, K)) * 0.2).astype(np.float32)
    return mean, scale, p


def test_host_inference_matches_oracle():
    from paper_2010_10131_b300 import selector
    mean, scale, p = _packed(3)
    selector.install(selector.pack(mean, scale, p))
    g = np.random.default_rng(4)
    F = g.standard_normal((50, IN)) * 2 + 3
    F[:, 0] = np.minimum(F[:, 0], 9.0)  # I_n <= 512: every class allowed
    cls, scores = selector.predict(F)
    X = (F - mean.astype(np.float32)) / scale.astype(np.float32)
    ref, _ = omlp.forward(p.astype(np.float64), X, IN, H, K)
    np.testing.assert_allclose(scores, ref, rtol=1e-4, atol=1e-4 * np.abs(ref).max())
    np.testing.assert_array_equal(cls, np.argmin(scores, axis=1))
    # The full-Jacobi classes need I_n <= 1024: at I_n = 2048 a mode gets the
    # subspace EIG classes or ALS; beyond 32768, ALS only.
    F[:, 0] = 11.0
    cls, _ = selector.predict(F)
    assert not np.any((cls == atk.CLASS_EIG_JACOBI) | (cls == atk.CLASS_EIG_JACOBI_SMALL))
    F[:, 0] = 16.0
    cls, _ = selector.predict(F)
    assert np.all(cls == atk.CLASS_ALS)
    atk.lib().atucker_selector_clear()


def test_selector_rejects_bad_parameters():
    lib = atk.lib()
    buf = np.zeros(10, dtype=np.float32)
    assert lib.atucker_selector_set(buf.ctypes.data_as(ctypes.c_void_p), 10) == atk.EINVAL
    n = 2 * IN + omlp.param_count(IN, H, K)
    assert lib.atucker_mlp_param_count(IN, H, K) == omlp.param_count(IN, H, K)
    buf = np.zeros(n, dtype=np.float32)  # zero scales are rejected
    assert lib.atucker_selector_set(buf.ctypes.data_as(ctypes.c_void_p), n) == atk.EINVAL


@pytest.mark.gpu
def test_auto_plan_uses_the_selector():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2010_10131_b300 import selector
    mean, scale, p = _packed(5)
    # bias the last layer so that the network always prefers ALS
    p = p.copy()
    p[-K:] = [5.0, 5.0, 5.0, 5.0, -5.0]
    p[-K - K * H:-K] = 0.0
    selector.install(selector.pack(mean, scale, p))
    plan = atk.Plan([30, 20, 10], [4, 4, 4], solver=[atk.AUTO, atk.EIG, atk.AUTO])
    assert plan.classes == [atk.CLASS_ALS, atk.CLASS_EIG, atk.CLASS_ALS]
    plan.close()
    atk.lib().atucker_selector_clear()
    plan = atk.Plan([30, 20, 10], [4, 4, 4], solver=[atk.AUTO] * 3)
    assert plan.classes == [atk.CLASS_EIG] * 3  # no selector loaded: EIG until the first run times the classes
    plan.close()


def test_search_policy_keeps_the_fastest_close_candidate():
    """Host logic of the product path's policy (with_search): candidates are
    the prediction plus up to two fitting classes predicted within the margin;
    the measured fastest of them wins; clear calls and unfit classes are left
    alone."""
    from paper_2010_10131_b300 import selector
    lg = np.array([[6.0], [6.0], [12.0], [6.0]])  # log2 I_n: 64, 64, 4096, 64
    F = np.concatenate([lg, np.zeros((4, IN - 1))], axis=1)
    scores = np.array([[0.0, 0.1, 0.2, 0.9, 0.05],   # EIG, ALS, EIG-small close: timed
                       [0.0, 2.0, 2.0, 2.0, 2.0],    # clear call
                       [0.0, 0.1, 0.05, 0.05, 3.0],  # I_n = 4096: Jacobi classes cannot run
                       [0.0, 0.1, 0.2, 0.25, 0.29]], dtype=np.float32)  # four close: at most three timed
    T = np.array([[5.0, 4.0, 1.0, 9.0, 3.0],
                  [5.0, 1.0, 1.0, 1.0, 1.0],
                  [5.0, 4.0, 1.0, 1.0, 9.0],
                  [5.0, 4.0, 3.0, 1.0, 0.5]])
    cls = np.zeros(4, dtype=int)
    out, searched = selector.with_search(F, T, cls, scores, margin=0.3, top=3)
    assert list(out) == [4, 0, 1, 2] and searched == 3


@pytest.mark.gpu
def test_auto_times_the_networks_close_calls():
    """A network that scores EIG and EIG-small-tile equal (and the rest far
    worse) leaves those two as candidates: the first run keeps one of them,
    and the result is bit for bit that of a plan built with the kept classes."""
    torch = _gpu()
    from paper_2010_10131_b300 import selector
    mean, scale, p = _packed(6)
    p = p.copy()
    p[-K:] = [-5.0, -5.0, 5.0, 5.0, 5.0]
    p[-K - K * H:-K] = 0.0
    selector.install(selector.pack(mean, scale, p))
    try:
        dims, ranks = [160, 40, 36], [8, 6, 5]
        x = torch.randn(dims[0] * dims[1] * dims[2], generator=torch.Generator().manual_seed(4)).cuda()
        p1 = atk.Plan(dims, ranks, solver=[atk.AUTO] * 3)
        c1, f1 = p1.run(x)
        chosen = p1.classes
        assert all(c in (atk.CLASS_EIG, atk.CLASS_EIG_SMALL) for c in chosen)
        p2 = atk.Plan(dims, ranks, classes=chosen)
        c2, f2 = p2.run(x)
        torch.cuda.synchronize()
        assert torch.equal(c1, c2) and torch.equal(f1, f2)
        p1.close()
        p2.close()
    finally:
        atk.lib().atucker_selector_clear()


@pytest.mark.gpu
def test_auto_without_selector_settles_classes_by_timing():
    """No selector loaded: the first run times every class that fits each AUTO
    mode and keeps the fastest; a second plan of the same key takes the cached
    choice, and either gives bit for bit what a plan built with those classes
    gives (the search changes which kernels run, not what they compute)."""
    torch = _gpu()
    atk.lib().atucker_selector_clear()
    dims, ranks = [48, 200, 36], [6, 10, 5]
    g = torch.Generator().manual_seed(3)
    x = torch.randn(dims[0] * dims[1] * dims[2], generator=g).cuda()
    p1 = atk.Plan(dims, ranks, solver=[atk.AUTO, atk.EIG, atk.AUTO])
    assert p1.classes == [atk.CLASS_EIG] * 3
    c1, f1 = p1.run(x)
    chosen = p1.classes
    assert chosen[1] == atk.CLASS_EIG  # a fixed mode is not searched
    assert all(0 <= c < atk.NUM_CLASSES for c in chosen)
    c1b, f1b = p1.run(x)
    p2 = atk.Plan(dims, ranks, solver=[atk.AUTO, atk.EIG, atk.AUTO])
    c2, f2 = p2.run(x)
    assert p2.classes == chosen
    p3 = atk.Plan(dims, ranks, classes=chosen)
    c3, f3 = p3.run(x)
    torch.cuda.synchronize()
    for a, b in ((c1b, c3), (f1b, f3), (c2, c3), (f2, f3), (c1, c3), (f1, f3)):
        assert torch.equal(a, b)
    for p in (p1, p2, p3):
        p.close()


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _case(seed, B=300):
    g = np.random.default_rng(seed)
    p = (g.standard_normal(omlp.param_count(IN, H, K)) * 0.2).astype(np.float32)
    X = g.standard_normal((B, IN)).astype(np.float32)
    Y = (g.standard_normal((B, K)) * 2).astype(np.float32)
    M = (g.random((B, K)) > 0.25).astype(np.float32)
    return p, X, Y, M


@pytest.mark.gpu
def test_gpu_forward_and_gradient_match_oracle():
    _gpu()
    from paper_2010_10131_b300.selector import GpuMLP
    for seed in (1, 2):
        p, X, Y, M = _case(seed)
        net = GpuMLP(p)
        out = net.forward(X)
        ref, _ = omlp.forward(p.astype(np.float64), X, IN, H, K)
        np.testing.assert_allclose(out, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
        L, g = net.loss_grad(X, Y, M)
        Lr, gr = omlp.grad(p.astype(np.float64), X, Y, M, IN, H, K)
        assert abs(L - Lr) <= 1e-5 * abs(Lr)
        np.testing.assert_allclose(g, gr, rtol=1e-5, atol=1e-5 * np.abs(gr).max())


@pytest.mark.gpu
def test_gpu_adam_steps_follow_oracle():
    _gpu()
    from paper_2010_10131_b300.selector import GpuMLP
    p, X, Y, M = _case(7)
    net = GpuMLP(p)
    losses = net.train(X, Y, M, steps=5, lr=1e-3)
    q, m, v = p.astype(np.float64), 0.0, 0.0
    for t in range(1, 6):
        L, g = omlp.grad(q, X, Y, M, IN, H, K)
        assert abs(losses[t - 1] - L) <= 1e-4 * abs(L)
        q, m, v = omlp.adam_step(q, g, m, v, t, 1e-3)
    np.testing.assert_allclose(net.host_params(), q, rtol=0, atol=2e-5)
    # and training goes down
    more = net.train(X, Y, M, steps=300, lr=3e-3)
    assert more[-1] < 0.5 * losses[0]


@pytest.mark.gpu
def test_trained_selector_beats_the_method_without_it():
    """Trained on the committed timing sets with the library's kernels, the
    selector's choices on the 64 held-out shapes cost less time (as measured by
    the library, per mode) than the fixed policies: every mode EIG (the method
    without a selector), every mode ALS, every mode full Jacobi."""
    _gpu()
    from paper_2010_10131_b300 import selector
    report, packed = selector.train_and_evaluate()
    ext = report["train_192_plus_extra"]
    assert ext["gain_vs_fixed_EIG"] > 1.0, ext
    assert ext["gain_vs_fixed_ALS"] > 2.0, ext
    assert ext["gain_vs_fixed_EIG-Jacobi"] > 2.0, ext
    assert ext["regret"] < report["best_possible_gain_vs_fixed_EIG"] - 1.0, ext
    atk.lib().atucker_selector_clear()
