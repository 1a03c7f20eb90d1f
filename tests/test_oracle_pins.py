"""Pins for the CPU oracle: each check ties it to something other than itself.

Sources of truth used here: closed forms, library routines the oracle does not
call (numpy.linalg.eigh / svd / qr / cholesky, numpy.tensordot), brute force on
tiny inputs, and invariants of the method (exact recovery, orthonormality, the
st-HOSVD error identity, ALS as subspace iteration).  The checks are chosen so
that a dropped term, a wrong sign or index, or a transposed operand anywhere in
the oracle fails at least one of them.
"""
import numpy as np
import pytest

import oracle
import synth


def _rand_tensor(dims, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(dims)


# ------------------------------------------------------------- matricization

@pytest.mark.parametrize("dims", [(2, 3, 4), (3, 1, 5, 2), (4, 3), (1, 4, 2)])
def test_unfold_matches_index_definition(dims):
    """X_(n)[i_n, j] from numpy's moveaxis + Fortran reshape (Sec. II-A)."""
    x = _rand_tensor(dims, 1)
    flat = x.ravel(order="F")
    for n in range(len(dims)):
        ref = np.moveaxis(x, n, 0).reshape((dims[n], -1), order="F")
        got = oracle.unfold(flat, dims, n)
        np.testing.assert_array_equal(got, ref)
        # Sec. II-A: the Frobenius norm is the same for every matricization.
        assert abs(np.sum(got * got) - oracle.norm2(flat)) <= 1e-12 * oracle.norm2(flat)
        np.testing.assert_array_equal(oracle.fold(got, dims, n), flat)


def test_matmul_against_numpy():
    g = np.random.default_rng(2)
    a, b = g.standard_normal((7, 5)), g.standard_normal((5, 3))
    np.testing.assert_allclose(oracle.matmul(a, b), a @ b, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 3, 2, 5), (9, 1, 4)])
def test_gram_is_contraction_over_other_modes(dims):
    """S[i, j] = sum over all other indices of x[..i..] x[..j..] (Eq. 3 with Y = X)."""
    x = _rand_tensor(dims, 3)
    for n in range(len(dims)):
        others = [k for k in range(len(dims)) if k != n]
        ref = np.tensordot(x, x, axes=(others, others))
        np.testing.assert_allclose(oracle.gram(x.ravel(order="F"), dims, n), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 3, 2, 5), (1, 6, 3)])
def test_ttm_eq2(dims):
    """Eq. (2) with the matrix U^T: y[.., r, ..] = sum_i x[.., i, ..] U[i, r]."""
    x = _rand_tensor(dims, 4)
    g = np.random.default_rng(5)
    for n in range(len(dims)):
        R = max(1, dims[n] - 1)
        U = g.standard_normal((dims[n], R))
        ref = np.moveaxis(np.tensordot(U.T, x, axes=(1, n)), 0, n)
        got = oracle.ttm(x.ravel(order="F"), dims, n, U)
        np.testing.assert_allclose(got, ref.ravel(order="F"), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- eigensolver

def test_jacobi_2x2_closed_form():
    a, b, c = 3.0, -1.25, 0.5
    lam, V, _ = oracle.jacobi_eig(np.array([[a, b], [b, c]]))
    mid, rad = (a + c) / 2, np.hypot((a - c) / 2, b)
    np.testing.assert_allclose(lam, [mid + rad, mid - rad], rtol=1e-14)
    S = np.array([[a, b], [b, c]])
    for k in range(2):
        np.testing.assert_allclose(S @ V[:, k], lam[k] * V[:, k], atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 64])
def test_jacobi_vs_eigh(n):
    g = np.random.default_rng(10 + n)
    M = g.standard_normal((n, n))
    S = M + M.T
    lam, V, _ = oracle.jacobi_eig(S)
    ref = np.linalg.eigh(S)[0][::-1]
    np.testing.assert_allclose(lam, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(V @ np.diag(lam) @ V.T, S, atol=1e-12 * np.abs(S).max())
    # Sign rule: the largest-magnitude entry of each column is positive.
    for k in range(n):
        assert V[np.argmax(np.abs(V[:, k])), k] > 0


def test_jacobi_diagonal_and_identity():
    lam, V, _ = oracle.jacobi_eig(np.diag([1.0, 4.0, 2.0]))
    np.testing.assert_array_equal(lam, [4.0, 2.0, 1.0])
    np.testing.assert_array_equal(np.abs(V), np.eye(3)[:, [1, 2, 0]])
    lam, V, _ = oracle.jacobi_eig(np.eye(4))  # ties keep index order
    np.testing.assert_array_equal(V, np.eye(4))


# ------------------------------------------------------- small linear algebra

def test_cholesky_vs_numpy():
    g = np.random.default_rng(20)
    M = g.standard_normal((9, 9))
    G = M @ M.T + 9 * np.eye(9)
    np.testing.assert_allclose(oracle.cholesky(G), np.linalg.cholesky(G), rtol=1e-12, atol=1e-12)
    with pytest.raises(RuntimeError):
        oracle.cholesky(-np.eye(3))


@pytest.mark.parametrize("m,r", [(7, 3), (5, 5), (40, 8), (3, 1)])
def test_householder_qr(m, r):
    g = np.random.default_rng(30 + m)
    M = g.standard_normal((m, r))
    Q, R = oracle.householder_qr(M)
    np.testing.assert_allclose(Q @ R, M, atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(r), atol=1e-13)
    assert np.all(np.diag(R) > 0) and np.allclose(np.tril(R, -1), 0)
    q2, r2 = np.linalg.qr(M)
    sg = np.sign(np.diag(r2))
    np.testing.assert_allclose(Q, q2 * sg, atol=1e-12)
    np.testing.assert_allclose(R, r2 * sg[:, None], atol=1e-12)


# ----------------------------------------------------------------- ALS pieces

def test_splitmix64_published_vectors():
    """First outputs of splitmix64 seeded with 0 (Steele, Lea and Flood 2014)."""
    assert oracle.splitmix64_at(0, 1) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64_at(0, 2) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64_at(0, 3) == 0x06C45D188009454F


def test_als_init_is_standard_normal():
    L = oracle.als_init(123, 2, 400, 50)
    assert L.shape == (400, 50)
    assert abs(L.mean()) < 0.02 and abs(L.std() - 1.0) < 0.02
    from scipy import stats
    assert stats.kstest(L.ravel(), "norm").pvalue > 1e-3
    np.testing.assert_array_equal(L, oracle.als_init(123, 2, 400, 50))
    assert not np.allclose(L, oracle.als_init(123, 1, 400, 50))


def test_als_is_subspace_iteration():
    """col(L_{k+1}) = col(S L_k) with S = Y Y^T, hence col(L_K) = col(S^K L_0)."""
    g = np.random.default_rng(40)
    Y = g.standard_normal((12, 30))
    L0 = g.standard_normal((12, 3))
    for K in (1, 2, 5):
        L, Rk = oracle.als(Y, L0, K)
        Z = L0.copy()
        for _ in range(K):
            Z = Y @ (Y.T @ Z)
            Z, _ = np.linalg.qr(Z)
        Ql, _ = np.linalg.qr(L)
        assert oracle.projector_distance(Ql, Z) < 1e-9
        # R_{K-1} is the least-squares partner of L_{K-1}; L_K is the LS fit to it.
        np.testing.assert_allclose(L, Y @ Rk @ np.linalg.inv(Rk.T @ Rk), atol=1e-10)


def test_als_exact_for_rank_r():
    g = np.random.default_rng(41)
    Y = g.standard_normal((10, 3)) @ g.standard_normal((3, 25))
    L, Rk = oracle.als(Y, g.standard_normal((10, 3)), 1)
    np.testing.assert_allclose(L @ Rk.T, Y, atol=1e-10)


# --------------------------------------------------------------- st-HOSVD

@pytest.mark.parametrize("solver", [(0, 0, 0), (1, 1, 1), (0, 1, 0), (1, 0, 1)])
def test_exact_recovery_noise_free(solver):
    dims, ranks = (12, 10, 9), (3, 4, 2)
    x, core_t, fac_t = synth.random_tucker(dims, ranks, noise=0.0, seed=7)
    x64 = x.astype(np.float64)
    out = oracle.sthosvd(x64, dims, ranks, mode_order=[0, 1, 2], solver=list(solver))
    rel = oracle.relerr(x64, out["core"], ranks, out["factors"], dims)
    assert rel < 1e-7  # the input itself is float32-rounded
    for U, Ut in zip(out["factors"], fac_t):
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)
        assert oracle.projector_distance(U, Ut) < 1e-6


def test_exact_recovery_float64_input():
    """Noise-free and never rounded: recovery to float64 precision."""
    dims, ranks = (8, 7, 6), (2, 3, 2)
    g = synth.rng(9)
    core = g.standard_normal(ranks)
    facs = [np.linalg.qr(g.standard_normal((d, r)))[0] for d, r in zip(dims, ranks)]
    x = core
    for n, u in enumerate(facs):
        x = np.moveaxis(np.tensordot(u, x, axes=(1, n)), 0, n)
    flat = x.ravel(order="F")
    for solver in ([0, 0, 0], [1, 1, 1]):
        out = oracle.sthosvd(flat, dims, ranks, solver=solver)
        assert oracle.relerr(flat, out["core"], ranks, out["factors"], dims) < 1e-12
        for U, Ut in zip(out["factors"], facs):
            assert oracle.projector_distance(U, Ut) < 1e-10


@pytest.mark.parametrize("mode_order", [[0, 1, 2], [2, 0, 1], [1, 2, 0]])
def test_error_identity_eig(mode_order):
    """EIG modes: ||X - X_hat||^2 = sum of discarded eigenvalues = ||X||^2 - ||G||^2."""
    dims, ranks = (14, 11, 9), (4, 3, 5)
    x, _, _ = synth.random_tucker(dims, ranks, noise=0.05, seed=11)
    x64 = x.astype(np.float64)
    out = oracle.sthosvd(x64, dims, ranks, mode_order=mode_order, solver=[0, 0, 0])
    xh = oracle.reconstruct(out["core"], ranks, out["factors"], dims)
    err2 = np.sum((x64 - xh) ** 2)
    nx2 = np.sum(x64 ** 2)
    assert abs(err2 - out["discarded"].sum()) <= 1e-10 * nx2
    assert abs(err2 - (nx2 - np.sum(out["core"] ** 2))) <= 1e-10 * nx2


def test_als_mode_pythagoras():
    """ALS step: ||Y||^2 = ||R^ R^T||^2 + ||Y - L R^T||^2 (L_K is the LS fit to R_{K-1})."""
    dims, ranks = (10, 8, 7), (3, 8, 7)
    x, _, _ = synth.random_tucker(dims, (3, 4, 3), noise=0.1, seed=12)
    x64 = x.astype(np.float64)
    out = oracle.sthosvd(x64, dims, ranks, mode_order=[0, 1, 2], solver=[1, 0, 0])
    Y = oracle.unfold(x64, dims, 0)
    L0 = oracle.als_init(0, 0, dims[0], ranks[0])
    L, Rk = oracle.als(Y, L0, 5)
    res = np.sum((Y - L @ Rk.T) ** 2)
    kept = np.sum((L @ Rk.T) ** 2)
    assert abs(np.sum(Y ** 2) - kept - res) <= 1e-10 * np.sum(Y ** 2)
    assert abs(out["discarded"][0] - res) <= 1e-9 * np.sum(Y ** 2)


def test_order2_is_truncated_svd():
    """Eckart-Young: for a matrix, st-HOSVD-EIG gives the best rank-(R, R) error."""
    g = np.random.default_rng(50)
    M = g.standard_normal((15, 11))
    dims, ranks = (15, 11), (4, 4)
    out = oracle.sthosvd(M.ravel(order="F"), dims, ranks, solver=[0, 0])
    s = np.linalg.svd(M, compute_uv=False)
    err2 = np.sum((M.ravel(order="F") - oracle.reconstruct(out["core"], ranks, out["factors"], dims)) ** 2)
    np.testing.assert_allclose(err2, np.sum(s[4:] ** 2), rtol=1e-10)
    u = np.linalg.svd(M)[0][:, :4]
    assert oracle.projector_distance(out["factors"][0], u) < 1e-10


@pytest.mark.parametrize("dims,ranks", [((3, 4, 5), (2, 2, 3)), ((2, 3, 4, 3), (2, 2, 2, 2))])
def test_eig_path_equals_svd_path(dims, ranks):
    """Sec. II-C: the Gram-eigen solver reproduces the SVD solver (Alg. 1)."""
    x = _rand_tensor(dims, 60).ravel(order="F")
    a = oracle.sthosvd(x, dims, ranks, solver=[0] * len(dims))
    b = oracle.sthosvd_svd(x, dims, ranks)
    for U, V in zip(a["factors"], b["factors"]):
        np.testing.assert_allclose(U, V, atol=1e-10)
    np.testing.assert_allclose(a["core"], b["core"], atol=1e-10)


def test_jacobi_svd_vs_numpy():
    g = np.random.default_rng(61)
    for shape in [(5, 9), (9, 5), (6, 6)]:
        M = g.standard_normal(shape)
        s, U = oracle.jacobi_svd_left(M)
        np.testing.assert_allclose(s, np.linalg.svd(M, compute_uv=False), rtol=1e-12)
        u = np.linalg.svd(M)[0][:, : len(s)]
        for k in range(len(s)):
            assert abs(abs(U[:, k] @ u[:, k]) - 1) < 1e-10


def test_captured_energy_beats_random_subspaces():
    """Brute force: no random orthonormal basis captures more of Y_(1) than U^(1)."""
    dims, ranks = (6, 5, 4), (2, 5, 4)
    x = _rand_tensor(dims, 70).ravel(order="F")
    out = oracle.sthosvd(x, dims, ranks, solver=[0, 0, 0])
    Y = oracle.unfold(x, dims, 0)
    best = np.sum((out["factors"][0].T @ Y) ** 2)
    g = np.random.default_rng(71)
    for _ in range(3000):
        q = np.linalg.qr(g.standard_normal((6, 2)))[0]
        assert np.sum((q.T @ Y) ** 2) <= best * (1 + 1e-12)


def test_rank_checks():
    x = _rand_tensor((4, 4, 4), 80).ravel(order="F")
    with pytest.raises(RuntimeError):
        oracle.sthosvd(x, (4, 4, 4), (5, 2, 2))
    with pytest.raises(RuntimeError):
        oracle.sthosvd(x, (4, 4, 4), (0, 2, 2))


def test_feasible_ranks():
    assert synth.feasible_ranks((10, 10, 10), (9, 2, 2)) == [4, 2, 2]
    r = synth.feasible_ranks((30, 40, 50), (20, 3, 4))
    for n in range(3):
        others = int(np.prod([r[k] for k in range(3) if k != n]))
        assert 1 <= r[n] <= min((30, 40, 50)[n], others)


# ----------------------------------------------------------------- selector MLP
from oracle import mlp as omlp  # noqa: E402

_IN, _H, _K = 12, 64, 5


def _mlp_case(seed, B=40):
    g = np.random.default_rng(seed)
    p = g.standard_normal(omlp.param_count(_IN, _H, _K)) * 0.3
    X = g.standard_normal((B, _IN))
    Y = g.standard_normal((B, _K))
    M = (g.random((B, _K)) > 0.2).astype(np.float64)
    return p, X, Y, M


def test_mlp_gradient_central_differences():
    """The backpropagated gradient against central differences of the loss on
    20 randomly chosen parameters (the loss is piecewise smooth: ReLU kinks
    are avoided by the small step)."""
    p, X, Y, M = _mlp_case(91)
    L, g = omlp.grad(p, X, Y, M, _IN, _H, _K)
    assert abs(L - omlp.loss(p, X, Y, M, _IN, _H, _K)) <= 1e-12 * max(1.0, L)
    idx = np.random.default_rng(92).choice(p.size, 20, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (omlp.loss(p + e, X, Y, M, _IN, _H, _K) - omlp.loss(p - e, X, Y, M, _IN, _H, _K)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_mlp_dead_hidden_layer_closed_form():
    """With b2 very negative every a2 is zero: the output is b3 for every row,
    so dL/db3 = 2 sum_b M (b3 - Y) / sum M and every other gradient is zero."""
    p, X, Y, M = _mlp_case(93)
    W1, b1, W2, b2, W3, b3 = omlp.unpack(p, _IN, _H, _K)
    q = p.copy()
    off_b2 = _H * _IN + _H + _H * _H
    q[off_b2:off_b2 + _H] = -1e6
    out, _ = omlp.forward(q, X, _IN, _H, _K)
    np.testing.assert_allclose(out, np.broadcast_to(b3, out.shape), rtol=0, atol=0)
    L, g = omlp.grad(q, X, Y, M, _IN, _H, _K)
    expect_b3 = 2 * (M * (b3[None, :] - Y)).sum(axis=0) / M.sum()
    np.testing.assert_allclose(g[-_K:], expect_b3, rtol=1e-12)
    assert np.all(g[:-_K] == 0.0)


def test_mlp_adam_first_step_is_sign_step():
    """Adam's first bias-corrected step is lr * g / (|g| + eps): every parameter
    with a non-zero gradient moves by lr (to 1e-6) against its sign."""
    p, X, Y, M = _mlp_case(94)
    _, g = omlp.grad(p, X, Y, M, _IN, _H, _K)
    q, m, v = omlp.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-2)
    nz = np.abs(g) > 1e-4
    np.testing.assert_allclose((p - q)[nz], 1e-2 * np.sign(g[nz]), rtol=1e-3)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
