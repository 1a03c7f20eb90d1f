"""GPU path vs the FP64 CPU oracle, step by step and end to end.

Every case feeds the identical float32 bytes (from ``synth``) to the CUDA
library (through the C ABI) and, widened to float64, to the oracle.
Tolerances follow the arithmetic: float32 products summed over J terms, in
split-K chunks of <= 8192, reduced in float64.  End-to-end tolerances are the
ones the method is judged by: |relerr_gpu - relerr_oracle| <= 1e-5 and
||U U^T - U_o U_o^T||_F <= 1e-4.
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


def _cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _view_dims(lo, n, hi):
    return [lo, n, hi]


GRAM_VIEWS = [
    (1, 96, 2000),     # mode 1: lo == 1, one tile, ragged c
    (1, 300, 777),     # mode 1: 3 row tiles, ragged n and c
    (8, 96, 96),       # middle mode, lo multiple of 4
    (7, 50, 33),       # middle mode, lo odd (uncoalesced path), n < 64
    (4096, 20, 1),     # last mode: hi == 1
    (3, 1, 11),        # n == 1
    (1, 17, 1),        # J == 1
    (33, 130, 5),      # n just over a tile, lo odd
    (5, 300, 40),      # strided, three tile rows: all six tiles in one launch
    (64, 257, 30),     # strided, the third tile row holds one row
    (1, 48, 100003),   # small-I_n form: 6 x 6 blocks, ragged last split
    (1, 64, 50000),    # small-I_n form: 8 x 8 blocks, two-warp groups
    (1, 60, 12345),    # small-I_n form: columns 60..63 zero-filled
    (1, 8, 70001),     # small-I_n form: one block
    (1, 4, 999),       # small-I_n form: half a block, fewer rows than a CTA's share
]


@pytest.mark.parametrize("lo,n,hi", GRAM_VIEWS)
def test_gram_matches_oracle(atk, lo, n, hi):
    g = np.random.default_rng(lo * 1000 + n * 7 + hi)
    y = g.standard_normal(lo * n * hi).astype(np.float32)
    S = atk.gram(_cuda(y), lo, n, hi).cpu().numpy()
    So = oracle.gram(y.astype(np.float64), _view_dims(lo, n, hi), 1)
    scale = np.abs(np.diag(So)).max()
    assert np.abs(S - So).max() <= 2e-6 * scale * max(1.0, np.sqrt(lo * hi / 8192))
    np.testing.assert_array_equal(S, S.T)


@pytest.mark.parametrize("lo,n,hi,R", [(1, 96, 2000, 8), (1, 300, 333, 64), (8, 96, 96, 8), (7, 50, 33, 17),
                                       (4096, 20, 1, 3), (5, 130, 9, 128), (1, 33, 1, 33), (16, 9, 40, 1)])
def test_ttm_matches_oracle(atk, lo, n, hi, R):
    g = np.random.default_rng(lo + n + hi + R)
    y = g.standard_normal(lo * n * hi).astype(np.float32)
    U = g.standard_normal((n, R)).astype(np.float32)
    out = atk.ttm(_cuda(y), lo, n, hi, _cuda(U)).cpu().numpy()
    ref = oracle.ttm(y.astype(np.float64), _view_dims(lo, n, hi), 1, U.astype(np.float64))
    assert np.abs(out - ref).max() <= 1e-5 * np.sqrt(n) * np.abs(ref).max() + 1e-6


# Contiguous mode-1 views large enough (a CTA per SM) for the cp.async-fed
# TTM: both column classes (R <= 16, <= 32) with R not a multiple of the
# column tile, J ragged against the row tile, I_n % 16 != 0 (a stage half
# past I_n) and I_n = 4 (one chunk per row); R = 50 and 64 check that larger
# ranks keep the k-major kernel.
@pytest.mark.parametrize("n,J,R", [(68, 40001, 12), (128, 39000, 16), (36, 20011, 20), (100, 19999, 32),
                                   (52, 19000, 50), (640, 19457, 64), (4, 40000, 3)])
def test_ttm_async_form_matches_oracle(atk, n, J, R):
    g = np.random.default_rng(n * 31 + J + R)
    y = g.standard_normal(n * J).astype(np.float32)
    U = g.standard_normal((n, R)).astype(np.float32)
    out = atk.ttm(_cuda(y), 1, n, J, _cuda(U)).cpu().numpy()
    ref = oracle.ttm(y.astype(np.float64), [n, J], 0, U.astype(np.float64))
    assert np.abs(out - ref).max() <= 1e-5 * np.sqrt(n) * np.abs(ref).max() + 1e-6


def _spd_with_gap(n, R, seed):
    g = np.random.default_rng(seed)
    Q = np.linalg.qr(g.standard_normal((n, n)))[0]
    lam = np.concatenate([np.linspace(10.0, 4.0, R), 1e-2 * g.random(n - R)])
    return (Q * lam) @ Q.T


def _rr_used(n, R, arith, method):
    # The library's choice: block width m = R + p, p = clamp(R / 2, 8, 16),
    # m <= 156; the subspace path needs m >= R + 8 (and, for AUTO, 2 m <= n).
    p = max(8, min(16, R // 2))
    m = min(n, R + p, 156)
    return arith == 0 and m >= R + 8 and ((method == 0 and 2 * m <= n) or (method == 2 and m < n))


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("n,R", [(2, 1), (5, 2), (33, 8), (96, 8), (128, 16), (130, 16), (200, 20), (640, 64),
                                 (1000, 128), (150, 40), (200, 72), (240, 100), (70, 22), (140, 49),
                                 (200, 81), (260, 113)])
def test_eig_matches_oracle(atk, n, R, arith, method):
    if arith == 1 and n > 200:
        pytest.skip("float64 rotations at n >= 640 are slow on B300 (covered at 200)")
    if method == 1 and n > 640:
        pytest.skip("full Jacobi is covered up to n = 640")
    S = _spd_with_gap(n, R, n + R)
    U, lam, disc = atk.eig(_cuda(S), R, eig_arith=arith, method=method)
    U = U.cpu().double().numpy()
    lo_, Vo, _ = oracle.jacobi_eig(S)
    lam = lam.cpu().numpy()
    # The kept subspace is refined in float64, so rotation-invariant quantities
    # are tight: the projector, the sum of the kept eigenvalues (float64
    # Rayleigh quotients) and the discarded energy.  Inside the kept subspace,
    # float rotations resolve vectors only to ~1e-4 * lambda_1 / (absolute gap),
    # so single eigenvalues and columns are checked at that accuracy.
    assert oracle.projector_distance(U, Vo[:, :R]) <= 1e-4
    np.testing.assert_allclose(lam[:R].sum(), lo_[:R].sum(), rtol=1e-10)
    np.testing.assert_allclose(lam[:R], lo_[:R], rtol=1e-7 if arith == 0 else 1e-10)
    if _rr_used(n, R, arith, method):
        assert np.all(np.isnan(lam[R:]))  # only the kept eigenvalues exist on the subspace path
    else:
        tail_tol = 4 * n * 6e-8 * lo_[0] if arith == 0 else 1e-12 * n * lo_[0]
        np.testing.assert_allclose(lam[R:], lo_[R:], atol=tail_tol)
    assert np.linalg.norm(U.T @ U - np.eye(R)) <= 1e-6
    # Same sign rule on both sides: well-separated columns agree, not just the subspace.
    gaps = np.abs(np.diff(lo_[: R + 1]))
    sep = np.minimum(np.r_[np.inf, gaps[:-1]], gaps) if R > 0 else gaps
    for r in range(R):
        if sep[r] >= 0.05 * lo_[0]:
            np.testing.assert_allclose(U[:, r], Vo[:, r], atol=1e-4)
    assert abs(disc.item() - lo_[R:].sum()) <= 1e-9 * lo_[0] * n


def test_eig_subspace_decaying_spectrum(atk):
    """lambda_k = k^-3 (singular values k^-1.5): relative gap at the cut 2.7e-6.

    Below the float32 resolution of the rotations the split between u_32 and
    u_33 is not determined, so the projector is not pinned; the captured
    energy is, to within the gap.
    """
    n, R = 500, 32
    g = np.random.default_rng(8)
    Q = np.linalg.qr(g.standard_normal((n, n)))[0]
    lam = np.arange(1, n + 1, dtype=np.float64) ** -3.0
    S = (Q * lam) @ Q.T
    U, lamg, disc = atk.eig(_cuda(S), R, method=2)
    lo_, Vo, _ = oracle.jacobi_eig(S)
    U = U.cpu().double().numpy()
    assert np.linalg.norm(U.T @ U - np.eye(R)) <= 1e-6
    assert abs(lamg.cpu().numpy()[:R].sum() - lo_[:R].sum()) <= 1e-5 * lo_[0]
    assert abs(disc.item() - lo_[R:].sum()) <= 1e-5 * lo_[0]
    # the leading vectors, well separated, still agree with the oracle
    assert oracle.projector_distance(U[:, :8], Vo[:, :8]) <= 1e-4


def test_eig_repeated_eigenvalues(atk):
    """Degenerate spectrum: the subspace of the top cluster is still unique."""
    n, R = 40, 4
    g = np.random.default_rng(3)
    Q = np.linalg.qr(g.standard_normal((n, n)))[0]
    lam = np.array([5.0] * 4 + [1.0] * (n - 4))
    S = (Q * lam) @ Q.T
    U, lamg, _ = atk.eig(_cuda(S), R)
    assert oracle.projector_distance(U.cpu().double().numpy(), Q[:, :4]) <= 1e-4


@pytest.mark.parametrize("n,R,lam_rtol,disc_rel", [(300, 24, 1e-7, 1e-9), (200, 20, 1e-7, 1e-9),
                                                  (300, 128, 3e-7, 1e-8)])
def test_eig_subspace_clustered_kept_eigenvalues(atk, n, R, lam_rtol, disc_rel):
    """Subspace path with exact clusters inside the kept set and a degenerate
    noise floor 1e-4 below it: the Rayleigh-Ritz eigensolver must return an
    orthonormal basis of each cluster (the tridiagonal solver re-orthogonalises
    inside clusters), and the float64 refinement must keep the float32
    leakage of the noise columns out of the kept subspace (its subspace step
    multiplies that leakage by lambda_1 / lambda_noise = 1e4).

    (300, 128) has the widest projection of the path (m = 144, only 16 guard
    columns): there one power step and one refinement step leave the kept
    subspace at about 2e-5 (kept energy 5e-6 off in 1.7e3) and the edge
    eigenvalues of the clusters 1.7e-7 relative off; the bounds follow."""
    g = np.random.default_rng(11)
    Q = np.linalg.qr(g.standard_normal((n, n)))[0]
    k = R // 3
    top = np.concatenate([np.full(k, 10.0), np.full(k, 7.0), np.full(R - 2 * k, 4.0)])
    lam = np.concatenate([top, np.full(n - R, 1e-3)])
    S = (Q * lam) @ Q.T
    U, lamg, disc = atk.eig(_cuda(S), R, method=2)
    U = U.cpu().double().numpy()
    assert np.linalg.norm(U.T @ U - np.eye(R)) <= 1e-6
    assert oracle.projector_distance(U, Q[:, :R]) <= 1e-4
    assert abs(disc.item() - lam[R:].sum()) <= disc_rel * lam[0] * n
    np.testing.assert_allclose(np.sort(lamg.cpu().numpy()[:R])[::-1], top, rtol=lam_rtol)


@pytest.mark.parametrize("n,R", [(712, 32), (400, 40), (887, 66)])
def test_eig_subspace_rank_equal_to_r(atk, n, R):
    """S = Y Y^T with Y n x R: rank exactly R, below the subspace block width
    m = R + p.  (This is the Gram of a mode whose rank equals the product of
    the other ranks.)  The shifted power steps keep the block at full rank, so
    the subspace path resolves it instead of breaking down (it used to fall
    back to the full Jacobi, 60x slower); the kept subspace is range(Y)."""
    g = np.random.default_rng(0)
    Y = g.standard_normal((n, R)).astype(np.float32).astype(np.float64)
    S = Y @ Y.T
    U, lamg, disc = atk.eig(_cuda(S), R, method=2)
    U = U.cpu().double().numpy()
    Qy = np.linalg.qr(Y)[0]
    assert np.linalg.norm(U.T @ U - np.eye(R)) <= 1e-6
    assert oracle.projector_distance(U, Qy) <= 1e-4
    ref = np.sort(np.linalg.eigvalsh(Y.T @ Y))[::-1]
    np.testing.assert_allclose(lamg.cpu().numpy()[:R], ref, rtol=1e-7)
    assert abs(disc.item()) <= 1e-9 * ref[0] * n


def test_sthosvd_mode_rank_equal_to_product_of_others(atk):
    """A plan whose last mode's rank is the product of the other ranks (its
    Gram has rank exactly R_n): matches the oracle.  The last mode's kept
    space is range(S), whose smallest eigenvalue is far below the largest
    (lambda_R / lambda_1 about 1e-3 for a random core); a float32 Gram of the
    truncated core would turn it by about eps_32 lambda_1 / lambda_R, so the
    plan recomputes that Gram with compensated sums (ATK_OPT_GRAM_REFINE)
    and the projector meets the same 1e-4 as every other factor."""
    dims, ranks = [40, 30, 120], [6, 5, 30]
    core, facs, disc, ref, rel_g, rel_o = _e2e(atk, dims, ranks, [0, 0, 0], seed=5)
    assert abs(rel_g - rel_o) <= 1e-5
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4


@pytest.mark.parametrize("lo,n,hi,R", [(1, 40, 300, 5), (6, 24, 50, 8), (64, 30, 1, 6)])
def test_als_mode_matches_oracle(atk, lo, n, hi, R):
    dims = [lo, n, hi]
    x, _, _ = synth.random_tucker(dims, synth.feasible_ranks(dims, [min(lo, R), R, min(hi, R)]), noise=1e-2,
                                  seed=lo + n)
    x64 = x.astype(np.float64)
    U, core = atk.als_mode(_cuda(x), lo, n, hi, R, seed=5, mode=1, sweeps=5)
    Y = oracle.unfold(x64, dims, 1)
    L0 = oracle.als_init(5, 1, n, R)
    L, Rk = oracle.als(Y, L0, 5)
    Q, Rh = oracle.householder_qr(L)
    core_ref = oracle.fold(Rh @ Rk.T, [lo, R, hi], 1)
    U = U.cpu().double().numpy()
    np.testing.assert_allclose(U, Q, atol=2e-4)
    np.testing.assert_allclose(core.cpu().double().numpy(), core_ref, atol=2e-4 * np.abs(core_ref).max())


# ------------------------------------------------------------- end to end

def _e2e(atk, dims, ranks, solver, mode_order=None, noise=1e-3, seed=0, eig_arith=None, eig_method=None):
    x, _, _ = synth.random_tucker(dims, ranks, noise=noise, seed=seed)
    core, facs, disc = atk.sthosvd(_cuda(x), dims, ranks, mode_order=mode_order, solver=solver,
                                   eig_arith=eig_arith, with_discarded=True, eig_method=eig_method)
    core = core.cpu().double().numpy()
    facs = [f.cpu().double().numpy() for f in facs]
    x64 = x.astype(np.float64)
    ref = oracle.sthosvd(x64, dims, ranks, mode_order=mode_order, solver=solver)
    rel_g = oracle.relerr(x64, core, ranks, facs, dims)
    rel_o = oracle.relerr(x64, ref["core"], ranks, ref["factors"], dims)
    return core, facs, disc.cpu().numpy(), ref, rel_g, rel_o


@pytest.mark.parametrize("solver", [[0, 0, 0], [1, 1, 1], [0, 1, 0], [1, 0, 0]])
def test_config1_96cube_r8(atk, solver):
    """The 96^3 random-Tucker case (ranks 8, noise 1e-3, seed 0)."""
    dims, ranks = [96, 96, 96], [8, 8, 8]
    core, facs, disc, ref, rel_g, rel_o = _e2e(atk, dims, ranks, solver)
    assert abs(rel_g - rel_o) <= 1e-5
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4
        assert np.linalg.norm(U.T @ U - np.eye(U.shape[1])) <= 1e-6
    np.testing.assert_allclose(core, ref["core"], atol=1e-3 * np.abs(ref["core"]).max())
    # EIG discarded energy is trace(S) - sum of float64 Rayleigh quotients.  For
    # ALS it is ||Y||^2 - ||Y'||^2 of float32 tensors, so it carries rounding
    # of order eps_32 * ||X||^2.
    nx2 = float(np.sum(synth.random_tucker([96, 96, 96], [8, 8, 8], seed=0)[0].astype(np.float64) ** 2))
    np.testing.assert_allclose(disc, ref["discarded"], rtol=1e-3, atol=2e-6 * nx2)


@pytest.mark.parametrize("dims,ranks,solver,mode_order", [
    ([30, 41, 25], [5, 7, 4], [0, 0, 0], [2, 0, 1]),
    ([19, 23, 17, 11], [3, 4, 5, 2], [0, 1, 0, 1], [3, 1, 0, 2]),
    ([12, 9, 10, 8, 7], [2, 3, 2, 3, 2], [0, 0, 1, 0, 0], None),
    ([150, 20, 30], [10, 5, 6], [0, 0, 0], None),
    ([20, 140, 13], [4, 12, 3], [0, 0, 1], [1, 2, 0]),
])
def test_orders_modes_solvers(atk, dims, ranks, solver, mode_order):
    core, facs, disc, ref, rel_g, rel_o = _e2e(atk, dims, ranks, solver, mode_order=mode_order, noise=1e-2, seed=3)
    assert abs(rel_g - rel_o) <= 1e-5
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4


def test_exact_recovery_noise_free(atk):
    dims, ranks = [40, 33, 27], [4, 3, 5]
    core, facs, disc, ref, rel_g, rel_o = _e2e(atk, dims, ranks, [0, 1, 0], noise=0.0, seed=9)
    assert rel_g <= 1e-5
    x, _, truth = synth.random_tucker(dims, ranks, noise=0.0, seed=9)
    for U, Ut in zip(facs, truth):
        assert oracle.projector_distance(U, Ut) <= 1e-4


@pytest.mark.parametrize("method", [1, 2])
def test_config1_eig_methods(atk, method):
    """The 96^3 case with the full Jacobi and with the Rayleigh-Ritz subspace eigensolver."""
    dims, ranks = [96, 96, 96], [8, 8, 8]
    core, facs, disc, ref, rel_g, rel_o = _e2e(atk, dims, ranks, [0, 0, 0], eig_method=method)
    assert abs(rel_g - rel_o) <= 1e-5
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4
    np.testing.assert_allclose(core, ref["core"], atol=1e-3 * np.abs(ref["core"]).max())


def test_eig_fp64_rotations_end_to_end(atk):
    dims, ranks = [64, 48, 56], [6, 5, 7]
    core, facs, disc, ref, rel_g, rel_o = _e2e(atk, dims, ranks, [0, 0, 0], eig_arith=1)
    assert abs(rel_g - rel_o) <= 1e-5
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4


def test_host_buffer_entry_point(atk):
    dims, ranks = [48, 40, 36], [4, 4, 4]
    x, _, _ = synth.random_tucker(dims, ranks, seed=1)
    p = atk.Plan(dims, ranks)
    xh = torch.from_numpy(x).pin_memory()
    core = torch.empty(p.core_numel).pin_memory()
    fac = torch.empty(p.factors_numel).pin_memory()
    disc = torch.empty(3, dtype=torch.float64)
    p.run_host(xh, core, fac, disc)
    ref = oracle.sthosvd(x.astype(np.float64), dims, ranks)
    facs = [f.double().numpy() for f in p.split_factors(fac)]
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4
    p.close()


@pytest.mark.parametrize("dims,ranks,solver,mode_order", [
    ([30, 41, 25], [5, 7, 4], [0, 0, 0], [2, 0, 1]),
    ([19, 23, 17, 11], [3, 4, 5, 2], [0, 1, 0, 1], [3, 1, 0, 2]),
    ([96, 96, 96], [8, 8, 8], [0, 0, 0], None),
])
def test_explicit_matricization_matches_oracle(atk, dims, ranks, solver, mode_order):
    """ATK_OPT_EXPLICIT_UNFOLD (the ablation of Sec. VI-E): each mode with
    I_<n > 1 is unfolded into a buffer, run as a mode-1 view and folded back;
    the decomposition meets the same tolerances as the matricization-free
    path, whose result it matches to float32 rounding."""
    x, _, _ = synth.random_tucker(dims, ranks, noise=1e-2, seed=3)
    xd = _cuda(x)
    outs = []
    for explicit in (0, 1):
        p = atk.Plan(dims, ranks, mode_order=mode_order, solver=solver)
        p.set_option(atk.OPT_EXPLICIT_UNFOLD, explicit)
        core, fac = p.run(xd)
        p.sync()
        outs.append((core.cpu().double().numpy(), [f.cpu().double().numpy() for f in p.split_factors(fac)]))
        p.close()
    x64 = x.astype(np.float64)
    ref = oracle.sthosvd(x64, dims, ranks, mode_order=mode_order, solver=solver)
    rel_o = oracle.relerr(x64, ref["core"], ranks, ref["factors"], dims)
    (core0, facs0), (core1, facs1) = outs
    assert abs(oracle.relerr(x64, core1, ranks, facs1, dims) - rel_o) <= 1e-5
    for U, U0, Uo in zip(facs1, facs0, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4
        assert oracle.projector_distance(U, U0) <= 1e-5
    np.testing.assert_allclose(core1, core0, atol=1e-4 * np.abs(core0).max())
