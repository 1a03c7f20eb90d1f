"""GPU path vs the FP64 oracle at the widths the benchmark runs.

The benchmark's 640^3 tensor has a 640-row Gram and a 640-wide EIG mode; the
precision sweep has a spectrum that decays like k^-3 at the cut, where the
gap between the kept and the first discarded eigenvalue is far below float32
resolution of the largest one.  These cases check the default arithmetic
(float32 contractions, the default eigensolver) against the oracle element
by element (Gram) and through the method's own error measure (relerr and the
factor projectors, Alg. 2), on inputs the oracle finishes in seconds.
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


@pytest.mark.parametrize("lo,n,hi", [(1, 640, 40000), (64, 640, 640)])
def test_gram_640_rows_matches_oracle(atk, lo, n, hi):
    """The 640-row Gram of mode 1 (lo = 1) and of a middle mode after a
    truncation to 64 (lo = 64), element by element.  Float32 chains of at
    most 8192 terms, reduced across splits in float-float: the error bound of
    the smaller views scaled by sqrt(J / 8192)."""
    g = np.random.default_rng(640 + lo)
    y = g.standard_normal(lo * n * hi).astype(np.float32)
    S = atk.gram(_cuda(y), lo, n, hi).cpu().numpy()
    So = oracle.gram(y.astype(np.float64), [lo, n, hi], 1)
    scale = np.abs(np.diag(So)).max()
    assert np.abs(S - So).max() <= 2e-6 * scale * max(1.0, np.sqrt(lo * hi / 8192))
    np.testing.assert_array_equal(S, S.T)


def _e2e(atk, x, dims, ranks, **kw):
    core, facs, disc = atk.sthosvd(_cuda(x), dims, ranks, solver=[0] * len(dims), with_discarded=True, **kw)
    core = core.cpu().double().numpy()
    facs = [f.cpu().double().numpy() for f in facs]
    x64 = x.astype(np.float64)
    ref = oracle.sthosvd(x64, dims, ranks, solver=[0] * len(dims))
    rel_g = oracle.relerr(x64, core, ranks, facs, dims)
    rel_o = oracle.relerr(x64, ref["core"], ranks, ref["factors"], dims)
    return facs, disc.cpu().numpy(), ref, rel_g, rel_o


def test_eig_mode_640_wide_end_to_end(atk):
    """A 640-wide EIG mode (the benchmark's mode-1 width and rank) on a random
    Tucker tensor with 1e-3 noise: the method's tolerances, |d relerr| <= 1e-5
    and ||U U^T - U_o U_o^T||_F <= 1e-4 for every factor."""
    dims, ranks = [640, 96, 48], [64, 16, 12]
    x, _, _ = synth.random_tucker(dims, ranks, noise=1e-3, seed=4)
    facs, disc, ref, rel_g, rel_o = _e2e(atk, x, dims, ranks)
    assert abs(rel_g - rel_o) <= 1e-5
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4
        assert np.linalg.norm(U.T @ U - np.eye(U.shape[1])) <= 1e-6


@pytest.mark.parametrize("R", [64, 128])
def test_decaying_spectrum_cut_default_arithmetic(atk, R):
    """The precision sweep's spectrum (core singular values ~ k^-1.5, so Gram
    eigenvalues ~ k^-3, plus 1e-3 noise) at 256^3: at R = 64 the gap at the
    cut is about 1.5 eps_32 lambda_1, at R = 128 about 0.1 eps_32 lambda_1.
    With the default arithmetic the relative error must stay within 1e-5 of
    the oracle's.  The projectors are not pinned here: the split between the
    eigenvectors on either side of such a cut is not determined by the
    float32 Gram (its rounding errors reach the size of the gap)."""
    dims = [256, 256, 256]
    x, _, _ = synth.decaying_tucker(dims, R, noise=1e-3, seed=0)
    facs, disc, ref, rel_g, rel_o = _e2e(atk, x, dims, [R] * 3)
    assert abs(rel_g - rel_o) <= 1e-5, (rel_g, rel_o)
    for U in facs:
        assert np.linalg.norm(U.T @ U - np.eye(U.shape[1])) <= 1e-6


@pytest.mark.parametrize("lo,n,hi", [(1, 300, 777), (33, 130, 5), (7, 50, 33)])
def test_gram_compensated_matches_oracle(atk, lo, n, hi):
    """ATK_FP32C: exact float32 products summed as float-float pairs, about
    48 bits per partial sum, element by element against the oracle."""
    g = np.random.default_rng(lo + 3 * n + hi)
    y = g.standard_normal(lo * n * hi).astype(np.float32)
    So = oracle.gram(y.astype(np.float64), [lo, n, hi], 1)
    S = atk.gram(_cuda(y), lo, n, hi, precision=atk.FP32C).cpu().numpy()
    scale = np.abs(np.diag(So)).max()
    assert np.abs(S - So).max() <= 1e-12 * scale
    np.testing.assert_array_equal(S, S.T)


def test_gram_compensated_concentrated_energy(atk):
    """The shape of a truncated core's energy: one entry per mode-n row 1e4
    times the others.  The float32 Gram's rounding reaches eps_32 times that
    entry's square (about 1e8); the compensated Gram's error is eps_32 times
    the sum of the small terms only (the large term is carried exactly in the
    high word), so the small-scale structure keeps float32 relative accuracy."""
    lo, n, hi = 16384, 64, 1
    g = np.random.default_rng(7)
    y = g.standard_normal((hi, n, lo))
    y[:, :, 0] *= 1e4
    y = y.astype(np.float32).ravel()
    So = oracle.gram(y.astype(np.float64), [lo, n, hi], 1)
    small = oracle.gram(np.where(np.arange(lo * n * hi) % lo == 0, 0.0, np.abs(y.astype(np.float64))),
                        [lo, n, hi], 1)
    S32 = atk.gram(_cuda(y), lo, n, hi).cpu().numpy()
    Sc = atk.gram(_cuda(y), lo, n, hi, precision=atk.FP32C).cpu().numpy()
    err_c, err_32 = np.abs(Sc - So), np.abs(S32 - So)
    assert np.all(err_c <= 2e-6 * np.sqrt(lo) * small + 1e-13 * np.abs(So))
    assert err_c.max() * 100 <= err_32.max()


def test_eig_mode_beyond_1024_rows(atk):
    """An EIG mode with I_n = 1056 > 1024 (the Table II shapes have EIG modes
    of up to 30648 rows): the subspace eigensolver on the full 1056-row Gram,
    end to end against the oracle's full Jacobi."""
    dims, ranks = [1056, 24, 10], [10, 8, 5]
    x, _, _ = synth.random_tucker(dims, ranks, noise=1e-2, seed=6)
    facs, disc, ref, rel_g, rel_o = _e2e(atk, x, dims, ranks)
    assert abs(rel_g - rel_o) <= 1e-5
    for U, Uo in zip(facs, ref["factors"]):
        assert oracle.projector_distance(U, Uo) <= 1e-4
