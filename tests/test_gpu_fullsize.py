"""Parity at the benchmarked sizes, on sampled outputs.

The bench's largest contractions run here in the launch configuration the
bench uses (the same C-ABI calls, the same split plans):
  - the mode-1 Gram of the 640^3 tensor (1 x 640 x 409600);
  - the mode-1 Gram of the 48^5 tensor (1 x 48 x 5308416, the small-I_n kernel);
  - the R = 64 truncating TTM of the 640^3 tensor.
A full float64 reference of these is out of reach on the host, so sampled
entries are checked against their definitions computed in float64 from the
same float32 input.  A Gram entry is S_ij = sum_c y(c, i) y(c, j) (Alg. 2,
EIG branch), and a TTM entry is Y'(c, r) = sum_i y(c, i) U(i, r) (Eq. 2).
The tolerances are those of the small-size parity tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def atk():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2010_10131_b300 as m
    m.lib()
    return m


def _input(n, J, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    y = torch.randn(n * J, device="cuda", generator=g)
    # column-major view (i, c) at i + n c: host rows are c, columns are i
    return y, y.cpu().numpy().reshape(J, n)


@pytest.mark.parametrize("n,J", [(640, 409600), (48, 5308416)])
def test_gram_full_size_sampled(atk, n, J):
    y, Y = _input(n, J, seed=n)
    S = atk.gram(y, 1, n, J).cpu().numpy()
    np.testing.assert_array_equal(S, S.T)
    rng = np.random.default_rng(n)
    pairs = [(i, i) for i in rng.choice(n, 4, replace=False)]
    pairs += [tuple(sorted(rng.choice(n, 2, replace=False))) for _ in range(12)]
    pairs += [(0, n - 1), (n - 1, n - 1)]
    cols = {}
    def col(i):
        if i not in cols:
            cols[i] = Y[:, i].astype(np.float64)
        return cols[i]
    scale = max(float(np.dot(col(i), col(i))) for i, _ in pairs[:4])
    tol = 2e-6 * scale * max(1.0, np.sqrt(J / 8192))
    for i, j in pairs:
        exact = float(np.dot(col(i), col(j)))
        assert abs(S[i, j] - exact) <= tol, (i, j, S[i, j], exact)


def test_ttm_full_size_sampled(atk):
    n, J, R = 640, 409600, 64
    y, Y = _input(n, J, seed=7)
    g = torch.Generator(device="cuda").manual_seed(8)
    U = torch.linalg.qr(torch.randn(n, R, device="cuda", generator=g))[0].contiguous()
    out = atk.ttm(y, 1, n, J, U).cpu().numpy()  # (R, J) column-major: (r, c) at r + R c
    O = out.reshape(J, R)
    U64 = U.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(9)
    cs = np.concatenate([rng.choice(J, 40, replace=False), [0, J - 1]])
    ref = Y[cs].astype(np.float64) @ U64  # (len(cs), R)
    got = O[cs]
    assert np.abs(got - ref).max() <= 1e-5 * np.sqrt(n) * np.abs(ref).max() + 1e-6
