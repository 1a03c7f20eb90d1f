"""The fused TTM and next-mode Gram (Alg. 2: the TTM closing mode n and the
Gram opening the next mode m are adjacent steps) against the FP64 oracle.

Direct cases call atucker_ttm_gram through the C ABI.  The TTM output is
checked against the oracle's TTM of the same float32 input.  The Gram is
checked against the oracle's mode-m Gram of the kernel's own float32 output,
widened to float64, so that the TTM's rounding does not enter the Gram check.
The geometries cover:
  - the first mode (rows contiguous in k);
  - a middle and a last mode (rows contiguous in c);
  - a next mode below or above the TTM's mode;
  - ragged fibre groups and every (R, I_m) tile class.
End-to-end cases run plans with the fusion on and off (the default), both
checked against the oracle's st-HOSVD.
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


def _geometry(dims, n, m):
    """Mode-n view of dims and the stride of mode m among its rows c."""
    lo = int(np.prod(dims[:n], dtype=np.int64))
    hi = int(np.prod(dims[n + 1:], dtype=np.int64))
    s = int(np.prod([dims[k] for k in range(m) if k != n], dtype=np.int64))
    return lo, dims[n], hi, s


CASES = [
    # dims, n (TTM mode), R, m (next mode)
    ([96, 128, 40], 0, 16, 1),        # first mode, I_m = 128 (one fibre per group)
    ([48, 48, 47], 0, 8, 1),          # I_m = 48: two fibres per group, ragged last group
    ([8, 60, 33], 1, 24, 2),          # middle mode -> last mode (s = lo)
    ([20, 3, 50], 2, 50, 0),          # last mode -> first mode (m < n), R = 50
    ([5, 17, 30, 7], 2, 24, 1),       # m < n inside lo (s = 5), I_m = 17
    ([64, 96, 600], 0, 16, 1),        # 600 groups, several per CTA
    ([100, 128, 30], 0, 64, 1),       # R = 64 with I_m = 128 (the widest tile)
    ([16, 32, 16, 40], 1, 32, 3),     # next mode two modes up (s = 16 * 16)
    ([40, 25, 3, 16], 0, 20, 3),      # I_m = 16, s = 25 * 3, odd lows per group
]


@pytest.mark.parametrize("dims,n,R,m", CASES)
def test_ttm_gram_matches_oracle(atk, dims, n, R, m):
    g = np.random.default_rng(sum(dims) + 31 * n + R)
    x = g.standard_normal(int(np.prod(dims))).astype(np.float32)
    U = np.linalg.qr(g.standard_normal((dims[n], R)))[0].astype(np.float32)
    lo, nn, hi, s = _geometry(dims, n, m)
    out, S = atk.ttm_gram(_cuda(x), lo, nn, hi, _cuda(U), s, dims[m])
    out = out.cpu().numpy()
    S = S.cpu().numpy()
    ref = oracle.ttm(x.astype(np.float64), dims, n, U.astype(np.float64))
    assert np.abs(out - ref).max() <= 1e-5 * np.sqrt(nn) * np.abs(ref).max() + 1e-6
    odims = list(dims)
    odims[n] = R
    So = oracle.gram(out.astype(np.float64), odims, m)
    scale = np.abs(np.diag(So)).max()
    J = out.size // dims[m]
    assert np.abs(S - So).max() <= 2e-6 * scale * max(1.0, np.sqrt(J / 8192))
    np.testing.assert_array_equal(S, S.T)


def test_ttm_gram_is_reproducible(atk):
    dims, n, R, m = [48, 48, 48], 0, 8, 1
    g = np.random.default_rng(5)
    x = _cuda(g.standard_normal(int(np.prod(dims))).astype(np.float32))
    U = _cuda(np.linalg.qr(g.standard_normal((48, R)))[0].astype(np.float32))
    lo, nn, hi, s = _geometry(dims, n, m)
    a = atk.ttm_gram(x, lo, nn, hi, U, s, 48)
    b = atk.ttm_gram(x, lo, nn, hi, U, s, 48)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_ttm_gram_refuses_unsupported_geometry(atk):
    x = torch.zeros(64 * 8 * 10, device="cuda")
    U = torch.zeros(64, 8, device="cuda")
    with pytest.raises(atk.AtuckerError):
        atk.ttm_gram(x, 1, 64, 80, U, 1, 8)      # I_m = 8 < 16
    with pytest.raises(atk.AtuckerError):
        atk.ttm_gram(x, 1, 64, 80, U, 1, 30)     # 30 does not divide the 80 rows
    U70 = torch.zeros(64, 70, device="cuda")
    with pytest.raises(atk.AtuckerError):
        atk.ttm_gram(x, 1, 64, 80, U70, 1, 16)   # R = 70 > 64


def _plan_run(atk, x, dims, ranks, mode_order, fuse):
    p = atk.Plan(dims, ranks, mode_order=mode_order)
    p.set_option(atk.OPT_FUSE_TTM_GRAM, 1 if fuse else 0)
    core, fac = p.run(_cuda(x))
    torch.cuda.synchronize()
    facs = [f.cpu().double().numpy() for f in p.split_factors(fac)]
    p.close()
    return core.cpu().double().numpy(), facs


@pytest.mark.parametrize("dims,ranks,mode_order", [
    ([96, 96, 96], [8, 8, 8], None),
    ([40, 48, 36, 32], [8, 16, 6, 8], None),
    ([30, 64, 20, 24], [5, 16, 4, 6], [3, 1, 0, 2]),
    ([128, 64, 64], [16, 32, 8], None),
])
def test_plan_with_and_without_fusion_match_oracle(atk, dims, ranks, mode_order):
    x, _, _ = synth.random_tucker(dims, ranks, noise=1e-3, seed=11)
    x64 = x.astype(np.float64)
    ref = oracle.sthosvd(x64, dims, ranks, mode_order=mode_order)
    rel_o = oracle.relerr(x64, ref["core"], ranks, ref["factors"], dims)
    for fuse in (True, False):
        core, facs = _plan_run(atk, x, dims, ranks, mode_order, fuse)
        rel_g = oracle.relerr(x64, core, ranks, facs, dims)
        assert abs(rel_g - rel_o) <= 1e-5
        for U, Uo in zip(facs, ref["factors"]):
            assert oracle.projector_distance(U, Uo) <= 1e-4
