"""The Gram entry point that allocates no device memory.

Callers that cannot allocate GPU memory at call time use
atucker_gram_noalloc.  Examples: a service with a memory budget fixed up front,
or a process whose free device memory a framework's caching allocator already
holds.  It keeps its split-K partial tiles in one fixed 16 MiB array inside
the library.  These tests call it through the C ABI and compare it with
atucker_gram, the allocating entry point, at the tolerance the Gram parity
tests use.  Two consecutive calls on different shapes show that what the
first call leaves in the shared array does not leak into the second.  The
file sorts last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _gram_both(atk, y, lo, n, hi):
    lib = atk.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    s_ref = torch.empty(n * n, device="cuda", dtype=torch.float64)
    s_new = torch.full((n * n,), float("nan"), device="cuda", dtype=torch.float64)
    yp = ctypes.c_void_p(y.data_ptr())
    assert lib.atucker_gram(yp, lo, n, hi, 0, ctypes.c_void_p(s_ref.data_ptr()), stream) == 0
    st = lib.atucker_gram_noalloc(yp, lo, n, hi, ctypes.c_void_p(s_new.data_ptr()), stream)
    assert st == 0, lib.atucker_last_error()
    torch.cuda.synchronize()
    return s_ref.cpu().numpy().reshape(n, n), s_new.cpu().numpy().reshape(n, n)


@pytest.mark.gpu
def test_noalloc_gram_matches_allocating_gram_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2010_10131_b300 as atk
    g = np.random.default_rng(42)
    # First call: 640 rows and a long J, so the 16 MiB array caps the split count.
    # Second call: a smaller, ragged middle-mode view on the same array.
    for lo, n, hi in [(1, 640, 40000), (7, 130, 333)]:
        y_host = g.standard_normal(lo * n * hi).astype(np.float32)
        y = torch.from_numpy(y_host).cuda()
        ref, new = _gram_both(atk, y, lo, n, hi)
        assert np.all(np.isfinite(new))
        scale = np.abs(np.diag(ref)).max()
        tol = 2e-6 * scale * max(1.0, np.sqrt(lo * hi / 8192))
        assert np.abs(new - ref).max() <= tol
        np.testing.assert_array_equal(new, new.T)
        if n == 130:
            # and against a float64 Gram of the same float32 data, on the host
            y3 = y_host.astype(np.float64).reshape(hi, n, lo)
            exact = np.einsum("bia,bja->ij", y3, y3)
            assert np.abs(new - exact).max() <= tol


@pytest.mark.gpu
def test_noalloc_gram_in_rounds_at_n_2048():
    """n = 2048 with a J needing 13 splits of at most 8192 terms: one split's
    partial tiles (136 of 128 x 128) fill the fixed array, so the splits run
    in 13 rounds added in float64; the chains, and so the error, match the
    allocating entry point's."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2010_10131_b300 as atk
    g = np.random.default_rng(7)
    lo, n, hi = 1, 2048, 100000
    y = torch.from_numpy(g.standard_normal(lo * n * hi).astype(np.float32)).cuda()
    ref, new = _gram_both(atk, y, lo, n, hi)
    scale = np.abs(np.diag(ref)).max()
    assert np.abs(new - ref).max() <= 2e-6 * scale * np.sqrt(lo * hi / 8192)
    np.testing.assert_array_equal(new, new.T)


def test_noalloc_gram_rejects_sizes_beyond_its_scratch():
    """n > 2048 is refused before any device work (the pointers are never touched)."""
    import paper_2010_10131_b300 as atk
    lib = atk.lib()
    fake = ctypes.c_void_p(0x1000)
    assert lib.atucker_gram_noalloc(fake, 1, 4096, 8, fake, None) == atk.EUNSUPPORTED
    assert b"2048" in lib.atucker_last_error()
    assert lib.atucker_gram_noalloc(None, 1, 16, 8, fake, None) == atk.EINVAL
