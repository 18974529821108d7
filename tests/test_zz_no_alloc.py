"""The allocation-free batched SVD against the allocating one.

mctrg_svd_batched_noalloc serves callers that cannot allocate device memory
(device memory owned by another allocator, loops that must never stall the
device on cudaFree, code barred from allocator calls).  It must return what
mctrg_svd_batched returns, call after call, although every call reuses the
same fixed working array.  This file is collected last so that a run that
stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1710_03757_gb300 import build, mctrg

pytestmark = pytest.mark.gpu


def _inputs(n, batch, seed, graded):
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(batch):
        if graded:
            U, _ = np.linalg.qr(rng.standard_normal((n, n)))
            V, _ = np.linalg.qr(rng.standard_normal((n, n)))
            mats.append((U * np.logspace(0, -12, n)) @ V.T)
        else:
            mats.append(rng.standard_normal((n, n)))
    return np.stack(mats)


def _both(torch, A, max_sweeps=0):
    batch, n = A.shape[0], A.shape[1]
    M = torch.tensor(A, device="cuda")
    sig_a = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    vt_a = torch.zeros((batch, n, n), dtype=torch.float64, device="cuda")
    sig_b = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
    vt_b = torch.full((batch, n, n), float("nan"), dtype=torch.float64, device="cuda")
    st_a = mctrg.mctrg_svd_batched(M, sig_a, vt_a, max_sweeps=max_sweeps)
    st_b = mctrg.mctrg_svd_batched_noalloc(M, sig_b, vt_b, max_sweeps=max_sweeps)
    torch.cuda.synchronize()
    return st_a, st_b, sig_a.cpu().numpy(), sig_b.cpu().numpy(), vt_a.cpu().numpy(), vt_b.cpu().numpy()


def _same(n, sa, sb, va, vb):
    for b in range(sa.shape[0]):
        s1 = sa[b][0]
        # the tolerance of the SVD parity tests
        np.testing.assert_allclose(sb[b], sa[b], atol=1e-13 * s1 * n ** 0.5, rtol=0)
        keep = sa[b] > 1e-10 * s1
        np.testing.assert_allclose(np.abs(np.sum(va[b][keep] * vb[b][keep], axis=1)), 1.0, atol=1e-9)


def test_no_alloc_matches_allocating_call_twice():
    build.build()
    torch = pytest.importorskip("torch")
    # two calls in a row with different shapes: the second must not see the
    # first call's leftovers in the shared working array
    for call, (n, batch, graded) in enumerate([(64, 40, False), (256, 5, True)]):
        A = _inputs(n, batch, seed=11 + call, graded=graded)
        st_a, st_b, sa, sb, va, vb = _both(torch, A)
        assert st_a == mctrg.MCTRG_OK and st_b == mctrg.MCTRG_OK
        _same(n, sa, sb, va, vb)


def test_no_alloc_batches_larger_than_the_array():
    # batches that the fixed array takes in several pieces: 31 matrices of
    # 256 x 256 fit, so 40 take two pieces; a 1024 x 1024 matrix fills the
    # array alone, so 3 take three.  Every piece's offsets into M, sigma and
    # vt, its flag clearing and the OR of the flags across pieces are used.
    build.build()
    torch = pytest.importorskip("torch")
    for call, (n, batch, graded) in enumerate([(256, 40, True), (1024, 3, False)]):
        A = _inputs(n, batch, seed=31 + call, graded=graded)
        st_a, st_b, sa, sb, va, vb = _both(torch, A)
        assert st_a == mctrg.MCTRG_OK and st_b == mctrg.MCTRG_OK
        _same(n, sa, sb, va, vb)


def test_no_alloc_reports_the_sweep_cap():
    # one Jacobi sweep cannot converge on these matrices: both entry points
    # return ENOCONV (results still written), here with the capped matrix in
    # the second of two pieces
    build.build()
    torch = pytest.importorskip("torch")
    A = _inputs(256, 40, seed=5, graded=False)
    st_a, st_b, sa, sb, _, _ = _both(torch, A, max_sweeps=1)
    assert st_a == mctrg.MCTRG_ENOCONV and st_b == mctrg.MCTRG_ENOCONV
    assert np.all(np.isfinite(sb))
    np.testing.assert_allclose(sb, sa, rtol=0, atol=1e-13 * float(np.max(sa)) * 16)
    # and the next call, with the cap lifted, is clean again
    st_a, st_b, sa, sb, va, vb = _both(torch, A[:4])
    assert st_a == mctrg.MCTRG_OK and st_b == mctrg.MCTRG_OK
    _same(256, sa, sb, va, vb)


def test_no_alloc_rejects_sizes_above_its_maximum():
    build.build()
    torch = pytest.importorskip("torch")
    n = 1025
    M = torch.zeros((1, 2, 2), dtype=torch.float64, device="cuda")
    sig = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    st = mctrg.lib().mctrg_svd_batched_noalloc(M.data_ptr(), n, 1, sig.data_ptr(), None, 0, None)
    assert st == mctrg.MCTRG_EINVAL
