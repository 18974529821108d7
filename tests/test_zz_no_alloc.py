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


def test_no_alloc_matches_allocating_call_twice():
    build.build()
    torch = pytest.importorskip("torch")
    # two calls in a row with different shapes: the second must not see the
    # first call's leftovers in the shared working array
    for call, (n, batch, graded) in enumerate([(64, 40, False), (256, 5, True)]):
        A = _inputs(n, batch, seed=11 + call, graded=graded)
        M = torch.tensor(A, device="cuda")
        sig_a = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
        vt_a = torch.zeros((batch, n, n), dtype=torch.float64, device="cuda")
        sig_b = torch.full((batch, n), float("nan"), dtype=torch.float64, device="cuda")
        vt_b = torch.full((batch, n, n), float("nan"), dtype=torch.float64, device="cuda")
        assert mctrg.mctrg_svd_batched(M, sig_a, vt_a) == mctrg.MCTRG_OK
        assert mctrg.mctrg_svd_batched_noalloc(M, sig_b, vt_b) == mctrg.MCTRG_OK
        torch.cuda.synchronize()
        sa, sb = sig_a.cpu().numpy(), sig_b.cpu().numpy()
        va, vb = vt_a.cpu().numpy(), vt_b.cpu().numpy()
        for b in range(batch):
            s1 = sa[b][0]
            # the tolerance of the SVD parity tests
            np.testing.assert_allclose(sb[b], sa[b], atol=1e-13 * s1 * n ** 0.5, rtol=0)
            keep = sa[b] > 1e-10 * s1
            np.testing.assert_allclose(np.abs(np.sum(va[b][keep] * vb[b][keep], axis=1)), 1.0, atol=1e-9)


def test_no_alloc_rejects_sizes_above_its_maximum():
    build.build()
    torch = pytest.importorskip("torch")
    n = 1025
    M = torch.zeros((1, 2, 2), dtype=torch.float64, device="cuda")
    sig = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    st = mctrg.lib().mctrg_svd_batched_noalloc(M.data_ptr(), n, 1, sig.data_ptr(), None, 0, None)
    assert st == mctrg.MCTRG_EINVAL
