"""Kernel-level parity of the batched Jacobi SVD (K2) against LAPACK."""
import numpy as np
import pytest

from paper_1710_03757_gb300 import build, mctrg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    build.build()
    return pytest.importorskip("torch")


def _matrices(n, batch, kind, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(batch):
        if kind == "gauss":
            A = rng.standard_normal((n, n))
        elif kind == "graded":       # singular values over 14 decades
            U, _ = np.linalg.qr(rng.standard_normal((n, n)))
            V, _ = np.linalg.qr(rng.standard_normal((n, n)))
            A = (U * np.logspace(0, -14, n)) @ V.T
        else:                        # rank n // 3
            r = max(1, n // 3)
            A = rng.standard_normal((n, r)) @ rng.standard_normal((r, n))
        out.append(A)
    return np.stack(out)


@pytest.mark.parametrize("n", [1, 4, 9, 16, 33, 64, 100, 256])
@pytest.mark.parametrize("kind", ["gauss", "graded", "lowrank"])
def test_singular_values_and_vectors(torch, n, kind):
    batch = 6 if n >= 256 else 24
    A = _matrices(n, batch, kind, seed=n * 7 + len(kind))
    M = torch.tensor(A, device="cuda")
    sig = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    vt = torch.zeros((batch, n, n), dtype=torch.float64, device="cuda")
    st = mctrg.mctrg_svd_batched(M, sig, vt)
    assert st == 0, mctrg.mctrg_strerror(st)
    torch.cuda.synchronize()
    sg, V = sig.cpu().numpy(), vt.cpu().numpy()
    for b in range(batch):
        ref = np.linalg.svd(A[b], compute_uv=False)
        s1 = ref[0]
        assert np.all(np.diff(sg[b]) <= 0)
        np.testing.assert_allclose(sg[b], ref, atol=1e-13 * s1 * max(1, n) ** 0.5, rtol=0)
        keep = sg[b] > 1e-10 * s1
        Vk = V[b][keep]
        # orthonormal rows, and M v = s u with |u| = 1 (reconstruction of the kept part)
        np.testing.assert_allclose(Vk @ Vk.T, np.eye(int(keep.sum())), atol=1e-12)
        Uk = (A[b] @ Vk.T) / sg[b][keep]
        # |A v| / s = 1 up to the rounding of A v itself, about eps |A| / s
        err = np.abs(np.linalg.norm(Uk, axis=0) - 1.0)
        assert np.all(err <= 1e-12 + 1e-13 * s1 / sg[b][keep])
        R = A[b] - (Uk * sg[b][keep]) @ Vk
        assert np.linalg.norm(R) <= 1e-12 * max(1.0, np.linalg.norm(A[b])) + 1e-10 * s1 * (n - keep.sum())


def test_rejects_bad_sizes(torch):
    M = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    sig = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    assert mctrg.lib().mctrg_svd_batched(M.data_ptr(), 0, 1, sig.data_ptr(), None, 0, None) == mctrg.MCTRG_EINVAL
    assert mctrg.lib().mctrg_svd_batched(M.data_ptr(), 2048, 1, sig.data_ptr(), None, 0, None) == mctrg.MCTRG_EINVAL
    assert mctrg.lib().mctrg_svd_batched(None, 4, 1, sig.data_ptr(), None, 0, None) == mctrg.MCTRG_EINVAL
