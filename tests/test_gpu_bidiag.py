"""The bidiagonalization route of the batched SVD (K2): Householder reduction,
bisection on Sturm counts of the Golub-Kahan tridiagonal, inverse iteration
and back-transformation of the kept vectors.

Kernel level against LAPACK (singular values to a few eps |M| absolute, right
vectors by residual, orthonormality and, where the value is isolated, by angle),
then the whole hot path with the route forced on every level against the
oracle, per trajectory, at the parity tolerance of the Jacobi route.
"""
import numpy as np
import pytest

from oracle import ising
from oracle.trg import Problem, run_many
from paper_1710_03757_gb300 import build, mctrg
from paper_1710_03757_gb300.workloads import generic_tensor, seed_for

from parity import compare
from test_gpu_parity import gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    build.build()
    mctrg.lib()
    return pytest.importorskip("torch")


def _matrices(n, batch, kind, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(batch):
        if kind == "gauss":
            A = rng.standard_normal((n, n))
        elif kind == "graded":           # singular values over 14 decades
            U, _ = np.linalg.qr(rng.standard_normal((n, n)))
            V, _ = np.linalg.qr(rng.standard_normal((n, n)))
            A = (U * np.logspace(0, -14, n)) @ V.T
        elif kind == "pairs":            # every singular value twice
            U, _ = np.linalg.qr(rng.standard_normal((n, n)))
            V, _ = np.linalg.qr(rng.standard_normal((n, n)))
            s = np.repeat(np.linspace(1.0, 0.05, (n + 1) // 2), 2)[:n]
            A = (U * s) @ V.T
        else:                            # rank n // 3
            r = max(1, n // 3)
            A = rng.standard_normal((n, r)) @ rng.standard_normal((r, n))
        out.append(A)
    return np.stack(out)


def _run(torch, A, nv):
    batch, n = A.shape[0], A.shape[1]
    M = torch.tensor(A, device="cuda")
    sig = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    vt = torch.zeros((batch, nv, n), dtype=torch.float64, device="cuda") if nv else None
    st = mctrg.mctrg_svd_bidiag_batched(M, sig, vt)
    assert st == 0, mctrg.mctrg_strerror(st)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), (vt.cpu().numpy() if nv else None)


@pytest.mark.parametrize("n", [2, 3, 16, 33, 64, 100, 256, 300, 600, 1024])
@pytest.mark.parametrize("kind", ["gauss", "graded", "lowrank", "pairs"])
def test_values_and_kept_vectors_against_lapack(torch, n, kind):
    # n = 300, 600 and 1024 take the 16-, 24- and 32-chunk register layouts of the reduction
    batch = (1 if n > 600 else 2) if n > 256 else (5 if n == 256 else 12)
    nv = min(16, n)
    A = _matrices(n, batch, kind, seed=1000 + n * 7 + len(kind))
    sg, V = _run(torch, A, nv)
    for b in range(batch):
        _, ref, Vr = np.linalg.svd(A[b])
        s1 = ref[0]
        np.testing.assert_allclose(sg[b], ref, atol=1e-13 * s1 * max(1, n) ** 0.5, rtol=0)
        # vectors of values at the noise level are not determined (the null
        # space of a rank-deficient matrix): checked above 1e-10 s_1, as for Jacobi
        kv = int(np.sum(sg[b][:nv] > 1e-10 * s1))
        Vb = V[b][:kv]
        np.testing.assert_allclose(Vb @ Vb.T, np.eye(kv), atol=1e-12)
        # residual of the normal equations, A^T A v = s^2 v, relative to s_1^2
        R = A[b].T @ (A[b] @ Vb.T) - Vb.T * sg[b][:kv] ** 2
        assert np.abs(R).max() <= 1e-12 * s1 * s1
        for r in range(kv):
            gap = min([abs(ref[r] - ref[q]) for q in (r - 1, r + 1) if 0 <= q < n] + [np.inf])
            if gap > 1e-3 * s1 and ref[r] > 1e-6 * s1:
                # isolated value: the vector itself, to about eps |A| / gap
                err = min(np.linalg.norm(Vb[r] - Vr[r]), np.linalg.norm(Vb[r] + Vr[r]))
                assert err <= 1e-12 + 1e-13 * s1 / gap
            else:
                # cluster: the vector lies in the span of the cluster's vectors
                C = [q for q in range(n) if abs(ref[q] - ref[r]) <= 2e-3 * s1]
                proj = Vr[C] @ Vb[r]
                assert abs(np.linalg.norm(proj) - 1.0) <= 1e-10


@pytest.mark.parametrize("n,kind,nv", [(1040, "lowrank", 48), (1600, "gauss", 40), (1600, "graded", 40),
                                       (1600, "pairs", 40), (2304, "gauss", 64)])
def test_wide_values_and_vectors_against_lapack(torch, n, kind, nv):
    # sides above 1024 take the streamed form of the reduction; 64 kept vectors
    # take two warps of inverse iteration and, at n = 2304, back-transformation
    # groups of 8
    A = _matrices(n, 1, kind, seed=3000 + n + len(kind))
    sg, V = _run(torch, A, nv)
    _, ref, Vr = np.linalg.svd(A[0])
    s1 = ref[0]
    np.testing.assert_allclose(sg[0], ref, atol=1e-13 * s1 * n ** 0.5, rtol=0)
    kv = int(np.sum(sg[0][:nv] > 1e-10 * s1))
    Vb = V[0][:kv]
    np.testing.assert_allclose(Vb @ Vb.T, np.eye(kv), atol=1e-12)
    R = A[0].T @ (A[0] @ Vb.T) - Vb.T * sg[0][:kv] ** 2
    assert np.abs(R).max() <= 1e-12 * s1 * s1
    for r in range(kv):
        gap = min([abs(ref[r] - ref[q]) for q in (r - 1, r + 1) if 0 <= q < n] + [np.inf])
        if gap > 1e-3 * s1 and ref[r] > 1e-6 * s1:
            err = min(np.linalg.norm(Vb[r] - Vr[r]), np.linalg.norm(Vb[r] + Vr[r]))
            assert err <= 1e-12 + 1e-13 * s1 / gap
        else:
            C = [q for q in range(n) if abs(ref[q] - ref[r]) <= 2e-3 * s1]
            assert abs(np.linalg.norm(Vr[C] @ Vb[r]) - 1.0) <= 1e-10


def test_zero_and_tiny_matrices(torch):
    A = np.zeros((3, 8, 8))
    A[1, 0, 0] = 1e-300                  # far below the underflow guard's range
    A[2] = np.diag(np.arange(8.0, 0.0, -1.0))
    sg, V = _run(torch, A, 4)
    assert np.all(sg[0] == 0.0)
    assert sg[1][0] == pytest.approx(1e-300, rel=1e-12) and np.all(sg[1][1:] == 0.0)
    np.testing.assert_allclose(sg[2], np.arange(8.0, 0.0, -1.0), rtol=0, atol=1e-14 * 8)
    np.testing.assert_allclose(np.abs(V[2]), np.eye(8)[:4], atol=1e-12)


def test_errors():
    build.build()
    assert mctrg.lib().mctrg_svd_bidiag_batched(None, 8, 1, None, 0, None, None) == mctrg.MCTRG_EINVAL


# ---- the whole path with the route forced ----------------------------------

@pytest.mark.parametrize("L,chi,D,n", [(4, 2, 2, 300), (4, 3, 2, 300), (8, 4, 2, 120), (4, 4, 3, 80),
                                       (8, 3, 3, 40)])
def test_generic_tensor_parity_bidiag(torch, L, chi, D, n):
    T0 = generic_tensor(D, seed=100 + 10 * L + chi + D)
    seed = 0xC0FFEE + L + chi
    gpu = gpu_run(L, chi, n, seed, T0=T0, svd=mctrg.SVD_BIDIAG)
    orc = run_many(Problem(T0, L, chi), seed, 0, n)
    assert compare(gpu, orc, min_ok=0.9, label="bidiag generic L%d chi%d D%d" % (L, chi, D)) >= 0.9 * n


def test_chi48_generic_parity(torch):
    # D = 7 generic tensor, chi = 48 on L = 2: 48 of the 49 values of level 0
    # are sampled (two lane sets of the sampler tables), then level 1 has
    # 2304 x 2304 matrices of rank <= 49 (streamed reduction, 48 kept vectors:
    # two warps of inverse iteration, back-transformation groups of 8)
    T0 = generic_tensor(7, seed=4807)
    seed = 0x48
    gpu = gpu_run(2, 48, 8, seed, T0=T0)
    orc = run_many(Problem(T0, 2, 48), seed, 0, 8, workers=8)
    compare(gpu, orc, min_ok=0.5, label="generic D7 L2 chi48")


@pytest.mark.parametrize("beta,h,L,chi,n", [(0.3, 0.1, 8, 4, 100), (0.44, 0.05, 8, 2, 200)])
def test_ising_parity_bidiag(torch, beta, h, L, chi, n):
    seed = 991 + L
    gpu = gpu_run(L, chi, n, seed, beta=beta, h=h, svd=mctrg.SVD_BIDIAG)
    orc = run_many(Problem(ising.site_tensor(beta, h), L, chi), seed, 0, n)
    compare(gpu, orc, min_ok=0.9, label="bidiag ising b%g h%g L%d chi%d" % (beta, h, L, chi))


@pytest.mark.parametrize("case", ["ising", "generic3"])
def test_chi32_parity_n1024_levels(torch, case):
    # chi = 32: the deepest levels are 1024 x 1024 (32-chunk reduction, vectors in
    # two back-transformation groups of 16).  (A D = 2 generic tensor at this
    # chi keeps values below 1e-7 s_1 in every trajectory: all flagged.)
    if case == "ising":
        T0, L, n = ising.site_tensor(0.3, 0.0), 8, 8
        gpu = gpu_run(L, 32, n, 31, beta=0.3)
    else:
        T0, L, n = generic_tensor(3, seed=9), 8, 6
        gpu = gpu_run(L, 32, n, 31, T0=T0)
    orc = run_many(Problem(T0, L, 32), 31, 0, n, workers=n)
    # measured: Ising none flagged; the D = 3 generic tensor 2 of 6 (kept values below 1e-7 s_1)
    compare(gpu, orc, min_ok=0.9 if case == "ising" else 0.5, label="chi32 " + case)


def test_n64_parity_bidiag(torch):
    T0 = generic_tensor(2, seed=7)
    gpu = gpu_run(8, 8, 24, 5, T0=T0, svd=mctrg.SVD_BIDIAG)
    orc = run_many(Problem(T0, 8, 8), 5, 0, 24, workers=4)
    compare(gpu, orc, min_ok=0.8, label="bidiag n64")


@pytest.mark.parametrize("L,beta,h,n", [(16, 0.44, 0.0, 32), (32, 0.40, 0.05, 16), (64, 0.44, 0.0, 16)])
def test_ising_chi16_parity_auto_route(torch, L, beta, h, n):
    # the automatic route: bidiagonalization on the full-rank 256 x 256 levels
    seed = seed_for(2) + L
    gpu = gpu_run(L, 16, n, seed, beta=beta, h=h)
    orc = run_many(Problem(ising.site_tensor(beta, h), L, 16), seed, 0, n, workers=8)
    compare(gpu, orc, min_ok=0.9, label="auto ising chi16 L%d" % L)


def test_routes_agree_at_L1024(torch):
    # the headline lattice: two trajectories through each route.  A
    # trajectory's ln Z~ amplifies rounding differences level by level (the
    # reweighted small singular values of each truncation): two backward-stable
    # FP64 SVDs agree to ~1e-16 at L = 64, ~1e-12 at L = 128, ~1e-10 at
    # L = 256 and ~1e-8 at L = 1024, so the bound here is that of the mixed
    # modes; the draws and flags are identical
    a = gpu_run(1024, 16, 2, seed_for(2), beta=0.44, svd=mctrg.SVD_JACOBI)
    b = gpu_run(1024, 16, 2, seed_for(2), beta=0.44)
    np.testing.assert_array_equal(a[3], b[3])
    np.testing.assert_array_equal(a[2], b[2])
    assert np.all(np.abs(a[1] - b[1]) <= 1e-6 * np.abs(a[1]))
    f = ising.onsager_minus_beta_f(0.44)
    assert np.all(np.abs(b[1] / 1024 ** 2 - f) < 2e-3)
