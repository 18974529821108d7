"""The two-stage (band) route of the batched SVD (K2): dense -> band with the
trailing products on the tensor cores (8-bit digit slices, fixed-point
trailing matrix), band -> bidiagonal by bulge chasing, bisection, inverse
iteration and the back-transformation through both stages.

Each stage against LAPACK: the band and the bidiagonal are orthogonal
two-sided transformations of M, so their singular values equal M's to a few
eps |M|; then values and kept vectors of the whole route, and agreement with
the one-stage bidiagonalization route on the same matrices.
"""
import numpy as np
import pytest

from paper_1710_03757_gb300 import build, mctrg

pytestmark = pytest.mark.gpu

B = 8


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
        elif kind == "scaled":           # large norm: the fixed point's exponent far from 0
            A = rng.standard_normal((n, n)) * 3.0e5
        else:                            # rank n // 3
            r = max(1, n // 3)
            A = rng.standard_normal((n, r)) @ rng.standard_normal((r, n))
        out.append(A)
    return np.stack(out)


def _dense_band(band, n):
    D = np.zeros((n, n))
    for i in range(n):
        for o in range(B + 1):
            if i + o < n:
                D[i, i + o] = band[i, o]
    return D


def _reduce(torch, A, with_bd):
    batch, n = A.shape[0], A.shape[1]
    M = torch.tensor(A, device="cuda")
    band = torch.full((batch, n, B + 1), float("nan"), dtype=torch.float64, device="cuda")
    bd = torch.full((batch, 3 * n), float("nan"), dtype=torch.float64, device="cuda") if with_bd else None
    st = mctrg.mctrg_band_reduce_batched(M, band, bd)
    assert st == 0, mctrg.mctrg_strerror(st)
    torch.cuda.synchronize()
    return band.cpu().numpy(), (bd.cpu().numpy() if with_bd else None)


@pytest.mark.parametrize("n", [64, 136, 256])
@pytest.mark.parametrize("kind", ["gauss", "graded", "lowrank", "scaled"])
def test_band_and_bidiagonal_keep_the_singular_values(torch, n, kind):
    batch = 3
    A = _matrices(n, batch, kind, seed=500 + n + len(kind))
    band, bd = _reduce(torch, A, True)
    for b in range(batch):
        ref = np.linalg.svd(A[b], compute_uv=False)
        s1 = ref[0]
        Db = _dense_band(band[b], n)
        np.testing.assert_allclose(np.linalg.svd(Db, compute_uv=False), ref, atol=1e-13 * s1 * n ** 0.5, rtol=0)
        # Frobenius norm kept (orthogonal transformations)
        assert abs(np.linalg.norm(Db) - np.linalg.norm(A[b])) <= 1e-13 * np.linalg.norm(A[b])
        d, e = bd[b][:n], bd[b][n:2 * n]
        assert e[n - 1] == 0.0 and np.all(bd[b][2 * n:] == 0.0)
        Bi = np.diag(d) + np.diag(e[:n - 1], 1)
        np.testing.assert_allclose(np.linalg.svd(Bi, compute_uv=False), ref, atol=1e-13 * s1 * n ** 0.5, rtol=0)


def _run(torch, A, nv, route):
    batch, n = A.shape[0], A.shape[1]
    M = torch.tensor(A, device="cuda")
    sig = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    vt = torch.zeros((batch, nv, n), dtype=torch.float64, device="cuda") if nv else None
    fn = mctrg.mctrg_svd_band_batched if route == "band" else mctrg.mctrg_svd_bidiag_batched
    st = fn(M, sig, vt)
    assert st == 0, mctrg.mctrg_strerror(st)
    torch.cuda.synchronize()
    return sig.cpu().numpy(), (vt.cpu().numpy() if nv else None)


@pytest.mark.parametrize("n", [64, 128, 200, 256])
@pytest.mark.parametrize("kind", ["gauss", "graded", "lowrank", "pairs"])
def test_values_and_kept_vectors_against_lapack(torch, n, kind):
    batch = 5 if n == 256 else 8
    nv = 16
    A = _matrices(n, batch, kind, seed=2000 + n * 7 + len(kind))
    sg, V = _run(torch, A, nv, "band")
    for b in range(batch):
        _, ref, Vr = np.linalg.svd(A[b])
        s1 = ref[0]
        np.testing.assert_allclose(sg[b], ref, atol=1e-13 * s1 * n ** 0.5, rtol=0)
        kv = int(np.sum(sg[b][:nv] > 1e-10 * s1))
        Vb = V[b][:kv]
        np.testing.assert_allclose(Vb @ Vb.T, np.eye(kv), atol=1e-12)
        R = A[b].T @ (A[b] @ Vb.T) - Vb.T * sg[b][:kv] ** 2
        assert np.abs(R).max() <= 1e-12 * s1 * s1
        for r in range(kv):
            gap = min([abs(ref[r] - ref[q]) for q in (r - 1, r + 1) if 0 <= q < n] + [np.inf])
            if gap > 1e-3 * s1 and ref[r] > 1e-6 * s1:
                err = min(np.linalg.norm(Vb[r] - Vr[r]), np.linalg.norm(Vb[r] + Vr[r]))
                assert err <= 1e-12 + 1e-13 * s1 / gap
            else:
                C = [q for q in range(n) if abs(ref[q] - ref[r]) <= 2e-3 * s1]
                assert abs(np.linalg.norm(Vr[C] @ Vb[r]) - 1.0) <= 1e-10


def test_agrees_with_the_one_stage_route(torch):
    # both routes are backward stable: values agree to a few eps |M|
    n, batch = 256, 6
    A = _matrices(n, batch, "graded", seed=77)
    s_band, V_band = _run(torch, A, 8, "band")
    s_bd, V_bd = _run(torch, A, 8, "bidiag")
    for b in range(batch):
        s1 = s_bd[b][0]
        np.testing.assert_allclose(s_band[b], s_bd[b], atol=1e-13 * s1 * n ** 0.5, rtol=0)
        for r in range(8):
            assert min(np.linalg.norm(V_band[b][r] - V_bd[b][r]), np.linalg.norm(V_band[b][r] + V_bd[b][r])) < 1e-9


def test_zero_matrix_and_rejected_sizes(torch):
    A = np.zeros((2, 64, 64))
    A[1] = np.diag(np.arange(64.0, 0.0, -1.0))
    sg, V = _run(torch, A, 4, "band")
    assert np.all(sg[0] == 0.0)
    np.testing.assert_allclose(sg[1], np.arange(64.0, 0.0, -1.0), rtol=0, atol=1e-13 * 64)
    for n in (56, 100, 264):             # below 64, not a multiple of 8, above 256
        M = torch.zeros((1, n, n), dtype=torch.float64, device="cuda")
        s = torch.zeros((1, n), dtype=torch.float64, device="cuda")
        assert mctrg.mctrg_svd_band_batched(M, s) == mctrg.MCTRG_EINVAL


# ---- the whole hot path with the band route, per trajectory against the oracle
from oracle import ising  # noqa: E402
from oracle.trg import Problem, run_many  # noqa: E402
from paper_1710_03757_gb300.workloads import generic_tensor, seed_for  # noqa: E402

from parity import compare  # noqa: E402
from test_gpu_parity import gpu_run  # noqa: E402


def test_n64_generic_parity_band(torch):
    # chi = 8 on a D = 2 generic tensor: the sampled levels are 64 x 64
    T0 = generic_tensor(2, seed=7)
    gpu = gpu_run(8, 8, 24, 5, T0=T0, svd=mctrg.SVD_BAND)
    orc = run_many(Problem(T0, 8, 8), 5, 0, 24, workers=4)
    # the same floor as the one-stage route's case on these trajectories
    compare(gpu, orc, min_ok=0.8, label="band n64")


@pytest.mark.parametrize("L,beta,h,n,prec", [(16, 0.44, 0.0, 32, 0), (32, 0.40, 0.05, 16, 0),
                                             (32, 0.44, 0.0, 16, 5)])
def test_ising_chi16_parity_band(torch, L, beta, h, n, prec):
    # 256 x 256 levels through the band route (prec 5: FP64TC, the contraction too)
    seed = seed_for(2) + L
    gpu = gpu_run(L, 16, n, seed, beta=beta, h=h, svd=mctrg.SVD_BAND, precision=prec)
    orc = run_many(Problem(ising.site_tensor(beta, h), L, 16), seed, 0, n, workers=8)
    compare(gpu, orc, min_ok=0.9, label="band ising chi16 L%d prec%d" % (L, prec))


def test_band_route_at_L1024(torch):
    # the headline lattice: the draws and flags of the default route, ln Z~ to
    # the rounding amplification of a trajectory at this size (1e-6, as between
    # the two one-stage routes)
    a = gpu_run(1024, 16, 2, seed_for(2), beta=0.44)
    b = gpu_run(1024, 16, 2, seed_for(2), beta=0.44, svd=mctrg.SVD_BAND, precision=mctrg.MCTRG_FP64TC)
    np.testing.assert_array_equal(a[3], b[3])
    np.testing.assert_array_equal(a[2], b[2])
    assert np.all(np.abs(a[1] - b[1]) <= 1e-6 * np.abs(a[1]))


def test_batch_rejects_the_band_route(torch):
    assert mctrg.mctrg_batch_run([(0.4, 0.0, 8, 4, 10, 1, 0)],
                                 mctrg.make_options(svd=mctrg.SVD_BAND))[0] == mctrg.MCTRG_EINVAL
