"""The plaquette GEMM on its own (M = X Yt^T, the end of the coarse-graining
contraction of Sec. III) through the C ABI: FP64 on the CUDA cores and the
FP64-accurate tensor-core form (BF16 slices multiplied exactly, Ozaki
scheme), against exact products.

* integer matrices whose products are exact in FP64: both forms bit-exact;
* every slice at its largest magnitude with one sign (the bound on a group's
  sum that keeps the FP32 accumulation exact is reached): the tensor-core
  form stays within its stated truncation bound of the exact product, which
  an inexact group accumulation (2^-24 of a group) would break by orders of
  magnitude;
* Gaussian and graded-magnitude data: the error against exact rational
  arithmetic (sampled entries) below 2^-43 K |row max| |column max|, and
  within 8 times the FP64 GEMM's own error plus 2^-50 of that scale;
* ragged tiles (n = 81, 576) and the largest inner dimension (1024).
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_1710_03757_gb300 import build, mctrg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    build.build()
    mctrg.lib()
    return pytest.importorskip("torch")


def _run(torch, X, Y, prec):
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.tensor(Y, device="cuda")
    M = torch.full((X.shape[0], X.shape[1], X.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
    st = mctrg.mctrg_contract_batched(Xd, Yd, M, precision=prec)
    assert st == mctrg.MCTRG_OK, mctrg.mctrg_strerror(st)
    return M.cpu().numpy()


def _exact(X, Y, b, r, c):
    return sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(X[b, r], Y[b, c]))


@pytest.mark.parametrize("D,K", [(8, 64), (9, 128), (16, 256), (24, 576), (32, 1024)])
def test_integer_matrices_are_exact(torch, D, K):
    rng = np.random.default_rng(D * 1000 + K)
    n, batch = D * D, 3
    # |x| < 2^20: every product and every sum of K products is an integer below 2^53
    X = rng.integers(-(1 << 20), 1 << 20, size=(batch, n, K)).astype(np.float64)
    Y = rng.integers(-(1 << 20), 1 << 20, size=(batch, n, K)).astype(np.float64)
    ref = np.einsum('bik,bjk->bij', X, Y)
    for prec in (mctrg.MCTRG_FP64, mctrg.MCTRG_FP64TC):
        np.testing.assert_array_equal(_run(torch, X, Y, prec), ref)


@pytest.mark.parametrize("K", [256, 1024])
def test_largest_slices_one_sign(torch, K):
    # x with every slice at +-(2^(b-1) - 1) and one sign, so that each group of
    # slice products sums to its largest magnitude
    bits, slices = (8, 7) if K <= 256 else (7, 8)
    a = (1 << (bits - 1)) - 1
    x = sum(Fraction(a, 1 << ((bits - 1) + bits * i)) for i in range(6))
    xv = float(x)
    assert Fraction(xv) == x                                    # 6 slices: exactly representable
    D = 16
    X = np.full((1, D * D, K), xv)
    Y = np.full((1, D * D, K), -xv)
    M = _run(torch, X, Y, mctrg.MCTRG_FP64TC)
    exact = -K * x * x
    err = abs(Fraction(float(M[0, 0, 0])) - exact)
    assert err <= Fraction(1, 2 ** 43) * K * x * x
    assert np.all(M == M[0, 0, 0])


@pytest.mark.parametrize("kind", ["gauss", "graded"])
@pytest.mark.parametrize("D,K", [(16, 256), (9, 64), (32, 1024)])
def test_against_exact_arithmetic(torch, kind, D, K):
    rng = np.random.default_rng(7 + D + K)
    n, batch = D * D, 2
    X = rng.standard_normal((batch, n, K))
    Y = rng.standard_normal((batch, n, K))
    if kind == "graded":   # rows and columns over 12 decades, entries over 6
        X *= np.logspace(0, -12, n)[None, :, None] * 10 ** rng.uniform(-6, 0, (batch, n, K))
        Y *= np.logspace(-12, 0, n)[None, :, None] * 10 ** rng.uniform(-6, 0, (batch, n, K))
    Mt = _run(torch, X, Y, mctrg.MCTRG_FP64TC)
    Mf = _run(torch, X, Y, mctrg.MCTRG_FP64)
    worst_tc, worst_f = 0.0, 0.0
    for _ in range(60):
        b, r, c = int(rng.integers(batch)), int(rng.integers(n)), int(rng.integers(n))
        ex = _exact(X, Y, b, r, c)
        scale = float(np.abs(X[b, r]).max() * np.abs(Y[b, c]).max())
        et = abs(float(Fraction(float(Mt[b, r, c])) - ex))
        ef = abs(float(Fraction(float(Mf[b, r, c])) - ex))
        assert et <= 2.0 ** -43 * K * scale, (et, scale)
        assert et <= 8 * ef + 2.0 ** -50 * K * scale
        worst_tc, worst_f = max(worst_tc, et / (K * scale)), max(worst_f, ef / (K * scale))
    print("D%d K%d %s: max error / (K |row max| |col max|): FP64TC %.2e, FP64 %.2e"
          % (D, K, kind, worst_tc, worst_f))


def test_rejects_unsupported_shapes(torch):
    X = torch.zeros((1, 16, 48), dtype=torch.float64, device="cuda")
    M = torch.zeros((1, 16, 16), dtype=torch.float64, device="cuda")
    assert mctrg.mctrg_contract_batched(X, X, M, precision=mctrg.MCTRG_FP64TC) == mctrg.MCTRG_EINVAL
    assert mctrg.mctrg_contract_batched(X, X, M, precision=mctrg.MCTRG_TF32) == mctrg.MCTRG_EINVAL
