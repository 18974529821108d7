"""Mixed precision (the contraction on the tensor cores, SVD and sampling in
FP64): every result is compared with the FP64 path on the same trajectories,
with the oracle trajectory by trajectory, and with the exact Z.

TF32X3 (error-compensated TF32, three tcgen05 passes) must stay within 1e-6
of FP64 in the median per-trajectory ln Z and in the estimate; the single-pass
modes are held to looser bounds that document their error.  Against the
oracle (FP64, LAPACK SVD) the maximum and the per-site absolute ln Z errors
are bounded at 32 x 32 and 64 x 64; against Kaufman's exact Z the mixed
modes' estimates are unbiased within 3 standard errors, which bounds the
bias from their larger zero threshold (singular values below sqrt(n) u s_1
count as zeros) by the statistical error."""
import math
import os

import numpy as np
import pytest

from oracle import ising
from oracle.trg import Problem, run_many
from paper_1710_03757_gb300 import build, mctrg
from paper_1710_03757_gb300.workloads import generic_tensor, seed_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def run(prec, L=32, chi=16, n=64, seed=7, beta=0.44, T0=None):
    ctx = mctrg.mctrg_create(mctrg.make_options(precision=prec))
    try:
        s = (mctrg.mctrg_init_lattice(ctx, beta, 0.0, L, chi) if T0 is None
             else mctrg.mctrg_init_tensor(ctx, T0, T0.shape[0], L, chi))
        assert s == 0
        ln = np.zeros(n)
        sg = np.zeros(n, np.int8)
        st, est = mctrg.mctrg_run(ctx, n, seed, 0, ln, sg, None)
        return st, est, ln, sg
    finally:
        mctrg.mctrg_destroy(ctx)


@pytest.fixture(scope="module")
def fp64_ref():
    return run(mctrg.MCTRG_FP64)


@pytest.mark.parametrize("prec,med_tol,est_tol", [(mctrg.MCTRG_TF32X3, 1e-6, 1e-6),
                                                   (mctrg.MCTRG_BF16X3, 1e-5, 1e-5),
                                                   (mctrg.MCTRG_TF32, 1e-3, 1e-3),
                                                   (mctrg.MCTRG_BF16, 1e-2, 1e-2)])
def test_against_fp64(fp64_ref, prec, med_tol, est_tol):
    st0, est0, ln0, sg0 = fp64_ref
    st, est, ln, sg = run(prec)
    assert st == mctrg.MCTRG_OK, mctrg.mctrg_strerror(st)
    assert np.mean(sg == sg0) >= 0.95
    err = np.abs(ln - ln0) / np.abs(ln0)
    assert np.median(err) <= med_tol, np.median(err)
    assert abs(est.ln_mean_Z - est0.ln_mean_Z) / abs(est0.ln_mean_Z) <= est_tol


def test_generic_tensor_mixed():
    T0 = generic_tensor(2, seed=8)
    st0, est0, ln0, _ = run(mctrg.MCTRG_FP64, L=8, chi=16, n=16, T0=T0)
    st, est, ln, _ = run(mctrg.MCTRG_TF32X3, L=8, chi=16, n=16, T0=T0)
    assert st == 0 and st0 == 0
    assert np.median(np.abs(ln - ln0) / np.abs(ln0)) <= 1e-6


def test_chi32_tensor_core_levels():
    # chi = 32: the 1024 x 1024 plaquette GEMMs run on the tensor cores in
    # 128 x 256 output tiles (four column tiles per tensor)
    st0, est0, ln0, sg0 = run(mctrg.MCTRG_FP64, L=16, chi=32, n=4)
    st, est, ln, sg = run(mctrg.MCTRG_TF32X3, L=16, chi=32, n=4)
    assert st0 == 0 and st == 0
    np.testing.assert_array_equal(sg, sg0)
    assert np.median(np.abs(ln - ln0) / np.abs(ln0)) <= 1e-6


def test_chi32_fp64tc_against_oracle():
    # chi = 32: inner dimension 1024, so the split uses 7-bit slices (8 of
    # them, 36 exact slice products, eight accumulators filling tensor memory);
    # per trajectory against the oracle at the FP64 bound
    L, chi, n, seed = 8, 32, 6, 31
    st, est, ln, sg = run(mctrg.MCTRG_FP64TC, L=L, chi=chi, n=n, seed=seed, beta=0.3)
    assert st == 0
    os_, ol, of = run_many(Problem(ising.site_tensor(0.3, 0.0), L, chi), seed, 0, n, workers=n)
    ok = of == 0
    assert ok.sum() >= n - 1
    np.testing.assert_array_equal(sg[ok], os_[ok])
    rel = np.abs(ln[ok] - ol[ok]) / np.maximum(1.0, np.abs(ol[ok]))
    assert rel.max() <= 1e-10, rel.max()


# per-trajectory bounds against the oracle (maximum relative ln Z error, and
# maximum absolute ln Z error per site), measured on GB300 with these seeds:
# TF32X3 6.8e-8 / 6.3e-8 at 32 x 32 and 64 x 64, within the 1e-6 target;
# BF16X3 3.2e-6 at 32 x 32 and 1.0e-4 at 64 x 64 (its median is 8e-7), so
# BF16X3 does not meet the 1e-6 target per trajectory; FP64TC (the BF16-slice
# GEMM at FP64 accuracy) is held to the FP64 parity bound.
ORACLE_BOUNDS = {mctrg.MCTRG_TF32X3: (1e-6, 1e-7), mctrg.MCTRG_BF16X3: (3e-4, 3e-4),
                 mctrg.MCTRG_FP64TC: (1e-10, 1e-10)}


@pytest.mark.parametrize("prec", [mctrg.MCTRG_TF32X3, mctrg.MCTRG_BF16X3, mctrg.MCTRG_FP64TC])
@pytest.mark.parametrize("L,n", [(32, 16), (64, 8)])
def test_mixed_against_oracle(prec, L, n):
    seed = seed_for(3) + L
    st, est, ln, sg = run(prec, L=L, chi=16, n=n, seed=seed)
    assert st == mctrg.MCTRG_OK, mctrg.mctrg_strerror(st)
    os_, ol, of = run_many(Problem(ising.site_tensor(0.44, 0.0), L, 16), seed, 0, n,
                           workers=min(n, os.cpu_count() or 1))
    ok = of == 0
    assert ok.sum() >= n // 2
    np.testing.assert_array_equal(sg[ok], os_[ok])
    rel = np.abs(ln[ok] - ol[ok]) / np.abs(ol[ok])
    per_site = np.abs(ln[ok] - ol[ok]) / (L * L)
    print("mixed %d L%d vs oracle: max rel %.3e median rel %.3e max abs per site %.3e"
          % (prec, L, rel.max(), np.median(rel), per_site.max()))
    max_rel, max_site = ORACLE_BOUNDS[prec]
    assert rel.max() <= max_rel and per_site.max() <= max_site


@pytest.mark.parametrize("prec", [mctrg.MCTRG_FP64, mctrg.MCTRG_TF32X3, mctrg.MCTRG_BF16X3, mctrg.MCTRG_FP64TC])
def test_mixed_unbiased_against_kaufman(prec):
    # 16 x 16, chi = 16: every distinct level's plaquette GEMM (256 x 256, inner
    # dimension 256) runs on the tensor cores in the mixed modes
    L, beta, n = 16, 0.44, 4000
    st, est, ln, sg = run(prec, L=L, chi=16, n=n, seed=seed_for(3), beta=beta)
    assert st == mctrg.MCTRG_OK
    z = math.exp(ising.kaufman_lnZ(L, beta) - est.ln_scale)
    zscore = (est.mean_Z_scaled - z) / est.se_Z_scaled
    print("mode %d L16 chi16: ln Z^ - ln Z = %.3e, SE(ln Z) = %.3e, z = %.2f"
          % (prec, est.ln_mean_Z - ising.kaufman_lnZ(L, beta), est.se_ln_Z, zscore))
    assert abs(zscore) <= 3.0
