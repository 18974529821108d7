"""Observables by impurity tensors on the device (mctrg_init_impurity), the
partial traces of Sec. III: per trajectory against the oracle's impurity
network (every level split per tensor from level 0), the partial trace
unbiased against brute force, and <sigma> and <sigma sigma> as ratios of
estimates against the transfer-matrix insertion."""
import math

import numpy as np
import pytest

from oracle import ising
from oracle.trg import Problem, run_many
from paper_1710_03757_gb300 import build, mctrg

from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    mctrg.lib()


def imp_run(L, chi, n, seed, beta, h, n_imp, first=0):
    ctx = mctrg.mctrg_create()
    try:
        assert mctrg.mctrg_init_impurity(ctx, beta, h, L, chi, n_imp) == 0
        ln, sg, fl = np.zeros(n), np.zeros(n, np.int8), np.zeros(n, np.uint8)
        st, est = mctrg.mctrg_run(ctx, n, seed, first, ln, sg, fl)
        assert st in (mctrg.MCTRG_OK, mctrg.MCTRG_EDOMAIN), mctrg.mctrg_strerror(st)
        return est, ln, sg, fl
    finally:
        mctrg.mctrg_destroy(ctx)


@pytest.mark.parametrize("L,chi,n_imp,beta,h,n", [(4, 2, 1, 0.4, 0.1, 300), (8, 4, 2, 0.44, 0.0, 100),
                                                  (8, 8, 1, 0.5, 0.05, 24), (16, 16, 2, 0.44, 0.0, 8)])
def test_impurity_parity(L, chi, n_imp, beta, h, n):
    seed = 0x1A + L + chi
    gpu = imp_run(L, chi, n, seed, beta, h, n_imp)
    T0, Ti = ising.site_tensor(beta, h), ising.impurity_tensor(beta, h)
    sites = {0: Ti} if n_imp == 1 else {0: Ti, 1: Ti}
    orc = run_many(Problem(T0, L, chi, site_tensors=sites), seed, 0, n, workers=8)
    compare(gpu, orc, min_ok=0.9, label="impurity L%d chi%d n%d" % (L, chi, n_imp))


def test_partial_trace_unbiased():
    beta, h, L = 0.4, 0.1, 4
    est, _, _, _ = imp_run(L, 2, 40000, 5, beta, h, 1)
    m, lnZ = ising.brute_force_observable(L, beta, h, [(0, 0)])
    z = m * math.exp(lnZ - est.ln_scale)
    assert abs(est.mean_Z_scaled - z) <= 3 * est.se_Z_scaled


@pytest.mark.parametrize("n_imp,h", [(1, 0.1), (2, 0.0)])
def test_observable_ratio_against_transfer_matrix(n_imp, h):
    # <sigma_00> in a field, <sigma_00 sigma_10> (the bond energy) at h = 0, on 8 x 8
    beta, L, chi, n = 0.4, 8, 8, 20000
    num, _, _, _ = imp_run(L, chi, n, 7, beta, h, n_imp)
    ctx = mctrg.mctrg_create()
    try:
        assert mctrg.mctrg_init_lattice(ctx, beta, h, L, chi) == 0
        st, den = mctrg.mctrg_run(ctx, n, 8, 0)
    finally:
        mctrg.mctrg_destroy(ctx)
    st, r, se = mctrg.mctrg_ratio_estimate(num, den)
    assert st == 0
    exact = ising.transfer_observable(L, beta, h, [0] if n_imp == 1 else [0, 1])
    print("n_imp %d: %.6f +- %.6f, exact %.6f" % (n_imp, r, se, exact))
    assert abs(r - exact) <= 3 * se


def test_impurity_rejects_bad_arguments():
    ctx = mctrg.mctrg_create()
    try:
        assert mctrg.mctrg_init_impurity(ctx, 0.4, 0.0, 8, 4, 3) == mctrg.MCTRG_EINVAL
        assert mctrg.mctrg_init_impurity(ctx, 0.4, 0.0, 6, 4, 1) == mctrg.MCTRG_EINVAL
    finally:
        mctrg.mctrg_destroy(ctx)
    ctx = mctrg.mctrg_create(mctrg.make_options(deterministic_levels=2))
    try:
        assert mctrg.mctrg_init_impurity(ctx, 0.4, 0.0, 8, 4, 1) == mctrg.MCTRG_EINVAL
    finally:
        mctrg.mctrg_destroy(ctx)
