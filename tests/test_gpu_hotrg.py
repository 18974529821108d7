"""Monte Carlo HOTRG on the device (mctrg_hotrg_run): the stochastic truncation
of Sec. II on the higher-order TRG, against the oracle per trajectory (same
Philox stream), exact without truncation, unbiased against brute force, and
independent of how trajectories are chunked."""
import math

import numpy as np
import pytest

from oracle import hotrg, ising
from oracle.network import network_trace, plan
from paper_1710_03757_gb300 import build, mctrg
from paper_1710_03757_gb300.workloads import generic_tensor

from parity import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    mctrg.lib()


def hrun(L, chi, n, seed, beta=0.44, h=0.0, T0=None, first=0, **opts):
    ln, sg, fl = np.zeros(n), np.zeros(n, np.int8), np.zeros(n, np.uint8)
    st, est = mctrg.mctrg_hotrg_run(mctrg.make_options(**opts), L, chi, n, seed, first, beta=beta, h=h, T0=T0,
                                    lnabsZ=ln, sign=sg, flags=fl)
    assert st in (mctrg.MCTRG_OK, mctrg.MCTRG_EDOMAIN), mctrg.mctrg_strerror(st)
    return est, ln, sg, fl


@pytest.mark.parametrize("L,beta,h", [(2, 0.44, 0.0), (4, 0.44, 0.0), (4, 0.3, 0.2)])
def test_untruncated_is_exact(L, beta, h):
    est, ln, sg, fl = hrun(L, 16, 4, 3, beta=beta, h=h)
    assert np.all(sg == 1) and np.all(fl == 0)
    np.testing.assert_allclose(ln, ising.brute_force_lnZ(L, beta, h), rtol=1e-12)


def test_untruncated_generic_is_exact():
    T0 = generic_tensor(2, seed=77)
    est, ln, sg, _ = hrun(4, 16, 2, 3, T0=T0)
    z = network_trace([T0] * 16, plan(4)[0])
    np.testing.assert_allclose(sg * np.exp(ln), z, rtol=1e-10)


@pytest.mark.parametrize("case,L,chi,n", [("ising", 4, 3, 200), ("ising", 8, 4, 60), ("ising-field", 8, 6, 40),
                                          ("generic", 4, 3, 100), ("ising", 16, 8, 8)])
def test_parity_with_oracle(case, L, chi, n):
    seed = 0x4070 + L + chi
    if case == "generic":
        T0, beta, h = generic_tensor(2, seed=55), 0.0, 0.0
    else:
        T0, beta, h = None, 0.44, (0.1 if case == "ising-field" else 0.0)
    gpu = hrun(L, chi, n, seed, beta=beta, h=h, T0=T0)
    t0 = ising.site_tensor(beta, h) if T0 is None else T0
    orc = hotrg.run_many(hotrg.HotrgProblem(t0, L, chi), seed, 0, n, workers=8)
    compare(gpu, orc, min_ok=0.9, label="hotrg %s L%d chi%d" % (case, L, chi))


def test_unbiased_against_brute_force():
    beta, L, chi, n = 0.44, 4, 3, 20000
    est, _, _, _ = hrun(L, chi, n, 0x407, beta=beta)
    z = math.exp(ising.brute_force_lnZ(L, beta) - est.ln_scale)
    print("hotrg L4 chi3: mean %.6e  exact %.6e  se %.2e" % (est.mean_Z_scaled, z, est.se_Z_scaled))
    assert abs(est.mean_Z_scaled - z) <= 3 * est.se_Z_scaled


def test_chunking_does_not_change_trajectories():
    a = hrun(8, 4, 40, 21)
    b = hrun(8, 4, 40, 21, max_chunk=7)
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)
    c = hrun(8, 4, 13, 21, first=27)          # trajectories 27 .. 39 alone
    np.testing.assert_array_equal(c[1], a[1][27:])


def test_rejects_bad_arguments():
    o = mctrg.make_options()
    assert mctrg.mctrg_hotrg_run(o, 6, 4, 4, 1)[0] == mctrg.MCTRG_EINVAL      # L not a power of two
    assert mctrg.mctrg_hotrg_run(o, 8, 1, 4, 1)[0] == mctrg.MCTRG_EINVAL      # chi < 2
    assert mctrg.mctrg_hotrg_run(o, 8, 33, 4, 1)[0] == mctrg.MCTRG_EINVAL     # chi > 32
    assert mctrg.mctrg_hotrg_run(o, 8, 4, 0, 1)[0] == mctrg.MCTRG_EINVAL      # no trajectories
