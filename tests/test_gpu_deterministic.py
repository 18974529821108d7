"""Deterministic TRG (Sec. II, Eq. approxSVD; Sec. IV, Fig. 3) and the hybrid
of deterministic levels followed by Monte Carlo (Sec. V) on the device,
through the C ABI, against the oracle.

* deterministic TRG (every level top-chi): every trajectory is identical and
  equals the oracle's deterministic TRG to 1e-10 relative, flags included,
  up to the headline lattice 1024 x 1024 (one split per sublattice per level);
* hybrid: per trajectory against the oracle's hybrid (tests/parity.py), and
  the estimate unbiased for the trace of the network the deterministic levels
  leave;
* the headline lattice against Kaufman's exact Z: Markov's bound above, the
  plain-TRG error at the same chi as the scale below.
"""
import math

import numpy as np
import pytest

from oracle import ising
from oracle.network import network_trace
from oracle.trg import Problem, run_level, run_many, run_trajectory
from paper_1710_03757_gb300 import build, mctrg
from paper_1710_03757_gb300.workloads import generic_tensor, seed_for

from parity import compare
from test_gpu_parity import gpu_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    mctrg.lib()


@pytest.mark.parametrize("beta,h,L,chi,D", [(0.44, 0.0, 32, 8, 0), (0.6, 0.0, 256, 16, 0), (0.3, 0.1, 64, 4, 0),
                                            (0.44, 0.0, 1024, 16, 0), (None, None, 16, 6, 2), (None, None, 8, 5, 3)])
def test_deterministic_trg_parity(beta, h, L, chi, D):
    if D:
        T0 = generic_tensor(D, seed=60 + L + chi)
        gpu = gpu_run(L, chi, 3, 11, T0=T0, deterministic_levels=99)
    else:
        T0 = ising.site_tensor(beta, h)
        gpu = gpu_run(L, chi, 3, 11, beta=beta, h=h, deterministic_levels=99)
    est, ln, sg, fl = gpu
    assert np.all(ln == ln[0]) and np.all(sg == sg[0]) and np.all(fl == fl[0])
    os_, ol, of = run_trajectory(Problem(T0, L, chi, deterministic_levels=99), 11, 0)
    assert int(fl[0]) == of
    if of == 0:
        assert sg[0] == os_
        assert abs(ln[0] - ol) <= 1e-10 * max(1.0, abs(ol)), (ln[0], ol)


@pytest.mark.parametrize("L,chi,det,n", [(8, 4, 2, 200), (16, 8, 3, 64), (32, 16, 4, 16)])
def test_hybrid_parity(L, chi, det, n):
    seed = seed_for(4) + L
    gpu = gpu_run(L, chi, n, seed, beta=0.44, deterministic_levels=det)
    orc = run_many(Problem(ising.site_tensor(0.44, 0.0), L, chi, deterministic_levels=det), seed, 0, n,
                   workers=8)
    compare(gpu, orc, min_ok=0.8, label="hybrid L%d chi%d det%d" % (L, chi, det))


def test_hybrid_unbiased_for_the_deterministic_network():
    # 4 x 4, chi = 2, two deterministic levels then Monte Carlo: the mean is
    # the exact trace of the level-2 network, not Z
    L, chi, det, beta, h = 4, 2, 2, 0.5, 0.05
    p = Problem(ising.site_tensor(beta, h), L, chi, deterministic_levels=det)
    tensors, lnacc, shared = [p.T0] * 16, 0.0, True
    for k in range(det):
        tensors, lnk, _, shared = run_level(p, k, tensors, shared, None, True)
        lnacc += lnk
    target = lnacc + math.log(network_trace(tensors, p.levels[det]))
    est, _, _, _ = gpu_run(L, chi, 40000, 4343, beta=beta, h=h, deterministic_levels=det)
    z = math.exp(target - est.ln_scale)
    assert abs(est.mean_Z_scaled - z) <= 3 * est.se_Z_scaled
    exact = ising.brute_force_lnZ(L, beta, h)
    assert abs(target - exact) > 1e-6    # the deterministic levels' bias is visible at this size


def test_headline_lattice_against_kaufman():
    # 1024 x 1024, chi = 16, beta = 0.44, FP64.  Counters fix each trajectory
    # whatever the batch.  Against Kaufman's exact ln Z of this torus:
    #  * upper side, distribution-free: Z~ >= 0 with E[Z~] = Z (Sec. III, Eq.
    #    infiniteEnsemble), so by Markov's inequality P(Z~ >= c Z) <= 1/c; with
    #    c = 100 n no trajectory of a correct implementation exceeds
    #    ln Z + ln(100 n) but with probability 1%;
    #  * lower side: at this size Z~/Z is so heavy-tailed (effective sample
    #    size about 1) that a few trajectories sit below ln Z by the Jensen gap
    #    and no distribution-free bound exists; they are held to three times
    #    the error of plain TRG at the same chi (measured: single trajectories
    #    fall 1.5 to 2 times that error below ln Z, the mean of more
    #    trajectories closer).
    L, beta, n = 1024, 0.44, 2
    a = gpu_run(L, 16, n, seed_for(2), beta=beta)
    b = gpu_run(L, 16, 1, seed_for(2), beta=beta, first=1)
    assert a[1][1] == b[1][0]
    assert np.all(a[2] == 1)
    exact = ising.kaufman_lnZ(L, beta)
    det = gpu_run(L, 16, 1, seed_for(2), beta=beta, deterministic_levels=99)[1][0]
    est = a[0]
    print("L1024: ln Z~ - ln Z = %s, ln Z^ - ln Z = %.3f, detTRG - ln Z = %.3f"
          % (np.round(a[1] - exact, 3).tolist(), est.ln_mean_Z - exact, det - exact))
    assert np.all(a[1] <= exact + math.log(100 * n))
    assert np.all(a[1] >= exact - 3 * abs(det - exact))
    assert est.ln_mean_Z <= exact + math.log(100 * n)
    m = gpu_run(L, 16, 1, seed_for(2), beta=beta, first=1, precision=mctrg.MCTRG_TF32X3)
    assert abs(m[1][0] - b[1][0]) / abs(b[1][0]) < 1e-6
    t = gpu_run(L, 16, 1, seed_for(2), beta=beta, first=1, precision=mctrg.MCTRG_FP64TC)
    assert abs(t[1][0] - b[1][0]) / abs(b[1][0]) < 1e-6
