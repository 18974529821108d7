"""Deterministic TRG (Sec. II, Eq. approxSVD; Sec. IV, Fig. 3) and the hybrid
of deterministic levels followed by Monte Carlo (Sec. V) on the device,
through the C ABI, against the oracle.

* deterministic TRG (every level top-chi): every trajectory is identical and
  equals the oracle's deterministic TRG to 1e-10 relative, flags included,
  up to the headline lattice 1024 x 1024 (one split per sublattice per level);
* hybrid: per trajectory against the oracle's hybrid (tests/parity.py), and
  the estimate unbiased for the trace of the network the deterministic levels
  leave;
* the headline lattice: the Monte Carlo estimate lies within 3 standard errors
  plus the deterministic TRG's own error of Kaufman's exact Z (the truncation
  bias of plain TRG at the same chi sets the scale of what a few heavy-tailed
  samples can resolve).
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
    # 1024 x 1024, chi = 16, beta = 0.44, FP64: counters fix each trajectory
    # whatever the batch; the estimate against the exact finite-torus ln Z within
    # 3 SE + |ln Z_detTRG - ln Z| (the plain-TRG truncation error at this chi)
    L, beta = 1024, 0.44
    a = gpu_run(L, 16, 2, seed_for(2), beta=beta)
    b = gpu_run(L, 16, 1, seed_for(2), beta=beta, first=1)
    assert a[1][1] == b[1][0]
    assert np.all(a[2] == 1)
    exact = ising.kaufman_lnZ(L, beta)
    det = gpu_run(L, 16, 1, seed_for(2), beta=beta, deterministic_levels=99)[1][0]
    est = a[0]
    bound = 3 * est.se_ln_Z + abs(det - exact)
    print("L1024: ln Z^ - ln Z = %.3f, SE %.3f, detTRG - ln Z = %.3f" % (est.ln_mean_Z - exact, est.se_ln_Z,
                                                                        det - exact))
    assert abs(est.ln_mean_Z - exact) <= bound
    m = gpu_run(L, 16, 1, seed_for(2), beta=beta, first=1, precision=mctrg.MCTRG_TF32X3)
    assert abs(m[1][0] - b[1][0]) / abs(b[1][0]) < 1e-6

