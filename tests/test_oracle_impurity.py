"""Pins of the oracle's observables by impurity tensors (CPU only).

Sec. III notes that the method applies to partial traces as well as to Z.  A
site whose tensor carries its spin (the impurity tensor) turns the trace of
the network into sum_sigma sigma_i e^{-beta H} = Z <sigma_i>; two neighbouring
impurities give Z <sigma_i sigma_j>, the bond energy.  Such a network is not
translation invariant, so every level is split tensor by tensor.

* the exact trace of the impurity network equals brute force (L = 2, 4, one
  and two impurities, with and without a field);
* the transfer-matrix insertion equals brute force (two independent exact
  references for the larger lattices);
* TRG without truncation reproduces the exact partial trace;
* every sample outcome enumerated at L = 2: E[Z~_imp] = Z <sigma_0>;
* statistically: the sample mean of Z~_imp lies within 3 SE of Z <sigma_0>,
  and the ratio of the impurity and plain estimates approaches <sigma_0>.
"""
import math

import numpy as np
import pytest

from oracle import ising
from oracle.estimator import estimate
from oracle.network import network_trace, plan
from oracle.trg import Problem, run_many, run_trajectory

from test_oracle_trg import _expected


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.4, 0.1)])
def test_impurity_network_trace_is_brute_force(L, beta, h):
    T0, Ti = ising.site_tensor(beta, h), ising.impurity_tensor(beta, h)
    lev = plan(L)[0]
    lnZ = ising.brute_force_lnZ(L, beta, h)
    for sites in ([(0, 0)], [(0, 0), (1, 0)]):
        ts = [T0] * (L * L)
        for x, y in sites:
            ts[y * L + x] = Ti
        ref, lnZ2 = ising.brute_force_observable(L, beta, h, sites)
        assert lnZ2 == pytest.approx(lnZ, rel=1e-13)
        got = network_trace(ts, lev) / math.exp(lnZ)
        assert got == pytest.approx(ref, rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.44, 0.05), (0.6, 0.1)])
def test_transfer_insertion_is_brute_force(beta, h):
    for cols, sites in (([0], [(0, 0)]), ([0, 1], [(0, 0), (1, 0)])):
        assert ising.transfer_observable(4, beta, h, cols) == pytest.approx(
            ising.brute_force_observable(4, beta, h, sites)[0], rel=1e-10, abs=1e-13)


def test_untruncated_trg_gives_the_exact_partial_trace():
    beta, h = 0.4, 0.1
    p = Problem(ising.site_tensor(beta, h), 4, 16, site_tensors={0: ising.impurity_tensor(beta, h)})
    sign, lnz, flags = run_trajectory(p, 1, 0)
    m, lnZ = ising.brute_force_observable(4, beta, h, [(0, 0)])
    assert sign == 1 and flags == 0
    assert sign * math.exp(lnz - lnZ) == pytest.approx(m, rel=1e-12)


def test_enumerated_expectation_with_an_impurity():
    # L = 2, chi = 2: both levels sampled per tensor; every outcome enumerated
    beta, h = 0.44, 0.05
    T0, Ti = ising.site_tensor(beta, h), ising.impurity_tensor(beta, h)
    p = Problem(T0, 2, 2, site_tensors={0: Ti})
    z = _expected(p, 0, [Ti, T0, T0, T0], False, 0.0)
    m, lnZ = ising.brute_force_observable(2, beta, h, [(0, 0)])
    assert z == pytest.approx(m * math.exp(lnZ), rel=1e-11)


def test_impurity_estimates_are_unbiased():
    beta, h, L, chi, n = 0.4, 0.1, 4, 2, 3000
    T0, Ti = ising.site_tensor(beta, h), ising.impurity_tensor(beta, h)
    m, lnZ = ising.brute_force_observable(L, beta, h, [(0, 0)])
    s, l, _ = run_many(Problem(T0, L, chi, site_tensors={0: Ti}), 71, 0, n)
    e = estimate(s, l)
    target = m * math.exp(lnZ - e['ln_scale'])
    assert abs(e['mean_Z_scaled'] - target) <= 3 * e['se_Z_scaled']
    # the ratio to the plain estimate (independent seeds) approaches <sigma_0>
    s0, l0, _ = run_many(Problem(T0, L, chi), 72, 0, n)
    e0 = estimate(s0, l0)
    ratio = math.exp(e['ln_scale'] - e0['ln_scale']) * e['mean_Z_scaled'] / e0['mean_Z_scaled']
    se = abs(ratio) * math.hypot(e['se_Z_scaled'] / e['mean_Z_scaled'], e0['se_Z_scaled'] / e0['mean_Z_scaled'])
    assert abs(ratio - m) <= 3 * se
