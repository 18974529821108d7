"""Pins of the exact partition-function references (CPU only).

Each routine is checked against routines that share no formula with it:
enumeration, the transfer matrix, Kaufman's closed form, Onsager's integral
(two independent forms) and the known value at the critical point.
"""
import math

import numpy as np
import pytest

from oracle import ising
from oracle.network import network_trace, plan


@pytest.mark.parametrize("beta", [0.1, 0.3, 0.44, 0.6, 1.0])
@pytest.mark.parametrize("h", [0.0, 0.05, -0.3])
def test_bruteforce_equals_transfer_L4(beta, h):
    assert ising.brute_force_lnZ(4, beta, h) == pytest.approx(ising.transfer_lnZ(4, beta, h), rel=1e-14)


@pytest.mark.parametrize("beta", [0.1, 0.3, 0.4406, 0.44, 0.6, 1.0])
def test_kaufman_equals_bruteforce_L4(beta):
    assert ising.kaufman_lnZ(4, beta) == pytest.approx(ising.brute_force_lnZ(4, beta), rel=1e-13)


@pytest.mark.parametrize("L", [2, 6, 8])
@pytest.mark.parametrize("beta", [0.25, 0.44, 0.7])
def test_kaufman_equals_transfer(L, beta):
    assert ising.kaufman_lnZ(L, beta) == pytest.approx(ising.transfer_lnZ(L, beta), rel=1e-12)


def test_zero_coupling():
    # beta = 0: every configuration has weight 1, Z = 2^N
    for L in (2, 4):
        assert ising.brute_force_lnZ(L, 0.0) == pytest.approx(L * L * math.log(2), rel=1e-15)


def test_onsager_forms_agree():
    for beta in (0.2, 0.35, 0.5, 0.8):
        assert ising.onsager_minus_beta_f(beta) == pytest.approx(ising.onsager_minus_beta_f_1d(beta), rel=1e-11)


def test_onsager_critical_value():
    # at K_c = ln(1+sqrt 2)/2:  -beta f = ln(2)/2 + 2G/pi, G = Catalan's constant
    catalan = 0.915965594177219015054603514932
    Kc = 0.5 * math.log(1 + math.sqrt(2))
    assert ising.onsager_minus_beta_f_1d(Kc) == pytest.approx(0.5 * math.log(2) + 2 * catalan / math.pi, rel=1e-9)


def test_kaufman_tends_to_onsager():
    # high temperature: finite-size corrections are exponentially small
    assert ising.kaufman_lnZ(64, 0.3) / 64 ** 2 == pytest.approx(ising.onsager_minus_beta_f(0.3), rel=1e-13)
    # low temperature: the two ordered states add ln 2 / N
    assert ising.kaufman_lnZ(64, 0.6) / 64 ** 2 - math.log(2) / 64 ** 2 == \
        pytest.approx(ising.onsager_minus_beta_f(0.6), rel=1e-9)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.3, 0.1), (0.7, -0.05)])
def test_site_tensor_network_is_Z(L, beta, h):
    T = ising.site_tensor(beta, h)
    lev = plan(L)[0]
    assert math.log(network_trace([T] * lev.n, lev)) == pytest.approx(ising.brute_force_lnZ(L, beta, h), rel=1e-13)


def test_site_tensor_rank_two():
    # M[(l,u),(r,d)] = sum_s e^{beta h s} (W_s x W_s)(W_s x W_s)^T has rank 2
    T = ising.site_tensor(0.44, 0.1)
    s = np.linalg.svd(T.reshape(4, 4), compute_uv=False)
    assert s[1] > 1e-3 * s[0] and s[2] < 1e-14 * s[0]


# ---- the spins-on-bonds network of Sec. IV (Fig. 1) -------------------------

@pytest.mark.parametrize("L,beta,h", [(2, 0.4, 0.0), (2, 0.7, 0.1), (3, 0.44, 0.0), (3, 0.3, -0.2)])
def test_bond_spin_transfer_equals_brute_force(L, beta, h):
    assert ising.bond_spin_transfer_lnZ(L, beta, h) == pytest.approx(ising.bond_spin_brute_lnZ(L, beta, h),
                                                                     rel=1e-13)


def test_bond_spin_beta0():
    for L in (2, 3, 8):
        assert ising.bond_spin_transfer_lnZ(L, 0.0) == pytest.approx(2 * L * L * math.log(2.0), rel=1e-14)


@pytest.mark.parametrize("L", [2, 4])
def test_bond_spin_network_trace(L):
    # the tensor network of the bond-spin tensors (geometry of the network
    # module, independent of the transfer matrix's ring contraction)
    lev = plan(L)[0]
    T = ising.bond_spin_tensor(0.5, 0.05)
    assert math.log(network_trace([T] * lev.n, lev)) == pytest.approx(
        ising.bond_spin_transfer_lnZ(L, 0.5, 0.05), rel=1e-13)


def test_bond_spin_is_the_square_lattice():
    # 2 L^2 spins of a (rotated) square lattice: ln Z per spin -> Onsager;
    # at high temperature the 128-spin torus is within 1e-7 of the limit, in
    # the ordered phase it exceeds it by ln 2 / N (the two ground states)
    N = 128
    assert ising.bond_spin_transfer_lnZ(8, 0.2) / N == pytest.approx(ising.onsager_minus_beta_f(0.2), abs=1e-7)
    assert (ising.bond_spin_transfer_lnZ(8, 0.8) / N - math.log(2.0) / N ==
            pytest.approx(ising.onsager_minus_beta_f(0.8), abs=1e-6))
