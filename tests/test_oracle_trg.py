"""Pins of the oracle's Monte Carlo TRG trajectories (CPU only).

* exact path: with chi at least every rank nothing is sampled and Z~ = Z;
* enumeration of every sample outcome: E[Z~] = Z to rounding (Sec. III,
  Eqs. infiniteSum and infiniteEnsemble), including conditional expectations
  given an earlier level's sample;
* statistics: the sample mean lies within 3 standard errors of exact Z, and
  the error falls as 1/sqrt(N) (Sec. V, Eq. shrunkDev).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import ising
from oracle.estimator import estimate
from oracle.network import network_trace
from oracle.sampler import inclusion_rates
from oracle.trg import Problem, matricize, run_level, run_many, run_trajectory, svd
from paper_1710_03757_gb300.workloads import generic_tensor, seed_for


def test_exact_path_L2():
    for beta, h in ((0.44, 0.0), (0.3, 0.2)):
        p = Problem(ising.site_tensor(beta, h), 2, 4)
        sign, lnz, flags = run_trajectory(p, 1, 0)
        assert sign == 1 and flags == 0
        assert lnz == pytest.approx(ising.brute_force_lnZ(2, beta, h), rel=1e-13)


def test_exact_levels_L4_then_trace():
    # chi = 16: levels 0-2 keep everything; the level-3 network traced exactly is Z
    for beta, h in ((0.44, 0.0), (0.6, 0.1)):
        p = Problem(ising.site_tensor(beta, h), 4, 16)
        tensors = [p.T0] * 16
        shared, lnacc = True, 0.0
        from oracle.trg import _stochastic_chooser
        for k in range(3):
            tensors, lnk, f, shared = run_level(
                p, k, tensors, shared, lambda t, k=k: _stochastic_chooser(1, 0, k, t, p.chi))
            lnacc += lnk
        assert shared
        z = network_trace(tensors, p.levels[3])
        assert lnacc + math.log(z) == pytest.approx(ising.brute_force_lnZ(4, beta, h), rel=1e-13)


def test_exact_path_generic_L2():
    T0 = generic_tensor(2, seed=5)
    p = Problem(T0, 2, 16)
    sign, lnz, flags = run_trajectory(p, 3, 0)
    z = network_trace([T0] * 4, p.levels[0])
    assert sign == (1 if z > 0 else -1)
    assert lnz == pytest.approx(math.log(abs(z)), rel=1e-13)


def _outcomes(T, parity, chi):
    """Every stochastic-truncation outcome of one tensor with its probability."""
    D = T.shape[0]
    s = svd(matricize(T, parity))[1]
    s = s / s[0]
    nnz = int(np.sum(s > D * D * 2.0 ** -52))
    if nnz <= chi:
        return [((list(range(nnz)), s[:nnz]), 1.0)]
    w = s[:nnz] ** 2
    r = inclusion_rates(w, chi)
    subs = list(itertools.combinations(range(nnz), chi))
    W = np.array([np.prod(w[list(e)]) for e in subs])
    return [((list(e), s[list(e)] / r[list(e)]), q) for e, q in zip(subs, W / W.sum())]


def _expected(p, k, tensors, shared, lnacc):
    """E[Z~ | level-k network] by enumerating every remaining sample outcome."""
    if k == p.n_levels:
        return math.exp(lnacc) * float(np.einsum('abab->', tensors[0]))
    lev = p.levels[k]
    per = [_outcomes(tensors[t], int(lev.parity[t]), p.chi) for t in range(lev.n)]
    total = 0.0
    for combo in itertools.product(*per):
        prob = float(np.prod([c[1] for c in combo]))
        fixed = [c[0] for c in combo]
        chooser_for = lambda t: (lambda s, n_rows, t=t: (fixed[t][0], fixed[t][1], 0))
        new, lnk, _, sh = run_level(p, k, tensors, shared, chooser_for)
        total += prob * _expected(p, k + 1, new, sh, lnacc + lnk)
    return total


@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.3, 0.1)])
def test_enumerated_expectation_ising_L2(beta, h):
    p = Problem(ising.site_tensor(beta, h), 2, 2)
    z = _expected(p, 0, [p.T0] * 4, True, 0.0)
    assert math.log(z) == pytest.approx(ising.brute_force_lnZ(2, beta, h), rel=1e-12)


def test_enumerated_expectation_generic_L2():
    # level 0 is already stochastic: 6^4 outcomes, then 6^2 at level 1
    T0 = generic_tensor(2, seed=9)
    p = Problem(T0, 2, 2)
    z = _expected(p, 0, [T0] * 4, True, 0.0)
    exact = network_trace([T0] * 4, p.levels[0])
    assert z == pytest.approx(exact, rel=1e-11)


def test_conditional_expectation_L4():
    # fix the level-1 sample of one trajectory; enumerating levels 2 and 3 gives
    # the exact trace of the sampled level-2 network (Eq. infiniteSum)
    p = Problem(ising.site_tensor(0.44, 0.05), 4, 2)
    tensors, shared, lnacc = [p.T0] * 16, True, 0.0
    from oracle.trg import _stochastic_chooser
    for k in range(2):
        tensors, lnk, _, shared = run_level(
            p, k, tensors, shared, lambda t, k=k: _stochastic_chooser(17, 0, k, t, p.chi))
        lnacc += lnk
    exact = math.exp(lnacc) * network_trace(tensors, p.levels[2])
    assert _expected(p, 2, tensors, shared, lnacc) == pytest.approx(exact, rel=1e-11)


def test_unbiased_config1():
    # L = 4, h = 0, beta = 0.44, chi = 2, 1000 trajectories: within 3 SE of exact Z
    p = Problem(ising.site_tensor(0.44, 0.0), 4, 2)
    sign, lnabs, flags = run_many(p, seed_for(1), 0, 1000)
    e = estimate(sign, lnabs)
    z = math.exp(ising.brute_force_lnZ(4, 0.44) - e['ln_scale'])
    assert abs(e['mean_Z_scaled'] - z) <= 3 * e['se_Z_scaled']


@pytest.mark.parametrize("beta,h", [(0.3, 0.0), (0.44, 0.1), (0.6, 0.0)])
def test_unbiased_many_seeds(beta, h):
    # z-scores of 12 independent 150-trajectory runs: mean near 0, spread near 1
    p = Problem(ising.site_tensor(beta, h), 4, 2)
    exact = ising.brute_force_lnZ(4, beta, h)
    zs = []
    for seed in range(12):
        sign, lnabs, _ = run_many(p, 1000 + seed, 0, 150)
        e = estimate(sign, lnabs)
        zs.append((e['mean_Z_scaled'] - math.exp(exact - e['ln_scale'])) / e['se_Z_scaled'])
    zs = np.array(zs)
    assert abs(zs.mean()) < 3 / math.sqrt(len(zs)) + 0.3
    assert np.all(np.abs(zs) < 4.5)


def test_unbiased_larger_lattice():
    # L = 8, chi = 4 against Kaufman's exact finite-torus Z
    p = Problem(ising.site_tensor(0.4, 0.0), 8, 4)
    sign, lnabs, _ = run_many(p, seed_for(2), 0, 300)
    e = estimate(sign, lnabs)
    z = math.exp(ising.kaufman_lnZ(8, 0.4) - e['ln_scale'])
    assert abs(e['mean_Z_scaled'] - z) <= 3 * e['se_Z_scaled']


def test_error_falls_as_inverse_sqrt_n():
    p = Problem(ising.site_tensor(0.3, 0.0), 4, 2)
    sign, lnabs, _ = run_many(p, 77, 0, 3200)
    small = [estimate(sign[i:i + 200], lnabs[i:i + 200])['se_ln_Z'] for i in range(0, 3200, 200)]
    big = estimate(sign, lnabs)['se_ln_Z']
    # 16x the samples -> 4x smaller error (the small-run average scatters)
    assert np.mean(small) / big == pytest.approx(4.0, rel=0.25)


def test_oracle_per_sample_spread_matches_table1():
    # The paper's printed per-sample std of Z~/Z on its own lattice (Sec. IV,
    # Table 1, first row: chi~ = 6, T = 1.5, 128 spins).  A sampler drawing from
    # a different p(e), or reweighting differently, gives a different spread.
    # 4000 fixed-seed trajectories; the band covers the std estimate's sampling
    # spread for this multimodal distribution (Fig. 2)
    import os
    from oracle.trg import Problem, run_many
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                    "table1_per_sample_std.txt")) if l.strip() and l[0] != "#"]
    chi, T, std_paper = int(rows[0][0]), float(rows[0][1]), float(rows[0][2])
    beta = 1.0 / T
    sign, lnabs, _ = run_many(Problem(ising.bond_spin_tensor(beta), 8, chi), 0x7AB1E, 0, 4000, workers=8)
    z = sign * np.exp(lnabs - ising.bond_spin_transfer_lnZ(8, beta))
    assert abs(z.mean() - 1.0) <= 4 * z.std(ddof=1) / math.sqrt(len(z))
    assert 0.75 * std_paper <= z.std(ddof=1) <= 1.25 * std_paper
