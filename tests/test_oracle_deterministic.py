"""Pins of the oracle's deterministic truncation (plain TRG, Sec. II Eq.
approxSVD) and of the hybrid of deterministic levels then Monte Carlo
(Sec. V), CPU only.

* no truncation (chi at least every rank): deterministic TRG is exact;
* each deterministic split is the best rank-chi approximation (Eckart-Young):
  its error equals the discarded spectral weight, computed here from the
  eigenvalues of M^T M (a different LAPACK routine than the oracle's SVD),
  and no other rank-chi projection does better;
* deterministic TRG of the Ising model approaches Kaufman's exact Z as chi
  grows, with the per-site error falling level by level in chi;
* the hybrid's trajectories are unbiased for the trace of the network that the
  deterministic levels leave (enumerated exactly), and with every level
  deterministic all trajectories are identical.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import ising
from oracle.network import network_trace
from oracle.sampler import GAP_TOL, FLAG_SPLIT_CLUSTER, truncate_top
from oracle.trg import (Problem, _deterministic_chooser, matricize, run_level, run_many, run_trajectory,
                        split)
from paper_1710_03757_gb300.workloads import generic_tensor


@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.6, 0.1)])
def test_deterministic_without_truncation_is_exact(beta, h):
    p = Problem(ising.site_tensor(beta, h), 4, 16, deterministic_levels=99)
    sign, lnz, flags = run_trajectory(p, 1, 0)
    assert sign == 1 and flags == 0
    assert lnz == pytest.approx(ising.brute_force_lnZ(4, beta, h), rel=1e-13)


@pytest.mark.parametrize("chi", [2, 3, 5])
def test_deterministic_split_is_the_best_rank_chi_approximation(chi):
    rng = np.random.default_rng(chi)
    T = generic_tensor(3, seed=40 + chi)
    for parity in (0, 1):
        M = matricize(T, parity)
        left, right, lns1, flags = split(T, parity, chi, _deterministic_chooser(chi))
        A = left.reshape(9, chi) @ right.reshape(chi, 9)            # approximant of M / s_1
        lam = np.sort(np.linalg.eigvalsh(M.T @ M))[::-1]             # s_i^2, by another routine
        s1 = math.sqrt(lam[0])
        assert lns1 == pytest.approx(math.log(s1), rel=1e-12)
        err = np.linalg.norm(M / s1 - A) ** 2
        assert err == pytest.approx(np.sum(lam[chi:]) / lam[0], rel=1e-9, abs=1e-14)
        for _ in range(20):                                           # random rank-chi projections
            Q, _ = np.linalg.qr(rng.standard_normal((9, chi)))
            assert np.linalg.norm(M / s1 - (M / s1) @ Q @ Q.T) ** 2 >= err * (1 - 1e-12)


def test_truncate_top_flags_a_split_cluster():
    s = np.array([1.0, 0.5, 0.5 - 0.5 * GAP_TOL, 0.1])
    kept, vals, flags, used = truncate_top(s, 2, 4)
    assert kept == [0, 1] and not used and flags == FLAG_SPLIT_CLUSTER
    kept, vals, flags, _ = truncate_top(np.array([1.0, 0.5, 0.4, 0.1]), 2, 4)
    assert flags == 0 and np.array_equal(vals, [1.0, 0.5])


def test_deterministic_trg_approaches_kaufman():
    # 32 x 32 at beta = 0.44 (near the critical point): the per-site error of
    # deterministic TRG against the exact finite-torus Z falls with chi
    L, beta = 32, 0.44
    exact = ising.kaufman_lnZ(L, beta)
    errs = []
    for chi in (2, 4, 8, 16):
        sign, lnz, _ = run_trajectory(Problem(ising.site_tensor(beta, 0.0), L, chi, deterministic_levels=99), 1, 0)
        assert sign == 1
        errs.append(abs(lnz - exact) / L ** 2)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[0] > 1e-3 and errs[-1] < 2e-5


def test_every_trajectory_identical_when_all_levels_are_deterministic():
    p = Problem(generic_tensor(2, seed=11), 8, 3, deterministic_levels=99)
    sign, lnabs, flags = run_many(p, 5, 0, 4)
    assert np.all(lnabs == lnabs[0]) and np.all(sign == sign[0])


def _outcomes(T, parity, chi):
    """Every stochastic-truncation outcome of one tensor, with its probability."""
    from oracle.sampler import inclusion_rates
    from oracle.trg import svd
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


def test_hybrid_is_unbiased_for_the_deterministic_network():
    # L = 2, generic D = 2 tensor, chi = 2: level 0 deterministic (top 2 of 4),
    # level 1 sampled.  Enumerating level 1's outcomes gives the exact trace of
    # the network the deterministic level leaves, which differs from Z.
    T0 = generic_tensor(2, seed=9)
    p = Problem(T0, 2, 2, deterministic_levels=1)
    tensors, lnacc, flags, shared = run_level(p, 0, [T0] * 4, True, None, True)
    assert shared
    target = math.exp(lnacc) * network_trace(tensors, p.levels[1])
    lev = p.levels[1]
    per = [_outcomes(tensors[t], int(lev.parity[t]), p.chi) for t in range(lev.n)]
    total = 0.0
    for combo in itertools.product(*per):
        prob = float(np.prod([c[1] for c in combo]))
        fixed = [c[0] for c in combo]
        chooser_for = lambda t: (lambda s, n_rows, t=t: (fixed[t][0], fixed[t][1], 0))
        new, lnk, _, _ = run_level(p, 1, tensors, shared, chooser_for)
        total += prob * math.exp(lnacc + lnk) * float(np.einsum('abab->', new[0]))
    assert total == pytest.approx(target, rel=1e-11)
    exact = network_trace([T0] * 4, p.levels[0])
    assert abs(target - exact) > 1e-6 * abs(exact)       # the truncation's bias is real
    # the oracle's trajectories follow the same hybrid: sample mean near the target
    sign, lnabs, _ = run_many(p, 3, 0, 3000)
    x = sign * np.exp(lnabs)
    assert abs(x.mean() - target) <= 4 * x.std(ddof=1) / math.sqrt(len(x))
