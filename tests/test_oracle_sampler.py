"""Pins of the oracle's stochastic truncation (Sec. II), CPU only.

The ESP-table sampler is checked against brute-force subset enumeration:
p(e) proportional to prod_{j in e} s_j^2 (Eqs. w, p), r_i = sum_{e contains i} p(e)
(Eq. r), and E[S^(e)] = S (Eq. Ssum).
"""
import itertools
import math

import numpy as np
import pytest

from oracle import philox
from oracle.sampler import (FLAG_DRAW_TIE, FLAG_SPLIT_CLUSTER, FLAG_TINY_KEPT, draw,
                            forward_table, inclusion_rates, truncate)


def _enumerate(w, chi):
    subs = list(itertools.combinations(range(len(w)), chi))
    W = np.array([np.prod(w[list(e)]) for e in subs])
    return subs, W / W.sum()


def _spectra():
    rng = np.random.default_rng(3)
    out = []
    for n in (3, 5, 8, 12):
        out.append(np.sort(rng.random(n))[::-1])                       # flat
        out.append(np.exp(-np.sort(rng.random(n) * 20))[:])            # decaying over 9 decades
    out.append(np.array([1.0, 1.0, 0.5, 0.5, 0.5, 0.1]))               # exact ties
    out.append(np.array([1.0, 1e-3, 1e-6, 1e-9, 1e-12, 1e-15, 1e-18]))  # extreme decay
    return out


@pytest.mark.parametrize("k", range(10))
def test_rates_and_draw_probabilities_match_enumeration(k):
    s = _spectra()[k]
    s = s / s[0]
    w = s ** 2
    for chi in range(1, min(6, len(w))):
        subs, P = _enumerate(w, chi)
        r = inclusion_rates(w, chi)
        r_enum = np.array([sum(P[q] for q, e in enumerate(subs) if i in e) for i in range(len(w))])
        np.testing.assert_allclose(r, r_enum, rtol=1e-12, atol=1e-300)
        assert r.sum() == pytest.approx(chi, rel=1e-13)
        assert np.all(r > 0) and np.all(r <= 1 + 1e-15)
        # the sequential draw's exact probability of each subset equals p(e)
        E = forward_table(w, chi)
        for q, e in enumerate(subs):
            b, p = len(w), 1.0
            for t, i in enumerate(sorted(e, reverse=True)):
                j = chi - t
                # P(largest pick = i | j picks among the first b) = w_i e_{j-1}(w_<i) / e_j(w_<=b)
                p *= (w[i] / w[j - 1]) * E[i, j - 1] / E[b, j]
                b = i
            assert p == pytest.approx(P[q], rel=1e-10, abs=1e-300)


def test_unbiased_reweighting_eq_Ssum():
    # sum_e p(e) S^(e) = S exactly, S^(e)_ii = s_i / r_i for i in e, 0 otherwise
    s = np.array([1.0, 0.8, 0.35, 0.2, 0.07, 0.01])
    w = s ** 2
    for chi in (1, 2, 3, 5):
        subs, P = _enumerate(w, chi)
        r = inclusion_rates(w, chi)
        mean = np.zeros_like(s)
        for q, e in enumerate(subs):
            for i in e:
                mean[i] += P[q] * s[i] / r[i]
        np.testing.assert_allclose(mean, s, rtol=1e-13)


def test_draw_frequencies_chi_square():
    s = np.array([1.0, 0.9, 0.6, 0.5, 0.3, 0.2, 0.1])
    w = s ** 2
    chi = 3
    subs, P = _enumerate(w, chi)
    index = {e: q for q, e in enumerate(subs)}
    counts = np.zeros(len(subs))
    n = 20000
    for t in range(n):
        kept, _ = draw(w, chi, philox.uniforms(11, t, 0, 0, chi))
        counts[index[tuple(kept)]] += 1
    expected = n * P
    chi2 = float(np.sum((counts - expected) ** 2 / expected))
    dof = len(subs) - 1
    # 5-sigma bound on a chi-square variable with dof degrees of freedom
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_truncate_keeps_all_when_rank_small():
    s = np.array([1.0, 0.5, 0.25, 1e-17, 0.0])
    calls = []
    kept, st, flags, used = truncate(s, 3, lambda c: calls.append(c) or [0.5] * c, 5)
    assert kept == [0, 1, 2] and not used and not calls
    np.testing.assert_array_equal(st, s[:3])


def test_truncate_zero_threshold():
    # values at or below n * 2^-52 * s_1 are zeros: never kept, never weighted
    s = np.array([1.0, 0.5, 0.25, 0.9 * 4 * 2.0 ** -52])
    kept, st, flags, used = truncate(s, 2, lambda c: [0.999999] * c, 4)
    assert used and 3 not in kept


def test_truncate_flags():
    s = np.array([1.0, 0.5, 0.5, 0.2])
    # u = 0.9 makes the first pick the largest index; a split of the tied pair is flagged
    seen = 0
    for u0 in np.linspace(0.01, 0.99, 25):
        kept, st, flags, used = truncate(s, 2, lambda c: [u0, 0.5][:c], 4)
        if (1 in kept) != (2 in kept):
            assert flags & FLAG_SPLIT_CLUSTER
            seen += 1
    assert seen > 0
    s = np.array([1.0, 0.3, 1e-8, 1e-9])
    kept, st, flags, used = truncate(s, 3, lambda c: [0.999999999, 0.9, 0.5][:c], 4)
    assert 3 in kept and flags & FLAG_TINY_KEPT
    # a uniform landing exactly on a CDF step is a tie
    w = (np.array([1.0, 0.7, 0.4]) ** 2)
    E = forward_table(w, 1)
    u_edge = E[1, 1] / E[3, 1]
    kept, flags = draw(w, 1, [u_edge])
    assert flags & FLAG_DRAW_TIE


def test_zero_threshold_scale():
    # R5 with a scale: values at or below zero_scale * n * 2^-52 * s_1 are zeros.
    # n = 4: tau = 8.9e-16 s_1 at scale 1, 8.9e-14 s_1 at scale 100
    from oracle.sampler import truncate
    s = np.array([1.0, 1e-14, 1e-20, 0.0])
    kept, st, flags, used = truncate(s, 4, None, 4)
    assert kept == [0, 1] and not used
    kept, st, flags, used = truncate(s, 4, None, 4, zero_scale=100.0)
    assert kept == [0] and not used
    np.testing.assert_array_equal(st, [1.0])
