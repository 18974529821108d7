"""Pins of the oracle's Monte Carlo HOTRG (stochastic truncation of Sec. II on
the higher-order TRG, the generalization Secs. III and V name).  CPU only.

* without truncation (chi at least every bond dimension) a trajectory is
  exact: brute-force Z of the Ising torus (with and without field) and the
  direct trace of a generic, non-symmetric tensor network (which checks the
  merge, the reflection and the leg bookkeeping);
* every outcome enumerated at L = 2 (all subsets of every bond of both steps,
  with probabilities and inclusion rates by brute force over the subsets, not
  by the sampler): E[Z~] = Z;
* the bond weights and basis are those of the right unfolding's SVD (a
  different routine from the Gram eigensolver), and the expected projector
  is the identity on the range M sees;
* statistically: the mean of Z~ over many trajectories lies within 3 SE of Z.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import hotrg, ising
from oracle.estimator import estimate
from oracle.network import network_trace, plan
from paper_1710_03757_gb300.workloads import generic_tensor


def _generic_exact(T0, L):
    return network_trace([T0] * (L * L), plan(L)[0])


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.3, 0.2)])
def test_untruncated_ising_is_exact(L, beta, h):
    p = hotrg.HotrgProblem(ising.site_tensor(beta, h), L, 64)
    sign, lnz, flags = hotrg.run_trajectory(p, 1, 0)
    assert sign == 1 and flags == 0
    assert lnz == pytest.approx(ising.brute_force_lnZ(L, beta, h), rel=1e-12)


@pytest.mark.parametrize("L", [2, 4])
def test_untruncated_generic_is_exact(L):
    T0 = generic_tensor(2, seed=77)
    assert not np.allclose(T0, T0.transpose(1, 0, 3, 2))     # not symmetric under the reflection
    p = hotrg.HotrgProblem(T0, L, 64)
    sign, lnz, _ = hotrg.run_trajectory(p, 1, 0)
    z = _generic_exact(T0, L)
    assert sign * math.exp(lnz) == pytest.approx(z, rel=1e-10)


def _subsets(lam, nnz, chi):
    """Every kept set with its probability and the inclusion rates, by brute force."""
    if nnz <= chi:
        return [(list(range(nnz)), np.ones(nnz), 1.0)]
    w = lam[:nnz] / lam[0]
    sets = list(itertools.combinations(range(nnz), chi))
    pw = np.array([np.prod(w[list(e)]) for e in sets])
    pw /= pw.sum()
    r = np.zeros(nnz)
    for e, q in zip(sets, pw):
        r[list(e)] += q
    return [(list(e), r[list(e)], q) for e, q in zip(sets, pw)]


def _enumerate(tensors, Lx, Ly, chi, steps_left, prob_weight, lnacc):
    if steps_left == 0:
        tr = float(np.einsum('abab->', tensors[0]))
        return prob_weight * math.exp(lnacc) * tr
    Lj = Ly // 2
    # the kept-set distribution of every bond of this step
    options = []
    for j in range(Lj):
        for x in range(Lx):
            M = hotrg.merge(tensors[2 * j * Lx + x], tensors[(2 * j + 1) * Lx + x])
            lam, U, nnz = hotrg.bond_eigen(M)
            options.append(_subsets(lam, nnz, chi))
    total = 0.0
    for combo in itertools.product(*options):
        def chooser_for(b, combo=combo):
            kept, r, _ = combo[b]
            return lambda lam, nnz, n: (kept, r, 0)
        new, nLx, nLy, lnk, _ = hotrg.run_step(tensors, Lx, Ly, chi, chooser_for)
        q = np.prod([c[2] for c in combo])
        total += _enumerate(new, nLx, nLy, chi, steps_left - 1, prob_weight * q, lnacc + lnk)
    return total


@pytest.mark.parametrize("chi", [2, 3])
@pytest.mark.parametrize("case", ["generic", "ising-field"])
def test_enumerated_expectation_is_z(chi, case):
    if case == "generic":
        T0 = generic_tensor(2, seed=91)
        z = _generic_exact(T0, 2)
    else:
        T0 = ising.site_tensor(0.5, 0.1)
        z = math.exp(ising.brute_force_lnZ(2, 0.5, 0.1))
    L = 2
    ez = _enumerate([T0] * (L * L), L, L, chi, 2, 1.0, 0.0)
    assert ez == pytest.approx(z, rel=1e-11)
    # and a single stochastic trajectory is one of the enumerated outcomes (not exact)
    p = hotrg.HotrgProblem(T0, L, chi)
    sign, lnz, _ = hotrg.run_trajectory(p, 5, 0)
    assert sign != 0


def test_bond_weights_are_the_right_unfoldings_singular_values():
    # lambda_i = s_i^2 of M's right unfolding (rows (l, u, d), columns r), and the
    # leading eigenvectors span its leading right singular vectors: the reading's
    # weights and basis, checked against an SVD of the unfolding itself
    M = hotrg.merge(generic_tensor(2, seed=13), generic_tensor(2, seed=14))
    lam, U, nnz = hotrg.bond_eigen(M)
    Mr = M.transpose(0, 1, 3, 2).reshape(-1, M.shape[2])
    _, s, Vt = np.linalg.svd(Mr)
    assert nnz == int(np.sum(s > 1e-6 * s[0]))
    np.testing.assert_allclose(lam[:nnz], s[:nnz] ** 2, rtol=1e-10, atol=1e-13 * s[0] ** 2)
    for k in range(1, nnz):
        if s[k - 1] - s[k] > 1e-6 * s[0]:
            Pe = U[:, :k] @ U[:, :k].T
            Ps = Vt[:k].T @ Vt[:k]
            np.testing.assert_allclose(Pe, Ps, atol=1e-9)


def test_expected_projector_is_identity_on_the_range():
    # sum over kept sets of p(e) * sum_{i in e} u_i u_i^T / r_i = the range projector
    T0 = generic_tensor(2, seed=5)
    M = hotrg.merge(T0, T0)
    lam, U, nnz = hotrg.bond_eigen(M)
    P = np.zeros((U.shape[0], U.shape[0]))
    for kept, r, q in _subsets(lam, nnz, 2):
        P += q * (U[:, kept] / r) @ U[:, kept].T
    R = U[:, :nnz] @ U[:, :nnz].T
    np.testing.assert_allclose(P, R, atol=1e-13)
    # and M does not see beyond the range of its Gram matrix
    Mr = M.transpose(0, 1, 3, 2).reshape(-1, M.shape[2])
    np.testing.assert_allclose(Mr @ R, Mr, atol=1e-12 * np.abs(Mr).max())


def test_sample_mean_is_unbiased():
    beta, L, chi, n = 0.44, 4, 3, 1500
    p = hotrg.HotrgProblem(ising.site_tensor(beta, 0.0), L, chi)
    s, l, _ = hotrg.run_many(p, 0x407, 0, n)
    e = estimate(s, l)
    z = math.exp(ising.brute_force_lnZ(L, beta) - e['ln_scale'])
    assert abs(e['mean_Z_scaled'] - z) <= 3 * e['se_Z_scaled']
    assert e['se_Z_scaled'] > 0.0          # chi = 3 does truncate at L = 4
