"""Stochastic truncation of one singular spectrum (oracle), Sec. II.

Test infrastructure only: nothing on the product path may import this module.

Given singular values s_1 >= s_2 >= ... >= s_n' > 0 (the nonzero ones) and a
sample size chi < n', draw a chi-subset e with p(e) = w(e) / sum_n w(n),
w(e) = prod_{j in e} s_j^2  (Sec. II, Eqs. w and p), and return the inclusion
rates r_i = sum_{e contains i} p(e)  (Sec. II, Eq. r), by which the kept values
are divided (Sec. II, the reweighting that makes Eq. Ssum hold).

The paper defers the O(chi * chi~) sampler to Ferris (2015), which is not
available; this is the reading used here (a fixed-size product-weight design):
  * weights w_i = (s_i / s_1)^2;
  * normalized elementary symmetric table
        E[i][j] = e_j(w_1..w_i) / (w_1 ... w_j),
        E[i][0] = 1, E[i][j] = 0 for i < j,
        E[i][j] = E[i-1][j] + (w_i / w_j) E[i-1][j-1];
    all entries lie in [1, C(i,j)] when w is sorted descending, so nothing
    under- or overflows;
  * draw the largest kept index first: with j picks left among {1..b},
    P(largest = i) is proportional to w_i e_{j-1}(w_1..w_{i-1}), whose
    running sum over i = j..b is E[i][j]; so take the smallest i in [j, b]
    with E[i][j] > u * E[b][j], keep i, set b = i - 1, and repeat;
  * inclusion rates from a forward and a backward table (sums of positive
    terms only):
        r_i = w_i e_{chi-1}(w without i) / e_chi(w)
            = sum_a E[i-1][a] G[i][chi-1-a] R(i,a) / E[n'][chi],
    G[i][b] = e_b(w_{i+1}..w_n') / (w_{i+1} ... w_{i+b}),
    G[i][0] = 1, G[i][b] = G[i+1][b] w_{i+b+1}/w_{i+1} + G[i+1][b-1],
    R(i,a) = prod_{t=0}^{chi-a-1} w_{i+t} / w_{a+1+t}  (each factor <= 1).
Indices are 1-based in the formulas and 0-based in the arrays returned.
"""
import numpy as np

# flag bits, OR-ed per trajectory
FLAG_SPLIT_CLUSTER = 1   # a kept and a dropped value closer than GAP_TOL * s_1
FLAG_DRAW_TIE = 2        # u * total within TIE_TOL * total of a CDF step
FLAG_TINY_KEPT = 4       # a kept value below TINY_TOL * s_1
GAP_TOL = 1e-8
TIE_TOL = 1e-9
TINY_TOL = 1e-7


def forward_table(w, chi):
    n = len(w)
    E = np.zeros((n + 1, chi + 1))
    E[:, 0] = 1.0
    for i in range(1, n + 1):
        for j in range(1, min(i, chi) + 1):
            E[i, j] = E[i - 1, j] + (w[i - 1] / w[j - 1]) * E[i - 1, j - 1]
    return E


def backward_table(w, chi):
    n = len(w)
    G = np.zeros((n + 1, chi))
    G[:, 0] = 1.0
    for i in range(n - 1, -1, -1):
        for b in range(1, min(chi - 1, n - i) + 1):
            first = 0.0
            if i + b + 1 <= n:
                first = G[i + 1, b] * (w[i + b] / w[i])
            G[i, b] = first + G[i + 1, b - 1]
    return G


def inclusion_rates(w, chi):
    """r_i for i = 0..n'-1 (0-based), for a chi-subset of n' > chi weights."""
    n = len(w)
    E = forward_table(w, chi)
    G = backward_table(w, chi)
    r = np.zeros(n)
    for i in range(1, n + 1):
        acc = 0.0
        for a in range(max(0, chi - 1 - (n - i)), min(chi - 1, i - 1) + 1):
            R = 1.0
            for t in range(chi - a):
                R *= w[i - 1 + t] / w[a + t]
            acc += E[i - 1, a] * G[i, chi - 1 - a] * R
        r[i - 1] = acc / E[n, chi]
    return r


def draw(w, chi, u):
    """Kept indices (0-based, ascending) for uniforms u[0..chi-1], plus flags."""
    n = len(w)
    E = forward_table(w, chi)
    b = n
    kept = []
    flags = 0
    for t in range(chi):
        j = chi - t
        total = E[b, j]
        x = u[t] * total
        i = j
        while not E[i, j] > x:
            i += 1
        lo = E[i - 1, j]
        hi = E[i, j]
        if (x - lo) <= TIE_TOL * total or (hi - x) <= TIE_TOL * total:
            flags |= FLAG_DRAW_TIE
        kept.append(i - 1)
        b = i - 1
    return sorted(kept), flags


def truncate(s, chi, uniforms_fn, n_rows, zero_scale=1.0):
    """Stochastic truncation of one descending spectrum s (length n_rows).

    Returns (kept indices, reweighted kept values s_i / r_i, flags, used),
    where used says whether uniforms were consumed.  Values at or below the
    zero threshold tau = zero_scale * n_rows * 2^-52 * s_1 count as exact
    zeros (the paper samples among the nonzero singular values, Sec. II;
    zero_scale = 1 is the default reading of "nonzero").
    """
    s1 = s[0]
    if not s1 > 0.0:
        return [], np.zeros(0), 0, False
    tau = zero_scale * n_rows * 2.0 ** -52 * s1
    flags = 0
    nnz = int(np.sum(s > tau))
    if nnz <= chi:
        kept = list(range(nnz))
        return kept, s[:nnz].copy(), flags, False
    w = (s[:nnz] / s1) ** 2
    u = uniforms_fn(chi)
    kept, f = draw(w, chi, u)
    flags |= f
    r = inclusion_rates(w, chi)
    keptset = set(kept)
    for i in range(nnz - 1):
        if ((i in keptset) != (i + 1 in keptset)) and (s[i] - s[i + 1]) <= GAP_TOL * s1:
            flags |= FLAG_SPLIT_CLUSTER
    if np.any(s[kept] < TINY_TOL * s1):
        flags |= FLAG_TINY_KEPT
    return kept, s[kept] / r[kept], flags, True


def truncate_top(s, chi, n_rows, zero_scale=1.0):
    """Deterministic truncation (Sec. II, Eq. approxSVD): keep the chi largest
    nonzero singular values of one descending spectrum, unreweighted (the
    plain TRG of Levin and Nave that the paper compares with, Sec. IV, Fig. 3).

    Returns (kept indices, kept values, flags, used=False).  When a kept and a
    dropped value are closer than GAP_TOL * s_1 the truncated tensor depends on
    the basis chosen inside that cluster, which two correct SVDs may choose
    differently: FLAG_SPLIT_CLUSTER.  The zero threshold is that of truncate.
    """
    s1 = s[0]
    if not s1 > 0.0:
        return [], np.zeros(0), 0, False
    tau = zero_scale * n_rows * 2.0 ** -52 * s1
    nnz = int(np.sum(s > tau))
    k = min(chi, nnz)
    flags = 0
    if nnz > chi and (s[k - 1] - s[k]) <= GAP_TOL * s1:
        flags |= FLAG_SPLIT_CLUSTER
    return list(range(k)), s[:k].copy(), flags, False
